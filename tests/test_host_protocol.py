"""Host-side tests of the token-passing protocol and its failure detection.

ring_model.cc models the ring queues of the persistent kernel with host
threads (same slot format, reservation and publication order, bounded
waits), under the consumer disciplines: one token at a time at the head
(fifo), and the batched kernel's window (up to 16 ready tokens taken from
the first 16 positions, out of order -- 8 in mode window8, the kernel's
batch for rows wider than one chunk per lane --, long visits first and each
handed on right after it, the others handed on together at the end of the
batch, rings with 17 slots of headroom; the tokens of the most-visited items
through a second, urgent ring per worker, taken between visits).  Failures
are made on the host: a token that is never sent, a token sent twice, a slow
worker, producers pausing between reserving and writing a slot, and (a
planted mistake in the model) rings too small for the tokens in flight.  No
GPU is involved.
"""
import os
import subprocess

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def model(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("ring") / "ring_model")
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread",
                    os.path.join(ROOT, "tests", "ring_model.cc"), "-o", exe], check=True)
    return exe


def run(exe, p, n, maxdeg, epochs, seed, fault, mode="fifo"):
    out = subprocess.run([exe, str(p), str(n), str(maxdeg), str(epochs), str(seed), fault,
                          mode], capture_output=True, text=True, timeout=120,
                         check=True).stdout
    return dict(kv.split("=") for kv in out.split())


@pytest.mark.parametrize("mode", ["fifo", "window", "window8"])
@pytest.mark.parametrize("p,n,maxdeg,epochs,seed",
                         [(4, 50, 4, 3, 1), (8, 200, 8, 4, 2), (16, 300, 5, 2, 3),
                          (3, 1, 3, 5, 4), (6, 40, 1, 3, 5)])
def test_protocol_exactly_once(model, p, n, maxdeg, epochs, seed, mode):
    """Every segment is visited exactly once per epoch, every item finishes
    all epochs, no token is held twice, no slot is written again before its
    token was taken."""
    r = run(model, p, n, maxdeg, epochs, seed, "none", mode)
    # the window discipline routes the most-visited items through the
    # urgent rings
    assert (int(r["urgent_items"]) > 0) == mode.startswith("window")
    assert r["status"] == "ok"
    assert r["visits"] == r["expected"]
    assert r["exact_once"] == "1" and r["per_item_epochs_ok"] == "1"


@pytest.mark.parametrize("mode", ["fifo", "window", "window8"])
def test_slow_worker_is_still_correct(model, mode):
    r = run(model, 6, 100, 6, 3, 7, "stall", mode)
    assert r["status"] == "ok" and r["exact_once"] == "1"


@pytest.mark.parametrize("seed", [11, 12, 13])
@pytest.mark.parametrize("mode", ["fifo", "window", "window8"])
def test_slow_publication_is_still_correct(model, mode, seed):
    """Producers that pause between reserving a position and writing it:
    the window takes the ready tokens behind the reserved one, the head
    waits for it, and the 17 slots of headroom keep every slot from being
    written again before it was taken."""
    r = run(model, 12, 400, 12, 3, seed, "slowpub", mode)
    assert r["status"] == "ok", r
    assert r["visits"] == r["expected"] and r["exact_once"] == "1"


@pytest.mark.parametrize("mode", ["fifo", "window", "window8"])
def test_too_small_rings_are_detected(model, mode):
    """A planted mistake in the model (rings of a quarter of the segments):
    a producer about to overwrite a token not yet taken is seen."""
    r = run(model, 4, 200, 4, 3, 1, "smallring", mode)
    assert r["status"] == "overwrite" and r["exact_once"] == "0"


@pytest.mark.parametrize("mode", ["fifo", "window", "window8"])
def test_dropped_token_is_detected_by_timeout(model, mode):
    """A lost message: the bounded wait gives up and the status says so; the
    accounting shows the missing visits."""
    r = run(model, 4, 30, 4, 2, 8, "drop", mode)
    assert r["status"] == "timeout"
    assert int(r["visits"]) < int(r["expected"]) and r["exact_once"] == "0"


@pytest.mark.parametrize("mode", ["fifo", "window", "window8"])
def test_duplicated_token_is_detected(model, mode):
    """A duplicated message breaks exactly-once: two owners of one item, or a
    visit count other than one, or a worker starved of its quota."""
    r = run(model, 4, 30, 4, 2, 9, "dup", mode)
    assert r["status"] in ("ownership", "timeout") or r["exact_once"] == "0"
