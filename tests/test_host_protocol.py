"""Host-side tests of the token-passing protocol and its failure detection.

ring_model.cc models the ring queues of the persistent kernel with host
threads (same slot format, reservation and publication order, bounded
waits).  Failures are made on the host: a token that is never sent, a token
sent twice, a slow worker.  No GPU is involved.
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


def run(exe, p, n, maxdeg, epochs, seed, fault):
    out = subprocess.run([exe, str(p), str(n), str(maxdeg), str(epochs), str(seed), fault],
                         capture_output=True, text=True, timeout=120, check=True).stdout
    return dict(kv.split("=") for kv in out.split())


@pytest.mark.parametrize("p,n,maxdeg,epochs,seed",
                         [(4, 50, 4, 3, 1), (8, 200, 8, 4, 2), (16, 300, 5, 2, 3),
                          (3, 1, 3, 5, 4), (6, 40, 1, 3, 5)])
def test_protocol_exactly_once(model, p, n, maxdeg, epochs, seed):
    """Every segment is visited exactly once per epoch, every item finishes
    all epochs, no token is held twice."""
    r = run(model, p, n, maxdeg, epochs, seed, "none")
    assert r["status"] == "ok"
    assert r["visits"] == r["expected"]
    assert r["exact_once"] == "1" and r["per_item_epochs_ok"] == "1"


def test_slow_worker_is_still_correct(model):
    r = run(model, 6, 100, 6, 3, 7, "stall")
    assert r["status"] == "ok" and r["exact_once"] == "1"


def test_dropped_token_is_detected_by_timeout(model):
    """A lost message: the bounded wait gives up and the status says so; the
    accounting shows the missing visits."""
    r = run(model, 4, 30, 4, 2, 8, "drop")
    assert r["status"] == "timeout"
    assert int(r["visits"]) < int(r["expected"]) and r["exact_once"] == "0"


def test_duplicated_token_is_detected(model):
    """A duplicated message breaks exactly-once: two owners of one item, or a
    visit count other than one, or a worker starved of its quota."""
    r = run(model, 4, 30, 4, 2, 9, "dup")
    assert r["status"] in ("ownership", "timeout") or r["exact_once"] == "0"
