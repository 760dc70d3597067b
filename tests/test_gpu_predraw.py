"""Rounding bits drawn before the launch for the items with most ratings
(bfloat16 and E4M3 storage of W).

When the ratings of the most-rated items (at least half the largest item
degree) are at most a quarter of all ratings, nomad_load_ratings reserves
room for their W rounding bits and every one-epoch launch draws them first
(the same Philox counters as the kernel's own draws, R14), so that the
visits of those items read them instead of drawing.  The input here is an
item rated by every user next to many light items: users 0 .. 999 rated
that item only, so their rows are written exactly once per epoch, by that
item's visits, with the pre-drawn bits.

A wrong bit moves a stored value by one bfloat16 (or E4M3) step with
probability about one half per write.  With the right bits a value differs
from the oracle's replay only where the binary32 value being rounded
differs (the block form of a long visit and the lane-tree dot products
differ from the sequential update by a few units in the last place, and the
differences grow along the item's chain of visits).  So the fraction of
entries of those rows that differ from the oracle's replay by more than
1e-3 relative (a rounding step; an E4M3 scale that moved by an ulp moves
the row by 1.2e-7) separates the two: it must stay below 10% (wrong bits
give about 50%).
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1312_0193_gb300 import Nomad  # noqa: E402

ONLY_HEAVY = 1000  # users 0 .. 999 rated the heavy item only
DIFF_FRAC = 0.10


def heavy_item_ratings(m=3000, n=400, density=0.05, seed=3):
    """Item 0 rated by every user; users ONLY_HEAVY .. m-1 also rate each of
    items 1 .. n-1 with probability `density`.  Values ~ N(3.5, 1)."""
    rng = np.random.default_rng(seed)
    rows = [np.arange(m, dtype=np.int32)]
    cols = [np.zeros(m, np.int32)]
    mask = rng.random((m - ONLY_HEAVY, n - 1)) < density
    r, c = np.nonzero(mask)
    rows.append((r + ONLY_HEAVY).astype(np.int32))
    cols.append((c + 1).astype(np.int32))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.normal(3.5, 1.0, size=rows.size).astype(np.float32)
    return m, n, rows, cols, vals


def urgent_ratings(n, cols):
    deg = np.bincount(cols, minlength=n)
    return int(deg[2 * deg >= deg.max()].sum())


@pytest.mark.parametrize("precision", ["bf16", "fp8", "fp32"])
def test_predrawn_bits_reserved_only_for_narrow_formats(precision):
    m, n, tr, tc, tv = heavy_item_ratings()
    with Nomad(m, n, 32, 0.05, precision=precision, n_workers=16) as nm:
        nm.load_coo(torch.from_numpy(tr).cuda(), torch.from_numpy(tc).cuda(),
                    torch.from_numpy(tv).cuda())
        got = nm.info()["predrawn_ratings"]
    assert 4 * urgent_ratings(n, tc) <= tr.size
    assert got == (urgent_ratings(n, tc) if precision != "fp32" else 0)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_predrawn_bits_replay(precision):
    """One epoch in debug mode at alpha 0.01 (16 workers: the heavy item's
    visits have ~190 ratings and run in block form out of turn), replayed by
    the oracle in the logged order from the same initial factors."""
    m, n, tr, tc, tv = heavy_item_ratings()
    k, p, lam, alpha, beta, seed = 32, 16, 0.05, 0.01, 0.05, 11
    with Nomad(m, n, k, lam, alpha=alpha, beta=beta, debug=True, n_workers=p, seed=seed,
               precision=precision) as nm:
        nm.load_coo(torch.from_numpy(tr).cuda(), torch.from_numpy(tc).cuda(),
                    torch.from_numpy(tv).cuda())
        assert nm.info()["predrawn_ratings"] == urgent_ratings(n, tc)
        rw = oracle.partition_rows(m, tr, p)
        L = oracle.build_layout(m, n, tr, tc, tv, rw, p)
        W0, H0 = nm.factors()
        nm.epoch(1)
        nm.check()
        seg, ep = nm.replay_log()
        Wg, Hg = nm.factors()
        counts, viol = nm.debug_counts()
    assert viol == 0 and np.all(counts == 1)
    f32 = lambda x: float(np.float32(x))
    if precision == "bf16":
        Wb, Hb, cnt = oracle.replay_bf16(L, seg, ep, oracle.bf16_rn(W0), oracle.bf16_rn(H0),
                                         f32(lam), f32(alpha), f32(beta), seed)
        Wo = oracle.bf16_to_f32(Wb)
    else:
        c0, s0 = oracle.e4m3_rows(oracle.init_factor(m, k, seed, 0).astype(np.float32))
        assert np.array_equal(W0, oracle.e4m3_decode_rows(c0, s0))
        Wc, Ws, Ho, cnt = oracle.replay_e4m3(L, seg, ep, c0, s0, H0, f32(lam), f32(alpha),
                                             f32(beta), seed)
        Wo = oracle.e4m3_decode_rows(Wc, Ws)
    assert np.array_equal(cnt, counts)
    # a differing rounding decision moves a value by one step: at least 2^-8
    # relative in bfloat16, 1/16 in E4M3; an E4M3 row whose scale differs by
    # an ulp (its largest magnitude differed by an ulp) moves by 1.2e-7 only
    g, o = Wg[:ONLY_HEAVY].astype(np.float64), Wo[:ONLY_HEAVY].astype(np.float64)
    differ = float(np.mean(np.abs(g - o) > 1e-3 * np.abs(o)))
    print("%s: entries of the heavy-only rows that differ from the replay: %.4f" % (
        precision, differ))
    assert differ <= DIFF_FRAC, differ
