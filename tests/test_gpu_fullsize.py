"""Full-size checks on the Netflix-shaped workload (m=480,189, n=17,770,
~100.5M ratings, k=100) in the launch configuration bench.py times (all
resident warps as workers, default block size).

* the layout built on the device equals the oracle's, bit for bit;
* the test RMSE of the device reduction equals the oracle's on the device
  factors (binary32 residuals, binary64 sums; 1e-6 relative);
* one epoch in debug mode (same grid, the kernel variant that also logs)
  replays on the oracle to the same factors within 1e-4 relative L2, with
  every rating updated exactly once;
* one non-debug epoch lowers the objective and the test RMSE.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_1312_0193_gb300 import Nomad  # noqa: E402


@pytest.fixture(scope="module")
def netflix():
    r = synth.netflix_shaped(1.0, device=torch.device("cuda", 0))
    host = r.numpy()
    return r, host


@pytest.fixture(scope="module")
def oracle_layout_full(netflix):
    r, (tr, tc, tv, *_) = netflix
    with Nomad(r.m, r.n, 100, 0.05) as nm:
        p = nm.info()["p"]
    rw = oracle.partition_rows(r.m, tr, p)
    return p, rw, oracle.build_layout(r.m, r.n, tr, tc, tv, rw, p)


def test_fullsize_layout_bit_exact(netflix, oracle_layout_full):
    r, _ = netflix
    p, rw, L = oracle_layout_full
    with Nomad(r.m, r.n, 100, 0.05) as nm:
        nm.load_coo(r.train_rows, r.train_cols, r.train_vals)
        G = nm.layout()
        assert nm.info()["p"] == p
    assert np.array_equal(G["row_worker"], rw)
    for key in ("seg_worker", "seg_col", "seg_ptr", "rec_row"):
        assert np.array_equal(G[key], L[key]), key
    assert np.array_equal(G["rec_val"], L["rec_val"].astype(np.float32))


def test_fullsize_epoch_replay_and_rmse(netflix, oracle_layout_full):
    r, (tr, tc, tv, er, ec, ev) = netflix
    p, rw, L = oracle_layout_full
    lam, alpha, beta = 0.05, 0.012, 0.05
    with Nomad(r.m, r.n, 100, lam, alpha=alpha, beta=beta, debug=True) as nm:
        nm.load_coo(r.train_rows, r.train_cols, r.train_vals)
        W0, H0 = nm.factors()
        nm.epoch(1)
        nm.check()
        seg, ep = nm.replay_log()
        Wg, Hg = nm.factors()
        counts, viol = nm.debug_counts()
        got_rmse = nm.rmse(r.test_rows, r.test_cols, r.test_vals)
    assert viol == 0 and np.all(counts == 1)
    assert seg.size == L["seg_col"].size and np.array_equal(np.sort(seg), np.arange(seg.size))
    Wo, Ho, cnt = oracle.replay(L, seg, W0, H0, float(np.float32(lam)),
                                float(np.float32(alpha)), float(np.float32(beta)),
                                precision="f32")
    assert np.all(cnt == 1)
    for g, o in ((Wg, Wo), (Hg, Ho)):
        d = np.linalg.norm(g.astype(np.float64) - o) / np.linalg.norm(o.astype(np.float64))
        assert d < 1e-4, d
        # every row on its own: one skipped or doubled update moves one row by
        # a whole step, which the norm over 48M entries could hide
        g64, o64 = g.astype(np.float64), o.astype(np.float64)
        rows = np.linalg.norm(g64 - o64, axis=1) / np.maximum(np.linalg.norm(o64, axis=1), 1e-30)
        assert rows.max() < 1e-3, rows.max()
    want = oracle.rmse(er, ec, ev, Wg.astype(np.float64), Hg.astype(np.float64))
    assert abs(got_rmse - want) <= 1e-6 * want


def test_fullsize_free_epoch_descends(netflix):
    r, (tr, tc, tv, er, ec, ev) = netflix
    with Nomad(r.m, r.n, 100, 0.05) as nm:
        nm.load_coo(r.train_rows, r.train_cols, r.train_vals)
        J0 = nm.objective()
        R0 = nm.rmse(r.test_rows, r.test_cols, r.test_vals)
        nm.epoch(1)
        nm.check()
        J1 = nm.objective()
        R1 = nm.rmse(r.test_rows, r.test_cols, r.test_vals)
    assert J1 < J0 and R1 < R0
