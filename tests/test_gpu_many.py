"""Several independent problems in one persistent launch (nomad_epoch_many),
against the oracle: each problem's logged visit order replays to its factors
(binary32 and binary64, 1e-4 relative L2), its accounting is bit-exact, and
a free run reaches the test RMSE of the same problem run alone.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1312_0193_gb300 import Nomad, NomadError  # noqa: E402
from paper_1312_0193_gb300 import nomad as nb  # noqa: E402

REPLAY_TOL = 1e-4


ROW_TOL = 1e-3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) /
                 max(np.linalg.norm(np.asarray(b, np.float64)), 1e-300))


def row_rel_max(a, b):
    """max over rows of the relative L2 difference (rows of b that are zero
    must match exactly)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm(a - b, axis=1)
    nb_ = np.linalg.norm(b, axis=1)
    assert np.all(d[nb_ == 0] == 0)
    return float((d[nb_ > 0] / nb_[nb_ > 0]).max()) if np.any(nb_ > 0) else 0.0


def make(r, k, lam, **kw):
    nm = Nomad(r.m, r.n, k, lam, **kw)
    nm.load_coo(r.train_rows.cuda(), r.train_cols.cuda(), r.train_vals.cuda())
    return nm


# (data, k, lambda, alpha, beta, workers): short and long visits, urgent items,
# three row widths of one chunk per lane, different step-size schedules
PROBLEMS = [
    (lambda: synth.tiny_planted(1), 10, 0.05, 0.05, 0.05, 16),
    (lambda: synth.netflix_shaped(0.002, seed=13), 100, 0.05, 0.01, 0.05, 24),
    (lambda: synth.netflix_shaped(0.0005, seed=7), 64, 0.1, 0.02, 0.01, 8),
]


def test_many_replay_each_problem():
    """Three problems, two calls of 3 epochs each (one launch per epoch, all
    problems in it); every problem replays on the oracle as if it had run
    alone."""
    epochs, calls = 3, 2
    runs = []
    try:
        for gen, k, lam, alpha, beta, p in PROBLEMS:
            r = gen()
            nm = make(r, k, lam, alpha=alpha, beta=beta, debug=True, n_workers=p)
            tr, tc, tv, *_ = r.numpy()
            rw = oracle.partition_rows(r.m, tr, p)
            L = oracle.build_layout(r.m, r.n, tr, tc, tv, rw, p)
            W0, H0 = nm.factors()
            runs.append(dict(nm=nm, L=L, lam=float(np.float32(lam)), a=float(np.float32(alpha)),
                             b=float(np.float32(beta)), W32=W0.copy(), H32=H0.copy(),
                             W64=W0.astype(np.float64), H64=H0.astype(np.float64),
                             c32=None, c64=None))
        for c in range(calls):
            Nomad.epoch_many([x["nm"] for x in runs], epochs)
            for x in runs:
                nm, L = x["nm"], x["L"]
                nm.check()
                seg, ep = nm.replay_log()
                S = L["seg_col"].size
                assert seg.size == S * epochs
                for e in range(c * epochs, (c + 1) * epochs):
                    assert np.array_equal(np.sort(seg[ep == e]), np.arange(S))
                x["W32"], x["H32"], x["c32"] = oracle.replay(
                    L, seg, x["W32"], x["H32"], x["lam"], x["a"], x["b"], precision="f32",
                    rec_count=x["c32"])
                x["W64"], x["H64"], x["c64"] = oracle.replay(
                    L, seg, x["W64"], x["H64"], x["lam"], x["a"], x["b"], precision="f64",
                    rec_count=x["c64"])
        for x in runs:
            Wg, Hg = x["nm"].factors()
            counts, viol = x["nm"].debug_counts()
            assert viol == 0
            assert np.all(counts == calls * epochs)
            assert np.array_equal(counts, x["c32"])
            for g, o in ((Wg, x["W32"]), (Hg, x["H32"]), (Wg, x["W64"]), (Hg, x["H64"])):
                assert rel(g, o) < REPLAY_TOL, rel(g, o)
                assert row_rel_max(g, o) < ROW_TOL, row_rel_max(g, o)
    finally:
        for x in runs:
            x["nm"].close()


def test_many_free_run_matches_alone():
    """Four problems, 10 epochs together (one launch per epoch): each
    problem's test RMSE is within 0.5% of the same problem run alone with
    the same workers."""
    specs = [(synth.tiny_planted(1), 10, 0.05, 16),
             (synth.netflix_shaped(0.002, seed=13), 100, 0.05, 40),
             (synth.netflix_shaped(0.001, seed=21), 32, 0.05, 24),
             (synth.netflix_shaped(0.0005, seed=7), 64, 0.1, 8)]
    alone, together = [], []
    for r, k, lam, p in specs:
        with make(r, k, lam, n_workers=p) as nm:
            nm.epoch(10)
            alone.append(nm.rmse(*r.numpy()[3:]))
    nms = [make(r, k, lam, n_workers=p) for r, k, lam, p in specs]
    try:
        Nomad.epoch_many(nms, 10)
        ms = nms[0].last_epoch_kernel_ms()
        spans = [nm.last_epoch_span_ns() for nm in nms]
        # each problem's device span lies within the call (CUDA events
        # around its launches), and the call lasts about as long as its
        # slowest problem
        assert all(0 < s <= ms * 1e6 * 1.02 + 5e4 for s in spans), (spans, ms)
        assert max(spans) >= 0.5 * ms * 1e6, (spans, ms)
        for nm, (r, *_rest) in zip(nms, specs):
            nm.check()
            together.append(nm.rmse(*r.numpy()[3:]))
            # every handle records its own events around the call's launches
            assert abs(nm.last_epoch_kernel_ms() - ms) < 0.05
    finally:
        for nm in nms:
            nm.close()
    for a, t in zip(alone, together):
        assert abs(t - a) <= 0.005 * a, (alone, together)


def test_many_rejects_what_it_cannot_run():
    r = synth.tiny_planted(1)
    a = make(r, 10, 0.05, n_workers=16)
    b = make(r, 10, 0.05, n_workers=16, precision="bf16")
    c = make(r, 10, 0.05, n_workers=16, mode="uniform")
    d = Nomad(r.m, r.n, 10, 0.05)
    big = [make(r, 10, 0.05, n_workers=800) for _ in range(2)]  # 2 x 100 blocks
    try:
        for hs, code in (([a, a], nb.NOMAD_ERR_INVALID_ARG),
                         ([a, b], nb.NOMAD_ERR_UNSUPPORTED),
                         ([a, c], nb.NOMAD_ERR_UNSUPPORTED),
                         ([a, d], nb.NOMAD_ERR_STATE),
                         (big, nb.NOMAD_ERR_UNSUPPORTED)):
            with pytest.raises(NomadError) as e:
                Nomad.epoch_many(hs, 1)
            assert e.value.code == code, (code, e.value)
        with pytest.raises(NomadError) as e:
            nb.nomad_epoch_many([], 1, None)
        assert e.value.code == nb.NOMAD_ERR_INVALID_ARG
        # a rejected call runs nothing; a valid one still runs afterwards
        Nomad.epoch_many([a], 2)
        a.check()
        assert a.info()["epochs_done"] == 2
    finally:
        for x in [a, b, c, d] + big:
            x.close()


def test_many_bf16_replay_with_predrawn_bits():
    """bfloat16 storage, two problems together for one epoch: one whose
    most-rated item holds a small share of the ratings (its rounding bits
    are drawn before the launch) and the tiny planted one (drawn in the
    kernel); each replays on the oracle's bfloat16 replay within 1e-2
    relative L2 (the bound of the one-problem bfloat16 test)."""
    rng = np.random.default_rng(3)
    m, n = 3000, 400
    mask = rng.random((m - 1000, n - 1)) < 0.05
    rr, cc = np.nonzero(mask)
    rows = np.concatenate([np.arange(m), rr + 1000]).astype(np.int32)
    cols = np.concatenate([np.zeros(m, np.int64), cc + 1]).astype(np.int32)
    vals = rng.normal(3.5, 1.0, size=rows.size).astype(np.float32)
    heavy = synth.Ratings(m, n, torch.from_numpy(rows), torch.from_numpy(cols),
                          torch.from_numpy(vals), torch.zeros(0, dtype=torch.int32),
                          torch.zeros(0, dtype=torch.int32), torch.zeros(0))
    seed, lam, alpha, beta = 11, 0.05, 0.01, 0.05
    runs = []
    try:
        for r, k, p in ((heavy, 32, 16), (synth.tiny_planted(1), 10, 16)):
            nm = make(r, k, lam, alpha=alpha, beta=beta, debug=True, n_workers=p, seed=seed,
                      precision="bf16")
            tr, tc, tv, *_ = r.numpy()
            L = oracle.build_layout(r.m, r.n, tr, tc, tv, oracle.partition_rows(r.m, tr, p), p)
            runs.append((nm, L, nm.factors()))
        assert runs[0][0].info()["predrawn_ratings"] == m
        assert runs[1][0].info()["predrawn_ratings"] == 0
        Nomad.epoch_many([x[0] for x in runs], 1)
        f32 = lambda x: float(np.float32(x))
        for nm, L, (W0, H0) in runs:
            nm.check()
            seg, ep = nm.replay_log()
            Wg, Hg = nm.factors()
            counts, viol = nm.debug_counts()
            assert viol == 0 and np.all(counts == 1)
            Wb, Hb, cnt = oracle.replay_bf16(L, seg, ep, oracle.bf16_rn(W0), oracle.bf16_rn(H0),
                                             f32(lam), f32(alpha), f32(beta), seed)
            assert np.array_equal(cnt, counts)
            assert rel(Wg, oracle.bf16_to_f32(Wb)) < 1e-2
            assert rel(Hg, oracle.bf16_to_f32(Hb)) < 1e-2
    finally:
        for x in runs:
            x[0].close()
