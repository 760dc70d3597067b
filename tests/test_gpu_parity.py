"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work (partition, layout, accounting) must match bit for bit; the
factors of a replayed run must match the oracle's replay of the logged
serial order within 1e-4 relative L2 (binary32 arithmetic on both sides,
different summation order inside the dot product); reductions within the
tolerance derived from binary32 residuals summed in binary64.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1312_0193_gb300 import Nomad, NomadError  # noqa: E402
from paper_1312_0193_gb300 import nomad as nb  # noqa: E402

REPLAY_TOL = 1e-4      # relative L2, factors after a replayed run
ROW_TOL = 1e-3         # relative L2 of every single row after a replayed run
REDUCE_TOL = 1e-6      # relative, RMSE and objective


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) /
                 max(np.linalg.norm(np.asarray(b, np.float64)), 1e-300))


def row_rel_max(a, b):
    """max over rows i of |a_i - b_i| / |b_i| (rows with b_i = 0 must match
    exactly).  A skipped or doubled update changes one row by the size of a
    step, which a whole-matrix norm can hide at full size; one row's norm
    cannot."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm(a - b, axis=1)
    nb_ = np.linalg.norm(b, axis=1)
    zero = nb_ == 0
    assert np.all(d[zero] == 0)
    return float((d[~zero] / nb_[~zero]).max()) if np.any(~zero) else 0.0


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_planted(1)


def make(r, k, lam, **kw):
    nm = Nomad(r.m, r.n, k, lam, **kw)
    tr, tc, tv = r.train_rows, r.train_cols, r.train_vals
    nm.load_coo(tr.cuda(), tc.cuda(), tv.cuda())
    return nm


def oracle_layout(nm, r):
    tr, tc, tv, *_ = r.numpy()
    p = nm.info()["p"]
    mode = "users" if nm.schedule.partition == nb.NOMAD_PARTITION_USERS else "ratings"
    rw = oracle.partition_rows(r.m, tr, p, mode=mode)
    return oracle.build_layout(r.m, r.n, tr, tc, tv, rw, p), rw


# ---------------------------------------------------------------- init
@pytest.mark.parametrize("k,seed", [(10, 2), (100, 7), (3, 11), (130, 5)])
def test_init_bit_exact(k, seed):
    with Nomad(257, 129, k, 0.05, seed=seed) as nm:
        W, H = nm.factors()
    assert np.array_equal(W.astype(np.float64), oracle.init_factor(257, k, seed, 0))
    assert np.array_equal(H.astype(np.float64), oracle.init_factor(129, k, seed, 1))


# ---------------------------------------------------------------- layout
@pytest.mark.parametrize("p,partition", [(8, "ratings"), (37, "ratings"),
                                         (16, "users"), (1, "ratings")])
def test_layout_bit_exact(tiny, p, partition):
    with make(tiny, 10, 0.05, n_workers=p, partition=partition) as nm:
        L, rw = oracle_layout(nm, tiny)
        G = nm.layout()
        info = nm.info()
    assert info["p"] == p and info["nnz"] == tiny.nnz
    assert np.array_equal(G["row_worker"], rw)
    assert info["n_segments"] == L["seg_col"].size
    assert np.array_equal(G["seg_worker"], L["seg_worker"])
    assert np.array_equal(G["seg_col"], L["seg_col"])
    assert np.array_equal(G["seg_ptr"], L["seg_ptr"])
    assert np.array_equal(G["rec_row"], L["rec_row"])
    assert np.array_equal(G["rec_val"], L["rec_val"].astype(np.float32))


def test_layout_skewed_auto_workers():
    r = synth.netflix_shaped(0.004, seed=5)
    with make(r, 100, 0.05) as nm:
        L, rw = oracle_layout(nm, r)
        G = nm.layout()
    assert np.array_equal(G["row_worker"], rw)
    for key in ("seg_worker", "seg_col", "seg_ptr", "rec_row"):
        assert np.array_equal(G[key], L[key]), key


def test_csc_input_matches_coo(tiny):
    tr, tc, tv, *_ = tiny.numpy()
    order = np.lexsort((tr, tc))
    colptr = np.zeros(tiny.n + 1, np.int64)
    np.add.at(colptr, tc + 1, 1)
    colptr = np.cumsum(colptr)
    with Nomad(tiny.m, tiny.n, 10, 0.05, n_workers=8) as a, \
            Nomad(tiny.m, tiny.n, 10, 0.05, n_workers=8) as b:
        a.load_coo(tr, tc, tv)                       # host COO
        b.load_csc(torch.from_numpy(colptr).cuda(), torch.from_numpy(tr[order]).cuda(),
                   torch.from_numpy(tv[order]).cuda())  # device CSC
        La, Lb = a.layout(), b.layout()
    for key in La:
        assert np.array_equal(La[key], Lb[key]), key


def test_input_errors(tiny):
    tr, tc, tv, *_ = tiny.numpy()
    with Nomad(tiny.m, tiny.n, 10, 0.05) as nm:
        with pytest.raises(NomadError) as e:
            nm.epoch(1)
        assert e.value.code == nb.NOMAD_ERR_STATE
        bad = tr.copy()
        bad[5] = tiny.m
        with pytest.raises(NomadError) as e:
            nm.load_coo(bad, tc, tv)
        assert e.value.code == nb.NOMAD_ERR_RANGE
        dup_r = np.concatenate([tr, tr[:1]])
        dup_c = np.concatenate([tc, tc[:1]])
        dup_v = np.concatenate([tv, tv[:1]])
        with pytest.raises(NomadError) as e:
            nm.load_coo(dup_r, dup_c, dup_v)
        assert e.value.code == nb.NOMAD_ERR_DUP_ENTRY
        nm.load_coo(tr, tc, tv)  # a good load after failed ones works
        nm.epoch(1)
        nm.check()
    with pytest.raises(NomadError):
        Nomad(10, 10, 0, 0.1)
    with pytest.raises(NomadError):
        Nomad(10, 10, 600, 0.1)


# ---------------------------------------------------------------- replay
def replay_check(r, k, lam, alpha, beta, epochs, p=None, calls=1, **kw):
    """Run `calls` nomad_epoch calls in debug mode; replay each call's log on
    the oracle (binary32 and binary64) and compare factors and accounting."""
    a32, b32 = float(np.float32(alpha)), float(np.float32(beta))
    lam32 = float(np.float32(lam))
    with make(r, k, lam, alpha=alpha, beta=beta, debug=True,
              n_workers=p or 0, **kw) as nm:
        L, _ = oracle_layout(nm, r)
        S = L["seg_col"].size
        W0, H0 = nm.factors()
        W32, H32 = W0.copy(), H0.copy()
        W64, H64 = W0.astype(np.float64), H0.astype(np.float64)
        cnt32 = cnt64 = None
        for c in range(calls):
            nm.epoch(epochs)
            nm.check()
            seg, ep = nm.replay_log()
            # accounting: every segment once per epoch, epochs in range
            assert seg.size == S * epochs
            assert ep.min() == c * epochs and ep.max() == (c + 1) * epochs - 1
            for e in range(c * epochs, (c + 1) * epochs):
                assert np.array_equal(np.sort(seg[ep == e]), np.arange(S))
            # per item, visits are in epoch order
            for j in np.unique(L["seg_col"])[:50]:
                mine = ep[L["seg_col"][seg] == j]
                assert np.all(np.diff(mine) >= 0)
            W32, H32, cnt32 = oracle.replay(L, seg, W32, H32, lam32, a32, b32,
                                            precision="f32", rec_count=cnt32)
            W64, H64, cnt64 = oracle.replay(L, seg, W64, H64, lam32, a32, b32,
                                            precision="f64", rec_count=cnt64)
        Wg, Hg = nm.factors()
        counts, viol = nm.debug_counts()
    assert viol == 0
    assert np.all(counts == calls * epochs)
    assert np.array_equal(counts, cnt32)
    for g, o in ((Wg, W32), (Hg, H32), (Wg, W64), (Hg, H64)):
        assert rel(g, o) < REPLAY_TOL, rel(g, o)
        assert row_rel_max(g, o) < ROW_TOL, row_rel_max(g, o)
    return Wg, Hg


@pytest.mark.parametrize("variant", ["batched", "simple"])
def test_replay_tiny_paper_schedule(tiny, variant):
    """Tiny planted config, the paper's decaying step size (alpha 0.012, beta
    0.05), 20 epochs, replayed on the oracle."""
    replay_check(tiny, 10, 0.05, 0.012, 0.05, 20, p=64, variant=variant)


@pytest.mark.parametrize("variant", ["batched", "simple"])
def test_replay_tiny_large_steps(tiny, variant):
    """Larger steps (alpha 0.1, beta 0.01) move the factors far from the
    start, so the comparison is sensitive to any arithmetic difference."""
    replay_check(tiny, 10, 0.05, 0.1, 0.01, 20, p=64, variant=variant)


@pytest.mark.parametrize("p", [4, 16, 64])
def test_replay_few_workers_long_visits(p):
    """Few workers: long visits (>= 32 ratings, pushed right after their
    visit, and taken out of turn when they arrive during another batch's
    stream of short visits), many rows shared between the visits of one
    batch (the prefetch-hazard path), records streamed in several chunks."""
    r = synth.netflix_shaped(0.002, seed=13)
    replay_check(r, 100, 0.05, 0.01, 0.05, 2, p=p)


def test_replay_auto_workers_two_calls(tiny):
    """All resident warps as workers (about 20 ratings per worker), two calls
    of 3 epochs: the step size continues from the epoch count."""
    replay_check(tiny, 10, 0.05, 0.05, 0.05, 3, calls=2)


@pytest.mark.parametrize("k", [1, 7, 64, 100, 128, 129, 256, 300])
def test_replay_ranks(k):
    """Every supported chunking of k (1, 2 or 4 float4 chunks per lane,
    ragged tails) on a small skewed problem."""
    r = synth.netflix_shaped(0.0005, seed=k)
    replay_check(r, k, 0.05, 0.01, 0.05, 2, p=48)


def test_replay_users_partition(tiny):
    replay_check(tiny, 10, 0.05, 0.05, 0.05, 3, p=20, partition="users")


# ---------------------------------------------------------------- reductions
def test_rmse_and_objective(tiny):
    tr, tc, tv, er, ec, ev = tiny.numpy()
    with make(tiny, 10, 0.05, alpha=0.1, beta=0.01) as nm:
        nm.epoch(3)
        W, H = nm.factors()
        got_dev = nm.rmse(tiny.test_rows.cuda(), tiny.test_cols.cuda(), tiny.test_vals.cuda())
        got_host = nm.rmse(er, ec, ev)
        J = nm.objective()
    want = oracle.rmse(er, ec, ev, W.astype(np.float64), H.astype(np.float64))
    assert abs(got_dev - want) <= REDUCE_TOL * want
    assert got_host == got_dev
    Jw = oracle.objective(tr, tc, tv, W.astype(np.float64), H.astype(np.float64),
                          float(np.float32(0.05)))
    assert abs(J - Jw) <= REDUCE_TOL * Jw


def test_rmse_empty_and_one():
    with Nomad(5, 4, 3, 0.1) as nm:
        assert np.isnan(nm.rmse(np.zeros(0, np.int32), np.zeros(0, np.int32),
                                np.zeros(0, np.float32)))
        W, H = nm.factors()
        v = nm.rmse(np.array([2], np.int32), np.array([3], np.int32),
                    np.array([1.5], np.float32))
    want = oracle.rmse([2], [3], [1.5], W.astype(np.float64), H.astype(np.float64))
    assert abs(v - want) <= REDUCE_TOL * want


def test_set_get_factors_roundtrip(tiny):
    rng = np.random.default_rng(0)
    W = rng.normal(size=(tiny.m, 10)).astype(np.float32)
    H = rng.normal(size=(tiny.n, 10)).astype(np.float32)
    with make(tiny, 10, 0.05) as nm:
        nm.set_factors(W, H, epochs_done=7)
        W2, H2 = nm.factors()
        assert nm.info()["epochs_done"] == 7
    assert np.array_equal(W, W2) and np.array_equal(H, H2)


def test_resume_from_checkpoint_replays(tiny):
    """Checkpoint and resume: a handle runs 2 epochs, its factors go to the
    host, a new handle takes them with epochs_done = 2 and runs 2 more in
    debug mode.  Its log has epochs 2 and 3 only, and the oracle's replay of
    it from the checkpoint (every rating's update count starting at 2, so
    the step sizes continue at t = 2) matches within the replay bound."""
    lam, alpha, beta = 0.05, 0.02, 0.05
    with make(tiny, 10, lam, alpha=alpha, beta=beta, n_workers=16) as nm:
        nm.epoch(2)
        nm.check()
        W1, H1 = nm.factors()
    a32, b32, lam32 = (float(np.float32(x)) for x in (alpha, beta, lam))
    with make(tiny, 10, lam, alpha=alpha, beta=beta, n_workers=16, debug=True) as nm:
        nm.set_factors(W1, H1, epochs_done=2)
        assert nm.info()["epochs_done"] == 2
        L, _ = oracle_layout(nm, tiny)
        nm.epoch(2)
        nm.check()
        seg, ep = nm.replay_log()
        Wg, Hg = nm.factors()
        counts, viol = nm.debug_counts()
        assert nm.info()["epochs_done"] == 4
    assert viol == 0 and np.all(counts == 2)
    assert ep.min() == 2 and ep.max() == 3
    S = L["seg_col"].size
    for e in (2, 3):
        assert np.array_equal(np.sort(seg[ep == e]), np.arange(S))
    start = np.full(L["rec_row"].size, 2, np.int32)
    Wo, Ho, cnt = oracle.replay(L, seg, W1, H1, lam32, a32, b32, precision="f32",
                                rec_count=start)
    assert np.all(cnt == 4)
    for g, o in ((Wg, Wo), (Hg, Ho)):
        assert rel(g, o) < REPLAY_TOL, rel(g, o)
        assert row_rel_max(g, o) < ROW_TOL, row_rel_max(g, o)
    # the step sizes matter: replayed as if from epoch 0 the result differs
    Wz, _, _ = oracle.replay(L, seg, W1, H1, lam32, a32, b32, precision="f32")
    assert rel(Wz, Wo) > 10 * REPLAY_TOL


# ---------------------------------------------------------------- failure path
def test_lost_token_times_out_and_recovers(tiny):
    """A planted lost message (one item's token never handed out): the worker
    that waits for it gives up after the timeout, nomad_check reports
    NOMAD_ERR_TIMEOUT, and the next call runs normally."""
    tr, *_ = tiny.numpy()
    item = int(tiny.train_cols[0])
    with make(tiny, 10, 0.05, n_workers=16, spin_timeout_ns=200_000_000,
              debug_drop_item=item) as nm:
        nm.epoch(1)
        with pytest.raises(NomadError) as e:
            nm.check()
        assert e.value.code == nb.NOMAD_ERR_TIMEOUT
        nm.check()  # cleared


def test_lost_token_error_kept_across_a_calls_launches(tiny):
    """Several epochs run as one launch per epoch: the first launch's timeout
    stays in the status word (a later launch of the same call does not clear
    it), and the later launches stop at their first wait instead of waiting
    out their own timeouts."""
    import time
    item = int(tiny.train_cols[0])
    timeout_ns = 300_000_000
    with make(tiny, 10, 0.05, n_workers=16, spin_timeout_ns=timeout_ns,
              debug_drop_item=item, epochs_per_launch=1) as nm:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nm.epoch(4)
        with pytest.raises(NomadError) as e:
            nm.check()
        dt = time.perf_counter() - t0
        assert e.value.code == nb.NOMAD_ERR_TIMEOUT
        assert nm.info()["kernel_launches"] >= 4
        # one timeout, not four
        assert dt < 2.5 * timeout_ns * 1e-9, dt
        nm.check()


# ---------------------------------------------------------------- free run
def test_free_run_matches_oracle_rmse(tiny):
    """Non-debug run of 20 epochs at the paper's schedule (alpha 0.012,
    beta 0.05): the test RMSE is within 0.5% of the binary64 oracle's serial
    NOMAD run (the visit orders differ; at this schedule the oracle's own
    spread over orders is about 0.01%, so 0.5% is a real bound)."""
    tr, tc, tv, er, ec, ev = tiny.numpy()
    with make(tiny, 10, 0.05, alpha=0.012, beta=0.05) as nm:
        W0, H0 = nm.factors()
        nm.epoch(20)
        g = nm.rmse(er, ec, ev)
        L, _ = oracle_layout(nm, tiny)
    Wo, Ho, _, _ = oracle.serial_nomad(L, W0, H0, 0.05, 0.012, 0.05, 20, 9)
    o = oracle.rmse(er, ec, ev, Wo, Ho)
    assert abs(g - o) <= 0.005 * o, (g, o)


def test_free_run_large_steps_within_order_spread(tiny):
    """With large steps (alpha 0.1, beta 0.01) the result depends on the visit
    order: the oracle's RMSE varies by several percent across orders.  The
    GPU's RMSE must lie within that spread (mean +- 3 std of 8 oracle runs
    with different orders, plus 0.5%)."""
    tr, tc, tv, er, ec, ev = tiny.numpy()
    with make(tiny, 10, 0.05, alpha=0.1, beta=0.01) as nm:
        W0, H0 = nm.factors()
        nm.epoch(20)
        g = nm.rmse(er, ec, ev)
        L, _ = oracle_layout(nm, tiny)
    runs = []
    for seed in range(1, 9):
        Wo, Ho, _, _ = oracle.serial_nomad(L, W0, H0, 0.05, 0.1, 0.01, 20, seed)
        runs.append(oracle.rmse(er, ec, ev, Wo, Ho))
    mu, sd = float(np.mean(runs)), float(np.std(runs))
    assert abs(g - mu) <= 3 * sd + 0.005 * mu, (g, mu, sd)


# ---------------------------------------------------------------- uniform mode
@pytest.mark.parametrize("p,routing", [(16, "uniform"), (64, "uniform"), (16, "shorter"),
                                       (64, "shorter")])
def test_uniform_mode_replay_and_budget(tiny, p, routing):
    """Alg. 1 literally: the next worker is uniform over all p (or, with the
    dynamic load balancing of Sec. 3.3, the one of two uniform draws with
    fewer tokens waiting), a visit to a worker without ratings of the item
    applies nothing, the per-rating update count gives t, and a call stops
    after n_epochs * nnz updates.  The logged order of non-empty visits
    replays to the same factors on the oracle."""
    tr, tc, tv, *_ = tiny.numpy()
    a32, b32, lam32 = (float(np.float32(x)) for x in (0.05, 0.05, 0.05))
    with make(tiny, 10, 0.05, alpha=0.05, beta=0.05, mode="uniform", debug=True,
              n_workers=p, routing=routing) as nm:
        L, _ = oracle_layout(nm, tiny)
        W0, H0 = nm.factors()
        nm.epoch(2)
        nm.check()
        seg, item = nm.replay_log()
        Wg, Hg = nm.factors()
        counts, viol = nm.debug_counts()
    assert viol == 0
    total = int(counts.sum())
    assert 2 * tiny.nnz <= total <= 2 * tiny.nnz + p * int(np.diff(L["seg_ptr"]).max())
    real = seg[seg >= 0]
    # every logged segment belongs to the logged item
    assert np.array_equal(L["seg_col"][real], item[seg >= 0])
    Wo, Ho, cnt = oracle.replay(L, real, W0, H0, lam32, a32, b32, precision="f32")
    assert np.array_equal(cnt, counts)
    assert rel(Wg, Wo) < REPLAY_TOL and rel(Hg, Ho) < REPLAY_TOL
    assert row_rel_max(Wg, Wo) < ROW_TOL and row_rel_max(Hg, Ho) < ROW_TOL
    assert seg.size > 5 * p  # many visits, some of them to workers without ratings


# ---------------------------------------------------------------- hybrid circulation
@pytest.mark.parametrize("p,k,epochs,calls", [(64, 10, 3, 2), (16, 100, 2, 1), (64, 100, 2, 1)])
def test_block_circulation_replay(p, k, epochs, calls):
    """The hybrid circulation of Sec. 3.4 (a token visits all of its workers
    in one thread block, handed over through shared-memory inboxes, before
    it moves to another block): every segment once per epoch, replay parity
    as for the flat circulation, and in every epoch each item's visits come
    in one contiguous run per block."""
    r = synth.tiny_planted(1) if k == 10 else synth.netflix_shaped(0.002, seed=13)
    replay_check(r, k, 0.05, 0.01, 0.05, epochs, p=p, calls=calls, circulation="block")
    # the run structure, from one more debug run's log
    with make(r, k, 0.05, alpha=0.01, beta=0.05, debug=True, n_workers=p,
              circulation="block") as nm:
        L, _ = oracle_layout(nm, r)
        wpb = nm.info()["warps_per_block"]
        nm.epoch(epochs)
        nm.check()
        seg, ep = nm.replay_log()
    blocks = L["seg_worker"][seg] // wpb
    items = L["seg_col"][seg]
    for e in range(epochs):
        for j in np.unique(items[ep == e])[:200]:
            b = blocks[(ep == e) & (items == j)]
            changes = np.flatnonzero(np.diff(b) != 0)
            # a block, once left, is not visited again in the epoch
            runs = np.concatenate([b[:1], b[changes + 1]])
            assert np.unique(runs).size == runs.size, (j, e, b)


def test_block_circulation_free_run_matches_oracle_rmse(tiny):
    """Non-debug run with the hybrid circulation, 20 epochs at the paper's
    schedule: test RMSE within 0.5% of the binary64 oracle's serial NOMAD."""
    tr, tc, tv, er, ec, ev = tiny.numpy()
    with make(tiny, 10, 0.05, alpha=0.012, beta=0.05, circulation="block") as nm:
        W0, H0 = nm.factors()
        nm.epoch(20)
        g = nm.rmse(er, ec, ev)
        L, _ = oracle_layout(nm, tiny)
    Wo, Ho, _, _ = oracle.serial_nomad(L, W0, H0, 0.05, 0.012, 0.05, 20, 9)
    o = oracle.rmse(er, ec, ev, Wo, Ho)
    assert abs(g - o) <= 0.005 * o, (g, o)


def test_block_circulation_only_batched_epoch():
    with pytest.raises(NomadError) as e:
        Nomad(10, 10, 4, 0.1, circulation="block", variant="simple")
    assert e.value.code == nb.NOMAD_ERR_UNSUPPORTED
    with pytest.raises(NomadError):
        Nomad(10, 10, 4, 0.1, circulation="block", mode="uniform")
