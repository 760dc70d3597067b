"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values
worked by hand from the paper's formulas (tests/golden/), published
known-answer vectors, closed forms, finite differences, invariants and brute
force on tiny inputs.  They run without a GPU.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle
import synth
from conftest import golden_rows


# --------------------------------------------------------------- randomness
def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors."""
    rows = golden_rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_init_first_entry_from_kat():
    """W[0,0] with seed 0 and k=1 is the first KAT word mapped to [0,1):
    counter (0,0,0,0), key (0,0) -> 0x6627e8d5; u = 0x6627e8 / 2^24."""
    W = oracle.init_factor(1, 1, 0, 0)
    assert W[0, 0] == 0x6627e8 / 2.0 ** 24


def test_init_distribution():
    """Entries are UniformReal(0, 1/sqrt(k)) (Alg. 1 initialisation):
    support, mean 1/(2 sqrt k), variance 1/(12 k), and a KS test."""
    k = 10
    W = oracle.init_factor(2000, k, 12345, 0)
    H = oracle.init_factor(1500, k, 12345, 1)
    c = 1.0 / np.sqrt(k)
    for F in (W, H):
        assert F.min() >= 0.0 and F.max() < c
        x = F.ravel() / c
        assert abs(x.mean() - 0.5) < 0.01
        assert abs(x.var() - 1.0 / 12.0) < 0.003
        assert stats.kstest(x, "uniform").pvalue > 1e-4
    # W and H draw from different streams, and so do different seeds.
    assert not np.array_equal(W[:100], H[:100])
    assert not np.array_equal(W, oracle.init_factor(2000, k, 12346, 0))
    # Entries are binary32 values (the CUDA path stores binary32 factors).
    assert np.array_equal(W, W.astype(np.float32).astype(np.float64))


# --------------------------------------------------------------- step size
def test_step_size_table1():
    """s_t = alpha / (1 + beta t^1.5) at Table 1's constants (hand values)."""
    rows = golden_rows("step_size_table1.txt")
    assert len(rows) == 13
    for _, a, b, t, frac in rows:
        want = float(Fraction(frac))
        got = oracle.step_size(float(a), float(b), int(t))
        assert got == pytest.approx(want, rel=1e-15, abs=0)


# --------------------------------------------------------------- SGD update
def test_one_step_worked_example():
    """One update per Eq. w_update/h_update, descent-sign reading (golden)."""
    rows = {r[0]: r for r in golden_rows("one_step_update.txt")}
    _, k, lam, s, a, *rest = rows["A"]
    k = int(k)
    w, h, wn, hn, hn_new = map(float, rest)
    w1, h1 = oracle.sgd_update([w], [h], float(a), float(lam), float(s))
    assert w1[0] == pytest.approx(wn, abs=1e-15)
    assert h1[0] == pytest.approx(hn, abs=1e-15)
    _, h2 = oracle.sgd_update([w], [h], float(a), float(lam), float(s),
                              h_uses_new_w=True)
    assert h2[0] == pytest.approx(hn_new, abs=1e-15)
    # the reading that is used (old w in the h-update) differs from the other
    assert abs(h1[0] - h2[0]) > 1e-3

    _, k, lam, s, a, *rest = rows["B"]
    vals = [float(x) for x in rest[:8]]
    w, h, wn, hn = vals[0:2], vals[2:4], vals[4:6], vals[6:8]
    w1, h1 = oracle.sgd_update(w, h, float(a), float(lam), float(s))
    np.testing.assert_allclose(w1, wn, atol=1e-14)
    np.testing.assert_allclose(h1, hn, atol=1e-14)


def _objective_one(w, h, a, lam):
    return oracle.objective([0], [0], [a], np.array([w]), np.array([h]), lam)


def test_update_is_minus_gradient_finite_difference():
    """(w - w')/s equals the gradient of the one-rating objective
    1/2 (A - <w,h>)^2 + lambda/2 (|w|^2 + |h|^2) (Sec. 2.3), by central
    differences; same for h."""
    rng = np.random.default_rng(7)
    for k in (1, 3, 8):
        w = rng.normal(size=k)
        h = rng.normal(size=k)
        a, lam, s = 0.7, 0.3, 1e-3
        w1, h1 = oracle.sgd_update(w, h, a, lam, s)
        dir_w = (w - w1) / s
        dir_h = (h - h1) / s
        eps = 1e-6
        for l in range(k):
            d = np.zeros(k)
            d[l] = eps
            gw = (_objective_one(w + d, h, a, lam) -
                  _objective_one(w - d, h, a, lam)) / (2 * eps)
            gh = (_objective_one(w, h + d, a, lam) -
                  _objective_one(w, h - d, a, lam)) / (2 * eps)
            assert dir_w[l] == pytest.approx(gw, abs=1e-6)
            assert dir_h[l] == pytest.approx(gh, abs=1e-6)


def test_sum_of_rating_gradients_is_full_gradient():
    """Summing the per-rating gradients over Omega gives grad J (Sec. 2.3: the
    per-rating gradient is the term of grad J for one rating)."""
    rng = np.random.default_rng(3)
    m, n, k, lam = 5, 4, 3, 0.2
    pairs = [(i, j) for i in range(m) for j in range(n) if rng.random() < 0.6]
    rows = np.array([p[0] for p in pairs], np.int32)
    cols = np.array([p[1] for p in pairs], np.int32)
    vals = rng.normal(size=len(pairs))
    W = rng.normal(size=(m, k))
    H = rng.normal(size=(n, k))
    s = 1e-3
    gW = np.zeros_like(W)
    gH = np.zeros_like(H)
    for r in range(len(pairs)):
        i, j = rows[r], cols[r]
        w1, h1 = oracle.sgd_update(W[i], H[j], vals[r], lam, s)
        gW[i] += (W[i] - w1) / s
        gH[j] += (H[j] - h1) / s
    eps = 1e-6
    for i in range(m):
        for l in range(k):
            Wp, Wm = W.copy(), W.copy()
            Wp[i, l] += eps
            Wm[i, l] -= eps
            fd = (oracle.objective(rows, cols, vals, Wp, H, lam) -
                  oracle.objective(rows, cols, vals, Wm, H, lam)) / (2 * eps)
            assert gW[i, l] == pytest.approx(fd, abs=2e-6)
    for j in range(n):
        for l in range(k):
            Hp, Hm = H.copy(), H.copy()
            Hp[j, l] += eps
            Hm[j, l] -= eps
            fd = (oracle.objective(rows, cols, vals, W, Hp, lam) -
                  oracle.objective(rows, cols, vals, W, Hm, lam)) / (2 * eps)
            assert gH[j, l] == pytest.approx(fd, abs=2e-6)


# --------------------------------------------------------------- objective/RMSE
def test_objective_and_rmse_worked_example():
    g = {r[0]: float(r[1]) for r in golden_rows("objective_small.txt")}
    W = np.array([[1.0], [2.0]])
    H = np.array([[0.5], [-1.0]])
    rows, cols, vals = [0, 0, 1], [0, 1, 0], [1.0, 0.0, 2.0]
    assert oracle.objective(rows, cols, vals, W, H, 0.1) == pytest.approx(
        g["J"], abs=1e-15)
    assert oracle.rmse(rows, cols, vals, W, H) == pytest.approx(
        np.sqrt(g["RMSE_SQUARED"]), abs=1e-15)


def test_objective_special_cases():
    """Zero factors: J = 1/2 sum A^2 and RMSE = sqrt(mean A^2).  Exact fit with
    lambda = 0: J = 0 and RMSE = 0."""
    rng = np.random.default_rng(5)
    m, n, k = 7, 6, 2
    rows = rng.integers(0, m, 20).astype(np.int32)
    cols = rng.integers(0, n, 20).astype(np.int32)
    vals = rng.normal(size=20)
    Z = np.zeros((m, k)), np.zeros((n, k))
    assert oracle.objective(rows, cols, vals, *Z, 0.7) == pytest.approx(
        0.5 * np.sum(vals ** 2))
    assert oracle.rmse(rows, cols, vals, *Z) == pytest.approx(
        np.sqrt(np.mean(vals ** 2)))
    W = rng.normal(size=(m, k))
    H = rng.normal(size=(n, k))
    exact = np.einsum("rk,rk->r", W[rows], H[cols])
    assert oracle.objective(rows, cols, exact, W, H, 0.0) == pytest.approx(
        0.0, abs=1e-12)
    assert oracle.rmse(rows, cols, exact, W, H) == pytest.approx(0.0, abs=1e-7)
    assert np.isnan(oracle.rmse([], [], [], W, H))


# --------------------------------------------------------------- layout
def test_partition_users_mode_brute_force():
    for m, p in ((10, 3), (7, 7), (100, 8), (5, 9)):
        rw = oracle.partition_rows(m, [], p, mode="users")
        for i in range(m):
            assert rw[i] == (i * p) // m


def test_partition_ratings_mode_properties():
    """Equal-ratings split (footnote of Sec. 3.1): contiguous non-decreasing
    blocks, every worker's load within one max row degree of nnz/p, and the
    middle-rating rule checked by brute force."""
    r = synth.netflix_shaped(0.002, seed=11)
    rows = r.train_rows.numpy()
    m = r.m
    deg = np.bincount(rows, minlength=m)
    for p in (1, 2, 7, 32, 100):
        rw = oracle.partition_rows(m, rows, p)
        assert rw.min() >= 0 and rw.max() <= p - 1
        assert np.all(np.diff(rw) >= 0)
        load = np.bincount(rw, weights=deg, minlength=p)
        assert load.sum() == rows.size
        assert np.all(np.abs(load - rows.size / p) <= deg.max() + 1)
        c = 0
        for i in range(0, m, max(1, m // 200)):
            c = int(deg[:i].sum())
            want = min(p - 1, (p * (2 * c + int(deg[i]))) // (2 * rows.size))
            assert rw[i] == want
    assert np.all(oracle.partition_rows(m, rows, 1) == 0)


def test_layout_brute_force():
    """Omega-bar_j^(q) = {(i,j) in Omega : i in I_q} (Sec. 3.1), ordered by
    (q, j) with rows ascending; every rating appears exactly once."""
    rng = np.random.default_rng(9)
    m, n, p = 23, 11, 4
    pairs = sorted({(int(rng.integers(m)), int(rng.integers(n)))
                    for _ in range(120)})
    rows = np.array([a for a, _ in pairs], np.int32)
    cols = np.array([b for _, b in pairs], np.int32)
    vals = rng.normal(size=len(pairs))
    rw = oracle.partition_rows(m, rows, p)
    L = oracle.build_layout(m, n, rows, cols, vals, rw, p)
    seen = []
    S = L["seg_col"].size
    for s in range(S):
        q, j = int(L["seg_worker"][s]), int(L["seg_col"][s])
        recs = list(range(L["seg_ptr"][s], L["seg_ptr"][s + 1]))
        got_rows = [int(L["rec_row"][r]) for r in recs]
        want_rows = sorted(i for (i, jj) in pairs if jj == j and rw[i] == q)
        assert got_rows == want_rows and len(want_rows) > 0
        for r in recs:
            src = L["rec_src"][r]
            assert rows[src] == L["rec_row"][r] and cols[src] == j
            assert vals[src] == L["rec_val"][r]
        seen += [int(L["rec_src"][r]) for r in recs]
    assert sorted(seen) == list(range(len(pairs)))
    keys = [(int(L["seg_worker"][s]), int(L["seg_col"][s])) for s in range(S)]
    assert keys == sorted(set(keys))
    for j in range(n):
        segs = L["col_segs"][L["col_seg_ptr"][j]:L["col_seg_ptr"][j + 1]]
        assert [int(L["seg_col"][s]) for s in segs] == [j] * len(segs)
        ws = [int(L["seg_worker"][s]) for s in segs]
        assert ws == sorted(set(ws))
        assert set(ws) == {int(rw[i]) for (i, jj) in pairs if jj == j}
    idx = oracle.segment_index(L, L["seg_worker"], L["seg_col"])
    assert np.array_equal(idx, np.arange(S))
    assert oracle.segment_index(L, [p - 1], [n + 5])[0] == -1


# --------------------------------------------------------------- schedules
def _tiny(p=8, seed=1):
    r = synth.tiny_planted(seed)
    tr, tc, tv, er, ec, ev = r.numpy()
    rw = oracle.partition_rows(r.m, tr, p)
    L = oracle.build_layout(r.m, r.n, tr, tc, tv, rw, p)
    return r, (tr, tc, tv, er, ec, ev), L


def test_replay_first_update_uses_alpha():
    """A one-rating replay reproduces the hand-worked update with s_0 = alpha
    (reading: t counts earlier updates, so the first uses t = 0), and the
    second visit uses s_1 = alpha / (1 + beta)."""
    L = oracle.build_layout(1, 1, [0], [0], [1.0], [0], 1)
    W0, H0 = np.array([[0.5]]), np.array([[0.5]])
    W, H, cnt = oracle.replay(L, [0], W0, H0, 0.1, 0.1, 0.3)
    assert W[0, 0] == pytest.approx(0.5325, abs=1e-15)
    assert H[0, 0] == pytest.approx(0.5325, abs=1e-15)
    assert cnt[0] == 1
    W2, H2, cnt2 = oracle.replay(L, [0, 0], W0, H0, 0.1, 0.1, 0.3)
    w_ref, h_ref = oracle.sgd_update([0.5325], [0.5325], 1.0, 0.1, 0.1 / 1.3)
    assert W2[0, 0] == pytest.approx(w_ref[0], abs=1e-15)
    assert H2[0, 0] == pytest.approx(h_ref[0], abs=1e-15)
    assert cnt2[0] == 2


@pytest.mark.parametrize("mode", ["epoch", "uniform"])
def test_serial_nomad_accounting(mode):
    """Epoch mode: each item visits each worker holding it exactly once per
    epoch (permutation circulation, Sec. 3.4), so every rating is updated
    exactly once per epoch.  Uniform mode (Alg. 1): the run stops at
    n_epochs * nnz updates."""
    r, (tr, tc, tv, *_), L = _tiny()
    k, E = 10, 3
    W0 = oracle.init_factor(r.m, k, 2, 0)
    H0 = oracle.init_factor(r.n, k, 2, 1)
    W, H, cnt, log = oracle.serial_nomad(L, W0, H0, 0.05, 0.012, 0.05, E, 3,
                                         mode=mode, log_cap=10 ** 7)
    if mode == "epoch":
        assert np.all(cnt == E)
        S = L["seg_col"].size
        assert log.size == E * S
        # per item, consecutive runs of d_j visits are permutations of its segments
        for j in range(r.n):
            segs = set(L["col_segs"][L["col_seg_ptr"][j]:L["col_seg_ptr"][j + 1]])
            mine = [s for s in log if L["seg_col"][s] == j]
            d = len(segs)
            assert len(mine) == E * d
            for e in range(E):
                assert set(mine[e * d:(e + 1) * d]) == segs
    else:
        assert cnt.sum() >= E * tr.size
        assert cnt.sum() < E * tr.size + 1000
    # the visit log replays to the very same factors
    valid = log[log >= 0]
    W2, H2, cnt2 = oracle.replay(L, valid, W0, H0, 0.05, 0.012, 0.05)
    assert np.array_equal(W, W2) and np.array_equal(H, H2)
    assert np.array_equal(cnt, cnt2)


def test_shorter_queue_routing_balances_the_queues():
    """Sec. 3.3: sending each token to the shorter of two uniformly drawn
    queues keeps the longest queue shorter than uniform routing (Alg. 1)
    does on the same draws, and the run still applies n_epochs * nnz
    updates whose logged order replays to the same factors."""
    r, (tr, tc, tv, *_), L = _tiny()
    k, E = 10, 3
    W0 = oracle.init_factor(r.m, k, 2, 0)
    H0 = oracle.init_factor(r.n, k, 2, 1)
    out = {}
    for mode in ("uniform", "uniform-shorter"):
        st = np.zeros(2, dtype=np.int64)
        W, H, cnt, log = oracle.serial_nomad(L, W0, H0, 0.05, 0.012, 0.05, E, 3, mode=mode,
                                             log_cap=10 ** 7, queue_stats=st)
        assert E * tr.size <= cnt.sum() < E * tr.size + 1000
        valid = log[log >= 0]
        W2, H2, cnt2 = oracle.replay(L, valid, W0, H0, 0.05, 0.012, 0.05)
        assert np.array_equal(W, W2) and np.array_equal(H, H2)
        out[mode] = (st.copy(), log.size)
    (su, nu), (ss, ns) = out["uniform"], out["uniform-shorter"]
    # the longest queue met by a push (the mean is n/p either way: every
    # token is always in some queue)
    assert ss[0] < 0.75 * su[0], (ss, su)


def test_serializability_commuting_visits():
    """Visits that share neither worker nor item touch disjoint variables, so
    swapping two adjacent such visits leaves the replay result bit-identical
    (the serializability property of Sec. 3.1 / Sec. 1)."""
    r, _, L = _tiny()
    k = 10
    W0 = oracle.init_factor(r.m, k, 2, 0)
    H0 = oracle.init_factor(r.n, k, 2, 1)
    _, _, _, log = oracle.serial_nomad(L, W0, H0, 0.05, 0.012, 0.05, 2, 5,
                                       log_cap=10 ** 7)
    sw, sc = L["seg_worker"], L["seg_col"]
    rng = np.random.default_rng(0)
    log2 = log.copy()
    swaps = 0
    for v in rng.permutation(log.size - 1)[:2000]:
        a, b = log2[v], log2[v + 1]
        if sw[a] != sw[b] and sc[a] != sc[b]:
            log2[v], log2[v + 1] = b, a
            swaps += 1
    assert swaps > 100
    A = oracle.replay(L, log, W0, H0, 0.05, 0.012, 0.05)
    B = oracle.replay(L, log2, W0, H0, 0.05, 0.012, 0.05)
    assert np.array_equal(A[0], B[0]) and np.array_equal(A[1], B[1])
    # ...while swapping two visits of the same item changes the result
    for v in range(log.size - 1):
        if sc[log[v]] == sc[log[v + 1]]:
            break
    else:
        v = None
    if v is not None:
        log3 = log.copy()
        log3[v], log3[v + 1] = log[v + 1], log[v]
        C = oracle.replay(L, log3, W0, H0, 0.05, 0.012, 0.05)
        assert not np.array_equal(A[1], C[1])


def test_monotone_descent_small_steps():
    """With a tiny constant step (alpha = 1e-4, beta = 0) an epoch is close to
    one full gradient step, so J decreases every epoch."""
    r, (tr, tc, tv, *_), L = _tiny()
    k, lam = 10, 0.05
    W = oracle.init_factor(r.m, k, 2, 0)
    H = oracle.init_factor(r.n, k, 2, 1)
    J = [oracle.objective(tr, tc, tv, W, H, lam)]
    for e in range(5):
        W, H, _, _ = oracle.serial_nomad(L, W, H, lam, 1e-4, 0.0, 1, 17 + e)
        J.append(oracle.objective(tr, tc, tv, W, H, lam))
    assert all(b < a for a, b in zip(J, J[1:])), J
    W = oracle.init_factor(r.m, k, 2, 0)
    H = oracle.init_factor(r.n, k, 2, 1)
    J2 = [oracle.objective(tr, tc, tv, W, H, lam)]
    for e in range(5):
        W, H, _ = oracle.shuffled_sgd(tr, tc, tv, W, H, lam, 1e-4, 0.0, 1, e)
        J2.append(oracle.objective(tr, tc, tv, W, H, lam))
    assert all(b < a for a, b in zip(J2, J2[1:])), J2


def test_planted_recovery_noise_free():
    """Noise-free rank-3 planted matrix, k = 3, tiny lambda: SGD drives the
    training RMSE near zero and the test RMSE far below the signal's unit
    standard deviation."""
    r = synth.planted(300, 200, 3, 18000, 0.0, 0.1, seed=21)
    tr, tc, tv, er, ec, ev = r.numpy()
    k = 3
    W = oracle.init_factor(r.m, k, 4, 0)
    H = oracle.init_factor(r.n, k, 4, 1)
    W, H, _ = oracle.shuffled_sgd(tr, tc, tv, W, H, 1e-4, 0.05, 0.0, 150, 8)
    assert oracle.rmse(tr, tc, tv, W, H) < 0.02
    assert oracle.rmse(er, ec, ev, W, H) < 0.05


def test_planted_recovery_with_noise():
    """Planted rank 5 with N(0, 0.1^2) noise, 30% observed, k = 5 (the
    generation recipe of Sec. 5.5 at a size where recovery is possible): the
    test RMSE approaches the noise level (recovery is not exact; tolerance
    0.15), through the serial NOMAD schedule and through plain SGD."""
    r = synth.planted(400, 300, 5, 36000, 0.1, 0.1, seed=22)
    tr, tc, tv, er, ec, ev = r.numpy()
    k, lam = 5, 0.01
    W0 = oracle.init_factor(r.m, k, 4, 0)
    H0 = oracle.init_factor(r.n, k, 4, 1)
    W, H, _ = oracle.shuffled_sgd(tr, tc, tv, W0, H0, lam, 0.02, 0.0, 100, 8)
    assert oracle.rmse(tr, tc, tv, W, H) < 0.12
    assert oracle.rmse(er, ec, ev, W, H) < 0.15
    rw = oracle.partition_rows(r.m, tr, 16)
    L = oracle.build_layout(r.m, r.n, tr, tc, tv, rw, 16)
    W, H, _, _ = oracle.serial_nomad(L, W0, H0, lam, 0.02, 0.0, 100, 3)
    assert oracle.rmse(tr, tc, tv, W, H) < 0.12
    assert oracle.rmse(er, ec, ev, W, H) < 0.15


def test_replay_f32_matches_f64_within_rounding():
    """The binary32 replay is the same algorithm: on the tiny config it stays
    within binary32 rounding of the binary64 replay."""
    r, _, L = _tiny()
    k = 10
    W0 = oracle.init_factor(r.m, k, 2, 0)
    H0 = oracle.init_factor(r.n, k, 2, 1)
    _, _, _, log = oracle.serial_nomad(L, W0, H0, 0.05, 0.012, 0.05, 3, 5,
                                       log_cap=10 ** 7)
    A = oracle.replay(L, log, W0, H0, 0.05, 0.012, 0.05, precision="f64")
    B = oracle.replay(L, log, W0, H0, 0.05, 0.012, 0.05, precision="f32")
    for x, y in ((A[0], B[0]), (A[1], B[1])):
        rel = np.linalg.norm(x - y) / np.linalg.norm(x)
        assert rel < 1e-5
    assert np.array_equal(A[2], B[2])
