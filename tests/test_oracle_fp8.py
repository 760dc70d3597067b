"""The oracle's FP8-E4M3 storage of W (codes plus a binary32 scale per row),
pinned by what the format and the mathematics fix rather than by its own
formulas: printed values of the format (OCP 8-bit floating point, E4M3:
largest finite 448, smallest normal 2^-6, smallest subnormal 2^-9, NaN
S.1111.111), brute-force nearest over all 256 codes, the round-up
probability of stochastic rounding counted over all 2^16 random inputs, the
per-row scale's extremes, and the replay against the binary32 replay.
"""
import numpy as np
import pytest

import oracle
import synth

ALL = np.arange(256, dtype=np.uint8)


def finite_table():
    v = oracle.e4m3_to_f32(ALL)
    ok = ~np.isnan(v)
    return ALL[ok], v[ok].astype(np.float64)


def test_printed_values_of_the_format():
    want = {0x00: 0.0, 0x01: 2.0 ** -9, 0x07: 7 * 2.0 ** -9, 0x08: 2.0 ** -6,
            0x38: 1.0, 0x3F: 1.875, 0x40: 2.0, 0x77: 240.0, 0x7E: 448.0,
            0x80: -0.0, 0xFE: -448.0, 0xB8: -1.0}
    got = oracle.e4m3_to_f32(np.array(list(want), np.uint8))
    assert np.array_equal(got, np.array(list(want.values()), np.float32))
    assert np.isnan(oracle.e4m3_to_f32(np.array([0x7F, 0xFF], np.uint8))).all()
    # positive codes increase strictly up to 448; negative codes mirror them
    pos = oracle.e4m3_to_f32(np.arange(0x7F, dtype=np.uint8))
    assert np.all(np.diff(pos) > 0)
    neg = oracle.e4m3_to_f32(np.arange(0x80, 0xFF, dtype=np.uint8))
    assert np.array_equal(neg[1:], -pos[1:])
    # every code round-trips through rounding to nearest
    codes, vals = finite_table()
    back = oracle.e4m3_rn(vals.astype(np.float32))
    same = (back == codes) | ((vals == 0) & (back & 0x7F == 0))
    assert same.all()


def brute_nearest(x):
    """Nearest finite E4M3 value (ties to the even code), saturating."""
    codes, vals = finite_table()
    keep = ((codes & 0x7F) != 0) | (codes == 0)  # one zero
    codes, vals = codes[keep], vals[keep]
    out = np.empty(x.size, np.uint8)
    for n, xv in enumerate(x.astype(np.float64)):
        if abs(xv) >= 448:
            out[n] = 0x7E | (0x80 if xv < 0 else 0)
            continue
        d = np.abs(vals - xv)
        best = np.flatnonzero(d == d.min())
        if best.size > 1:
            even = [b for b in best if codes[b] % 2 == 0]
            best = even
        c = codes[best[0]]
        if vals[best[0]] == 0:
            c = 0x80 if np.signbit(xv) else 0
        out[n] = c
    return out


def test_round_to_nearest_matches_brute_force():
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.uniform(-500, 500, 3000), rng.uniform(-1, 1, 3000),
        rng.uniform(-2 ** -5, 2 ** -5, 3000),           # subnormal range
        (np.arange(-40, 41) * 2.0 ** -10),              # ties of the subnormal grid
        np.array([448.0, 464.0, 479.0, 480.0, 1e30, -1e30, 0.0])]).astype(np.float32)
    got = oracle.e4m3_rn(x)
    want = brute_nearest(x)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], want[bad[:5]])


def neighbours(xv):
    _, vals = finite_table()
    vals = np.unique(vals)
    lo = vals[vals <= xv].max()
    hi = vals[vals >= xv].min()
    return lo, hi


@pytest.mark.parametrize("x", [0.3, 1.0 + 2 ** -8, 200.7, 0.0171, 3.3e-3, 1.1e-3,
                               2 ** -9 * 0.25, 447.0])
def test_stochastic_rounding_probability(x):
    """Over all 2^16 random inputs the result is always one of the two
    neighbours of x, and the mean is x within the 16-bit resolution."""
    xs = np.full(65536, x, np.float32)
    r = np.arange(65536, dtype=np.uint32)
    v = oracle.e4m3_to_f32(oracle.e4m3_sr(xs, r)).astype(np.float64)
    lo, hi = neighbours(float(np.float32(x)))
    assert set(np.unique(v)) <= {lo, hi}
    assert abs(v.mean() - float(np.float32(x))) <= (hi - lo) * 2.0 ** -15 + 1e-12
    # exact values are kept by every draw
    for c in (0x01, 0x08, 0x38, 0x7E):
        val = oracle.e4m3_to_f32(np.array([c], np.uint8))[0]
        assert np.all(oracle.e4m3_sr(np.full(65536, val, np.float32), r) == c)


def test_row_scaling():
    rng = np.random.default_rng(5)
    W = rng.normal(size=(40, 37)).astype(np.float32)
    W[3] = 0.0
    W[4, :] = 1e-30
    codes, scales = oracle.e4m3_rows(W)
    deq = oracle.e4m3_decode_rows(codes, scales)
    # the largest entry of a row maps to +-448 exactly
    for i in range(W.shape[0]):
        if np.abs(W[i]).max() >= 2 ** -100:
            j = np.argmax(np.abs(W[i]))
            assert codes[i, j] & 0x7F == 0x7E
    assert scales[3] == 1.0 and np.all(deq[3] == 0)
    # entries in the normal range of the scaled grid are within half an ulp
    # (2^-4 relative), the rest within half of the subnormal step
    with np.errstate(divide="ignore", invalid="ignore"):
        q = W * (448.0 / np.abs(W).max(1, keepdims=True)).astype(np.float32)
        rel = np.abs(deq - W) / np.abs(W)
    normal = np.abs(q) >= 2 ** -6
    assert np.all(rel[normal & (np.abs(W) > 1e-20)] <= 2 ** -4 * (1 + 1e-6))
    step = (scales[:, None] * 2.0 ** -9) * np.ones_like(W)
    assert np.all(np.abs(deq - W)[~normal] <= 0.5 * step[~normal] * (1 + 1e-6))


def test_replay_tracks_the_binary32_replay():
    """Two epochs on the tiny problem.  With a zero step the replay leaves H
    unchanged and W within one E4M3 step.  With the paper's steps, against
    the binary32 replay of the same order: every write of a row adds an
    unbiased rounding error of at most half an E4M3 ulp rms (2^-4 relative),
    so after the ~45 writes per row of two epochs the rows differ by at most
    2^-4 * sqrt(45) ~ 0.42 relative L2 (the contraction of SGD only shrinks
    this); the mean difference stays near zero (the rounding is unbiased)
    and the test RMSE within 1%."""
    r = synth.tiny_planted(1)
    tr, tc, tv, er, ec, ev = r.numpy()
    p = 8
    rw = oracle.partition_rows(r.m, tr, p)
    L = oracle.build_layout(r.m, r.n, tr, tc, tv, rw, p)
    S = L["seg_col"].size
    order = np.concatenate([np.random.default_rng(e).permutation(S) for e in range(2)])
    ep = np.repeat(np.arange(2, dtype=np.int32), S)
    W0 = oracle.init_factor(r.m, 10, 1, 0).astype(np.float32)
    H0 = oracle.init_factor(r.n, 10, 1, 1).astype(np.float32)
    Wc, Ws = oracle.e4m3_rows(W0)
    Wq = oracle.e4m3_decode_rows(Wc, Ws)
    lam = float(np.float32(0.05))
    # zero step
    c1, s1, H1, _ = oracle.replay_e4m3(L, order, ep, Wc, Ws, H0, lam, 0.0, 0.0, 7)
    assert np.array_equal(H1, H0)
    W1 = oracle.e4m3_decode_rows(c1, s1)
    assert np.all(np.abs(W1 - Wq) <= 2 ** -3 * np.abs(Wq) + s1[:, None] * 2.0 ** -9)
    # the paper's schedule
    a, b = float(np.float32(0.05)), float(np.float32(0.05))
    c2, s2, H2, cnt = oracle.replay_e4m3(L, order, ep, Wc, Ws, H0, lam, a, b, 7)
    W2 = oracle.e4m3_decode_rows(c2, s2)
    W32, H32, cnt32 = oracle.replay(L, order, Wq.copy(), H0.copy(), lam, a, b, precision="f32")
    assert np.array_equal(cnt, cnt32) and np.all(cnt == 2)
    writes = tr.size / r.m * 2
    rel = np.linalg.norm(W2 - W32) / np.linalg.norm(W32)
    assert rel < 2.0 ** -4 * np.sqrt(writes), rel
    bias = abs(float((W2 - W32).mean())) / float(np.abs(W32).mean())
    assert bias < 0.01, bias
    r8 = oracle.rmse(er, ec, ev, W2.astype(np.float64), H2.astype(np.float64))
    r32 = oracle.rmse(er, ec, ev, W32.astype(np.float64), H32.astype(np.float64))
    assert abs(r8 - r32) <= 0.01 * r32, (r8, r32)
