"""Pins of the oracle's bfloat16 storage arithmetic (the precision variant:
W and H stored in bfloat16, updates in binary32, stochastic rounding on
write-back).  CPU only."""
import numpy as np
import pytest

import oracle
import synth
from conftest import golden_rows


def test_round_to_nearest_even_worked_examples():
    rows = golden_rows("bf16_rounding.txt")
    bits = np.array([int(r[0], 16) for r in rows], dtype=np.uint32)
    want = np.array([int(r[1], 16) for r in rows], dtype=np.uint16)
    assert np.array_equal(oracle.bf16_rn(bits.view(np.float32)), want)


def test_round_to_nearest_matches_torch():
    """torch's float32 -> bfloat16 conversion rounds to nearest even."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=20000), rng.normal(size=2000) * 1e-30,
                        rng.normal(size=2000) * 1e30]).astype(np.float32)
    t = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.bf16_rn(x), t)


def test_stochastic_rounding_properties():
    rng = np.random.default_rng(2)
    x = rng.normal(size=64).astype(np.float32)
    # exactly representable values never move
    exact = oracle.bf16_to_f32(oracle.bf16_rn(x))
    for r in (0, 1, 0x7FFF, 0xFFFF):
        assert np.array_equal(oracle.bf16_to_f32(oracle.bf16_sr(exact, np.full(64, r))), exact)
    # r = 0 truncates the magnitude; results are the two neighbours only
    lo = oracle.bf16_to_f32(oracle.bf16_sr(x, np.zeros(64, np.uint32)))
    assert np.all(np.abs(lo) <= np.abs(x))
    hi = oracle.bf16_to_f32(oracle.bf16_sr(x, np.full(64, 0xFFFF, np.uint32)))
    assert np.all(np.abs(hi) >= np.abs(x))
    # unbiased: the mean over all 2^16 draws is the binary32 value exactly
    r = np.arange(1 << 16, dtype=np.uint32)
    for v in x[:8]:
        vals = oracle.bf16_to_f32(oracle.bf16_sr(np.full(r.size, v, np.float32), r))
        assert set(np.unique(vals)) <= {lo[list(x).index(v)], hi[list(x).index(v)]}
        assert vals.astype(np.float64).mean() == pytest.approx(float(v), rel=0, abs=0)


def _tiny_bf16():
    r = synth.tiny_planted(1)
    tr, tc, tv, *_ = r.numpy()
    rw = oracle.partition_rows(r.m, tr, 8)
    L = oracle.build_layout(r.m, r.n, tr, tc, tv, rw, 8)
    W0 = oracle.init_factor(r.m, 10, 2, 0).astype(np.float32)
    H0 = oracle.init_factor(r.n, 10, 2, 1).astype(np.float32)
    return r, L, oracle.bf16_rn(W0), oracle.bf16_rn(H0)


def test_bf16_replay_zero_step_is_identity():
    r, L, Wb, Hb = _tiny_bf16()
    _, _, _, log = oracle.serial_nomad(L, np.zeros((r.m, 10)), np.zeros((r.n, 10)),
                                       0.05, 0.0, 0.0, 1, 3, log_cap=10 ** 7)
    W1, H1, cnt = oracle.replay_bf16(L, log, np.zeros(log.size, np.int32), Wb, Hb,
                                     0.05, 0.0, 0.0, seed=9)
    assert np.array_equal(W1, Wb) and np.array_equal(H1, Hb)
    assert np.all(cnt == 1)


def test_bf16_replay_tracks_f32_replay_and_is_unbiased():
    """From the same bfloat16-representable start, a bfloat16 replay stays
    within stochastic-rounding noise of the binary32 replay, and averaging
    replays with different rounding draws moves closer to it."""
    r, L, Wb, Hb = _tiny_bf16()
    W0, H0 = oracle.bf16_to_f32(Wb), oracle.bf16_to_f32(Hb)
    _, _, _, log = oracle.serial_nomad(L, W0, H0, 0.05, 0.05, 0.0, 2, 3, log_cap=10 ** 7)
    S = L["seg_col"].size
    ep = np.repeat(np.arange(2, dtype=np.int32), S)
    Wf, Hf, _ = oracle.replay(L, log, W0, H0, 0.05, 0.05, 0.0, precision="f32")
    mean_W = np.zeros_like(Wf, dtype=np.float64)
    errs = []
    for seed in range(8):
        Wb1, Hb1, _ = oracle.replay_bf16(L, log, ep, Wb, Hb, 0.05, 0.05, 0.0, seed=seed)
        Wx = oracle.bf16_to_f32(Wb1)
        errs.append(np.linalg.norm(Wx - Wf) / np.linalg.norm(Wf))
        mean_W += Wx / 8
    assert max(errs) < 2e-2
    assert np.linalg.norm(mean_W - Wf) / np.linalg.norm(Wf) < 0.6 * np.mean(errs)
