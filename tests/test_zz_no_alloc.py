"""nomad_rmse_noalloc: the test RMSE for callers that cannot let the library
allocate (a service that pre-reserves all device memory, a loop that must
not hit cudaMalloc's implicit synchronisation).  It must give what
nomad_rmse gives, and what the binary64 oracle gives on the same factors, on
two calls in a row (the second reuses the scratch array the first one left
behind), for factors with a row pitch wider than k, on a side stream, and
NaN for an empty test set.

The file name sorts last so that pytest collects it after every other test
file: a run that stops at the first failure (-x) has then already run the
rest of the suite before this entry point is exercised.  The tests do not
depend on the order otherwise; each passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1312_0193_gb300 import Nomad  # noqa: E402
from paper_1312_0193_gb300 import nomad as nb  # noqa: E402

REDUCE_TOL = 1e-6  # relative; same bound as the other RMSE tests


def _noalloc(W, H, k, rows, cols, vals, out, stream):
    lib = nb.load_library()
    P = ctypes.c_void_p
    return lib.nomad_rmse_noalloc(P(W.data_ptr()), P(H.data_ptr()), W.shape[0], H.shape[0],
                                  k, W.stride(0), rows.numel(), P(rows.data_ptr()),
                                  P(cols.data_ptr()), P(vals.data_ptr()), P(out.data_ptr()),
                                  P(stream.cuda_stream))


def test_noalloc_rmse_matches_nomad_rmse_twice():
    r = synth.tiny_planted(1)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    k = 10
    with Nomad(r.m, r.n, k, 0.05, alpha=0.1, beta=0.01) as nm:
        nm.load_coo(r.train_rows.to(dev), r.train_cols.to(dev), r.train_vals.to(dev))
        te = [t.to(dev) for t in (r.test_rows, r.test_cols, r.test_vals)]
        W = torch.empty(r.m, k, dtype=torch.float32, device=dev)
        H = torch.empty(r.n, k, dtype=torch.float32, device=dev)
        out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        er, ec, ev = (t.cpu().numpy() for t in (r.test_rows, r.test_cols, r.test_vals))
        for call in range(2):
            nm.epoch(2)
            want = nm.rmse(*te)
            nm.factors_into(W, H)
            assert _noalloc(W, H, k, *te, out, stream) == nb.NOMAD_OK
            torch.cuda.synchronize(dev)
            got = float(out.item())
            assert abs(got - want) <= REDUCE_TOL * want, (call, got, want)
            orc = oracle.rmse(er, ec, ev, W.cpu().double().numpy(), H.cpu().double().numpy())
            assert abs(got - orc) <= REDUCE_TOL * orc, (call, got, orc)


def test_noalloc_rmse_padded_rows_side_stream_and_empty():
    """W and H as column slices of wider arrays (row pitch 16 > k = 10, the
    same pitch for both), launched on a side stream; an empty test set gives
    NaN."""
    r = synth.tiny_planted(1)
    dev = torch.device("cuda", 0)
    k = 10
    with Nomad(r.m, r.n, k, 0.05, alpha=0.1, beta=0.01) as nm:
        nm.load_coo(r.train_rows.to(dev), r.train_cols.to(dev), r.train_vals.to(dev))
        nm.epoch(3)
        Wd = torch.empty(r.m, k, dtype=torch.float32, device=dev)
        Hd = torch.empty(r.n, k, dtype=torch.float32, device=dev)
        nm.factors_into(Wd, Hd)
    Wwide = torch.full((r.m, 16), float("nan"), dtype=torch.float32, device=dev)
    Hwide = torch.full((r.n, 16), float("nan"), dtype=torch.float32, device=dev)
    Wwide[:, 3:3 + k] = Wd
    Hwide[:, 3:3 + k] = Hd
    W, H = Wwide[:, 3:3 + k], Hwide[:, 3:3 + k]
    assert W.stride(0) == H.stride(0) == 16
    te = [t.to(dev) for t in (r.test_rows, r.test_cols, r.test_vals)]
    er, ec, ev = (t.cpu().numpy() for t in (r.test_rows, r.test_cols, r.test_vals))
    want = oracle.rmse(er, ec, ev, Wd.cpu().double().numpy(), Hd.cpu().double().numpy())
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    with torch.cuda.stream(side):
        for c in range(2):
            assert _noalloc(W, H, k, *te, out[c:c + 1], side) == nb.NOMAD_OK
    side.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.abs(got - want) <= REDUCE_TOL * want), (got, want)
    assert got[0] == got[1]  # the same inputs give the same bits
    empty_i = torch.zeros(0, dtype=torch.int32, device=dev)
    empty_v = torch.zeros(0, dtype=torch.float32, device=dev)
    one = torch.zeros(1, dtype=torch.float64, device=dev)
    assert _noalloc(W, H, k, empty_i, empty_i, empty_v, one, side) == nb.NOMAD_OK
    side.synchronize()
    assert np.isnan(float(one.item()))


def test_noalloc_rmse_larger_rank_and_limits():
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    r = synth.netflix_shaped(0.002, seed=4)
    k = 100
    with Nomad(r.m, r.n, k, 0.05) as nm:
        nm.load_coo(r.train_rows.to(dev), r.train_cols.to(dev), r.train_vals.to(dev))
        nm.epoch(1)
        te = [t.to(dev) for t in (r.test_rows, r.test_cols, r.test_vals)]
        want = nm.rmse(*te)
        W = torch.empty(r.m, k, dtype=torch.float32, device=dev)
        H = torch.empty(r.n, k, dtype=torch.float32, device=dev)
        nm.factors_into(W, H)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(2):
        assert _noalloc(W, H, k, *te, out, stream) == nb.NOMAD_OK
        torch.cuda.synchronize(dev)
        assert abs(float(out.item()) - want) <= REDUCE_TOL * want
    # an index outside [0, m) gives NaN, and the next good call is clean again
    bad_rows = te[0].clone()
    bad_rows[3] = r.m
    assert _noalloc(W, H, k, bad_rows, te[1], te[2], out, stream) == nb.NOMAD_OK
    torch.cuda.synchronize(dev)
    assert np.isnan(float(out.item()))
    assert _noalloc(W, H, k, *te, out, stream) == nb.NOMAD_OK
    torch.cuda.synchronize(dev)
    assert abs(float(out.item()) - want) <= REDUCE_TOL * want
    # more ratings than the fixed scratch can reduce are refused up front
    lib = nb.load_library()
    P = ctypes.c_void_p
    too_many = 65536 * 8192 + 1
    assert lib.nomad_rmse_noalloc(P(W.data_ptr()), P(H.data_ptr()), r.m, r.n, k, k,
                                  too_many, P(te[0].data_ptr()), P(te[1].data_ptr()),
                                  P(te[2].data_ptr()), P(out.data_ptr()),
                                  P(stream.cuda_stream)) == nb.NOMAD_ERR_INVALID_ARG
