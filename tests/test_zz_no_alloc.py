"""nomad_rmse_noalloc: the test RMSE for callers that cannot let the library
allocate (a service that pre-reserves all device memory, a loop that must
not hit cudaMalloc's implicit synchronisation).  It must give what
nomad_rmse gives, on two calls in a row (the second reuses the scratch
array the first one left behind).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

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
        for call in range(2):
            nm.epoch(2)
            want = nm.rmse(*te)
            nm.factors_into(W, H)
            assert _noalloc(W, H, k, *te, out, stream) == nb.NOMAD_OK
            torch.cuda.synchronize(dev)
            got = float(out.item())
            assert abs(got - want) <= REDUCE_TOL * want, (call, got, want)


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
