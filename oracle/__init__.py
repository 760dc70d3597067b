"""Serial CPU oracle for NOMAD matrix completion (arXiv 1312.0193).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_1312_0193_gb300``)
and never imports it.

The arithmetic lives in ``nomad_oracle.c`` (plain C, binary64 unless stated,
built with gcc by ``oracle/build.py``).  This module adds the data layout of
Sec. 3.1 (row blocks I_q and the sets Omega-bar_j^(q)), written with numpy
library sorts, and thin ctypes wrappers.

Parity status of each function (see the pins in ``tests/test_oracle_*.py``):
every function below is pinned; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i32, i64, u32, u64, f64, f32 = (ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_uint32, ctypes.c_uint64,
                                        ctypes.c_double, ctypes.c_float)
        P = ctypes.c_void_p
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_philox4x32_10.restype = None
        lib.orc_init_factor.argtypes = [i64, i32, u64, u32, P]
        lib.orc_init_factor.restype = None
        lib.orc_step_size.argtypes = [f64, f64, i64]
        lib.orc_step_size.restype = f64
        lib.orc_sgd_update.argtypes = [i32, P, P, f64, f64, f64, i32]
        lib.orc_sgd_update.restype = None
        lib.orc_objective.argtypes = [i64, P, P, P, i32, f64, P, P]
        lib.orc_objective.restype = f64
        lib.orc_sq_error_sum.argtypes = [i64, P, P, P, i32, P, P]
        lib.orc_sq_error_sum.restype = f64
        lib.orc_replay_f64.argtypes = [i32, f64, f64, f64, i64, P, i64, P, P,
                                       P, P, P, P, P, i32]
        lib.orc_replay_f64.restype = i32
        lib.orc_replay_f32.argtypes = [i32, f32, f64, f64, i64, P, i64, P, P,
                                       P, P, P, P, P]
        lib.orc_replay_f32.restype = i32
        lib.orc_serial_nomad.argtypes = [i32, f64, f64, f64, i32, i64, i64, P,
                                         P, P, P, P, P, P, i32, u64, i32, P, P,
                                         P, P, i64, P]
        lib.orc_serial_nomad.restype = i64
        lib.orc_shuffled_sgd.argtypes = [i32, f64, f64, f64, i64, P, P, P, i32,
                                         u64, P, P, P]
        lib.orc_shuffled_sgd.restype = i32
        lib.orc_bf16_rn_n.argtypes = [i64, P, P]
        lib.orc_bf16_rn_n.restype = None
        lib.orc_bf16_sr_n.argtypes = [i64, P, P, P]
        lib.orc_bf16_sr_n.restype = None
        lib.orc_bf16_to_f32_n.argtypes = [i64, P, P]
        lib.orc_bf16_to_f32_n.restype = None
        lib.orc_replay_bf16.argtypes = [i32, f32, f64, f64, i64, P, P, i64, P, P,
                                        P, P, P, P, P, u64]
        lib.orc_replay_bf16.restype = i32
        lib.orc_e4m3_rn_n.argtypes = [i64, P, P]
        lib.orc_e4m3_rn_n.restype = None
        lib.orc_e4m3_sr_n.argtypes = [i64, P, P, P]
        lib.orc_e4m3_sr_n.restype = None
        lib.orc_e4m3_to_f32_n.argtypes = [i64, P, P]
        lib.orc_e4m3_to_f32_n.restype = None
        lib.orc_e4m3_rows.argtypes = [i64, i32, P, P, P, P]
        lib.orc_e4m3_rows.restype = None
        lib.orc_replay_e4m3.argtypes = [i32, f32, f64, f64, i64, P, P, i64, P, P,
                                        P, P, P, P, P, P, u64]
        lib.orc_replay_e4m3.restype = i32
        _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- randomness
def philox4x32_10(counter, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11): 4 x u32 out."""
    c = _c(counter, np.uint32)
    k = _c(key, np.uint32)
    assert c.shape == (4,) and k.shape == (2,)
    out = np.zeros(4, dtype=np.uint32)
    _lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def init_factor(rows: int, k: int, seed: int, which: int) -> np.ndarray:
    """W (which=0) or H (which=1): UniformReal(0, 1/sqrt(k)) entries (Alg. 1
    initialisation, Sec. 5.1), binary32 values widened to float64."""
    F = np.zeros((rows, k), dtype=np.float64)
    _lib().orc_init_factor(rows, k, seed, which, _ptr(F))
    return F


# ---------------------------------------------------------------- the method
def step_size(alpha: float, beta: float, t: int) -> float:
    """s_t = alpha / (1 + beta t^1.5), Sec. 5.1 Eq. stepsize_method."""
    return _lib().orc_step_size(alpha, beta, t)


def sgd_update(w, h, a: float, lam: float, s: float, h_uses_new_w=False):
    """One SGD update (Sec. 2.3, Eq. w_update/h_update, sign reading R1).
    Returns new copies (w', h')."""
    w = _c(w, np.float64).copy()
    h = _c(h, np.float64).copy()
    assert w.shape == h.shape and w.ndim == 1
    _lib().orc_sgd_update(w.size, _ptr(w), _ptr(h), a, lam, s,
                          1 if h_uses_new_w else 0)
    return w, h


def objective(rows, cols, vals, W, H, lam: float) -> float:
    """J(W,H) of Eq. obj_fcn in its per-rating form (Sec. 2), binary64."""
    rows, cols = _c(rows, np.int32), _c(cols, np.int32)
    vals, W, H = _c(vals, np.float64), _c(W, np.float64), _c(H, np.float64)
    return _lib().orc_objective(rows.size, _ptr(rows), _ptr(cols), _ptr(vals),
                                W.shape[1], lam, _ptr(W), _ptr(H))


def sq_error_sum(rows, cols, vals, W, H) -> float:
    rows, cols = _c(rows, np.int32), _c(cols, np.int32)
    vals, W, H = _c(vals, np.float64), _c(W, np.float64), _c(H, np.float64)
    return _lib().orc_sq_error_sum(rows.size, _ptr(rows), _ptr(cols),
                                   _ptr(vals), W.shape[1], _ptr(W), _ptr(H))


def rmse(rows, cols, vals, W, H) -> float:
    """Test RMSE of Sec. 5.1, binary64 (nan for an empty set)."""
    n = int(np.asarray(rows).size)
    if n == 0:
        return float("nan")
    return float(np.sqrt(sq_error_sum(rows, cols, vals, W, H) / n))


# ---------------------------------------------------------------- layout
def partition_rows(m: int, rows, p: int, mode: str = "ratings") -> np.ndarray:
    """Split users 0..m-1 into p contiguous blocks I_0..I_{p-1} (Sec. 3.1).

    mode "users": equal numbers of users, worker(i) = floor(i p / m).
    mode "ratings" (the footnote's alternative): with d_i the degree of row i
    and c_i = sum_{i' < i} d_i', worker(i) = min(p-1, floor(p (2 c_i + d_i) /
    (2 nnz))), i.e. a row goes to the block its middle rating falls in.
    Returns row_worker (int32, length m).
    """
    rows = np.asarray(rows, dtype=np.int64)
    if mode == "users":
        return (np.arange(m, dtype=np.int64) * p // max(m, 1)).astype(np.int32)
    assert mode == "ratings"
    nnz = rows.size
    if nnz == 0:
        return np.zeros(m, dtype=np.int32)
    deg = np.bincount(rows, minlength=m).astype(np.int64)
    c = np.concatenate([[0], np.cumsum(deg)[:-1]])
    q = (p * (2 * c + deg)) // (2 * nnz)
    return np.minimum(q, p - 1).astype(np.int32)


def build_layout(m: int, n: int, rows, cols, vals, row_worker, p: int) -> dict:
    """The per-worker item sets Omega-bar_j^(q) of Sec. 3.1.

    A segment is one non-empty Omega-bar_j^(q).  Segments are ordered by
    (worker q, item j); inside a segment the ratings are ordered by row i.
    Returns a dict of numpy arrays:
      seg_worker, seg_col (int32, S); seg_ptr (int64, S+1);
      rec_row (int32), rec_val (float64), rec_src (int64: index into the
      input arrays) in segment order;
      col_seg_ptr (int64, n+1), col_segs (int64, S): the segments of item j,
      ordered by worker.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    row_worker = np.asarray(row_worker, dtype=np.int64)
    wk = row_worker[rows] if rows.size else np.zeros(0, np.int64)
    order = np.lexsort((rows, cols, wk))  # primary wk, then col, then row
    wk_s, col_s = wk[order], cols[order]
    if order.size:
        new = np.ones(order.size, dtype=bool)
        new[1:] = (wk_s[1:] != wk_s[:-1]) | (col_s[1:] != col_s[:-1])
        starts = np.flatnonzero(new)
    else:
        starts = np.zeros(0, dtype=np.int64)
    seg_ptr = np.concatenate([starts, [order.size]]).astype(np.int64)
    seg_worker = wk_s[starts].astype(np.int32)
    seg_col = col_s[starts].astype(np.int32)
    # the segments of each item, ordered by worker
    by_col = np.lexsort((seg_worker, seg_col))
    col_counts = np.bincount(seg_col, minlength=n) if seg_col.size else \
        np.zeros(n, dtype=np.int64)
    col_seg_ptr = np.concatenate([[0], np.cumsum(col_counts)]).astype(np.int64)
    return dict(
        p=p, m=m, n=n,
        seg_worker=seg_worker, seg_col=seg_col, seg_ptr=seg_ptr,
        rec_row=rows[order].astype(np.int32), rec_val=vals[order],
        rec_src=order.astype(np.int64),
        col_seg_ptr=col_seg_ptr, col_segs=by_col.astype(np.int64))


def segment_index(layout: dict, worker, col) -> np.ndarray:
    """Map (worker, item) pairs to segment indices of ``layout`` (-1 when the
    pair holds no ratings)."""
    worker = np.asarray(worker, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = layout["n"]
    key_seg = layout["seg_worker"].astype(np.int64) * n + layout["seg_col"]
    key = worker * n + col
    pos = np.searchsorted(key_seg, key)
    pos_c = np.minimum(pos, max(key_seg.size - 1, 0))
    ok = (pos < key_seg.size) & (key_seg[pos_c] == key) if key_seg.size else \
        np.zeros(key.shape, dtype=bool)
    return np.where(ok, pos_c, -1).astype(np.int64)


# ---------------------------------------------------------------- drivers
def replay(layout: dict, visit_seg, W, H, lam: float, alpha: float,
           beta: float, precision: str = "f64", rec_count=None,
           h_uses_new_w: bool = False):
    """Apply the visits ``visit_seg`` (segment indices) in the given serial
    order (Alg. 1's inner loop per visit).  Returns (W, H, rec_count)."""
    visit_seg = _c(visit_seg, np.int64)
    seg_ptr, seg_col = layout["seg_ptr"], _c(layout["seg_col"], np.int32)
    rec_row = _c(layout["rec_row"], np.int32)
    nrec = rec_row.size
    cnt = (np.zeros(nrec, dtype=np.int32) if rec_count is None
           else _c(rec_count, np.int32).copy())
    k = W.shape[1]
    if precision == "f64":
        W = _c(W, np.float64).copy()
        H = _c(H, np.float64).copy()
        val = _c(layout["rec_val"], np.float64)
        rc = _lib().orc_replay_f64(k, lam, alpha, beta, visit_seg.size,
                                   _ptr(visit_seg), seg_col.size, _ptr(seg_ptr),
                                   _ptr(seg_col), _ptr(rec_row), _ptr(val),
                                   _ptr(W), _ptr(H), _ptr(cnt),
                                   1 if h_uses_new_w else 0)
    elif precision == "f32":
        assert not h_uses_new_w
        W = _c(W, np.float32).copy()
        H = _c(H, np.float32).copy()
        val = _c(layout["rec_val"], np.float32)
        rc = _lib().orc_replay_f32(k, lam, alpha, beta, visit_seg.size,
                                   _ptr(visit_seg), seg_col.size, _ptr(seg_ptr),
                                   _ptr(seg_col), _ptr(rec_row), _ptr(val),
                                   _ptr(W), _ptr(H), _ptr(cnt))
    else:
        raise ValueError(precision)
    if rc != 0:
        raise ValueError("replay: segment index out of range")
    return W, H, cnt


def serial_nomad(layout: dict, W, H, lam: float, alpha: float, beta: float,
                 n_epochs: int, seed: int, mode: str = "epoch",
                 log_cap: int = 0, queue_stats=None):
    """Serial simulation of Alg. 1 with p simulated queues (see the C source
    for the schedule); mode "epoch", "uniform" or "uniform-shorter" (the
    dynamic load balancing of Sec. 3.3).  Returns (W, H, rec_count,
    visit_log); `queue_stats`, an int64 array of 2, receives the longest
    queue met by a push and the sum of the queue lengths met by pushes."""
    W = _c(W, np.float64).copy()
    H = _c(H, np.float64).copy()
    cnt = np.zeros(layout["rec_row"].size, dtype=np.int32)
    log = np.zeros(max(log_cap, 1), dtype=np.int64)
    seg_col = _c(layout["seg_col"], np.int32)
    seg_worker = _c(layout["seg_worker"], np.int32)
    rec_row = _c(layout["rec_row"], np.int32)
    rec_val = _c(layout["rec_val"], np.float64)
    nv = _lib().orc_serial_nomad(
        W.shape[1], lam, alpha, beta, layout["p"], layout["n"], seg_col.size,
        _ptr(layout["seg_ptr"]), _ptr(seg_col), _ptr(seg_worker), _ptr(rec_row),
        _ptr(rec_val), _ptr(layout["col_seg_ptr"]), _ptr(layout["col_segs"]),
        n_epochs, seed, {"epoch": 0, "uniform": 1, "uniform-shorter": 2}[mode], _ptr(W),
        _ptr(H), _ptr(cnt), _ptr(log) if log_cap > 0 else None, log_cap,
        _ptr(queue_stats) if queue_stats is not None else None)
    if nv < 0:
        raise ValueError("serial_nomad: bad argument or corrupt layout")
    return W, H, cnt, log[:min(nv, log_cap)]


def shuffled_sgd(rows, cols, vals, W, H, lam: float, alpha: float, beta: float,
                 n_epochs: int, seed: int):
    """Textbook SGD, a fresh random permutation of Omega per epoch (Sec. 2.3).
    Returns (W, H, rec_count)."""
    rows, cols = _c(rows, np.int32), _c(cols, np.int32)
    vals = _c(vals, np.float64)
    W = _c(W, np.float64).copy()
    H = _c(H, np.float64).copy()
    cnt = np.zeros(rows.size, dtype=np.int32)
    rc = _lib().orc_shuffled_sgd(W.shape[1], lam, alpha, beta, rows.size,
                                 _ptr(rows), _ptr(cols), _ptr(vals), n_epochs,
                                 seed, _ptr(W), _ptr(H), _ptr(cnt))
    if rc != 0:
        raise MemoryError("shuffled_sgd")
    return W, H, cnt


# ---------------------------------------------------------------- bfloat16
def bf16_rn(x) -> np.ndarray:
    """bfloat16 bit patterns (uint16) of binary32 values, round to nearest
    even."""
    x = _c(x, np.float32)
    out = np.zeros(x.shape, dtype=np.uint16)
    _lib().orc_bf16_rn_n(x.size, _ptr(x), _ptr(out))
    return out


def bf16_sr(x, r16) -> np.ndarray:
    """Stochastic rounding of binary32 values to bfloat16 with the given 16
    random bits per value."""
    x = _c(x, np.float32)
    r = _c(r16, np.uint32)
    assert r.shape == x.shape
    out = np.zeros(x.shape, dtype=np.uint16)
    _lib().orc_bf16_sr_n(x.size, _ptr(x), _ptr(r), _ptr(out))
    return out


def bf16_to_f32(b) -> np.ndarray:
    b = _c(b, np.uint16)
    out = np.zeros(b.shape, dtype=np.float32)
    _lib().orc_bf16_to_f32_n(b.size, _ptr(b), _ptr(out))
    return out


def replay_bf16(layout: dict, visit_seg, visit_epoch, Wb, Hb, lam: float,
                alpha: float, beta: float, seed: int, rec_count=None):
    """Replay with bfloat16 storage and stochastic rounding (see the C
    source).  Wb, Hb are uint16 bit patterns (m x k, n x k).  Returns
    (Wb, Hb, rec_count)."""
    visit_seg = _c(visit_seg, np.int64)
    visit_epoch = _c(visit_epoch, np.int32)
    assert visit_seg.shape == visit_epoch.shape
    Wb = _c(Wb, np.uint16).copy()
    Hb = _c(Hb, np.uint16).copy()
    seg_col = _c(layout["seg_col"], np.int32)
    rec_row = _c(layout["rec_row"], np.int32)
    rec_val = _c(layout["rec_val"], np.float32)
    cnt = (np.zeros(rec_row.size, dtype=np.int32) if rec_count is None
           else _c(rec_count, np.int32).copy())
    rc = _lib().orc_replay_bf16(Wb.shape[1], lam, alpha, beta, visit_seg.size,
                                _ptr(visit_seg), _ptr(visit_epoch), seg_col.size,
                                _ptr(layout["seg_ptr"]), _ptr(seg_col),
                                _ptr(rec_row), _ptr(rec_val), _ptr(Wb), _ptr(Hb),
                                _ptr(cnt), seed)
    if rc != 0:
        raise ValueError("replay_bf16: bad segment index or allocation failure")
    return Wb, Hb, cnt


# ---------------------------------------------------------------- FP8 E4M3
def e4m3_rn(x) -> np.ndarray:
    """E4M3 codes (uint8) of binary32 values, round to nearest even,
    saturating at 448."""
    x = _c(x, np.float32)
    out = np.zeros(x.shape, dtype=np.uint8)
    _lib().orc_e4m3_rn_n(x.size, _ptr(x), _ptr(out))
    return out


def e4m3_sr(x, r16) -> np.ndarray:
    """Stochastic rounding of binary32 values to E4M3 with the given 16
    random bits per value (see the C source for the rule)."""
    x = _c(x, np.float32)
    r = _c(r16, np.uint32)
    assert r.shape == x.shape
    out = np.zeros(x.shape, dtype=np.uint8)
    _lib().orc_e4m3_sr_n(x.size, _ptr(x), _ptr(r), _ptr(out))
    return out


def e4m3_to_f32(c) -> np.ndarray:
    c = _c(c, np.uint8)
    out = np.zeros(c.shape, dtype=np.float32)
    _lib().orc_e4m3_to_f32_n(c.size, _ptr(c), _ptr(out))
    return out


def e4m3_rows(W, r16=None):
    """Per-row scaled E4M3 storage of the rows of W (binary32, rows x k):
    (codes uint8 rows x k, scales float32 rows); r16 = None rounds to
    nearest, else stochastic with r16 (uint32, rows x k)."""
    W = _c(W, np.float32)
    rows, k = W.shape
    codes = np.zeros((rows, k), dtype=np.uint8)
    scales = np.zeros(rows, dtype=np.float32)
    r = None if r16 is None else _c(r16, np.uint32)
    if r is not None:
        assert r.shape == W.shape
    _lib().orc_e4m3_rows(rows, k, _ptr(W), None if r is None else _ptr(r), _ptr(codes),
                         _ptr(scales))
    return codes, scales


def e4m3_decode_rows(codes, scales) -> np.ndarray:
    """The stored binary32 values: scale * decode(code), row by row."""
    return (e4m3_to_f32(codes) * _c(scales, np.float32)[:, None]).astype(np.float32)


def replay_e4m3(layout: dict, visit_seg, visit_epoch, Wc, Ws, H, lam: float,
                alpha: float, beta: float, seed: int, rec_count=None):
    """Replay with W stored as per-row scaled E4M3 (codes Wc m x k, scales Ws
    m) and H in binary32 (see the C source).  Returns (Wc, Ws, H,
    rec_count)."""
    visit_seg = _c(visit_seg, np.int64)
    visit_epoch = _c(visit_epoch, np.int32)
    assert visit_seg.shape == visit_epoch.shape
    Wc = _c(Wc, np.uint8).copy()
    Ws = _c(Ws, np.float32).copy()
    H = _c(H, np.float32).copy()
    seg_col = _c(layout["seg_col"], np.int32)
    rec_row = _c(layout["rec_row"], np.int32)
    rec_val = _c(layout["rec_val"], np.float32)
    cnt = (np.zeros(rec_row.size, dtype=np.int32) if rec_count is None
           else _c(rec_count, np.int32).copy())
    rc = _lib().orc_replay_e4m3(Wc.shape[1], lam, alpha, beta, visit_seg.size,
                                _ptr(visit_seg), _ptr(visit_epoch), seg_col.size,
                                _ptr(layout["seg_ptr"]), _ptr(seg_col), _ptr(rec_row),
                                _ptr(rec_val), _ptr(Wc), _ptr(Ws), _ptr(H), _ptr(cnt),
                                seed)
    if rc != 0:
        raise ValueError("replay_e4m3: bad segment index or allocation failure")
    return Wc, Ws, H, cnt
