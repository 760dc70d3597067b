"""Seeded synthetic rating matrices for NOMAD matrix completion.

This module only makes inputs: sets of observed entries Omega with values,
split into train and test.  It holds none of the method's arithmetic, and it
serves the oracle and the CUDA path alike (the same arrays are handed to
both).  Generation runs with torch on the CPU or on a CUDA device (the large
shapes are generated on the device, where sorting 10^8 keys takes
milliseconds).

Recipes (the datasets of the paper's Table 2 are not available; these stand
in for them with their shapes and the generation recipe of Sec. 5.5):

* planted(m, n, r, nnz, ...): entries chosen uniformly without replacement,
  truth U (m x r), V (n x r) with i.i.d. N(0, var) entries, var = 1/sqrt(r),
  so that <u_i, v_j> has unit variance; A_ij = <u_i, v_j> + N(0, noise^2).
* skewed(...): user and item degrees from rank-frequency Zipf weights
  (weight of rank t proportional to t^-s, random rank -> id map), capped at
  the other dimension with the excess water-filled onto the uncapped ids;
  distinct (i,j) pairs drawn Chung-Lu style (row and column sampled
  independently from the degree weights, duplicates dropped, more drawn until
  the target count is met); values from a planted rank-r model through a
  per-shape value map (clip/round for integer ratings).
* planted_sparse(m, n, r, density, ...): as planted(), for shapes whose
  m x n cells are too many to permute: uniform cell keys drawn with
  replacement, duplicates dropped, a uniform subset of the target size kept.
* sweep_specs(count, seed) / sweep_problem(spec): a set of independent
  problems of random shape and hyperparameters, as for a sweep over lambda
  and k: m ~ U[2,000, 200,000], n ~ U[1,000, 50,000], density ~ U[0.1%, 2%],
  k in {16, 32, 64, 128}, lambda in {0.01, 0.05, 0.1, 0.5}, each a planted
  rank-k matrix with noise 0.1 and a 1% test hold-out.
* The train/test split is a seeded uniform hold-out restricted so that every
  test row and test column keeps at least one training rating.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch


@dataclass
class Ratings:
    m: int
    n: int
    train_rows: torch.Tensor  # int32
    train_cols: torch.Tensor  # int32
    train_vals: torch.Tensor  # float32
    test_rows: torch.Tensor
    test_cols: torch.Tensor
    test_vals: torch.Tensor
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.train_rows.numel())

    def numpy(self):
        """(train_rows, train_cols, train_vals, test_rows, test_cols,
        test_vals) as numpy arrays on the host."""
        f = lambda t: t.detach().cpu().numpy()
        return (f(self.train_rows), f(self.train_cols), f(self.train_vals),
                f(self.test_rows), f(self.test_cols), f(self.test_vals))

    def to(self, device) -> "Ratings":
        t = lambda x: x.to(device)
        return Ratings(self.m, self.n, t(self.train_rows), t(self.train_cols),
                       t(self.train_vals), t(self.test_rows), t(self.test_cols),
                       t(self.test_vals), self.name)

    def fingerprint(self) -> list:
        """Sums of the index and value arrays (train and test): two runs of a
        generator gave the same data when these agree."""
        f = lambda t: t.detach().cpu().numpy()
        return [int(f(self.train_rows).astype(np.int64).sum()),
                int(f(self.train_cols).astype(np.int64).sum()),
                float(f(self.train_vals).astype(np.float64).sum()),
                int(f(self.test_rows).astype(np.int64).sum()),
                int(f(self.test_cols).astype(np.int64).sum()),
                float(f(self.test_vals).astype(np.float64).sum())]

    def stats(self) -> dict:
        r = self.train_rows.long()
        c = self.train_cols.long()
        rd = torch.bincount(r, minlength=self.m)
        cd = torch.bincount(c, minlength=self.n)
        return dict(m=self.m, n=self.n, nnz_train=self.nnz,
                    nnz_test=int(self.test_rows.numel()),
                    row_deg_max=int(rd.max()) if rd.numel() else 0,
                    row_deg_mean=float(rd.float().mean()) if rd.numel() else 0,
                    col_deg_max=int(cd.max()) if cd.numel() else 0,
                    col_deg_mean=float(cd.float().mean()) if cd.numel() else 0,
                    active_rows=int((rd > 0).sum()),
                    active_cols=int((cd > 0).sum()))


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _truth_dot(rows, cols, U, V, chunk=1 << 22):
    out = torch.empty(rows.numel(), dtype=torch.float32, device=rows.device)
    for s in range(0, rows.numel(), chunk):
        e = min(s + chunk, rows.numel())
        out[s:e] = (U[rows[s:e].long()] * V[cols[s:e].long()]).sum(1)
    return out


# Above this many elements the generators work in chunks: torch's unique,
# randperm and boolean indexing go through CUB, which takes fewer than 2^31.
_CHUNK = 1 << 30


def _masked(x, mask):
    """x[mask], chunk by chunk for long tensors."""
    if x.numel() <= _CHUNK:
        return x[mask]
    return torch.cat([x[s:s + _CHUNK][mask[s:s + _CHUNK]]
                      for s in range(0, x.numel(), _CHUNK)])


def _bincount(x, minlength):
    if x.numel() <= _CHUNK:
        return torch.bincount(x.long(), minlength=minlength)
    out = torch.zeros(minlength, dtype=torch.int64, device=x.device)
    for s in range(0, x.numel(), _CHUNK):
        out += torch.bincount(x[s:s + _CHUNK].long(), minlength=minlength)
    return out


def _split(rows, cols, vals, n_test, m, n, g):
    """Uniform hold-out of about n_test entries; a test entry whose row or
    column would be left without a training entry goes back to training."""
    nnz = rows.numel()
    dev = rows.device
    is_test = torch.zeros(nnz, dtype=torch.bool, device=dev)
    if nnz <= _CHUNK:
        perm = torch.randperm(nnz, generator=g, device=dev)
        is_test[perm[:n_test]] = True
    else:  # n_test distinct positions drawn uniformly
        pick = torch.empty(0, dtype=torch.int64, device=dev)
        while pick.numel() < n_test:
            draw = torch.randint(0, nnz, (int((n_test - pick.numel()) * 1.1) + 16,),
                                 generator=g, device=dev)
            pick = torch.unique(torch.cat([pick, draw]))
        pick = pick[torch.randperm(pick.numel(), generator=g, device=dev)[:n_test]]
        is_test[pick] = True
    tr = ~is_test
    rdeg = _bincount(_masked(rows, tr), m)
    cdeg = _bincount(_masked(cols, tr), n)
    bad = is_test & ((rdeg[rows.long()] == 0) | (cdeg[cols.long()] == 0))
    is_test &= ~bad
    tr = ~is_test
    return (_masked(rows, tr), _masked(cols, tr), _masked(vals, tr), _masked(rows, is_test),
            _masked(cols, is_test), _masked(vals, is_test))


def _sort_rowmajor(rows, cols, vals, n):
    key = rows.long() * n + cols.long()
    order = torch.argsort(key)
    return rows[order], cols[order], vals[order]


def planted(m: int, n: int, r: int, nnz_total: int, noise: float,
            test_frac: float, seed: int, device="cpu", name="planted") -> Ratings:
    """Uniformly observed planted low-rank matrix (see module docstring)."""
    g = _gen(seed, device)
    assert nnz_total <= m * n
    keys = torch.randperm(m * n, generator=g, device=device)[:nnz_total]
    rows = (keys // n).to(torch.int32)
    cols = (keys % n).to(torch.int32)
    std = (1.0 / math.sqrt(r)) ** 0.5
    U = torch.randn(m, r, generator=g, device=device) * std
    V = torch.randn(n, r, generator=g, device=device) * std
    vals = _truth_dot(rows, cols, U, V)
    if noise > 0:
        vals = vals + noise * torch.randn(vals.shape, generator=g, device=device)
    rows, cols, vals = _sort_rowmajor(rows, cols, vals, n)
    n_test = int(round(test_frac * nnz_total))
    parts = _split(rows, cols, vals.float(), n_test, m, n, g)
    return Ratings(m, n, *parts, name=name)


def planted_sparse(m: int, n: int, r: int, density: float, noise: float,
                   test_frac: float, seed: int, device="cpu", name="planted-sparse") -> Ratings:
    """Uniformly observed planted low-rank matrix with about density*m*n
    entries, drawn without permuting all m*n cells."""
    g = _gen(seed, device)
    target = max(1, int(round(density * m * n)))
    cells = m * n
    keys = torch.empty(0, dtype=torch.int64, device=device)
    for _ in range(64):
        need = target - keys.numel()
        if need <= 0:
            break
        draw = torch.randint(0, cells, (int(need * 1.1) + 16,), generator=g, device=device)
        keys = torch.unique(torch.cat([keys, draw]))
    keys = keys[torch.randperm(keys.numel(), generator=g, device=device)[:target]]
    rows = (keys // n).to(torch.int32)
    cols = (keys % n).to(torch.int32)
    std = (1.0 / math.sqrt(r)) ** 0.5
    U = torch.randn(m, r, generator=g, device=device) * std
    V = torch.randn(n, r, generator=g, device=device) * std
    vals = _truth_dot(rows, cols, U, V)
    if noise > 0:
        vals = vals + noise * torch.randn(vals.shape, generator=g, device=device)
    rows, cols, vals = _sort_rowmajor(rows, cols, vals, n)
    n_test = int(round(test_frac * rows.numel()))
    parts = _split(rows, cols, vals.float(), n_test, m, n, g)
    return Ratings(m, n, *parts, name=name)


def sweep_specs(count: int = 64, seed: int = 5) -> list:
    """Shapes and hyperparameters of `count` independent problems (see the
    module docstring); problem i is generated from seed 1000 * seed + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        out.append(dict(m=int(rng.integers(2000, 200001)), n=int(rng.integers(1000, 50001)),
                        density=float(rng.uniform(0.001, 0.02)),
                        k=int(rng.choice([16, 32, 64, 128])),
                        lam=float(rng.choice([0.01, 0.05, 0.1, 0.5])),
                        seed=1000 * seed + i))
    return out


def sweep_problem(spec: dict, device="cpu") -> Ratings:
    return planted_sparse(spec["m"], spec["n"], spec["k"], spec["density"], 0.1, 0.01,
                          spec["seed"], device,
                          name="sweep-%d m=%d n=%d k=%d" % (spec["seed"] % 1000, spec["m"],
                                                           spec["n"], spec["k"]))


def tiny_planted(seed: int = 1, device="cpu") -> Ratings:
    """m=1000, n=500, true rank 10, 25,000 observed entries (5%), noise
    N(0, 0.1^2), 10% held out for test."""
    return planted(1000, 500, 10, 25000, 0.1, 0.10, seed, device,
                   name="tiny-planted")


def zipf_degrees(count: int, total: float, s: float, cap: float, g) -> torch.Tensor:
    """Expected degrees: rank-frequency Zipf(s) weights over `count` ids in a
    random rank -> id order, scaled to sum to `total`, capped at `cap` with
    the excess water-filled onto uncapped ids (float64, on g's device)."""
    dev = g.device
    ranks = torch.arange(1, count + 1, dtype=torch.float64, device=dev)
    w = ranks.pow(-s)
    d = w / w.sum() * total
    for _ in range(64):
        over = d > cap
        if not bool(over.any()):
            break
        excess = float((d[over] - cap).sum())
        d[over] = cap
        free = ~over & (d < cap)
        if not bool(free.any()):
            break
        d[free] += excess * d[free] / d[free].sum()
    perm = torch.randperm(count, generator=g, device=dev)
    out = torch.empty_like(d)
    out[perm] = d
    return out


def _sample_pairs(du, dv, target, n, g, max_rounds=64):
    """Distinct (i, j) pairs, i ~ du / sum(du), j ~ dv / sum(dv)."""
    if target > _CHUNK:
        return _sample_pairs_chunked(du, dv, target, n, g, max_rounds)
    dev = du.device
    cu = torch.cumsum(du, 0)
    cu = cu / cu[-1]
    cv = torch.cumsum(dv, 0)
    cv = cv / cv[-1]
    keys = torch.empty(0, dtype=torch.int64, device=dev)
    for _ in range(max_rounds):
        need = target - keys.numel()
        if need <= 0:
            break
        draw = int(need * 1.15) + 1024
        i = torch.searchsorted(cu, torch.rand(draw, generator=g, device=dev,
                                              dtype=torch.float64))
        j = torch.searchsorted(cv, torch.rand(draw, generator=g, device=dev,
                                              dtype=torch.float64))
        i = i.clamp_(max=du.numel() - 1)
        j = j.clamp_(max=dv.numel() - 1)
        keys = torch.unique(torch.cat([keys, i * n + j]))
    if keys.numel() > target:
        pick = torch.randperm(keys.numel(), generator=g, device=dev)[:target]
        keys = torch.sort(keys[pick]).values
    return keys


def _sample_pairs_chunked(du, dv, target, n, g, max_rounds=64):
    """_sample_pairs for more than _CHUNK pairs: the users are cut into
    ranges of about equal degree weight, each range receives its share of the
    pairs (i drawn from the range's weights, j from all items), and pairs are
    made distinct within a range (ranges share no user)."""
    dev = du.device
    cu = torch.cumsum(du.double(), 0)
    total_w = float(cu[-1])
    nchunks = (target + _CHUNK // 2 - 1) // (_CHUNK // 2)
    # user boundaries at equal weight fractions
    cuts = torch.searchsorted(cu, torch.linspace(0, total_w, nchunks + 1, device=dev,
                                                 dtype=torch.float64)[1:-1])
    bounds = [0] + [int(c) + 1 for c in cuts.tolist()] + [du.numel()]
    cv = torch.cumsum(dv.double(), 0)
    cv = cv / cv[-1]
    out, assigned = [], 0
    for c in range(nchunks):
        lo, hi = bounds[c], bounds[c + 1]
        if hi <= lo:
            continue
        w_lo = float(cu[lo - 1]) if lo > 0 else 0.0
        w_hi = float(cu[hi - 1])
        t_c = target - assigned if c == nchunks - 1 else int(round(target * (w_hi - w_lo) / total_w))
        t_c = min(t_c, (hi - lo) * int(dv.numel()))
        assigned += t_c
        cuc = (cu[lo:hi] - w_lo) / (w_hi - w_lo)
        keys = torch.empty(0, dtype=torch.int64, device=dev)
        for _ in range(max_rounds):
            need = t_c - keys.numel()
            if need <= 0:
                break
            draw = int(need * 1.15) + 1024
            i = torch.searchsorted(cuc, torch.rand(draw, generator=g, device=dev,
                                                   dtype=torch.float64))
            j = torch.searchsorted(cv, torch.rand(draw, generator=g, device=dev,
                                                  dtype=torch.float64))
            i = i.clamp_(max=hi - lo - 1) + lo
            j = j.clamp_(max=dv.numel() - 1)
            keys = torch.unique(torch.cat([keys, i * n + j]))
        if keys.numel() > t_c:
            pick = torch.randperm(keys.numel(), generator=g, device=dev)[:t_c]
            keys = torch.sort(keys[pick]).values
        out.append(keys)
    return torch.cat(out)


def skewed(m: int, n: int, nnz_train: int, nnz_test: int, user_s: float,
           item_s: float, r: int, value_map, seed: int, device="cpu",
           name="skewed") -> Ratings:
    """Heavy-tailed degrees, planted rank-r values (see module docstring).
    value_map(dot, noise_std_normal) -> float32 values."""
    g = _gen(seed, device)
    total = nnz_train + nnz_test
    du = zipf_degrees(m, total, user_s, float(n), g)
    dv = zipf_degrees(n, total, item_s, float(m), g)
    keys = _sample_pairs(du, dv, total, n, g)
    rows = (keys // n).to(torch.int32)
    cols = (keys % n).to(torch.int32)
    del keys
    std = (1.0 / math.sqrt(r)) ** 0.5
    U = torch.randn(m, r, generator=g, device=device) * std
    V = torch.randn(n, r, generator=g, device=device) * std
    dot = _truth_dot(rows, cols, U, V)
    del U, V
    z = torch.randn(dot.shape, generator=g, device=device)
    vals = value_map(dot, z).float()
    parts = _split(rows, cols, vals, nnz_test, m, n, g)
    return Ratings(m, n, *parts, name=name)


def netflix_value(dot, z):
    """Integer ratings 1..5: clip(round(3.6 + <u,v> + N(0, 0.5^2)), 1, 5)."""
    return torch.clamp(torch.round(3.6 + dot + 0.5 * z), 1.0, 5.0)


def yahoo_value(dot, z):
    """Integer ratings 0..100: clip(round(50 + 20 <u,v> + N(0, 10^2)), 0, 100)."""
    return torch.clamp(torch.round(50.0 + 20.0 * dot + 10.0 * z), 0.0, 100.0)


def hugewiki_value(dot, z):
    """Real values <u,v> + N(0, 0.1^2)."""
    return dot + 0.1 * z


def netflix_shaped(scale: float = 1.0, seed: int = 2, device="cpu") -> Ratings:
    """Netflix-shaped: m=480,189, n=17,770, ~100.5M train + ~1.4M test,
    Zipf(1.2) user and item degrees, integer ratings 1..5 from a clipped
    rank-100 model plus noise.  `scale` < 1 shrinks m and the rating counts
    (n shrinks with sqrt(scale)) for tests."""
    m = max(64, int(round(480189 * scale)))
    n = max(32, int(round(17770 * math.sqrt(scale))))
    return skewed(m, n, int(round(100_480_507 * scale)),
                  int(round(1_408_395 * scale)), 1.2, 1.2, 100, netflix_value,
                  seed, device, name="netflix-shaped" if scale == 1.0 else
                  "netflix-shaped-x%g" % scale)


def yahoo_shaped(scale: float = 1.0, seed: int = 3, device="cpu") -> Ratings:
    """Yahoo!-Music-shaped: m=1,000,990, n=624,961, ~252.8M train + ~4M test,
    Zipf(1.2) degrees, integer ratings 0..100 from a planted rank-100 model."""
    m = max(64, int(round(1_000_990 * scale)))
    n = max(32, int(round(624_961 * scale)))
    return skewed(m, n, int(round(252_800_275 * scale)),
                  int(round(4_003_960 * scale)), 1.2, 1.2, 100, yahoo_value,
                  seed, device, name="yahoo-shaped" if scale == 1.0 else
                  "yahoo-shaped-x%g" % scale)


def hugewiki_shaped(scale: float = 1.0, seed: int = 4, device="cpu",
                    item_s: float = 0.8, name: str = "hugewiki-shaped") -> Ratings:
    """Hugewiki-shaped: m=50,082,603, n=39,780, ~2.74B train ratings (mean
    54.6 per row; mild Zipf(0.5) over rows and Zipf(item_s) over columns) +
    1% test; real values <u,v> + N(0, 0.1^2) from a planted rank-100 model.
    With the default Zipf(0.8) over columns the weights of the top items
    exceed m and are capped: the most-rated item is rated by every user
    (50.1M ratings at full size), a property of this generator, not of the
    paper's data (whose mean is 68,635 ratings per item)."""
    m = max(64, int(round(50_082_603 * scale)))
    n = max(32, int(round(39_780 * math.sqrt(scale))))
    nnz = int(round(2_736_496_604 * scale))
    return skewed(m, n, nnz, nnz // 100, 0.5, item_s, 100, hugewiki_value, seed,
                  device, name=name if scale == 1.0 else "%s-x%g" % (name, scale))


def hugewiki_flat(scale: float = 1.0, seed: int = 4, device="cpu") -> Ratings:
    """Hugewiki-shaped with flatter column degrees, Zipf(0.5): no column
    reaches the cap m, and the most-rated item holds about 0.25% of the
    ratings (about 6.9M of 2.74B at full size, 14% of the users)."""
    return hugewiki_shaped(scale, seed, device, item_s=0.5, name="hugewiki-flat")
