"""The seeded input generators: the sparse planted sampler and the chunked
paths taken above torch's 2^31-element limits (forced here at a small
chunk size), on CPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import synth  # noqa: E402


def test_planted_sparse_is_a_set_with_its_density():
    r = synth.planted_sparse(3000, 1500, 16, 0.01, 0.1, 0.01, seed=9)
    tr, tc, tv, er, ec, ev = r.numpy()
    rows = np.concatenate([tr, er]).astype(np.int64)
    cols = np.concatenate([tc, ec]).astype(np.int64)
    keys = rows * 1500 + cols
    assert np.unique(keys).size == keys.size  # Omega is a set
    assert keys.size == round(0.01 * 3000 * 1500)
    assert rows.min() >= 0 and rows.max() < 3000 and cols.min() >= 0 and cols.max() < 1500



def test_chunked_generation_is_a_valid_split(monkeypatch):
    """Above the chunk size, pairs are drawn per user range and the hold-out
    by distinct draws: Omega is still a set of the requested size, every
    test row and column keeps a training rating, and the degrees stay skewed."""
    ref = synth.netflix_shaped(0.001, seed=3)  # the same shape, one chunk
    monkeypatch.setattr(synth, "_CHUNK", 1 << 13)
    r = synth.netflix_shaped(0.001, seed=3)
    tr, tc, tv, er, ec, ev = r.numpy()
    keys = np.concatenate([tr, er]).astype(np.int64) * r.n + np.concatenate([tc, ec])
    assert np.unique(keys).size == keys.size
    want = int(round(100_480_507 * 0.001)) + int(round(1_408_395 * 0.001))
    assert abs(keys.size - want) <= 2
    assert np.isin(er, tr).all() and np.isin(ec, tc).all()
    assert er.size > 0.9 * int(round(1_408_395 * 0.001))
    # the degree profiles of users and items match the one-chunk sampler's
    for a, b, size in ((tr, ref.numpy()[0], r.m), (tc, ref.numpy()[1], r.n)):
        qa = np.quantile(np.bincount(a, minlength=size), [0.5, 0.9, 0.99, 1.0])
        qb = np.quantile(np.bincount(b, minlength=size), [0.5, 0.9, 0.99, 1.0])
        assert np.all(np.abs(qa - qb) <= 0.15 * qb + 2), (qa, qb)


@pytest.mark.parametrize("k", [16, 128])
def test_sweep_problem_follows_its_recipe(k):
    """A sweep problem is a planted rank-k matrix: <u_i, v_j> has unit
    variance and the noise is N(0, 0.1^2), so the values have mean ~0 and
    variance ~1.01; density*m*n distinct entries, 1% held out."""
    r = synth.sweep_problem(dict(m=4000, n=2000, density=0.01, k=k, lam=0.1, seed=3))
    tr, tc, tv, er, ec, ev = r.numpy()
    v = np.concatenate([tv, ev]).astype(np.float64)
    assert v.size == 80000
    assert abs(er.size - 800) <= 8
    assert abs(v.mean()) < 0.03
    assert 0.9 < v.var() < 1.15, v.var()
