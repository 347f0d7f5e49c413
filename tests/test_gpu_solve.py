"""Batched tree solve on the GPU (cn_solve_trees) against the oracle's Hines
elimination and a dense LU solve, through the C ABI."""
import itertools

import numpy as np
import pytest

from oracle import hines_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10975_gb300 import build
    build.build()
    from paper_1901_10975_gb300 import cn as _cn
    return _cn


def _system(rng, parent):
    n = len(parent)
    a = np.where(parent >= 0, -rng.uniform(0.1, 5.0, n), 0.0)
    b = np.where(parent >= 0, -rng.uniform(0.1, 5.0, n), 0.0)
    d = rng.uniform(0.05, 1.0, n)
    for i in range(1, n):
        d[i] -= b[i]
        d[parent[i]] -= a[i]
    return a, b, d, rng.normal(size=n)


def batch_of_trees():
    rng = np.random.default_rng(5)
    trees = []
    for n in range(1, 8):
        for tail in itertools.product(*[range(i) for i in range(1, n)]):
            trees.append(np.array((-1,) + tail, np.int32))
    for _ in range(300):
        n = int(rng.integers(8, 600))
        trees.append(np.array([-1] + [int(rng.integers(max(0, i - 7), i)) for i in range(1, n)], np.int32))
    trees.append(np.arange(-1, 4999, dtype=np.int32))          # a 5,000-node chain
    parts = [_system(rng, p) for p in trees]
    off = np.zeros(len(trees) + 1, np.int32)
    off[1:] = np.cumsum([len(p) for p in trees])
    cat = lambda k: np.concatenate([x[k] for x in parts])
    return trees, off, np.concatenate(trees), cat(0), cat(1), cat(2), cat(3)


def reference(trees, off, a, b, d, r):
    out = np.empty_like(r)
    for t, p in enumerate(trees):
        s = slice(off[t], off[t + 1])
        out[s] = hines_solve(p, a[s], b[s], d[s], r[s])
    return out


def test_solve_trees_matches_oracle(cn):
    trees, off, parent, a, b, d, r = batch_of_trees()
    x = cn.cn_solve_trees(off, parent, a, b, d, r)
    ref = reference(trees, off, a, b, d, r)
    scale = np.maximum(1.0, np.abs(ref))
    assert np.max(np.abs(x - ref) / scale) <= 1e-13


def test_solve_trees_rejects_bad_parent(cn):
    off = np.array([0, 3], np.int32)
    parent = np.array([-1, 0, 2], np.int32)      # parent[2] = 2 is not < 2
    with pytest.raises(cn.CNError) as e:
        cn.cn_solve_trees(off, parent, np.zeros(3), np.zeros(3), np.ones(3), np.ones(3))
    assert e.value.status == cn.CN_EINVAL


@pytest.mark.parametrize("off", [[0, 3, 7],       # last offset past the 6 rows
                                 [0, 4, 2, 6],    # a descending offset (overlapping ranges)
                                 [1, 3, 6]])      # does not start at row 0
def test_solve_trees_rejects_bad_offsets(cn, off):
    """Offsets that disagree with n_nodes are refused before any row is
    touched (every index stays inside the six-row arrays)."""
    off = np.array(off, np.int32)
    parent = np.array([-1, 0, 1, -1, 0, 1], np.int32)
    with pytest.raises(cn.CNError) as e:
        cn.cn_solve_trees(off, parent, np.full(6, -0.5), np.full(6, -0.5), np.full(6, 3.0), np.ones(6))
    assert e.value.status == cn.CN_EINVAL


def _pivot_sweep():
    rng = np.random.default_rng(11)
    e = np.arange(-1021, 1021)
    p2 = np.ldexp(1.0, e)
    vals = [
        np.exp2(rng.uniform(-1021.0, 1021.0, 400_000)),           # the whole claimed range
        rng.uniform(1.0, 100.0, 400_000),                          # pivots of the cable matrix
        p2, np.nextafter(p2, 0.0), np.nextafter(p2, np.inf),       # powers of two and neighbours
        np.ldexp(2.0 - 2.0 ** -52, e[:-1]),                        # mantissa of all ones
        np.ldexp(1.0 + rng.integers(0, 2 ** 20, 100_000) * 2.0 ** -20, rng.integers(-1021, 1020, 100_000)),
        np.array([2.0 ** -1021, 2.0 ** 1021, np.nextafter(2.0 ** 1021, 0.0), 1.0, 3.0, 1.0 + 2 ** -52]),
    ]
    d = np.concatenate(vals)
    return d[(d >= 2.0 ** -1021) & (d <= 2.0 ** 1021)]


def test_pivot_reciprocal_within_one_ulp_of_ieee(cn):
    """The interval kernel's Newton-Raphson reciprocal (float seed, fixed-point
    step, FP64 step) against IEEE 1/d (numpy, correctly rounded) over the
    range the solve relies on, [2^-1021, 2^1021]: never more than 1 ulp off,
    and exactly rounded in most cases."""
    d = _pivot_sweep()
    got = cn.cn_pivot_reciprocal(d)
    ref = 1.0 / d
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    ulps = np.abs(got.view(np.int64) - ref.view(np.int64))
    exact = float(np.mean(ulps == 0))
    print(f"pivot reciprocal: {d.size} values, exact {exact:.5f}, max {ulps.max()} ulp")
    assert ulps.max() <= 1
    assert exact >= 0.99
