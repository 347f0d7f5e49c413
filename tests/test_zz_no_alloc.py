"""The allocation-free tree solve (cn_solve_trees_noalloc) against the
allocating one (cn_solve_trees), through the C ABI.

It serves callers that cannot allocate device memory when they solve (for
instance because another allocator already holds the whole GPU); it uses a
fixed scratch array built into the library instead.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL_TOL = 1e-13   # same bar as the tree-solve tests


@pytest.fixture(scope="module")
def cn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10975_gb300 import build
    build.build()
    from paper_1901_10975_gb300 import cn as _cn
    return _cn


def random_trees(seed, n_trees, max_n):
    rng = np.random.default_rng(seed)
    parents, parts = [], []
    for _ in range(n_trees):
        n = int(rng.integers(1, max_n))
        p = np.array([-1] + [int(rng.integers(max(0, i - 9), i)) for i in range(1, n)], np.int32)
        a = np.where(p >= 0, -rng.uniform(0.1, 5.0, n), 0.0)
        b = np.where(p >= 0, -rng.uniform(0.1, 5.0, n), 0.0)
        d = rng.uniform(0.05, 1.0, n)
        for i in range(1, n):
            d[i] -= b[i]
            d[p[i]] -= a[i]
        parents.append(p)
        parts.append((a, b, d, rng.normal(size=n)))
    off = np.zeros(n_trees + 1, np.int32)
    off[1:] = np.cumsum([len(p) for p in parents])
    cat = lambda k: np.concatenate([x[k] for x in parts])
    return off, np.concatenate(parents), cat(0), cat(1), cat(2), cat(3)


def test_noalloc_matches_allocating_solve_twice(cn):
    """Two calls in a row with different systems: the shared fixed scratch
    must not carry anything over from the first call into the second."""
    for seed, n_trees, max_n in ((1, 700, 400), (2, 50, 3000)):
        off, parent, a, b, d, r = random_trees(seed, n_trees, max_n)
        ref = cn.cn_solve_trees(off, parent, a, b, d, r)
        got = cn.cn_solve_trees_noalloc(off, parent, a, b, d, r)
        assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= REL_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(cn):
    import ctypes as C
    st = cn.lib().cn_solve_trees_noalloc(1, (1 << 20) + 1, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16),
                                         C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), None)
    assert st == cn.CN_ERANGE


def test_noalloc_reports_device_errors_and_recovers(cn):
    """A bad parent gives CN_EINVAL and a zero pivot CN_ERANGE (both found on
    the device); a valid solve right after each on the same stream succeeds
    with the right answer, so the shared status word does not carry an error
    into the next call.  Every index stays inside the arrays."""
    off, parent, a, b, d, r = random_trees(3, 40, 60)
    ref = cn.cn_solve_trees(off, parent, a, b, d, r)
    bad_parent = np.array([-1, 0, 2], np.int32)           # parent[2] = 2 is not < 2
    with pytest.raises(cn.CNError) as e:
        cn.cn_solve_trees_noalloc(np.array([0, 3], np.int32), bad_parent, np.zeros(3), np.zeros(3),
                                  np.ones(3), np.ones(3))
    assert e.value.status == cn.CN_EINVAL
    got = cn.cn_solve_trees_noalloc(off, parent, a, b, d, r)
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= REL_TOL
    with pytest.raises(cn.CNError) as e:                   # leaf pivot 0
        cn.cn_solve_trees_noalloc(np.array([0, 2], np.int32), np.array([-1, 0], np.int32),
                                  np.array([0.0, -1.0]), np.array([0.0, -1.0]), np.array([2.0, 0.0]),
                                  np.ones(2))
    assert e.value.status == cn.CN_ERANGE
    with pytest.raises(cn.CNError) as e:                   # offsets past n_nodes
        cn.cn_solve_trees_noalloc(np.array([0, 2, 5], np.int32), np.array([-1, 0, -1, 0], np.int32),
                                  np.full(4, -0.5), np.full(4, -0.5), np.full(4, 3.0), np.ones(4))
    assert e.value.status == cn.CN_EINVAL
    got = cn.cn_solve_trees_noalloc(off, parent, a, b, d, r)
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= REL_TOL
