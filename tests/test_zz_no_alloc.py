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
