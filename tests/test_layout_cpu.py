"""Host checks of the cell-to-lane placement (no GPU needed).

cn_plan_layout returns, for every node, the lane and warp row the engine
gives it and the topology bits the interval kernel reads.  These tests check
the invariants the kernel relies on (Hines order inside every part, a part
root above its junction row in the same warp with matching mailbox entries,
one spike source per lane, far-child partial sums within the reported
stack depth), and then run the kernel's elimination schedule on random tree
systems in NumPy, following only the placement: the solution must equal a
direct sparse solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from scenarios import network, batched, passive_cable, ring16

FAR, REAL, JUNC, PROOT = 1 << 6, 1 << 11, 1 << 12, 1 << 13


def nfar(f):
    return (f >> 7) & 7


def jmail(f):
    return (int(f) >> 14) & 511


def pmail(f):
    return (int(f) & 0xffffffff) >> 23


@pytest.fixture(scope="module")
def cn():
    from paper_1901_10975_gb300 import build
    build.build()
    from paper_1901_10975_gb300 import cn as _cn
    return _cn


def cells_of(sc):
    off = np.asarray(sc.cell_offset, np.int64)
    return off, np.asarray(sc.parent, np.int32)


def check_invariants(off, parent, L):
    lane, row, fl = L["lane"], L["row"], L["flags"]
    n = parent.shape[0]
    assert np.all(fl & REAL)
    # one node per (lane, row)
    key = lane.astype(np.int64) * (1 << 32) + row
    assert np.unique(key).shape[0] == n
    nfar_seen = np.zeros(n, np.int64)
    for c in range(len(off) - 1):
        lo, hi = off[c], off[c + 1]
        lanes = np.unique(lane[lo:hi])
        assert np.all(lanes // 32 == lanes[0] // 32), "a cell spans two warps"
        assert not (fl[lo] & PROOT)
        for i in range(lo + 1, hi):
            p = lo + parent[i]
            if fl[i] & PROOT:
                assert fl[p] & JUNC and jmail(fl[p]) == pmail(fl[i])
                assert row[i] > row[p]
            elif fl[i] & FAR:
                assert lane[i] == lane[p] and row[p] < row[i] - 1
                nfar_seen[p] += 1
            else:
                assert lane[i] == lane[p] and row[p] == row[i] - 1
    assert np.array_equal(nfar(fl), nfar_seen)
    # a mailbox entry joins exactly one junction and one part root per warp
    for w in range(L["n_warps"]):
        sel = lane // 32 == w
        js = sorted(jmail(f) for f in fl[sel] if f & JUNC)
        ps = sorted(pmail(f) for f in fl[sel] if f & PROOT)
        assert js == ps and len(set(js)) == len(js)
    # one spike source (the cell's first node) per lane
    roots = lane[off[:-1]]
    assert np.unique(roots).shape[0] == roots.shape[0]


def emulate_solve(off, parent, L, a, b, d, rhs):
    """The interval kernel's elimination and back substitution, warp row by
    warp row, driven only by the placement and its flags.  Elimination takes
    one (-a, x, b/d) term per row: the previous row's, into this row when
    that row is its child; when that row was a far child, into the partial
    sums of its parent (which start from the parent's own row and replace it
    when the parent's row comes), on the row after it, which must be a leaf
    of the same lane."""
    lane, row, fl = L["lane"], L["row"], L["flags"]
    n = parent.shape[0]
    gpar = np.full(n, -1, np.int64)
    has_child = np.zeros(n, bool)
    for c in range(len(off) - 1):
        for i in range(off[c] + 1, off[c + 1]):
            gpar[i] = off[c] + parent[i]
            if not fl[i] & PROOT:
                has_child[gpar[i]] = True
    at = {}
    for i in range(n):
        at[(int(lane[i]), int(row[i]))] = i
    depth = L["stack_depth"]
    x = np.zeros(n)
    bp = np.zeros(n)
    v = np.zeros(n)
    span = np.zeros(L["n_warps"], np.int64)
    np.maximum.at(span, lane // 32, row.astype(np.int64) + 1)
    for w in range(L["n_warps"]):
        lanes = range(32 * w, 32 * w + 32)
        R = int(span[w])
        if R == 0:
            continue
        stack = {l: [] for l in lanes}   # [parent row, partial rhs, partial d]
        carry = {l: None for l in lanes}
        pend = {l: None for l in lanes}  # parent node of the previous row if it was far
        mail = {}
        maxtop = 0
        for j in range(R - 1, -1, -1):
            for l in lanes:
                i = at.get((l, j))
                if i is None:
                    assert pend[l] is None, "the row after a far child is empty"
                    carry[l] = None
                    continue
                f = int(fl[i])
                if stack[l] and stack[l][-1][0] == j:
                    _, r_, d_ = stack[l].pop()
                else:
                    r_, d_ = rhs[i], d[i]
                if pend[l] is not None:
                    assert not has_child[i], "the row after a far child has in-part children"
                    p = pend[l]
                    na, xx, bb = carry[l]
                    if stack[l] and stack[l][-1][0] == row[p]:
                        stack[l][-1][1] += na * xx
                        stack[l][-1][2] += na * bb
                    else:
                        stack[l].append([int(row[p]), rhs[p] + na * xx, d[p] + na * bb])
                        maxtop = max(maxtop, len(stack[l]))
                elif carry[l] is not None:
                    na, xx, bb = carry[l]
                    r_ += na * xx
                    d_ += na * bb
                if f & JUNC:
                    na, xx, bb = mail.pop(jmail(f))
                    r_ += na * xx
                    d_ += na * bb
                x[i] = r_ / d_
                bp[i] = b[i] / d_
                ent = (-a[i], x[i], bp[i])
                if f & PROOT:
                    assert pmail(f) not in mail
                    mail[pmail(f)] = ent
                    carry[l], pend[l] = None, None
                else:
                    carry[l] = ent
                    pend[l] = int(gpar[i]) if f & FAR else None
        assert all(len(s) == 0 for s in stack.values()) and not mail
        assert all(p is None for p in pend.values())
        assert maxtop <= depth
        # back substitution, root to leaves
        vstack = {l: [] for l in lanes}
        vprev = {l: 0.0 for l in lanes}
        vmail = {}
        for j in range(R):
            for l in lanes:
                i = at.get((l, j))
                if i is None:
                    continue
                f = int(fl[i])
                if f & FAR:
                    vp = vstack[l].pop()
                elif f & PROOT:
                    vp = vmail.pop(pmail(f))
                else:
                    vp = vprev[l]
                v[i] = x[i] - bp[i] * vp
                if f & JUNC:
                    vmail[jmail(f)] = v[i]
                vstack[l].extend([v[i]] * nfar(f))
                vprev[l] = v[i]
    return v


def random_system(off, parent, rng):
    n = parent.shape[0]
    a = -rng.uniform(0.1, 1.0, n)
    b = -rng.uniform(0.1, 1.0, n)
    d = np.zeros(n)
    rows, cols, vals = [], [], []
    for c in range(len(off) - 1):
        for i in range(off[c], off[c + 1]):
            p = parent[i]
            if p < 0:
                a[i] = b[i] = 0.0
                continue
            p += off[c]
            rows += [i, p]
            cols += [p, i]
            vals += [b[i], a[i]]
            d[i] += -b[i]
            d[p] += -a[i]
    d += rng.uniform(0.05, 1.0, n)
    A = sp.csr_matrix((np.concatenate([vals, d]), (np.concatenate([rows, np.arange(n)]),
                                                    np.concatenate([cols, np.arange(n)]))), shape=(n, n))
    rhs = rng.normal(size=n)
    return a, b, d, rhs, A


CASES = {
    "network": lambda: network(n_cells=60, tstop=1.0),
    "batched": lambda: batched(n_cells=24, tstop=1.0, n_in=4),
    "cable": lambda: passive_cable(700, L=1400.0, tstop=1.0),
    "ring": lambda: ring16(),
}


HEIGHT = 22  # bit of the warp height field


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("mapping", [1, 16, 40, 100, 300, 0, 16 | (1 << 20), 100 | (1 << 20), 40 | (3 << 20),
                                     24 | (2 << 20), 32 | (1 << 20) | (48 << HEIGHT), 16 | (1 << 20) | (24 << HEIGHT),
                                     100 | (1 << 20) | (200 << HEIGHT)])
def test_layout_invariants_and_emulated_solve(cn, case, mapping):
    off, parent = cells_of(CASES[case]())
    L = cn.cn_plan_layout(off, parent, mapping)
    check_invariants(off, parent, L)
    rng = np.random.default_rng(7)
    a, b, d, rhs, A = random_system(off, parent, rng)
    v = emulate_solve(off, parent, L, a, b, d, rhs)
    ref = spla.spsolve(A.tocsc(), rhs)
    assert np.max(np.abs(v - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_split_spreads_large_cells(cn):
    """The largest cell of the batched workload (a branched tree) with a
    100-row target occupies several lanes and its span (warp rows) drops well
    below its size; an unbranched cable cannot be shortened (its depth is
    its size) and stays on one lane."""
    off, parent = cells_of(batched(n_cells=24, tstop=1.0, n_in=4))
    sizes = np.diff(off)
    c = int(np.argmax(sizes))
    sub_off = np.array([0, sizes[c]])
    sub_par = parent[off[c]:off[c + 1]]
    one = cn.cn_plan_layout(sub_off, sub_par, 1)
    split = cn.cn_plan_layout(sub_off, sub_par, 100)
    assert np.unique(one["lane"]).shape[0] == 1 and one["row"].max() == sizes[c] - 1
    assert np.unique(split["lane"]).shape[0] >= 4 and split["row"].max() < sizes[c] // 2
    off, parent = cells_of(passive_cable(700, L=1400.0, tstop=1.0))
    assert np.unique(cn.cn_plan_layout(off, parent, 40)["lane"]).shape[0] == 1


def warp_rows(L):
    """Rows per warp (its highest used row + 1) and the lane tops."""
    span = np.zeros(L["n_warps"], np.int64)
    np.maximum.at(span, L["lane"] // 32, L["row"].astype(np.int64) + 1)
    return span


def test_warp_height_packs_tighter(cn):
    """A warp height below the largest cell span: every warp is that tall
    unless a cell that cannot be cut below it opens one (then as tall as
    that cell's span), and the parts, which may now fill the free runs
    below a lane's top, take fewer warp rows in all than warps as tall as
    the largest span at the same target."""
    off, parent = cells_of(network(n_cells=2048, tstop=1.0))
    tall = cn.cn_plan_layout(off, parent, 43 | (1 << 20))
    top = int(warp_rows(tall).max())
    h = (9 * top) // 10
    capped = cn.cn_plan_layout(off, parent, 43 | (1 << 20) | (h << HEIGHT))
    check_invariants(off, parent, capped)
    rows = warp_rows(capped)
    assert np.all(rows <= top)
    assert np.mean(rows <= h) > 0.95
    assert rows.sum() < 0.95 * warp_rows(tall).sum()


def test_plan_layout_rejects_bad_mappings(cn):
    off, parent = cells_of(ring16(tstop=1.0))
    for mp in [32 | (64 << HEIGHT), 32 | (3 << 20) | (64 << HEIGHT), 32 | (1 << 20) | (8 << HEIGHT),
               8 | (1 << 20), 10]:
        with pytest.raises(cn.CNError) as e:
            cn.cn_plan_layout(off, parent, mp)
        assert e.value.status == cn.CN_EINVAL


def test_plan_layout_rejects_bad_trees(cn):
    with pytest.raises(cn.CNError) as e:
        cn.cn_plan_layout(np.array([0, 3]), np.array([-1, 0, 2]), 0)
    assert e.value.status == cn.CN_EINVAL
    with pytest.raises(cn.CNError):
        cn.cn_plan_layout(np.array([0, 2]), np.array([0, -1]), 0)


@pytest.mark.parametrize("mapping", ["interleaved", "constdepth"])
@pytest.mark.parametrize("case", ["network", "morph_types", "ring16"])
def test_reference_layout_invariants(cn, case, mapping):
    """The reference placements keep what makes their sums follow a
    sequential per-cell stepper: every parent in an earlier row of the same
    warp; never two children of one node in one row; a node's children in
    rows that increase with their input index; at most one spike source
    (here each cell's root) per lane; one node per (warp, lane, row).
    Interleaved puts node i of each cell at row i of one lane."""
    from scenarios import morph_types
    sc = {"network": lambda: network(n_cells=70, tstop=1.0),
          "morph_types": lambda: morph_types(n_cells=96, cells_per_type=4, tstop=1.0),
          "ring16": lambda: ring16(tstop=1.0)}[case]()
    off, par = np.asarray(sc.cell_offset), np.asarray(sc.parent)
    code = cn.CN_MAP_INTERLEAVED if mapping == "interleaved" else cn.CN_MAP_CONSTDEPTH
    L = cn.cn_plan_layout(off, par, code)
    lane, row = L["lane"], L["row"]
    assert len(set(zip(lane.tolist(), row.tolist()))) == len(lane)
    roots = set()
    for c in range(len(off) - 1):
        i0, i1 = off[c], off[c + 1]
        w = lane[i0] // 32
        assert np.all(lane[i0:i1] // 32 == w)
        assert lane[i0] not in roots
        roots.add(lane[i0])
        kids = {}
        for i in range(i0 + 1, i1):
            p = i0 + par[i]
            assert row[p] < row[i]
            kids.setdefault(p, []).append(i)
        for p, ks in kids.items():
            rs = [row[i] for i in ks]                      # input order
            assert rs == sorted(rs) and len(set(rs)) == len(rs)
        if mapping == "interleaved":
            assert np.all(row[i0:i1] == np.arange(i1 - i0)) and np.all(lane[i0:i1] == lane[i0])
