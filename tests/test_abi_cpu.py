"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every function declared in include/*.h; host validation rejects
bad models with CN_EINVAL; the geometry helper agrees with the oracle."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from scenarios import ring16, network, MECH_PARAMS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cn():
    from paper_1901_10975_gb300 import build
    build.build()
    from paper_1901_10975_gb300 import cn as _cn
    return _cn


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+(cn_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol(cn):
    names = declared_functions()
    assert len(names) >= 20
    L = C.CDLL(cn.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_mech_param_counts_match_generator(cn):
    for kind, cols in MECH_PARAMS.items():
        assert cn.lib().cn_mech_nparams(cn.MECH[kind]) == len(cols)
    assert cn.lib().cn_mech_nparams(99) == -1


def test_geometry_matches_oracle():
    from paper_1901_10975_gb300 import cn
    from oracle import OracleModel
    sc = network(n_cells=20, tstop=1.0)
    area, ri = cn.cn_geometry(sc.cell_offset, sc.parent, sc.dx, sc.diam, sc.Ra)
    ao, ro = OracleModel(sc).geometry()
    assert np.array_equal(area, ao) and np.array_equal(ri, ro)


def _create(cn, sc, **over):
    area, ri = cn.cn_geometry(sc.cell_offset, sc.parent, sc.dx, sc.diam, sc.Ra)
    kw = dict(cell_offset=sc.cell_offset, parent=sc.parent, area=area, cm=sc.cm, ri=ri,
              spike_node=sc.spike_node, threshold=sc.threshold,
              mechs=[(m.kind, m.node, m.param_matrix()) for m in sc.mechs])
    kw.update(over)
    return cn.Model(torch_alloc=False, **kw)


@pytest.mark.parametrize("case", ["parent_forward", "two_roots", "neg_area", "bad_spike_node",
                                  "mech_node_range", "dup_table", "bad_tau"])
def test_create_rejects_invalid_models(cn, case):
    sc = ring16(n_cells=3, tstop=1.0)
    over = {}
    if case == "parent_forward":
        p = sc.parent.copy(); p[5] = 7; over["parent"] = p
    elif case == "two_roots":
        p = sc.parent.copy(); p[3] = -1; over["parent"] = p
    elif case == "neg_area":
        area, ri = cn.cn_geometry(sc.cell_offset, sc.parent, sc.dx, sc.diam, sc.Ra)
        area[4] = -1.0; over["area"] = area
    elif case == "bad_spike_node":
        s = sc.spike_node.copy(); s[1] = 999; over["spike_node"] = s
    elif case == "mech_node_range":
        m = sc.mech("expsyn"); over["mechs"] = [("expsyn", np.array([0, 10**6, 2]), m.param_matrix())]
    elif case == "dup_table":
        m = sc.mech("pas"); over["mechs"] = [("pas", m.node, m.param_matrix())] * 2
    elif case == "bad_tau":
        m = sc.mech("expsyn"); pm = m.param_matrix().copy(); pm[0, 0] = 0.0
        over["mechs"] = [("expsyn", m.node, pm)]
    with pytest.raises(cn.CNError) as e:
        _create(cn, sc, **over)
    assert e.value.status == cn.CN_EINVAL
    assert len(str(e.value)) > len("CN_EINVAL: ")


def test_geometry_rejects_bad_input(cn):
    sc = ring16(n_cells=2, tstop=1.0)
    dx = sc.dx.copy(); dx[3] = 0.0
    with pytest.raises(cn.CNError):
        cn.cn_geometry(sc.cell_offset, sc.parent, dx, sc.diam, sc.Ra)
