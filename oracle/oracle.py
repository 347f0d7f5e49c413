"""ctypes wrapper of the FP64 CPU oracle (``cn_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use this module to compute expected results.  The CUDA
engine never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cn_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

KIND = {"pas": 0, "hh": 1, "expsyn": 2, "na3h": 3, "kdr4": 4, "ka": 5, "ih": 6, "cahva": 7, "kca": 8}

_P_I32 = C.POINTER(C.c_int32)
_P_I64 = C.POINTER(C.c_int64)
_P_F64 = C.POINTER(C.c_double)


class _MechIn(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("node", _P_I32), ("param", _P_F64)]


class _Scenario(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("v_init", C.c_double), ("n_cells", C.c_int32),
        ("cell_offset", _P_I32), ("parent", _P_I32), ("dx", _P_F64), ("diam", _P_F64),
        ("Ra", _P_F64), ("cm", _P_F64), ("spike_node", _P_I32), ("threshold", _P_F64),
        ("n_mech", C.c_int32), ("mechs", C.POINTER(_MechIn)),
        ("n_netcon", C.c_int64), ("nc_src", _P_I32), ("nc_syn", _P_I32), ("nc_w", _P_F64),
        ("nc_delay", _P_F64),
        ("n_ev", C.c_int64), ("ev_syn", _P_I32), ("ev_t", _P_F64), ("ev_w", _P_F64),
        ("n_stim", C.c_int32), ("stim_node", _P_I32), ("stim_del", _P_F64), ("stim_dur", _P_F64),
        ("stim_amp", _P_F64),
        ("n_rec", C.c_int32), ("rec_node", _P_I32),
        ("n_gap", C.c_int64), ("gap_node", _P_I32), ("gap_peer", _P_I32), ("gap_g", _P_F64),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain g++, no CUDA)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC", "-pthread",
           "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Scenario), C.c_char_p, C.c_int]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_run.argtypes = [C.c_void_p, C.c_int64, C.c_int]
        L.or_run.restype = C.c_int
        for f in ("or_step_index", "or_min_delay", "or_spike_count"):
            getattr(L, f).argtypes = [C.c_void_p]
            getattr(L, f).restype = C.c_int64
        L.or_get_spikes.argtypes = [C.c_void_p, _P_I32, _P_I64]
        L.or_get_trace.argtypes = [C.c_void_p, C.c_int32, _P_F64]
        L.or_get_v.argtypes = [C.c_void_p, _P_F64]
        L.or_get_cai.argtypes = [C.c_void_p, _P_F64]
        L.or_set_cai.argtypes = [C.c_void_p, _P_F64]
        L.or_get_state.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _P_F64]
        L.or_get_state.restype = C.c_int
        L.or_get_geometry.argtypes = [C.c_void_p, _P_F64, _P_F64]
        L.or_hines_solve.argtypes = [C.c_int32, _P_I32, _P_F64, _P_F64, _P_F64, _P_F64]
        L.or_adjoint.argtypes = [C.POINTER(_Scenario), C.c_int64, _P_F64, C.c_int32, C.c_int, _P_F64, _P_F64,
                                 _P_F64, _P_F64, C.c_char_p, C.c_int]
        L.or_adjoint.restype = C.c_int
        _lib = L
    return _lib


def _p(a, ty):
    return a.ctypes.data_as(ty)


def hines_solve(parent, a, b, d, rhs):
    """Solve one tree matrix with the oracle's Hines elimination."""
    parent = np.ascontiguousarray(parent, np.int32)
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    d = np.array(d, np.float64, copy=True)
    x = np.array(rhs, np.float64, copy=True)
    lib().or_hines_solve(len(parent), _p(parent, _P_I32), _p(a, _P_F64), _p(b, _P_F64),
                         _p(d, _P_F64), _p(x, _P_F64))
    return x


def _marshal(sc, keep):
    def i32(x):
        a = np.ascontiguousarray(x, np.int32)
        keep.append(a)
        return _p(a, _P_I32)

    def f64(x):
        a = np.ascontiguousarray(x, np.float64)
        keep.append(a)
        return _p(a, _P_F64)

    mechs = (_MechIn * max(1, len(sc.mechs)))()
    keep.append(mechs)
    for t, m in enumerate(sc.mechs):
        mechs[t].kind = KIND[m.kind]
        mechs[t].n = m.n
        mechs[t].node = i32(m.node)
        mechs[t].param = f64(m.param_matrix().reshape(-1))
    s = _Scenario()
    s.dt, s.v_init, s.n_cells = sc.dt, sc.v_init, sc.n_cells
    s.cell_offset, s.parent = i32(sc.cell_offset), i32(sc.parent)
    s.dx, s.diam, s.Ra, s.cm = f64(sc.dx), f64(sc.diam), f64(sc.Ra), f64(sc.cm)
    s.spike_node, s.threshold = i32(sc.spike_node), f64(sc.threshold)
    s.n_mech, s.mechs = len(sc.mechs), mechs
    s.n_netcon = len(sc.netcon_src)
    s.nc_src, s.nc_syn, s.nc_w, s.nc_delay = (i32(sc.netcon_src), i32(sc.netcon_syn),
                                              f64(sc.netcon_w), f64(sc.netcon_delay))
    s.n_ev = len(sc.ev_syn)
    s.ev_syn, s.ev_t, s.ev_w = i32(sc.ev_syn), f64(sc.ev_t), f64(sc.ev_w)
    s.n_stim = len(sc.stim_node)
    s.stim_node, s.stim_del, s.stim_dur, s.stim_amp = (i32(sc.stim_node), f64(sc.stim_del),
                                                       f64(sc.stim_dur), f64(sc.stim_amp))
    s.n_rec, s.rec_node = len(sc.rec_node), i32(sc.rec_node)
    s.n_gap = len(sc.gap_node)
    s.gap_node, s.gap_peer, s.gap_g = i32(sc.gap_node), i32(sc.gap_peer), f64(sc.gap_g)
    return s


def adjoint(sc, nsteps, target, seg=200, nthreads=None):
    """Oracle adjoint of J = sum over recorded nodes, steps 1..nsteps of
    (v - target)^2.  target: [n_rec, nsteps+1].  Returns (J, dJ/dgnabar per HH
    instance, dJ/dgkbar per HH instance, dJ/dg per pas instance)."""
    keep = []
    s = _marshal(sc, keep)
    tg = np.ascontiguousarray(target, np.float64)
    assert tg.shape == (len(sc.rec_node), nsteps + 1)
    nh = sc.mech("hh").n if sc.mech("hh") is not None else 0
    npas = sc.mech("pas").n if sc.mech("pas") is not None else 0
    gna, gk, gp = np.zeros(max(nh, 1)), np.zeros(max(nh, 1)), np.zeros(max(npas, 1))
    J = C.c_double()
    err = C.create_string_buffer(256)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib().or_adjoint(C.byref(s), int(nsteps), _p(tg, _P_F64), int(seg), int(nthreads), C.byref(J),
                          _p(gna, _P_F64), _p(gk, _P_F64), _p(gp, _P_F64), err, 256)
    if rc != 0:
        raise ValueError("oracle adjoint failed: " + err.value.decode())
    return J.value, gna[:nh], gk[:nh], gp[:npas]


class OracleModel:
    """A running oracle simulation of one Scenario."""

    def __init__(self, sc):
        L = lib()
        keep = []
        s = _marshal(sc, keep)
        err = C.create_string_buffer(512)
        h = L.or_create(C.byref(s), err, 512)
        if not h:
            raise ValueError("oracle rejected scenario: " + err.value.decode())
        self._h = h
        self.sc = sc
        self.n_rec = len(sc.rec_node)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def run(self, nsteps: int, nthreads: int | None = None):
        if nthreads is None:
            nthreads = os.cpu_count() or 1
        rc = lib().or_run(self._h, int(nsteps), int(nthreads))
        if rc != 0:
            raise RuntimeError("oracle run failed")
        return self

    @property
    def step(self) -> int:
        return int(lib().or_step_index(self._h))

    @property
    def min_delay(self) -> int:
        return int(lib().or_min_delay(self._h))

    def spikes(self):
        n = int(lib().or_spike_count(self._h))
        g = np.empty(n, np.int32)
        k = np.empty(n, np.int64)
        if n:
            lib().or_get_spikes(self._h, _p(g, _P_I32), _p(k, _P_I64))
        return g, k

    def trace(self, r: int) -> np.ndarray:
        out = np.empty(self.step + 1, np.float64)
        lib().or_get_trace(self._h, int(r), _p(out, _P_F64))
        return out

    def traces(self) -> np.ndarray:
        return np.stack([self.trace(r) for r in range(self.n_rec)]) if self.n_rec else np.zeros((0, self.step + 1))

    def v(self) -> np.ndarray:
        out = np.empty(self.sc.n_nodes, np.float64)
        lib().or_get_v(self._h, _p(out, _P_F64))
        return out

    def cai(self) -> np.ndarray:
        out = np.empty(self.sc.n_nodes, np.float64)
        lib().or_get_cai(self._h, _p(out, _P_F64))
        return out

    def set_cai(self, values) -> None:
        """Overwrite [Ca]i of every node (test perturbation)."""
        x = np.ascontiguousarray(np.broadcast_to(np.asarray(values, np.float64), (self.sc.n_nodes,)))
        lib().or_set_cai(self._h, _p(x, _P_F64))

    def state(self, kind: str, col: int) -> np.ndarray:
        m = self.sc.mech(kind)
        out = np.empty(m.n, np.float64)
        if lib().or_get_state(self._h, KIND[kind], int(col), _p(out, _P_F64)) != 0:
            raise ValueError(f"no state {kind}[{col}]")
        return out

    def geometry(self):
        area = np.empty(self.sc.n_nodes)
        ri = np.empty(self.sc.n_nodes)
        lib().or_get_geometry(self._h, _p(area, _P_F64), _p(ri, _P_F64))
        return area, ri


def simulate(sc, nsteps=None, nthreads=None) -> OracleModel:
    m = OracleModel(sc)
    m.run(sc.nsteps if nsteps is None else nsteps, nthreads)
    return m
