"""ctypes binding of the engine's C ABI (include/cn.h).

Argument marshalling only: every simulation step runs in the CUDA kernels of
``libcn.so``.  There is no CPU fallback; importing this module on a machine
without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcn.so")

CN_OK, CN_EINVAL, CN_ENOMEM, CN_ECUDA, CN_ESTATE, CN_ETIMEOUT, CN_ERANGE = range(7)
CN_PARAM_GNABAR, CN_PARAM_GKBAR, CN_PARAM_GPAS = range(3)
CN_MAP_AUTO, CN_MAP_THREAD, CN_MAP_TUNE, CN_MAP_INTERLEAVED, CN_MAP_CONSTDEPTH = range(5)
CN_MAP_TALL = 1 << 20
CN_MAP_TALL2 = 1 << 21
CN_MAP_HEIGHT_SHIFT = 22


def CN_MAP_HEIGHT(h):
    """Warp height field of a mapping value (with CN_MAP_TALL and a span)."""
    return int(h) << CN_MAP_HEIGHT_SHIFT
STATUS_NAMES = {0: "CN_OK", 1: "CN_EINVAL", 2: "CN_ENOMEM", 3: "CN_ECUDA", 4: "CN_ESTATE",
                5: "CN_ETIMEOUT", 6: "CN_ERANGE"}
MECH = {"pas": 0, "hh": 1, "expsyn": 2, "na3h": 3, "kdr4": 4, "ka": 5, "ih": 6, "cahva": 7, "kca": 8}
PRECISION = {"fp64": 0, "gate_fp32": 1, "gate_bf16": 2}

_P_I32 = C.POINTER(C.c_int32)
_P_I64 = C.POINTER(C.c_int64)
_P_F64 = C.POINTER(C.c_double)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class cn_morph(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("cell_offset", _P_I32), ("parent", _P_I32),
                ("area_um2", _P_F64), ("cm_uF_cm2", _P_F64), ("ri_MOhm", _P_F64),
                ("spike_node", _P_I32), ("threshold_mV", _P_F64)]


class cn_mech_table(C.Structure):
    _fields_ = [("type", C.c_int32), ("n", C.c_int32), ("node", _P_I32), ("param", _P_F64)]


class cn_options(C.Structure):
    _fields_ = [("dt_ms", C.c_double), ("v_init_mV", C.c_double), ("precision", C.c_int32),
                ("device", C.c_int32), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("mapping", C.c_int32), ("use_graph", C.c_int32),
                ("warps_per_block", C.c_int32)]


class CNError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libcn.so (built by ``paper_1901_10975_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA engine library not built: {LIB_PATH} (run paper_1901_10975_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        st = C.c_int
        L.cn_mech_nparams.argtypes = [C.c_int32]
        L.cn_mech_nparams.restype = C.c_int32
        L.cn_options_default.argtypes = [C.POINTER(cn_options)]
        L.cn_options_default.restype = None
        L.cn_geometry.argtypes = [C.c_int32, _P_I32, _P_I32, _P_F64, _P_F64, _P_F64, _P_F64, _P_F64]
        L.cn_geometry.restype = st
        L.cn_plan_layout.argtypes = [C.c_int32, _P_I32, _P_I32, C.c_int32, _P_I32, _P_I32, _P_I32, _P_I32, _P_I32]
        L.cn_plan_layout.restype = st
        L.cn_get_mapping.argtypes = [C.c_void_p, _P_I32, _P_I32, _P_I32, C.POINTER(C.c_float)]
        L.cn_get_mapping.restype = st
        L.cn_checkpoint_save.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
        L.cn_checkpoint_save.restype = st
        L.cn_checkpoint_load.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.cn_checkpoint_load.restype = st
        L.cn_add_gaps.argtypes = [C.c_void_p, C.c_int64, _P_I32, _P_I32, _P_F64]
        L.cn_add_gaps.restype = st
        L.cn_get_traces.argtypes = [C.c_void_p, _P_F64, C.c_size_t, C.POINTER(C.c_size_t)]
        L.cn_get_traces.restype = st
        L.cn_model_create.argtypes = [C.POINTER(cn_morph), C.POINTER(cn_mech_table), C.c_int32,
                                      C.POINTER(cn_options), C.POINTER(C.c_void_p)]
        L.cn_model_create.restype = st
        L.cn_add_netcon.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_double]
        L.cn_add_netcon.restype = st
        L.cn_add_netcons.argtypes = [C.c_void_p, C.c_int64, _P_I32, _P_I32, _P_F64, _P_F64]
        L.cn_add_netcons.restype = st
        L.cn_add_events.argtypes = [C.c_void_p, C.c_int64, _P_I32, _P_F64, _P_F64]
        L.cn_add_events.restype = st
        L.cn_add_stim.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_double]
        L.cn_add_stim.restype = st
        L.cn_record.argtypes = [C.c_void_p, C.c_int32, _P_I32]
        L.cn_record.restype = st
        L.cn_run.argtypes = [C.c_void_p, C.c_double]
        L.cn_run.restype = st
        L.cn_sync.argtypes = [C.c_void_p]
        L.cn_sync.restype = st
        L.cn_current_step.argtypes = [C.c_void_p]
        L.cn_current_step.restype = C.c_int64
        L.cn_updates.argtypes = [C.c_void_p]
        L.cn_updates.restype = C.c_int64
        L.cn_launch_count.argtypes = [C.c_void_p]
        L.cn_launch_count.restype = C.c_int64
        L.cn_get_spikes.argtypes = [C.c_void_p, _P_I32, _P_I64, C.c_size_t, C.POINTER(C.c_size_t)]
        L.cn_get_spikes.restype = st
        L.cn_get_trace.argtypes = [C.c_void_p, C.c_int32, _P_F64, C.c_size_t, C.POINTER(C.c_size_t)]
        L.cn_get_trace.restype = st
        L.cn_get_v.argtypes = [C.c_void_p, _P_F64, C.c_size_t]
        L.cn_get_v.restype = st
        L.cn_get_state.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _P_F64, C.c_size_t]
        L.cn_get_state.restype = st
        L.cn_reset.argtypes = [C.c_void_p]
        L.cn_reset.restype = st
        L.cn_set_cell_param.argtypes = [C.c_void_p, C.c_int32, _P_F64]
        L.cn_set_cell_param.restype = st
        L.cn_get_cell_param.argtypes = [C.c_void_p, C.c_int32, _P_F64]
        L.cn_get_cell_param.restype = st
        L.cn_enable_adjoint.argtypes = [C.c_void_p, C.c_int32]
        L.cn_enable_adjoint.restype = st
        L.cn_run_adjoint.argtypes = [C.c_void_p, _P_F64, _P_F64]
        L.cn_run_adjoint.restype = st
        L.cn_profile.argtypes = [C.c_void_p, C.c_int32]
        L.cn_profile.restype = st
        L.cn_profile_read.argtypes = [C.c_void_p, _P_F64, _P_I64, _P_F64, _P_I64]
        L.cn_profile_read.restype = st
        L.cn_solve_trees.argtypes = [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.cn_solve_trees.restype = st
        L.cn_solve_trees_noalloc.argtypes = list(L.cn_solve_trees.argtypes)
        L.cn_solve_trees_noalloc.restype = st
        L.cn_fp64_peak.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
        L.cn_fp64_peak.restype = st
        L.cn_pivot_reciprocal.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        L.cn_pivot_reciprocal.restype = st
        L.cn_last_error.argtypes = [C.c_void_p]
        L.cn_last_error.restype = C.c_char_p
        L.cn_model_destroy.argtypes = [C.c_void_p]
        L.cn_model_destroy.restype = None
        _lib = L
    return _lib


def _check(status, handle=None):
    if status != CN_OK:
        raise CNError(status, lib().cn_last_error(handle).decode())


def _i32(a):
    return np.ascontiguousarray(a, np.int32)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def _p(a, ty):
    return a.ctypes.data_as(ty)


def cn_geometry(cell_offset, parent, dx, diam, Ra):
    """area (um2) and ri (MOhm) per node from segment geometry."""
    off, par = _i32(cell_offset), _i32(parent)
    dx, diam, Ra = _f64(dx), _f64(diam), _f64(Ra)
    n = par.shape[0]
    area, ri = np.empty(n), np.empty(n)
    _check(lib().cn_geometry(len(off) - 1, _p(off, _P_I32), _p(par, _P_I32), _p(dx, _P_F64), _p(diam, _P_F64),
                             _p(Ra, _P_F64), _p(area, _P_F64), _p(ri, _P_F64)))
    return area, ri


def cn_plan_layout(cell_offset, parent, mapping=0):
    """Lane, warp row and topology flags of every node under `mapping` (host only)."""
    off, par = _i32(cell_offset), _i32(parent)
    n = par.shape[0]
    lane, row, flags = np.empty(n, np.int32), np.empty(n, np.int32), np.empty(n, np.int32)
    nw, depth = np.zeros(1, np.int32), np.zeros(1, np.int32)
    _check(lib().cn_plan_layout(len(off) - 1, _p(off, _P_I32), _p(par, _P_I32), int(mapping), _p(lane, _P_I32),
                                _p(row, _P_I32), _p(flags, _P_I32), _p(nw, _P_I32), _p(depth, _P_I32)))
    return {"lane": lane, "row": row, "flags": flags, "n_warps": int(nw[0]), "stack_depth": int(depth[0])}


def _device_tree_args(offset, parent, a, b, d, rhs, device):
    import torch
    dev = torch.device("cuda", device)
    t = dict(offset=torch.as_tensor(_i32(offset), device=dev), parent=torch.as_tensor(_i32(parent), device=dev),
             a=torch.as_tensor(_f64(a), device=dev), b=torch.as_tensor(_f64(b), device=dev),
             d=torch.as_tensor(_f64(d), device=dev), rhs=torch.as_tensor(_f64(rhs), device=dev))
    t["x"] = torch.empty_like(t["rhs"])
    return t


def cn_solve_trees(offset, parent, a, b, d, rhs, device=0):
    """Solve concatenated tree systems on the GPU; host arrays in, host array out."""
    import torch
    t = _device_tree_args(offset, parent, a, b, d, rhs, device)
    stream = torch.cuda.current_stream(device).cuda_stream
    n_trees = t["offset"].numel() - 1
    st = lib().cn_solve_trees(n_trees, t["rhs"].numel(), t["offset"].data_ptr(), t["parent"].data_ptr(),
                              t["a"].data_ptr(), t["b"].data_ptr(), t["d"].data_ptr(), t["rhs"].data_ptr(),
                              t["x"].data_ptr(), stream)
    if st != CN_OK:
        raise CNError(st, "cn_solve_trees failed")
    return t["x"].cpu().numpy()


def cn_pivot_reciprocal(d, device=0):
    """The interval kernel's pivot reciprocal of every value of d (host array
    in, host array out)."""
    import torch
    x = torch.from_numpy(_f64(d)).to(f"cuda:{device}")
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream(device).cuda_stream
    st = lib().cn_pivot_reciprocal(x.numel(), x.data_ptr(), out.data_ptr(), stream)
    if st != CN_OK:
        raise CNError(st, "cn_pivot_reciprocal failed")
    return out.cpu().numpy()


def cn_solve_trees_noalloc(offset, parent, a, b, d, rhs, device=0):
    """cn_solve_trees through the allocation-free entry point (the library's
    fixed scratch array instead of a per-call allocation)."""
    import torch
    t = _device_tree_args(offset, parent, a, b, d, rhs, device)
    stream = torch.cuda.current_stream(device).cuda_stream
    n_trees = t["offset"].numel() - 1
    st = lib().cn_solve_trees_noalloc(n_trees, t["rhs"].numel(), t["offset"].data_ptr(), t["parent"].data_ptr(),
                                      t["a"].data_ptr(), t["b"].data_ptr(), t["d"].data_ptr(),
                                      t["rhs"].data_ptr(), t["x"].data_ptr(), stream)
    if st != CN_OK:
        raise CNError(st, "cn_solve_trees_noalloc failed")
    return t["x"].cpu().numpy()


def _torch_allocator(device):
    """Device allocator callbacks routing through PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device)
        except Exception:
            return None

    def _free(ptr, ctx):
        if ptr:
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

    return ALLOC_FN(_alloc), FREE_FN(_free)


class Model:
    """Owner of one ``cn_model`` handle; methods map 1:1 onto the C ABI."""

    def __init__(self, cell_offset, parent, area, cm, ri, spike_node, threshold, mechs,
                 dt=0.025, v_init=-65.0, precision="fp64", device=0, stream=None,
                 torch_alloc=True, use_graph=True, mapping=0, warps_per_block=0):
        L = lib()
        self._keep = []
        k = self._keep
        off, par = _i32(cell_offset), _i32(parent)
        area, cm, ri = _f64(area), _f64(cm), _f64(ri)
        sn, th = _i32(spike_node), _f64(threshold)
        k += [off, par, area, cm, ri, sn, th]
        morph = cn_morph(len(off) - 1, _p(off, _P_I32), _p(par, _P_I32), _p(area, _P_F64), _p(cm, _P_F64),
                         _p(ri, _P_F64), _p(sn, _P_I32), _p(th, _P_F64))
        tabs = (cn_mech_table * max(1, len(mechs)))()
        for i, (kind, node, params) in enumerate(mechs):
            node = _i32(node)
            params = _f64(params).reshape(-1)
            k += [node, params]
            tabs[i] = cn_mech_table(MECH[kind], node.shape[0], _p(node, _P_I32), _p(params, _P_F64))
        opt = cn_options()
        L.cn_options_default(C.byref(opt))
        opt.dt_ms, opt.v_init_mV = float(dt), float(v_init)
        opt.precision = PRECISION[precision]
        opt.device = int(device)
        opt.use_graph = int(bool(use_graph))
        opt.mapping = int(mapping)
        opt.warps_per_block = int(warps_per_block)
        if stream is not None:
            opt.stream = int(stream)
        if torch_alloc:
            self._alloc_cbs = _torch_allocator(device)
            opt.alloc, opt.free = self._alloc_cbs
        h = C.c_void_p()
        _check(L.cn_model_create(C.byref(morph), tabs, len(mechs), C.byref(opt), C.byref(h)))
        self._h = h
        self.n_nodes = int(par.shape[0])
        self.n_cells = int(off.shape[0] - 1)
        self.dt = float(dt)
        self.n_rec = 0

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().cn_model_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    # -- inputs
    def cn_add_netcons(self, src, syn, w, delay):
        src, syn, w, delay = _i32(src), _i32(syn), _f64(w), _f64(delay)
        _check(lib().cn_add_netcons(self._h, src.shape[0], _p(src, _P_I32), _p(syn, _P_I32), _p(w, _P_F64),
                                    _p(delay, _P_F64)), self._h)

    def cn_add_events(self, syn, t, w):
        syn, t, w = _i32(syn), _f64(t), _f64(w)
        _check(lib().cn_add_events(self._h, syn.shape[0], _p(syn, _P_I32), _p(t, _P_F64), _p(w, _P_F64)), self._h)

    def cn_add_stim(self, node, delay, dur, amp):
        _check(lib().cn_add_stim(self._h, int(node), float(delay), float(dur), float(amp)), self._h)

    def cn_add_gaps(self, node, peer, g_uS):
        node, peer, g = _i32(node), _i32(peer), _f64(g_uS)
        _check(lib().cn_add_gaps(self._h, node.shape[0], _p(node, _P_I32), _p(peer, _P_I32), _p(g, _P_F64)),
               self._h)

    def cn_record(self, node) -> int:
        rid = C.c_int32()
        _check(lib().cn_record(self._h, int(node), C.byref(rid)), self._h)
        self.n_rec = max(self.n_rec, rid.value + 1)
        return rid.value

    # -- running
    def cn_run(self, tstop):
        _check(lib().cn_run(self._h, float(tstop)), self._h)

    def cn_sync(self):
        _check(lib().cn_sync(self._h), self._h)

    @property
    def step(self) -> int:
        return int(lib().cn_current_step(self._h))

    @property
    def updates(self) -> int:
        return int(lib().cn_updates(self._h))

    @property
    def launches(self) -> int:
        return int(lib().cn_launch_count(self._h))

    def cn_reset(self):
        _check(lib().cn_reset(self._h), self._h)

    def cn_set_cell_param(self, param, values):
        v = _f64(values)
        assert v.shape == (self.n_cells,)
        _check(lib().cn_set_cell_param(self._h, int(param), _p(v, _P_F64)), self._h)

    def cn_get_cell_param(self, param):
        out = np.empty(self.n_cells)
        _check(lib().cn_get_cell_param(self._h, int(param), _p(out, _P_F64)), self._h)
        return out

    def cn_enable_adjoint(self, checkpoint_steps):
        _check(lib().cn_enable_adjoint(self._h, int(checkpoint_steps)), self._h)

    def cn_run_adjoint(self, dj_dtrace):
        """dj_dtrace: [n_rec, K+1]; returns the gradient [3, n_cells]."""
        dj = _f64(dj_dtrace)
        out = np.empty((3, self.n_cells))
        _check(lib().cn_run_adjoint(self._h, _p(dj, _P_F64), _p(out, _P_F64)), self._h)
        return out

    def cn_profile(self, enable=True):
        _check(lib().cn_profile(self._h, int(bool(enable))), self._h)

    def cn_checkpoint_save(self) -> bytes:
        """The network state at the current (interval-boundary) step."""
        n = C.c_size_t(0)
        _check(lib().cn_checkpoint_save(self._h, None, 0, C.byref(n)), self._h)
        buf = C.create_string_buffer(n.value)
        _check(lib().cn_checkpoint_save(self._h, buf, n.value, C.byref(n)), self._h)
        return buf.raw[:n.value]

    def cn_checkpoint_load(self, data: bytes):
        _check(lib().cn_checkpoint_load(self._h, data, len(data)), self._h)

    def cn_get_mapping(self):
        """(mapping, warps per block, warps, autotuner's interval ms) of the layout in use."""
        mp, w, nw = np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32)
        ms = C.c_float(0.0)
        _check(lib().cn_get_mapping(self._h, _p(mp, _P_I32), _p(w, _P_I32), _p(nw, _P_I32), C.byref(ms)), self._h)
        return int(mp[0]), int(w[0]), int(nw[0]), float(ms.value)

    def fp64_peak(self) -> float:
        """FP64 TFLOP/s attained by a stream of independent FMAs on this GPU."""
        x = C.c_double()
        _check(lib().cn_fp64_peak(self._h, C.byref(x)), self._h)
        return x.value

    def cn_profile_read(self):
        """(interval-kernel ms, launches, pull-kernel ms, launches) since the last read."""
        a, b, c, d = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
        _check(lib().cn_profile_read(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), self._h)
        return a.value, b.value, c.value, d.value

    # -- outputs
    def cn_get_spikes(self):
        n = C.c_size_t()
        _check(lib().cn_get_spikes(self._h, None, None, 0, C.byref(n)), self._h)
        g = np.empty(n.value, np.int32)
        k = np.empty(n.value, np.int64)
        if n.value:
            _check(lib().cn_get_spikes(self._h, _p(g, _P_I32), _p(k, _P_I64), n.value, C.byref(n)), self._h)
        return g, k

    def cn_get_traces(self) -> np.ndarray:
        """All recorded traces, [n_rec, steps + 1] (one device-to-host copy)."""
        n = C.c_size_t(0)
        _check(lib().cn_get_traces(self._h, None, 0, C.byref(n)), self._h)
        nr = self.n_rec
        out = np.empty(n.value, np.float64)
        _check(lib().cn_get_traces(self._h, _p(out, _P_F64), n.value, C.byref(n)), self._h)
        return out.reshape(-1, nr).T if nr else np.zeros((0, self.step + 1))  # a view, no copy

    def cn_get_trace(self, rec_id):
        n = C.c_size_t()
        _check(lib().cn_get_trace(self._h, int(rec_id), None, 0, C.byref(n)), self._h)
        out = np.empty(n.value)
        _check(lib().cn_get_trace(self._h, int(rec_id), _p(out, _P_F64), n.value, C.byref(n)), self._h)
        return out

    def cn_get_v(self):
        out = np.empty(self.n_nodes)
        _check(lib().cn_get_v(self._h, _p(out, _P_F64), out.shape[0]), self._h)
        return out

    def cn_get_state(self, kind, col, n):
        out = np.empty(int(n))
        _check(lib().cn_get_state(self._h, MECH[kind], int(col), _p(out, _P_F64), out.shape[0]), self._h)
        return out


def from_scenario(sc, precision="fp64", device=0, stream=None, record=True, torch_alloc=True,
                  use_graph=True, mapping=0, warps_per_block=0) -> Model:
    """Build a Model from a scenarios.Scenario through the C ABI calls."""
    area, ri = cn_geometry(sc.cell_offset, sc.parent, sc.dx, sc.diam, sc.Ra)
    mechs = [(m.kind, m.node, m.param_matrix()) for m in sc.mechs if m.n > 0]
    md = Model(sc.cell_offset, sc.parent, area, sc.cm, ri, sc.spike_node, sc.threshold, mechs,
               dt=sc.dt, v_init=sc.v_init, precision=precision, device=device, stream=stream,
               torch_alloc=torch_alloc, use_graph=use_graph, mapping=mapping, warps_per_block=warps_per_block)
    if len(sc.netcon_src):
        md.cn_add_netcons(sc.netcon_src, sc.netcon_syn, sc.netcon_w, sc.netcon_delay)
    if len(sc.ev_syn):
        md.cn_add_events(sc.ev_syn, sc.ev_t, sc.ev_w)
    for i in range(len(sc.stim_node)):
        md.cn_add_stim(sc.stim_node[i], sc.stim_del[i], sc.stim_dur[i], sc.stim_amp[i])
    gap_node = getattr(sc, "gap_node", ())
    if len(gap_node):
        md.cn_add_gaps(gap_node, sc.gap_peer, sc.gap_g)
    if record:
        for node in sc.rec_node:
            md.cn_record(int(node))
    return md
