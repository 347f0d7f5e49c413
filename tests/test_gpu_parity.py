"""CUDA engine vs FP64 oracle, element by element, through the C ABI.

Bar (FP64 path): spike raster (gid, step) bit-exact; every voltage within
1e-9 mV of the oracle; gating states within 1e-9 (they are O(1)).
"""
import numpy as np
import pytest

from scenarios import ring16, network, adjoint_net, single_compartment, passive_cable, morph_types
from oracle import simulate

pytestmark = pytest.mark.gpu

V_TOL = 1e-9      # mV, FP64 path
GATE_TOL = 1e-9


@pytest.fixture(scope="module")
def cn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10975_gb300 import build
    build.build()
    from paper_1901_10975_gb300 import cn as _cn
    return _cn


def run_gpu(cn, sc, precision="fp64", tstop=None, chunks=None, **kw):
    md = cn.from_scenario(sc, precision=precision, **kw)
    tstop = sc.tstop if tstop is None else tstop
    if chunks:
        for t in chunks:
            md.cn_run(t)
    md.cn_run(tstop)
    md.cn_sync()
    g, k = md.cn_get_spikes()
    tr = np.stack([md.cn_get_trace(r) for r in range(len(sc.rec_node))]) if len(sc.rec_node) else None
    v = md.cn_get_v()
    out = {"g": g, "k": k, "tr": tr, "v": v, "model": md}
    hh = sc.mech("hh")
    if hh is not None and hh.n:
        out["hh"] = [md.cn_get_state("hh", c, hh.n) for c in range(3)]
    syn = sc.mech("expsyn")
    if syn is not None and syn.n:
        out["syn"] = md.cn_get_state("expsyn", 0, syn.n)
    return out


def run_oracle(sc, nsteps=None, nthreads=None):
    m = simulate(sc, nsteps=nsteps, nthreads=nthreads)
    g, k = m.spikes()
    out = {"g": g, "k": k, "tr": m.traces() if len(sc.rec_node) else None, "v": m.v()}
    hh = sc.mech("hh")
    if hh is not None and hh.n:
        out["hh"] = [m.state("hh", c) for c in range(3)]
    syn = sc.mech("expsyn")
    if syn is not None and syn.n:
        out["syn"] = m.state("expsyn", 0)
    return out


def assert_parity(gpu, ref, v_tol=V_TOL, gate_tol=GATE_TOL):
    assert np.array_equal(gpu["g"], ref["g"]) and np.array_equal(gpu["k"], ref["k"]), \
        (gpu["g"][:10], gpu["k"][:10], ref["g"][:10], ref["k"][:10])
    if ref["tr"] is not None:
        assert gpu["tr"].shape == ref["tr"].shape
        err = np.max(np.abs(gpu["tr"] - ref["tr"]))
        assert err <= v_tol, f"trace error {err}"
    err_v = np.max(np.abs(gpu["v"] - ref["v"]))
    assert err_v <= v_tol, f"voltage error {err_v}"
    if "hh" in ref:
        for c in range(3):
            assert np.max(np.abs(gpu["hh"][c] - ref["hh"][c])) <= gate_tol
    if "syn" in ref:
        assert np.max(np.abs(gpu["syn"] - ref["syn"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["syn"])))


def test_ring16_fp64(cn):
    """Ring of 16 (the Ring model's shape): raster bit-exact, v within 1e-9 mV."""
    sc = ring16()
    ref = run_oracle(sc, nthreads=1)
    gpu = run_gpu(cn, sc)
    assert len(ref["g"]) >= 5
    assert_parity(gpu, ref)


def test_ring16_strong_many_laps(cn):
    sc = ring16(weight=0.02, tstop=300.0)
    ref = run_oracle(sc, nthreads=1)
    gpu = run_gpu(cn, sc)
    assert len(ref["g"]) > 32
    assert_parity(gpu, ref)


def test_network_reduced_ragged(cn):
    """Network shape (200-600 compartments, 50 ExpSyn, 100 NetCons, 5 Hz
    background) cut to 500 cells (15 full warps and a ragged tail) x 50 ms."""
    sc = network(n_cells=500, tstop=50.0)
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc)
    assert_parity(gpu, ref)


def test_network_driven_spiking(cn):
    """Stronger synapses so that cells fire and NetCon events flow: exercises
    the interval exchange, delivery order and threshold detection."""
    sc = network(n_cells=300, tstop=60.0, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0)
    ref = run_oracle(sc)
    assert len(ref["g"]) > 50
    gpu = run_gpu(cn, sc)
    assert_parity(gpu, ref)


def test_network_full_size_short(cn):
    """All 16,384 cells of the network workload, 10 ms, in the benchmark's
    launch configuration (autotuned layout, graph replay): every soma trace
    and every node voltage against the oracle."""
    sc = network(tstop=10.0)
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc, mapping=cn.CN_MAP_TUNE)
    assert_parity(gpu, ref)


def test_network_full_length(cn):
    """The headline workload for its whole run: all 16,384 cells, 1,000 ms
    (40,000 steps), in the benchmark's launch configuration (autotuned
    layout, graph replay), against the threaded oracle: raster bit-exact
    (this input leaves the network subthreshold, so both are empty), every
    soma trace at every step and every node voltage at the end within
    1e-9 mV."""
    sc = network(tstop=1000.0)
    gpu = cn.from_scenario(sc, mapping=cn.CN_MAP_TUNE)
    gpu.cn_run(sc.tstop)
    gpu.cn_sync()
    g, k = gpu.cn_get_spikes()
    tr = gpu.cn_get_traces()                    # [probe][step]
    v = gpu.cn_get_v()
    ref = simulate(sc)
    rg, rk = ref.spikes()
    assert np.array_equal(g, rg) and np.array_equal(k, rk)
    assert tr.shape == (len(sc.rec_node), sc.nsteps + 1)
    worst = 0.0
    for r in range(len(sc.rec_node)):
        worst = max(worst, float(np.max(np.abs(tr[r] - ref.trace(r)))))
    err_v = float(np.max(np.abs(v - ref.v())))
    print(f"\n[full length] 16,384 cells x 1,000 ms: max trace error {worst:.3g} mV, node {err_v:.3g} mV")
    assert worst <= V_TOL and err_v <= V_TOL


def _layout(cn, name):
    return {"interleaved": cn.CN_MAP_INTERLEAVED, "constdepth": cn.CN_MAP_CONSTDEPTH}[name]


@pytest.mark.parametrize("layout", ["interleaved", "constdepth"])
def test_morph_types_full_size_short(cn, layout):
    """All 131,072 cells (10,878,976 compartments) of the morphological-types
    workload with every cell distinct, 10 ms (~19,000 HH spikes), in the
    paper's two node orderings (the reference layouts: the same operation
    order as the oracle, no fused multiply-adds): raster bit-exact, every
    trace and node voltage within 1e-9 mV."""
    sc = morph_types(cells_per_type=1, tstop=10.0)
    ref = _morph_ref(sc)
    assert len(ref["g"]) > 1000
    gpu = run_gpu(cn, sc, mapping=_layout(cn, layout))
    print(f"\n[{layout}] morph_types full size: max trace error "
          f"{np.max(np.abs(gpu['tr'] - ref['tr'])):.3g} mV, node {np.max(np.abs(gpu['v'] - ref['v'])):.3g} mV")
    assert_parity(gpu, ref)


_morph_cache = {}


def _morph_ref(sc):
    if "full" not in _morph_cache:
        _morph_cache["full"] = run_oracle(sc)
    return _morph_cache["full"]


def test_morph_types_fast_layout_report(cn):
    """The same full-size run in the fast layout (autotuned split cells,
    rows scaled by 1/cdt, v_{k+1} form, fused multiply-adds, the integer
    Newton reciprocal).  Raster bit-exact; the voltage error is reported
    over time beside the smallest distance |v - threshold| of any soma at
    the steps on either side of a crossing, which is how far a rounding
    difference would have to push a soma to move a spike by a step."""
    sc = morph_types(cells_per_type=1, tstop=10.0)
    ref = _morph_ref(sc)
    gpu = run_gpu(cn, sc, mapping=cn.CN_MAP_TUNE)
    assert np.array_equal(gpu["g"], ref["g"]) and np.array_equal(gpu["k"], ref["k"])
    err = np.abs(gpu["tr"] - ref["tr"])
    per_ms = [float(err[:, i * 40:(i + 1) * 40 + 1].max()) for i in range(10)]
    soma = ref["tr"]                       # one probe per cell, at the soma
    th = float(sc.threshold[0])
    margin = np.inf
    for g_, k_ in zip(ref["g"].tolist(), ref["k"].tolist()):
        margin = min(margin, abs(soma[g_, k_] - th), abs(soma[g_, k_ - 1] - th))
    print(f"\n[fast] morph_types full size: max trace error {err.max():.3g} mV "
          f"(per ms: {' '.join(f'{x:.1e}' for x in per_ms)}), node {np.max(np.abs(gpu['v'] - ref['v'])):.3g} mV; "
          f"smallest |v - threshold| at a crossing {margin:.3g} mV")
    assert margin > 1e3 * err.max()


@pytest.mark.parametrize("layout", ["interleaved", "constdepth"])
@pytest.mark.parametrize("case", ["ring16_laps", "driven", "reduced", "stim"])
def test_reference_layouts_match_oracle(cn, layout, case):
    """The reference layouts on the ring (many laps), a driven spiking
    network, the subthreshold network cut to 500 cells (a ragged warp) and
    current-clamped cells: raster bit-exact, voltages within 1e-9 mV (the
    operation order is the oracle's, so they agree up to exp()'s last bit)."""
    sc = {"ring16_laps": lambda: ring16(weight=0.02, tstop=300.0),
          "driven": lambda: network(n_cells=300, tstop=60.0, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0),
          "reduced": lambda: network(n_cells=500, tstop=20.0),
          "stim": lambda: adjoint_net(n_cells=70, tstop=30.0)}[case]()
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc, mapping=_layout(cn, layout))
    print(f"\n[{layout}] {case}: {len(ref['g'])} spikes, max trace error "
          f"{np.max(np.abs(gpu['tr'] - ref['tr'])):.3g} mV, node {np.max(np.abs(gpu['v'] - ref['v'])):.3g} mV")
    assert_parity(gpu, ref)


def test_reference_layouts_reject_unsupported_models(cn):
    """Channel types, gap junctions and reduced precision are fast-layout
    features: a reference layout refuses them with CN_EINVAL."""
    from scenarios import batched
    sc = batched(n_cells=8, tstop=1.0, n_in=2)
    for code in (cn.CN_MAP_INTERLEAVED, cn.CN_MAP_CONSTDEPTH):
        with pytest.raises(cn.CNError) as e:
            run_gpu(cn, sc, mapping=code)
        assert e.value.status == cn.CN_EINVAL
        with pytest.raises(cn.CNError) as e:
            run_gpu(cn, ring16(tstop=1.0), precision="gate_fp32", mapping=code)
        assert e.value.status == cn.CN_EINVAL


def test_partial_intervals_and_resume(cn):
    """cn_run to times that are not interval boundaries, then continue."""
    sc = network(n_cells=70, tstop=20.0, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0)
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc, chunks=[0.0, 0.3, 1.0, 1.525, 7.0, 13.3])
    assert_parity(gpu, ref)


def test_stimulus_and_single_compartment(cn):
    sc = single_compartment(mech="hh", tstop=30.0, stim_amp=0.3, stim_del=1.0, stim_dur=1.0)
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc)
    assert len(ref["g"]) == 1
    assert_parity(gpu, ref)


def test_adjoint_shape_forward(cn):
    """Clamp-driven unconnected cells (the adjoint workload's forward pass)."""
    sc = adjoint_net(n_cells=70, tstop=30.0)
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc)
    assert_parity(gpu, ref)


def test_passive_cable_long_chain(cn):
    """One 2,000-node unbranched cable (deep chain, one lane busy)."""
    sc = passive_cable(2000, L=4000.0, tstop=5.0)
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc)
    assert_parity(gpu, ref)


@pytest.mark.parametrize("prec,bound", [("gate_fp32", 0.1), ("gate_bf16", None)])
def test_reduced_precision_gating_error(cn, prec, bound):
    """FP32 gating (BF16 storage optional) against the FP64 oracle: report
    max soma-voltage error and spike agreement; FP32 must stay within 0.1 mV
    with every spike in the same step on the ring."""
    sc = ring16(weight=0.02, tstop=200.0)
    ref = run_oracle(sc, nthreads=1)
    gpu = run_gpu(cn, sc, precision=prec)
    err = np.max(np.abs(gpu["tr"] - ref["tr"]))
    same = len(set(zip(gpu["g"].tolist(), gpu["k"].tolist())) & set(zip(ref["g"].tolist(), ref["k"].tolist())))
    frac = same / max(1, len(ref["g"]))
    print(f"{prec}: max soma error {err:.3g} mV, spikes in the same step {same}/{len(ref['g'])}")
    if bound is not None:
        assert err <= bound and frac == 1.0 and len(gpu["g"]) == len(ref["g"])


def test_add_after_run_is_rejected(cn):
    sc = ring16(n_cells=4, tstop=2.0)
    md = cn.from_scenario(sc)
    md.cn_run(1.0)
    with pytest.raises(cn.CNError) as e:
        md.cn_add_stim(0, 0.0, 1.0, 0.1)
    assert e.value.status == cn.CN_ESTATE
    with pytest.raises(cn.CNError) as e:
        md.cn_run(0.5)
    assert e.value.status == cn.CN_EINVAL


def test_event_buffers_sized_for_every_delivery(cn):
    """Each lane's event buffer holds its busiest interval's external events
    plus ceil(D/2) per incoming NetCon (a source spikes at most every other
    step), so nothing is dropped however many events converge on one cell:
    5,000 events on one synapse inside one interval, and a cell driven by
    every NetCon of a strongly spiking network, match the oracle."""
    sc = ring16(n_cells=2, tstop=2.0)
    sc.netcon_src = sc.netcon_src[:0]; sc.netcon_syn = sc.netcon_syn[:0]
    sc.netcon_w = sc.netcon_w[:0]; sc.netcon_delay = sc.netcon_delay[:0]
    sc.ev_syn = np.zeros(5000, np.int32)
    sc.ev_t = np.linspace(0.3, 0.8, 5000)
    sc.ev_w = np.full(5000, 1e-6)
    assert_parity(run_gpu(cn, sc), run_oracle(sc, nthreads=1))
    sc = network(n_cells=64, tstop=30.0, w_median=0.05, bg_w=0.05, bg_rate_hz=60.0)
    sc.netcon_syn = np.where(np.arange(len(sc.netcon_syn)) % 2 == 0, 0, sc.netcon_syn).astype(np.int32)
    ref = run_oracle(sc)
    assert len(ref["g"]) > 100
    assert_parity(run_gpu(cn, sc), ref)


@pytest.mark.parametrize("mapping", [1, 40, 100, 16 | (1 << 20), 64 | (1 << 20), 40 | (3 << 20), 24 | (2 << 20),
                                     32 | (1 << 20) | (56 << 22), 16 | (1 << 20) | (24 << 22)])
def test_split_cells_over_lanes(cn, mapping):
    """The same driven network with one cell per lane (mapping 1) and with
    cells cut into parts of about 40 or 100 rows spread over lanes of one
    warp, in warps as tall as the opening cell or 1, 1.5 and 2 times the
    largest span, or of a given height (parts filling free runs below lane
    tops; cells cut finer, or in warps of their own, where they exceed it):
    the raster, voltages and states must match the oracle in every layout."""
    sc = network(n_cells=96, tstop=30.0, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0)
    ref = run_oracle(sc)
    assert len(ref["g"]) > 10
    assert_parity(run_gpu(cn, sc, mapping=mapping), ref)


def test_split_cells_batched_big(cn):
    """Cells of up to 5,000 compartments with channels everywhere, cut into
    parts of about 300 rows (up to 17 lanes per cell)."""
    from scenarios import batched
    sc = batched(n_cells=40, tstop=8.0, n_in=20)
    ref = run_oracle(sc)
    assert_parity(run_gpu(cn, sc, mapping=300), ref)


def _same(a, b):
    for key in ("g", "k", "v", "tr"):
        assert np.array_equal(a[key], b[key]), key


def test_graph_replay_matches_direct_launches(cn):
    """Whole intervals replayed from the captured graph (8 per chunk, the
    interval index kept on the device) give bit-identical results to one
    launch per interval, including a run that stops mid-interval."""
    sc = network(n_cells=200, tstop=41.3, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0)
    a = run_gpu(cn, sc, use_graph=False)
    b = run_gpu(cn, sc, use_graph=True)
    c = run_gpu(cn, sc, use_graph=True, chunks=[2.5, 11.0, 30.0])
    assert len(a["g"]) > 10
    _same(a, b)
    _same(a, c)


@pytest.mark.parametrize("wpb", [2, 4])
def test_warps_per_block_bit_identical(cn, wpb):
    """Several groups per block change only the launch shape: results are
    bit-identical to one warp per block."""
    sc = network(n_cells=300, tstop=20.0, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0)
    a = run_gpu(cn, sc, warps_per_block=1)
    b = run_gpu(cn, sc, warps_per_block=wpb)
    assert b["model"].cn_get_mapping()[1] == wpb
    _same(a, b)


def test_autotuned_mapping_parity(cn):
    """CN_MAP_TUNE times every candidate layout, keeps the fastest, starts
    from the initial state again: the run still matches the oracle."""
    sc = network(n_cells=96, tstop=30.0, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0)
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc, mapping=cn.CN_MAP_TUNE)
    mp, wpb, nw, ms = gpu["model"].cn_get_mapping()
    assert (mp == cn.CN_MAP_THREAD or mp >= 16) and 1 <= wpb <= 4 and nw >= 1 and ms > 0
    assert_parity(gpu, ref)


def test_profile_counts_graph_launches(cn):
    """Per-launch CUDA-event timing also covers graph-replayed intervals."""
    sc = network(n_cells=64, tstop=30.0)
    md = cn.from_scenario(sc, record=False)
    md.cn_profile(True)
    md.cn_run(27.0)
    k_ms, k_n, p_ms, p_n = md.cn_profile_read()
    assert k_n == 27 and p_n == 27 and k_ms > 0 and p_ms > 0
    md.cn_run(30.0)
    assert md.cn_profile_read()[1] == 3


@pytest.mark.parametrize("cpt", [1, 4, 32])
@pytest.mark.parametrize("mapping", [1, 0])
def test_morphological_types(cn, cpt, mapping):
    """Cells of 83 nodes with 1, 4 or 32 identical cells per branching type
    (rings of 16, HH soma): same raster and voltages as the oracle whether
    the 32 lanes of a warp hold identical or all different trees."""
    sc = morph_types(n_cells=160, cells_per_type=cpt, tstop=25.0)
    ref = run_oracle(sc)
    assert len(ref["g"]) > 20
    assert_parity(run_gpu(cn, sc, mapping=mapping), ref)


def _with_gaps(sc, g=0.0005, seed=5):
    """Adds symmetric gap junctions between random node pairs of different
    cells (one pair per cell: a node of cell i with a node of cell i+1)."""
    import dataclasses
    rng = np.random.default_rng(seed)
    off = np.asarray(sc.cell_offset)
    a, b = [], []
    for c in range(sc.n_cells - 1):
        a.append(off[c] + rng.integers(0, off[c + 1] - off[c]))
        b.append(off[c + 1] + rng.integers(0, off[c + 2] - off[c + 1]))
    a, b = np.array(a, np.int32), np.array(b, np.int32)
    return dataclasses.replace(sc, gap_node=np.concatenate([a, b]), gap_peer=np.concatenate([b, a]),
                               gap_g=np.full(2 * len(a), g))


@pytest.mark.parametrize("mapping", [1, 0, 16 | (1 << 20)])
def test_gap_junctions_against_oracle(cn, mapping):
    """Gap junctions between random node pairs of neighbouring cells of a
    driven network: the exchange interval drops to one step; raster and
    voltages must still match the oracle in every layout."""
    sc = _with_gaps(network(n_cells=64, tstop=20.0, w_median=0.03, bg_w=0.03, bg_rate_hz=30.0))
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc, mapping=mapping)
    assert len(ref["g"]) > 10
    assert_parity(gpu, ref)


def test_gap_pair_closed_form(cn):
    """The two-compartment junction of the oracle pins, on the GPU."""
    import importlib
    pins = importlib.import_module("test_oracle_pins")
    sc = pins.gap_pair()
    ref = run_oracle(sc)
    gpu = run_gpu(cn, sc)
    assert np.max(np.abs(gpu["tr"] - ref["tr"])) <= 1e-9
    assert np.max(np.abs(gpu["tr"][1] + 65.0)) > 0.1  # the junction moved the second cell


def test_bulk_trace_readback(cn):
    """cn_get_traces returns every probe's trace in one copy, equal to the
    per-probe reads."""
    sc = network(n_cells=40, tstop=5.0)
    md = cn.from_scenario(sc)
    md.cn_run(5.0)
    md.cn_sync()
    one = np.stack([md.cn_get_trace(r) for r in range(len(sc.rec_node))])
    assert np.array_equal(md.cn_get_traces(), one)
