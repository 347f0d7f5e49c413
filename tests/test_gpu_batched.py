"""Heterogeneous batched workload (sizes 50-5000, random channel subsets on
every node, synapses and network as the plain network) on the GPU against
the FP64 oracle, and the FP32/BF16-gating variants' accuracy report."""
import numpy as np
import pytest

from scenarios import batched
from oracle import simulate

pytestmark = pytest.mark.gpu

CHANNELS = {"na3h": 2, "kdr4": 1, "ka": 2, "ih": 1, "cahva": 2, "kca": 1}


@pytest.fixture(scope="module")
def cn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_10975_gb300 import build
    build.build()
    from paper_1901_10975_gb300 import cn as _cn
    return _cn


@pytest.fixture(scope="module")
def case():
    sc = batched(n_cells=150, tstop=25.0)
    ref = simulate(sc)
    return sc, ref


def run(cn, sc, precision):
    md = cn.from_scenario(sc, precision=precision)
    md.cn_run(sc.tstop)
    md.cn_sync()
    g, k = md.cn_get_spikes()
    tr = np.stack([md.cn_get_trace(r) for r in range(len(sc.rec_node))])
    return md, g, k, tr


def test_batched_fp64_parity(cn, case):
    sc, ref = case
    md, g, k, tr = run(cn, sc, "fp64")
    rg, rk = ref.spikes()
    assert len(rg) > 20
    assert np.array_equal(g, rg) and np.array_equal(k, rk)
    assert np.max(np.abs(tr - ref.traces())) <= 1e-9
    assert np.max(np.abs(md.cn_get_v() - ref.v())) <= 1e-9
    for kind, ng in CHANNELS.items():
        n = sc.mech(kind).n
        for c in range(ng):
            assert np.max(np.abs(md.cn_get_state(kind, c, n) - ref.state(kind, c))) <= 1e-9, (kind, c)
    cai = md.cn_get_state("cahva", 2, sc.mech("cahva").n)
    assert np.max(np.abs(cai - ref.cai()[sc.mech("cahva").node])) <= 1e-12


@pytest.mark.parametrize("precision", ["gate_fp32", "gate_bf16"])
def test_batched_reduced_precision_report(cn, case, precision):
    """Gating in FP32 (BF16 storage optional), voltage and solve in FP64:
    max/RMS soma-voltage error and spikes in the same step as the FP64
    oracle, printed.  The FP32 bar is 0.1 mV and 99.9% of spikes in the same
    step; a miss is an xfail that states the measured numbers."""
    sc, ref = case
    _, g, k, tr = run(cn, sc, precision)
    rt = ref.traces()
    rg, rk = ref.spikes()
    err = np.abs(tr - rt)
    same = len(set(zip(g.tolist(), k.tolist())) & set(zip(rg.tolist(), rk.tolist())))
    print(f"{precision}: max {err.max():.3g} mV, rms {np.sqrt(np.mean(err ** 2)):.3g} mV, "
          f"spikes same step {same}/{len(rg)} (gpu {len(g)})")
    if precision == "gate_fp32" and (err.max() > 0.1 or same < 0.999 * len(rg)):
        pytest.xfail(f"FP32 gating misses the bar: max soma error {err.max():.3g} mV (bar 0.1), "
                     f"{same}/{len(rg)} spikes in the same step (bar 99.9%)")


def _one_node(kind, gbar, v_init, pas_g, pas_e, tstop):
    from scenarios import single_compartment, MechTable, MECH_PARAMS
    from scenarios.generator import _NOMINAL_GATES, _EREV
    sc = single_compartment(mech="pas", tstop=tstop, v_init=v_init, pas_g=pas_g, pas_e=pas_e)
    p = {"gbar": gbar, "erev": _EREV[kind]}
    for (t, gate), nom in _NOMINAL_GATES.items():
        if t == kind:
            for name, val in zip(["A", "vh", "k", "B", "vh2", "k2"], nom):
                p[f"{gate}_{name}"] = val
    if kind == "cahva":
        p.update(depth=0.1, taur=80.0, cainf=5e-5)
    if kind == "kca":
        p.update(A=0.01, kd=1e-3, B=0.02)
    sc.mechs.append(MechTable(kind, np.array([0], np.int32), {k: np.array([p[k]]) for k in MECH_PARAMS[kind]}))
    return sc


@pytest.mark.parametrize("kind", sorted(CHANNELS))
def test_single_channel_type_against_oracle(cn, kind):
    """Each channel type alone in one compartment (40 steps, depolarized
    start): voltage, gates and calcium against the oracle."""
    sc = _one_node(kind, 0.01, -40.0, 1e-4, -70.0, 1.0)
    ref = simulate(sc, nthreads=1)
    md = cn.from_scenario(sc)
    md.cn_run(sc.tstop)
    md.cn_sync()
    tr = md.cn_get_trace(0)
    assert np.max(np.abs(tr - ref.trace(0))) <= 1e-9, (tr[:4], ref.trace(0)[:4])
    for c in range(CHANNELS[kind]):
        assert abs(md.cn_get_state(kind, c, 1)[0] - ref.state(kind, c)[0]) <= 1e-9


def test_batched_full_size_short(cn):
    """All 50,000 cells (27.8 M compartments) of the heterogeneous workload,
    FP64, 2 ms, autotuned layout: raster, soma traces and every node voltage
    against the oracle."""
    sc = batched(tstop=2.0)
    ref = simulate(sc)
    md = cn.from_scenario(sc, mapping=cn.CN_MAP_TUNE)
    md.cn_run(sc.tstop)
    md.cn_sync()
    g, k = md.cn_get_spikes()
    rg, rk = ref.spikes()
    assert np.array_equal(g, rg) and np.array_equal(k, rk)
    assert np.max(np.abs(md.cn_get_traces() - ref.traces())) <= 1e-9
    assert np.max(np.abs(md.cn_get_v() - ref.v())) <= 1e-9
