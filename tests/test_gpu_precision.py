"""Reduced-precision gating against the FP64 oracle (accuracy report).

Gating rates, exponentials and state updates in FP32 (CN_PREC_GATE_FP32),
optionally with the gating states stored as bfloat16 (CN_PREC_GATE_BF16);
voltages, matrix assembly and the Hines solve stay FP64.  For each workload
the test prints the maximum and RMS soma-voltage error (mV), the fraction
of oracle spikes that the GPU run emits in the same step (and within one
step), and that fraction per 10 ms window (one displaced spike can cascade
through a recurrent network, so agreement is also shown over time).

The bar for FP32 gating is a maximum soma-voltage error of 0.1 mV and at
least 99.9% of the oracle's spikes in the same step.  Where a workload
misses it the test is marked xfail with the measured numbers in its reason
(it still fails outright if a spike moves by more than one step or the
spike count changes).  The BF16 variant is reported only.
"""
import numpy as np
import pytest

from scenarios import network, batched
from oracle import simulate

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


CASES = {
    # the plain network at full size (16,384 cells), first 20 ms
    "network": lambda: network(tstop=20.0),
    # the heterogeneous channel workload, 200 cells, 100 ms (spiking)
    "batched": lambda: batched(n_cells=200, tstop=100.0),
}
_refs = {}


def reference(name):
    if name not in _refs:
        sc = CASES[name]()
        _refs[name] = (sc, simulate(sc))
    return _refs[name]


def _agreement(g, k, rg, rk, tol):
    """Oracle spikes with a GPU spike of the same cell within tol steps."""
    gpu = {}
    for a, b in zip(g.tolist(), k.tolist()):
        gpu.setdefault(a, []).append(b)
    hit = 0
    for a, b in zip(rg.tolist(), rk.tolist()):
        if any(abs(b - x) <= tol for x in gpu.get(a, ())):
            hit += 1
    return hit


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["gate_fp32", "gate_bf16"])
def test_precision_report(cn, name, precision):
    sc, ref = reference(name)
    md = cn.from_scenario(sc, precision=precision)
    md.cn_run(sc.tstop)
    md.cn_sync()
    g, k = md.cn_get_spikes()
    tr = np.stack([md.cn_get_trace(r) for r in range(len(sc.rec_node))])
    rt = ref.traces()
    rg, rk = ref.spikes()
    err = np.abs(tr - rt)
    mx, rms = float(err.max()), float(np.sqrt(np.mean(err ** 2)))
    same, near = _agreement(g, k, rg, rk, 0), _agreement(g, k, rg, rk, 1)
    win = 400  # 10 ms
    windows = []
    for w0 in range(0, sc.nsteps, win):
        sel_r = (rk > w0) & (rk <= w0 + win)
        sel_g = (k > w0) & (k <= w0 + win)
        if sel_r.any():
            windows.append(f"{_agreement(g[sel_g], k[sel_g], rg[sel_r], rk[sel_r], 0)}/{int(sel_r.sum())}")
    print(f"\n[precision] {name} {precision}: max {mx:.3g} mV, rms {rms:.3g} mV, "
          f"spikes in the same step {same}/{len(rg)}, within one step {near}/{len(rg)} "
          f"(GPU emitted {len(g)}); same step per 10 ms window: {' '.join(windows) or '-'}")
    if name == "batched":
        assert len(rg) > 50
    if precision == "gate_fp32":
        # never more than one step off, nothing gained or lost
        assert len(g) == len(rg) and near == len(rg)
        if mx > 0.1 or same < 0.999 * len(rg):
            pytest.xfail(f"FP32 gating misses the bar on {name}: max soma error {mx:.3g} mV (bar 0.1), "
                         f"{same}/{len(rg)} spikes in the same step (bar 99.9%)")
