"""Discrete adjoint on the GPU (cn_run_adjoint, CNTraceFn) against the CPU
oracle's adjoint and against central finite differences.

Loss: J = sum over cells and steps 1..K of (v_soma - v*_soma)^2 with targets
v* from the oracle run of the same cells with every conductance scaled by
(1 + 0.1 s), s = +-1 seeded.  Gradients with respect to per-cell gnabar,
gkbar and pas g.
"""
import copy

import numpy as np
import pytest

from scenarios import adjoint_net
from oracle import simulate, adjoint as oracle_adjoint

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


def perturbed(sc, seed=1905):
    rng = np.random.default_rng(seed)
    sp = copy.deepcopy(sc)
    hh, pas = sp.mech("hh"), sp.mech("pas")
    cell = sc.cell_of_node()
    s = rng.choice([-1.0, 1.0], size=(3, sc.n_cells))
    hh.params["gnabar"] = hh.params["gnabar"] * (1 + 0.1 * s[0][cell[hh.node]])
    hh.params["gkbar"] = hh.params["gkbar"] * (1 + 0.1 * s[1][cell[hh.node]])
    pas.params["g"] = pas.params["g"] * (1 + 0.1 * s[2][cell[pas.node]])
    return sp


def oracle_per_cell(sc, K, target, seg):
    J, gna, gk, gp = oracle_adjoint(sc, K, target, seg=seg)
    cell = sc.cell_of_node()
    out = np.zeros((3, sc.n_cells))
    np.add.at(out[0], cell[sc.mech("hh").node], gna)
    np.add.at(out[1], cell[sc.mech("hh").node], gk)
    np.add.at(out[2], cell[sc.mech("pas").node], gp)
    return J, out


def gpu_loss_and_grad(cn, md, K, target):
    md.cn_reset()
    md.cn_run(K * 0.025)
    tr = np.stack([md.cn_get_trace(r) for r in range(md.n_rec)])
    dj = 2.0 * (tr - target)
    dj[:, 0] = 0.0
    J = float(np.sum((tr[:, 1:] - target[:, 1:]) ** 2))
    return J, md.cn_run_adjoint(dj), tr


@pytest.mark.parametrize("n_cells,tstop,seg", [(70, 30.0, 200), (33, 12.0, 37)])
def test_adjoint_matches_oracle_adjoint(cn, n_cells, tstop, seg):
    sc = adjoint_net(n_cells=n_cells, tstop=tstop)
    K = sc.nsteps
    target = simulate(perturbed(sc)).traces()
    J_ref, g_ref = oracle_per_cell(sc, K, target, seg)
    md = cn.from_scenario(sc, record=True)
    md.cn_enable_adjoint(seg)
    J, g, _ = gpu_loss_and_grad(cn, md, K, target)
    assert abs(J - J_ref) <= 1e-9 * J_ref
    err = np.max(np.abs(g - g_ref) / (np.abs(g_ref) + 1e-6 * np.max(np.abs(g_ref), axis=1, keepdims=True)))
    assert err <= 1e-8, err


def test_adjoint_matches_central_differences(cn):
    """The loss is separable per cell, so one +-h perturbation of a parameter
    type in every cell at once gives every cell's finite difference."""
    sc = adjoint_net(n_cells=40, tstop=20.0)
    K = sc.nsteps
    target = simulate(perturbed(sc)).traces()
    md = cn.from_scenario(sc, record=True)
    md.cn_enable_adjoint(200)
    _, g, _ = gpu_loss_and_grad(cn, md, K, target)
    base = [md.cn_get_cell_param(p) for p in range(3)]

    def per_cell_loss():
        md.cn_reset()
        md.cn_run(K * 0.025)
        tr = np.stack([md.cn_get_trace(r) for r in range(md.n_rec)])
        return np.sum((tr[:, 1:] - target[:, 1:]) ** 2, axis=1)

    for p in range(3):
        h = 1e-6 * base[p]
        md.cn_set_cell_param(p, base[p] + h)
        lp = per_cell_loss()
        md.cn_set_cell_param(p, base[p] - h)
        lm = per_cell_loss()
        md.cn_set_cell_param(p, base[p])
        fd = (lp - lm) / (2 * h)
        rel = np.abs(fd - g[p]) / np.maximum(np.abs(g[p]), 1e-3 * np.max(np.abs(g[p])))
        assert np.max(rel) <= 1e-5, (p, np.max(rel))


def test_adjoint_preserves_state_and_params(cn):
    sc = adjoint_net(n_cells=8, tstop=5.0)
    md = cn.from_scenario(sc, record=True)
    md.cn_enable_adjoint(50)
    vals = np.linspace(0.1, 0.14, 8)
    md.cn_set_cell_param(0, vals)
    assert np.allclose(md.cn_get_cell_param(0), vals)
    md.cn_run(5.0)
    v_before = md.cn_get_v()
    md.cn_run_adjoint(np.ones((md.n_rec, sc.nsteps + 1)))
    assert np.array_equal(md.cn_get_v(), v_before)
    assert md.step == sc.nsteps


def test_autograd_function_matches_c_abi(cn):
    import torch
    from paper_1901_10975_gb300.autograd import CNTraceFn, trace_model
    sc = adjoint_net(n_cells=20, tstop=10.0)
    target = torch.from_numpy(simulate(perturbed(sc)).traces())
    md = trace_model(sc, checkpoint_ms=5.0)
    p = [torch.tensor(md.cn_get_cell_param(i), dtype=torch.float64, requires_grad=True) for i in range(3)]
    tr = CNTraceFn.apply(p[0], p[1], p[2], md, sc.tstop)
    loss = ((tr[:, 1:] - target[:, 1:]) ** 2).sum()
    loss.backward()
    J_ref, g_ref = oracle_per_cell(sc, sc.nsteps, target.numpy(), 200)
    assert abs(loss.item() - J_ref) <= 1e-9 * J_ref
    for i in range(3):
        assert np.allclose(p[i].grad.numpy(), g_ref[i], rtol=1e-8, atol=1e-8 * np.max(np.abs(g_ref[i])))


def test_adjoint_full_size_workload(cn):
    """1,024 cells of 100-300 compartments, 200 ms, somatic clamps, 5 ms
    checkpoints: GPU adjoint against the CPU adjoint."""
    sc = adjoint_net()
    K = sc.nsteps
    target = simulate(perturbed(sc)).traces()
    J_ref, g_ref = oracle_per_cell(sc, K, target, 200)
    md = cn.from_scenario(sc, record=True)
    md.cn_enable_adjoint(200)
    J, g, _ = gpu_loss_and_grad(cn, md, K, target)
    assert abs(J - J_ref) <= 1e-9 * J_ref
    err = np.max(np.abs(g - g_ref) / (np.abs(g_ref) + 1e-6 * np.max(np.abs(g_ref), axis=1, keepdims=True)))
    assert err <= 1e-8, err
