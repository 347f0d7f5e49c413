"""Pins of the FP64 CPU oracle against results fixed by mathematics, not by
the oracle itself: a dense LU solver, backward-Euler closed forms, sealed
cable theory, the Hodgkin-Huxley equilibrium, an independent RK4 integration
and the composition of isolated-cell latencies around the ring."""
import itertools
import math

import numpy as np
import pytest

from scenarios import (passive_cable, ring16, single_compartment, network, MechTable)
from scenarios.generator import HH_SOMA
from oracle import simulate, hines_solve, OracleModel


# ---------------------------------------------------------------- Hines solve
def _all_parent_arrays(n):
    """Every rooted tree on n nodes numbered so that parent[i] < i."""
    ranges = [range(i) for i in range(1, n)]
    for tail in itertools.product(*ranges):
        yield np.array((-1,) + tail, np.int32)


def _dense(parent, a, b, d):
    n = len(parent)
    M = np.zeros((n, n))
    for i in range(n):
        M[i, i] = d[i]
        if parent[i] >= 0:
            M[i, parent[i]] = b[i]
            M[parent[i], i] = a[i]
    return M


def _random_system(rng, parent):
    n = len(parent)
    a = np.where(parent >= 0, -rng.uniform(0.1, 5.0, n), 0.0)
    b = np.where(parent >= 0, -rng.uniform(0.1, 5.0, n), 0.0)
    d = rng.uniform(0.05, 1.0, n)            # capacitive + membrane part
    for i in range(1, n):                    # plus the axial sums (dominance)
        d[i] -= b[i]
        d[parent[i]] -= a[i]
    return a, b, d, rng.normal(size=n)


def test_hines_matches_dense_lu_on_every_small_tree():
    """Gaussian elimination in Hines order (Section 2, Hines 1984) equals
    LU with partial pivoting for all 873 rooted trees of 1..7 nodes."""
    rng = np.random.default_rng(7)
    count = 0
    for n in range(1, 8):
        for parent in _all_parent_arrays(n):
            a, b, d, r = _random_system(rng, parent)
            x = hines_solve(parent, a, b, d, r)
            ref = np.linalg.solve(_dense(parent, a, b, d), r)
            assert np.max(np.abs(x - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
            count += 1
    assert count == sum(math.factorial(n - 1) for n in range(1, 8))


def test_hines_matches_dense_lu_on_random_trees():
    rng = np.random.default_rng(11)
    for _ in range(200):
        n = int(rng.integers(8, 65))
        parent = np.array([-1] + [int(rng.integers(0, i)) for i in range(1, n)], np.int32)
        a, b, d, r = _random_system(rng, parent)
        x = hines_solve(parent, a, b, d, r)
        ref = np.linalg.solve(_dense(parent, a, b, d), r)
        assert np.max(np.abs(x - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_hines_arithmetic_count_independent_of_branching():
    """Section 4.4: elimination costs the same for every branching pattern of
    a given size; a chain and a star of n nodes give the same dense result."""
    rng = np.random.default_rng(3)
    n = 40
    for parent in (np.arange(-1, n - 1, dtype=np.int32), np.array([-1] + [0] * (n - 1), np.int32)):
        a, b, d, r = _random_system(rng, parent)
        x = hines_solve(parent, a, b, d, r)
        assert np.allclose(x, np.linalg.solve(_dense(parent, a, b, d), r), rtol=0, atol=1e-12)


# ----------------------------------------------------- passive closed forms
def test_isopotential_backward_euler_closed_form():
    """One passive compartment: v_n - e = (v_0 - e) (1 + dt/tau)^-n exactly,
    tau = cm/g = 1 ms for g = 1e-3 S/cm2, cm = 1 uF/cm2."""
    sc = single_compartment(mech="pas", tstop=10.0, v_init=-40.0, pas_g=1e-3, pas_e=-65.0)
    m = simulate(sc, nthreads=1)
    tr = m.trace(0)
    n = np.arange(tr.shape[0])
    ref = -65.0 + 25.0 * (1.0 + 0.025 / 1.0) ** (-n)
    assert np.max(np.abs(tr - ref)) < 1e-12


def test_sealed_tree_uniform_offset_decays_like_one_compartment():
    """A uniform offset on a sealed passive tree (uniform g, cm) has no axial
    current, so every node follows the isopotential closed form."""
    sc = ring16(n_cells=3, tstop=5.0)
    nn = sc.n_nodes
    sc.mechs = [MechTable("pas", np.arange(nn, dtype=np.int32),
                          {"g": np.full(nn, 1e-3), "e": np.full(nn, -65.0)})]
    sc.netcon_src = sc.netcon_src[:0]; sc.netcon_syn = sc.netcon_syn[:0]
    sc.netcon_w = sc.netcon_w[:0]; sc.netcon_delay = sc.netcon_delay[:0]
    sc.ev_syn = sc.ev_syn[:0]; sc.ev_t = sc.ev_t[:0]; sc.ev_w = sc.ev_w[:0]
    sc.v_init = -30.0
    sc.rec_node = np.arange(nn, dtype=np.int32)
    m = simulate(sc, nthreads=1)
    tr = m.traces()
    n = np.arange(tr.shape[1])
    ref = -65.0 + 35.0 * 1.025 ** (-n)
    assert np.max(np.abs(tr - ref[None, :])) < 1e-11


def _cable_steady(nseg, L=500.0, diam=1.0, Ra=100.0, g=1e-3, amp=0.1):
    sc = passive_cable(nseg, L=L, diam=diam, Ra=Ra, g=g, amp=amp, tstop=60.0)
    m = simulate(sc, nthreads=1)
    return sc, m.v()


def _cable_theory(x_um, L=500.0, diam=1.0, Ra=100.0, g=1e-3, amp=0.1):
    """Sealed finite cable, steady current I at x = 0 (cable theory):
    lambda = sqrt(d Rm / (4 Ra)), r_a = 4 Ra / (pi d^2),
    V(x) = I r_a lambda cosh((L - x)/lambda) / sinh(L/lambda)."""
    d_cm = diam * 1e-4
    L_cm = L * 1e-4
    Rm = 1.0 / g                              # ohm cm2
    lam = math.sqrt(d_cm * Rm / (4.0 * Ra))   # cm
    r_a = 4.0 * Ra / (math.pi * d_cm ** 2)    # ohm / cm
    I = amp * 1e-9                            # A
    x = np.asarray(x_um) * 1e-4
    V = I * r_a * lam * np.cosh((L_cm - x) / lam) / np.sinh(L_cm / lam)
    return V * 1e3                            # mV


def test_sealed_cable_matches_cable_theory_second_order():
    """Steady-state attenuation and input resistance of a sealed cable
    converge to the closed form with error O(dx^2): doubling nseg cuts the
    error by ~4."""
    errs = []
    for nseg in (25, 50, 100, 200):
        sc, v = _cable_steady(nseg)
        dx = 500.0 / nseg
        x = (np.arange(nseg) + 0.5) * dx
        V = v - (-65.0)
        ref = _cable_theory(x)
        errs.append(np.max(np.abs(V - ref)) / np.max(np.abs(ref)))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-4
    for r in ratios:
        assert 3.5 < r < 4.5, (errs, ratios)


def test_cable_charge_conservation():
    """At steady state the injected current equals the total membrane
    current: axial terms only move charge between nodes."""
    sc, v = _cable_steady(100)
    area = math.pi * 1.0 * (500.0 / 100)      # um2 per segment
    membrane_nA = np.sum(1e-3 * (v + 65.0) * area * 1e-8) * 1e6  # S/cm2*mV*cm2 -> nA
    assert abs(membrane_nA - 0.1) < 1e-9


# --------------------------------------------------------- Hodgkin-Huxley
def _hh_inf(v):
    def vtrap(A, vh, k):
        u = (v - vh) / k
        return A * k * (1 + u / 2) if abs(u) < 1e-6 else A * (v - vh) / (1 - math.exp(-u))
    am, bm = vtrap(0.1, -40.0, 10.0), 4.0 * math.exp(-(v + 65.0) / 18.0)
    ah, bh = 0.07 * math.exp(-(v + 65.0) / 20.0), 1.0 / (1.0 + math.exp(-(v + 35.0) / 10.0))
    an, bn = vtrap(0.01, -55.0, 10.0), 0.125 * math.exp(-(v + 65.0) / 80.0)
    return (am, bm), (ah, bh), (an, bn)


def _hh_current(v, m, h, n, p=HH_SOMA):
    return (p["gnabar"] * m ** 3 * h * (v - p["ena"]) + p["gkbar"] * n ** 4 * (v - p["ek"])
            + p["gl"] * (v - p["el"]))


def _hh_rest():
    def f(v):
        (am, bm), (ah, bh), (an, bn) = _hh_inf(v)
        return _hh_current(v, am / (am + bm), ah / (ah + bh), an / (an + bn))
    lo, hi = -70.0, -60.0
    assert f(lo) < 0 < f(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_hh_rest_is_the_ode_equilibrium():
    """With no input the discrete map settles on the root of
    I(v, x_inf(v)) = 0, found here by bisection (about -65 mV, the resting
    potential of the squid-axon model at 6.3 C with el = -54.3 mV)."""
    vr = _hh_rest()
    assert abs(vr - (-65.0)) < 0.1
    sc = single_compartment(mech="hh", tstop=500.0)
    m = simulate(sc, nthreads=1)
    assert abs(m.v()[0] - vr) < 1e-9


def _rk4_hh(t_end, dt, amp_density, t_on, t_off, v0=-65.0):
    """Independent RK4 integration of the single-compartment HH ODE
    (cm dv/dt = I_inj - I_ion, 1e3 converts mA/cm2 / uF/cm2 to mV/ms)."""
    (am, bm), (ah, bh), (an, bn) = _hh_inf(v0)
    y = np.array([v0, am / (am + bm), ah / (ah + bh), an / (an + bn)])

    def rhs(t, y):
        v, m, h, n = y
        (am, bm), (ah, bh), (an, bn) = _hh_inf(v)
        inj = amp_density if t_on <= t < t_off else 0.0
        return np.array([1e3 * (inj - _hh_current(v, m, h, n)) / 1.0,
                         am * (1 - m) - bm * m, ah * (1 - h) - bh * h, an * (1 - n) - bn * n])
    nsteps = int(round(t_end / dt))
    out = np.empty(nsteps + 1)
    out[0] = v0
    t = 0.0
    for k in range(nsteps):
        t = k * dt
        k1 = rhs(t, y)
        k2 = rhs(t + dt / 2, y + dt / 2 * k1)
        k3 = rhs(t + dt / 2, y + dt / 2 * k2)
        k4 = rhs(t + dt, y + dt * k3)
        y = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        out[k + 1] = y[0]
    return out


@pytest.mark.slow
def test_hh_spike_first_order_convergence_to_rk4():
    """The oracle's backward Euler + cnexp scheme is first order: against an
    RK4 solution of the same ODE the error halves when dt halves."""
    area = math.pi * 20.0 * 20.0
    amp = 0.3
    t_end = 12.0
    ref_dt = 0.00625 / 8
    ref = _rk4_hh(t_end, ref_dt, 100.0 * amp / area, 1.0, 2.0)
    errs = []
    for dt in (0.025, 0.0125, 0.00625):
        sc = single_compartment(mech="hh", tstop=t_end, dt=dt, stim_amp=amp, stim_del=1.0, stim_dur=1.0)
        tr = simulate(sc, nthreads=1).trace(0)
        stride = int(round(dt / ref_dt))
        assert abs(stride * ref_dt - dt) < 1e-15
        errs.append(np.max(np.abs(tr - ref[::stride][: tr.shape[0]])))
    assert ref.max() > 0.0                     # the pulse fires a spike
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.6 < r1 < 2.6 and 1.6 < r2 < 2.6, errs


# --------------------------------------------------------------- events
def _isolated_spikes(gid, event_steps, weight, tstop):
    """Spike steps of cell ``gid`` of the ring, disconnected, receiving
    external events of ``weight`` at the given steps."""
    sc = ring16(tstop=tstop, weight=weight)
    sc.netcon_src = sc.netcon_src[:0]; sc.netcon_syn = sc.netcon_syn[:0]
    sc.netcon_w = sc.netcon_w[:0]; sc.netcon_delay = sc.netcon_delay[:0]
    n = len(event_steps)
    sc.ev_syn = np.full(n, gid, np.int32)
    sc.ev_t = np.array(event_steps, np.float64) * sc.dt
    sc.ev_w = np.full(n, weight)
    g, k = simulate(sc, nthreads=1).spikes()
    return [int(x) for x in k[g == gid]]


@pytest.mark.parametrize("weight,tstop", [(0.01, 100.0), (0.02, 300.0)])
def test_ring_raster_composes_isolated_responses(weight, tstop):
    """Ring of 16 (the Ring model's shape, Section 5): the raster must be the
    chain of isolated single-cell responses.  Cell c, simulated alone with the
    events the ring delivers to it, fires at step t; cell c+1 then receives an
    event at t + 40 (1 ms delay); the kick reaches cell 0 at step 40."""
    sc = ring16(tstop=tstop, weight=weight)
    nsteps = sc.nsteps
    g, k = simulate(sc, nthreads=2).spikes()
    got = [(int(a), int(b)) for a, b in zip(g, k)]
    events = {c: [] for c in range(16)}
    expect = []
    c, s = 0, 40
    while s < nsteps:
        events[c].append(s)
        after = [t for t in _isolated_spikes(c, events[c], weight, tstop) if t > s]
        if not after:
            break
        expect.append((c, after[0]))
        c, s = (c + 1) % 16, after[0] + 40
    assert got == expect
    if weight == 0.01:                         # a subthreshold cell ends the ring early
        assert 5 <= len(got) < 16
    else:                                      # the ring keeps circulating
        assert len(got) > 32
        assert all(x == i % 16 for i, (x, _) in enumerate(got))


def test_expsyn_converges_first_order_to_the_ode():
    """One passive compartment with one ExpSyn (tau 2 ms, e 0 mV) kicked by a
    0.005 uS event at 1 ms, against an independent high-accuracy integration
    (DOP853, rtol 1e-12) of cm dv/dt = -g_l (v - e_l) - (100 G(t)/area)(v - e),
    G(t) = w exp(-(t - 1)/tau): the backward-Euler error halves with dt.  A
    wrong point-to-density scale (100/area), sign or decay would leave an
    error that does not vanish."""
    from scipy.integrate import solve_ivp
    w, tau, es, T = 0.005, 2.0, 0.0, 10.0
    area, gl, el, cm = math.pi * 20.0 * 20.0, 1e-4, -65.0, 1.0   # single_compartment: L = diam = 20 um

    def rhs(t, v):
        G = 100.0 * w * math.exp(-(t - 1.0) / tau) / area
        return [-(1e3 / cm) * (gl * (v[0] - el) + G * (v[0] - es))]

    errs = []
    for dt in (0.025, 0.0125, 0.00625, 0.003125):
        sc = single_compartment(mech="pas", tstop=T, dt=dt, pas_g=gl, pas_e=el, v_init=el)
        sc.mechs.append(MechTable("expsyn", np.array([0], np.int32), {"tau": np.array([tau]), "e": np.array([es])}))
        sc.ev_syn, sc.ev_t, sc.ev_w = np.array([0], np.int32), np.array([1.0]), np.array([w])
        tr = simulate(sc, nthreads=1).trace(0)
        ts = np.arange(tr.shape[0]) * dt
        ref = np.full(ts.shape, el)
        after = ts > 1.0
        ref[after] = solve_ivp(rhs, (1.0, ts[-1]), [el], method="DOP853", rtol=1e-12, atol=1e-12,
                               t_eval=ts[after]).y[0]
        assert np.all(tr[~after] == el)          # nothing before the event
        errs.append(np.max(np.abs(tr - ref)))
    assert tr.max() > -45.0                      # a real depolarisation towards e
    for e0, e1 in zip(errs, errs[1:]):
        assert 1.95 < e0 / e1 < 2.05
    assert errs[-1] < 0.01


def test_netcon_delay_rounds_half_away_from_zero():
    """A 2.5-step delay (dt 0.25 ms, delay 0.625 ms) lands 3 steps after the
    spike: the target's voltage is untouched until that step's update."""
    base = ring16(n_cells=2, tstop=30.0, weight=0.02, dt=0.25)
    base.netcon_src = np.array([0], np.int32); base.netcon_syn = np.array([1], np.int32)
    base.netcon_w = np.array([0.02]); base.netcon_delay = np.array([0.625])
    quiet = ring16(n_cells=2, tstop=30.0, weight=0.02, dt=0.25)
    quiet.netcon_src = quiet.netcon_src[:0]; quiet.netcon_syn = quiet.netcon_syn[:0]
    quiet.netcon_w = quiet.netcon_w[:0]; quiet.netcon_delay = quiet.netcon_delay[:0]
    m1, m0 = simulate(base, nthreads=1), simulate(quiet, nthreads=1)
    g, k = m1.spikes()
    t0 = int(k[g == 0][0])
    a, b = m1.trace(1), m0.trace(1)
    first_diff = int(np.nonzero(a != b)[0][0])
    # delivered at the start of step t0+3, so v_{t0+4} is the first change
    assert first_diff == t0 + 3 + 1
    assert m1.min_delay == 3


def test_event_order_is_deterministic_across_threads():
    sc = network(n_cells=48, tstop=30.0, w_median=0.02, bg_w=0.02, bg_rate_hz=40.0)
    m1 = simulate(sc, nthreads=1)
    m4 = simulate(sc, nthreads=4)
    g1, k1 = m1.spikes()
    g4, k4 = m4.spikes()
    assert len(g1) > 0
    assert np.array_equal(g1, g4) and np.array_equal(k1, k4)
    assert np.array_equal(m1.v(), m4.v())


# ---------------------------------------------------------- generator
def test_background_is_poisson_5hz():
    """Background trains (counter-based Philox draws, cf. Random123 in
    Section 3.5) form a homogeneous Poisson process of the stated rate: counts
    per synapse have variance equal to their mean, and event times are
    uniform over [0, tstop)."""
    from scipy import stats
    sc = network(n_cells=64, tstop=1000.0, n_in=0)
    S = sc.mech("expsyn").n
    lam = 5.0 * S                                  # expected events overall
    n = sc.ev_t.shape[0]
    assert abs(n - lam) < 3 * math.sqrt(lam)
    counts = np.bincount(sc.ev_syn, minlength=S)
    disp = counts.var(ddof=1) / counts.mean()      # 1 for Poisson; sd ~ sqrt(2/(S-1))
    assert abs(disp - 1.0) < 4 * math.sqrt(2.0 / (S - 1))
    assert stats.kstest(sc.ev_t, "uniform", args=(0.0, 1000.0)).pvalue > 1e-3
    assert np.all(np.diff(sc.ev_t) >= 0)


# ------------------------------------------------- channel types (batched)
from scenarios.generator import MECH_PARAMS, _NOMINAL_GATES, _EREV  # noqa: E402


def _gate_rates(g, v):
    A, vh, k, B, vh2, k2 = g
    u = (v - vh) / k
    al = A * k * (1 + u / 2) if abs(u) < 1e-6 else A * (v - vh) / (1 - math.exp(-u))
    return al, B * math.exp(-(v - vh2) / k2)


def _channel_params(kind, gbar):
    p = {"gbar": gbar, "erev": _EREV[kind]}
    for (t, gate), nom in _NOMINAL_GATES.items():
        if t == kind:
            for name, val in zip(["A", "vh", "k", "B", "vh2", "k2"], nom):
                p[f"{gate}_{name}"] = val
    if kind == "cahva":
        p.update(depth=0.1, taur=80.0, cainf=5e-5)
    if kind == "kca":
        p.update(A=0.01, kd=1e-3, B=0.02)
    return p


def _one_node(kind, gbar, v_init, pas_g, pas_e, tstop=1.0):
    sc = single_compartment(mech="pas", tstop=tstop, v_init=v_init, pas_g=pas_g, pas_e=pas_e)
    p = _channel_params(kind, gbar)
    sc.mechs.append(MechTable(kind, np.array([0], np.int32), {k: np.array([p[k]]) for k in MECH_PARAMS[kind]}))
    return sc, p


GATES = {"na3h": ["m", "h"], "kdr4": ["n"], "ka": ["a", "b"], "ih": ["q"], "cahva": ["m", "h"]}
POWERS = {"na3h": (3, 1), "kdr4": (4,), "ka": (3, 1), "ih": (1,), "cahva": (2, 1)}


@pytest.mark.parametrize("kind", sorted(GATES))
def test_channel_gates_relax_exponentially_under_clamp(kind):
    """With the voltage held (a huge pas conductance pins v at e_pas within
    1e-6 mV after one step) each gate relaxes as
    x(t) = x_inf + (x0 - x_inf) exp(-t/tau) (cnexp is exact at fixed v)."""
    v0, vc = -65.0, -20.0
    sc, p = _one_node(kind, 0.0, v0, 1e6, vc, tstop=5.0)
    m = simulate(sc, nthreads=1)
    nsteps = sc.nsteps
    for col, gate in enumerate(GATES[kind]):
        g = tuple(p[f"{gate}_{q}"] for q in ["A", "vh", "k", "B", "vh2", "k2"])
        a0, b0 = _gate_rates(g, v0)
        a1, b1 = _gate_rates(g, vc)
        x0, xi, tau = a0 / (a0 + b0), a1 / (a1 + b1), 1.0 / (a1 + b1)
        ref = xi + (x0 - xi) * math.exp(-nsteps * sc.dt / tau)
        assert abs(m.state(kind, col)[0] - ref) < 1e-7 * max(1.0, abs(x0 - xi)), (gate, ref)
    assert abs(m.v()[0] - vc) < 1e-6


@pytest.mark.parametrize("kind", sorted(GATES) + ["kca"])
def test_channel_current_first_step_backward_euler(kind):
    """One step of one compartment: (cdt + sum g) v1 = cdt v0 + sum g E, with
    each channel's g = gbar * prod(gate^power) at the steady state of v0."""
    v0 = -40.0
    sc, p = _one_node(kind, 0.01, v0, 1e-4, -70.0, tstop=0.025)
    m = simulate(sc, nthreads=1)
    if kind == "kca":
        cai = 5e-5
        al = p["A"] * cai / (cai + p["kd"])
        gx = p["gbar"] * al / (al + p["B"])
    else:
        gx = p["gbar"]
        for gate, pw in zip(GATES[kind], POWERS[kind]):
            g = tuple(p[f"{gate}_{q}"] for q in ["A", "vh", "k", "B", "vh2", "k2"])
            a, b = _gate_rates(g, v0)
            gx *= (a / (a + b)) ** pw
    cdt = 1e-3 * 1.0 / 0.025
    v1 = (cdt * v0 + 1e-4 * -70.0 + gx * p["erev"]) / (cdt + 1e-4 + gx)
    assert abs(m.v()[0] - v1) < 1e-12


def test_calcium_decay_step():
    """cai after one step: drive = -1e4 ica/(2 F depth) from the current at
    v0, then the linear decay toward cainf + drive*taur over dt (cnexp)."""
    v0 = -10.0
    sc, p = _one_node("cahva", 0.01, v0, 1e-4, -70.0, tstop=0.025)
    m = simulate(sc, nthreads=1)
    gx = p["gbar"]
    for gate, pw in zip(["m", "h"], (2, 1)):
        g = tuple(p[f"{gate}_{q}"] for q in ["A", "vh", "k", "B", "vh2", "k2"])
        a, b = _gate_rates(g, v0)
        gx *= (a / (a + b)) ** pw
    ica = gx * (v0 - p["erev"])
    drive = max(0.0, -1e4 * ica / (2 * 96485.3321 * p["depth"]))
    cai1 = 5e-5 + (1 - math.exp(-0.025 / 80.0)) * (5e-5 + drive * 80.0 - 5e-5)
    assert drive > 0
    assert abs(m.cai()[0] - cai1) < 1e-15


def test_kca_gate_relaxes_exponentially_at_fixed_calcium():
    """KCa alone (no CAHVA, so nothing changes [Ca]i): the gate starts at its
    steady state of the initial 5e-5 mM; after [Ca]i is moved to 2e-3 mM its
    rates are fixed, alpha = A cai/(cai+kd) and beta = B, and cnexp gives
    x(t) = x_inf + (x0 - x_inf) exp(-t (alpha+beta)) exactly.  A wrong alpha
    form, a dropped kd or a swapped alpha/beta fails it."""
    sc, p = _one_node("kca", 0.01, -65.0, 1e6, -30.0, tstop=2.0)
    m = OracleModel(sc)
    c0, c1 = 5e-5, 2e-3
    m.set_cai(c1)
    m.run(sc.nsteps, nthreads=1)
    a0 = p["A"] * c0 / (c0 + p["kd"])
    a1 = p["A"] * c1 / (c1 + p["kd"])
    x0, xi = a0 / (a0 + p["B"]), a1 / (a1 + p["B"])
    ref = xi + (x0 - xi) * math.exp(-sc.nsteps * sc.dt * (a1 + p["B"]))
    assert abs(x0 - xi) > 0.1
    assert abs(m.state("kca", 0)[0] - ref) < 1e-12
    assert np.all(m.cai() == c1)


def test_kca_reads_the_calcium_of_the_new_step():
    """CAHVA and KCa on one compartment, two steps by hand.  Step k: the
    currents use the gates of step k (ica_k = g_ca,k (v_k - eca)); the solve
    gives v_{k+1}; CAHVA's gates move at v_{k+1}; [Ca]i moves with the drive
    of ica_k; then the KCa gate moves with alpha at the NEW [Ca]i.  Reading
    [Ca]i before its update would leave the KCa gate at its steady state
    after the first step (it starts there), which this test rejects."""
    v0, gp, ep = -10.0, 1e-4, -70.0
    sc, pc = _one_node("cahva", 0.02, v0, gp, ep, tstop=0.05)
    pk = _channel_params("kca", 0.01)
    sc.mechs.append(MechTable("kca", np.array([0], np.int32), {k: np.array([pk[k]]) for k in MECH_PARAMS["kca"]}))
    m = simulate(sc, nthreads=1)
    assert sc.nsteps == 2
    dt, cdt, F = sc.dt, 1e-3 * 1.0 / sc.dt, 96485.3321
    gm = tuple(pc[f"m_{q}"] for q in ["A", "vh", "k", "B", "vh2", "k2"])
    gh = tuple(pc[f"h_{q}"] for q in ["A", "vh", "k", "B", "vh2", "k2"])

    def relax(x, al, be):                      # exact solution at fixed rates over dt
        xi = al / (al + be)
        return xi + (x - xi) * math.exp(-dt * (al + be))

    def steady(g, v):
        a, b = _gate_rates(g, v)
        return a / (a + b)

    def kca_alpha(c):
        return pk["A"] * c / (c + pk["kd"])

    v, cai = v0, pc["cainf"]
    xm, xh = steady(gm, v0), steady(gh, v0)
    xk = kca_alpha(cai) / (kca_alpha(cai) + pk["B"])
    xk0 = xk
    for _ in range(2):
        gca = pc["gbar"] * xm * xm * xh
        gk = pk["gbar"] * xk
        ica = gca * (v - pc["erev"])
        v1 = (cdt * v + gp * ep + gca * pc["erev"] + gk * pk["erev"]) / (cdt + gp + gca + gk)
        xm, xh = relax(xm, *_gate_rates(gm, v1)), relax(xh, *_gate_rates(gh, v1))
        drive = max(0.0, -1e4 * ica / (2 * F * pc["depth"]))
        target = pc["cainf"] + drive * pc["taur"]
        cai = target + (cai - target) * math.exp(-dt / pc["taur"])
        xk = relax(xk, kca_alpha(cai), pk["B"])
        v = v1
    assert abs(xk - xk0) > 1e-9 * xk0                 # the step really moved the gate
    assert abs(m.state("kca", 0)[0] - xk) < 1e-13 * max(1.0, xk)
    assert abs(m.cai()[0] - cai) < 1e-11 * cai          # 1 - exp(-dt/taur) cancels ~3.5 digits
    assert abs(m.v()[0] - v) < 1e-11


# ---------------------------------------------------------------- adjoint
def test_oracle_adjoint_matches_central_differences():
    """The discrete adjoint (reverse Hines solve + HH gate Jacobians, with
    checkpointed recompute) against central finite differences of the
    oracle's forward map, h = 1e-6 relative, for gnabar, gkbar and pas g."""
    import copy
    from scenarios import adjoint_net
    from oracle import adjoint
    sc = adjoint_net(n_cells=3, tstop=12.0, n_range=(20, 40))
    K = sc.nsteps
    tgt = simulate(sc, nthreads=1).traces() + 0.5 * np.sin(np.arange(K + 1) * 0.01)[None, :]

    def loss(s):
        tr = simulate(s, nthreads=1).traces()
        return float(np.sum((tr[:, 1:] - tgt[:, 1:]) ** 2))

    J, gna, gk, gp = adjoint(sc, K, tgt, seg=37, nthreads=1)
    assert abs(J - loss(sc)) <= 1e-12 * J

    def fd(kind, name, inst):
        h = 1e-6 * abs(sc.mech(kind).params[name][inst])
        sp, sm = copy.deepcopy(sc), copy.deepcopy(sc)
        sp.mech(kind).params[name][inst] += h
        sm.mech(kind).params[name][inst] -= h
        return (loss(sp) - loss(sm)) / (2 * h)

    for inst in range(3):
        assert abs(gna[inst] - fd("hh", "gnabar", inst)) <= 1e-6 * abs(gna[inst])
        assert abs(gk[inst] - fd("hh", "gkbar", inst)) <= 1e-6 * abs(gk[inst])
    for inst in (0, 17, 40):
        assert abs(gp[inst] - fd("pas", "g", inst)) <= 1e-6 * max(abs(gp[inst]), 1.0)
    # checkpoint spacing does not change the result
    J2, gna2, gk2, gp2 = adjoint(sc, K, tgt, seg=K, nthreads=2)
    assert np.allclose(gna2, gna, rtol=1e-12) and np.allclose(gp2, gp, rtol=1e-12, atol=1e-12)


# -------------------------------------------------------- gap junctions
def gap_pair(g_uS=0.002, tstop=5.0, both_sides=True, gl=1e-3, e=-65.0, amp=0.2):
    """Two single passive compartments (L = d = 20 um); cell 0 gets a 0.5 ms
    current pulse; a gap junction of g uS couples their nodes (one half gap
    per side, or only the half gap on cell 0)."""
    import dataclasses
    a = single_compartment(mech="pas", tstop=tstop, pas_g=gl, pas_e=e, v_init=e,
                           stim_amp=amp, stim_del=0.0, stim_dur=0.5)
    off = np.array([0, 1, 2], np.int32)
    pas = MechTable("pas", np.array([0, 1], np.int32), {"g": np.full(2, gl), "e": np.full(2, e)})
    sc = dataclasses.replace(
        a, cell_offset=off, parent=np.array([-1, -1], np.int32), dx=np.repeat(a.dx, 2),
        diam=np.repeat(a.diam, 2), Ra=np.repeat(a.Ra, 2), cm=np.repeat(a.cm, 2),
        spike_node=np.zeros(2, np.int32), threshold=np.full(2, 100.0), mechs=[pas],
        rec_node=np.array([0, 1], np.int32),
        gap_node=np.array([0, 1] if both_sides else [0], np.int32),
        gap_peer=np.array([1, 0] if both_sides else [1], np.int32),
        gap_g=np.full(2 if both_sides else 1, g_uS))
    return sc


def test_gap_junction_sum_and_difference_laws():
    """With the peer voltage of the start of the step and the own voltage
    implicit, two equal passive compartments obey, step by step,
    (s' - 2e) = (s - 2e)(c + G)/(c + gl + G) for the sum s = v0 + v1 and
    d' = d (c - G)/(c + gl + G) for the difference, c = 1e-3 cm/dt,
    G = 100 g/area.  Checked after the pulse ends."""
    g, gl, e, dt = 0.002, 1e-3, -65.0, 0.025
    sc = gap_pair(g_uS=g, gl=gl, e=e)
    tr = simulate(sc, nthreads=1).traces()
    area = math.pi * 20.0 * 20.0
    c, G = 1e-3 * 1.0 / dt, 100.0 * g / area
    s, d = tr[0] + tr[1], tr[0] - tr[1]
    k0 = 25  # the pulse is over
    for k in range(k0, sc.nsteps):
        assert abs((s[k + 1] - 2 * e) - (s[k] - 2 * e) * (c + G) / (c + gl + G)) <= 1e-12 * abs(s[k] - 2 * e) + 1e-14
        assert abs(d[k + 1] - d[k] * (c - G) / (c + gl + G)) <= 1e-12 * abs(d[k]) + 1e-14
    assert abs(d[k0]) > 1.0  # the pulse made a real difference


def test_half_gap_acts_on_its_own_side_only():
    """A half gap on cell 0 alone: cell 1 evolves exactly as an uncoupled
    compartment at rest, cell 0 feels the junction."""
    sc = gap_pair(both_sides=False)
    tr = simulate(sc, nthreads=1).traces()
    assert np.all(tr[1] == -65.0)
    ref = gap_pair(g_uS=0.0)
    tr0 = simulate(ref, nthreads=1).traces()
    assert np.max(np.abs(tr[0] - tr0[0])) > 0.1


def test_spike_upstrokes_amplify_rounding():
    """The spiking dynamics amplify a one-ulp change of the initial voltage
    by orders of magnitude (it stays far below the 1e-9 mV bar for one
    perturbation) without changing the raster: the scale against which two
    correct FP64 implementations that round differently at every step are
    compared."""
    import dataclasses
    from scenarios import morph_types
    sc = morph_types(n_cells=1024, cells_per_type=1, tstop=10.0)
    a = simulate(sc)
    b = simulate(dataclasses.replace(sc, v_init=np.nextafter(sc.v_init, 0.0)))
    ga, ka = a.spikes()
    gb, kb = b.spikes()
    assert len(ga) > 50 and np.array_equal(ga, gb) and np.array_equal(ka, kb)
    dv = np.max(np.abs(a.traces() - b.traces()))
    ulp = np.spacing(65.0)
    assert 100 * ulp < dv < 1e-9
