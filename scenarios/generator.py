"""Seeded synthetic network generators (inputs only).

Every workload is a forest of multi-compartment cells.  A cell is a soma node
(index 0, the root) plus dendritic sections; a section of ``nseg`` segments
adds a chain of ``nseg`` nodes, the first attached to the last node of an
earlier section or to the soma.  Nodes are numbered so that parent < child
inside each cell.  Geometry is given per node as the segment length ``dx``
(um), diameter ``diam`` (um), axial resistivity ``Ra`` (ohm cm) and specific
capacitance ``cm`` (uF/cm2); turning geometry into areas and axial
resistances is left to the consumers.

Randomness uses numpy's counter-based Philox generator: one stream per cell,
keyed by (gid, seed), so a reduced workload (fewer cells) reproduces the first
cells of the full one exactly, plus one network stream keyed by the seed.

Units: mV, ms, um, uF/cm2, S/cm2 (density mechanisms), uS (synapses), nA
(stimuli).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Parameter order of every mechanism type (SoA column order).
GATE6 = ["A", "vh", "k", "B", "vh2", "k2"]


def _gate(prefix):
    return [f"{prefix}_{p}" for p in GATE6]


MECH_PARAMS = {
    "pas": ["g", "e"],
    "hh": ["gnabar", "gkbar", "gl", "el", "ena", "ek"],
    "expsyn": ["tau", "e"],
    # Channel types of the heterogeneous batched workload.  Each gate x obeys
    # alpha = A (v-vh) / (1 - exp(-(v-vh)/k)), beta = B exp(-(v-vh2)/k2).
    "na3h": ["gbar", "erev"] + _gate("m") + _gate("h"),
    "kdr4": ["gbar", "erev"] + _gate("n"),
    "ka": ["gbar", "erev"] + _gate("a") + _gate("b"),
    "ih": ["gbar", "erev"] + _gate("q"),
    # HVA calcium current m^2 h with intracellular calcium decay:
    # dcai/dt = -1e4 ica / (2 F depth) + (cainf - cai) / taur (inward only).
    "cahva": ["gbar", "erev"] + _gate("m") + _gate("h") + ["depth", "taur", "cainf"],
    # Calcium-activated K: one gate, alpha = A cai / (cai + kd), beta = B.
    "kca": ["gbar", "erev", "A", "kd", "B"],
}

# Nominal ("HH-like") gate kinetics used by the batched workload; each cell
# draws A, vh, k from +/-20% of these.
_NOMINAL_GATES = {
    ("na3h", "m"): (0.1, -40.0, 10.0, 4.0, -65.0, 18.0),
    ("na3h", "h"): (-0.007, -60.0, -10.0, 0.05, -30.0, -12.0),
    ("kdr4", "n"): (0.01, -55.0, 10.0, 0.125, -65.0, 80.0),
    ("ka", "a"): (0.02, -50.0, 10.0, 0.1, -70.0, 20.0),
    ("ka", "b"): (-0.002, -75.0, -8.0, 0.03, -55.0, -20.0),
    ("ih", "q"): (-0.0008, -90.0, -10.0, 0.0005, -70.0, -20.0),
    ("cahva", "m"): (0.055, -27.0, 3.8, 0.94, -75.0, 17.0),
    ("cahva", "h"): (-0.0004, -60.0, -10.0, 0.0065, -15.0, -28.0),
}
_NOMINAL_GBAR_SOMA = {"na3h": 0.12, "kdr4": 0.036, "ka": 0.01, "ih": 1e-4, "cahva": 1e-4, "kca": 1e-3}
_NOMINAL_GBAR_DEND = {"na3h": 0.01, "kdr4": 0.003, "ka": 0.005, "ih": 5e-5, "cahva": 5e-5, "kca": 5e-4}
_EREV = {"na3h": 50.0, "kdr4": -77.0, "ka": -77.0, "ih": -30.0, "cahva": 120.0, "kca": -77.0}
CHANNEL_TYPES = ["na3h", "kdr4", "ka", "ih", "cahva", "kca"]


@dataclass
class MechTable:
    kind: str
    node: np.ndarray                      # int32, global node index per instance
    params: dict = field(default_factory=dict)  # name -> float64[n]

    @property
    def n(self) -> int:
        return int(self.node.shape[0])

    def param_matrix(self) -> np.ndarray:
        """Parameters as a [n_params, n] float64 array in MECH_PARAMS order."""
        names = MECH_PARAMS[self.kind]
        if self.n == 0:
            return np.zeros((len(names), 0))
        return np.ascontiguousarray(np.stack([np.asarray(self.params[p], np.float64) for p in names]))


@dataclass
class Scenario:
    name: str
    dt: float
    tstop: float
    cell_offset: np.ndarray   # int32[n_cells+1]
    parent: np.ndarray        # int32[n_nodes], cell-local parent, -1 at the root
    dx: np.ndarray            # float64[n_nodes] segment length (um)
    diam: np.ndarray          # float64[n_nodes] (um)
    Ra: np.ndarray            # float64[n_nodes] (ohm cm)
    cm: np.ndarray            # float64[n_nodes] (uF/cm2)
    spike_node: np.ndarray    # int32[n_cells], cell-local
    threshold: np.ndarray     # float64[n_cells] (mV)
    mechs: list               # list[MechTable]
    netcon_src: np.ndarray    # int32 source gid
    netcon_syn: np.ndarray    # int32 target expsyn instance (index in the expsyn table)
    netcon_w: np.ndarray      # float64 (uS)
    netcon_delay: np.ndarray  # float64 (ms)
    ev_syn: np.ndarray        # int32 external events: target expsyn instance
    ev_t: np.ndarray          # float64 (ms)
    ev_w: np.ndarray          # float64 (uS)
    stim_node: np.ndarray     # int32 global node (IClamp)
    stim_del: np.ndarray
    stim_dur: np.ndarray
    stim_amp: np.ndarray      # nA
    rec_node: np.ndarray      # int32 global nodes whose voltage is recorded
    v_init: float = -65.0
    meta: dict = field(default_factory=dict)
    # half gap junctions: node, peer node (global), conductance (uS); one entry per side
    gap_node: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    gap_peer: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    gap_g: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))

    @property
    def n_cells(self) -> int:
        return int(self.cell_offset.shape[0] - 1)

    @property
    def n_nodes(self) -> int:
        return int(self.parent.shape[0])

    @property
    def nsteps(self) -> int:
        return int(round(self.tstop / self.dt))

    def mech(self, kind):
        for m in self.mechs:
            if m.kind == kind:
                return m
        return None

    def cell_of_node(self) -> np.ndarray:
        sizes = np.diff(self.cell_offset)
        return np.repeat(np.arange(self.n_cells, dtype=np.int32), sizes)


def _cell_rng(seed: int, gid: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([gid, seed], dtype=np.uint64)))


def _net_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([2**63 + 7, seed], dtype=np.uint64)))


def random_section_tree(rng, n_dend: int, nseg: int = 5, L=(50.0, 200.0), d=(1.0, 3.0),
                        soma_max_children: int = 2):
    """Dendrite nodes of one cell as a random binary tree of sections.

    Returns (parent, dx, diam, section_of_node) for nodes 1..n_dend (cell-local,
    soma = 0).  Sections have ``nseg`` segments, the last one takes the
    remainder so that exactly ``n_dend`` dendrite nodes exist.  Each new
    section attaches, uniformly at random, to the soma or to the end of an
    earlier section that has fewer than two children.
    """
    n_sec = max(1, math.ceil(n_dend / nseg)) if n_dend > 0 else 0
    parent = np.empty(n_dend, np.int32)
    dx = np.empty(n_dend, np.float64)
    diam = np.empty(n_dend, np.float64)
    secid = np.empty(n_dend, np.int32)
    open_pts = [0]                # attach points (cell-local node) with < 2 children
    nchild = {0: 0}
    limit = {0: soma_max_children}
    lens = rng.uniform(L[0], L[1], n_sec)
    diams = rng.uniform(d[0], d[1], n_sec)
    picks = rng.random(n_sec)
    pos = 0
    for s in range(n_sec):
        ns = nseg if s < n_sec - 1 else n_dend - nseg * (n_sec - 1)
        k = int(picks[s] * len(open_pts))
        at = open_pts[k]
        nchild[at] += 1
        if nchild[at] >= limit[at]:
            open_pts.pop(k)
        for j in range(ns):
            node = 1 + pos + j
            parent[pos + j] = at if j == 0 else node - 1
            dx[pos + j] = lens[s] / nseg
            diam[pos + j] = diams[s]
            secid[pos + j] = s
        end = 1 + pos + ns - 1
        nchild[end] = 0
        limit[end] = 2
        open_pts.append(end)
        pos += ns
    return parent, dx, diam, secid


def _assemble(name, dt, tstop, cells, mechs, **kw):
    """Concatenate per-cell morphology dicts into a Scenario."""
    sizes = np.array([c["parent"].shape[0] for c in cells], np.int64)
    off = np.zeros(len(cells) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    if off[-1] >= 2**31:
        raise ValueError("too many nodes for int32 indexing")
    cat = lambda k, dt_: np.concatenate([c[k] for c in cells]).astype(dt_) if cells else np.zeros(0, dt_)
    z_i = np.zeros(0, np.int32)
    z_f = np.zeros(0, np.float64)
    sc = Scenario(
        name=name, dt=dt, tstop=tstop, cell_offset=off.astype(np.int32),
        parent=cat("parent", np.int32), dx=cat("dx", np.float64), diam=cat("diam", np.float64),
        Ra=cat("Ra", np.float64), cm=cat("cm", np.float64),
        spike_node=np.zeros(len(cells), np.int32),
        threshold=np.full(len(cells), kw.pop("threshold", -20.0)),
        mechs=mechs,
        netcon_src=kw.pop("netcon_src", z_i), netcon_syn=kw.pop("netcon_syn", z_i),
        netcon_w=kw.pop("netcon_w", z_f), netcon_delay=kw.pop("netcon_delay", z_f),
        ev_syn=kw.pop("ev_syn", z_i), ev_t=kw.pop("ev_t", z_f), ev_w=kw.pop("ev_w", z_f),
        stim_node=kw.pop("stim_node", z_i), stim_del=kw.pop("stim_del", z_f),
        stim_dur=kw.pop("stim_dur", z_f), stim_amp=kw.pop("stim_amp", z_f),
        rec_node=kw.pop("rec_node", z_i), v_init=kw.pop("v_init", -65.0), meta=kw.pop("meta", {}),
    )
    if kw:
        raise TypeError(f"unknown fields {sorted(kw)}")
    return sc


def _hh_soma_cell(rng, n_dend, Ra=100.0, cm=1.0, soma_L=20.0, soma_d=20.0, nseg=5):
    par, dx, diam, sec = random_section_tree(rng, n_dend, nseg=nseg)
    return {
        "parent": np.concatenate([[-1], par]).astype(np.int32),
        "dx": np.concatenate([[soma_L], dx]),
        "diam": np.concatenate([[soma_d], diam]),
        "Ra": np.full(n_dend + 1, Ra),
        "cm": np.full(n_dend + 1, cm),
        "sec": np.concatenate([[-1], sec]).astype(np.int32),
    }


HH_SOMA = dict(gnabar=0.12, gkbar=0.036, gl=3e-4, el=-54.3, ena=50.0, ek=-77.0)
PAS_DEND = dict(g=1e-3, e=-65.0)


def _hh_and_pas(cells, off):
    """HH at every soma, pas at every dendrite node."""
    soma = off[:-1].astype(np.int32)
    n = len(cells)
    hh = MechTable("hh", soma, {k: np.full(n, v) for k, v in HH_SOMA.items()})
    dend = np.concatenate([np.arange(off[i] + 1, off[i + 1]) for i in range(n)]).astype(np.int32) \
        if n else np.zeros(0, np.int32)
    pas = MechTable("pas", dend, {k: np.full(dend.shape[0], v) for k, v in PAS_DEND.items()})
    return hh, pas


def _offsets(cells):
    sizes = np.array([c["parent"].shape[0] for c in cells], np.int64)
    off = np.zeros(len(cells) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    return off


def ring16(n_cells: int = 16, tstop: float = 100.0, weight: float = 0.01, seed: int = 1901,
           dt: float = 0.025) -> Scenario:
    """Ring of HH-soma cells with 4 passive dendrite sections (nseg 5) each.

    One ExpSyn (tau 2 ms, e 0 mV) sits in the middle node of each cell's first
    dendrite section.  Cell i drives cell i+1 (the last drives cell 0):
    threshold -20 mV, delay 1 ms, weight ``weight`` uS.  Cell 0 receives one
    external event at t = 1 ms with the same weight.
    """
    cells = [_hh_soma_cell(_cell_rng(seed, g), 20) for g in range(n_cells)]
    off = _offsets(cells)
    hh, pas = _hh_and_pas(cells, off)
    syn_node = np.array([off[i] + 1 + 2 for i in range(n_cells)], np.int32)  # section 0, segment 2
    syn = MechTable("expsyn", syn_node, {"tau": np.full(n_cells, 2.0), "e": np.zeros(n_cells)})
    src = np.arange(n_cells, dtype=np.int32)
    tgt = ((src + 1) % n_cells).astype(np.int32)
    return _assemble(
        "ring16", dt, tstop, cells, [hh, pas, syn],
        netcon_src=src, netcon_syn=tgt, netcon_w=np.full(n_cells, weight),
        netcon_delay=np.full(n_cells, 1.0),
        ev_syn=np.array([0], np.int32), ev_t=np.array([1.0]), ev_w=np.array([weight]),
        rec_node=off[:-1].astype(np.int32), threshold=-20.0,
        meta={"seed": seed, "config": "ring16"},
    )


def network(n_cells: int = 16384, tstop: float = 1000.0, n_range=(200, 600), n_syn: int = 50,
            n_in: int = 100, delay=(1.0, 5.0), w_median: float = 0.002, w_sigma: float = 0.5,
            bg_rate_hz: float = 5.0, bg_w: float = 0.002, seed: int = 1902, dt: float = 0.025,
            record: str = "soma") -> Scenario:
    """Plain FP64 network: random binary dendritic trees with an HH soma.

    Each cell has N ~ U{n_range} compartments, ``n_syn`` ExpSyn at uniform
    random dendritic nodes, and ``n_in`` incoming NetCons from uniform random
    other cells onto uniform random synapses of the target (delay U[delay] ms,
    weight lognormal with the given median and sigma).  Every synapse receives
    an independent Poisson train of ``bg_rate_hz`` external events of weight
    ``bg_w`` over [0, tstop).
    """
    sizes = []
    cells = []
    syn_nodes = []
    for g in range(n_cells):
        rng = _cell_rng(seed, g)
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        c = _hh_soma_cell(rng, N - 1)
        cells.append(c)
        sizes.append(N)
        syn_nodes.append(1 + rng.integers(0, N - 1, n_syn))
    off = _offsets(cells)
    hh, pas = _hh_and_pas(cells, off)
    sn = np.concatenate([off[i] + syn_nodes[i] for i in range(n_cells)]).astype(np.int32)
    S = sn.shape[0]
    syn = MechTable("expsyn", sn, {"tau": np.full(S, 2.0), "e": np.zeros(S)})
    rng = _net_rng(seed)
    kw = {}
    if n_in > 0 and n_cells > 1:
        src = rng.integers(0, n_cells - 1, (n_cells, n_in))
        src = src + (src >= np.arange(n_cells)[:, None])
        tsyn = np.arange(n_cells)[:, None] * n_syn + rng.integers(0, n_syn, (n_cells, n_in))
        dly = rng.uniform(delay[0], delay[1], (n_cells, n_in))
        w = rng.lognormal(np.log(w_median), w_sigma, (n_cells, n_in))
        kw.update(netcon_src=src.reshape(-1).astype(np.int32), netcon_syn=tsyn.reshape(-1).astype(np.int32),
                  netcon_w=w.reshape(-1), netcon_delay=dly.reshape(-1))
    if bg_rate_hz > 0 and S > 0:
        lam = bg_rate_hz * 1e-3 * tstop
        cnt = rng.poisson(lam, S)
        t = rng.uniform(0.0, tstop, int(cnt.sum()))
        s = np.repeat(np.arange(S, dtype=np.int32), cnt)
        order = np.argsort(t, kind="stable")
        kw.update(ev_syn=s[order], ev_t=t[order], ev_w=np.full(t.shape[0], bg_w))
    rec = off[:-1].astype(np.int32) if record == "soma" else np.zeros(0, np.int32)
    return _assemble("network", dt, tstop, cells, [hh, pas, syn], rec_node=rec, threshold=-20.0,
                     meta={"seed": seed, "config": "network", "n_range": n_range}, **kw)


def adjoint_net(n_cells: int = 1024, tstop: float = 200.0, n_range=(100, 300), seed: int = 1905,
                dt: float = 0.025, amp=(0.1, 0.3)) -> Scenario:
    """Unconnected cells (config-1 morphology rules) driven by a somatic IClamp.

    The clamp runs for the whole simulation (del 0, dur tstop) with amplitude
    U[amp] nA per cell.  Soma voltage of every cell is recorded.
    """
    cells = []
    amps = []
    for g in range(n_cells):
        rng = _cell_rng(seed, g)
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        cells.append(_hh_soma_cell(rng, N - 1))
        amps.append(rng.uniform(amp[0], amp[1]))
    off = _offsets(cells)
    hh, pas = _hh_and_pas(cells, off)
    soma = off[:-1].astype(np.int32)
    return _assemble("adjoint", dt, tstop, cells, [hh, pas],
                     stim_node=soma, stim_del=np.zeros(n_cells), stim_dur=np.full(n_cells, tstop),
                     stim_amp=np.array(amps), rec_node=soma, threshold=-20.0,
                     meta={"seed": seed, "config": "adjoint"})


def batched(n_cells: int = 50000, tstop: float = 1000.0, n_clip=(50, 5000), logn_mu=math.log(400.0),
            logn_sigma: float = 0.8, n_syn: int = 50, n_in: int = 100, seed: int = 1903,
            dt: float = 0.025, bg_rate_hz: float = 5.0, record: str = "soma") -> Scenario:
    """Heterogeneous cells with random channel subsets.

    N ~ LogNormal(logn_mu, logn_sigma) clipped to ``n_clip``.  Each of the six
    channel types is selected with probability 1/2 per cell and then inserted
    at every node of that cell; Na and Kdr are always present at the soma.
    Every node also carries pas (soma: g 3e-4, e -54.3; dendrites g 1e-3,
    e -65).  Gate parameters A, vh, k of each type are drawn per cell within
    +/-20% of nominal values.  Synapses, NetCons and background as in
    :func:`network`.
    """
    cells, syn_nodes, chans = [], [], []
    for g in range(n_cells):
        rng = _cell_rng(seed, g)
        N = int(np.clip(round(rng.lognormal(logn_mu, logn_sigma)), n_clip[0], n_clip[1]))
        c = _hh_soma_cell(rng, N - 1)
        cells.append(c)
        syn_nodes.append(1 + rng.integers(0, N - 1, n_syn))
        sel = rng.random(len(CHANNEL_TYPES)) < 0.5
        draws = {}
        for ti, t in enumerate(CHANNEL_TYPES):
            pr = {}
            for (tt, gate), nom in _NOMINAL_GATES.items():
                if tt != t:
                    continue
                f = rng.uniform(0.8, 1.2, 3)
                pr[gate] = (nom[0] * f[0], nom[1] * f[1], nom[2] * f[2], nom[3], nom[4], nom[5])
            draws[t] = pr
        chans.append((sel, draws))
    off = _offsets(cells)
    mechs = []
    # pas everywhere
    allnodes = np.arange(off[-1], dtype=np.int32)
    is_soma = np.zeros(off[-1], bool)
    is_soma[off[:-1]] = True
    mechs.append(MechTable("pas", allnodes, {"g": np.where(is_soma, 3e-4, 1e-3),
                                             "e": np.where(is_soma, -54.3, -65.0)}))
    for ti, t in enumerate(CHANNEL_TYPES):
        nodes, cols = [], {p: [] for p in MECH_PARAMS[t]}
        for gid in range(n_cells):
            sel, draws = chans[gid]
            if sel[ti]:
                nd = np.arange(off[gid], off[gid + 1], dtype=np.int32)
            elif t in ("na3h", "kdr4"):
                nd = np.array([off[gid]], np.int32)
            else:
                continue
            n = nd.shape[0]
            nodes.append(nd)
            gb = np.full(n, _NOMINAL_GBAR_DEND[t])
            gb[0] = _NOMINAL_GBAR_SOMA[t]
            cols["gbar"].append(gb)
            cols["erev"].append(np.full(n, _EREV[t]))
            for gate, vals in draws[t].items():
                for pi, p in enumerate(GATE6):
                    cols[f"{gate}_{p}"].append(np.full(n, vals[pi]))
            if t == "cahva":
                cols["depth"].append(np.full(n, 0.1))
                cols["taur"].append(np.full(n, 80.0))
                cols["cainf"].append(np.full(n, 5e-5))
            if t == "kca":
                cols["A"].append(np.full(n, 0.01))
                cols["kd"].append(np.full(n, 1e-3))
                cols["B"].append(np.full(n, 0.02))
        if nodes:
            mechs.append(MechTable(t, np.concatenate(nodes),
                                   {p: np.concatenate(v) for p, v in cols.items()}))
        else:
            mechs.append(MechTable(t, np.zeros(0, np.int32), {p: np.zeros(0) for p in MECH_PARAMS[t]}))
    sn = np.concatenate([off[i] + syn_nodes[i] for i in range(n_cells)]).astype(np.int32)
    S = sn.shape[0]
    mechs.append(MechTable("expsyn", sn, {"tau": np.full(S, 2.0), "e": np.zeros(S)}))
    rng = _net_rng(seed)
    kw = {}
    if n_in > 0 and n_cells > 1:
        src = rng.integers(0, n_cells - 1, (n_cells, n_in))
        src = src + (src >= np.arange(n_cells)[:, None])
        tsyn = np.arange(n_cells)[:, None] * n_syn + rng.integers(0, n_syn, (n_cells, n_in))
        kw.update(netcon_src=src.reshape(-1).astype(np.int32), netcon_syn=tsyn.reshape(-1).astype(np.int32),
                  netcon_w=rng.lognormal(np.log(0.002), 0.5, (n_cells, n_in)).reshape(-1),
                  netcon_delay=rng.uniform(1.0, 5.0, (n_cells, n_in)).reshape(-1))
    if bg_rate_hz > 0 and S > 0:
        cnt = rng.poisson(bg_rate_hz * 1e-3 * tstop, S)
        t = rng.uniform(0.0, tstop, int(cnt.sum()))
        s = np.repeat(np.arange(S, dtype=np.int32), cnt)
        order = np.argsort(t, kind="stable")
        kw.update(ev_syn=s[order], ev_t=t[order], ev_w=np.full(t.shape[0], 0.002))
    rec = off[:-1].astype(np.int32) if record == "soma" else np.zeros(0, np.int32)
    return _assemble("batched", dt, tstop, cells, mechs, rec_node=rec, threshold=-20.0,
                     meta={"seed": seed, "config": "batched"}, **kw)


def morph_types(n_cells: int = 131072, cells_per_type: int = 32, tstop: float = 10.0, ring: int = 16,
                weight: float = 0.02, seed: int = 1906, dt: float = 0.025) -> Scenario:
    """Cells of many morphological types, as in the node-ordering study.

    Every cell has 83 nodes: an HH soma and 41 passive sections of 2 segments
    (L U[50,200] um, d U[1,3] um) in a random binary branching pattern that is
    drawn per type.  ``cells_per_type`` consecutive gids share a type (1: every
    cell distinct).  Cells form rings of ``ring`` (cell i drives i+1 through an
    ExpSyn in the middle of its first section, delay 1 ms), each ring kicked
    by one external event at 1 ms.
    """
    n_types = (n_cells + cells_per_type - 1) // cells_per_type
    shapes = [_hh_soma_cell(_cell_rng(seed, t), 82, nseg=2) for t in range(n_types)]
    cells = []
    for g in range(n_cells):
        cells.append(shapes[g // cells_per_type])
    off = _offsets(cells)
    hh, pas = _hh_and_pas(cells, off)
    syn_node = (off[:-1] + 1).astype(np.int32)
    syn = MechTable("expsyn", syn_node, {"tau": np.full(n_cells, 2.0), "e": np.zeros(n_cells)})
    src = np.arange(n_cells, dtype=np.int32)
    base = (src // ring) * ring
    tgt = (base + (src - base + 1) % np.minimum(ring, n_cells - base)).astype(np.int32)
    kick = np.arange(0, n_cells, ring, dtype=np.int32)
    return _assemble(
        "morph_types", dt, tstop, cells, [hh, pas, syn],
        netcon_src=src, netcon_syn=tgt, netcon_w=np.full(n_cells, weight),
        netcon_delay=np.full(n_cells, 1.0),
        ev_syn=kick, ev_t=np.full(kick.shape[0], 1.0), ev_w=np.full(kick.shape[0], weight),
        rec_node=off[:-1].astype(np.int32), threshold=-20.0,
        meta={"seed": seed, "cells_per_type": cells_per_type},
    )


def passive_cable(nseg: int, L: float = 1000.0, diam: float = 1.0, Ra: float = 100.0, cm: float = 1.0,
                  g: float = 1e-3, e: float = -65.0, amp: float = 0.1, tstop: float = 60.0,
                  dt: float = 0.025, v_init: float = -65.0) -> Scenario:
    """One unbranched sealed cable of ``nseg`` equal segments, pas everywhere,
    a constant current ``amp`` (nA) injected into the first segment."""
    cell = {
        "parent": np.arange(-1, nseg - 1, dtype=np.int32),
        "dx": np.full(nseg, L / nseg), "diam": np.full(nseg, diam),
        "Ra": np.full(nseg, Ra), "cm": np.full(nseg, cm),
    }
    pas = MechTable("pas", np.arange(nseg, dtype=np.int32), {"g": np.full(nseg, g), "e": np.full(nseg, e)})
    stim = dict(stim_node=np.array([0], np.int32), stim_del=np.array([0.0]), stim_dur=np.array([1e9]),
                stim_amp=np.array([amp])) if amp != 0 else {}
    return _assemble("cable", dt, tstop, [cell], [pas], rec_node=np.arange(nseg, dtype=np.int32),
                     threshold=1e9, v_init=v_init, meta={"L": L, "diam": diam, "Ra": Ra, "g": g, "cm": cm},
                     **stim)


def single_compartment(mech: str = "hh", tstop: float = 50.0, dt: float = 0.025, L: float = 20.0,
                       diam: float = 20.0, stim_amp: float = 0.0, stim_del: float = 1.0,
                       stim_dur: float = 0.5, v_init: float = -65.0, pas_g: float = 1e-3,
                       pas_e: float = -65.0) -> Scenario:
    """One isopotential compartment carrying HH (or pas), optional IClamp."""
    cell = {"parent": np.array([-1], np.int32), "dx": np.array([L]), "diam": np.array([diam]),
            "Ra": np.array([100.0]), "cm": np.array([1.0])}
    if mech == "hh":
        m = MechTable("hh", np.array([0], np.int32), {k: np.array([v]) for k, v in HH_SOMA.items()})
    else:
        m = MechTable("pas", np.array([0], np.int32), {"g": np.array([pas_g]), "e": np.array([pas_e])})
    stim = {}
    if stim_amp != 0.0:
        stim = dict(stim_node=np.array([0], np.int32), stim_del=np.array([stim_del]),
                    stim_dur=np.array([stim_dur]), stim_amp=np.array([stim_amp]))
    return _assemble("single", dt, tstop, [cell], [m], rec_node=np.array([0], np.int32),
                     threshold=-20.0, v_init=v_init, **stim)
