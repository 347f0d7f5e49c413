// cn_oracle.cpp -- plain FP64 CPU stepper for the fixed-step cable network.
//
// TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA engine is
// checked against.  Only the tests, the smoke check and the CPU-baseline leg
// of the benchmark may load it; the engine never calls it, and it shares no
// code, header or table with the engine.  It is deliberately slow and
// literal: one cell at a time, one node at a time, in the order the paper
// lists the per-step operations (Section 2: event delivery, matrix assembly
// from I_ion and I_syn, matrix resolution, state update, threshold
// detection), with the spike exchange at every minimum-delay interval
// (Section 2, hybrid clock-event algorithm).
//
// Model (Section 2, Eq. 1): each section obeys the cable equation
//   d/(4 Ra) d2v/dx2 = cm dv/dt + I_pas + I_ion + I_syn,
// discretised into compartments (nodes at segment centres) that form a tree
// indexed by parent; point-process currents are turned into densities by
// dividing by the compartment area (Section 2, the delta-function remark).
// The stiff tree system is integrated implicitly (backward Euler, fixed step)
// and solved by Gaussian elimination in Hines order (Section 2, citing Hines
// 1984).  Mechanism conductances are analytic (the CONDUCTANCE keyword,
// Section 3.5); gating states use the cnexp update of a fixed-step method
// (Section 6).
//
// Readings where the paper is silent (all listed in the design notes):
//  * area = pi d dx; half-segment resistance 1e-2*2*Ra*dx/(pi d^2) MOhm;
//    ri(node->parent) = R_half(node) + R_half(parent); no zero-area nodes.
//  * coupling in row i: 100/(ri*area_i); in row p: 100/(ri*area_p).
//  * t_k = k*dt (never accumulated); events with delivery step k are applied
//    at the start of step k, ordered by (external before NetCon, then input
//    index / (source gid, NetCon index)), one addition at a time.
//  * IClamp on when del <= (k+1/2) dt < del+dur.
//  * a spike is (gid, k+1) when v_{k+1} > threshold and the source was not
//    already above; its NetCon events arrive at step k+1+round(delay/dt),
//    rounding half away from zero.
//  * rate singularity of A(v-vh)/(1-exp(-(v-vh)/k)): A*k*(1+u/2), u=(v-vh)/k,
//    when |u| < 1e-6.  q10 = 1, rates evaluated directly (no tables).
//  * initial state: v = v_init, gates at their steady state at v_init,
//    synaptic g = 0, cai = cainf.
//  * a half gap junction at node i with peer j injects g (v_j,k - v_i) with
//    v_i implicit and the peer voltage of the start of the step (voltages are
//    exchanged every step; the minimum-delay interval becomes one step).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

extern "C" {

enum {
  OR_PAS = 0, OR_HH = 1, OR_EXPSYN = 2, OR_NA3H = 3, OR_KDR4 = 4, OR_KA = 5,
  OR_IH = 6, OR_CAHVA = 7, OR_KCA = 8, OR_NKINDS = 9
};

struct or_mech_in {
  int32_t kind;
  int32_t n;
  const int32_t* node;   // global node index per instance
  const double* param;   // [n_param][n], column order documented per kind
};

struct or_scenario {
  double dt;
  double v_init;
  int32_t n_cells;
  const int32_t* cell_offset;  // [n_cells+1]
  const int32_t* parent;       // cell-local, -1 at the root, parent < child
  const double* dx;            // um
  const double* diam;          // um
  const double* Ra;            // ohm cm
  const double* cm;            // uF/cm2
  const int32_t* spike_node;   // cell-local
  const double* threshold;     // mV
  int32_t n_mech;
  const or_mech_in* mechs;
  int64_t n_netcon;
  const int32_t* nc_src;
  const int32_t* nc_syn;       // expsyn instance index
  const double* nc_w;          // uS
  const double* nc_delay;      // ms
  int64_t n_ev;
  const int32_t* ev_syn;
  const double* ev_t;
  const double* ev_w;
  int32_t n_stim;
  const int32_t* stim_node;
  const double* stim_del;
  const double* stim_dur;
  const double* stim_amp;      // nA
  int32_t n_rec;
  const int32_t* rec_node;
  int64_t n_gap;               // half gap junctions (one entry per side)
  const int32_t* gap_node;     // global node carrying the half gap
  const int32_t* gap_peer;     // global node of the other side
  const double* gap_g;         // uS
};

}  // extern "C"

namespace {

const int kNParam[OR_NKINDS] = {2, 6, 2, 14, 8, 14, 8, 17, 5};
const double kFaraday = 96485.3321;  // C/mol

// alpha = A (v - vh) / (1 - exp(-(v - vh)/k)), with its limit near v = vh.
double vtrap_rate(double A, double vh, double k, double v) {
  double u = (v - vh) / k;
  if (std::fabs(u) < 1e-6) return A * k * (1.0 + u / 2.0);
  return A * (v - vh) / (1.0 - std::exp(-u));
}

// beta = B exp(-(v - vh2)/k2)
double exp_rate(double B, double vh2, double k2, double v) { return B * std::exp(-(v - vh2) / k2); }

// cnexp step of dx/dt = alpha (1-x) - beta x at fixed v over dt.
double cnexp(double x, double alpha, double beta, double dt) {
  double tau = 1.0 / (alpha + beta);
  double inf = alpha * tau;
  return x + (1.0 - std::exp(-dt / tau)) * (inf - x);
}
double steady(double alpha, double beta) { return alpha / (alpha + beta); }

// Hodgkin-Huxley rates (squid axon at 6.3 C, q10 = 1).
void hh_rates(double v, double* am, double* bm, double* ah, double* bh, double* an, double* bn) {
  *am = vtrap_rate(0.1, -40.0, 10.0, v);
  *bm = 4.0 * std::exp(-(v + 65.0) / 18.0);
  *ah = 0.07 * std::exp(-(v + 65.0) / 20.0);
  *bh = 1.0 / (1.0 + std::exp(-(v + 35.0) / 10.0));
  *an = vtrap_rate(0.01, -55.0, 10.0, v);
  *bn = 0.125 * std::exp(-(v + 65.0) / 80.0);
}

struct Gate6 { double A, vh, k, B, vh2, k2; };
Gate6 gate_at(const std::vector<std::vector<double>>& P, int col, int i) {
  return Gate6{P[col][i], P[col + 1][i], P[col + 2][i], P[col + 3][i], P[col + 4][i], P[col + 5][i]};
}
double galpha(const Gate6& g, double v) { return vtrap_rate(g.A, g.vh, g.k, v); }
double gbeta(const Gate6& g, double v) { return exp_rate(g.B, g.vh2, g.k2, v); }

struct Ev {
  int32_t kind;   // 0 external, 1 NetCon
  int64_t k1;     // external: input index; NetCon: source gid
  int64_t k2;     // NetCon index
  int32_t syn;    // expsyn instance
  double w;
};

struct Mech {
  int kind = -1;
  int n = 0;
  std::vector<int32_t> node;
  std::vector<std::vector<double>> P;  // [n_param][n]
  std::vector<std::vector<double>> S;  // states [n_state][n]
  std::vector<double> ica;             // cahva: current at the last nrn_cur
  std::vector<int32_t> cell_start;     // CSR of instances by cell
  std::vector<int32_t> by_cell;
};

struct Model {
  double dt = 0.025;
  int n_cells = 0, n_nodes = 0;
  std::vector<int32_t> off, parent;  // parent as a global index (-1 at roots)
  std::vector<double> area, ri, a, b, cm, v, rhs, d, cai;
  std::vector<int32_t> spike_node;   // global
  std::vector<double> threshold;
  std::vector<uint8_t> above;
  Mech mech[OR_NKINDS];
  std::vector<int32_t> syn_cell;     // expsyn instance -> cell
  // stimuli
  std::vector<int32_t> st_node;
  std::vector<double> st_del, st_dur, st_amp;
  std::vector<std::vector<int32_t>> cell_stims;
  // gap junctions: per half gap its node, peer node and g; the peer voltage of
  // the current step is copied into gap_vpeer before any cell advances
  std::vector<int32_t> gap_node, gap_peer;
  std::vector<double> gap_g, gap_vpeer;
  std::vector<std::vector<int32_t>> cell_gaps;
  // network
  std::vector<int64_t> nc_start;     // CSR by source gid, NetCon index order
  std::vector<int64_t> nc_idx;
  std::vector<int32_t> nc_syn;
  std::vector<double> nc_w;
  std::vector<int64_t> nc_dsteps;
  int64_t min_delay = 0;             // steps; 0 when there are no NetCons
  std::vector<std::map<int64_t, std::vector<Ev>>> queue;  // per cell
  // outputs
  int64_t step = 0;                  // current step index k (v holds v_k)
  std::vector<int32_t> sp_gid;
  std::vector<int64_t> sp_step;
  std::vector<int32_t> rec_node;
  std::vector<std::vector<double>> trace;  // [rec][k]
  std::vector<std::vector<int32_t>> cell_recs;
  std::string err;
};

bool build(Model& M, const or_scenario* s) {
  M.dt = s->dt;
  M.n_cells = s->n_cells;
  M.off.assign(s->cell_offset, s->cell_offset + s->n_cells + 1);
  M.n_nodes = M.off[M.n_cells];
  int N = M.n_nodes;
  M.parent.resize(N);
  M.area.resize(N); M.ri.assign(N, 0.0); M.a.assign(N, 0.0); M.b.assign(N, 0.0);
  M.cm.assign(s->cm, s->cm + N);
  M.v.assign(N, s->v_init); M.rhs.assign(N, 0.0); M.d.assign(N, 0.0);
  M.cai.assign(N, 5e-5);
  const double pi = 3.14159265358979323846;
  std::vector<double> rhalf(N);
  for (int i = 0; i < N; ++i) {
    M.area[i] = pi * s->diam[i] * s->dx[i];
    rhalf[i] = 1e-2 * 2.0 * s->Ra[i] * s->dx[i] / (pi * s->diam[i] * s->diam[i]);
  }
  for (int c = 0; c < M.n_cells; ++c) {
    for (int i = M.off[c]; i < M.off[c + 1]; ++i) {
      int pl = s->parent[i];
      int li = i - M.off[c];
      if (pl >= li || (li == 0) != (pl < 0) || (pl < -1)) {
        M.err = "bad parent at node " + std::to_string(i);
        return false;
      }
      M.parent[i] = pl < 0 ? -1 : M.off[c] + pl;
      if (pl >= 0) {
        int p = M.parent[i];
        M.ri[i] = rhalf[i] + rhalf[p];
        M.b[i] = -100.0 / (M.ri[i] * M.area[i]);
        M.a[i] = -100.0 / (M.ri[i] * M.area[p]);
      }
    }
  }
  M.spike_node.resize(M.n_cells);
  M.threshold.assign(s->threshold, s->threshold + M.n_cells);
  M.above.resize(M.n_cells);
  for (int c = 0; c < M.n_cells; ++c) {
    M.spike_node[c] = M.off[c] + s->spike_node[c];
    M.above[c] = M.v[M.spike_node[c]] > M.threshold[c];
  }
  std::vector<int32_t> cell_of(N);
  for (int c = 0; c < M.n_cells; ++c)
    for (int i = M.off[c]; i < M.off[c + 1]; ++i) cell_of[i] = c;

  for (int t = 0; t < s->n_mech; ++t) {
    const or_mech_in& in = s->mechs[t];
    if (in.kind < 0 || in.kind >= OR_NKINDS) { M.err = "bad mechanism kind"; return false; }
    Mech& m = M.mech[in.kind];
    if (m.kind >= 0) { M.err = "duplicate mechanism kind"; return false; }
    m.kind = in.kind;
    m.n = in.n;
    m.node.assign(in.node, in.node + in.n);
    int np = kNParam[in.kind];
    m.P.assign(np, std::vector<double>(in.n));
    for (int p = 0; p < np; ++p)
      for (int i = 0; i < in.n; ++i) m.P[p][i] = in.param[(int64_t)p * in.n + i];
    m.cell_start.assign(M.n_cells + 1, 0);
    for (int i = 0; i < in.n; ++i) m.cell_start[cell_of[m.node[i]] + 1]++;
    for (int c = 0; c < M.n_cells; ++c) m.cell_start[c + 1] += m.cell_start[c];
    m.by_cell.resize(in.n);
    std::vector<int32_t> fill(m.cell_start.begin(), m.cell_start.end() - 1);
    for (int i = 0; i < in.n; ++i) m.by_cell[fill[cell_of[m.node[i]]]++] = i;
  }
  // Initial states: steady state at v_init.
  for (int k = 0; k < OR_NKINDS; ++k) {
    Mech& m = M.mech[k];
    if (m.kind < 0) continue;
    std::vector<std::vector<double>>& S = m.S;
    switch (k) {
      case OR_HH: {
        S.assign(3, std::vector<double>(m.n));
        for (int i = 0; i < m.n; ++i) {
          double am, bm, ah, bh, an, bn;
          hh_rates(M.v[m.node[i]], &am, &bm, &ah, &bh, &an, &bn);
          S[0][i] = steady(am, bm); S[1][i] = steady(ah, bh); S[2][i] = steady(an, bn);
        }
        break;
      }
      case OR_EXPSYN: S.assign(1, std::vector<double>(m.n, 0.0)); break;
      case OR_NA3H: case OR_KA: case OR_CAHVA: {
        S.assign(2, std::vector<double>(m.n));
        for (int i = 0; i < m.n; ++i) {
          double v = M.v[m.node[i]];
          Gate6 g1 = gate_at(m.P, 2, i), g2 = gate_at(m.P, 8, i);
          S[0][i] = steady(galpha(g1, v), gbeta(g1, v));
          S[1][i] = steady(galpha(g2, v), gbeta(g2, v));
        }
        if (k == OR_CAHVA) {
          m.ica.assign(m.n, 0.0);
          for (int i = 0; i < m.n; ++i) M.cai[m.node[i]] = m.P[16][i];
        }
        break;
      }
      case OR_KDR4: case OR_IH: {
        S.assign(1, std::vector<double>(m.n));
        for (int i = 0; i < m.n; ++i) {
          double v = M.v[m.node[i]];
          Gate6 g1 = gate_at(m.P, 2, i);
          S[0][i] = steady(galpha(g1, v), gbeta(g1, v));
        }
        break;
      }
      default: break;
    }
  }
  if (M.mech[OR_KCA].kind >= 0) {
    Mech& m = M.mech[OR_KCA];
    m.S.assign(1, std::vector<double>(m.n));
    for (int i = 0; i < m.n; ++i) {
      double cai = M.cai[m.node[i]];
      double al = m.P[2][i] * cai / (cai + m.P[3][i]);
      m.S[0][i] = steady(al, m.P[4][i]);
    }
  }
  // Synapse -> cell.
  Mech& syn = M.mech[OR_EXPSYN];
  M.syn_cell.resize(syn.kind >= 0 ? syn.n : 0);
  for (size_t i = 0; i < M.syn_cell.size(); ++i) M.syn_cell[i] = cell_of[syn.node[i]];
  // Stimuli.
  M.st_node.assign(s->stim_node, s->stim_node + s->n_stim);
  M.st_del.assign(s->stim_del, s->stim_del + s->n_stim);
  M.st_dur.assign(s->stim_dur, s->stim_dur + s->n_stim);
  M.st_amp.assign(s->stim_amp, s->stim_amp + s->n_stim);
  M.cell_stims.assign(M.n_cells, {});
  for (int i = 0; i < s->n_stim; ++i) M.cell_stims[cell_of[M.st_node[i]]].push_back(i);
  // Gap junctions.
  M.gap_node.assign(s->gap_node, s->gap_node + s->n_gap);
  M.gap_peer.assign(s->gap_peer, s->gap_peer + s->n_gap);
  M.gap_g.assign(s->gap_g, s->gap_g + s->n_gap);
  M.gap_vpeer.assign(s->n_gap, 0.0);
  M.cell_gaps.assign(M.n_cells, {});
  for (int64_t i = 0; i < s->n_gap; ++i) {
    if (M.gap_node[i] < 0 || M.gap_node[i] >= N || M.gap_peer[i] < 0 || M.gap_peer[i] >= N) {
      M.err = "bad gap junction";
      return false;
    }
    M.cell_gaps[cell_of[M.gap_node[i]]].push_back((int32_t)i);
  }
  // NetCons: CSR by source in index order.
  M.nc_start.assign(M.n_cells + 1, 0);
  for (int64_t j = 0; j < s->n_netcon; ++j) {
    if (s->nc_src[j] < 0 || s->nc_src[j] >= M.n_cells || s->nc_syn[j] < 0 ||
        s->nc_syn[j] >= (int64_t)M.syn_cell.size()) { M.err = "bad netcon"; return false; }
    M.nc_start[s->nc_src[j] + 1]++;
  }
  for (int c = 0; c < M.n_cells; ++c) M.nc_start[c + 1] += M.nc_start[c];
  M.nc_idx.resize(s->n_netcon);
  {
    std::vector<int64_t> fill(M.nc_start.begin(), M.nc_start.end() - 1);
    for (int64_t j = 0; j < s->n_netcon; ++j) M.nc_idx[fill[s->nc_src[j]]++] = j;
  }
  M.nc_syn.assign(s->nc_syn, s->nc_syn + s->n_netcon);
  M.nc_w.assign(s->nc_w, s->nc_w + s->n_netcon);
  M.nc_dsteps.resize(s->n_netcon);
  M.min_delay = 0;
  for (int64_t j = 0; j < s->n_netcon; ++j) {
    M.nc_dsteps[j] = std::lround(s->nc_delay[j] / s->dt);
    if (M.nc_dsteps[j] < 1) { M.err = "NetCon delay below one step"; return false; }
    if (M.min_delay == 0 || M.nc_dsteps[j] < M.min_delay) M.min_delay = M.nc_dsteps[j];
  }
  // External events.
  M.queue.assign(M.n_cells, {});
  for (int64_t e = 0; e < s->n_ev; ++e) {
    int32_t sy = s->ev_syn[e];
    if (sy < 0 || sy >= (int64_t)M.syn_cell.size()) { M.err = "bad event target"; return false; }
    int64_t k = std::lround(s->ev_t[e] / s->dt);
    if (k < 0) k = 0;
    M.queue[M.syn_cell[sy]][k].push_back(Ev{0, e, 0, sy, s->ev_w[e]});
  }
  M.rec_node.assign(s->rec_node, s->rec_node + s->n_rec);
  M.trace.assign(s->n_rec, {});
  M.cell_recs.assign(M.n_cells, {});
  for (int r = 0; r < s->n_rec; ++r) {
    if (M.rec_node[r] < 0 || M.rec_node[r] >= N) { M.err = "bad record node"; return false; }
    M.trace[r].push_back(M.v[M.rec_node[r]]);
    M.cell_recs[cell_of[M.rec_node[r]]].push_back(r);
  }
  return true;
}

// One backward-Euler step k -> k+1 of cell c.  Spikes are appended to out.
void cell_step(Model& M, int c, int64_t k, std::vector<std::pair<int64_t, int32_t>>& out) {
  const double dt = M.dt;
  const int i0 = M.off[c], i1 = M.off[c + 1];
  // (1) Event-driven delivery: synapse callbacks for events due at step k.
  auto& q = M.queue[c];
  auto it = q.find(k);
  if (it != q.end()) {
    std::vector<Ev>& evs = it->second;
    std::sort(evs.begin(), evs.end(), [](const Ev& x, const Ev& y) {
      if (x.kind != y.kind) return x.kind < y.kind;
      if (x.k1 != y.k1) return x.k1 < y.k1;
      return x.k2 < y.k2;
    });
    for (const Ev& e : evs) M.mech[OR_EXPSYN].S[0][e.syn] += e.w;
    q.erase(it);
  }
  // (2) Matrix assembly: currents I and conductances G of every mechanism at
  //     v_k go into rhs (as -I) and into the diagonal (as G).
  for (int i = i0; i < i1; ++i) { M.rhs[i] = 0.0; M.d[i] = 0.0; }
  for (int kind = 0; kind < OR_NKINDS; ++kind) {
    Mech& m = M.mech[kind];
    if (m.kind < 0) continue;
    for (int q2 = m.cell_start[c]; q2 < m.cell_start[c + 1]; ++q2) {
      int i = m.by_cell[q2];
      int nd = m.node[i];
      double v = M.v[nd];
      double I = 0.0, G = 0.0;
      switch (kind) {
        case OR_PAS: G = m.P[0][i]; I = G * (v - m.P[1][i]); break;
        case OR_HH: {
          double mm = m.S[0][i], hh = m.S[1][i], nn = m.S[2][i];
          double gna = m.P[0][i] * mm * mm * mm * hh;
          double gk = m.P[1][i] * nn * nn * nn * nn;
          double gl = m.P[2][i];
          I = gna * (v - m.P[4][i]) + gk * (v - m.P[5][i]) + gl * (v - m.P[3][i]);
          G = gna + gk + gl;
          break;
        }
        case OR_EXPSYN: {
          double g = m.S[0][i];
          // point current (nA) to density (mA/cm2): divide by area (um2), x100
          I = 100.0 * g * (v - m.P[1][i]) / M.area[nd];
          G = 100.0 * g / M.area[nd];
          break;
        }
        case OR_NA3H: case OR_KA: {
          double x = m.S[0][i], y = m.S[1][i];
          G = m.P[0][i] * x * x * x * y;
          I = G * (v - m.P[1][i]);
          break;
        }
        case OR_KDR4: { double x = m.S[0][i]; G = m.P[0][i] * x * x * x * x; I = G * (v - m.P[1][i]); break; }
        case OR_IH: { G = m.P[0][i] * m.S[0][i]; I = G * (v - m.P[1][i]); break; }
        case OR_CAHVA: {
          double x = m.S[0][i], y = m.S[1][i];
          G = m.P[0][i] * x * x * y;
          I = G * (v - m.P[1][i]);
          m.ica[i] = I;
          break;
        }
        case OR_KCA: { G = m.P[0][i] * m.S[0][i]; I = G * (v - m.P[1][i]); break; }
      }
      M.rhs[nd] -= I;
      M.d[nd] += G;
    }
  }
  // Gap junctions: I = g (v - v_peer,k), the peer voltage taken at the start
  // of the step (exchanged every step), the own voltage implicit.
  for (int gi : M.cell_gaps[c]) {
    int nd = M.gap_node[gi];
    double G = 100.0 * M.gap_g[gi] / M.area[nd];
    M.rhs[nd] -= G * (M.v[nd] - M.gap_vpeer[gi]);
    M.d[nd] += G;
  }
  const double tmid = (k + 0.5) * dt;
  for (int si : M.cell_stims[c]) {
    if (M.st_del[si] <= tmid && tmid < M.st_del[si] + M.st_dur[si]) {
      int nd = M.st_node[si];
      M.rhs[nd] += 100.0 * M.st_amp[si] / M.area[nd];
    }
  }
  //     Axial terms (Eq. 1's second derivative on the tree) and capacitance.
  for (int i = i0; i < i1; ++i) {
    int p = M.parent[i];
    if (p >= 0) {
      double dv = M.v[p] - M.v[i];
      M.rhs[i] -= M.b[i] * dv;
      M.rhs[p] += M.a[i] * dv;
      M.d[i] -= M.b[i];
      M.d[p] -= M.a[i];
    }
    M.d[i] += 1e-3 * M.cm[i] / dt;
  }
  // (3) Matrix resolution: Gaussian elimination in Hines order (leaves to
  //     root), back substitution (root to leaves), v += dv.
  for (int i = i1 - 1; i > i0; --i) {
    int p = M.parent[i];
    double f = M.a[i] / M.d[i];
    M.d[p] -= f * M.b[i];
    M.rhs[p] -= f * M.rhs[i];
  }
  M.rhs[i0] /= M.d[i0];
  for (int i = i0 + 1; i < i1; ++i) {
    int p = M.parent[i];
    M.rhs[i] = (M.rhs[i] - M.b[i] * M.rhs[p]) / M.d[i];
  }
  for (int i = i0; i < i1; ++i) M.v[i] += M.rhs[i];
  // (4) State update at v_{k+1} (cnexp).
  for (int kind = 0; kind < OR_NKINDS; ++kind) {
    Mech& m = M.mech[kind];
    if (m.kind < 0) continue;
    for (int q2 = m.cell_start[c]; q2 < m.cell_start[c + 1]; ++q2) {
      int i = m.by_cell[q2];
      int nd = m.node[i];
      double v = M.v[nd];
      switch (kind) {
        case OR_HH: {
          double am, bm, ah, bh, an, bn;
          hh_rates(v, &am, &bm, &ah, &bh, &an, &bn);
          m.S[0][i] = cnexp(m.S[0][i], am, bm, dt);
          m.S[1][i] = cnexp(m.S[1][i], ah, bh, dt);
          m.S[2][i] = cnexp(m.S[2][i], an, bn, dt);
          break;
        }
        case OR_EXPSYN: m.S[0][i] *= std::exp(-dt / m.P[0][i]); break;
        case OR_NA3H: case OR_KA: case OR_CAHVA: {
          Gate6 g1 = gate_at(m.P, 2, i), g2 = gate_at(m.P, 8, i);
          m.S[0][i] = cnexp(m.S[0][i], galpha(g1, v), gbeta(g1, v), dt);
          m.S[1][i] = cnexp(m.S[1][i], galpha(g2, v), gbeta(g2, v), dt);
          if (kind == OR_CAHVA) {
            double drive = -1e4 * m.ica[i] / (2.0 * kFaraday * m.P[14][i]);
            if (drive < 0.0) drive = 0.0;
            double taur = m.P[15][i];
            double target = m.P[16][i] + drive * taur;
            double cai = M.cai[nd];
            M.cai[nd] = cai + (1.0 - std::exp(-dt / taur)) * (target - cai);
          }
          break;
        }
        case OR_KDR4: case OR_IH: {
          Gate6 g1 = gate_at(m.P, 2, i);
          m.S[0][i] = cnexp(m.S[0][i], galpha(g1, v), gbeta(g1, v), dt);
          break;
        }
        case OR_KCA: {
          double cai = M.cai[nd];
          double al = m.P[2][i] * cai / (cai + m.P[3][i]);
          m.S[0][i] = cnexp(m.S[0][i], al, m.P[4][i], dt);
          break;
        }
        default: break;
      }
    }
  }
  // (5) Threshold detection at the spike source.
  double vs = M.v[M.spike_node[c]];
  bool now = vs > M.threshold[c];
  if (now && !M.above[c]) out.emplace_back(k + 1, c);
  M.above[c] = now;
}

// Spike exchange at an interval boundary: every spike of the interval, in
// (step, gid) order, queues one event per outgoing NetCon at the target.
void exchange(Model& M, std::vector<std::pair<int64_t, int32_t>>& spikes) {
  std::sort(spikes.begin(), spikes.end());
  for (auto& sp : spikes) {
    int64_t t = sp.first;
    int32_t g = sp.second;
    M.sp_gid.push_back(g);
    M.sp_step.push_back(t);
    for (int64_t q = M.nc_start[g]; q < M.nc_start[g + 1]; ++q) {
      int64_t j = M.nc_idx[q];
      int32_t sy = M.nc_syn[j];
      M.queue[M.syn_cell[sy]][t + M.nc_dsteps[j]].push_back(Ev{1, g, j, sy, M.nc_w[j]});
    }
  }
}

void run(Model& M, int64_t nsteps, int nthreads) {
  int64_t D = M.min_delay > 0 ? M.min_delay : 40;
  if (!M.gap_node.empty()) D = 1;  // gap junctions exchange voltages every step
  int64_t end = M.step + nsteps;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > M.n_cells) nthreads = std::max(1, M.n_cells);
  while (M.step < end) {
    // An interval ends at the next multiple of the minimum delay; within it
    // the cells are independent (every NetCon delay is at least D steps).
    int64_t stop = std::min(end, (M.step / D + 1) * D);
    int64_t k0 = M.step;
    for (size_t i = 0; i < M.gap_peer.size(); ++i) M.gap_vpeer[i] = M.v[M.gap_peer[i]];
    for (auto& tr : M.trace) tr.resize(stop + 1);
    std::vector<std::vector<std::pair<int64_t, int32_t>>> sp(nthreads);
    auto work = [&](int tid) {
      int c0 = (int)((int64_t)M.n_cells * tid / nthreads);
      int c1 = (int)((int64_t)M.n_cells * (tid + 1) / nthreads);
      for (int c = c0; c < c1; ++c)
        for (int64_t k = k0; k < stop; ++k) {
          cell_step(M, c, k, sp[tid]);
          for (int32_t r : M.cell_recs[c]) M.trace[r][k + 1] = M.v[M.rec_node[r]];
        }
    };
    if (nthreads == 1) {
      work(0);
    } else {
      std::vector<std::thread> th;
      for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
      for (auto& x : th) x.join();
    }
    std::vector<std::pair<int64_t, int32_t>> all;
    for (auto& v : sp) all.insert(all.end(), v.begin(), v.end());
    exchange(M, all);
    M.step = stop;
  }
}


// ------------------------------------------------------------------ adjoint
// Discrete adjoint of one cell's backward-Euler trajectory.  The forward map
// of step k is A_k v_{k+1} = C v_k + b_k with A_k = C + G_k + L (C = cdt,
// G_k the membrane conductances frozen at the gates of step k, L the axial
// couplings) and gates_{k+1} = Phi(gates_k, v_{k+1}) (cnexp).  With the loss
// J = sum_r sum_{k=1..K} (v_r,k - target_r,k)^2 over the cell's recorded
// nodes, walking k from K-1 down to 0:
//   mu_k     = A_k^-T lambda_{k+1}                       (Hines, a and b swapped)
//   xi_k     = dPhi_k/dgates_k xi_{k+1} + mu_s d(GE - G v_{s,k+1})/dgates_k
//   lambda_k = dJ/dv_k (direct) + C mu_k + (dPhi_{k-1}/dv_k)^T xi_k
// and parameter gradients mu_k . d(b_k - A_k v_{k+1})/dtheta.

// HH rate derivatives (same rates as hh_rates).
double vtrap_deriv(double A, double vh, double k, double v) {
  double u = (v - vh) / k;
  if (std::fabs(u) < 1e-6) return A * (0.5 + u / 3.0);
  double em = std::exp(-u);
  double den = 1.0 - em;
  return A * (den - u * em) / (den * den);
}

void hh_rate_derivs(double v, double* dam, double* dbm, double* dah, double* dbh, double* dan, double* dbn) {
  *dam = vtrap_deriv(0.1, -40.0, 10.0, v);
  *dbm = -4.0 * std::exp(-(v + 65.0) / 18.0) / 18.0;
  *dah = -0.07 * std::exp(-(v + 65.0) / 20.0) / 20.0;
  double bh = 1.0 / (1.0 + std::exp(-(v + 35.0) / 10.0));
  *dbh = bh * (1.0 - bh) / 10.0;
  *dan = vtrap_deriv(0.01, -55.0, 10.0, v);
  *dbn = -0.125 * std::exp(-(v + 65.0) / 80.0) / 80.0;
}

// d x_{k+1} / d v_{k+1} and d x_{k+1} / d x_k of the cnexp update.
void cnexp_derivs(double x, double al, double be, double dal, double dbe, double dt, double* dv, double* dx) {
  double s = al + be;
  double inf = al / s;
  double E = std::exp(-dt * s);
  double dinf = (dal * be - al * dbe) / (s * s);
  double dE = -dt * (dal + dbe) * E;
  *dv = dinf * (1.0 - E) + (x - inf) * dE;
  *dx = E;
}

struct CellSnap {
  std::vector<double> v;
  std::vector<std::vector<double>> hh;  // [3][instances of the cell]
  std::vector<double> syn;
};

void cell_adjoint(Model& M, int c, int64_t K, int seg, const double* target, const std::vector<int32_t>& recs,
                  double* J, double* g_na, double* g_k, double* g_pas) {
  const int i0 = M.off[c], i1 = M.off[c + 1], n = i1 - i0;
  const double dt = M.dt;
  Mech& hh = M.mech[OR_HH];
  Mech& pas = M.mech[OR_PAS];
  Mech& syn = M.mech[OR_EXPSYN];
  std::vector<int> hh_inst, pas_inst, syn_inst;
  if (hh.kind >= 0) for (int q = hh.cell_start[c]; q < hh.cell_start[c + 1]; ++q) hh_inst.push_back(hh.by_cell[q]);
  if (pas.kind >= 0) for (int q = pas.cell_start[c]; q < pas.cell_start[c + 1]; ++q) pas_inst.push_back(pas.by_cell[q]);
  if (syn.kind >= 0) for (int q = syn.cell_start[c]; q < syn.cell_start[c + 1]; ++q) syn_inst.push_back(syn.by_cell[q]);
  auto snap = [&]() {
    CellSnap s;
    s.v.assign(M.v.begin() + i0, M.v.begin() + i1);
    s.hh.assign(3, {});
    for (int g = 0; g < 3; ++g)
      for (int q : hh_inst) s.hh[g].push_back(hh.S[g][q]);
    for (int q : syn_inst) s.syn.push_back(syn.S[0][q]);
    return s;
  };
  auto restore = [&](const CellSnap& s) {
    std::copy(s.v.begin(), s.v.end(), M.v.begin() + i0);
    for (int g = 0; g < 3; ++g)
      for (size_t t = 0; t < hh_inst.size(); ++t) hh.S[g][hh_inst[t]] = s.hh[g][t];
    for (size_t t = 0; t < syn_inst.size(); ++t) syn.S[0][syn_inst[t]] = s.syn[t];
  };
  std::vector<std::pair<int64_t, int32_t>> dummy;
  // forward with checkpoints every `seg` steps; loss
  std::vector<CellSnap> cps;
  double loss = 0.0;
  for (int64_t k = 0; k < K; ++k) {
    if (k % seg == 0) cps.push_back(snap());
    cell_step(M, c, k, dummy);
    for (size_t r = 0; r < recs.size(); ++r) {
      double e = M.v[M.rec_node[recs[r]]] - target[(size_t)recs[r] * (K + 1) + (k + 1)];
      loss += e * e;
    }
  }
  *J = loss;
  // backward
  std::vector<double> lam(n, 0.0), mu(n), d(n), rhs(n);
  for (size_t r = 0; r < recs.size(); ++r) {
    int i = M.rec_node[recs[r]];
    lam[i - i0] += 2.0 * (M.v[i] - target[(size_t)recs[r] * (K + 1) + K]);
  }
  const int nh = (int)hh_inst.size();
  std::vector<double> xi(3 * nh, 0.0);
  for (int64_t sb = ((K - 1) / seg) * seg; sb >= 0; sb -= seg) {
    const int64_t se = std::min<int64_t>(K, sb + seg);
    // recompute v_k (all nodes) and gates_k for k in [sb, se]
    restore(cps[sb / seg]);
    std::vector<std::vector<double>> vs(se - sb + 1), gs(se - sb + 1), ss(se - sb + 1);
    auto record = [&](int64_t t) {
      vs[t].assign(M.v.begin() + i0, M.v.begin() + i1);
      gs[t].clear();
      for (int g = 0; g < 3; ++g)
        for (int q : hh_inst) gs[t].push_back(hh.S[g][q]);
      ss[t].clear();
      for (int q : syn_inst) ss[t].push_back(syn.S[0][q]);
    };
    record(0);
    for (int64_t k = sb; k < se; ++k) {
      cell_step(M, c, k, dummy);
      record(k - sb + 1);
    }
    for (int64_t k = se - 1; k >= sb; --k) {
      const std::vector<double>& vk1 = vs[k - sb + 1];
      const std::vector<double>& gk = gs[k - sb];
      // A_k: diagonal from the conductances of step k
      for (int i = 0; i < n; ++i) d[i] = 1e-3 * M.cm[i0 + i] / dt;
      for (int q : pas_inst) d[pas.node[q] - i0] += pas.P[0][q];
      for (int t = 0; t < nh; ++t) {
        int q = hh_inst[t];
        double m = gk[t], h = gk[nh + t], nn = gk[2 * nh + t];
        d[hh.node[q] - i0] += hh.P[0][q] * m * m * m * h + hh.P[1][q] * nn * nn * nn * nn + hh.P[2][q];
      }
      for (size_t t = 0; t < syn_inst.size(); ++t) {
        int q = syn_inst[t];
        int nd = syn.node[q];
        d[nd - i0] += 100.0 * ss[k - sb][t] / M.area[nd];
      }
      for (int i = 1; i < n; ++i) {
        int p = M.parent[i0 + i] - i0;
        d[i] -= M.b[i0 + i];
        d[p] -= M.a[i0 + i];
      }
      // transposed Hines solve: A^T has b where A has a and vice versa
      for (int i = 0; i < n; ++i) rhs[i] = lam[i];
      for (int i = n - 1; i > 0; --i) {
        int p = M.parent[i0 + i] - i0;
        double f = M.b[i0 + i] / d[i];
        d[p] -= f * M.a[i0 + i];
        rhs[p] -= f * rhs[i];
      }
      rhs[0] /= d[0];
      for (int i = 1; i < n; ++i) {
        int p = M.parent[i0 + i] - i0;
        rhs[i] = (rhs[i] - M.a[i0 + i] * rhs[p]) / d[i];
      }
      mu = rhs;
      // parameter gradients and the gates' adjoint
      for (int t = 0; t < nh; ++t) {
        int q = hh_inst[t];
        int si = hh.node[q] - i0;
        double vs1 = vk1[si];
        double m = gk[t], h = gk[nh + t], nn = gk[2 * nh + t];
        double ena = hh.P[4][q], ek = hh.P[5][q];
        g_na[q] += mu[si] * m * m * m * h * (ena - vs1);
        g_k[q] += mu[si] * nn * nn * nn * nn * (ek - vs1);
        double am, bm, ah, bh, an, bn, dam, dbm, dah, dbh, dan, dbn;
        hh_rates(vs1, &am, &bm, &ah, &bh, &an, &bn);
        double dvx, Em, Eh, En;
        cnexp_derivs(m, am, bm, 0, 0, dt, &dvx, &Em);
        cnexp_derivs(h, ah, bh, 0, 0, dt, &dvx, &Eh);
        cnexp_derivs(nn, an, bn, 0, 0, dt, &dvx, &En);
        (void)dam; (void)dbm; (void)dah; (void)dbh; (void)dan; (void)dbn;
        double gna = hh.P[0][q], gkb = hh.P[1][q];
        double xm = Em * xi[t] + mu[si] * gna * 3.0 * m * m * h * (ena - vs1);
        double xh = Eh * xi[nh + t] + mu[si] * gna * m * m * m * (ena - vs1);
        double xn = En * xi[2 * nh + t] + mu[si] * gkb * 4.0 * nn * nn * nn * (ek - vs1);
        xi[t] = xm;
        xi[nh + t] = xh;
        xi[2 * nh + t] = xn;
      }
      for (int q : pas_inst) {
        int i = pas.node[q] - i0;
        g_pas[q] += mu[i] * (pas.P[1][q] - vk1[i]);
      }
      // lambda_k
      const std::vector<double>& vk = vs[k - sb];
      for (int i = 0; i < n; ++i) lam[i] = 1e-3 * M.cm[i0 + i] / dt * mu[i];
      if (k >= 1) {
        for (size_t r = 0; r < recs.size(); ++r) {
          int i = M.rec_node[recs[r]];
          lam[i - i0] += 2.0 * (vk[i - i0] - target[(size_t)recs[r] * (K + 1) + k]);
        }
        // gates_k = Phi(gates_{k-1}, v_k): needs gates_{k-1}
        if (nh > 0) {
          std::vector<double> gprev;
          if (k - 1 >= sb) gprev = gs[k - 1 - sb];
          else {  // previous segment's last gate state: recompute it from its checkpoint
            CellSnap cur = snap();
            restore(cps[(k - 1) / seg]);
            for (int64_t kk = ((k - 1) / seg) * seg; kk < k - 1; ++kk) cell_step(M, c, kk, dummy);
            for (int g = 0; g < 3; ++g)
              for (int q : hh_inst) gprev.push_back(hh.S[g][q]);
            restore(cur);
          }
          for (int t = 0; t < nh; ++t) {
            int q = hh_inst[t];
            int si = hh.node[q] - i0;
            double vv = vk[si];
            double am, bm, ah, bh, an, bn, dam, dbm, dah, dbh, dan, dbn;
            hh_rates(vv, &am, &bm, &ah, &bh, &an, &bn);
            hh_rate_derivs(vv, &dam, &dbm, &dah, &dbh, &dan, &dbn);
            double dvm, dvh, dvn, e_;
            cnexp_derivs(gprev[t], am, bm, dam, dbm, dt, &dvm, &e_);
            cnexp_derivs(gprev[nh + t], ah, bh, dah, dbh, dt, &dvh, &e_);
            cnexp_derivs(gprev[2 * nh + t], an, bn, dan, dbn, dt, &dvn, &e_);
            lam[si] += xi[t] * dvm + xi[nh + t] * dvh + xi[2 * nh + t] * dvn;
          }
        }
      }
    }
  }
}

}  // namespace

extern "C" {

void* or_create(const or_scenario* s, char* errbuf, int errlen) {
  Model* M = new Model();
  if (!build(*M, s)) {
    if (errbuf && errlen > 0) std::snprintf(errbuf, errlen, "%s", M->err.c_str());
    delete M;
    return nullptr;
  }
  return M;
}

void or_destroy(void* h) { delete static_cast<Model*>(h); }

int or_run(void* h, int64_t nsteps, int nthreads) {
  Model* M = static_cast<Model*>(h);
  if (nsteps < 0) return -1;
  run(*M, nsteps, nthreads);
  return 0;
}

int64_t or_step_index(void* h) { return static_cast<Model*>(h)->step; }
int64_t or_min_delay(void* h) { return static_cast<Model*>(h)->min_delay; }

int64_t or_spike_count(void* h) { return (int64_t) static_cast<Model*>(h)->sp_gid.size(); }

void or_get_spikes(void* h, int32_t* gid, int64_t* step) {
  Model* M = static_cast<Model*>(h);
  for (size_t i = 0; i < M->sp_gid.size(); ++i) { gid[i] = M->sp_gid[i]; step[i] = M->sp_step[i]; }
}

// trace of recorded node r: v at steps 0..step_index
void or_get_trace(void* h, int32_t r, double* out) {
  Model* M = static_cast<Model*>(h);
  std::memcpy(out, M->trace[r].data(), sizeof(double) * M->trace[r].size());
}

void or_get_v(void* h, double* out) {
  Model* M = static_cast<Model*>(h);
  std::memcpy(out, M->v.data(), sizeof(double) * M->v.size());
}

void or_get_cai(void* h, double* out) {
  Model* M = static_cast<Model*>(h);
  std::memcpy(out, M->cai.data(), sizeof(double) * M->cai.size());
}

// Overwrite [Ca]i of every node (a perturbation for the pins: without a
// CAHVA instance nothing else changes cai, so the KCa gate then relaxes at
// fixed rates).
void or_set_cai(void* h, const double* in) {
  Model* M = static_cast<Model*>(h);
  std::memcpy(M->cai.data(), in, sizeof(double) * M->cai.size());
}

// state column `col` of mechanism `kind` (HH: m,h,n; expsyn: g; ...)
int or_get_state(void* h, int32_t kind, int32_t col, double* out) {
  Model* M = static_cast<Model*>(h);
  if (kind < 0 || kind >= OR_NKINDS) return -1;
  Mech& m = M->mech[kind];
  if (m.kind < 0 || col < 0 || col >= (int)m.S.size()) return -1;
  std::memcpy(out, m.S[col].data(), sizeof(double) * m.n);
  return 0;
}

// Area and axial resistance per node as the oracle derives them.
void or_get_geometry(void* h, double* area, double* ri) {
  Model* M = static_cast<Model*>(h);
  std::memcpy(area, M->area.data(), sizeof(double) * M->area.size());
  std::memcpy(ri, M->ri.data(), sizeof(double) * M->ri.size());
}

// Stand-alone Hines solve of one tree matrix (row i: diagonal d[i],
// coupling b[i] to parent p; row p: coupling a[i] to child i), in place:
// on return rhs holds the solution.  Used to pin the elimination against a
// dense solver.
void or_hines_solve(int32_t n, const int32_t* parent, const double* a, const double* b, double* d,
                    double* rhs) {
  for (int i = n - 1; i > 0; --i) {
    int p = parent[i];
    double f = a[i] / d[i];
    d[p] -= f * b[i];
    rhs[p] -= f * rhs[i];
  }
  rhs[0] /= d[0];
  for (int i = 1; i < n; ++i) rhs[i] = (rhs[i] - b[i] * rhs[parent[i]]) / d[i];
}

// Adjoint of J = sum over recorded nodes and steps 1..K of (v - target)^2 for
// a network without NetCons: target is [n_rec][K+1]; gradients with respect
// to every HH instance's gnabar and gkbar and every pas instance's g.
// Checkpoints every `seg` steps, recomputed forward per segment.
int or_adjoint(const or_scenario* s, int64_t K, const double* target, int32_t seg, int nthreads, double* J,
               double* g_na, double* g_k, double* g_pas, char* errbuf, int errlen) {
  Model M;
  if (!build(M, s)) {
    if (errbuf && errlen > 0) std::snprintf(errbuf, errlen, "%s", M.err.c_str());
    return -1;
  }
  if (s->n_netcon > 0 || seg < 1 || K < 1) {
    if (errbuf && errlen > 0) std::snprintf(errbuf, errlen, "adjoint needs no NetCons, seg >= 1, K >= 1");
    return -1;
  }
  std::vector<std::vector<int32_t>> cell_rec(M.n_cells);
  for (int r = 0; r < s->n_rec; ++r) {
    int c = 0;
    while (M.off[c + 1] <= M.rec_node[r]) ++c;
    cell_rec[c].push_back(r);
  }
  if (M.mech[OR_HH].kind >= 0) {
    std::fill(g_na, g_na + M.mech[OR_HH].n, 0.0);
    std::fill(g_k, g_k + M.mech[OR_HH].n, 0.0);
  }
  if (M.mech[OR_PAS].kind >= 0) std::fill(g_pas, g_pas + M.mech[OR_PAS].n, 0.0);
  std::vector<double> Jc(M.n_cells, 0.0);
  if (nthreads < 1) nthreads = 1;
  auto work = [&](int tid) {
    for (int c = tid; c < M.n_cells; c += nthreads)
      cell_adjoint(M, c, K, seg, target, cell_rec[c], &Jc[c], g_na, g_k, g_pas);
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
  for (auto& x : th) x.join();
  double tot = 0.0;
  for (double x : Jc) tot += x;
  *J = tot;
  return 0;
}

}  // extern "C"
