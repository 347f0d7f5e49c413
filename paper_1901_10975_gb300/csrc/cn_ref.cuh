// cn_ref.cuh -- the reference layouts: the paper's two GPU node orderings
// (Section 4.4), run with the fixed-step update written in its plain
// sequential form (Section 2).
//
// Both layouts put 32 cells in a warp group and process the group's nodes
// row by row, one node per lane:
//  * interleaved: cell p of the group sits in lane p, its node i (input
//    order, parent[i] < i) at row i -- one cell per thread;
//  * constant depth: the group's nodes level by level (distance from the
//    root), within a level by (cell-local index, cell), 32 to a row, never two
//    children of one parent in one row.
// In either, a node's parent lies in an earlier row of the group, and the
// children of a node lie in later rows in increasing input order.  So walking
// the rows forwards (assembly, back substitution) and backwards (elimination)
// applies every update to a node in the same order as a sequential per-cell
// stepper: mechanism currents in type then instance order, then the node's
// own axial link and capacitance, then its children's links; elimination
// children in decreasing index order.  Every operation is a separately
// rounded IEEE operation (__dadd_rn and friends: no contraction into FMAs),
// and divisions are IEEE divisions.  The matrix is assembled in the
// linearised form of Section 2: rhs = -I(v) + axial currents, d = C + G +
// couplings, then v += the solution.
#pragma once
#include "cn_device.cuh"

namespace cn {
namespace ref {

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dv_(double a, double b) { return __ddiv_rn(a, b); }

// alpha = A (v - vh) / (1 - exp(-(v - vh)/k)); A k (1 + u/2) near vh.
__device__ __forceinline__ double vtrap(double A, double vh, double k, double v) {
  const double u = dv_(sub(v, vh), k);
  if (fabs(u) < 1e-6) return mul(mul(A, k), add(1.0, dv_(u, 2.0)));
  return dv_(mul(A, sub(v, vh)), sub(1.0, exp(-u)));
}

// Hodgkin-Huxley rates (6.3 C, q10 = 1).
__device__ __forceinline__ void hh_rates(double v, double& am, double& bm, double& ah, double& bh, double& an,
                                         double& bn) {
  am = vtrap(0.1, -40.0, 10.0, v);
  bm = mul(4.0, exp(dv_(-add(v, 65.0), 18.0)));
  ah = mul(0.07, exp(dv_(-add(v, 65.0), 20.0)));
  bh = dv_(1.0, add(1.0, exp(dv_(-add(v, 35.0), 10.0))));
  an = vtrap(0.01, -55.0, 10.0, v);
  bn = mul(0.125, exp(dv_(-add(v, 65.0), 80.0)));
}

// cnexp over dt at fixed v: tau = 1/(alpha+beta), x_inf = alpha tau,
// x + (1 - exp(-dt/tau)) (x_inf - x).
__device__ __forceinline__ double cnexp(double x, double al, double be, double dt) {
  const double tau = dv_(1.0, add(al, be));
  const double inf = mul(al, tau);
  return add(x, mul(sub(1.0, exp(dv_(-dt, tau))), sub(inf, x)));
}

}  // namespace ref

// One warp per group of 32 cells advances steps [s_begin, s_end) of
// interval J.  Per-row arrays (element g_node_base[g] + row*32 + lane):
// v; rhs (in M.bp) and d (in M.d0_syn) as per-step scratch; the unscaled
// couplings a (row parent, column node) and b (row node, column parent);
// cdt = 1e-3 cm/dt; area; flags (real node, pas); ref_par, the parent's
// element offset within the group (-1 at roots and padding).
__global__ void __launch_bounds__(32) k_interval_ref(DevModel M, int64_t J, int s_begin, int s_end,
                                                     const int64_t* Jp) {
  using namespace ref;
  if (Jp) J = *Jp;
  const int g = blockIdx.x;
  if (g >= M.n_groups) return;
  const int lane = threadIdx.x;
  const int slot = g * kLanes + lane;
  const int R = M.g_rows[g];
  const int64_t nb0 = M.g_node_base[g], nb = nb0 + lane;
  const int gid = M.s_gid[slot];
  double* const V = M.v;
  double* const RHS = M.bp;
  double* const Dg = M.d0_syn;
  const int SYR = M.g_syn_rows[g];
  const int64_t sb = M.g_syn_base[g] + lane;
  const int HR = M.g_hh_rows[g], nhh = M.s_nhh[slot];
  const int64_t hb = M.g_hh_base[g] + lane;
  const int STR = M.g_st_rows[g], nst = M.s_nst[slot];
  const int64_t stb = M.g_st_base[g] + lane;
  const int RR = M.g_rec_rows[g], nrec = M.s_nrec[slot];
  const int64_t rcb = M.g_rec_base[g] + lane;
  const double dt = M.dt;
  const int64_t T0 = J * M.D;
  const int spike_row = M.s_spike_row[slot];
  const double thresh = M.s_thresh[slot];
  int above = M.s_above[slot];
  uint64_t mask = (s_begin > 0 && gid >= 0) ? M.hist[J * M.n_cells + gid] : 0ull;
  const EvRec* ev = M.ev_buf + M.ev_off[slot];
  const int ne = M.ev_count[slot];
  int ei = 0;
  while (ei < ne && ev[ei].step < s_begin) ++ei;
  double* const gm = static_cast<double*>(M.hh_m);
  double* const gh = static_cast<double*>(M.hh_h);
  double* const gn = static_cast<double*>(M.hh_n);

  for (int s = s_begin; s < s_end; ++s) {
    const int64_t k = T0 + s;
    // (1) event delivery, in buffer order
    while (ei < ne && ev[ei].step == s) {
      M.syn_g[sb - lane + ev[ei].syn] += ev[ei].w;
      ++ei;
    }
    // (2) currents and conductances at v_k into rhs (as -I) and d (as G):
    //     pas, then HH, then ExpSyn, then IClamp
    for (int r = 0; r < R; ++r) {
      const int64_t e = nb + (int64_t)r * kLanes;
      const int f = M.flags[e];
      double rhs = 0.0, d = 0.0;
      if (f & kHasPasBit) {
        const double G = M.pas_g[e];
        rhs = sub(rhs, mul(G, sub(V[e], M.pas_e[e])));
        d = add(d, G);
      }
      RHS[e] = rhs;
      Dg[e] = d;
    }
    for (int q = 0; q < HR; ++q) {
      if (q < nhh) {
        const int64_t i = hb + (int64_t)q * kLanes;
        const int64_t e = nb + (int64_t)M.hh_row[i] * kLanes;
        const double* P = M.hh_raw;  // gnabar gkbar gl el ena ek
        const int64_t H = M.hh_elems;
        const double mm = gm[i], hh = gh[i], nn = gn[i], v = V[e];
        const double gna = mul(mul(mul(mul(P[i], mm), mm), mm), hh);
        const double gk = mul(mul(mul(mul(P[H + i], nn), nn), nn), nn);
        const double gl = P[2 * H + i];
        const double I = add(add(mul(gna, sub(v, P[4 * H + i])), mul(gk, sub(v, P[5 * H + i]))),
                             mul(gl, sub(v, P[3 * H + i])));
        RHS[e] = sub(RHS[e], I);
        Dg[e] = add(Dg[e], add(add(gna, gk), gl));
      }
    }
    __syncwarp();
    // a target's synapses are consecutive entries of one column (one lane)
    for (int q = 0; q < SYR; ++q) {
      const int64_t i = sb + (int64_t)q * kLanes;
      const int t = M.syn_tgt[i];
      if (t >= 0) {
        const int64_t e = nb0 + (t & kSynTgtMask);
        const double gs = M.syn_g[i], ar = M.area[e];
        RHS[e] = sub(RHS[e], dv_(mul(mul(100.0, gs), sub(V[e], M.syn_e[i])), ar));
        Dg[e] = add(Dg[e], dv_(mul(100.0, gs), ar));
      }
    }
    __syncwarp();
    if (STR > 0) {
      const double tmid = mul(add((double)k, 0.5), dt);
      for (int q = 0; q < STR; ++q) {
        if (q < nst) {
          const int64_t i = stb + (int64_t)q * kLanes;
          if (M.st_del[i] <= tmid && tmid < add(M.st_del[i], M.st_dur[i])) {
            const int64_t e = nb + (int64_t)M.st_row[i] * kLanes;
            RHS[e] = add(RHS[e], dv_(mul(100.0, M.st_amp[i]), M.area[e]));
          }
        }
      }
    }
    __syncwarp();
    // axial currents and capacitance, rows in order: a node's own link and
    // cdt, then (from later rows) its children's links
    for (int r = 0; r < R; ++r) {
      const int64_t e = nb + (int64_t)r * kLanes;
      if (M.flags[e] & kRealBit) {
        const int p = M.ref_par[e];
        if (p >= 0) {
          const int64_t pe = nb0 + p;
          const double dvv = sub(V[pe], V[e]);
          RHS[e] = sub(RHS[e], mul(M.b[e], dvv));
          RHS[pe] = add(RHS[pe], mul(M.a[e], dvv));
          Dg[e] = sub(Dg[e], M.b[e]);
          Dg[pe] = sub(Dg[pe], M.a[e]);
        }
        Dg[e] = add(Dg[e], M.cdt[e]);
      }
      __syncwarp();
    }
    // (3) Gaussian elimination leaves to root (rows backwards), then back
    //     substitution root to leaves, then v += the solution
    for (int r = R - 1; r >= 0; --r) {
      const int64_t e = nb + (int64_t)r * kLanes;
      const int p = (M.flags[e] & kRealBit) ? M.ref_par[e] : -1;
      if (p >= 0) {
        const int64_t pe = nb0 + p;
        const double fct = dv_(M.a[e], Dg[e]);
        Dg[pe] = sub(Dg[pe], mul(fct, M.b[e]));
        RHS[pe] = sub(RHS[pe], mul(fct, RHS[e]));
      }
      __syncwarp();
    }
    for (int r = 0; r < R; ++r) {
      const int64_t e = nb + (int64_t)r * kLanes;
      if (M.flags[e] & kRealBit) {
        const int p = M.ref_par[e];
        RHS[e] = p < 0 ? dv_(RHS[e], Dg[e]) : dv_(sub(RHS[e], mul(M.b[e], RHS[nb0 + p])), Dg[e]);
      }
      __syncwarp();
    }
    for (int r = 0; r < R; ++r) {
      const int64_t e = nb + (int64_t)r * kLanes;
      if (M.flags[e] & kRealBit) V[e] = add(V[e], RHS[e]);
    }
    __syncwarp();
    // (4) states at v_{k+1}: HH gates by cnexp, ExpSyn decay
    for (int q = 0; q < HR; ++q) {
      if (q < nhh) {
        const int64_t i = hb + (int64_t)q * kLanes;
        const double v = V[nb + (int64_t)M.hh_row[i] * kLanes];
        double am, bm, ah, bh, an, bn;
        hh_rates(v, am, bm, ah, bh, an, bn);
        gm[i] = cnexp(gm[i], am, bm, dt);
        gh[i] = cnexp(gh[i], ah, bh, dt);
        gn[i] = cnexp(gn[i], an, bn, dt);
      }
    }
    for (int q = 0; q < SYR; ++q) {
      const int64_t i = sb + (int64_t)q * kLanes;
      if (M.syn_tgt[i] >= 0) M.syn_g[i] = mul(M.syn_g[i], M.syn_decay[i]);
    }
    __syncwarp();
    // (5) threshold detection and recording
    if (spike_row >= 0 && gid >= 0) {
      const double vs = V[nb + (int64_t)spike_row * kLanes];
      const int now = vs > thresh;
      if (now && !above) mask |= 1ull << s;
      above = now;
    }
    for (int q = 0; q < RR; ++q) {
      if (q < nrec) {
        const int64_t i = rcb + (int64_t)q * kLanes;
        M.trace[(k + 1) * M.n_rec + M.rec_id[i]] = V[nb + (int64_t)M.rec_row[i] * kLanes];
      }
    }
  }
  if (gid >= 0) {
    M.hist[J * M.n_cells + gid] = mask;
    M.s_above[slot] = (uint8_t)above;
  }
}

}  // namespace cn
