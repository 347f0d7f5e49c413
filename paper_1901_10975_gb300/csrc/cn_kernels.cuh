// cn_kernels.cuh -- setup, spike-pull and interval kernels.
#pragma once
#include "cn_device.cuh"

namespace cn {

// ------------------------------------------------------------------ setup
// Matrix constants of every node (Eq. 1 discretised on the tree):
//   b_i = -100/(ri_i area_i)   (row i, column parent)
//   a_i = -100/(ri_i area_p)   (row parent, column i)
//   d0_i = 1e-3 cm_i/dt + sum(pas g) + sum of axial couplings of row i
//   ge_i = pas g e
// and the initial state v = v_init, acc = ge, dacc = d0.
__global__ void k_setup_nodes(DevModel M, const double* area, const double* ri, const double* cm,
                              const double* gpas, const double* epas, double v_init) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int N = M.s_rows[slot];
  const int64_t nb = M.g_node_base[g] + lane;
  double* d0 = const_cast<double*>(M.d0);
  double* a = const_cast<double*>(M.a);
  double* b = const_cast<double*>(M.b);
  double* cdt = const_cast<double*>(M.cdt);
  double* ge = const_cast<double*>(M.ge);
  for (int j = 0; j < N; ++j) {
    const int64_t i = nb + (int64_t)j * kLanes;
    cdt[i] = 1e-3 * cm[i] / M.dt;
    d0[i] = cdt[i] + gpas[i];
    ge[i] = gpas[i] * epas[i];
    a[i] = 0.0;
    b[i] = 0.0;
  }
  for (int j = 1; j < N; ++j) {
    const int64_t i = nb + (int64_t)j * kLanes;
    const int64_t ip = nb + (int64_t)M.prow[i] * kLanes;
    b[i] = -100.0 / (ri[i] * area[i]);
    a[i] = -100.0 / (ri[i] * area[ip]);
    d0[i] -= b[i];
    d0[ip] -= a[i];
  }
  for (int j = 0; j < N; ++j) {
    const int64_t i = nb + (int64_t)j * kLanes;
    M.v[i] = v_init;
    M.acc[i] = ge[i];
    M.dacc[i] = d0[i];
  }
}

// ExpSyn constants: s = 100/area (nA -> mA/cm2), decay = exp(-dt/tau), g = 0.
__global__ void k_setup_syn(DevModel M, const double* node_area, const double* tau) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int n = M.s_nsyn[slot];
  const int64_t base = M.g_syn_base[g] + lane;
  for (int q = 0; q < n; ++q) {
    const int64_t i = base + (int64_t)q * kLanes;
    const_cast<double*>(M.syn_s)[i] = 100.0 / node_area[i];
    const_cast<double*>(M.syn_decay)[i] = exp(-M.dt / tau[i]);
    M.syn_g[i] = 0.0;
  }
}

// HH gates at their steady state of v_init.
template <int PREC>
__global__ void k_setup_hh(DevModel M, double v_init) {
  using S = typename GateT<PREC>::S;
  using T = typename GateT<PREC>::M;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int n = M.s_nhh[slot];
  const int64_t base = M.g_hh_base[g] + lane;
  for (int q = 0; q < n; ++q) {
    const int64_t i = base + (int64_t)q * kLanes;
    T am, bm, ah, bh, an, bn;
    hh_rates<T>(T(v_init), am, bm, ah, bh, an, bn);
    g_store(static_cast<S*>(M.hh_m) + i, am / (am + bm));
    g_store(static_cast<S*>(M.hh_h) + i, ah / (ah + bh));
    g_store(static_cast<S*>(M.hh_n) + i, an / (an + bn));
  }
}

// IClamp amplitude as a density: 100 amp / area (mA/cm2).
__global__ void k_setup_stim(DevModel M, const double* amp, const double* node_area) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int n = M.s_nst[slot];
  const int64_t base = M.g_st_base[g] + lane;
  for (int q = 0; q < n; ++q) {
    const int64_t i = base + (int64_t)q * kLanes;
    const_cast<double*>(M.st_amp)[i] = 100.0 * amp[i] / node_area[i];
  }
}

// ------------------------------------------------------- interval boundary
// Spike exchange at the start of interval J (Section 2: spikes are exchanged
// once per minimum delay).  Each cell pulls, from the spike masks of earlier
// intervals, every NetCon event due in [J D, J D + D), and its external
// events for the same window, into its event buffer ordered by (step,
// external-before-NetCon, input index | source gid, NetCon index).  No
// atomics: the result is deterministic.
__global__ void k_pull_events(DevModel M, int64_t J) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  EvRec* out = M.ev_buf + (int64_t)slot * kEvCap;
  if (M.s_gid[slot] < 0) {
    M.ev_count[slot] = 0;
    return;
  }
  const int D = M.D;
  const int64_t T = J * D;
  int n = 0;
  bool overflow = false;
  // external events (sorted by step, then input order)
  int64_t p = M.x_pos[slot];
  const int64_t pe = M.x_off[slot + 1];
  while (p < pe && M.x_step[p] < T + D) {
    if (M.x_step[p] >= T) {
      if (n < kEvCap) out[n] = EvRec{(int32_t)(M.x_step[p] - T), M.x_syn[p], M.x_w[p]};
      else overflow = true;
      ++n;
    }
    ++p;
  }
  M.x_pos[slot] = p;
  // NetCon events: a spike at step t reaches the target at t + dsteps.
  for (int64_t q = M.in_off[slot]; q < M.in_off[slot + 1]; ++q) {
    const int src = M.in_src[q];
    const int ds = M.in_dsteps[q];
    int64_t lo = T - ds, hi = T + D - ds;  // spike steps [lo, hi)
    if (lo < 1) lo = 1;
    if (hi <= lo) continue;
    const int64_t I0 = (lo - 1) / D, I1 = (hi - 2) / D;
    for (int64_t I = I0; I <= I1; ++I) {
      uint64_t mk = M.hist[I * M.n_cells + src];
      const int64_t t0 = lo > I * D + 1 ? lo : I * D + 1;
      const int64_t t1 = hi < (I + 1) * D + 1 ? hi : (I + 1) * D + 1;  // exclusive
      const int b0 = (int)(t0 - 1 - I * D), b1 = (int)(t1 - 1 - I * D);
      if (b1 <= b0) continue;
      mk >>= b0;
      if (b1 - b0 < 64) mk &= ((1ull << (b1 - b0)) - 1ull);
      while (mk) {
        const int bit = __ffsll((long long)mk) - 1;
        mk &= mk - 1ull;
        const int64_t t = I * D + 1 + b0 + bit;
        if (n < kEvCap) out[n] = EvRec{(int32_t)(t + ds - T), M.in_syn[q], M.in_w[q]};
        else overflow = true;
        ++n;
      }
    }
  }
  const int m = n < kEvCap ? n : kEvCap;
  // Stable insertion sort by step: externals were appended first (in step
  // order), NetCon events after them in (source gid, NetCon index) order, so
  // ties keep exactly the delivery order described above.
  for (int i = 1; i < m; ++i) {
    const EvRec x = out[i];
    int j = i - 1;
    while (j >= 0 && out[j].step > x.step) {
      out[j + 1] = out[j];
      --j;
    }
    out[j + 1] = x;
  }
  if (overflow) atomicOr(M.status, kStatusEvOverflow);
  M.ev_count[slot] = m;
}

// ---------------------------------------------------------- interval kernel
// Advances every cell of a warp by steps [s_begin, s_end) of interval J, one
// cell per lane.  Per step k = J D + s (Section 2's per-step list):
//  1 deliver due events (g += w, in buffer order),
//  2 nrn_cur: ExpSyn, HH and IClamp add their conductance G to the diagonal
//    accumulator and G E (+ I_inj) to the right-hand side accumulator,
//  3 the tree system (C + G + L) v_{k+1} = C v_k + G E + I_inj is solved by
//    Hines elimination (leaves to root) and back substitution,
//  4 nrn_state: HH gates by cnexp at v_{k+1}, ExpSyn decay,
//  5 threshold detection at the cell's spike node, and recording.
// Backward Euler with gates frozen over the step makes every current linear
// in v, so the system above is exactly the paper's linearised update
// (C + G + L) dv = -I(v_k) - L v_k written for v_{k+1} instead of dv.
template <int PREC>
__global__ void __launch_bounds__(32) k_interval(DevModel M, int64_t J, int s_begin, int s_end) {
  using S = typename GateT<PREC>::S;
  using T = typename GateT<PREC>::M;
  const int g = blockIdx.x * (blockDim.x / kLanes) + threadIdx.x / kLanes;
  if (g >= M.n_groups) return;
  const int lane = threadIdx.x % kLanes;
  const int slot = g * kLanes + lane;
  const int N = M.s_rows[slot];
  const int R = M.g_rows[g];
  const int64_t nb = M.g_node_base[g] + lane;
  const int gid = M.s_gid[slot];
  const int SR = M.g_syn_rows[g], nsyn = M.s_nsyn[slot];
  const int64_t sb = M.g_syn_base[g] + lane;
  const int HR = M.g_hh_rows[g], nhh = M.s_nhh[slot];
  const int64_t hb = M.g_hh_base[g] + lane;
  const int STR = M.g_st_rows[g], nst = M.s_nst[slot];
  const int64_t stb = M.g_st_base[g] + lane;
  const int RR = M.g_rec_rows[g], nrec = M.s_nrec[slot];
  const int64_t rb = M.g_rec_base[g] + lane;
  const double dt = M.dt;
  const int64_t T0 = J * M.D;
  const int64_t spike_i = nb + (int64_t)M.s_spike_row[slot] * kLanes;
  const double thresh = M.s_thresh[slot];
  int above = M.s_above[slot];
  uint64_t mask = (s_begin > 0 && gid >= 0) ? M.hist[J * M.n_cells + gid] : 0ull;
  const EvRec* ev = M.ev_buf + (int64_t)slot * kEvCap;
  const int ne = M.ev_count[slot];
  int ei = 0;
  while (ei < ne && ev[ei].step < s_begin) ++ei;
  S* const gm = static_cast<S*>(M.hh_m);
  S* const gh = static_cast<S*>(M.hh_h);
  S* const gn = static_cast<S*>(M.hh_n);

  for (int s = s_begin; s < s_end; ++s) {
    const int64_t k = T0 + s;
    // (1) event delivery
    while (ei < ne && ev[ei].step == s) {
      M.syn_g[sb + (int64_t)ev[ei].syn * kLanes] += ev[ei].w;
      ++ei;
    }
    // (2) nrn_cur: synapses
    for (int q = 0; q < SR; ++q) {
      if (q < nsyn) {
        const int64_t i = sb + (int64_t)q * kLanes;
        const double gs = M.syn_g[i];
        const double G = gs * M.syn_s[i];
        const int64_t ni = nb + (int64_t)M.syn_row[i] * kLanes;
        M.acc[ni] = fma(G, M.syn_e[i], M.acc[ni]);
        M.dacc[ni] += G;
        M.syn_g[i] = gs * M.syn_decay[i];  // state update (g' = g exp(-dt/tau)), v-independent
      }
    }
    //     HH
    for (int q = 0; q < HR; ++q) {
      if (q < nhh) {
        const int64_t i = hb + (int64_t)q * kLanes;
        const double m = (double)g_load(gm + i), h = (double)g_load(gh + i), n = (double)g_load(gn + i);
        const double gna = M.hh_p[i] * (m * m * m * h);
        const double gk = M.hh_p[M.hh_elems + i] * ((n * n) * (n * n));
        const double gl = M.hh_p[2 * M.hh_elems + i];
        const int64_t ni = nb + (int64_t)M.hh_row[i] * kLanes;
        M.acc[ni] += gna * M.hh_p[4 * M.hh_elems + i] + gk * M.hh_p[5 * M.hh_elems + i] +
                     gl * M.hh_p[3 * M.hh_elems + i];
        M.dacc[ni] += gna + gk + gl;
      }
    }
    //     IClamp (midpoint rule)
    if (STR > 0) {
      const double tmid = ((double)k + 0.5) * dt;
      for (int q = 0; q < STR; ++q) {
        if (q < nst) {
          const int64_t i = stb + (int64_t)q * kLanes;
          if (M.st_del[i] <= tmid && tmid < M.st_del[i] + M.st_dur[i]) {
            const int64_t ni = nb + (int64_t)M.st_row[i] * kLanes;
            M.acc[ni] += M.st_amp[i];
          }
        }
      }
    }
    // (3) Hines elimination, leaves to root.  Row j's pivot is final once all
    //     its children (rows > j) are eliminated.
    for (int j = R - 1; j >= 1; --j) {
      if (j < N) {
        const int64_t i = nb + (int64_t)j * kLanes;
        const double rhs = fma(M.cdt[i], M.v[i], M.acc[i]);
        const double r = rcp64(M.dacc[i]);
        const double x = rhs * r;
        const double bp = M.b[i] * r;
        const int64_t ip = nb + (int64_t)M.prow[i] * kLanes;
        const double na = -M.a[i];
        M.acc[ip] = fma(na, x, M.acc[ip]);
        M.dacc[ip] = fma(na, bp, M.dacc[ip]);
        M.v[i] = x;       // holds rhs/d until back substitution
        M.dacc[i] = bp;   // holds b/d until back substitution
      }
    }
    if (N > 0) {
      const double x0 = fma(M.cdt[nb], M.v[nb], M.acc[nb]) * rcp64(M.dacc[nb]);
      M.v[nb] = x0;
      M.acc[nb] = M.ge[nb];
      M.dacc[nb] = M.d0[nb];
    }
    //     back substitution, root to leaves; reset the accumulators.
    for (int j = 1; j < R; ++j) {
      if (j < N) {
        const int64_t i = nb + (int64_t)j * kLanes;
        const int64_t ip = nb + (int64_t)M.prow[i] * kLanes;
        M.v[i] = fma(-M.dacc[i], M.v[ip], M.v[i]);
        M.acc[i] = M.ge[i];
        M.dacc[i] = M.d0[i];
      }
    }
    // (4) nrn_state: HH gates (cnexp) at v_{k+1}
    for (int q = 0; q < HR; ++q) {
      if (q < nhh) {
        const int64_t i = hb + (int64_t)q * kLanes;
        const T vv = (T)M.v[nb + (int64_t)M.hh_row[i] * kLanes];
        T am, bm, ah, bh, an, bn;
        hh_rates<T>(vv, am, bm, ah, bh, an, bn);
        const T tdt = (T)dt;
        g_store(gm + i, cnexp_step<T>(g_load(gm + i), am, bm, tdt));
        g_store(gh + i, cnexp_step<T>(g_load(gh + i), ah, bh, tdt));
        g_store(gn + i, cnexp_step<T>(g_load(gn + i), an, bn, tdt));
      }
    }
    // (5) threshold detection and recording
    if (N > 0) {
      const int now = M.v[spike_i] > thresh;
      if (now && !above) mask |= 1ull << s;
      above = now;
      for (int q = 0; q < RR; ++q) {
        if (q < nrec) {
          const int64_t i = rb + (int64_t)q * kLanes;
          M.trace[(k + 1) * M.n_rec + M.rec_id[i]] = M.v[nb + (int64_t)M.rec_row[i] * kLanes];
        }
      }
    }
  }
  if (gid >= 0) {
    M.hist[J * M.n_cells + gid] = mask;
    M.s_above[slot] = (uint8_t)above;
  }
}

// Record step-0 voltages.
__global__ void k_record0(DevModel M, int64_t k) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int nrec = M.s_nrec[slot];
  const int64_t rb = M.g_rec_base[g] + lane;
  const int64_t nb = M.g_node_base[g] + lane;
  for (int q = 0; q < nrec; ++q) {
    const int64_t i = rb + (int64_t)q * kLanes;
    M.trace[k * M.n_rec + M.rec_id[i]] = M.v[nb + (int64_t)M.rec_row[i] * kLanes];
  }
}

// Threshold flags at the initial state.
__global__ void k_init_above(DevModel M) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  if (M.s_rows[slot] == 0) { M.s_above[slot] = 0; return; }
  const int g = slot / kLanes, lane = slot % kLanes;
  const int64_t i = M.g_node_base[g] + lane + (int64_t)M.s_spike_row[slot] * kLanes;
  M.s_above[slot] = M.v[i] > M.s_thresh[slot];
}

}  // namespace cn
