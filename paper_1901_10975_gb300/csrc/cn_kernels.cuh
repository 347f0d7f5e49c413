// cn_kernels.cuh -- setup, spike-pull and interval kernels.
#pragma once
#include "cn_device.cuh"

namespace cn {

// ------------------------------------------------------------------ setup
// Every element starts as an identity row (padding): cdt 1, no couplings.
__global__ void k_setup_pad(DevModel M) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M.node_elems) return;
  M.cdt[e] = 1.0;
  M.dax[e] = 0.0;
  const_cast<double*>(M.a)[e] = 0.0;
  const_cast<double*>(M.b)[e] = 0.0;
}

// Geometry part of every row (Eq. 1 discretised on the tree), rows scaled by
// 1/cdt_i, cdt_i = 1e-3 cm_i/dt:
//   b_i  = -100/(ri_i area_i) / cdt_i          (row i, column parent)
//   a_i  = -100/(ri_i area_p) / cdt_p          (row parent, column i)
//   dax_i = sum of the unscaled axial couplings of row i
// One thread per cell (a cell's parts may sit in different lanes); elem
// maps a global node to its element.  Without `scaled` (the reference
// layouts) a and b keep their unscaled values.
__global__ void k_setup_geom(DevModel M, int n_cells, const int32_t* off, const int32_t* parent, const double* area,
                             const double* ri, const double* cm, const int64_t* elem, bool scaled) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  double* a = const_cast<double*>(M.a);
  double* b = const_cast<double*>(M.b);
  for (int32_t i = off[c]; i < off[c + 1]; ++i) M.cdt[elem[i]] = 1e-3 * cm[i] / M.dt;
  for (int32_t i = off[c] + 1; i < off[c + 1]; ++i) {
    const int32_t ip = off[c] + parent[i];
    const int64_t e = elem[i], ep = elem[ip];
    const double bb = -100.0 / (ri[i] * area[i]);
    const double aa = -100.0 / (ri[i] * area[ip]);
    M.dax[e] -= bb;
    M.dax[ep] -= aa;
    b[e] = scaled ? bb / M.cdt[e] : bb;
    a[e] = scaled ? aa / M.cdt[ep] : aa;
  }
}

// Diagonal and right-hand-side constants from the pas parameters:
//   d0_i = (cdt_i + g_i + dax_i) / cdt_i,   ge_i = g_i e_i / cdt_i,
// identity rows past the cell's end.  Re-run when pas g changes.
__global__ void k_pas_apply(DevModel M) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int64_t nb = M.g_node_base[g] + lane;
  double* d0 = const_cast<double*>(M.d0);
  double* ge = const_cast<double*>(M.ge);
  for (int j = 0; j < M.g_rows[g]; ++j) {
    const int64_t i = nb + (int64_t)j * kLanes;
    if (M.flags[i] & kRealBit) {
      const double c = M.cdt[i];
      d0[i] = (c + M.pas_g[i] + M.dax[i]) / c;
      ge[i] = M.pas_g[i] * M.pas_e[i] / c;
    } else {
      d0[i] = 1.0;
      ge[i] = 0.0;
    }
    M.d0_syn[i] = d0[i];  // rows with synapses are rewritten every step
    M.ge_syn[i] = ge[i];
  }
}

// HH conductance densities divided by cdt of their row.  Re-run when gnabar
// or gkbar change.
__global__ void k_hh_params(DevModel M) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int n = M.s_nhh[slot];
  const int64_t base = M.g_hh_base[g] + lane, nb = M.g_node_base[g] + lane;
  double* P = const_cast<double*>(M.hh_p);
  for (int q = 0; q < n; ++q) {
    const int64_t i = base + (int64_t)q * kLanes;
    const double c = M.cdt[nb + (int64_t)M.hh_row[i] * kLanes];
    for (int col = 0; col < 6; ++col) {
      const double raw = M.hh_raw[col * M.hh_elems + i];
      P[col * M.hh_elems + i] = col < 3 ? raw / c : raw;
    }
  }
}

// Parameter scatter / gather by element index (per-cell conductances are
// expanded to their instances on the host): dst[idx[i]] = val[i] and
// out[i] = src[idx[i]].
__global__ void k_scatter(double* dst, const int64_t* idx, const double* val, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] = val[i];
}
__global__ void k_gather(const double* src, const int64_t* idx, double* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = src[idx[i]];
}

// Initial state: v = v_init (0 on rows past the cell's end), HH gates at
// their steady state of v_init, synaptic g = 0, threshold flags.
template <int PREC>
__global__ void k_state_init(DevModel M, double v_init) {
  using S = typename GateT<PREC>::S;
  using T = typename GateT<PREC>::M;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int N = M.s_rows[slot];
  const int64_t nb = M.g_node_base[g] + lane;
  for (int j = 0; j < M.g_rows[g]; ++j) {
    const int64_t i = nb + (int64_t)j * kLanes;
    M.v[i] = (M.flags[i] & kRealBit) ? v_init : 0.0;
    M.bp[i] = 0.0;
  }
  const int nh = M.s_nhh[slot];
  const int64_t hb = M.g_hh_base[g] + lane;
  for (int q = 0; q < nh; ++q) {
    const int64_t i = hb + (int64_t)q * kLanes;
    T am, bm, ah, bh, an, bn;
    hh_rates<T>(T(v_init), am, bm, ah, bh, an, bn);
    g_store(static_cast<S*>(M.hh_m) + i, am / (am + bm));
    g_store(static_cast<S*>(M.hh_h) + i, ah / (ah + bh));
    g_store(static_cast<S*>(M.hh_n) + i, an / (an + bn));
  }
  const int64_t sb = M.g_syn_base[g] + lane;
  for (int q = 0; q < M.g_syn_rows[g]; ++q) M.syn_g[sb + (int64_t)q * kLanes] = 0.0;
  M.s_above[slot] = M.s_gid[slot] >= 0 && N > 0 && v_init > M.s_thresh[slot];
  M.ev_count[slot] = 0;
}


// ExpSyn constants: s = 100/(area cdt) (nA -> mA/cm2, row-scaled),
// decay = exp(-dt/tau), g = 0 (one thread per warp column).
__global__ void k_setup_syn(DevModel M, const double* node_area, const double* node_cm, const double* tau) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int64_t base = M.g_syn_base[g] + lane;
  for (int q = 0; q < M.g_syn_rows[g]; ++q) {
    const int64_t i = base + (int64_t)q * kLanes;
    if (M.syn_tgt[i] >= 0) {
      const_cast<double*>(M.syn_s)[i] = 100.0 / (node_area[i] * (1e-3 * node_cm[i] / M.dt));
      const_cast<double*>(M.syn_decay)[i] = exp(-M.dt / tau[i]);
    }
    M.syn_g[i] = 0.0;
  }
}

// Copies of the target rows' ge and d0 beside the first synapse of each
// group, so the per-step sum reads them with the synapse (coalesced).
// Re-run whenever d0 or ge change.
__global__ void k_syn_consts(DevModel M) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int64_t base = M.g_syn_base[g] + lane, nbw = M.g_node_base[g];
  for (int q = 0; q < M.g_syn_rows[g]; ++q) {
    const int64_t i = base + (int64_t)q * kLanes;
    const int t = M.syn_tgt[i];
    if (t >= 0 && (t & kSynFirst)) {
      M.syn_ge0[i] = M.ge[nbw + (t & kSynTgtMask)];
      M.syn_d00[i] = M.d0[nbw + (t & kSynTgtMask)];
    }
  }
}

// IClamp amplitude as a row-scaled density: 100 amp / (area cdt).
__global__ void k_setup_stim(DevModel M, const double* amp, const double* node_area, const double* node_cm) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int n = M.s_nst[slot];
  const int64_t base = M.g_st_base[g] + lane;
  for (int q = 0; q < n; ++q) {
    const int64_t i = base + (int64_t)q * kLanes;
    const_cast<double*>(M.st_amp)[i] = 100.0 * amp[i] / (node_area[i] * (1e-3 * node_cm[i] / M.dt));
  }
}

// Half gap junction constants: gs = 100 g / (area cdt) of the junction's row.
__global__ void k_setup_gap(DevModel M, const double* area, const double* cm, const double* g_uS, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) M.gap_gs[i] = 100.0 * g_uS[i] / (area[i] * (1e-3 * cm[i] / M.dt));
}

// Publishes every gap peer voltage of the current step into vgap[parity].
__global__ void k_gap_publish(DevModel M, int parity) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int n = M.s_ngsrc[slot];
  const int64_t sb = M.g_gsrc_base[g] + lane, nb = M.g_node_base[g] + lane;
  for (int q = 0; q < n; ++q) {
    const int64_t i = sb + (int64_t)q * kLanes;
    M.vgap[(int64_t)parity * M.n_gsrc + M.gsrc_id[i]] = M.v[nb + (int64_t)M.gsrc_row[i] * kLanes];
  }
}

// ------------------------------------------------------- interval boundary
// Spike exchange at the start of interval J (Section 2: spikes are exchanged
// once per minimum delay).  Each cell pulls, from the spike masks of earlier
// intervals, every NetCon event due in [J D, J D + D), and its external
// events for the same window, into its event buffer ordered by (step,
// external-before-NetCon, input index | source gid, NetCon index).  No
// atomics: the result is deterministic.
__global__ void k_pull_events(DevModel M, int64_t J, const int64_t* Jp) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  if (Jp) J = *Jp;
  EvRec* out = M.ev_buf + M.ev_off[slot];
  const int cap = (int)(M.ev_off[slot + 1] - M.ev_off[slot]);
  const int D = M.D;
  const int64_t T = J * D;
  int n = 0;
  bool overflow = false;
  // external events (sorted by step, then input order)
  int64_t p = M.x_pos[slot];
  const int64_t pe = M.x_off[slot + 1];
  while (p < pe && M.x_step[p] < T + D) {
    if (M.x_step[p] >= T) {
      if (n < cap) out[n] = EvRec{(int32_t)(M.x_step[p] - T), M.x_syn[p], M.x_w[p]};
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
        if (n < cap) out[n] = EvRec{(int32_t)(t + ds - T), M.in_syn[q], M.in_w[q]};
        else overflow = true;
        ++n;
      }
    }
  }
  const int m = n < cap ? n : cap;
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

// The solve's pivot reciprocal applied elementwise (diagnostics: lets the
// reciprocal be compared with IEEE division).
__global__ void k_rcp64(const double* __restrict__ d, double* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = rcp64(d[i]);
}

// A stream of independent FP64 fused multiply-adds (diagnostics: the FP64
// pipe's attainable rate on this GPU).  Four chains per thread; the sums go
// to out so nothing is eliminated.
__global__ void k_dfma_stream(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  for (int it = 0; it < iters; ++it) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}

// Advances the device-side interval index after a complete interval.
__global__ void k_next_interval(int64_t* Jp) { *Jp += 1; }


// ------------------------------------------------------- dense channel types
// Channel types of the batched workload, present on every row of a cell
// (I_ion of Eq. 1).  Gate x of a type obeys alpha = A (v-vh)/(1-exp(-(v-vh)/k)),
// beta = B exp(-(v-vh2)/k2) (KCa: alpha = A cai/(cai+kd), beta = B) and
// is updated by cnexp at v_{k+1}; the conductance gbar * prod(x^p) enters
// the matrix in FP64 whatever the gate precision.  kin points at the lane's
// kinetics in shared memory ([param][32]).
template <typename T>
__device__ __forceinline__ void gate_ab(const T* kin, T v, T& al, T& be) {
  const T A = kin[0], vh = kin[kLanes], k = kin[2 * kLanes];
  const T B = kin[3 * kLanes], vh2 = kin[4 * kLanes], k2 = kin[5 * kLanes];
  al = vtrap<T>(A, vh, k, v);
  be = B * dexp_(-(v - vh2) / k2);
}

// One gate's cnexp update at v from its kinetics (alpha, beta as above).  It
// is kept out of line so that one copy of its exponential and division
// sequences serves all nine gates: inlined per gate, the channel update's
// code outgrew the instruction cache (ncu: 13.8 cycles per issue waiting on
// instruction fetch) and the interval ran 28% (FP64) / 18% (FP32) slower.
template <typename T>
__device__ __noinline__ T gate_next(const T* kin, T v, T x, T dt) {
  T al, be;
  gate_ab<T>(kin, v, al, be);
  return cnexp_step<T>(x, al, be, dt);
}

// Channel conductance G and sum of g E of row e at voltage v from the stored
// gates (the nrn_cur of the channel types), and ica for the calcium update.
template <int PREC>
__device__ __forceinline__ void dense_cur(const DevModel& M, int mask, int64_t e, double v, const double* kin,
                                          int64_t ks, double& G, double& GE) {
  using S = typename GateT<PREC>::S;
  using T = typename GateT<PREC>::M;
  auto x = [&](int gi) { return (T)g_load(static_cast<const S*>(M.ch_gate[gi]) + e); };
  double g = 0.0, ge = 0.0;
  if (mask & 1) {  // NA3H: m^3 h
    const T m = x(0);
    const double c = M.ch_gbar[0][e] * (double)(m * m * m * x(1));
    g += c;
    ge = fma(c, kin[chan_kin0(0) * ks], ge);
  }
  if (mask & 2) {  // KDR4: n^4
    const T n = x(2);
    const double c = M.ch_gbar[1][e] * (double)((n * n) * (n * n));
    g += c;
    ge = fma(c, kin[chan_kin0(1) * ks], ge);
  }
  if (mask & 4) {  // KA: a^3 b
    const T a = x(3);
    const double c = M.ch_gbar[2][e] * (double)(a * a * a * x(4));
    g += c;
    ge = fma(c, kin[chan_kin0(2) * ks], ge);
  }
  if (mask & 8) {  // IH: q
    const double c = M.ch_gbar[3][e] * (double)x(5);
    g += c;
    ge = fma(c, kin[chan_kin0(3) * ks], ge);
  }
  if (mask & 16) {  // CAHVA: m^2 h; its current drives [Ca]i
    const T m = x(6);
    const double c = M.ch_gbar[4][e] * (double)(m * m * x(7));
    const double eca = kin[chan_kin0(4) * ks];
    g += c;
    ge = fma(c, eca, ge);
    M.ica[e] = c * M.cdt[e] * (v - eca);
  }
  if (mask & 32) {  // KCA: c
    const double c = M.ch_gbar[5][e] * (double)x(8);
    g += c;
    ge = fma(c, kin[chan_kin0(5) * ks], ge);
  }
  G = g;
  GE = ge;
}

// nrn_state of the channel types at v_{k+1} (cnexp, in type order; the
// calcium update uses the ica of step k), followed at once by their nrn_cur
// for step k+1 from the new gates and v_{k+1}: G and G E go to ch_g/ch_ge,
// which the next elimination streams with the row, and ica is kept for the
// next calcium update.  The values are those a separate nrn_cur at the start
// of step k+1 would compute.
template <int PREC>
struct ChanIn {  // the inputs of one row's channel update
  typename GateT<PREC>::M x[kChanGates];
  double gb[kChanTypes];
  double ica, cai;
};

template <int PREC>
__device__ __forceinline__ void dense_load(const DevModel& M, int mask, int64_t e, ChanIn<PREC>& in) {
  using S = typename GateT<PREC>::S;
#pragma unroll
  for (int t = 0; t < kChanTypes; ++t) {
    if (mask & (1 << t)) {
      in.gb[t] = M.ch_gbar[t][e];
#pragma unroll
      for (int gi = chan_gate0(t); gi < (t + 1 < kChanTypes ? chan_gate0(t + 1) : kChanGates); ++gi)
        in.x[gi] = g_load(static_cast<const S*>(M.ch_gate[gi]) + e);
    }
  }
  in.ica = (mask & 16) ? M.ica[e] : 0.0;
  in.cai = (mask & 48) ? M.cai[e] : 0.0;
}

template <int PREC>
__device__ __forceinline__ void dense_step(const DevModel& M, int mask, int64_t e, double vnew, const double* erev,
                                           const typename GateT<PREC>::M* kinT, const ChanIn<PREC>& in) {
  using S = typename GateT<PREC>::S;
  using T = typename GateT<PREC>::M;
  const T v = (T)vnew, tdt = (T)M.dt;
  // the gate powers are formed in the gate type; gbar times that product
  // and the sums that enter the matrix are FP64
  auto upd = [&](int gi, const T* k6) -> T {
    S* p = static_cast<S*>(M.ch_gate[gi]) + e;
    return g_store_ret(p, gate_next<T>(k6, v, in.x[gi], tdt));
  };
  double g = 0.0, ge = 0.0;
  if (mask & 1) {  // NA3H: m^3 h
    const T m = upd(0, kinT + (chan_kin0(0) + 1) * kLanes);
    const T h = upd(1, kinT + (chan_kin0(0) + 7) * kLanes);
    const double c = in.gb[0] * (double)(m * m * m * h);
    g += c;
    ge = fma(c, erev[0 * kLanes], ge);
  }
  if (mask & 2) {  // KDR4: n^4
    const T n = upd(2, kinT + (chan_kin0(1) + 1) * kLanes);
    const double c = in.gb[1] * (double)((n * n) * (n * n));
    g += c;
    ge = fma(c, erev[1 * kLanes], ge);
  }
  if (mask & 4) {  // KA: a^3 b
    const T a = upd(3, kinT + (chan_kin0(2) + 1) * kLanes);
    const T b = upd(4, kinT + (chan_kin0(2) + 7) * kLanes);
    const double c = in.gb[2] * (double)(a * a * a * b);
    g += c;
    ge = fma(c, erev[2 * kLanes], ge);
  }
  if (mask & 8) {  // IH: q
    const T q = upd(5, kinT + (chan_kin0(3) + 1) * kLanes);
    const double c = in.gb[3] * (double)q;
    g += c;
    ge = fma(c, erev[3 * kLanes], ge);
  }
  double cai1 = in.cai;
  if (mask & 16) {  // CAHVA: m^2 h, [Ca]i from the current of step k
    const T m = upd(6, kinT + (chan_kin0(4) + 1) * kLanes);
    const T h = upd(7, kinT + (chan_kin0(4) + 7) * kLanes);
    const T* kct = kinT + chan_kin0(4) * kLanes;
    const T depth = kct[13 * kLanes], taur = kct[14 * kLanes], cainf = kct[15 * kLanes];
    T drive = T(-1e4) * (T)in.ica / (T(2.0 * 96485.3321) * depth);
    if (drive < T(0)) drive = T(0);
    const T cai = (T)in.cai;
    cai1 = (double)(cai + omexp_(tdt / taur) * (cainf + drive * taur - cai));
    M.cai[e] = cai1;
    const double c = in.gb[4] * (double)(m * m * h);
    const double eca = erev[4 * kLanes];
    g += c;
    ge = fma(c, eca, ge);
    M.ica[e] = c * M.cdt[e] * (vnew - eca);
  }
  if (mask & 32) {  // KCA: c, activated by the new [Ca]i
    const T* kkt = kinT + chan_kin0(5) * kLanes;
    const T cai = (T)cai1;
    const T al = kkt[1 * kLanes] * cai / (cai + kkt[2 * kLanes]);
    S* p = static_cast<S*>(M.ch_gate[8]) + e;
    const T xk = g_store_ret(p, cnexp_step<T>(in.x[8], al, kkt[3 * kLanes], tdt));
    const double c = in.gb[5] * (double)xk;
    g += c;
    ge = fma(c, erev[5 * kLanes], ge);
  }
  M.ch_g[e] = g;
  M.ch_ge[e] = ge;
}

// Channel currents of every row from the stored gates and v (after setup or
// a restore).
template <int PREC>
__global__ void k_dense_currents(DevModel M) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int mask = M.g_chmask[g];
  const int64_t nb = M.g_node_base[g] + lane;
  const double* kin = M.ch_kin + slot;  // [param][n_slots]
  for (int j = 0; j < M.g_rows[g]; ++j) {
    const int64_t e = nb + (int64_t)j * kLanes;
    double G = 0.0, GE = 0.0;
    if (M.flags[e] & kRealBit) dense_cur<PREC>(M, mask, e, M.v[e], kin, M.n_slots, G, GE);
    M.ch_g[e] = G;
    M.ch_ge[e] = GE;
  }
}

// Dense-channel constants and initial state: gbar divided by cdt of the row,
// gates at their steady state of v_init, [Ca]i at cainf (5e-5 mM without
// CAHVA).
template <int PREC>
__global__ void k_setup_dense(DevModel M, double v_init, bool scale_gbar) {
  using S = typename GateT<PREC>::S;
  using T = typename GateT<PREC>::M;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int N = M.s_rows[slot];
  const int mask = M.g_chmask[g];
  const int64_t nb = M.g_node_base[g] + lane;
  const double* kin = M.ch_kin + slot;  // [param][n_slots]
  const int64_t ks = M.n_slots;
  const T v = (T)v_init;
  for (int j = 0; j < N; ++j) {
    const int64_t e = nb + (int64_t)j * kLanes;
    if (!(M.flags[e] & kRealBit)) continue;
    if (scale_gbar)
      for (int t = 0; t < kChanTypes; ++t)
        if ((mask >> t) & 1) M.ch_gbar[t][e] /= M.cdt[e];
    auto init = [&](int gi, int k0) {
      const T A = (T)kin[k0 * ks], vh = (T)kin[(k0 + 1) * ks], k = (T)kin[(k0 + 2) * ks];
      const T B = (T)kin[(k0 + 3) * ks], vh2 = (T)kin[(k0 + 4) * ks], k2 = (T)kin[(k0 + 5) * ks];
      const T al = vtrap<T>(A, vh, k, v), be = B * dexp_(-(v - vh2) / k2);
      g_store(static_cast<S*>(M.ch_gate[gi]) + e, al / (al + be));
    };
    if (mask & 1) { init(0, chan_kin0(0) + 1); init(1, chan_kin0(0) + 7); }
    if (mask & 2) init(2, chan_kin0(1) + 1);
    if (mask & 4) { init(3, chan_kin0(2) + 1); init(4, chan_kin0(2) + 7); }
    if (mask & 8) init(5, chan_kin0(3) + 1);
    if (mask & 16) { init(6, chan_kin0(4) + 1); init(7, chan_kin0(4) + 7); }
    if (M.cai) M.cai[e] = (mask & 16) ? kin[(chan_kin0(4) + 15) * ks] : 5e-5;
    if (mask & 32) {
      const T cai = (T)M.cai[e];
      const T al = (T)kin[(chan_kin0(5) + 1) * ks] * cai / (cai + (T)kin[(chan_kin0(5) + 2) * ks]);
      const T be = (T)kin[(chan_kin0(5) + 3) * ks];
      g_store(static_cast<S*>(M.ch_gate[8]) + e, al / (al + be));
    }
    double G, GE;  // channel currents of step 0 (ica included)
    dense_cur<PREC>(M, mask, e, v_init, kin, ks, G, GE);
    M.ch_g[e] = G;
    M.ch_ge[e] = GE;
  }
}

// ---------------------------------------------------------- interval kernel
// Each warp advances the parts placed on its 32 lanes (whole cells, or parts
// of cells split over lanes of the warp) by steps [s_begin, s_end) of
// interval J; a block holds one to four warps.  Per step k = J D + s
// (Section 2's list):
//  1 deliver due events (g += w, in buffer order),
//  2 nrn_cur: ExpSyn G and G E summed per warp column onto the target rows'
//    constants (ge_syn, d0_syn); HH, IClamp and gap terms into the per-lane
//    slot buffer of their row; channel terms computed at the end of the
//    previous step,
//  3 matrix resolution: the row-scaled system (C + G + L) v_{k+1} = C v_k +
//    G E + I_inj is eliminated leaves to root in Hines order and
//    back-substituted root to leaves,
//  4 nrn_state: channel gates and calcium, then HH gates, by cnexp at
//    v_{k+1}; the ExpSyn decay is applied with the sums of step 2,
//  5 threshold detection at the lane's spike row, and recording.
// Backward Euler with the gates frozen over a step makes every current linear
// in v, so this is exactly the paper's linearised update
// (C + G + L) dv = -I(v_k) - L v_k written for v_{k+1} instead of dv.
// Row data streams through a per-lane shared-memory ring fed by cp.async, each
// lane copying its own elements kElimRows rows ahead (kBackRows in the back
// substitution); a row's child terms come from a register carry (previous
// row), from partial sums on the per-lane stack (far children), or from the
// warp's mailbox (a part hanging from the row).
// TRAJ: adjoint recompute -- also store v and the HH gates of every step
// into the trajectory buffers, and leave spikes, threshold flags and traces
// untouched.
// Registers: at most 128 per thread without channel types, so that four
// 4-warp blocks (16 warps) fit an SM.  The cap is set directly: asking for
// four resident blocks through __launch_bounds__ gives the same cap, but
// that build ran 3% slower.
template <int PREC, bool TRAJ, bool DENSE>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32) __maxnreg__(DENSE ? 255 : 128)
    k_interval(DevModel M, int64_t J, int s_begin, int s_end, const int64_t* Jp) {
  using S = typename GateT<PREC>::S;
  using T = typename GateT<PREC>::M;
  extern __shared__ __align__(16) unsigned char smem_all[];
  if (Jp) J = *Jp;  // interval index kept on the device (graph replay)
  const int wib = threadIdx.x >> 5;  // warp in block: each warp runs one group
  const int g = blockIdx.x * (blockDim.x >> 5) + wib;
  if (g >= M.n_groups) return;
  const int lane = threadIdx.x & 31;
  unsigned char* const smem = smem_all + (size_t)wib * M.smem_warp;
  const int slot = g * kLanes + lane;
  const int N = M.s_rows[slot];
  const int R = M.g_rows[g];
  const int64_t nb = M.g_node_base[g] + lane;
  const int gid = M.s_gid[slot];
  const int DS = M.stack_depth;

  // elimination ring [array][kElimRows][32]; back-substitution ring shares it
  double* const e_v = reinterpret_cast<double*>(smem) + lane;
  double* const e_ge = e_v + kElimRows * kLanes;
  double* const e_d0 = e_ge + kElimRows * kLanes;
  double* const e_a = e_d0 + kElimRows * kLanes;
  double* const e_b = e_a + kElimRows * kLanes;
  double* const e_cg = e_b + kElimRows * kLanes;    // channel G and G E (DENSE)
  double* const e_cge = e_cg + kElimRows * kLanes;
  int32_t* const e_fl =
      reinterpret_cast<int32_t*>(reinterpret_cast<double*>(smem) + (DENSE ? 7 : 5) * kElimRows * kLanes) + lane;
  int32_t* const e_pf = e_fl + kElimRows * kLanes;
  double* const b_x = reinterpret_cast<double*>(smem) + lane;
  double* const b_bp = b_x + kBackRows * kLanes;
  int32_t* const b_fl = reinterpret_cast<int32_t*>(reinterpret_cast<double*>(smem) + 2 * kBackRows * kLanes) + lane;
  double* const wsm = reinterpret_cast<double*>(smem + ring_bytes(DENSE));
  // per-lane stack [DS + 1][32] of three words.  Elimination: the partial
  // sums of parents some of whose far children are done, with the parent's
  // row; back substitution: the parents' voltages for their far children.
  double* const st_r = wsm + lane;
  double* const st_d = st_r + (DS + 1) * kLanes;
  int32_t* const st_o = reinterpret_cast<int32_t*>(wsm + 2 * (DS + 1) * kLanes) + lane;
  double* const st_x = st_r;
  double* const sl_ge = st_r + 3 * (DS + 1) * kLanes;  // slot buffer [max_slots][32]
  double* const sl_d = sl_ge + M.max_slots * kLanes;
  // channel types: reversal potentials [6][32] (FP64) and the gate kinetics
  // [kChanParams][32] in the gate arithmetic's type
  double* const erev = sl_d + M.max_slots * kLanes;
  unsigned char* const kin_base = reinterpret_cast<unsigned char*>(
      wsm + (3 * (DS + 1) + 2 * M.max_slots + (DENSE ? kChanTypes : 0)) * kLanes);
  T* const kinT = reinterpret_cast<T*>(kin_base) + lane;
  // mailbox [n_mail][4] shared by the warp: a part root leaves (a, x, b/d)
  // for its junction row, the junction row leaves v for the part root
  double* const mail = reinterpret_cast<double*>(kin_base + (DENSE ? kChanParams * kLanes * sizeof(T) : 0));
  const int chmask = DENSE ? M.g_chmask[g] : 0;
  if (DENSE) {
    for (int q = 0; q < kChanParams; ++q) kinT[q * kLanes] = (T)M.ch_kin[(int64_t)q * M.n_slots + slot];
    for (int t = 0; t < kChanTypes; ++t) erev[t * kLanes] = M.ch_kin[(int64_t)chan_kin0(t) * M.n_slots + slot];
  }

  // this lane's column of every per-row array
  double* const gv = M.v + nb;
  double* const gbp = M.bp + nb;
  const double* const gge = M.ge_syn + nb;  // row constants with this step's synaptic terms
  const double* const gd0 = M.d0_syn + nb;
  const double* const ga = M.a + nb;
  const double* const gb = M.b + nb;
  const int32_t* const gfl = M.flags + nb;

  const int SLR = M.g_slot_rows[g], nslot = M.s_nslot[slot];
  const int SYR = M.g_syn_rows[g];
  const int64_t sb = M.g_syn_base[g] + lane;  // sb - lane, nb - lane: the warp's bases
  const int HR = M.g_hh_rows[g], nhh = M.s_nhh[slot];
  const int64_t hb = M.g_hh_base[g] + lane;
  const int STR = M.g_st_rows[g], nst = M.s_nst[slot];
  const int64_t stb = M.g_st_base[g] + lane;
  const int GR = M.g_gap_rows[g], ngap = M.s_ngap[slot];
  const int64_t gpb = M.g_gap_base[g] + lane;
  const int GSR = M.g_gsrc_rows[g], ngsrc = M.s_ngsrc[slot];
  const int64_t gsb = M.g_gsrc_base[g] + lane;
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
  S* const gm = static_cast<S*>(M.hh_m);
  S* const gh = static_cast<S*>(M.hh_h);
  S* const gn = static_cast<S*>(M.hh_n);

  auto fetch_elim = [&](int j, int u) {  // row j into ring row u (a no-op group past the root)
    if (j >= 0) {
      const int64_t o = (int64_t)j * kLanes;
      cp_async8(e_v + u * kLanes, gv + o);
      cp_async8(e_ge + u * kLanes, gge + o);
      cp_async8(e_d0 + u * kLanes, gd0 + o);
      cp_async8(e_a + u * kLanes, ga + o);
      cp_async8(e_b + u * kLanes, gb + o);
      if (DENSE) {
        cp_async8(e_cg + u * kLanes, M.ch_g + nb + o);
        cp_async8(e_cge + u * kLanes, M.ch_ge + nb + o);
      }
      cp_async4(e_fl + u * kLanes, gfl + o);
      cp_async4(e_pf + u * kLanes, M.pfar + nb + o);
    }
    cp_async_commit();
  };
  auto fetch_back = [&](int j, int u) {
    if (j < R) {
      const int64_t o = (int64_t)j * kLanes;
      cp_async8(b_x + u * kLanes, gv + o);
      cp_async8(b_bp + u * kLanes, gbp + o);
      cp_async4(b_fl + u * kLanes, gfl + o);
    }
    cp_async_commit();
  };

  // Slot buffer (HH and IClamp terms of a row): cleared once per launch; after
  // that every elimination row clears its own slot for the next step.
  for (int t = 0; t < SLR; ++t) {
    if (t < nslot) {
      sl_ge[t * kLanes] = 0.0;
      sl_d[t * kLanes] = 0.0;
    }
  }

  for (int s = s_begin; s < s_end; ++s) {
    const int64_t k = T0 + s;
    // (1) event delivery (into the synapse's column, wherever it lies)
    while (ei < ne && ev[ei].step == s) {
      M.syn_g[sb - lane + ev[ei].syn] += ev[ei].w;
      ++ei;
    }
    __syncwarp();
    // (2) nrn_cur.  ExpSyn: G = g s and G E of every synapse of the warp,
    //     each lane summing its column (kSynBatch entries at a time, their
    //     loads in flight together) onto the target row's constants into
    //     ge_syn / d0_syn, which the elimination streams; then the
    //     v-independent decay of g.  A row's synapses are consecutive entries
    //     of one column, between kSynFirst and kSynLast.
    {
      constexpr int kSynBatch = 2;
      double age = 0.0, ad = 0.0;
      for (int q0 = 0; q0 < SYR; q0 += kSynBatch) {
        double sg_[kSynBatch], ss_[kSynBatch], se_[kSynBatch], sd_[kSynBatch], cg[kSynBatch], cd[kSynBatch];
        int st_[kSynBatch];
#pragma unroll
        for (int u = 0; u < kSynBatch; ++u) {
          st_[u] = -1;
          if (q0 + u < SYR) {
            const int64_t i = sb + (int64_t)(q0 + u) * kLanes;
            st_[u] = M.syn_tgt[i];
            sg_[u] = M.syn_g[i];
            ss_[u] = M.syn_s[i];
            se_[u] = M.syn_e[i];
            sd_[u] = M.syn_decay[i];
            cg[u] = M.syn_ge0[i];
            cd[u] = M.syn_d00[i];
          }
        }
#pragma unroll
        for (int u = 0; u < kSynBatch; ++u) {
          const int t = st_[u];
          if (t < 0) continue;
          if (t & kSynFirst) {
            age = cg[u];
            ad = cd[u];
          }
          const double G = sg_[u] * ss_[u];
          age = fma(G, se_[u], age);
          ad += G;
          M.syn_g[sb + (int64_t)(q0 + u) * kLanes] = sg_[u] * sd_[u];
          if (t & kSynLast) {
            M.ge_syn[nb - lane + (t & kSynTgtMask)] = age;
            M.d0_syn[nb - lane + (t & kSynTgtMask)] = ad;
          }
        }
      }
    }
    __syncwarp();
    // start streaming the top rows (after this lane's row constants are final)
#pragma unroll
    for (int u = 0; u < kElimRows; ++u) fetch_elim(R - 1 - u, u);
    // HH and IClamp into the slot buffer
    for (int q = 0; q < HR; ++q) {
      if (q < nhh) {
        const int64_t i = hb + (int64_t)q * kLanes;
        const double m = (double)g_load(gm + i), h = (double)g_load(gh + i), n = (double)g_load(gn + i);
        const double gna = M.hh_p[i] * (m * m * m * h);
        const double gk = M.hh_p[M.hh_elems + i] * ((n * n) * (n * n));
        const double gl = M.hh_p[2 * M.hh_elems + i];
        const int t = M.hh_slot[i] * kLanes;
        sl_ge[t] += gna * M.hh_p[4 * M.hh_elems + i] + gk * M.hh_p[5 * M.hh_elems + i] +
                    gl * M.hh_p[3 * M.hh_elems + i];
        sl_d[t] += gna + gk + gl;
      }
    }
    // gap junctions: g (v_peer,k - v) with the peers' voltages of step k
    for (int q = 0; q < GR; ++q) {
      if (q < ngap) {
        const int64_t i = gpb + (int64_t)q * kLanes;
        const double gs = M.gap_gs[i];
        const int t = M.gap_slot[i] * kLanes;
        sl_ge[t] = fma(gs, M.vgap[(k & 1) * M.n_gsrc + M.gap_src[i]], sl_ge[t]);
        sl_d[t] += gs;
      }
    }
    if (STR > 0) {
      const double tmid = ((double)k + 0.5) * dt;
      for (int q = 0; q < STR; ++q) {
        if (q < nst) {
          const int64_t i = stb + (int64_t)q * kLanes;
          if (M.st_del[i] <= tmid && tmid < M.st_del[i] + M.st_dur[i]) sl_ge[M.st_slot[i] * kLanes] += M.st_amp[i];
        }
      }
    }
    // (3) elimination, leaves to root.  One FMA pair per row takes the
    //     previous row's (-a, x, b/d): into this row when the previous row is
    //     its child, or, when the previous row was a far child, into the
    //     partial sums of that child's parent.  The row after a far child is
    //     always a leaf (the last row of the preceding sibling's subtree), so
    //     its own row needs no pair.  A parent's partial sums start from its
    //     v and d0 and take their place when its row comes.
    double ca = 0.0, cx = 0.0, cb = 0.0, x = 0.0, pv = 0.0, pd = 0.0;
    // v and d0 of the far parents of the next kElimRows rows, loaded that
    // many rows ahead into a register ring (slot u of the unrolled loop);
    // the first rows' come from their own pfar words
    double fpv[kElimRows], fpd[kElimRows];
#pragma unroll
    for (int u = 0; u < kElimRows; ++u) {
      const int j = R - 1 - u;
      const int pf = j >= 0 ? (M.pfar[nb + (int64_t)j * kLanes] & kPfarMask) : 0;
      fpv[u] = 0.0;
      fpd[u] = 0.0;
      if (pf > 0) {
        fpv[u] = gv[(int64_t)(j - pf) * kLanes];
        fpd[u] = gd0[(int64_t)(j - pf) * kLanes];
      }
    }
    int top = 0, pp = -1;
    // the top stack entry lives in registers (tr, td, owner row to; -1 when
    // the stack is empty); entries below it in st_r / st_d / st_o [0, top-1)
    double tr = 0.0, td = 0.0;
    int to = -1;
    for (int jb = R - 1; jb >= 0; jb -= kElimRows) {
#pragma unroll
      for (int u = 0; u < kElimRows; ++u) {
        const int j = jb - u;
        cp_async_wait<kElimRows - 1>();
        if (j >= 0) {
          const int ro = u * kLanes;
          const int f = e_fl[ro];
          const int sl = f & kNoSlot;
          const bool hs = sl != kNoSlot;
          // this row's partial sums, if far children of it were folded
          const bool own = to == j;
          const double v0 = own ? tr : e_v[ro];
          double dd0 = own ? td : e_d0[ro];
          if (own) {  // pop: the next entry comes back into registers
            --top;
            const int ti = (top > 0 ? top - 1 : 0) * kLanes;
            tr = st_r[ti];
            td = st_d[ti];
            to = top > 0 ? st_o[ti] : -1;
          }
          double acc_ge = e_ge[ro];  // constants with this step's synaptic terms
          // one vote covers the rare rows: slot rows and junction rows
          const bool jn = (f & kJuncBit) != 0;
          const bool rare = __any_sync(0xffffffffu, hs || jn);
          if (rare) {  // HH / IClamp rows (somas): add and clear the slot
            if (hs) {
              const int si = sl * kLanes;
              acc_ge += sl_ge[si];
              dd0 += sl_d[si];
              sl_ge[si] = 0.0;
              sl_d[si] = 0.0;
            }
          }
          double base = v0 + acc_ge;
          if (DENSE) {  // channel currents of this step (computed at the end of the previous one)
            base += e_cge[ro];
            dd0 += e_cg[ro];
          }
          // the previous row's terms: into this row, or into its parent's
          // partial sums (a new entry, or the top one if it is that parent's)
          const bool fin = pp >= 0;
          const bool acc = fin && to == pp;
          const double o_r = fma(-ca, cx, fin ? (acc ? tr : pv) : base);
          const double o_d = fma(-ca, cb, fin ? (acc ? td : pd) : dd0);
          double rhs = fin ? base : o_r;
          double d = fin ? dd0 : o_d;
          if (fin) {
            if (!acc) {  // push: the current top goes to shared memory
              if (top > 0) {
                const int w = (top - 1) * kLanes;
                st_r[w] = tr;
                st_d[w] = td;
                st_o[w] = to;
              }
              ++top;
            }
            tr = o_r;
            td = o_d;
            to = pp;
          }
          // a part of this cell hangs from this row: its root was eliminated
          // at a higher warp row and left (a, x, b/d) in the mailbox
          if (rare) {
            __syncwarp();
            if (jn) {
              const double* q = mail + 4 * ((f >> kJmailShift) & kMailMask);
              rhs = fma(-q[0], q[1], rhs);
              d = fma(-q[0], q[2], d);
            }
          }
          const double r = rcp64(d);
          x = rhs * r;
          const double bp = e_b[ro] * r;
          gv[(int64_t)j * kLanes] = x;
          gbp[(int64_t)j * kLanes] = bp;
          // a, negated inside the FMAs that use it (a separate negation would
          // cost an FP64 instruction per row)
          const double na = e_a[ro];
          if (f & kProotBit) {  // the parent row lies below, possibly in another lane
            double* q = mail + 4 * (((uint32_t)f >> kPmailShift) & kMailMask);
            q[0] = na;
            q[1] = x;
            q[2] = bp;
          }
          // a far child: its parent's v and d0 (not eliminated yet, loaded
          // kElimRows rows ago) start the parent's partial sums at the next
          // row; then the far parent of row j - kElimRows is loaded into
          // this ring slot (its rows lie below: still v_k and d0 of the step)
          const bool far = (f & kFarBit) != 0;
          const int pfw = e_pf[ro];
          pp = far ? j - (pfw & kPfarMask) : -1;
          if (far) {
            pv = fpv[u];
            pd = fpd[u];
          }
          {
            const int pf4 = (int)((unsigned)pfw >> kPfarAheadShift);
            const int j4 = j - kElimRows;
            if (pf4 > 0 && j4 >= 0) {
              fpv[u] = gv[(int64_t)(j4 - pf4) * kLanes];
              fpd[u] = gd0[(int64_t)(j4 - pf4) * kLanes];
            }
          }
          ca = (f & kProotBit) ? 0.0 : na;
          cx = x;
          cb = bp;
        }
        fetch_elim(j - kElimRows, u);
      }
    }
    cp_async_wait<0>();
    // back substitution, root to leaves (row 0: b = 0, so v_0 = x_0)
#pragma unroll
    for (int u = 0; u < kBackRows; ++u) fetch_back(u, u);
    // The stack holds, per parent with far children still to come, its
    // voltage and that count; the top entry lives in registers (tv, tc),
    // the entries below it in st_x / st_c [0, top-1).
    double vprev = 0.0, tv = 0.0;
    int tc = 0;
    int32_t* const st_c = st_o;
    for (int jb = 0; jb < R; jb += kBackRows) {
#pragma unroll
      for (int u = 0; u < kBackRows; ++u) {
        const int j = jb + u;
        cp_async_wait<kBackRows - 1>();
        if (j < R) {
          const int ro = u * kLanes;
          const int f = b_fl[ro];
          const bool far = (f & kFarBit) != 0;
          double vp = far ? tv : vprev;
          if (far && --tc == 0) {  // the parent's last far child: pop
            --top;
            const int ti = (top > 0 ? top - 1 : 0) * kLanes;
            tv = st_x[ti];
            tc = top > 0 ? st_c[ti] : 0;
          }
          // root of a part: its parent row was back-substituted at a lower
          // warp row and left v in the mailbox
          const bool pr = (f & kProotBit) != 0;
          if (__any_sync(0xffffffffu, pr)) {
            __syncwarp();
            if (pr) vp = mail[4 * (((uint32_t)f >> kPmailShift) & kMailMask) + 3];
          }
          const double vj = fma(-b_bp[ro], vp, b_x[ro]);
          gv[(int64_t)j * kLanes] = vj;
          if (f & kJuncBit) mail[4 * ((f >> kJmailShift) & kMailMask) + 3] = vj;
          if (TRAJ) M.traj_v[(k + 1 - M.traj_k0) * M.node_elems + nb + (int64_t)j * kLanes] = vj;
          const int np = (f >> kNFarShift) & kNFarMask;
          if (np > 0) {  // push this row's voltage for its far children
            if (top > 0) {
              const int w = (top - 1) * kLanes;
              st_x[w] = tv;
              st_c[w] = tc;
            }
            ++top;
            tv = vj;
            tc = np;
          }
          vprev = vj;
        }
        fetch_back(j + kBackRows, u);
      }
    }
    cp_async_wait<0>();
    // (3b) channel types: nrn_state at v_{k+1}, then their nrn_cur for the
    //      next step.  Rows are independent here, so kChanBatch rows load
    //      their inputs together before any of them computes.
    if (DENSE) {
      constexpr int kChanBatch = 2;
      for (int j0 = 0; j0 < R; j0 += kChanBatch) {
        ChanIn<PREC> in[kChanBatch];
        double vv[kChanBatch];
        int fr[kChanBatch];
#pragma unroll
        for (int u = 0; u < kChanBatch; ++u) {
          const int j = j0 + u;
          fr[u] = 0;
          if (j < R) {
            const int64_t e = nb + (int64_t)j * kLanes;
            fr[u] = M.flags[e] & kRealBit;
            vv[u] = M.v[e];
            dense_load<PREC>(M, chmask, e, in[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < kChanBatch; ++u)
          if (fr[u]) dense_step<PREC>(M, chmask, nb + (int64_t)(j0 + u) * kLanes, vv[u], erev, kinT, in[u]);
      }
    }
    // (4) nrn_state: HH gates (cnexp) at v_{k+1}.  A warp holds few HH
    //     instances (one per soma), so their work is spread over the lanes:
    //     the six rates of every instance, one per lane, then the three gate
    //     updates, one per lane.  Scratch lives in the row ring, idle here.
    for (int q = 0; q < HR; ++q) {
      const bool has = q < nhh;
      const unsigned act = __ballot_sync(0xffffffffu, has);
      const int nact = __popc(act);
      T* const hv = reinterpret_cast<T*>(smem);                             // [32] soma v
      int* const hl = reinterpret_cast<int*>(smem + kLanes * sizeof(double));  // [32] its lane
      T* const hr = reinterpret_cast<T*>(smem + kLanes * (sizeof(double) + sizeof(int)));  // [6][32]
      if (has) {
        const int rk = __popc(act & ((1u << lane) - 1u));
        hv[rk] = (T)M.v[nb + (int64_t)M.hh_row[hb + (int64_t)q * kLanes] * kLanes];
        hl[rk] = lane;
      }
      __syncwarp();
      for (int t = lane; t < 6 * nact; t += kLanes) {
        const int a = t / 6, kind = t - 6 * a;
        hr[kind * kLanes + a] = hh_rate<T>(kind, hv[a]);
      }
      __syncwarp();
      for (int t = lane; t < 3 * nact; t += kLanes) {
        const int a = t / 3, gate = t - 3 * a;
        const int64_t i = hb - lane + hl[a] + (int64_t)q * kLanes;
        S* const gp = gate == 0 ? gm : gate == 1 ? gh : gn;
        const T xn = cnexp_step<T>(g_load(gp + i), hr[2 * gate * kLanes + a], hr[(2 * gate + 1) * kLanes + a], (T)dt);
        const double xs = (double)g_store_ret(gp + i, xn);
        if (TRAJ) M.traj_g[(k + 1 - M.traj_k0) * 3 * M.hh_elems + gate * M.hh_elems + i] = xs;
      }
      __syncwarp();
    }
    // publish this lane's gap peer voltages of step k+1 (the other buffer:
    // lanes of other warps may still read the step-k values)
    for (int q = 0; q < GSR; ++q) {
      if (q < ngsrc) {
        const int64_t i = gsb + (int64_t)q * kLanes;
        const int row = M.gsrc_row[i];
        M.vgap[((k + 1) & 1) * M.n_gsrc + M.gsrc_id[i]] = M.v[nb + (int64_t)row * kLanes];
      }
    }
    // (5) threshold detection and recording
    if (!TRAJ && N > 0) {
      const double vs = M.v[nb + (int64_t)spike_row * kLanes];
      const int now = vs > thresh;
      if (now && !above) mask |= 1ull << s;
      above = now;
      for (int q = 0; q < RR; ++q) {
        if (q < nrec) {
          const int64_t i = rcb + (int64_t)q * kLanes;
          const int row = M.rec_row[i];
          M.trace[(k + 1) * M.n_rec + M.rec_id[i]] = M.v[nb + (int64_t)row * kLanes];
        }
      }
    }
  }
  if (!TRAJ && gid >= 0) {
    M.hist[J * M.n_cells + gid] = mask;
    M.s_above[slot] = (uint8_t)above;
  }
}

// Record step-k voltages.
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

// -------------------------------------------------------------------- adjoint
// Reverse pass of the FP64 backward-Euler map over steps [k0, k1) of one
// checkpoint segment (cn_run_adjoint).  The forward step is
// A_k v_{k+1} = C v_k + b_k, A_k = C + G_k + L, gates_{k+1} = Phi(gates_k,
// v_{k+1}); with lambda_{k+1} = dJ/dv_{k+1} in `lam`, step k computes
//   mu_k = A_k^-T lambda_{k+1}     (Hines on the transposed rows: a <-> b)
//   xi_k = dPhi/dgates_k xi_{k+1} + mu_soma d(GE - G v_{k+1})/dgates_k
//   lambda_k = C mu_k + dJ/dv_k + (dPhi_{k-1}/dv_k)^T xi_k
// and accumulates dJ/dtheta += mu_k . d(b_k - A_k v_{k+1})/dtheta for the
// cell's gnabar, gkbar and pas g.  The row-scaled matrix is A' = A/cdt, so
// A'^T y = lambda gives mu = y/cdt and C mu = y.  One cell per lane, at
// most one HH instance per cell; traj holds v_{k0..k1} and gates_{k0..k1}.
struct AdjView {
  double* lam;      // [node_elems]
  double* ytmp;     // [node_elems]
  double* qtmp;     // [node_elems]
  double* xi;       // [3][n_slots]
  double* grad;     // [3][n_slots]
  const double* dj; // [K+1][n_rec] dJ/d(trace)
  int64_t K;
};

__device__ __forceinline__ double vtrap_d(double A, double vh, double k, double v) {
  // d/dv of A (v - vh) / (1 - exp(-(v - vh)/k))
  const double u = (v - vh) / k;
  if (fabs(u) < 1e-6) return A * (0.5 + u / 3.0);
  const double em = exp(-u), den = 1.0 - em;
  return A * (den - u * em) / (den * den);
}

// Rates, their derivatives, and the cnexp sensitivities at v: for each gate
// dx_new/dx_old = E and dx_new/dv = dinf (1 - E) + (x - inf) dE.
__device__ void hh_sens(double v, double xm, double xh, double xn, double dt, double* E, double* dv) {
  double am, bm, ah, bh, an, bn;
  hh_rates<double>(v, am, bm, ah, bh, an, bn);
  const double dam = vtrap_d(0.1, -40.0, 10.0, v), dbm = -bm / 18.0;
  const double dah = -ah / 20.0, dbh = bh * (1.0 - bh) / 10.0;
  const double dan = vtrap_d(0.01, -55.0, 10.0, v), dbn = -bn / 80.0;
  const double al[3] = {am, ah, an}, be[3] = {bm, bh, bn}, dal[3] = {dam, dah, dan}, dbe[3] = {dbm, dbh, dbn};
  const double x[3] = {xm, xh, xn};
  for (int c = 0; c < 3; ++c) {
    const double s = al[c] + be[c];
    const double inf = al[c] / s;
    const double e = exp(-dt * s);
    const double dinf = (dal[c] * be[c] - al[c] * dbe[c]) / (s * s);
    E[c] = e;
    dv[c] = dinf * (1.0 - e) + (x[c] - inf) * (-dt * (dal[c] + dbe[c]) * e);
  }
}

__global__ void __launch_bounds__(32) k_adjoint(DevModel M, AdjView A, int64_t k0, int64_t k1) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int g = blockIdx.x;
  if (g >= M.n_groups) return;
  const int lane = threadIdx.x;
  const int slot = g * kLanes + lane;
  const int R = M.g_rows[g];
  const int64_t nb = M.g_node_base[g] + lane;
  const int DS = M.stack_depth;
  double* const st_a = reinterpret_cast<double*>(smem) + lane;
  double* const st_x = st_a + DS * kLanes;
  double* const st_y = st_x + DS * kLanes;
  const int nhh = M.s_nhh[slot];
  const int64_t hi = M.g_hh_base[g] + lane;
  const int hrow = nhh > 0 ? M.hh_row[hi] : -1;
  const int64_t H = M.hh_elems, E = M.node_elems;
  const int RR = M.g_rec_rows[g], nrec = M.s_nrec[slot];
  const int64_t rcb = M.g_rec_base[g] + lane;
  const double dt = M.dt;
  double xi[3] = {A.xi[slot], A.xi[M.n_slots + slot], A.xi[2 * M.n_slots + slot]};
  double gna = 0.0, gk = 0.0, gpas = 0.0;
  auto gate = [&](int64_t t, int c) { return M.traj_g[t * 3 * H + c * H + hi]; };
  auto gate_term = [&](int64_t k) {  // (dPhi_{k-1}/dv_k)^T xi_k at the HH row
    double Ek[3], dv[3];
    const int64_t t = k - 1 - k0;
    hh_sens(M.traj_v[(k - k0) * E + nb + (int64_t)hrow * kLanes], gate(t, 0), gate(t, 1), gate(t, 2), dt, Ek, dv);
    return xi[0] * dv[0] + xi[1] * dv[1] + xi[2] * dv[2];
  };
  if (nhh > 0 && k1 < A.K) A.lam[nb + (int64_t)hrow * kLanes] += gate_term(k1);
  for (int64_t k = k1 - 1; k >= k0; --k) {
    const int64_t tv1 = (k + 1 - k0) * E;
    double m = 0.0, h = 0.0, n = 0.0, Gh = 0.0;
    if (nhh > 0) {
      m = gate(k - k0, 0);
      h = gate(k - k0, 1);
      n = gate(k - k0, 2);
      Gh = M.hh_p[hi] * (m * m * m * h) + M.hh_p[H + hi] * ((n * n) * (n * n)) + M.hh_p[2 * H + hi];
    }
    // elimination of the transposed rows, leaves to root
    double ca = 0.0, cx = 0.0, cb = 0.0;
    int top = 0;
    for (int j = R - 1; j >= 0; --j) {
      const int64_t e = nb + (int64_t)j * kLanes;
      const int f = M.flags[e];
      const int np = (f >> kNFarShift) & kNFarMask;
      double rhs = A.lam[e];
      double d = M.d0[e] + (j == hrow ? Gh : 0.0);
      for (int q = 0; q < np; ++q) {
        --top;
        rhs = fma(st_a[top * kLanes], st_x[top * kLanes], rhs);
        d = fma(st_a[top * kLanes], st_y[top * kLanes], d);
      }
      rhs = fma(ca, cx, rhs);
      d = fma(ca, cb, d);
      const double y = rhs / d, q = M.a[e] / d;
      A.ytmp[e] = y;
      A.qtmp[e] = q;
      const double nbc = -M.b[e];
      if (f & kFarBit) {
        st_a[top * kLanes] = nbc;
        st_x[top * kLanes] = y;
        st_y[top * kLanes] = q;
        ++top;
        ca = 0.0;
      } else {
        ca = nbc;
        cx = y;
        cb = q;
      }
    }
    // back substitution, root to leaves; gradients; lambda_k = y
    double yprev = 0.0, mus = 0.0, vs1 = 0.0;
    for (int j = 0; j < R; ++j) {
      const int64_t e = nb + (int64_t)j * kLanes;
      const int f = M.flags[e];
      double yp = yprev;
      if (f & kFarBit) yp = st_x[--top * kLanes];
      const double yj = fma(-A.qtmp[e], yp, A.ytmp[e]);
      const int np = (f >> kNFarShift) & kNFarMask;
      for (int q = 0; q < np; ++q) st_x[top++ * kLanes] = yj;
      yprev = yj;
      if (f & kRealBit) {
        const double mu = yj / M.cdt[e];
        const double v1 = M.traj_v[tv1 + e];
        if (f & kHasPasBit) gpas = fma(mu, M.pas_e[e] - v1, gpas);
        if (j == hrow) {
          mus = mu;
          vs1 = v1;
        }
      }
      A.lam[e] = yj;
    }
    if (nhh > 0) {
      const double ena = M.hh_raw[4 * H + hi], ek = M.hh_raw[5 * H + hi];
      const double gnab = M.hh_raw[hi], gkb = M.hh_raw[H + hi];
      gna = fma(mus, (m * m * m * h) * (ena - vs1), gna);
      gk = fma(mus, ((n * n) * (n * n)) * (ek - vs1), gk);
      double Ek[3], dv[3];
      hh_sens(vs1, m, h, n, dt, Ek, dv);
      xi[0] = Ek[0] * xi[0] + mus * gnab * 3.0 * m * m * h * (ena - vs1);
      xi[1] = Ek[1] * xi[1] + mus * gnab * m * m * m * (ena - vs1);
      xi[2] = Ek[2] * xi[2] + mus * gkb * 4.0 * n * n * n * (ek - vs1);
    }
    if (k >= 1) {
      for (int q = 0; q < RR; ++q) {
        if (q < nrec) {
          const int64_t i = rcb + (int64_t)q * kLanes;
          A.lam[nb + (int64_t)M.rec_row[i] * kLanes] += A.dj[k * M.n_rec + M.rec_id[i]];
        }
      }
      if (nhh > 0 && k > k0) A.lam[nb + (int64_t)hrow * kLanes] += gate_term(k);
    }
  }
  A.xi[slot] = xi[0];
  A.xi[M.n_slots + slot] = xi[1];
  A.xi[2 * M.n_slots + slot] = xi[2];
  A.grad[slot] += gna;
  A.grad[M.n_slots + slot] += gk;
  A.grad[2 * M.n_slots + slot] += gpas;
}

// lambda_K = dJ/dv_K at the recorded rows.
__global__ void k_adjoint_init(DevModel M, AdjView A) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int nrec = M.s_nrec[slot];
  const int64_t rcb = M.g_rec_base[g] + lane, nb = M.g_node_base[g] + lane;
  for (int q = 0; q < nrec; ++q) {
    const int64_t i = rcb + (int64_t)q * kLanes;
    A.lam[nb + (int64_t)M.rec_row[i] * kLanes] += A.dj[A.K * M.n_rec + M.rec_id[i]];
  }
}

// Trajectory entry of the segment's first step (v and gates at k0).
__global__ void k_traj_first(DevModel M) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= M.n_slots) return;
  const int g = slot / kLanes, lane = slot % kLanes;
  const int64_t nb = M.g_node_base[g] + lane;
  for (int j = 0; j < M.g_rows[g]; ++j) M.traj_v[nb + (int64_t)j * kLanes] = M.v[nb + (int64_t)j * kLanes];
  const int nh = M.s_nhh[slot];
  const int64_t hb = M.g_hh_base[g] + lane;
  for (int q = 0; q < nh; ++q) {
    const int64_t i = hb + (int64_t)q * kLanes;
    M.traj_g[i] = static_cast<const double*>(M.hh_m)[i];
    M.traj_g[M.hh_elems + i] = static_cast<const double*>(M.hh_h)[i];
    M.traj_g[2 * M.hh_elems + i] = static_cast<const double*>(M.hh_n)[i];
  }
}

}  // namespace cn
