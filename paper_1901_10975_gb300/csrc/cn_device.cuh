// cn_device.cuh -- device data layout and kernels of the fixed-step engine.
//
// Layout: cells are cut into subtrees ("parts") and the parts are placed on
// the 32 lanes of warps ("groups"); row j of lane l lives at element
// base_g + 32*j + l of every per-row array, so the 32 lanes of a warp touch
// one contiguous 256-byte row of FP64 per array.  Inside a part, rows follow
// a depth-first preorder, so a row's parent is the previous row except for
// the "far" children of branch points, whose contributions are folded into
// partial sums kept on a per-lane stack in shared memory; a part root hangs
// from a junction row of its parent part at a lower warp row (possibly in
// another lane of the warp) and passes its values through a per-warp
// mailbox in shared memory.  Each row of the tree matrix is scaled by 1/cdt
// (cdt = 1e-3 cm/dt), so the right-hand side is v + (sum g E)/cdt and no
// capacitance term is streamed.  One warp advances its parts for a whole
// minimum-delay interval.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace cn {

constexpr int kLanes = 32;
constexpr int kMaxInterval = 64;     // steps per interval (spike mask width)

enum : int32_t { kStatusEvOverflow = 1, kStatusBadState = 2 };

struct EvRec {
  int32_t step;   // step offset inside the interval
  int32_t syn;    // synapse element offset within the target's warp
  double w;       // uS
};

constexpr int kMaxWarpsPerBlock = 4;  // warps (groups) per block of the interval kernel
// Per-row flag word of the interval kernel.
constexpr int32_t kNoSlot = 0x3f;          // bits 0-5: mechanism slot of the row (HH, IClamp); 63 = none
constexpr int32_t kFarBit = 1 << 6;        // the in-part parent is not the previous row
constexpr int kNFarShift = 7;              // bits 7-9: number of far children
constexpr int32_t kNFarMask = 7;
constexpr int32_t kHasPasBit = 1 << 10;
constexpr int32_t kRealBit = 1 << 11;      // a compartment (else an identity padding row)
constexpr int32_t kJuncBit = 1 << 12;      // a child part hangs from this row
constexpr int32_t kProotBit = 1 << 13;     // root of a child part (its parent row is elsewhere)
constexpr int kJmailShift = 14;            // bits 14-22: mailbox entry of the hanging part
constexpr int kPmailShift = 23;            // bits 23-31: mailbox entry of this part root
constexpr int32_t kMailMask = 511;

// ExpSyn column entries: the first and last synapse of a target row's group
constexpr int32_t kSynFirst = 1 << 29;
constexpr int32_t kSynLast = 1 << 30;
constexpr int32_t kSynTgtMask = kSynFirst - 1;

// Channel types of the batched workload (CN_MECH_NA3H .. CN_MECH_KCA), their
// gate-state arrays and their per-cell kinetic parameters (the table columns
// after gbar).  Offsets into the kinetics block per type:
constexpr int kChanTypes = 6;    // NA3H KDR4 KA IH CAHVA KCA
constexpr int kChanGates = 9;    // m h | n | a b | q | m h | c
constexpr int kChanParams = 60;  // 13 + 7 + 13 + 7 + 16 + 4
__host__ __device__ constexpr int chan_gate0(int t) {
  return t == 0 ? 0 : t == 1 ? 2 : t == 2 ? 3 : t == 3 ? 5 : t == 4 ? 6 : t == 5 ? 8 : kChanGates;
}
__host__ __device__ constexpr int chan_kin0(int t) {
  return t == 0 ? 0 : t == 1 ? 13 : t == 2 ? 20 : t == 3 ? 33 : t == 4 ? 40 : t == 5 ? 56 : kChanParams;
}

// Plain-old-data view of a model's device buffers, passed by value.
struct DevModel {
  int32_t n_groups, n_slots, n_cells, D, n_rec;
  int32_t max_slots, stack_depth, n_mail;
  int64_t node_elems;
  double dt;
  int64_t smem_warp;           // dynamic shared memory of one warp (multiple of 16 bytes)
  int64_t* jdev;               // current interval index (advanced by k_next_interval)
  // per group
  const int64_t* g_node_base;  // element index of row 0, lane 0 (multiple of 64)
  const int32_t* g_rows;       // rows (even)
  const int32_t* g_slot_rows;
  const int64_t* g_syn_base;
  const int32_t* g_syn_rows;
  const int64_t* g_hh_base;
  const int32_t* g_hh_rows;
  const int64_t* g_st_base;
  const int32_t* g_st_rows;
  const int64_t* g_gap_base;   // half gap junctions of the lane
  const int32_t* g_gap_rows;
  const int64_t* g_gsrc_base;  // gap peer nodes whose voltage the lane publishes
  const int32_t* g_gsrc_rows;
  const int64_t* g_rec_base;
  const int32_t* g_rec_rows;
  // per slot (group * 32 + lane)
  const int32_t* s_rows;
  const int32_t* s_nslot;
  const int32_t* s_nhh;
  const int32_t* s_nst;
  const int32_t* s_ngap;
  const int32_t* s_ngsrc;
  const int32_t* s_nrec;
  const int32_t* s_gid;
  const int32_t* s_spike_row;
  const double* s_thresh;
  uint8_t* s_above;
  // rows (interleaved); constants are scaled by 1/cdt of their row
  double* v;           // v_k; holds rhs/d between elimination and back substitution
  double* bp;          // b/d of each row, from elimination to back substitution
  const double* ge;    // (pas g e)/cdt
  const double* d0;    // (cdt + pas g + axial couplings)/cdt
  const double* a;     // row p, column i coupling / cdt_p
  const double* b;     // row i, column p coupling / cdt_i
  const int32_t* flags;
  const int32_t* pfar;         // far rows: rows down to the in-part parent (else 0), and the
                               // same for the row kElimRows below (see kPfarAheadShift)
  // synapses (ExpSyn), in warp columns: a warp's synapses grouped by target
  // (owner lane, row) and spread evenly over its 32 lanes
  const int32_t* syn_tgt;   // row * 32 + owner lane | kSynFirst | kSynLast; -1: empty
  double* syn_ge0;          // ge and d0 of the target row (read at kSynFirst)
  double* syn_d00;
  double* syn_g;
  const double* syn_s;      // 100 / (area cdt) of the synapse row
  const double* syn_e;
  const double* syn_decay;  // exp(-dt / tau)
  // HH
  const int32_t* hh_slot;
  const int32_t* hh_row;
  void* hh_m;
  void* hh_h;
  void* hh_n;
  const double* hh_p;       // [6][hh_elems]: gnabar/cdt gkbar/cdt gl/cdt el ena ek
  double* hh_raw;           // [6][hh_elems]: the same, unscaled
  int64_t hh_elems;
  // pas and row scaling, kept to rebuild d0/ge when parameters change
  double* pas_g;            // per row (0 without pas)
  double* pas_e;            // per row
  double* cdt;              // per row: 1e-3 cm/dt
  double* dax;              // per row: axial part of the unscaled diagonal
  // dense channel types of the batched workload (present on every row of a
  // cell): per-group presence mask, per-row scaled gbar and gate states,
  // per-lane kinetics [kChanParams][n_slots], per-row calcium and ica
  const int32_t* g_chmask;
  double* ch_gbar[kChanTypes];
  void* ch_gate[kChanGates];
  const double* ch_kin;
  double* cai;
  double* ge_syn;  // per row: ge plus the ExpSyn sum of G E of the coming step (streamed by the solve)
  double* d0_syn;  // per row: d0 plus the ExpSyn sum of G
  double* ch_g;    // channel conductance of the row for the coming step, / cdt
  double* ch_ge;   // its sum of g E, / cdt
  double* ica;
  // adjoint trajectory (recompute only)
  double* traj_v;           // [step - traj_k0][node_elems]
  double* traj_g;           // [step - traj_k0][3][hh_elems]
  int64_t traj_k0;
  // stimuli
  const int32_t* st_slot;
  // gap junctions: slot of the row, index of the peer voltage, 100 g/(area cdt)
  const int32_t* gap_slot;
  const int32_t* gap_src;
  double* gap_gs;
  const int32_t* gsrc_row;     // published voltages: row in the lane, index
  const int32_t* gsrc_id;
  double* vgap;                // [2][n_gsrc]: peer voltages of even / odd steps
  int32_t n_gsrc;
  const double* st_del;
  const double* st_dur;
  const double* st_amp;     // 100 amp / (area cdt)
  // records
  const int32_t* rec_row;
  const int32_t* rec_id;
  double* trace;            // [step][n_rec]
  // events: lane `slot` owns ev_buf[ev_off[slot], ev_off[slot+1]), sized for
  // the most its synapses can receive in one interval
  int32_t* ev_count;
  EvRec* ev_buf;
  const int64_t* ev_off;    // [n_slots + 1]
  // external events, CSR by slot
  const int64_t* x_off;
  int64_t* x_pos;
  const int64_t* x_step;
  const int32_t* x_syn;
  const double* x_w;
  // incoming NetCons, CSR by target slot, sorted by (src gid, NetCon index)
  const int64_t* in_off;
  const int32_t* in_src;
  const int32_t* in_syn;
  const int32_t* in_dsteps;
  const double* in_w;
  // spike masks, [interval][gid]: bit s = spike at step interval*D + s + 1
  uint64_t* hist;
  int32_t* status;
  // reference layouts only (see cn_ref.cuh): parent element offset within
  // the group (-1: root or padding), node area, and each stimulus's row
  const int32_t* ref_par;
  const double* area;
  const int32_t* st_row;
};

// Rows kept in flight by the per-lane cp.async rings.  Elimination streams
// five FP64 arrays, the flags and the far-parent offsets and spends ~8 FP64
// instructions per row; back substitution streams two arrays and the flags
// and spends one, so its ring is deeper.  Each lane copies and reads only its
// own elements, so the rings need no warp synchronisation.  The two rings
// share memory.  The depths are kept small: the kernel is bound by latency
// across the warps resident per SM sub-partition, and shared memory per warp
// decides how many are resident (3 and 6 rows measured 10% faster than 4 and
// 8 on the network workload, 66% faster than 6 and 12).
constexpr int kElimRows = 3;
constexpr int kBackRows = 6;
// pfar word of a row: bits 0-15 the rows down to this row's in-part parent
// (far rows, else 0); bits 16-31 the same for row j - kElimRows of the lane,
// so that the far parent's v and d0 can be loaded kElimRows rows ahead.
constexpr int32_t kPfarMask = 0xffff;
constexpr int kPfarAheadShift = 16;

__host__ __device__ inline size_t ring_bytes(bool dense) {
  // elimination: v, ge, d0, a, b (+ the channel G, G E), flags, pfar per row
  const size_t elim = (size_t)kElimRows * kLanes * ((dense ? 7 : 5) * sizeof(double) + 2 * sizeof(int32_t));
  const size_t back = (size_t)kBackRows * kLanes * (2 * sizeof(double) + sizeof(int32_t));
  return ((elim > back ? elim : back) + 15) / 16 * 16;
}
// Dynamic shared memory of one warp of the interval kernel: row rings, the
// per-lane stack (three words per entry: elimination keeps a pending
// parent's two partial sums and its row, back substitution the parents'
// voltages), slot buffer, channel reversal potentials and gate kinetics
// (gate_bytes: 8 for FP64 gating, else 4), mailbox.
__host__ __device__ inline size_t interval_smem_bytes(int stack_depth, int max_slots, bool dense, int n_mail,
                                                      int gate_bytes) {
  return ring_bytes(dense) + (size_t)(stack_depth + 1) * kLanes * 3 * sizeof(double) +
         (size_t)max_slots * kLanes * 2 * sizeof(double) +
         (dense ? (size_t)kChanTypes * kLanes * sizeof(double) +
                      (size_t)kChanParams * kLanes * (gate_bytes == 8 ? sizeof(double) : sizeof(float))
                : 0) +
         (size_t)n_mail * 4 * sizeof(double);
}

// Per-thread asynchronous global->shared copies (through L1, so a lane's own
// earlier global stores are observed) and their group bookkeeping.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// --------------------------------------------------------------- arithmetic
// Reciprocal of a pivot d in [2^-1021, 2^1021] (a pivot of the cable matrix
// is >= 1: 1 plus non-negative conductances over cdt), with no FP64
// instruction: GB300 issues one warp-wide FP64 instruction per 64 cycles on
// each SM sub-partition, while its integer pipes are ~30 times faster.
// Newton-Raphson division (Markstein 1990) on d = 2^E m, m in [1, 2): the
// MUFU float reciprocal of m's leading bits (~2^-22) is refined by one
// Newton step y1 = y0 + y0 (1 - m y0) in 32-bit fixed point (limited to
// ~2^-31 by the truncated m), then by a second step in 64-bit fixed point
// with the full 53-bit m (~2^-60), and rounded to 53 bits.  The result is
// within 1 ulp of 1/d and exactly rounded in ~99.95% of cases.
__device__ __forceinline__ double rcp64(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned frac = hi & 0xfffffu;  // d = 2^E m, m = 1.frac in [1, 2)
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(0x3f800000u | (frac << 3) | (lo >> 29))));
  const unsigned rb = __float_as_uint(rf);  // ~1/m in (0.5, 1]
  unsigned y0 = ((rb & 0x7fffffu) | 0x800000u) << 8;                    // 1/m in Q0.32
  y0 = rb >= 0x3f800000u ? 0xffffffffu : rb < 0x3f000000u ? 0x80000000u : y0;
  const unsigned mq = 0x80000000u | (frac << 11) | (lo >> 21);           // m in Q1.31
  const unsigned long long p = (unsigned long long)mq * y0;              // m y0 in Q1.63
  const long long e = (long long)(0x8000000000000000ull - p) >> 12;      // (1 - m y0) 2^51
  long long y1 = (long long)y0 + (((long long)y0 * e) >> 51);
  y1 = y1 > 0xffffffffll ? 0xffffffffll : y1 < 0x80000000ll ? 0x80000000ll : y1;
  // second step in Q0.64 with m in Q1.63
  const unsigned long long f52 = ((unsigned long long)frac << 32) | lo;
  const unsigned long long M = 0x8000000000000000ull | (f52 << 11);
  const unsigned long long Y1 = (unsigned long long)y1 << 32;
  const long long E = (long long)(0x8000000000000000ull - __umul64hi(M, Y1));  // (1 - m y1) 2^63
  const unsigned long long aE = E < 0 ? (unsigned long long)(-E) : (unsigned long long)E;
  const unsigned long long C = (__umul64hi(Y1, aE) << 1) | ((Y1 * aE) >> 63);  // y1 |1 - m y1| 2^64
  const unsigned long long Y2 = E < 0 ? Y1 - C : Y1 + C;                        // 1/m in Q0.64, in (2^63, 2^64)
  // 1/d = 2^(1022 - Eb) (Y2 / 2^63); m = 1 gives the power of two exactly
  const unsigned long long eb = (hi >> 20) & 0x7ffu;
  const unsigned long long mant = ((Y2 + 0x400ull) >> 11) & 0xfffffffffffffull;
  const unsigned long long bits = f52 == 0 ? (2046ull - eb) << 52 : ((2045ull - eb) << 52) | mant;
  return __longlong_as_double((long long)bits);
}

// alpha = A (v - vh) / (1 - exp(-(v - vh)/k)); limit A k (1 + u/2) near vh.
template <typename T>
__device__ __forceinline__ T vtrap(T A, T vh, T k, T v);

template <>
__device__ __forceinline__ double vtrap<double>(double A, double vh, double k, double v) {
  const double u = (v - vh) / k;
  if (fabs(u) < 1e-6) return A * k * (1.0 + 0.5 * u);
  return A * (v - vh) / (1.0 - exp(-u));
}
template <>
__device__ __forceinline__ float vtrap<float>(float A, float vh, float k, float v) {
  const float u = (v - vh) / k;
  if (fabsf(u) < 1e-4f) return A * k * (1.0f + 0.5f * u);
  return A * (v - vh) / -expm1f(-u);
}
__device__ __forceinline__ double dexp_(double x) { return exp(x); }
__device__ __forceinline__ float dexp_(float x) { return expf(x); }
// 1 - exp(-x).  FP64 keeps that form (the oracle's); FP32 uses -expm1(-x),
// which does not lose digits to cancellation when x is small (dt (alpha +
// beta) is ~0.025 for a gate, 3e-4 for the calcium decay).
__device__ __forceinline__ double omexp_(double x) { return 1.0 - exp(-x); }
__device__ __forceinline__ float omexp_(float x) { return -expm1f(-x); }

// Hodgkin-Huxley rate functions (squid axon, 6.3 C, q10 = 1).
template <typename T>
__device__ __forceinline__ void hh_rates(T v, T& am, T& bm, T& ah, T& bh, T& an, T& bn) {
  am = vtrap<T>(T(0.1), T(-40.0), T(10.0), v);
  bm = T(4.0) * dexp_(-(v + T(65.0)) / T(18.0));
  ah = T(0.07) * dexp_(-(v + T(65.0)) / T(20.0));
  bh = T(1.0) / (T(1.0) + dexp_(-(v + T(35.0)) / T(10.0)));
  an = vtrap<T>(T(0.01), T(-55.0), T(10.0), v);
  bn = T(0.125) * dexp_(-(v + T(65.0)) / T(80.0));
}

// One HH rate by kind (0 am, 1 bm, 2 ah, 3 bh, 4 an, 5 bn) with the same
// instruction sequence for every kind, so that the lanes of a warp can each
// evaluate a different rate without diverging:
//   rate = (c0 + c1 w)(c2 + c3 e) / (c4 + c5 e),  w = v - vh, e = exp(-w/k),
// with coefficients 0, 1 and -1 that make each product and sum exact, so the
// value rounds as the rate's own formula in hh_rates does (the vtrap kinds 0
// and 4 keep their small-u limit).
template <typename T>
__device__ __forceinline__ T hh_rate(int kind, T v) {
  const bool vt = kind == 0 || kind == 4;
  const T vh = kind == 0 ? T(-40.0) : kind == 3 ? T(-35.0) : kind == 4 ? T(-55.0) : T(-65.0);
  const T k = kind == 1 ? T(18.0) : kind == 2 ? T(20.0) : kind == 5 ? T(80.0) : T(10.0);
  const T A = kind == 0 ? T(0.1) : kind == 4 ? T(0.01) : kind == 1 ? T(4.0) : kind == 2 ? T(0.07)
                                                                  : kind == 5 ? T(0.125) : T(1.0);
  const T w = v - vh;
  const T u = w / k;
  const T e = dexp_(-u);
  if (vt && (u < T(0) ? -u : u) < (sizeof(T) == 8 ? T(1e-6) : T(1e-4))) return A * k * (T(1.0) + T(0.5) * u);
  const T num = vt ? A * w : A;
  const T fac = (kind == 1 || kind == 2 || kind == 5) ? e : T(1.0);
  const T den = vt ? (sizeof(T) == 8 ? T(1.0) - e : omexp_(u)) : kind == 3 ? T(1.0) + e : T(1.0);
  return num * fac / den;
}

// cnexp: x <- x + (1 - exp(-dt (alpha+beta))) (alpha/(alpha+beta) - x)
template <typename T>
__device__ __forceinline__ T cnexp_step(T x, T al, T be, T dt) {
  const T s = al + be;
  const T inf = al / s;
  return x + omexp_(dt * s) * (inf - x);
}

// Gate storage per precision mode.
template <int PREC> struct GateT;
template <> struct GateT<0> { using S = double; using M = double; };
template <> struct GateT<1> { using S = float; using M = float; };
template <> struct GateT<2> { using S = __nv_bfloat16; using M = float; };

__device__ __forceinline__ double g_load(const double* p) { return *p; }
__device__ __forceinline__ float g_load(const float* p) { return *p; }
__device__ __forceinline__ float g_load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void g_store(double* p, double x) { *p = x; }
__device__ __forceinline__ void g_store(float* p, float x) { *p = x; }
__device__ __forceinline__ void g_store(__nv_bfloat16* p, float x) { *p = __float2bfloat16_rn(x); }
// Stores x and returns the value as stored (rounded for bfloat16).
__device__ __forceinline__ double g_store_ret(double* p, double x) { *p = x; return x; }
__device__ __forceinline__ float g_store_ret(float* p, float x) { *p = x; return x; }
__device__ __forceinline__ float g_store_ret(__nv_bfloat16* p, float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  *p = b;
  return __bfloat162float(b);
}

}  // namespace cn
