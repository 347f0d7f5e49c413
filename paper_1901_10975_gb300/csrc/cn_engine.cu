// cn_engine.cu -- host side of the C ABI declared in include/cn.h.
//
// The host validates inputs, lays cells out for the device (sort by size,
// 32 cells per warp, interleaved rows), uploads the tables and queues the
// kernels.  All model arithmetic (matrix constants, initial gates, every
// simulation step) runs in the kernels of cn_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "cn.h"
#include "cn_kernels.cuh"
#include "cn_ref.cuh"

namespace {

thread_local std::string g_create_error;

int64_t round_half_away(double x) { return (int64_t)std::llround(x); }

const int kNParams[CN_MECH_NTYPES] = {2, 6, 2, 14, 8, 14, 8, 17, 5};
constexpr int kMaxSmemPerBlock = 227 * 1024;  // opt-in dynamic shared memory per block

}  // namespace

// One captured chunk of whole intervals (see replay_chunk).
struct GraphChunk {
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;   // profiling: pull start/end, interval start/end per interval
  bool pending = false;          // events recorded but not read yet
  const void* key_hist = nullptr;
  const void* key_trace = nullptr;
  bool key_prof = false;
  int key_wpb = 0;
};

struct cn_model {
  cn_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  std::vector<void*> allocs;

  // ---- host copy of the description (input order)
  int32_t n_cells = 0;
  int64_t n_nodes = 0;
  std::vector<int32_t> off, parent, spike_node;
  std::vector<double> area, cm, ri, thresh;
  std::vector<int32_t> pas_node, hh_node, syn_node;
  std::vector<double> pas_g, pas_e, hh_par, syn_tau, syn_e;
  // dense channel tables (types CN_MECH_NA3H .. CN_MECH_KCA)
  std::vector<int32_t> ch_node[cn::kChanTypes];
  std::vector<double> ch_par[cn::kChanTypes];  // [n_params][n]
  bool dense = false;
  std::vector<int32_t> nc_src, nc_syn;
  std::vector<double> nc_w, nc_delay;
  std::vector<int32_t> ev_syn;
  std::vector<double> ev_t, ev_w;
  std::vector<int32_t> st_node;
  std::vector<double> st_del, st_dur, st_amp;
  std::vector<int32_t> rec_node;
  std::vector<int32_t> gap_node, gap_peer;  // half gap junctions (global nodes)
  std::vector<double> gap_g;                // uS
  std::vector<int32_t> node_cell;
  std::vector<int32_t> node_row;   // global node -> warp row of its lane
  std::vector<int32_t> node_slot;  // global node -> lane (slot) holding it
  std::vector<int64_t> node_elem;  // global node -> element of the interleaved row arrays
  std::vector<int64_t> hh_elem;    // HH instance -> element of the interleaved HH arrays
  std::vector<int64_t> syn_elem;   // ExpSyn instance -> element of the interleaved synapse arrays
  std::vector<int64_t> x_off_h, x_step_h;  // external events per lane (offsets, steps sorted per lane)
  int64_t max_ds = 0;              // longest NetCon delay in steps
  int64_t raster_from = 0;         // spikes at or before this step are not reported (restored runs)
  std::vector<int32_t> slot_cell;  // lane -> cell (-1 when empty)
  size_t smem_bytes = 0;
  std::vector<int64_t> x_pos0;     // initial external-event cursors
  // adjoint checkpoints: state at steps 0, S, 2S, ...
  int32_t ck_steps = 0;
  std::vector<void*> ck_buf;
  size_t ck_bytes = 0;

  // ---- layout
  bool finalized = false;
  int32_t n_groups = 0, n_slots = 0, D = 0;
  std::vector<int32_t> cell_slot;             // gid -> slot
  std::vector<int64_t> g_node_base, g_syn_base, g_hh_base;
  std::vector<int32_t> hh_slot, hh_q;
  int64_t node_elems = 0, syn_elems = 0, hh_elems = 0, st_elems = 0, rec_elems = 0;
  int gate_bytes = 8;
  cn::DevModel dm{};
  int64_t step = 0;
  int64_t hist_cap = 0;   // intervals
  int64_t trace_cap = 0;  // steps + 1
  int64_t launches = 0;
  int64_t cells_nodes = 0;
  // optional per-launch timing
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_interval, ev_pull;
  std::vector<cudaEvent_t> ev_pool;
  double acc_int_ms = 0.0, acc_pull_ms = 0.0;
  int64_t acc_int_n = 0, acc_pull_n = 0;
  // launch shape and graph replay
  int wpb = 1;                        // warps (groups) per block of the interval kernel
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  GraphChunk gchunk[2];
  int gnext = 0;
  float tuned_ms = 0.f;               // autotuner: time of one interval with the chosen shape

  cn_status fail(cn_status s, const std::string& msg) {
    err = msg;
    return s;
  }
};

namespace {

void* dalloc_raw(cn_model* m, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (m->opt.alloc) {
    p = m->opt.alloc(bytes, m->opt.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) m->allocs.push_back(p);
  return p;
}

void dfree_raw(cn_model* m, void* p) {
  if (!p) return;
  auto it = std::find(m->allocs.begin(), m->allocs.end(), p);
  if (it != m->allocs.end()) m->allocs.erase(it);
  if (m->opt.free) m->opt.free(p, m->opt.alloc_ctx);
  else cudaFree(p);
}

#define CN_TRY_CUDA(m, call)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return (m)->fail(CN_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

template <class T>
cn_status upload(cn_model* m, T** dst, const std::vector<T>& src, size_t min_elems = 0) {
  size_t n = std::max(src.size(), min_elems);
  T* p = static_cast<T*>(dalloc_raw(m, n * sizeof(T)));
  if (!p) return m->fail(CN_ENOMEM, "device allocation failed");
  if (!src.empty())
    CN_TRY_CUDA(m, cudaMemcpyAsync(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, m->stream));
  if (n > src.size())
    CN_TRY_CUDA(m, cudaMemsetAsync(p + src.size(), 0, (n - src.size()) * sizeof(T), m->stream));
  *dst = p;
  return CN_OK;
}

template <class T>
cn_status zeros(cn_model* m, T** dst, size_t n) {
  T* p = static_cast<T*>(dalloc_raw(m, n * sizeof(T)));
  if (!p) return m->fail(CN_ENOMEM, "device allocation failed");
  CN_TRY_CUDA(m, cudaMemsetAsync(p, 0, std::max<size_t>(n, 1) * sizeof(T), m->stream));
  *dst = p;
  return CN_OK;
}

#define CN_CHECK(expr)              \
  do {                              \
    cn_status s_ = (expr);          \
    if (s_ != CN_OK) return s_;     \
  } while (0)

// Interleave per-instance lists: instance i of cell c becomes row q of slot
// cell_slot[c].  Returns per-group row counts/bases and per-slot counts.
// Runs fn(lo, hi) over [0, n) split into contiguous ranges on up to 16 host
// threads (one range, inline, when n is small).
template <class F>
void parallel_ranges(int64_t n, int64_t min_per_thread, F&& fn) {
  const int64_t hc = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(hc, n / std::max<int64_t>(1, min_per_thread)));
  if (nt <= 1) {
    fn((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t) th.emplace_back([&, t] { fn(n * t / nt, n * (t + 1) / nt); });
  for (auto& x : th) x.join();
}

// Stable order of items by (bucket, key): a counting sort by bucket (off is
// the buckets' CSR offsets), then a stable sort of each bucket's run by key,
// the runs spread over host threads.
template <class Key>
std::vector<int64_t> order_by_bucket(const std::vector<int32_t>& bucket, const std::vector<int64_t>& off, Key key) {
  std::vector<int64_t> order(bucket.size());
  std::vector<int64_t> cur(off.begin(), off.end() - 1);
  for (size_t i = 0; i < bucket.size(); ++i) order[cur[bucket[i]]++] = (int64_t)i;
  parallel_ranges((int64_t)off.size() - 1, 256, [&](int64_t lo, int64_t hi) {
    for (int64_t b = lo; b < hi; ++b)
      std::stable_sort(order.begin() + off[b], order.begin() + off[b + 1],
                       [&](int64_t x, int64_t y) { return key(x) < key(y); });
  });
  return order;
}

struct Rows {
  std::vector<int32_t> slot_n;   // per slot
  std::vector<int32_t> g_rows;   // per group
  std::vector<int64_t> g_base;   // per group (elements)
  std::vector<int32_t> inst_slot, inst_q;
  int64_t elems = 0;
};

Rows interleave(const cn_model* m, const std::vector<int32_t>& inst_node, bool rows_descending = false) {
  Rows r;
  r.slot_n.assign(m->n_slots, 0);
  r.inst_slot.resize(inst_node.size());
  r.inst_q.resize(inst_node.size());
  std::vector<int64_t> order(inst_node.size());
  std::iota(order.begin(), order.end(), 0);
  if (rows_descending)  // a lane's instances in elimination order (stable for equal rows)
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
      return m->node_row[inst_node[x]] > m->node_row[inst_node[y]];
    });
  for (int64_t i : order) {
    int s = m->node_slot[inst_node[i]];
    r.inst_slot[i] = s;
    r.inst_q[i] = r.slot_n[s]++;
  }
  r.g_rows.assign(m->n_groups, 0);
  r.g_base.assign(m->n_groups, 0);
  for (int s = 0; s < m->n_slots; ++s)
    r.g_rows[s / cn::kLanes] = std::max(r.g_rows[s / cn::kLanes], r.slot_n[s]);
  int64_t acc = 0;
  for (int g = 0; g < m->n_groups; ++g) {
    r.g_base[g] = acc;
    acc += (int64_t)r.g_rows[g] * cn::kLanes;
  }
  r.elems = acc;
  return r;
}

int64_t elem_of(const Rows& r, size_t inst) {
  int s = r.inst_slot[inst];
  return r.g_base[s / cn::kLanes] + (int64_t)r.inst_q[inst] * cn::kLanes + s % cn::kLanes;
}

// ExpSyn instances in warp columns.  A warp's synapses are grouped by target
// (owner lane, row); the groups are spread over the 32 columns longest first,
// each onto the column that is shortest so far, so that every lane of the warp
// sums about the same number of synapses whatever lane owns them.  One group
// stays in one column, in consecutive positions, so its sum is one lane's.
// tgt[e] = row * 32 + owner lane (plus kSynFirst / kSynLast), -1 if empty.
struct SynPack {
  std::vector<int32_t> g_rows;   // column height per group
  std::vector<int64_t> g_base;
  std::vector<int64_t> elem;     // instance -> element
  std::vector<int32_t> tgt;      // per element
  int64_t elems = 0;
};

SynPack pack_synapses(const cn_model* m) {
  SynPack p;
  const size_t n = m->syn_node.size();
  p.elem.assign(n, 0);
  p.g_rows.assign(m->n_groups, 0);
  p.g_base.assign(m->n_groups, 0);
  std::vector<std::vector<int64_t>> by_group(m->n_groups);
  for (size_t i = 0; i < n; ++i) by_group[m->node_slot[m->syn_node[i]] / cn::kLanes].push_back((int64_t)i);
  struct Pl { int col, pos; };
  std::vector<std::vector<Pl>> place(m->n_groups);
  std::vector<std::vector<std::pair<int64_t, int64_t>>> runs(m->n_groups);  // [begin, end) into by_group
  parallel_ranges(m->n_groups, 64, [&](int64_t g0, int64_t g1) {
  for (int g = (int)g0; g < (int)g1; ++g) {
    auto& v = by_group[g];
    auto key = [&](int64_t i) {
      return std::make_pair(m->node_slot[m->syn_node[i]] % cn::kLanes, m->node_row[m->syn_node[i]]);
    };
    std::stable_sort(v.begin(), v.end(), [&](int64_t x, int64_t y) { return key(x) < key(y); });
    auto& r = runs[g];
    for (size_t b = 0; b < v.size();) {
      size_t e = b + 1;
      while (e < v.size() && key(v[e]) == key(v[b])) ++e;
      r.push_back({(int64_t)b, (int64_t)e});
      b = e;
    }
    std::stable_sort(r.begin(), r.end(), [](const std::pair<int64_t, int64_t>& x, const std::pair<int64_t, int64_t>& y) {
      return x.second - x.first > y.second - y.first;
    });
    int h[cn::kLanes] = {0};
    place[g].resize(v.size());
    for (auto& run : r) {
      int c = 0;
      for (int l = 1; l < cn::kLanes; ++l)
        if (h[l] < h[c]) c = l;
      for (int64_t t = run.first; t < run.second; ++t) place[g][t] = Pl{c, h[c]++};
    }
    for (int l = 0; l < cn::kLanes; ++l) p.g_rows[g] = std::max(p.g_rows[g], h[l]);
  }
  });
  int64_t acc = 0;
  for (int g = 0; g < m->n_groups; ++g) {
    p.g_base[g] = acc;
    acc += (int64_t)p.g_rows[g] * cn::kLanes;
  }
  p.elems = acc;
  p.tgt.assign(std::max<int64_t>(acc, 1), -1);
  for (int g = 0; g < m->n_groups; ++g) {
    const auto& v = by_group[g];
    for (auto& run : runs[g])
      for (int64_t t = run.first; t < run.second; ++t) {
        const int64_t i = v[t];
        const int64_t e = p.g_base[g] + (int64_t)place[g][t].pos * cn::kLanes + place[g][t].col;
        p.elem[i] = e;
        const int lane = m->node_slot[m->syn_node[i]] % cn::kLanes;
        p.tgt[e] = (m->node_row[m->syn_node[i]] * cn::kLanes + lane) | (t == run.first ? cn::kSynFirst : 0) |
                   (t + 1 == run.second ? cn::kSynLast : 0);
      }
  }
  return p;
}

template <class F>
cn_status launch_checked(cn_model* m, F&& f) {
  f();
  m->launches++;
  CN_TRY_CUDA(m, cudaGetLastError());
  return CN_OK;
}

// Gap peer voltages of the current step into the buffer that step reads.
cn_status gap_publish(cn_model* m) {
  if (m->dm.n_gsrc == 0) return CN_OK;
  const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
  cn::DevModel dm = m->dm;
  const int parity = (int)(m->step & 1);
  return launch_checked(m, [&] { cn::k_gap_publish<<<nb, tb, 0, m->stream>>>(dm, parity); });
}

cn_status state_init(cn_model* m) {
  const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
  cn::DevModel dm = m->dm;
  cudaStream_t st = m->stream;
  double v0 = m->opt.v_init_mV;
  switch (m->opt.precision) {
    case CN_PREC_FP64:
      CN_CHECK(launch_checked(m, [&] { cn::k_state_init<0><<<nb, tb, 0, st>>>(dm, v0); }));
      if (m->dense) CN_CHECK(launch_checked(m, [&] { cn::k_setup_dense<0><<<nb, tb, 0, st>>>(dm, v0, false); }));
      break;
    case CN_PREC_GATE_FP32:
      CN_CHECK(launch_checked(m, [&] { cn::k_state_init<1><<<nb, tb, 0, st>>>(dm, v0); }));
      if (m->dense) CN_CHECK(launch_checked(m, [&] { cn::k_setup_dense<1><<<nb, tb, 0, st>>>(dm, v0, false); }));
      break;
    default:
      CN_CHECK(launch_checked(m, [&] { cn::k_state_init<2><<<nb, tb, 0, st>>>(dm, v0); }));
      if (m->dense) CN_CHECK(launch_checked(m, [&] { cn::k_setup_dense<2><<<nb, tb, 0, st>>>(dm, v0, false); }));
      break;
  }
  const int64_t step = m->step;
  m->step = 0;  // state_init always describes step 0
  const cn_status r = gap_publish(m);
  m->step = step;
  return r;
}

// Split plan and row order of one cell.  The cell (local nodes 0..n-1,
// parent[i] < i) is cut into parts (subtrees) that go to lanes of one warp:
// part 0 holds the root; every other part hangs from a "junction" node of
// its parent part and must start above that node's warp row (it is
// eliminated before the junction row and back-substituted after it).  The
// plan's base is the earliest such start (junction row + 1), which makes
// span the cell's critical path; the placer may start a part later.  Rows
// of a part follow a depth-first preorder that visits children leading to
// junctions first, then smaller subtrees first; a row's in-part parent is
// then the previous row except for "far" children, whose contributions nest
// last-in-first-out on a per-lane stack.
struct CellPart {
  int root = 0;          // local node
  int parent_part = -1;
  int jnode = -1;        // local node (in the parent part) the root hangs from
  int base = 0;          // warp row of the part's first row
  std::vector<int32_t> nodes;  // local nodes in row order
};

struct CellPlan {
  std::vector<CellPart> parts;
  std::vector<int32_t> part_of, row_of;  // per local node: part, row within the part
  std::vector<uint8_t> far;              // per local node
  std::vector<int32_t> pfar;             // per local far node: rows down to its in-part parent
  std::vector<int32_t> nfar;             // per local node (in-part far children)
  int depth = 1;                         // far-stack depth needed
  int span = 0;                          // max over parts of base + size
};

// Earliest warp row of each part's first row: one row after the row of its
// junction node in the parent part.  Re-parenting during the split can
// give a part a parent with a larger index, so bases follow the part tree,
// not the index order.
std::vector<int> part_bases(const std::vector<CellPart>& parts, const std::vector<int32_t>& row) {
  std::vector<int> base(parts.size(), -1);
  base[0] = 0;
  for (size_t q0 = 1; q0 < parts.size(); ++q0) {
    std::vector<int> chain;
    int q = (int)q0;
    while (base[q] < 0) {
      chain.push_back(q);
      q = parts[q].parent_part;
    }
    for (auto it = chain.rbegin(); it != chain.rend(); ++it)
      base[*it] = base[parts[*it].parent_part] + row[parts[*it].jnode] + 1;
  }
  return base;
}

CellPlan plan_cell(const int32_t* parent, int n, int target) {
  CellPlan P;
  // children in CSR form: kids of i are cidx[cofs[i] .. cofs[i+1])
  std::vector<int32_t> cofs(n + 1, 0), cidx(n > 0 ? n - 1 : 0);
  for (int i = 1; i < n; ++i) cofs[parent[i] + 1]++;
  for (int i = 0; i < n; ++i) cofs[i + 1] += cofs[i];
  {
    std::vector<int32_t> fill(cofs.begin(), cofs.end() - 1);
    for (int i = 1; i < n; ++i) cidx[fill[parent[i]]++] = i;
  }
  struct Kids {
    const int32_t* b;
    const int32_t* e;
    const int32_t* begin() const { return b; }
    const int32_t* end() const { return e; }
  };
  auto ch = [&](int i) { return Kids{cidx.data() + cofs[i], cidx.data() + cofs[i + 1]}; };
  P.part_of.assign(n, 0);
  P.parts.push_back(CellPart{});
  std::vector<int32_t> child_part_at(n, -1);  // junction node -> child part
  const int want = target > 0 ? std::min(32, std::max(1, (n + target - 1) / target)) : 1;
  // in-part subtree sizes, depths below the part root and part sizes, kept
  // up to date as subtrees move to new parts
  std::vector<int32_t> sub(n), dep(n), mv;
  std::vector<int> psize{n};
  for (int i = n - 1; i >= 0; --i) {
    sub[i] = 1;
    for (int c : ch(i)) sub[i] += sub[c];
  }
  for (int i = 0; i < n; ++i) dep[i] = i == 0 ? 0 : dep[parent[i]] + 1;
  while ((int)P.parts.size() < want) {
    // estimated bases: a child part starts at its junction depth + 1
    const std::vector<int> base = part_bases(P.parts, dep);
    int worst = 0;
    for (size_t q = 1; q < P.parts.size(); ++q)
      if (base[q] + psize[q] > base[worst] + psize[worst]) worst = (int)q;
    const int cur = base[worst] + psize[worst];
    int best_c = -1, best = cur;
    for (int c = 0; c < n; ++c) {
      if (P.part_of[c] != worst || c == P.parts[worst].root || child_part_at[parent[c]] >= 0) continue;
      const int cost = std::max(base[worst] + psize[worst] - sub[c], base[worst] + dep[c] + sub[c]);
      if (cost < best) {
        best = cost;
        best_c = c;
      }
    }
    if (best_c < 0 || best >= cur) break;
    CellPart np_;
    np_.root = best_c;
    np_.parent_part = worst;
    np_.jnode = parent[best_c];
    const int nq = (int)P.parts.size();
    P.parts.push_back(np_);
    child_part_at[parent[best_c]] = nq;
    // move the in-part subtree of best_c (and re-parent child parts hanging
    // inside it); its nodes keep their subtree sizes and rise by best_c's
    // depth, and best_c's in-part ancestors lose its size
    const int d0 = dep[best_c], s0 = sub[best_c];
    mv.assign(1, best_c);
    while (!mv.empty()) {
      int u = mv.back();
      mv.pop_back();
      P.part_of[u] = nq;
      dep[u] -= d0;
      for (int c : ch(u))
        if (P.part_of[c] == worst) mv.push_back(c);
    }
    for (int a = parent[best_c]; a >= 0 && P.part_of[a] == worst; a = a == P.parts[worst].root ? -1 : parent[a])
      sub[a] -= s0;
    psize[worst] -= s0;
    psize.push_back(s0);
    for (size_t q = 1; q < P.parts.size(); ++q)
      if (P.part_of[P.parts[q].jnode] == nq && (int)q != nq) P.parts[q].parent_part = nq;
  }
  // row order inside every part
  for (int i = n - 1; i >= 0; --i) {
    sub[i] = 1;
    for (int c : ch(i))
      if (P.part_of[c] == P.part_of[i]) sub[i] += sub[c];
  }
  std::vector<uint8_t> leads(n, 0);  // in-part subtree contains a junction node
  for (int i = n - 1; i >= 0; --i) {
    if (child_part_at[i] >= 0) leads[i] = 1;
    for (int c : ch(i))
      if (P.part_of[c] == P.part_of[i] && leads[c]) leads[i] = 1;
  }
  P.row_of.assign(n, -1);
  P.far.assign(n, 0);
  P.pfar.assign(n, 0);
  P.nfar.assign(n, 0);
  std::vector<int32_t> cc, st;
  for (size_t q = 0; q < P.parts.size(); ++q) {
    CellPart& pt = P.parts[q];
    st.assign(1, pt.root);
    while (!st.empty()) {
      int u = st.back();
      st.pop_back();
      P.row_of[u] = (int)pt.nodes.size();
      pt.nodes.push_back(u);
      cc.clear();
      for (int c : ch(u))
        if (P.part_of[c] == (int)q) cc.push_back(c);
      // stable insertion sort (a node has a handful of children): children
      // leading to junctions first, then smaller subtrees first
      auto before = [&](int x, int y) { return leads[x] != leads[y] ? leads[x] > leads[y] : sub[x] < sub[y]; };
      for (size_t a = 1; a < cc.size(); ++a)
        for (size_t b = a; b > 0 && before(cc[b], cc[b - 1]); --b) std::swap(cc[b], cc[b - 1]);
      for (auto it = cc.rbegin(); it != cc.rend(); ++it) st.push_back(*it);
    }
    // far flags and stack depth of this part
    const int sz = (int)pt.nodes.size();
    for (int r = 1; r < sz; ++r) {
      const int u = pt.nodes[r];
      if (P.row_of[parent[u]] != r - 1) {
        P.far[u] = 1;
        P.pfar[u] = r - P.row_of[parent[u]];
        P.nfar[parent[u]]++;
      }
    }
    int top = 0, mx = 0;
    for (int r = sz - 1; r >= 0; --r) {
      top -= P.nfar[pt.nodes[r]];
      if (r > 0 && P.far[pt.nodes[r]]) mx = std::max(mx, ++top);
    }
    top = P.nfar[pt.nodes[0]];
    mx = std::max(mx, top);
    for (int r = 1; r < sz; ++r) {
      if (P.far[pt.nodes[r]]) --top;
      top += P.nfar[pt.nodes[r]];
      mx = std::max(mx, top);
    }
    P.depth = std::max(P.depth, mx);
  }
  const std::vector<int> base = part_bases(P.parts, P.row_of);
  for (size_t q = 0; q < P.parts.size(); ++q) P.parts[q].base = base[q];
  for (const CellPart& pt : P.parts) P.span = std::max(P.span, pt.base + (int)pt.nodes.size());
  return P;
}

// Warp height policy of a mapping value: 0 = the opening cell's span,
// 1 = the largest span, 2 = twice the largest span.
int tall_factor(int32_t mapping) {  // warp height in half spans: TALL 2, TALL2 4, both 3
  return ((mapping & CN_MAP_TALL) ? 2 : 0) + ((mapping & CN_MAP_TALL2) ? (mapping & CN_MAP_TALL ? 1 : 4) : 0);
}

// Warp height of a mapping value (CN_MAP_HEIGHT field); 0 = none.
int map_height(int32_t mapping) { return (mapping & CN_MAP_HEIGHT_MASK) >> CN_MAP_HEIGHT_SHIFT; }

// A cn_mapping value, or a span >= 16 with CN_MAP_TALL / CN_MAP_TALL2, or
// with CN_MAP_TALL alone and a warp height of at least 16 rows.
bool valid_mapping(int32_t mapping) {
  const int32_t span = mapping & ~(CN_MAP_TALL | CN_MAP_TALL2 | CN_MAP_HEIGHT_MASK);
  const int h = map_height(mapping);
  if (mapping < 0 || (span > CN_MAP_CONSTDEPTH && span < 16)) return false;
  if ((mapping & (CN_MAP_TALL | CN_MAP_TALL2)) && span < 16) return false;
  return h == 0 || (h >= 16 && (mapping & CN_MAP_TALL) && !(mapping & CN_MAP_TALL2));
}

// Target span (rows per lane) of a mapping value; 0 = never split.
int map_target(int32_t mapping, int64_t n_nodes, int32_t n_cells, bool adjoint) {
  mapping &= ~(CN_MAP_TALL | CN_MAP_TALL2 | CN_MAP_HEIGHT_MASK);
  if (mapping >= 16) return mapping;
  if (mapping == CN_MAP_AUTO && !adjoint && n_cells > 0)
    return (int)std::max<int64_t>(16, (n_nodes + n_cells - 1) / n_cells);
  return 0;
}

// Checks cell_offset / parent as cn_morph requires.
bool valid_trees(int32_t n_cells, const int32_t* off, const int32_t* parent, std::string& err) {
  if (n_cells < 0 || !off || off[0] != 0) {
    err = "bad cell_offset";
    return false;
  }
  for (int c = 0; c < n_cells; ++c) {
    if (off[c + 1] <= off[c]) {
      err = "every cell needs at least one node";
      return false;
    }
    for (int64_t i = off[c]; i < off[c + 1]; ++i) {
      const int64_t li = i - off[c];
      const int32_t p = parent[i];
      if ((li == 0) != (p == -1) || p >= li || p < -1) {
        err = "parent must be cell-local with parent[i] < i and one root at local index 0";
        return false;
      }
    }
  }
  return true;
}

// Placement of every cell on the lanes of the warps.  Each warp is a grid
// of 32 lanes x H rows: H is the span of the cell that opened the warp, or,
// with "tall" warps, the largest span of all cells (or a given warp
// height).  Warps are filled one at a time, cells largest span first; a
// cell goes part by part in part-tree order: the root part into a lane that
// holds no other spike source, each child part where it starts earliest at
// or above the row after its junction (see place() for the rule with a
// warp height).  A child part may start anywhere above its junction row:
// its eliminated (-a, x, b/d) and the junction's back-substituted v pass
// through a per-warp mailbox in shared memory.
// With stacking on, a lane holds parts of several cells one above the
// other; without it (channel kinetics are per lane; the adjoint sums per
// lane) a lane holds parts of one cell only.  Channel sets never share a
// warp.  node_flags holds each node's topology bits (real, far, nfar,
// junction and part root with their mailbox entries); the mechanism-slot
// field is left 0.
struct Layout {
  std::vector<CellPlan> plans;
  int depth = 1;
  int n_groups = 0;
  int n_mail = 1;                             // mailbox entries per warp (max over warps)
  std::vector<int32_t> cell_lane0;            // cell -> lane of its root part (global)
  std::vector<int32_t> lane_rows;             // lane -> rows used
  std::vector<int32_t> lane_cell;             // lane -> its only cell (-1: none or several)
  std::vector<int32_t> node_slot, node_row;   // global node -> lane, warp row
  std::vector<int32_t> node_flags;            // global node -> topology bits
  std::vector<int32_t> node_pfar;             // global node -> rows down to the in-part parent (far nodes)
  std::vector<int32_t> node_paroff;           // reference layouts: parent's element offset in the group (-1: root)
  int max_span = 0;                           // largest cell span of the split plans
};

// Split plans of every cell (in parallel over the host's cores); with a
// warp height, a cell whose span exceeds it is planned again with finer
// targets, keeping its lowest span.
void plan_cells(int32_t n_cells, const int32_t* off, const int32_t* parent, int target, int height,
                std::vector<CellPlan>& plans) {
  plans.assign(n_cells, CellPlan{});
  parallel_ranges(n_cells, 256, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      const int n = off[c + 1] - off[c];
      plans[c] = plan_cell(parent + off[c], n, target);
      for (int t = target - 2; height > 0 && target > 0 && plans[c].span > height && t >= 4; t -= 2) {
        CellPlan P = plan_cell(parent + off[c], n, t);
        if (P.span < plans[c].span) plans[c] = std::move(P);
      }
    }
  });
}

constexpr int kPackLookahead = 512;    // remaining cells tried per warp
// with a warp height:
constexpr int kPackChunks = 16;        // chunks packed in parallel, at most,
constexpr int kPackChunkCells = 1024;  // of at least this many cells each
constexpr int kHoles = 4;              // free runs below a lane's top kept per lane
constexpr int kHoleWeight = 4;         // rows of delay one row of padding is worth

// With a warp height (height > 0, tall warps): cells whose span exceeds it
// are planned again with finer targets, warps are `height` rows tall (or
// the span of a taller cell that opens one), and parts may fill the free
// runs below a lane's top.
bool build_layout(int32_t n_cells, const int32_t* off, const int32_t* parent, const int32_t* cell_mask,
                  const int32_t* spike_node, int target, bool stack, int tall, int height, Layout& L,
                  std::string& err) {
  auto mask = [&](int c) { return cell_mask ? cell_mask[c] : 0; };
  plan_cells(n_cells, off, parent, target, height, L.plans);
  L.depth = 1;
  int H = 1;
  for (int c = 0; c < n_cells; ++c) {
    const int n = off[c + 1] - off[c];
    L.depth = std::max(L.depth, L.plans[c].depth);
    H = std::max(H, L.plans[c].span);
    for (int32_t li = 0; li < n; ++li)
      if (L.plans[c].nfar[li] > (int)cn::kNFarMask) {
        err = "a node has more than 8 children";
        return false;
      }
    if ((int)L.plans[c].parts.size() - 1 > cn::kMailMask + 1) {
      err = "a cell was cut into too many parts";
      return false;
    }
  }
  L.max_span = H;
  std::vector<int32_t> order(n_cells);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (mask(x) != mask(y)) return mask(x) < mask(y);
    return L.plans[x].span > L.plans[y].span;
  });
  struct Warp {
    int lev[cn::kLanes];
    int owner[cn::kLanes];   // -1 free, >= 0 the only cell, -2 several
    bool root[cn::kLanes];
    int n_mail = 0;
    int32_t mask = 0;
    int min_lev = 0;
    int H = 0;               // rows of this warp
    int max_free = 1 << 30;  // longest free run of rows in any lane
    int64_t free_rows = 0;   // free rows over all lanes
    // with a warp height: free runs [hs, he) below a lane's top, left where
    // a part root had to start above its junction row
    int nh[cn::kLanes];
    int hs[cn::kLanes][kHoles], he[cn::kLanes][kHoles];
  };
  // per cell: the placement found
  std::vector<std::vector<int>> kids;
  std::vector<int> po;
  std::vector<int32_t> part_lane_of_cell, part_start_of_cell;  // flattened by cell
  std::vector<int64_t> cell_part0(n_cells + 1, 0);
  for (int c = 0; c < n_cells; ++c) cell_part0[c + 1] = cell_part0[c] + (int64_t)L.plans[c].parts.size();
  part_lane_of_cell.assign(cell_part0[n_cells], -1);
  part_start_of_cell.assign(cell_part0[n_cells], 0);
  std::vector<int> cell_warp(n_cells, -1), warp_mail0(n_cells, 0);
  // per cell, once: parts in part-tree order (parents first), rows, largest part
  std::vector<int32_t> cell_porder(cell_part0[n_cells]), cell_rows(n_cells), cell_maxpart(n_cells);
  for (int c = 0; c < n_cells; ++c) {
    const CellPlan& P = L.plans[c];
    const int np = (int)P.parts.size();
    kids.assign(np, {});
    for (int q = 1; q < np; ++q) kids[P.parts[q].parent_part].push_back(q);
    po.assign(1, 0);
    for (size_t h = 0; h < po.size(); ++h)
      for (int k : kids[po[h]]) po.push_back(k);
    std::copy(po.begin(), po.end(), cell_porder.begin() + cell_part0[c]);
    cell_rows[c] = off[c + 1] - off[c];
    cell_maxpart[c] = 0;
    for (const CellPart& pt : P.parts) cell_maxpart[c] = std::max(cell_maxpart[c], (int)pt.nodes.size());
  }
  std::vector<uint8_t> placed(n_cells, 0);
  // Packs the cells of `ord` (in that order) into `warps`; the lanes it
  // records for a cell's parts count warps from the start of `warps`.
  auto pack = [&](const std::vector<int32_t>& ord, std::vector<Warp>& warps) -> bool {
    const int n = (int)ord.size();
    std::vector<int> porder, pstart, plane;
    // Places cell c's parts in warp w (parents first).  Each part goes to the
    // lane, and with a warp height to the free run or lane top, where it
    // starts earliest (ties: least padding left below it); with `pad_rule`,
    // where padding x kHoleWeight + delay past its release row is least.
    // Returns 0 when placed, 1 when the first part has no room at all (no rule
    // can place the cell), 2 when a later part found none.
    auto place = [&](int c, Warp& w, bool pad_rule) -> int {
      const CellPlan& P = L.plans[c];
      const int np = (int)P.parts.size();
      if (w.n_mail + np - 1 > cn::kMailMask + 1) return 1;
      const int qsp = P.part_of[spike_node ? spike_node[c] : 0];  // the part holding the spike source
      int lev[cn::kLanes], own[cn::kLanes], nh[cn::kLanes], hs[cn::kLanes][kHoles], he[cn::kLanes][kHoles];
      std::copy(w.lev, w.lev + cn::kLanes, lev);
      std::copy(w.owner, w.owner + cn::kLanes, own);
      std::copy(w.nh, w.nh + cn::kLanes, nh);
      std::copy(&w.hs[0][0], &w.hs[0][0] + cn::kLanes * kHoles, &hs[0][0]);
      std::copy(&w.he[0][0], &w.he[0][0] + cn::kLanes * kHoles, &he[0][0]);
      // a new free run [a, b) of lane l (only with a warp height); when the
      // lane's list is full the shortest run stays padding
      auto add_hole = [&](int l, int a, int b) {
        if (height <= 0 || b <= a) return;
        int s = nh[l];
        if (s == kHoles) {
          s = 0;
          for (int h = 1; h < kHoles; ++h)
            if (he[l][h] - hs[l][h] < he[l][s] - hs[l][s]) s = h;
          if (he[l][s] - hs[l][s] >= b - a) return;
        } else {
          ++nh[l];
        }
        hs[l][s] = a;
        he[l][s] = b;
      };
      pstart.assign(np, 0);
      plane.assign(np, -1);
      for (int q : porder) {
        const int size = (int)P.parts[q].nodes.size();
        const int release = q == 0 ? 0 : pstart[P.parts[q].parent_part] + P.row_of[P.parts[q].jnode] + 1;
        int best = -1, bhole = -1, bstart = 0, bgap = 0;
        auto consider = [&](int l, int h, int st, int gap) {
          bool better = best < 0;
          if (!better && pad_rule) {
            const int cst = kHoleWeight * gap + st, cb = kHoleWeight * bgap + bstart;
            better = cst < cb || (cst == cb && st < bstart);
          } else if (!better) {
            better = st < bstart || (st == bstart && gap < bgap);
          }
          if (better) {
            best = l;
            bhole = h;
            bstart = st;
            bgap = gap;
          }
        };
        for (int l = 0; l < cn::kLanes; ++l) {
          if (q == qsp && w.root[l]) continue;
          if (!stack && own[l] != -1 && own[l] != c) continue;
          const int st = std::max(lev[l], release);
          if (st + size <= w.H) consider(l, -1, st, st - lev[l]);
          for (int h = 0; h < nh[l]; ++h) {
            const int sh = std::max(hs[l][h], release);
            if (sh + size <= he[l][h]) consider(l, h, sh, sh - hs[l][h]);
          }
        }
        if (best < 0) return q == porder[0] ? 1 : 2;
        plane[q] = best;
        pstart[q] = bstart;
        if (bhole < 0) {
          add_hole(best, lev[best], bstart);
          lev[best] = bstart + size;
        } else {  // the run splits into what is left below and above the part
          const int a = hs[best][bhole], b = he[best][bhole];
          --nh[best];
          hs[best][bhole] = hs[best][nh[best]];
          he[best][bhole] = he[best][nh[best]];
          add_hole(best, a, bstart);
          add_hole(best, bstart + size, b);
        }
        own[best] = (own[best] == -1 || own[best] == c) ? c : -2;
      }
      std::copy(lev, lev + cn::kLanes, w.lev);
      std::copy(own, own + cn::kLanes, w.owner);
      std::copy(nh, nh + cn::kLanes, w.nh);
      std::copy(&hs[0][0], &hs[0][0] + cn::kLanes * kHoles, &w.hs[0][0]);
      std::copy(&he[0][0], &he[0][0] + cn::kLanes * kHoles, &w.he[0][0]);
      w.root[plane[qsp]] = true;
      w.max_free = 0;
      w.free_rows = 0;
      w.min_lev = cn::kMailMask + (1 << 30);
      for (int l = 0; l < cn::kLanes; ++l) {
        w.max_free = std::max(w.max_free, w.H - w.lev[l]);
        w.free_rows += w.H - w.lev[l];
        int lo = w.lev[l];
        for (int h = 0; h < w.nh[l]; ++h) {
          w.max_free = std::max(w.max_free, w.he[l][h] - w.hs[l][h]);
          w.free_rows += w.he[l][h] - w.hs[l][h];
          lo = std::min(lo, w.hs[l][h]);
        }
        if (!w.root[l]) w.min_lev = std::min(w.min_lev, lo);  // where a spike-source part can go
      }
      return 0;
    };
    auto try_place = [&](int c, Warp& w, int wi) -> bool {
      const int r = height > 0 ? place(c, w, true) : 2;
      if (r == 1 || (r == 2 && place(c, w, false) != 0)) return false;
      const int np = (int)L.plans[c].parts.size();
      warp_mail0[c] = w.n_mail;
      w.n_mail += np - 1;
      cell_warp[c] = wi;
      for (int q = 0; q < np; ++q) {
        part_lane_of_cell[cell_part0[c] + q] = wi * cn::kLanes + plane[q];
        part_start_of_cell[cell_part0[c] + q] = pstart[q];
      }
      return true;
    };
    auto set_order = [&](int c) {
      porder.assign(cell_porder.begin() + cell_part0[c], cell_porder.begin() + cell_part0[c + 1]);
    };
    // a cell cannot fit a warp with fewer free rows than it has, or without a
    // free run as long as its largest part (cheap tests before a placement try)
    // (nor, when its first part holds the spike source and so starts no lower
    // than the lowest lane free of one, if the cell's span does not fit above)
    auto may_fit = [&](int c, const Warp& w) {
      const CellPlan& P = L.plans[c];
      const bool src0 = P.part_of[spike_node ? spike_node[c] : 0] == 0;
      return cell_rows[c] <= w.free_rows && cell_maxpart[c] <= w.max_free && (!src0 || w.min_lev + P.span <= w.H);
    };
    // Fill one warp at a time: it opens with the largest remaining cell and
    // takes, among the next kPackLookahead remaining cells of the same channel
    // set, every cell that still fits; the rest wait for later warps.
    std::vector<int32_t> next_of(n + 1);  // linked list of unplaced cells in order
    for (int k = 0; k <= n; ++k) next_of[k] = k + 1;
    int head = 0;  // position in order of the first unplaced cell
    auto advance = [&](int k) { return next_of[k]; };
      int tail = n;  // cells at positions >= tail are placed (or of another channel set)
    while (head < n) {
      const int c0 = ord[head];
      const CellPlan& P0 = L.plans[c0];
      Warp w;
      std::fill(w.lev, w.lev + cn::kLanes, 0);
      std::fill(w.owner, w.owner + cn::kLanes, -1);
      std::fill(w.root, w.root + cn::kLanes, false);
      std::fill(w.nh, w.nh + cn::kLanes, 0);
      w.mask = mask(c0);
      w.H = !tall ? P0.span : height > 0 ? std::max(height, P0.span) : tall * H / 2;
      warps.push_back(w);
      const int wi = (int)warps.size() - 1;
      set_order(c0);
      if (!try_place(c0, warps[wi], wi)) return false;
      placed[c0] = 1;
      int k = advance(head), seen = 0;
      head = k;  // c0 leaves the list
      int last_kept = -1;
      while (k < n && seen < kPackLookahead) {
        const int c = ord[k];
        if (placed[c]) {  // taken by an earlier warp's gap filling: unlink
          const int nk = advance(k);
          if (last_kept < 0) head = nk;
          else next_of[last_kept] = nk;
          k = nk;
          continue;
        }
        if (mask(c) != w.mask) break;
        ++seen;
        Warp& ww = warps[wi];
        const CellPlan& P = L.plans[c];
        const int size0 = (int)P.parts[P.part_of[spike_node ? spike_node[c] : 0]].nodes.size();
        bool ok = false;
        if (ww.min_lev + size0 <= ww.H && may_fit(c, ww)) {
          set_order(c);
          ok = try_place(c, ww, wi);
        }
        const int nk = advance(k);
        if (ok) {
          placed[c] = 1;
          if (last_kept < 0) head = nk;  // unlink k
          else next_of[last_kept] = nk;
        } else {
          last_kept = k;
        }
        k = nk;
      }
      // then the smallest remaining cells of the same channel set, to fill gaps
      while (tail > 0 && placed[ord[tail - 1]]) --tail;
      int tk = tail;
      seen = 0;
      while (tk > head && seen < kPackLookahead) {
        const int c = ord[tk - 1];
        --tk;
        if (placed[c]) continue;
        if (mask(c) != w.mask) break;
        ++seen;
        Warp& ww = warps[wi];
        const CellPlan& P = L.plans[c];
        const int size0 = (int)P.parts[P.part_of[spike_node ? spike_node[c] : 0]].nodes.size();
        if (ww.min_lev + size0 > ww.H || !may_fit(c, ww)) continue;
        set_order(c);
        if (try_place(c, ww, wi)) placed[c] = 1;
      }
      while (head < n && placed[ord[head]]) head = advance(head);
    }
    return true;
  };
  // With a warp height the cells are dealt round robin (in their sorted
  // order) into up to kPackChunks chunks of at least kPackChunkCells cells,
  // packed in parallel; the count follows from the cell count only, so the
  // layout does not depend on the host's cores.
  std::vector<Warp> warps;
  const int chunks = height > 0 ? std::max(1, std::min(kPackChunks, n_cells / kPackChunkCells)) : 1;
  if (chunks == 1) {
    if (!pack(order, warps)) {
      err = "internal: a cell does not fit an empty warp";
      return false;
    }
  } else {
    std::vector<std::vector<int32_t>> ords(chunks);
    for (int i = 0; i < n_cells; ++i) ords[i % chunks].push_back(order[i]);
    std::vector<std::vector<Warp>> cw(chunks);
    std::vector<uint8_t> ok(chunks, 0);
    parallel_ranges(chunks, 1, [&](int64_t j0, int64_t j1) {
      for (int64_t j = j0; j < j1; ++j) ok[j] = pack(ords[j], cw[j]);
    });
    for (int j = 0; j < chunks; ++j) {
      if (!ok[j]) {
        err = "internal: a cell does not fit an empty warp";
        return false;
      }
      const int w0 = (int)warps.size();
      for (int c : ords[j]) {  // chunk-local warp numbers to global ones
        cell_warp[c] += w0;
        for (int64_t q = cell_part0[c]; q < cell_part0[c + 1]; ++q) part_lane_of_cell[q] += w0 * cn::kLanes;
      }
      warps.insert(warps.end(), cw[j].begin(), cw[j].end());
    }
  }
  L.n_groups = (int)warps.size();
  L.n_mail = 1;
  L.lane_rows.assign((size_t)L.n_groups * cn::kLanes, 0);
  L.lane_cell.assign((size_t)L.n_groups * cn::kLanes, -1);
  for (int wi = 0; wi < L.n_groups; ++wi) {
    L.n_mail = std::max(L.n_mail, warps[wi].n_mail);
    for (int l = 0; l < cn::kLanes; ++l) {
      L.lane_rows[(size_t)wi * cn::kLanes + l] = warps[wi].lev[l];
      L.lane_cell[(size_t)wi * cn::kLanes + l] = warps[wi].owner[l] >= 0 ? warps[wi].owner[l] : -1;
    }
  }
  L.cell_lane0.assign(n_cells, -1);
  const int64_t nn = off[n_cells];
  L.node_slot.assign(nn, 0);
  L.node_row.assign(nn, 0);
  L.node_flags.assign(nn, 0);
  L.node_pfar.assign(nn, 0);
  // cells write disjoint node ranges: spread them over the host's cores
  parallel_ranges(n_cells, 256, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      const CellPlan& P = L.plans[c];
      const int64_t p0 = cell_part0[c];
      L.cell_lane0[c] = part_lane_of_cell[p0];
      for (int32_t li = 0; li < off[c + 1] - off[c]; ++li) {
        const int64_t node = off[c] + li;
        const int q = P.part_of[li];
        L.node_slot[node] = part_lane_of_cell[p0 + q];
        L.node_row[node] = part_start_of_cell[p0 + q] + P.row_of[li];
        int32_t f = cn::kRealBit | (P.far[li] ? cn::kFarBit : 0) | (P.nfar[li] << cn::kNFarShift);
        // mailbox entry of part q (q >= 1): warp_mail0 + q - 1
        if (q > 0 && li == P.parts[q].root)
          f |= cn::kProotBit | (int32_t)((uint32_t)(warp_mail0[c] + q - 1) << cn::kPmailShift);
        L.node_flags[node] = f;
        L.node_pfar[node] = P.pfar[li];
      }
      // the junction of each part (a node carries at most one)
      for (size_t q2 = 1; q2 < P.parts.size(); ++q2)
        L.node_flags[off[c] + P.parts[q2].jnode] |= cn::kJuncBit | ((warp_mail0[c] + (int)q2 - 1) << cn::kJmailShift);
    }
  });
  return true;
}

// The reference layouts, the paper's two GPU node orderings (Section 4.4),
// for k_interval_ref.  Cells go 32 to a warp group in order of decreasing
// size (ties by gid).
//  interleaved: cell p of a group in lane p, its node i at row i.
//  constant depth: the group's nodes level by level (distance from the root;
//    each level starts a new row), within a level by (cell-local index, cell
//    position), filling rows of 32 in that order; a node starts a new row
//    when the row is full or already holds a child of its parent (so
//    children of one node are never updated together, and a later sibling
//    lies in a later row), and a spike source skips lanes that already hold
//    one.
bool build_ref_layout(int32_t n_cells, const int32_t* off, const int32_t* parent, const int32_t* spike_node,
                      bool constdepth, Layout& L, std::string& err) {
  std::vector<int32_t> order(n_cells);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return off[x + 1] - off[x] > off[y + 1] - off[y]; });
  L.plans.clear();
  L.depth = 1;
  L.n_mail = 1;
  L.n_groups = (n_cells + cn::kLanes - 1) / cn::kLanes;
  const int64_t nn = off[n_cells];
  L.node_slot.assign(nn, 0);
  L.node_row.assign(nn, 0);
  L.node_flags.assign(nn, cn::kRealBit);
  L.node_pfar.assign(nn, 0);
  L.node_paroff.assign(nn, -1);
  L.lane_rows.assign((size_t)L.n_groups * cn::kLanes, 0);
  L.lane_cell.assign((size_t)L.n_groups * cn::kLanes, -1);
  L.cell_lane0.assign(n_cells, -1);
  std::vector<int32_t> depth;
  struct Item { int32_t li, p; };
  std::vector<std::vector<Item>> level;
  for (int g = 0; g < L.n_groups; ++g) {
    const int nc = std::min<int>(cn::kLanes, n_cells - g * cn::kLanes);
    const int32_t* cs = order.data() + (size_t)g * cn::kLanes;
    if (!constdepth) {
      for (int p = 0; p < nc; ++p) {
        const int c = cs[p], n = off[c + 1] - off[c], slot = g * cn::kLanes + p;
        L.lane_cell[slot] = c;
        L.lane_rows[slot] = n;
        L.cell_lane0[c] = slot;
        for (int32_t i = 0; i < n; ++i) {
          L.node_slot[off[c] + i] = slot;
          L.node_row[off[c] + i] = i;
          L.node_paroff[off[c] + i] = parent[off[c] + i] < 0 ? -1 : parent[off[c] + i] * cn::kLanes + p;
        }
      }
      continue;
    }
    level.clear();
    for (int p = 0; p < nc; ++p) {
      const int c = cs[p], n = off[c + 1] - off[c];
      depth.assign(n, 0);
      for (int32_t i = 1; i < n; ++i) depth[i] = depth[parent[off[c] + i]] + 1;
      for (int32_t i = 0; i < n; ++i) {
        if ((int)level.size() <= depth[i]) level.resize(depth[i] + 1);
        level[depth[i]].push_back(Item{i, p});
      }
    }
    int row = 0;
    bool spike_lane[cn::kLanes] = {};
    std::vector<std::pair<int32_t, int32_t>> row_parents;  // (cell position, parent) in the current row
    for (auto& lv : level) {
      std::sort(lv.begin(), lv.end(), [](const Item& x, const Item& y) {
        return x.li != y.li ? x.li < y.li : x.p < y.p;
      });
      int pos = 0;
      row_parents.clear();
      for (const Item& it : lv) {
        const int c = cs[it.p];
        const int32_t par = parent[off[c] + it.li];
        const bool src = it.li == (spike_node ? spike_node[c] : 0);
        bool clash = false;
        for (auto& rp : row_parents) clash = clash || (rp.first == it.p && rp.second == par && par >= 0);
        if (pos == cn::kLanes || clash) {
          ++row;
          pos = 0;
          row_parents.clear();
        }
        if (src) {
          while (pos < cn::kLanes && spike_lane[pos]) ++pos;
          if (pos == cn::kLanes) {
            ++row;
            pos = 0;
            row_parents.clear();
            while (pos < cn::kLanes && spike_lane[pos]) ++pos;
            if (pos == cn::kLanes) {
              err = "internal: no lane free of a spike source";
              return false;
            }
          }
          spike_lane[pos] = true;
        }
        const int64_t node = off[c] + it.li;
        L.node_slot[node] = g * cn::kLanes + pos;
        L.node_row[node] = row;
        row_parents.emplace_back(it.p, par);
        ++pos;
      }
      if (pos > 0) ++row;
    }
    for (int l = 0; l < cn::kLanes; ++l) L.lane_rows[(size_t)g * cn::kLanes + l] = row;
    for (int p = 0; p < nc; ++p) {
      const int c = cs[p], n = off[c + 1] - off[c];
      L.cell_lane0[c] = L.node_slot[off[c] + (spike_node ? spike_node[c] : 0)];
      for (int32_t i = 1; i < n; ++i) {
        const int64_t pn = off[c] + parent[off[c] + i];
        L.node_paroff[off[c] + i] = L.node_row[pn] * cn::kLanes + L.node_slot[pn] % cn::kLanes;
      }
    }
  }
  return true;
}

bool is_ref_mapping(int32_t mapping) { return mapping == CN_MAP_INTERLEAVED || mapping == CN_MAP_CONSTDEPTH; }

cn_status finalize(cn_model* m) {
  cn::DevModel& dm = m->dm;
  const double dt = m->opt.dt_ms;
  // interval length: the minimum NetCon delay in steps, at most 64
  int64_t dmin = 0;
  std::vector<int32_t> nc_ds(m->nc_src.size());
  for (size_t j = 0; j < m->nc_src.size(); ++j) {
    int64_t ds = round_half_away(m->nc_delay[j] / dt);
    if (ds < 1) return m->fail(CN_EINVAL, "NetCon delay rounds to less than one step");
    if (ds > (int64_t)1 << 30) return m->fail(CN_EINVAL, "NetCon delay too long");
    nc_ds[j] = (int32_t)ds;
    m->max_ds = std::max<int64_t>(m->max_ds, ds);
    if (dmin == 0 || ds < dmin) dmin = ds;
  }
  m->D = (int32_t)(dmin == 0 ? cn::kMaxInterval : std::min<int64_t>(dmin, cn::kMaxInterval));
  if (!m->gap_node.empty()) m->D = 1;  // gap junctions exchange voltages every step

  // dense channel types: per-cell presence mask and per-cell kinetics (every
  // column after gbar must be uniform within a cell for this mapping)
  std::vector<int32_t> cell_mask(m->n_cells, 0);
  std::vector<double> cell_kin;
  if (m->dense) {
    cell_kin.assign((size_t)cn::kChanParams * m->n_cells, 0.0);
    for (int t = 0; t < cn::kChanTypes; ++t) {
      const auto& nodes = m->ch_node[t];
      const int np = kNParams[CN_MECH_NA3H + t];
      const size_t n = nodes.size();
      std::vector<int32_t> first(m->n_cells, -1);
      std::vector<uint8_t> seen_node(m->n_nodes, 0);
      for (size_t i = 0; i < n; ++i) {
        if (seen_node[nodes[i]]++) return m->fail(CN_EINVAL, "two instances of one channel type on one node");
        const int c = m->node_cell[nodes[i]];
        if (first[c] < 0) {
          first[c] = (int32_t)i;
          cell_mask[c] |= 1 << t;
          for (int q = 1; q < np; ++q)
            cell_kin[(size_t)(cn::chan_kin0(t) + q - 1) * m->n_cells + c] = m->ch_par[t][(size_t)q * n + i];
        } else {
          for (int q = 1; q < np; ++q)
            if (m->ch_par[t][(size_t)q * n + i] != m->ch_par[t][(size_t)q * n + first[c]])
              return m->fail(CN_EINVAL, "channel kinetics must be uniform within a cell (only gbar may vary)");
        }
      }
    }
  }
  // split plans (no split when the adjoint is on or the mapping asks for
  // one cell per lane); target span = mean cell size unless given
  const bool ref = is_ref_mapping(m->opt.mapping);
  if (ref && (m->dense || !m->gap_node.empty() || m->ck_steps > 0 || m->opt.precision != CN_PREC_FP64))
    return m->fail(CN_EINVAL, "the reference layouts take FP64 models of pas, HH, ExpSyn and IClamp "
                              "without gap junctions or the adjoint");
  const int target = map_target(m->opt.mapping, m->n_nodes, m->n_cells, m->ck_steps > 0);
  Layout L;
  {
    std::string lerr;
    const bool ok = ref ? build_ref_layout(m->n_cells, m->off.data(), m->parent.data(), m->spike_node.data(),
                                           m->opt.mapping == CN_MAP_CONSTDEPTH, L, lerr)
                        : build_layout(m->n_cells, m->off.data(), m->parent.data(), cell_mask.data(),
                                       m->spike_node.data(), target, !m->dense && m->ck_steps <= 0,
                                       tall_factor(m->opt.mapping), map_height(m->opt.mapping), L, lerr);
    if (!ok) return m->fail(CN_EINVAL, lerr);
  }
  const int depth = L.depth;
  m->n_groups = L.n_groups;
  m->n_slots = L.n_groups * cn::kLanes;
  m->cell_slot = L.cell_lane0;
  m->node_row = L.node_row;
  m->node_slot = L.node_slot;
  std::vector<int32_t> slot_gid(m->n_slots, -1), slot_rows(m->n_slots, 0), slot_spike(m->n_slots, 0),
      slot_cell(m->n_slots, -1);
  std::vector<double> slot_thresh(m->n_slots, 0.0);
  for (int sl = 0; sl < m->n_slots; ++sl) {
    slot_cell[sl] = L.lane_cell[sl];
    slot_rows[sl] = L.lane_rows[sl];
  }
  for (int c = 0; c < m->n_cells; ++c) {
    const int64_t sn = m->off[c] + m->spike_node[c];
    const int ss = m->node_slot[sn];
    slot_gid[ss] = c;
    slot_spike[ss] = m->node_row[sn];
    slot_thresh[ss] = m->thresh[c];
  }
  m->slot_cell = slot_cell;
  std::vector<int32_t> g_rows(m->n_groups, 0);
  m->g_node_base.assign(m->n_groups, 0);
  for (int s = 0; s < m->n_slots; ++s) g_rows[s / cn::kLanes] = std::max(g_rows[s / cn::kLanes], slot_rows[s]);
  int64_t acc = 0;
  for (int g = 0; g < m->n_groups; ++g) {
    g_rows[g] += g_rows[g] & 1;
    m->g_node_base[g] = acc;
    acc += (int64_t)g_rows[g] * cn::kLanes;
  }
  m->node_elems = acc;
  auto node_elem = [&](int64_t node) {
    const int s = m->node_slot[node];
    return m->g_node_base[s / cn::kLanes] + (int64_t)m->node_row[node] * cn::kLanes + s % cn::kLanes;
  };
  // mechanism slots: distinct rows carrying a point process, per lane
  std::vector<std::vector<int32_t>> lane_slot_rows(m->n_slots);
  std::vector<int32_t> row_slot(m->n_nodes, -1);  // by global node
  auto slot_of_node = [&](int64_t node) {
    if (row_slot[node] < 0) {
      const int sl = m->node_slot[node];
      row_slot[node] = (int32_t)lane_slot_rows[sl].size();
      lane_slot_rows[sl].push_back(m->node_row[node]);
    }
    return row_slot[node];
  };
  // (the reference kernel adds point-process terms in place: no slots)
  std::vector<int32_t> hh_slotid(m->hh_node.size(), 0), st_slotid(m->st_node.size(), 0);
  std::vector<int32_t> gap_slotid(m->gap_node.size(), 0);
  if (!ref) {
    for (size_t i = 0; i < m->hh_node.size(); ++i) hh_slotid[i] = slot_of_node(m->hh_node[i]);
    for (size_t i = 0; i < m->st_node.size(); ++i) st_slotid[i] = slot_of_node(m->st_node[i]);
    for (size_t i = 0; i < m->gap_node.size(); ++i) gap_slotid[i] = slot_of_node(m->gap_node[i]);
  }
  // distinct gap peers: each is published by the lane that holds it
  std::vector<int32_t> gsrc_node, gap_src(m->gap_node.size());
  {
    std::vector<int32_t> id(m->n_nodes, -1);
    for (size_t i = 0; i < m->gap_peer.size(); ++i) {
      int32_t& x = id[m->gap_peer[i]];
      if (x < 0) {
        x = (int32_t)gsrc_node.size();
        gsrc_node.push_back(m->gap_peer[i]);
      }
      gap_src[i] = x;
    }
  }
  int max_slots = 1;
  for (int sl = 0; sl < m->n_slots; ++sl) max_slots = std::max<int>(max_slots, (int)lane_slot_rows[sl].size());
  if (max_slots >= cn::kNoSlot) return m->fail(CN_EINVAL, "too many mechanism rows in one cell part");
  const size_t smem = ref ? 0
                          : cn::interval_smem_bytes(depth, max_slots, m->dense, L.n_mail,
                                                    m->opt.precision == CN_PREC_FP64 ? 8 : 4);
  if (smem > kMaxSmemPerBlock)
    return m->fail(CN_EINVAL, "cell needs " + std::to_string(smem) + " bytes of shared memory (slots " +
                                  std::to_string(max_slots) + ", stack " + std::to_string(depth) + ")");
  m->smem_bytes = smem;
  // per-row flags (interleaved) and per-node geometry (node order)
  std::vector<double> h_gp(acc, 0.0), h_ep(acc, 0.0);
  std::vector<int32_t> h_flags(acc, cn::kNoSlot), h_pfar(acc, 0);
  std::vector<int64_t> h_elem(m->n_nodes);
  for (int64_t node = 0; node < m->n_nodes; ++node) {
    const int64_t e = node_elem(node);
    h_elem[node] = e;
    h_flags[e] = L.node_flags[node] | (row_slot[node] >= 0 ? row_slot[node] : cn::kNoSlot);
    h_pfar[e] = L.node_pfar[node];
  }
  m->node_elem = h_elem;
  // each row's pfar word also carries, in its upper half, the far-parent
  // distance of the row kElimRows below it in the lane
  for (int g = 0; g < m->n_groups && !ref; ++g) {
    const int64_t b0 = m->g_node_base[g];
    for (int j = g_rows[g] - 1; j >= cn::kElimRows; --j)
      for (int l = 0; l < cn::kLanes; ++l) {
        const int64_t e = b0 + (int64_t)j * cn::kLanes + l, e4 = e - (int64_t)cn::kElimRows * cn::kLanes;
        if (h_pfar[e4] > cn::kPfarMask || h_pfar[e] > cn::kPfarMask)
          return m->fail(CN_EINVAL, "a far child lies too many rows above its parent");
        h_pfar[e] |= (h_pfar[e4] & cn::kPfarMask) << cn::kPfarAheadShift;
      }
  }
  for (size_t q = 0; q < m->pas_node.size(); ++q) {
    int64_t e = node_elem(m->pas_node[q]);
    h_gp[e] = m->pas_g[q];
    h_ep[e] = m->pas_e[q];
    h_flags[e] |= cn::kHasPasBit;
  }
  // slots per lane, and the most in any lane of each warp (the kernel clears
  // that many slot-buffer entries)
  std::vector<int32_t> slot_n(m->n_slots, 0), g_slot_rows(m->n_groups, 0);
  for (int sl = 0; sl < m->n_slots; ++sl) slot_n[sl] = (int32_t)lane_slot_rows[sl].size();
  for (int s = 0; s < m->n_slots; ++s) g_slot_rows[s / cn::kLanes] = std::max(g_slot_rows[s / cn::kLanes], slot_n[s]);
  // synapses, HH, stimuli, records
  SynPack rs = pack_synapses(m);
  Rows rh = interleave(m, m->hh_node), rt = interleave(m, m->st_node), rr = interleave(m, m->rec_node);
  Rows rg = interleave(m, m->gap_node), rgs = interleave(m, gsrc_node);
  std::vector<int32_t> h_gap_slot(std::max<int64_t>(rg.elems, 1), 0), h_gap_src(std::max<int64_t>(rg.elems, 1), 0);
  std::vector<double> h_gap_area(std::max<int64_t>(rg.elems, 1), 1.0), h_gap_cm(std::max<int64_t>(rg.elems, 1), 1.0),
      h_gap_g(std::max<int64_t>(rg.elems, 1), 0.0);
  for (size_t i = 0; i < m->gap_node.size(); ++i) {
    const int64_t e = elem_of(rg, i);
    h_gap_slot[e] = gap_slotid[i];
    h_gap_src[e] = gap_src[i];
    h_gap_area[e] = m->area[m->gap_node[i]];
    h_gap_cm[e] = m->cm[m->gap_node[i]];
    h_gap_g[e] = m->gap_g[i];
  }
  std::vector<int32_t> h_gsrc_row(std::max<int64_t>(rgs.elems, 1), 0), h_gsrc_id(std::max<int64_t>(rgs.elems, 1), 0);
  for (size_t i = 0; i < gsrc_node.size(); ++i) {
    const int64_t e = elem_of(rgs, i);
    h_gsrc_row[e] = m->node_row[gsrc_node[i]];
    h_gsrc_id[e] = (int32_t)i;
  }
  m->syn_elem = rs.elem;
  m->hh_slot = rh.inst_slot; m->hh_q = rh.inst_q;
  m->g_syn_base = rs.g_base;
  m->g_hh_base = rh.g_base;
  m->syn_elems = rs.elems; m->hh_elems = rh.elems; m->st_elems = rt.elems; m->rec_elems = rr.elems;
  std::vector<double> h_syn_tau(rs.elems, 1.0), h_syn_e(rs.elems, 0.0), h_syn_area(rs.elems, 1.0),
      h_syn_cm(rs.elems, 1.0);
  for (size_t i = 0; i < m->syn_node.size(); ++i) {
    const int64_t e = rs.elem[i];
    h_syn_tau[e] = m->syn_tau[i];
    h_syn_e[e] = m->syn_e[i];
    h_syn_area[e] = m->area[m->syn_node[i]];
    h_syn_cm[e] = m->cm[m->syn_node[i]];
  }
  std::vector<int32_t> h_hh_row(rh.elems, 0), h_hh_slot(rh.elems, 0);
  std::vector<double> h_hh_p(6 * rh.elems, 0.0), h_hh_cm(rh.elems, 1.0);
  size_t nhh = m->hh_node.size();
  m->hh_elem.assign(nhh, 0);
  for (size_t i = 0; i < nhh; ++i) {
    int64_t e = elem_of(rh, i);
    m->hh_elem[i] = e;
    h_hh_row[e] = m->node_row[m->hh_node[i]];
    h_hh_slot[e] = hh_slotid[i];
    h_hh_cm[e] = m->cm[m->hh_node[i]];
    for (int p = 0; p < 6; ++p) h_hh_p[p * rh.elems + e] = m->hh_par[p * nhh + i];
  }
  std::vector<int32_t> h_st_slot(rt.elems, 0), h_st_row(std::max<int64_t>(rt.elems, 1), 0);
  std::vector<double> h_st_del(rt.elems, 0.0), h_st_dur(rt.elems, 0.0), h_st_amp(rt.elems, 0.0),
      h_st_area(rt.elems, 1.0), h_st_cm(rt.elems, 1.0);
  for (size_t i = 0; i < m->st_node.size(); ++i) {
    int64_t e = elem_of(rt, i);
    h_st_slot[e] = st_slotid[i];
    h_st_row[e] = m->node_row[m->st_node[i]];
    h_st_del[e] = m->st_del[i];
    h_st_dur[e] = m->st_dur[i];
    h_st_amp[e] = m->st_amp[i];
    h_st_area[e] = m->area[m->st_node[i]];
    h_st_cm[e] = m->cm[m->st_node[i]];
  }
  std::vector<int32_t> h_rec_row(rr.elems, 0), h_rec_id(rr.elems, 0);
  for (size_t i = 0; i < m->rec_node.size(); ++i) {
    int64_t e = elem_of(rr, i);
    h_rec_row[e] = m->node_row[m->rec_node[i]];
    h_rec_id[e] = (int32_t)i;
  }
  // an event names its synapse by the element offset within the target's warp
  auto syn_off = [&](int32_t i) {
    return (int32_t)(rs.elem[i] - rs.g_base[m->node_slot[m->syn_node[i]] / cn::kLanes]);
  };
  // incoming NetCons per target slot, by (source gid, NetCon index)
  size_t nnc = m->nc_src.size();
  std::vector<int64_t> in_off(m->n_slots + 1, 0);
  std::vector<int32_t> nc_tslot(nnc);
  for (size_t j = 0; j < nnc; ++j) {
    nc_tslot[j] = m->node_slot[m->syn_node[m->nc_syn[j]]];
    in_off[nc_tslot[j] + 1]++;
  }
  for (int s = 0; s < m->n_slots; ++s) in_off[s + 1] += in_off[s];
  const std::vector<int64_t> nc_order = order_by_bucket(nc_tslot, in_off, [&](int64_t j) { return m->nc_src[j]; });
  std::vector<int32_t> h_in_src(nnc), h_in_syn(nnc), h_in_ds(nnc);
  std::vector<double> h_in_w(nnc);
  for (size_t q = 0; q < nnc; ++q) {
    int64_t j = nc_order[q];
    h_in_src[q] = m->nc_src[j];
    h_in_syn[q] = syn_off(m->nc_syn[j]);
    h_in_ds[q] = nc_ds[j];
    h_in_w[q] = m->nc_w[j];
  }
  // external events per target slot, by (step, input index)
  size_t nev = m->ev_syn.size();
  std::vector<int64_t> x_off(m->n_slots + 1, 0), ev_step(nev);
  std::vector<int32_t> ev_tslot(nev);
  for (size_t e = 0; e < nev; ++e) {
    ev_step[e] = std::max<int64_t>(0, round_half_away(m->ev_t[e] / dt));
    ev_tslot[e] = m->node_slot[m->syn_node[m->ev_syn[e]]];
    x_off[ev_tslot[e] + 1]++;
  }
  for (int s = 0; s < m->n_slots; ++s) x_off[s + 1] += x_off[s];
  const std::vector<int64_t> ev_order = order_by_bucket(ev_tslot, x_off, [&](int64_t e) { return ev_step[e]; });
  std::vector<int64_t> h_x_step(nev);
  std::vector<int32_t> h_x_syn(nev);
  std::vector<double> h_x_w(nev);
  for (size_t q = 0; q < nev; ++q) {
    int64_t e = ev_order[q];
    h_x_step[q] = ev_step[e];
    h_x_syn[q] = syn_off(m->ev_syn[e]);
    h_x_w[q] = m->ev_w[e];
  }

  // ---- upload
  dm = cn::DevModel{};
  m->gate_bytes = m->opt.precision == CN_PREC_FP64 ? 8 : (m->opt.precision == CN_PREC_GATE_FP32 ? 4 : 2);
  dm.n_groups = m->n_groups;
  dm.n_slots = m->n_slots;
  dm.n_cells = m->n_cells;
  dm.D = m->D;
  dm.n_rec = (int32_t)m->rec_node.size();
  dm.max_slots = max_slots;
  dm.stack_depth = depth;
  dm.n_mail = L.n_mail;
  dm.node_elems = acc;
  dm.dt = dt;
  int64_t* p64;
  int32_t* p32;
  double* pd;
  CN_CHECK(upload(m, &p64, m->g_node_base)); dm.g_node_base = p64;
  CN_CHECK(upload(m, &p32, g_rows)); dm.g_rows = p32;
  CN_CHECK(upload(m, &p32, g_slot_rows)); dm.g_slot_rows = p32;
  CN_CHECK(upload(m, &p64, rs.g_base)); dm.g_syn_base = p64;
  CN_CHECK(upload(m, &p32, rs.g_rows)); dm.g_syn_rows = p32;
  CN_CHECK(upload(m, &p64, rh.g_base)); dm.g_hh_base = p64;
  CN_CHECK(upload(m, &p32, rh.g_rows)); dm.g_hh_rows = p32;
  CN_CHECK(upload(m, &p64, rt.g_base)); dm.g_st_base = p64;
  CN_CHECK(upload(m, &p32, rt.g_rows)); dm.g_st_rows = p32;
  CN_CHECK(upload(m, &p64, rr.g_base)); dm.g_rec_base = p64;
  CN_CHECK(upload(m, &p32, rr.g_rows)); dm.g_rec_rows = p32;
  CN_CHECK(upload(m, &p32, slot_rows)); dm.s_rows = p32;
  CN_CHECK(upload(m, &p32, slot_n)); dm.s_nslot = p32;
  CN_CHECK(upload(m, &p32, rh.slot_n)); dm.s_nhh = p32;
  CN_CHECK(upload(m, &p32, rt.slot_n)); dm.s_nst = p32;
  CN_CHECK(upload(m, &p64, rg.g_base)); dm.g_gap_base = p64;
  CN_CHECK(upload(m, &p32, rg.g_rows)); dm.g_gap_rows = p32;
  CN_CHECK(upload(m, &p32, rg.slot_n)); dm.s_ngap = p32;
  CN_CHECK(upload(m, &p64, rgs.g_base)); dm.g_gsrc_base = p64;
  CN_CHECK(upload(m, &p32, rgs.g_rows)); dm.g_gsrc_rows = p32;
  CN_CHECK(upload(m, &p32, rgs.slot_n)); dm.s_ngsrc = p32;
  CN_CHECK(upload(m, &p32, h_gap_slot)); dm.gap_slot = p32;
  CN_CHECK(upload(m, &p32, h_gap_src)); dm.gap_src = p32;
  CN_CHECK(zeros(m, &pd, h_gap_g.size())); dm.gap_gs = pd;
  CN_CHECK(upload(m, &p32, h_gsrc_row)); dm.gsrc_row = p32;
  CN_CHECK(upload(m, &p32, h_gsrc_id)); dm.gsrc_id = p32;
  CN_CHECK(zeros(m, &pd, 2 * std::max<size_t>(gsrc_node.size(), 1))); dm.vgap = pd;
  dm.n_gsrc = (int32_t)gsrc_node.size();
  CN_CHECK(upload(m, &p32, rr.slot_n)); dm.s_nrec = p32;
  CN_CHECK(upload(m, &p32, slot_gid)); dm.s_gid = p32;
  CN_CHECK(upload(m, &p32, slot_spike)); dm.s_spike_row = p32;
  CN_CHECK(upload(m, &pd, slot_thresh)); dm.s_thresh = pd;
  uint8_t* pu8;
  CN_CHECK(zeros(m, &pu8, m->n_slots)); dm.s_above = pu8;
  CN_CHECK(zeros(m, &pd, acc)); dm.v = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.bp = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.ge = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.d0 = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.ge_syn = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.d0_syn = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.a = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.b = pd;
  CN_CHECK(upload(m, &p32, h_flags)); dm.flags = p32;
  CN_CHECK(upload(m, &p32, h_pfar)); dm.pfar = p32;
  CN_CHECK(upload(m, &p32, rs.tgt)); dm.syn_tgt = p32;
  CN_CHECK(zeros(m, &pd, rs.elems)); dm.syn_ge0 = pd;
  CN_CHECK(zeros(m, &pd, rs.elems)); dm.syn_d00 = pd;
  CN_CHECK(zeros(m, &pd, rs.elems)); dm.syn_g = pd;
  CN_CHECK(zeros(m, &pd, rs.elems)); dm.syn_s = pd;
  CN_CHECK(upload(m, &pd, h_syn_e)); dm.syn_e = pd;
  CN_CHECK(zeros(m, &pd, rs.elems)); dm.syn_decay = pd;
  CN_CHECK(upload(m, &p32, h_hh_slot)); dm.hh_slot = p32;
  CN_CHECK(upload(m, &p32, h_hh_row)); dm.hh_row = p32;
  for (void** gp : {&dm.hh_m, &dm.hh_h, &dm.hh_n}) {
    void* q = dalloc_raw(m, std::max<int64_t>(rh.elems, 1) * m->gate_bytes);
    if (!q) return m->fail(CN_ENOMEM, "device allocation failed");
    CN_TRY_CUDA(m, cudaMemsetAsync(q, 0, std::max<int64_t>(rh.elems, 1) * m->gate_bytes, m->stream));
    *gp = q;
  }
  CN_CHECK(zeros(m, &pd, 6 * std::max<int64_t>(rh.elems, 1))); dm.hh_p = pd;
  CN_CHECK(upload(m, &pd, h_hh_p, 6)); dm.hh_raw = pd;
  dm.hh_elems = rh.elems;
  CN_CHECK(upload(m, &pd, h_gp)); dm.pas_g = pd;
  CN_CHECK(upload(m, &pd, h_ep)); dm.pas_e = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.cdt = pd;
  CN_CHECK(zeros(m, &pd, acc)); dm.dax = pd;
  if (m->dense) {
    std::vector<int32_t> g_mask(m->n_groups, 0);
    std::vector<double> h_kin((size_t)cn::kChanParams * m->n_slots, 0.0);
    for (int sl = 0; sl < m->n_slots; ++sl) {
      const int c = m->slot_cell[sl];
      if (c < 0) continue;
      g_mask[sl / cn::kLanes] |= cell_mask[c];
      for (int q = 0; q < cn::kChanParams; ++q)
        h_kin[(size_t)q * m->n_slots + sl] = cell_kin[(size_t)q * m->n_cells + c];
    }
    CN_CHECK(upload(m, &p32, g_mask)); dm.g_chmask = p32;
    CN_CHECK(upload(m, &pd, h_kin)); dm.ch_kin = pd;
    bool need_ca = false;
    for (int t = 0; t < cn::kChanTypes; ++t) {
      if (m->ch_node[t].empty()) continue;
      if (t >= 4) need_ca = true;
      std::vector<double> h_g(acc, 0.0);
      for (size_t i = 0; i < m->ch_node[t].size(); ++i) h_g[node_elem(m->ch_node[t][i])] = m->ch_par[t][i];
      CN_CHECK(upload(m, &pd, h_g)); dm.ch_gbar[t] = pd;
      const int g0 = cn::chan_gate0(t), g1 = t + 1 < cn::kChanTypes ? cn::chan_gate0(t + 1) : cn::kChanGates;
      for (int gi = g0; gi < g1; ++gi) {
        void* q = dalloc_raw(m, (size_t)acc * m->gate_bytes);
        if (!q) return m->fail(CN_ENOMEM, "device allocation failed");
        CN_TRY_CUDA(m, cudaMemsetAsync(q, 0, (size_t)acc * m->gate_bytes, m->stream));
        dm.ch_gate[gi] = q;
      }
    }
    if (need_ca) {
      CN_CHECK(zeros(m, &pd, acc)); dm.cai = pd;
      CN_CHECK(zeros(m, &pd, acc)); dm.ica = pd;
    }
    CN_CHECK(zeros(m, &pd, acc)); dm.ch_g = pd;
    CN_CHECK(zeros(m, &pd, acc)); dm.ch_ge = pd;
  }
  CN_CHECK(upload(m, &p32, h_st_slot)); dm.st_slot = p32;
  CN_CHECK(upload(m, &pd, h_st_del)); dm.st_del = pd;
  CN_CHECK(upload(m, &pd, h_st_dur)); dm.st_dur = pd;
  if (ref) {  // the reference kernel takes the amplitudes as given (nA)
    CN_CHECK(upload(m, &pd, h_st_amp)); dm.st_amp = pd;
    CN_CHECK(upload(m, &p32, h_st_row)); dm.st_row = p32;
    std::vector<double> h_area_e(acc, 1.0);
    std::vector<int32_t> h_par(acc, -1);
    for (int64_t node = 0; node < m->n_nodes; ++node) {
      h_area_e[h_elem[node]] = m->area[node];
      h_par[h_elem[node]] = L.node_paroff[node];
    }
    CN_CHECK(upload(m, &pd, h_area_e)); dm.area = pd;
    CN_CHECK(upload(m, &p32, h_par)); dm.ref_par = p32;
  } else {
    CN_CHECK(zeros(m, &pd, rt.elems)); dm.st_amp = pd;
  }
  CN_CHECK(upload(m, &p32, h_rec_row)); dm.rec_row = p32;
  CN_CHECK(upload(m, &p32, h_rec_id)); dm.rec_id = p32;
  CN_CHECK(zeros(m, &p32, m->n_slots)); dm.ev_count = p32;
  // Event buffer of each lane, sized for the most its synapses can receive
  // in one interval: its external events of the busiest interval, plus, per
  // incoming NetCon, ceil(D/2) spikes (a source spikes at most every other
  // step: it must fall back to threshold or below before it can cross
  // again), so no delivery is ever dropped.
  std::vector<int64_t> ev_off(m->n_slots + 1, 0);
  for (int sl = 0; sl < m->n_slots; ++sl) {
    int64_t ext = 0, run = 0, cur = -1;
    for (int64_t q = x_off[sl]; q < x_off[sl + 1]; ++q) {
      const int64_t J = h_x_step[q] / m->D;
      run = J == cur ? run + 1 : 1;
      cur = J;
      ext = std::max(ext, run);
    }
    ev_off[sl + 1] = ev_off[sl] + ext + (in_off[sl + 1] - in_off[sl]) * ((m->D + 1) / 2);
  }
  cn::EvRec* pev = static_cast<cn::EvRec*>(dalloc_raw(m, (size_t)std::max<int64_t>(ev_off.back(), 1) * sizeof(cn::EvRec)));
  if (!pev) return m->fail(CN_ENOMEM, "device allocation failed");
  dm.ev_buf = pev;
  CN_CHECK(upload(m, &p64, ev_off)); dm.ev_off = p64;
  CN_CHECK(upload(m, &p64, x_off)); dm.x_off = p64;
  std::vector<int64_t> x_pos(x_off.begin(), x_off.end() - 1);
  CN_CHECK(upload(m, &p64, x_pos)); dm.x_pos = p64;
  CN_CHECK(upload(m, &p64, h_x_step)); dm.x_step = p64;
  m->x_off_h = x_off;
  m->x_step_h = h_x_step;
  CN_CHECK(upload(m, &p32, h_x_syn)); dm.x_syn = p32;
  CN_CHECK(upload(m, &pd, h_x_w)); dm.x_w = pd;
  CN_CHECK(upload(m, &p64, in_off)); dm.in_off = p64;
  CN_CHECK(upload(m, &p32, h_in_src)); dm.in_src = p32;
  CN_CHECK(upload(m, &p32, h_in_syn)); dm.in_syn = p32;
  CN_CHECK(upload(m, &p32, h_in_ds)); dm.in_dsteps = p32;
  CN_CHECK(upload(m, &pd, h_in_w)); dm.in_w = pd;
  CN_CHECK(zeros(m, &p32, 1)); dm.status = p32;
  CN_CHECK(zeros(m, &p64, 1)); dm.jdev = p64;
  dm.smem_warp = (int64_t)m->smem_bytes;
  dm.hist = nullptr;
  dm.trace = nullptr;

  // temporaries for the setup kernels
  double *d_area, *d_ri, *d_cm, *d_syn_area, *d_syn_cm, *d_syn_tau, *d_st_amp, *d_st_area, *d_st_cm;
  int32_t *d_parent, *d_off;
  int64_t* d_elem;
  CN_CHECK(upload(m, &d_area, m->area));
  CN_CHECK(upload(m, &d_ri, m->ri));
  CN_CHECK(upload(m, &d_cm, m->cm));
  CN_CHECK(upload(m, &d_parent, m->parent));
  CN_CHECK(upload(m, &d_off, m->off));
  CN_CHECK(upload(m, &d_elem, h_elem));
  CN_CHECK(upload(m, &d_syn_area, h_syn_area));
  CN_CHECK(upload(m, &d_syn_cm, h_syn_cm));
  CN_CHECK(upload(m, &d_syn_tau, h_syn_tau));
  CN_CHECK(upload(m, &d_st_amp, h_st_amp));
  CN_CHECK(upload(m, &d_st_area, h_st_area));
  CN_CHECK(upload(m, &d_st_cm, h_st_cm));
  const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
  cudaStream_t st = m->stream;
  const int nbe = (int)((acc + 255) / 256), nbc = (m->n_cells + tb - 1) / tb;
  CN_CHECK(launch_checked(m, [&] { cn::k_setup_pad<<<nbe, 256, 0, st>>>(dm); }));
  CN_CHECK(launch_checked(m, [&] { cn::k_setup_geom<<<nbc, tb, 0, st>>>(dm, m->n_cells, d_off, d_parent, d_area, d_ri, d_cm, d_elem, !ref); }));
  CN_CHECK(launch_checked(m, [&] { cn::k_pas_apply<<<nb, tb, 0, st>>>(dm); }));
  CN_CHECK(launch_checked(m, [&] { cn::k_setup_syn<<<nb, tb, 0, st>>>(dm, d_syn_area, d_syn_cm, d_syn_tau); }));
  CN_CHECK(launch_checked(m, [&] { cn::k_syn_consts<<<nb, tb, 0, st>>>(dm); }));
  CN_CHECK(launch_checked(m, [&] { cn::k_hh_params<<<nb, tb, 0, st>>>(dm); }));
  if (!ref) CN_CHECK(launch_checked(m, [&] { cn::k_setup_stim<<<nb, tb, 0, st>>>(dm, d_st_amp, d_st_area, d_st_cm); }));
  if (rg.elems > 0) {
    double *d_ga, *d_gc, *d_gg;
    CN_CHECK(upload(m, &d_ga, h_gap_area));
    CN_CHECK(upload(m, &d_gc, h_gap_cm));
    CN_CHECK(upload(m, &d_gg, h_gap_g));
    const int64_t ng = rg.elems;
    CN_CHECK(launch_checked(m, [&] { cn::k_setup_gap<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(dm, d_ga, d_gc, d_gg, ng); }));
    CN_TRY_CUDA(m, cudaStreamSynchronize(st));
    for (double* q : {d_ga, d_gc, d_gg}) dfree_raw(m, q);
  }
  if (m->dense) {
    const double v0 = m->opt.v_init_mV;
    switch (m->opt.precision) {
      case CN_PREC_FP64: CN_CHECK(launch_checked(m, [&] { cn::k_setup_dense<0><<<nb, tb, 0, st>>>(dm, v0, true); })); break;
      case CN_PREC_GATE_FP32: CN_CHECK(launch_checked(m, [&] { cn::k_setup_dense<1><<<nb, tb, 0, st>>>(dm, v0, true); })); break;
      default: CN_CHECK(launch_checked(m, [&] { cn::k_setup_dense<2><<<nb, tb, 0, st>>>(dm, v0, true); })); break;
    }
  }
  CN_CHECK(state_init(m));
  CN_TRY_CUDA(m, cudaStreamSynchronize(st));
  for (double* p : {d_area, d_ri, d_cm, d_syn_area, d_syn_cm, d_syn_tau, d_st_amp, d_st_area, d_st_cm}) dfree_raw(m, p);
  dfree_raw(m, d_parent);
  dfree_raw(m, d_off);
  dfree_raw(m, d_elem);
  m->x_pos0 = x_pos;
  for (auto fn : {(const void*)cn::k_interval<0, false, false>, (const void*)cn::k_interval<1, false, false>,
                  (const void*)cn::k_interval<2, false, false>, (const void*)cn::k_interval<0, true, false>,
                  (const void*)cn::k_interval<0, false, true>, (const void*)cn::k_interval<1, false, true>,
                  (const void*)cn::k_interval<2, false, true>})
    CN_TRY_CUDA(m, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemPerBlock));
  m->wpb = ref ? 1 : std::max(1, std::min<int>(m->wpb, (int)(kMaxSmemPerBlock / m->smem_bytes)));
  m->finalized = true;
  m->cells_nodes = m->n_nodes;
  return CN_OK;
}

// Grow a device buffer to n elements, keeping old contents.
template <class T>
cn_status grow(cn_model* m, T** p, int64_t old_n, int64_t new_n) {
  T* q = static_cast<T*>(dalloc_raw(m, (size_t)new_n * sizeof(T)));
  if (!q) return m->fail(CN_ENOMEM, "device allocation failed");
  CN_TRY_CUDA(m, cudaMemsetAsync(q, 0, (size_t)new_n * sizeof(T), m->stream));
  if (*p && old_n > 0)
    CN_TRY_CUDA(m, cudaMemcpyAsync(q, *p, (size_t)old_n * sizeof(T), cudaMemcpyDeviceToDevice, m->stream));
  if (*p) {
    CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
    dfree_raw(m, *p);
  }
  *p = q;
  return CN_OK;
}

cn_status ensure_capacity(cn_model* m, int64_t K) {
  int64_t need_int = (K + m->D - 1) / m->D + 1;
  if (need_int > m->hist_cap) {
    int64_t nc = std::max(need_int, m->hist_cap * 2);
    CN_CHECK(grow(m, &m->dm.hist, m->hist_cap * m->n_cells, nc * m->n_cells));
    m->hist_cap = nc;
  }
  if (!m->rec_node.empty() && K + 1 > m->trace_cap) {
    int64_t nc = std::max(K + 1, m->trace_cap * 2);
    bool first = m->trace_cap == 0;
    CN_CHECK(grow(m, &m->dm.trace, m->trace_cap * m->dm.n_rec, nc * m->dm.n_rec));
    m->trace_cap = nc;
    if (first) {
      const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
      cn::DevModel dm = m->dm;
      int64_t k = m->step;
      CN_CHECK(launch_checked(m, [&] { cn::k_record0<<<nb, tb, 0, m->stream>>>(dm, k); }));
    }
  }
  return CN_OK;
}

cudaEvent_t take_event(cn_model* m) {
  if (!m->ev_pool.empty()) {
    cudaEvent_t e = m->ev_pool.back();
    m->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Queue one interval (steps [s0, s1) of interval J) on stream st: the event
// pull at the interval start, the interval kernel, and the device-side
// interval index bump once the interval is complete.  ev, when given, holds
// four events recorded around the pull and the interval kernel.
cn_status enqueue_interval(cn_model* m, cudaStream_t st, int64_t J, int s0, int s1, cudaEvent_t* ev,
                           bool capturing = false) {
  // inside a capture an event becomes a record node only when marked external
  const unsigned rec_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  cn::DevModel dm = m->dm;
  const int64_t* Jp = dm.jdev;
  const int wpb = m->wpb;
  const int blocks = (m->n_groups + wpb - 1) / wpb;
  const size_t smem = (size_t)wpb * m->smem_bytes;
  if (s0 == 0) {
    const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
    if (ev) CN_TRY_CUDA(m, cudaEventRecordWithFlags(ev[0], st, rec_flags));
    CN_CHECK(launch_checked(m, [&] { cn::k_pull_events<<<nb, tb, 0, st>>>(dm, J, Jp); }));
    if (ev) CN_TRY_CUDA(m, cudaEventRecordWithFlags(ev[1], st, rec_flags));
  }
  if (ev) CN_TRY_CUDA(m, cudaEventRecordWithFlags(ev[2], st, rec_flags));
  if (is_ref_mapping(m->opt.mapping)) {
    CN_CHECK(launch_checked(m, [&] { cn::k_interval_ref<<<m->n_groups, 32, 0, st>>>(dm, J, s0, s1, Jp); }));
  } else switch (m->opt.precision) {
    case CN_PREC_FP64:
      if (m->dense) CN_CHECK(launch_checked(m, [&] { cn::k_interval<0, false, true><<<blocks, 32 * wpb, smem, st>>>(dm, J, s0, s1, Jp); }));
      else CN_CHECK(launch_checked(m, [&] { cn::k_interval<0, false, false><<<blocks, 32 * wpb, smem, st>>>(dm, J, s0, s1, Jp); }));
      break;
    case CN_PREC_GATE_FP32:
      if (m->dense) CN_CHECK(launch_checked(m, [&] { cn::k_interval<1, false, true><<<blocks, 32 * wpb, smem, st>>>(dm, J, s0, s1, Jp); }));
      else CN_CHECK(launch_checked(m, [&] { cn::k_interval<1, false, false><<<blocks, 32 * wpb, smem, st>>>(dm, J, s0, s1, Jp); }));
      break;
    default:
      if (m->dense) CN_CHECK(launch_checked(m, [&] { cn::k_interval<2, false, true><<<blocks, 32 * wpb, smem, st>>>(dm, J, s0, s1, Jp); }));
      else CN_CHECK(launch_checked(m, [&] { cn::k_interval<2, false, false><<<blocks, 32 * wpb, smem, st>>>(dm, J, s0, s1, Jp); }));
      break;
  }
  if (ev) CN_TRY_CUDA(m, cudaEventRecordWithFlags(ev[3], st, rec_flags));
  if (s1 == m->D) CN_CHECK(launch_checked(m, [&] { cn::k_next_interval<<<1, 1, 0, st>>>(dm.jdev); }));
  return CN_OK;
}

// Direct launch of one interval on the model's stream (events from the pool
// when profiling).
cn_status launch_interval(cn_model* m, int64_t J, int s0, int s1) {
  if (!m->profiling) return enqueue_interval(m, m->stream, J, s0, s1, nullptr);
  cudaEvent_t ev[4];
  for (auto& e : ev) e = take_event(m);
  CN_CHECK(enqueue_interval(m, m->stream, J, s0, s1, ev));
  if (s0 == 0) m->ev_pull.emplace_back(ev[0], ev[1]);
  else {
    m->ev_pool.push_back(ev[0]);
    m->ev_pool.push_back(ev[1]);
  }
  m->ev_interval.emplace_back(ev[2], ev[3]);
  return CN_OK;
}

// ---- CUDA graph replay of whole intervals.  A chunk of kGraphIntervals
// complete intervals is captured once (the interval index lives on the
// device, so the same graph serves every chunk) and replayed on the model's
// stream.  Two chunk graphs alternate so that, when profiling, the events of
// one can be read while the other runs.
constexpr int kGraphIntervals = 8;

cn_status fold_chunk_events(cn_model* m, int c) {
  GraphChunk& g = m->gchunk[c];
  if (!g.pending) return CN_OK;
  CN_TRY_CUDA(m, cudaEventSynchronize(g.ev.back()));
  for (size_t i = 0; i + 3 < g.ev.size(); i += 4) {
    float a = 0.f, b = 0.f;
    CN_TRY_CUDA(m, cudaEventElapsedTime(&a, g.ev[i], g.ev[i + 1]));
    CN_TRY_CUDA(m, cudaEventElapsedTime(&b, g.ev[i + 2], g.ev[i + 3]));
    m->acc_pull_ms += a;
    m->acc_int_ms += b;
    m->acc_pull_n++;
    m->acc_int_n++;
  }
  g.pending = false;
  return CN_OK;
}

void drop_graphs(cn_model* m) {
  for (GraphChunk& g : m->gchunk) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
    g = GraphChunk{};
  }
}

cn_status capture_chunk(cn_model* m, int c) {
  GraphChunk& g = m->gchunk[c];
  if (!m->cap_stream) CN_TRY_CUDA(m, cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
  if (m->profiling && g.ev.empty()) {
    g.ev.resize(4 * kGraphIntervals);
    for (auto& e : g.ev) CN_TRY_CUDA(m, cudaEventCreate(&e));
  }
  cudaGraph_t graph = nullptr;
  CN_TRY_CUDA(m, cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
  cn_status st = CN_OK;
  const int64_t launches = m->launches;
  for (int i = 0; i < kGraphIntervals && st == CN_OK; ++i)
    st = enqueue_interval(m, m->cap_stream, 0, 0, m->D, m->profiling ? g.ev.data() + 4 * i : nullptr, true);
  m->launches = launches;  // captured, not launched
  cudaError_t e = cudaStreamEndCapture(m->cap_stream, &graph);
  if (st != CN_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  CN_TRY_CUDA(m, e);
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  CN_TRY_CUDA(m, e);
  g.key_hist = m->dm.hist;
  g.key_trace = m->dm.trace;
  g.key_prof = m->profiling;
  g.key_wpb = m->wpb;
  return CN_OK;
}

// Replays one chunk of kGraphIntervals complete intervals.
cn_status replay_chunk(cn_model* m) {
  const int c = m->gnext;
  m->gnext ^= 1;
  GraphChunk& g = m->gchunk[c];
  CN_CHECK(fold_chunk_events(m, c));
  if (g.exec && (g.key_hist != m->dm.hist || g.key_trace != m->dm.trace || g.key_prof != m->profiling ||
                 g.key_wpb != m->wpb)) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (!g.exec) CN_CHECK(capture_chunk(m, c));
  CN_TRY_CUDA(m, cudaGraphLaunch(g.exec, m->stream));
  // the graph's kernels: per interval the pull, the interval kernel and the bump
  m->launches += 3 * kGraphIntervals;
  g.pending = m->profiling;
  return CN_OK;
}


// Back to step 0: initial state, event cursors, spike history, interval
// index, status word and the step-0 trace sample.
cn_status reset_state(cn_model* m) {
  CN_CHECK(state_init(m));
  if (!m->x_pos0.empty())
    CN_TRY_CUDA(m, cudaMemcpyAsync(m->dm.x_pos, m->x_pos0.data(), m->x_pos0.size() * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, m->stream));
  if (m->dm.hist) CN_TRY_CUDA(m, cudaMemsetAsync(m->dm.hist, 0, (size_t)m->hist_cap * m->n_cells * 8, m->stream));
  CN_TRY_CUDA(m, cudaMemsetAsync(m->dm.status, 0, sizeof(int32_t), m->stream));
  CN_TRY_CUDA(m, cudaMemsetAsync(m->dm.jdev, 0, sizeof(int64_t), m->stream));
  m->step = 0;
  m->raster_from = 0;
  if (m->dm.trace) {
    const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
    cn::DevModel dm = m->dm;
    CN_CHECK(launch_checked(m, [&] { cn::k_record0<<<nb, tb, 0, m->stream>>>(dm, 0); }));
  }
  CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
  return CN_OK;
}

// Frees every device buffer of the model and forgets the layout, so that
// finalize can lay the model out again (used by the autotuner).
cn_status release_device(cn_model* m) {
  CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
  drop_graphs(m);
  for (auto* v : {&m->ev_interval, &m->ev_pull})
    for (auto& pr : *v) {
      m->ev_pool.push_back(pr.first);
      m->ev_pool.push_back(pr.second);
    }
  m->ev_interval.clear();
  m->ev_pull.clear();
  std::vector<void*> all = m->allocs;
  for (void* p : all) dfree_raw(m, p);
  m->ck_buf.clear();
  m->dm = cn::DevModel{};
  m->finalized = false;
  m->hist_cap = m->trace_cap = 0;
  m->step = 0;
  m->acc_int_ms = m->acc_pull_ms = 0.0;
  m->acc_int_n = m->acc_pull_n = 0;
  return CN_OK;
}

// Warps of the interval kernel (non-dense instantiation of the model's
// precision) resident on the whole device at once, in blocks of wpb warps of
// smem_warp bytes of shared memory each.
int resident_warps(cn_model* m, size_t smem_warp, int wpb) {
  const void* fn = m->opt.precision == CN_PREC_FP64        ? (const void*)cn::k_interval<0, false, false>
                   : m->opt.precision == CN_PREC_GATE_FP32 ? (const void*)cn::k_interval<1, false, false>
                                                           : (const void*)cn::k_interval<2, false, false>;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * wpb, (size_t)wpb * smem_warp) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->opt.device) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return per_sm * wpb * sms;
}

// Mapping autotuner: lays the model out for each candidate (one cell per
// lane; target spans of 1/8, 1/4, 1/2 and 1 mean cell size, each with warps
// as tall as the opening cell's span or as 1, 1.5 and 2 times the largest
// span; then spans of 0.85, 0.9, 0.95 and 1.1 times the best one), and for
// each runs one warm-up and one timed interval from the initial state with
// 1, 2 and 4 warps per block; keeps the fastest.  When the fastest has warps
// as tall as the largest span, a last round tries warp heights: for the best
// span and 3/4 of it, the lowest height (found by bisection on host-only
// layouts) at which every warp, in blocks of four, is resident on the device
// at once, and that height + 4.  The model is then laid out again with the
// winner.  Results do not depend on the choice beyond rounding.
cn_status autotune(cn_model* m) {
  const int64_t mean = std::max<int64_t>(1, (m->n_nodes + m->n_cells - 1) / std::max(1, m->n_cells));
  std::vector<int32_t> cand{CN_MAP_THREAD};
  if (m->ck_steps <= 0)
    for (int64_t t : {mean / 8, mean / 4, mean / 2, mean}) {
      const int32_t v = (int32_t)std::max<int64_t>(16, t);
      if (std::find(cand.begin(), cand.end(), v) == cand.end()) {
        cand.push_back(v);
        if (!m->dense) {
          cand.push_back(v | CN_MAP_TALL);
          cand.push_back(v | CN_MAP_TALL | CN_MAP_TALL2);
          cand.push_back(v | CN_MAP_TALL2);
        }
      }
    }
  float best = 0.f;
  int32_t best_map = CN_MAP_THREAD, best_wpb = 1, best_slots = 1;
  const bool prof = m->profiling;
  m->profiling = false;
  cudaEvent_t e0 = take_event(m), e1 = take_event(m);
  std::vector<int32_t> tried;
  auto measure = [&](int32_t c) -> cn_status {
    tried.push_back(c);
    m->opt.mapping = c;
    CN_CHECK(finalize(m));
    CN_CHECK(ensure_capacity(m, 2 * (int64_t)m->D));
    for (int w = 1; w <= cn::kMaxWarpsPerBlock; w *= 2) {
      if ((size_t)w * m->smem_bytes > (size_t)kMaxSmemPerBlock) break;
      m->wpb = w;
      CN_CHECK(reset_state(m));
      CN_CHECK(enqueue_interval(m, m->stream, 0, 0, m->D, nullptr));
      CN_TRY_CUDA(m, cudaEventRecord(e0, m->stream));
      CN_CHECK(enqueue_interval(m, m->stream, 1, 0, m->D, nullptr));
      CN_TRY_CUDA(m, cudaEventRecord(e1, m->stream));
      CN_TRY_CUDA(m, cudaEventSynchronize(e1));
      float ms = 0.f;
      CN_TRY_CUDA(m, cudaEventElapsedTime(&ms, e0, e1));
      if (best == 0.f || ms < best) {
        best = ms;
        best_map = c;
        best_wpb = w;
        best_slots = m->dm.max_slots;
      }
    }
    return release_device(m);
  };
  bool refined = false;
  for (size_t ci = 0; ci < cand.size(); ++ci) {
    CN_CHECK(measure(cand[ci]));
    // after the coarse candidates, refine the best span: a slightly finer
    // cut can fill the device's resident warps without a second wave
    if (ci + 1 == cand.size() && best_map >= 16 && !refined) {
      refined = true;
      const int32_t flags = best_map & (CN_MAP_TALL | CN_MAP_TALL2), span = best_map & ~flags;
      for (double f : {0.85, 0.9, 0.95, 1.1}) {
        const int32_t v = (int32_t)std::max<int64_t>(16, (int64_t)(span * f + 0.5)) | flags;
        if (std::find(tried.begin(), tried.end(), v) == tried.end() &&
            std::find(cand.begin(), cand.end(), v) == cand.end())
          cand.push_back(v);
      }
    }
  }
  // warp heights for tall warps: the lowest height whose warps, in blocks of
  // four, are all resident at once (the warp count falls as the height grows)
  if (!m->dense && m->ck_steps <= 0 && best_map >= 16 &&
      (best_map & (CN_MAP_TALL | CN_MAP_TALL2)) == CN_MAP_TALL) {
    const int32_t span = best_map & ~CN_MAP_TALL;
    const int gate_bytes = m->opt.precision == CN_PREC_FP64 ? 8 : 4;
    auto fits = [&](int32_t target, int h) -> int {  // 1 fits, 0 not, -1 layout failed
      Layout L;
      std::string lerr;
      if (!build_layout(m->n_cells, m->off.data(), m->parent.data(), nullptr, m->spike_node.data(), target, true, 2,
                        h, L, lerr))
        return -1;
      const size_t smem = cn::interval_smem_bytes(L.depth, best_slots, false, L.n_mail, gate_bytes);
      return L.n_groups <= resident_warps(m, smem, cn::kMaxWarpsPerBlock) ? 1 : 0;
    };
    std::vector<int32_t> hc;
    for (int32_t target : {span, std::max<int32_t>(16, (3 * span + 2) / 4)}) {
      std::vector<CellPlan> plans;
      plan_cells(m->n_cells, m->off.data(), m->parent.data(), target, 0, plans);
      int top = 0;  // the largest span: heights below it are the candidates
      for (const CellPlan& P : plans) top = std::max(top, P.span);
      if (top > 511) continue;
      // lo does not fit, hi is taken to (a height that does not fit leaves
      // no candidate below the largest span)
      int lo = std::max(16, (3 * top) / 4), hi = top;
      const int r0 = fits(target, lo);
      if (r0 < 0) continue;
      if (r0 == 1) hi = lo;
      bool ok = true;
      while (hi - lo > 2) {
        const int mid = (lo + hi) / 2;
        const int r = fits(target, mid);
        if (r < 0) {
          ok = false;
          break;
        }
        (r == 1 ? hi : lo) = mid;
      }
      if (!ok) continue;
      for (int h : {hi, hi + 4})
        if (h < top) hc.push_back(target | CN_MAP_TALL | CN_MAP_HEIGHT(h));
    }
    for (int32_t c : hc)
      if (std::find(tried.begin(), tried.end(), c) == tried.end()) CN_CHECK(measure(c));
  }
  m->ev_pool.push_back(e0);
  m->ev_pool.push_back(e1);
  m->profiling = prof;
  m->opt.mapping = best_map;
  m->wpb = best_wpb;
  m->tuned_ms = best;
  m->launches = 0;
  return finalize(m);
}

// Lays the model out on first use (through the autotuner when asked).
cn_status prepare(cn_model* m) {
  if (m->finalized) return CN_OK;
  if (m->opt.mapping == CN_MAP_TUNE) return autotune(m);
  return finalize(m);
}

// State snapshot (v, HH gates, synaptic g) into / out of a device buffer.
size_t snapshot_bytes(const cn_model* m) {
  return (size_t)m->node_elems * 8 + 3 * (size_t)std::max<int64_t>(m->hh_elems, 1) * m->gate_bytes +
         (size_t)std::max<int64_t>(m->syn_elems, 1) * 8;
}

cn_status snapshot(cn_model* m, void* buf, bool save) {
  char* p = static_cast<char*>(buf);
  const size_t nv = (size_t)m->node_elems * 8, ng = (size_t)std::max<int64_t>(m->hh_elems, 1) * m->gate_bytes,
               ns = (size_t)std::max<int64_t>(m->syn_elems, 1) * 8;
  void* dev[5] = {m->dm.v, m->dm.hh_m, m->dm.hh_h, m->dm.hh_n, m->dm.syn_g};
  size_t sz[5] = {nv, ng, ng, ng, ns};
  for (int i = 0; i < 5; ++i) {
    if (save) CN_TRY_CUDA(m, cudaMemcpyAsync(p, dev[i], sz[i], cudaMemcpyDeviceToDevice, m->stream));
    else CN_TRY_CUDA(m, cudaMemcpyAsync(dev[i], p, sz[i], cudaMemcpyDeviceToDevice, m->stream));
    p += sz[i];
  }
  return CN_OK;
}

// Advance from the current step to K (< next interval boundary handling as
// in cn_run), with the trajectory-recording kernel when traj is set.
cn_status advance(cn_model* m, int64_t K, bool traj) {
  while (m->step < K) {
    const int64_t J = m->step / m->D;
    const int s0 = (int)(m->step - J * m->D);
    const int s1 = (int)std::min<int64_t>(m->D, K - J * m->D);
    if (traj) {
      cn::DevModel dm = m->dm;
      CN_CHECK(launch_checked(m, [&] {
        cn::k_interval<0, true, false><<<m->n_groups, 32, m->smem_bytes, m->stream>>>(dm, J, s0, s1, nullptr);
      }));
    } else if (m->opt.use_graph && s0 == 0 && K - m->step >= (int64_t)kGraphIntervals * m->D) {
      CN_CHECK(replay_chunk(m));
      m->step += (int64_t)kGraphIntervals * m->D;
      continue;
    } else {
      CN_CHECK(launch_interval(m, J, s0, s1));
    }
    m->step = J * m->D + s1;
  }
  return CN_OK;
}

}  // namespace

// ====================================================================== ABI
namespace {
constexpr uint64_t kCkMagic = 0x314b434e43ull;  // "CNCK1"

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}
template <class T>
uint64_t fnv_vec(uint64_t h, const std::vector<T>& v) {
  return fnv(h, v.data(), v.size() * sizeof(T));
}

// Identity of the network a checkpoint belongs to: morphology, mechanism
// placement, NetCons and the step.
uint64_t network_fingerprint(const cn_model* m) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, &m->n_cells, sizeof(m->n_cells));
  h = fnv_vec(h, m->off);
  h = fnv_vec(h, m->parent);
  h = fnv_vec(h, m->pas_node);
  h = fnv_vec(h, m->hh_node);
  h = fnv_vec(h, m->syn_node);
  for (int t = 0; t < cn::kChanTypes; ++t) h = fnv_vec(h, m->ch_node[t]);
  h = fnv_vec(h, m->nc_src);
  h = fnv_vec(h, m->nc_syn);
  h = fnv_vec(h, m->nc_delay);
  h = fnv_vec(h, m->nc_w);
  h = fnv_vec(h, m->gap_node);
  h = fnv_vec(h, m->gap_peer);
  h = fnv_vec(h, m->gap_g);
  h = fnv(h, &m->opt.dt_ms, sizeof(double));
  return h;
}

struct CkHeader {
  uint64_t magic, fingerprint;
  int64_t step, window0, n_nodes, n_hh, n_syn, n_ch[cn::kChanTypes];
  int32_t n_cells, D, has_cai, pad;
};

double gate_load(const void* base, int64_t e, int bytes) {
  if (bytes == 8) return static_cast<const double*>(base)[e];
  if (bytes == 4) return static_cast<const float*>(base)[e];
  uint32_t fb = (uint32_t) static_cast<const uint16_t*>(base)[e] << 16;
  float f;
  std::memcpy(&f, &fb, 4);
  return f;
}

// Stores x in the gate format (bfloat16 by round-to-nearest-even of its
// single-precision value).
void gate_store(void* base, int64_t e, int bytes, double x) {
  if (bytes == 8) {
    static_cast<double*>(base)[e] = x;
    return;
  }
  const float f = (float)x;
  if (bytes == 4) {
    static_cast<float*>(base)[e] = f;
    return;
  }
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);
  static_cast<uint16_t*>(base)[e] = (uint16_t)(u >> 16);
}

// Everything a checkpoint moves, as (device buffer, bytes per element,
// element map from input order) triples, plus the flat host image.
struct CkPlan {
  std::vector<void*> dev;
  std::vector<int64_t> dev_elems;
  std::vector<int> bytes;
  std::vector<const std::vector<int64_t>*> map;
  std::vector<std::vector<int64_t>> owned_maps;
};

void ck_plan(cn_model* m, CkPlan& P) {
  P.owned_maps.reserve(2 * cn::kChanTypes + 2);
  auto add = [&](void* d, int64_t elems, int bytes, const std::vector<int64_t>* mp) {
    P.dev.push_back(d);
    P.dev_elems.push_back(elems);
    P.bytes.push_back(bytes);
    P.map.push_back(mp);
  };
  add(m->dm.v, m->node_elems, 8, &m->node_elem);
  for (void* g : {m->dm.hh_m, m->dm.hh_h, m->dm.hh_n}) add(g, m->hh_elems, m->gate_bytes, &m->hh_elem);
  add(m->dm.syn_g, m->syn_elems, 8, &m->syn_elem);
  for (int t = 0; t < cn::kChanTypes; ++t) {
    if (m->ch_node[t].empty()) continue;
    std::vector<int64_t> mp(m->ch_node[t].size());
    for (size_t i = 0; i < mp.size(); ++i) mp[i] = m->node_elem[m->ch_node[t][i]];
    P.owned_maps.push_back(std::move(mp));
    const int g0 = cn::chan_gate0(t), g1 = t + 1 < cn::kChanTypes ? cn::chan_gate0(t + 1) : cn::kChanGates;
    for (int gi = g0; gi < g1; ++gi) add(m->dm.ch_gate[gi], m->node_elems, m->gate_bytes, &P.owned_maps.back());
  }
  if (m->dm.cai) add(m->dm.cai, m->node_elems, 8, &m->node_elem);
}

size_t ck_bytes(const cn_model* m, const CkPlan& P, int64_t nwin) {
  size_t b = sizeof(CkHeader);
  for (size_t k = 0; k < P.dev.size(); ++k) b += P.map[k]->size() * 8;
  b += (size_t)m->n_cells;                          // threshold flags
  b += (size_t)nwin * m->n_cells * sizeof(uint64_t);  // spike history window
  return b;
}
}  // namespace

extern "C" {

int32_t cn_mech_nparams(int32_t type) {
  return (type >= 0 && type < CN_MECH_NTYPES) ? kNParams[type] : -1;
}

void cn_options_default(cn_options* opt) {
  std::memset(opt, 0, sizeof(*opt));
  opt->dt_ms = 0.025;
  opt->v_init_mV = -65.0;
  opt->precision = CN_PREC_FP64;
  opt->device = 0;
  opt->mapping = CN_MAP_AUTO;
  opt->use_graph = 1;
}

cn_status cn_geometry(int32_t n_cells, const int32_t* cell_offset, const int32_t* parent,
                      const double* dx_um, const double* diam_um, const double* Ra_ohm_cm,
                      double* area_um2, double* ri_MOhm) {
  if (n_cells < 0 || !cell_offset || (n_cells > 0 && (!parent || !dx_um || !diam_um || !Ra_ohm_cm ||
                                                      !area_um2 || !ri_MOhm)))
    return CN_EINVAL;
  const double pi = 3.14159265358979323846;
  int64_t n = cell_offset[n_cells];
  std::vector<double> rhalf(n);
  for (int64_t i = 0; i < n; ++i) {
    if (!(dx_um[i] > 0) || !(diam_um[i] > 0) || !(Ra_ohm_cm[i] > 0)) return CN_EINVAL;
    area_um2[i] = pi * diam_um[i] * dx_um[i];
    rhalf[i] = 1e-2 * 2.0 * Ra_ohm_cm[i] * dx_um[i] / (pi * diam_um[i] * diam_um[i]);
  }
  for (int c = 0; c < n_cells; ++c) {
    for (int64_t i = cell_offset[c]; i < cell_offset[c + 1]; ++i) {
      int64_t li = i - cell_offset[c];
      int32_t p = parent[i];
      if ((li == 0) != (p == -1) || p >= li || p < -1) return CN_EINVAL;
      ri_MOhm[i] = p < 0 ? 0.0 : rhalf[i] + rhalf[cell_offset[c] + p];
    }
  }
  return CN_OK;
}

cn_status cn_get_mapping(cn_model* m, int32_t* mapping, int32_t* warps_per_block, int32_t* n_warps,
                         float* tuned_interval_ms) {
  if (!m) return CN_EINVAL;
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  CN_CHECK(prepare(m));
  if (mapping) *mapping = m->opt.mapping;
  if (warps_per_block) *warps_per_block = m->wpb;
  if (n_warps) *n_warps = m->n_groups;
  if (tuned_interval_ms) *tuned_interval_ms = m->tuned_ms;
  return CN_OK;
}

cn_status cn_plan_layout(int32_t n_cells, const int32_t* cell_offset, const int32_t* parent, int32_t mapping,
                         int32_t* node_lane, int32_t* node_row, int32_t* node_flags, int32_t* n_warps,
                         int32_t* stack_depth) {
  g_create_error.clear();
  if (n_cells < 0 || !cell_offset || (n_cells > 0 && !parent)) {
    g_create_error = "null argument";
    return CN_EINVAL;
  }
  if (!valid_trees(n_cells, cell_offset, parent, g_create_error)) return CN_EINVAL;
  if (!valid_mapping(mapping)) {
    g_create_error = "bad mapping";
    return CN_EINVAL;
  }
  const int64_t nn = cell_offset[n_cells];
  Layout L;
  const bool ok = is_ref_mapping(mapping)
                      ? build_ref_layout(n_cells, cell_offset, parent, nullptr, mapping == CN_MAP_CONSTDEPTH, L,
                                         g_create_error)
                      : build_layout(n_cells, cell_offset, parent, nullptr, nullptr,
                                     map_target(mapping, nn, n_cells, false), true, tall_factor(mapping),
                                     map_height(mapping), L, g_create_error);
  if (!ok) return CN_EINVAL;
  if (node_lane) std::copy(L.node_slot.begin(), L.node_slot.end(), node_lane);
  if (node_row) std::copy(L.node_row.begin(), L.node_row.end(), node_row);
  if (node_flags) std::copy(L.node_flags.begin(), L.node_flags.end(), node_flags);
  if (n_warps) *n_warps = L.n_groups;
  if (stack_depth) *stack_depth = L.depth;
  return CN_OK;
}

cn_status cn_model_create(const cn_morph* morph, const cn_mech_table* mechs, int32_t n_mechs,
                          const cn_options* opt, cn_model** out) {
  g_create_error.clear();
  auto bad = [](const std::string& s) {
    g_create_error = s;
    return CN_EINVAL;
  };
  if (!morph || !out || n_mechs < 0 || (n_mechs > 0 && !mechs)) return bad("null argument");
  *out = nullptr;
  cn_options o;
  if (opt) o = *opt;
  else cn_options_default(&o);
  if (!(o.dt_ms > 0) || !std::isfinite(o.v_init_mV)) return bad("bad dt or v_init");
  if (o.precision < 0 || o.precision > 2) return bad("bad precision");
  if ((o.alloc == nullptr) != (o.free == nullptr)) return bad("alloc and free must be given together");
  if (o.warps_per_block < 0 || o.warps_per_block > cn::kMaxWarpsPerBlock) return bad("warps_per_block must be 0..4");
  {
    if (!valid_mapping(o.mapping))
      return bad("mapping must be 0-4, or a span >= 16 (optionally with CN_MAP_TALL and/or CN_MAP_TALL2, "
                 "or with CN_MAP_TALL and a warp height of 16-511 rows)");
  }
  const int32_t nc = morph->n_cells;
  if (nc <= 0 || !morph->cell_offset || !morph->parent || !morph->area_um2 || !morph->cm_uF_cm2 ||
      !morph->ri_MOhm || !morph->spike_node || !morph->threshold_mV)
    return bad("incomplete morphology");
  if (morph->cell_offset[0] != 0) return bad("cell_offset[0] must be 0");
  for (int c = 0; c < nc; ++c)
    if (morph->cell_offset[c + 1] <= morph->cell_offset[c]) return bad("empty cell or decreasing cell_offset");
  const int64_t nn = morph->cell_offset[nc];
  for (int c = 0; c < nc; ++c) {
    const int32_t a0 = morph->cell_offset[c], a1 = morph->cell_offset[c + 1];
    if (a1 - a0 > (1 << 24)) return bad("cell too large");
    for (int32_t i = a0; i < a1; ++i) {
      const int32_t li = i - a0, p = morph->parent[i];
      if (li == 0 ? p != -1 : (p < 0 || p >= li)) return bad("parent must satisfy parent[0] = -1, 0 <= parent[i] < i");
      if (!(morph->area_um2[i] > 0) || !(morph->cm_uF_cm2[i] > 0) || (li > 0 && !(morph->ri_MOhm[i] > 0)))
        return bad("non-positive area, cm or ri");
    }
    if (morph->spike_node[c] < 0 || morph->spike_node[c] >= a1 - a0) return bad("spike_node out of range");
    if (!std::isfinite(morph->threshold_mV[c])) return bad("bad threshold");
  }
  cn_model* m = new (std::nothrow) cn_model();
  if (!m) {
    g_create_error = "host allocation failed";
    return CN_ENOMEM;
  }
  m->opt = o;
  m->wpb = std::max(1, o.warps_per_block);
  m->stream = static_cast<cudaStream_t>(o.stream);
  m->n_cells = nc;
  m->n_nodes = nn;
  m->off.assign(morph->cell_offset, morph->cell_offset + nc + 1);
  m->parent.assign(morph->parent, morph->parent + nn);
  m->area.assign(morph->area_um2, morph->area_um2 + nn);
  m->cm.assign(morph->cm_uF_cm2, morph->cm_uF_cm2 + nn);
  m->ri.assign(morph->ri_MOhm, morph->ri_MOhm + nn);
  m->spike_node.assign(morph->spike_node, morph->spike_node + nc);
  m->thresh.assign(morph->threshold_mV, morph->threshold_mV + nc);
  m->node_cell.resize(nn);
  for (int c = 0; c < nc; ++c)
    for (int32_t i = m->off[c]; i < m->off[c + 1]; ++i) m->node_cell[i] = c;
  bool seen[CN_MECH_NTYPES] = {};
  std::vector<uint8_t> has_pas(nn, 0);
  for (int t = 0; t < n_mechs; ++t) {
    const cn_mech_table& mt = mechs[t];
    if (mt.type < 0 || mt.type >= CN_MECH_NTYPES) { delete m; return bad("unknown mechanism type"); }
    if (seen[mt.type]) { delete m; return bad("duplicate mechanism table"); }
    seen[mt.type] = true;
    if (mt.n < 0 || (mt.n > 0 && (!mt.node || !mt.param))) { delete m; return bad("bad mechanism table"); }
    for (int i = 0; i < mt.n; ++i)
      if (mt.node[i] < 0 || mt.node[i] >= nn) { delete m; return bad("mechanism node out of range"); }
    const int np = kNParams[mt.type];
    auto col = [&](int p, int i) { return mt.param[(int64_t)p * mt.n + i]; };
    switch (mt.type) {
      case CN_MECH_PAS:
        for (int i = 0; i < mt.n; ++i) {
          if (has_pas[mt.node[i]]) { delete m; return bad("at most one pas instance per node"); }
          has_pas[mt.node[i]] = 1;
          m->pas_node.push_back(mt.node[i]);
          m->pas_g.push_back(col(0, i));
          m->pas_e.push_back(col(1, i));
        }
        break;
      case CN_MECH_HH:
        m->hh_node.assign(mt.node, mt.node + mt.n);
        m->hh_par.assign(mt.param, mt.param + (int64_t)np * mt.n);
        break;
      case CN_MECH_EXPSYN:
        for (int i = 0; i < mt.n; ++i)
          if (!(col(0, i) > 0)) { delete m; return bad("ExpSyn tau must be positive"); }
        m->syn_node.assign(mt.node, mt.node + mt.n);
        m->syn_tau.assign(mt.param, mt.param + mt.n);
        m->syn_e.assign(mt.param + mt.n, mt.param + 2 * (int64_t)mt.n);
        break;
      default: {
        const int t = mt.type - CN_MECH_NA3H;
        m->ch_node[t].assign(mt.node, mt.node + mt.n);
        m->ch_par[t].assign(mt.param, mt.param + (int64_t)np * mt.n);
        if (mt.n > 0) m->dense = true;
        break;
      }
    }
  }
  cudaError_t e = cudaSetDevice(o.device);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    delete m;
    return CN_ECUDA;
  }
  *out = m;
  return CN_OK;
}

static cn_status state_check(cn_model* m) {
  if (!m) return CN_EINVAL;
  if (m->finalized) return m->fail(CN_ESTATE, "model already running: add inputs before the first cn_run");
  return CN_OK;
}

cn_status cn_add_netcons(cn_model* m, int64_t n, const int32_t* src, const int32_t* syn, const double* w,
                         const double* delay) {
  CN_CHECK(state_check(m));
  if (n < 0 || (n > 0 && (!src || !syn || !w || !delay))) return m->fail(CN_EINVAL, "bad netcon arrays");
  for (int64_t j = 0; j < n; ++j) {
    if (src[j] < 0 || src[j] >= m->n_cells) return m->fail(CN_EINVAL, "NetCon source out of range");
    if (syn[j] < 0 || syn[j] >= (int64_t)m->syn_node.size()) return m->fail(CN_EINVAL, "NetCon target out of range");
    if (!std::isfinite(w[j]) || !(delay[j] > 0)) return m->fail(CN_EINVAL, "bad NetCon weight or delay");
  }
  m->nc_src.insert(m->nc_src.end(), src, src + n);
  m->nc_syn.insert(m->nc_syn.end(), syn, syn + n);
  m->nc_w.insert(m->nc_w.end(), w, w + n);
  m->nc_delay.insert(m->nc_delay.end(), delay, delay + n);
  return CN_OK;
}

cn_status cn_add_netcon(cn_model* m, int32_t src, int32_t syn, double w, double delay) {
  return cn_add_netcons(m, 1, &src, &syn, &w, &delay);
}

cn_status cn_add_events(cn_model* m, int64_t n, const int32_t* syn, const double* t, const double* w) {
  CN_CHECK(state_check(m));
  if (n < 0 || (n > 0 && (!syn || !t || !w))) return m->fail(CN_EINVAL, "bad event arrays");
  for (int64_t e = 0; e < n; ++e) {
    if (syn[e] < 0 || syn[e] >= (int64_t)m->syn_node.size()) return m->fail(CN_EINVAL, "event target out of range");
    if (!std::isfinite(t[e]) || !std::isfinite(w[e])) return m->fail(CN_EINVAL, "bad event time or weight");
  }
  m->ev_syn.insert(m->ev_syn.end(), syn, syn + n);
  m->ev_t.insert(m->ev_t.end(), t, t + n);
  m->ev_w.insert(m->ev_w.end(), w, w + n);
  return CN_OK;
}

cn_status cn_add_stim(cn_model* m, int32_t node, double del, double dur, double amp) {
  CN_CHECK(state_check(m));
  if (node < 0 || node >= m->n_nodes) return m->fail(CN_EINVAL, "stimulus node out of range");
  if (!std::isfinite(del) || !std::isfinite(dur) || !std::isfinite(amp)) return m->fail(CN_EINVAL, "bad stimulus");
  m->st_node.push_back(node);
  m->st_del.push_back(del);
  m->st_dur.push_back(dur);
  m->st_amp.push_back(amp);
  return CN_OK;
}

cn_status cn_add_gaps(cn_model* m, int64_t n, const int32_t* node, const int32_t* peer, const double* g_uS) {
  CN_CHECK(state_check(m));
  if (n < 0 || (n > 0 && (!node || !peer || !g_uS))) return m->fail(CN_EINVAL, "bad gap junction arrays");
  for (int64_t i = 0; i < n; ++i) {
    if (node[i] < 0 || node[i] >= m->n_nodes || peer[i] < 0 || peer[i] >= m->n_nodes)
      return m->fail(CN_EINVAL, "gap junction node out of range");
    if (!std::isfinite(g_uS[i]) || g_uS[i] < 0) return m->fail(CN_EINVAL, "bad gap junction conductance");
  }
  m->gap_node.insert(m->gap_node.end(), node, node + n);
  m->gap_peer.insert(m->gap_peer.end(), peer, peer + n);
  m->gap_g.insert(m->gap_g.end(), g_uS, g_uS + n);
  return CN_OK;
}

cn_status cn_record(cn_model* m, int32_t node, int32_t* rec_id) {
  CN_CHECK(state_check(m));
  if (node < 0 || node >= m->n_nodes || !rec_id) return m->fail(CN_EINVAL, "record node out of range");
  *rec_id = (int32_t)m->rec_node.size();
  m->rec_node.push_back(node);
  return CN_OK;
}

cn_status cn_run(cn_model* m, double tstop_ms) {
  if (!m) return CN_EINVAL;
  if (!std::isfinite(tstop_ms)) return m->fail(CN_EINVAL, "bad tstop");
  const int64_t K = round_half_away(tstop_ms / m->opt.dt_ms);
  if (K < m->step) return m->fail(CN_EINVAL, "tstop is behind the current time");
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  CN_CHECK(prepare(m));
  CN_CHECK(ensure_capacity(m, K));
  if (m->ck_steps <= 0) return advance(m, K, false);
  // with adjoint checkpoints: snapshot the state at every multiple of S
  while (m->step < K) {
    const int64_t S = m->ck_steps;
    if (m->step % S == 0) {
      const size_t idx = (size_t)(m->step / S);
      while (m->ck_buf.size() <= idx) {
        void* b = dalloc_raw(m, m->ck_bytes);
        if (!b) return m->fail(CN_ENOMEM, "checkpoint allocation failed");
        m->ck_buf.push_back(b);
      }
      CN_CHECK(snapshot(m, m->ck_buf[idx], true));
    }
    CN_CHECK(advance(m, std::min<int64_t>(K, (m->step / S + 1) * S), false));
  }
  return CN_OK;
}

cn_status cn_sync(cn_model* m) {
  if (!m) return CN_EINVAL;
  if (!m->finalized) return CN_OK;
  CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
  int32_t st = 0;
  CN_TRY_CUDA(m, cudaMemcpy(&st, m->dm.status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st & cn::kStatusEvOverflow)
    return m->fail(CN_ERANGE, "more than 256 events arrived at one cell within one interval");
  return CN_OK;
}

int64_t cn_current_step(const cn_model* m) { return m ? m->step : -1; }
int64_t cn_updates(const cn_model* m) { return m ? m->n_nodes * m->step : 0; }
int64_t cn_launch_count(const cn_model* m) { return m ? m->launches : 0; }

cn_status cn_get_spikes(cn_model* m, int32_t* gid, int64_t* step, size_t cap, size_t* n) {
  if (!m || !n) return CN_EINVAL;
  *n = 0;
  if (!m->finalized) return CN_OK;
  CN_CHECK(cn_sync(m));
  const int64_t nint = (m->step + m->D - 1) / m->D;
  std::vector<uint64_t> h((size_t)nint * m->n_cells);
  if (!h.empty())
    CN_TRY_CUDA(m, cudaMemcpy(h.data(), m->dm.hist, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  std::vector<std::pair<int64_t, int32_t>> sp;
  for (int64_t J = 0; J < nint; ++J)
    for (int32_t c = 0; c < m->n_cells; ++c) {
      uint64_t mk = h[(size_t)J * m->n_cells + c];
      while (mk) {
        int b = __builtin_ctzll(mk);
        mk &= mk - 1;
        if (J * m->D + b + 1 > m->raster_from) sp.emplace_back(J * m->D + b + 1, c);
      }
    }
  std::sort(sp.begin(), sp.end());
  *n = sp.size();
  if (!gid || !step) return CN_OK;
  if (cap < sp.size()) return m->fail(CN_ERANGE, "spike buffer too small");
  for (size_t i = 0; i < sp.size(); ++i) {
    gid[i] = sp[i].second;
    step[i] = sp[i].first;
  }
  return CN_OK;
}

cn_status cn_get_trace(cn_model* m, int32_t rec_id, double* out, size_t cap, size_t* n) {
  if (!m || !n) return CN_EINVAL;
  if (rec_id < 0 || rec_id >= (int32_t)m->rec_node.size()) return m->fail(CN_EINVAL, "bad record id");
  *n = (size_t)m->step + 1;
  if (!out) return CN_OK;
  if (cap < *n) return m->fail(CN_ERANGE, "trace buffer too small");
  if (!m->finalized) {
    out[0] = m->opt.v_init_mV;
    return CN_OK;
  }
  CN_CHECK(cn_sync(m));
  const int nr = m->dm.n_rec;
  CN_TRY_CUDA(m, cudaMemcpy2D(out, sizeof(double), m->dm.trace + rec_id, nr * sizeof(double), sizeof(double),
                              *n, cudaMemcpyDeviceToHost));
  return CN_OK;
}

cn_status cn_get_traces(cn_model* m, double* out, size_t cap, size_t* n) {
  if (!m || !n) return CN_EINVAL;
  const size_t nr = m->rec_node.size();
  *n = ((size_t)m->step + 1) * nr;
  if (!out) return CN_OK;
  if (cap < *n) return m->fail(CN_ERANGE, "trace buffer too small");
  if (!m->finalized) {
    for (size_t i = 0; i < nr; ++i) out[i] = m->opt.v_init_mV;
    return CN_OK;
  }
  CN_CHECK(cn_sync(m));
  if (*n) CN_TRY_CUDA(m, cudaMemcpy(out, m->dm.trace, *n * sizeof(double), cudaMemcpyDeviceToHost));
  return CN_OK;
}

cn_status cn_get_v(cn_model* m, double* out, size_t cap) {
  if (!m || !out) return CN_EINVAL;
  if (cap < (size_t)m->n_nodes) return m->fail(CN_ERANGE, "buffer too small");
  if (!m->finalized) {
    for (int64_t i = 0; i < m->n_nodes; ++i) out[i] = m->opt.v_init_mV;
    return CN_OK;
  }
  CN_CHECK(cn_sync(m));
  std::vector<double> h(m->node_elems);
  CN_TRY_CUDA(m, cudaMemcpy(h.data(), m->dm.v, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < m->n_nodes; ++i) {
    const int s = m->node_slot[i];
    out[i] = h[m->g_node_base[s / cn::kLanes] + (int64_t)m->node_row[i] * cn::kLanes + s % cn::kLanes];
  }
  return CN_OK;
}

static double gate_to_double(const void* base, int64_t e, int bytes) {
  if (bytes == 8) return static_cast<const double*>(base)[e];
  if (bytes == 4) return static_cast<const float*>(base)[e];
  uint16_t hb = static_cast<const uint16_t*>(base)[e];
  uint32_t fb = (uint32_t)hb << 16;
  float f;
  std::memcpy(&f, &fb, 4);
  return f;
}

cn_status cn_get_state(cn_model* m, int32_t type, int32_t col, double* out, size_t cap) {
  if (!m || !out) return CN_EINVAL;
  if (!m->finalized) return m->fail(CN_ESTATE, "state is built at the first cn_run");
  CN_CHECK(cn_sync(m));
  if (type == CN_MECH_HH && col >= 0 && col < 3) {
    size_t n = m->hh_node.size();
    if (cap < n) return m->fail(CN_ERANGE, "buffer too small");
    const void* src = col == 0 ? m->dm.hh_m : (col == 1 ? m->dm.hh_h : m->dm.hh_n);
    std::vector<uint8_t> h((size_t)std::max<int64_t>(m->hh_elems, 1) * m->gate_bytes);
    CN_TRY_CUDA(m, cudaMemcpy(h.data(), src, h.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) {
      int s = m->hh_slot[i];
      int64_t e = m->g_hh_base[s / cn::kLanes] + (int64_t)m->hh_q[i] * cn::kLanes + s % cn::kLanes;
      out[i] = gate_to_double(h.data(), e, m->gate_bytes);
    }
    return CN_OK;
  }
  if (type == CN_MECH_EXPSYN && col == 0) {
    size_t n = m->syn_node.size();
    if (cap < n) return m->fail(CN_ERANGE, "buffer too small");
    std::vector<double> h(std::max<int64_t>(m->syn_elems, 1));
    CN_TRY_CUDA(m, cudaMemcpy(h.data(), m->dm.syn_g, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) out[i] = h[m->syn_elem[i]];
    return CN_OK;
  }
  if (type >= CN_MECH_NA3H && type <= CN_MECH_KCA) {
    const int t = type - CN_MECH_NA3H;
    const int ngates = (t + 1 < cn::kChanTypes ? cn::chan_gate0(t + 1) : cn::kChanGates) - cn::chan_gate0(t);
    const size_t n = m->ch_node[t].size();
    if (cap < n) return m->fail(CN_ERANGE, "buffer too small");
    const bool want_cai = type == CN_MECH_CAHVA && col == ngates;
    if (col < 0 || (col >= ngates && !want_cai)) return m->fail(CN_EINVAL, "no such state column");
    const void* src = want_cai ? (const void*)m->dm.cai : m->dm.ch_gate[cn::chan_gate0(t) + col];
    const int bytes = want_cai ? 8 : m->gate_bytes;
    std::vector<uint8_t> h((size_t)m->node_elems * bytes);
    CN_TRY_CUDA(m, cudaMemcpy(h.data(), src, h.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) {
      const int32_t node = m->ch_node[t][i];
      const int sl = m->node_slot[node];
      const int64_t e = m->g_node_base[sl / cn::kLanes] + (int64_t)m->node_row[node] * cn::kLanes + sl % cn::kLanes;
      out[i] = gate_to_double(h.data(), e, bytes);
    }
    return CN_OK;
  }
  return m->fail(CN_EINVAL, "no such state column");
}

cn_status cn_profile(cn_model* m, int32_t enable) {
  if (!m) return CN_EINVAL;
  m->profiling = enable != 0;
  return CN_OK;
}

cn_status cn_profile_read(cn_model* m, double* interval_ms, int64_t* interval_launches, double* pull_ms,
                          int64_t* pull_launches) {
  if (!m) return CN_EINVAL;
  CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
  auto sum = [&](std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& v, double& ms, int64_t& cnt) -> cn_status {
    for (auto& pr : v) {
      float x = 0.f;
      CN_TRY_CUDA(m, cudaEventElapsedTime(&x, pr.first, pr.second));
      ms += x;
      ++cnt;
      m->ev_pool.push_back(pr.first);
      m->ev_pool.push_back(pr.second);
    }
    v.clear();
    return CN_OK;
  };
  CN_CHECK(sum(m->ev_interval, m->acc_int_ms, m->acc_int_n));
  CN_CHECK(sum(m->ev_pull, m->acc_pull_ms, m->acc_pull_n));
  CN_CHECK(fold_chunk_events(m, 0));
  CN_CHECK(fold_chunk_events(m, 1));
  if (interval_ms) *interval_ms = m->acc_int_ms;
  if (interval_launches) *interval_launches = m->acc_int_n;
  if (pull_ms) *pull_ms = m->acc_pull_ms;
  if (pull_launches) *pull_launches = m->acc_pull_n;
  m->acc_int_ms = m->acc_pull_ms = 0.0;
  m->acc_int_n = m->acc_pull_n = 0;
  return CN_OK;
}

cn_status cn_reset(cn_model* m) {
  if (!m) return CN_EINVAL;
  if (!m->finalized) return CN_OK;
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  return reset_state(m);
}

// Element indices and cells of the instances a per-cell parameter covers:
// HH instances (gnabar, gkbar) or rows carrying pas (g).
static void param_targets(const cn_model* m, int32_t param, std::vector<int64_t>& idx, std::vector<int32_t>& cell) {
  idx.clear();
  cell.clear();
  if (param < 2) {
    for (size_t i = 0; i < m->hh_node.size(); ++i) {
      idx.push_back((int64_t)param * m->hh_elems + m->hh_elem[i]);
      cell.push_back(m->node_cell[m->hh_node[i]]);
    }
  } else {
    for (size_t i = 0; i < m->pas_node.size(); ++i) {
      idx.push_back(m->node_elem[m->pas_node[i]]);
      cell.push_back(m->node_cell[m->pas_node[i]]);
    }
  }
}

cn_status cn_set_cell_param(cn_model* m, int32_t param, const double* values) {
  if (!m || !values || param < 0 || param > 2) return m ? m->fail(CN_EINVAL, "bad parameter id") : CN_EINVAL;
  for (int c = 0; c < m->n_cells; ++c)
    if (!std::isfinite(values[c])) return m->fail(CN_EINVAL, "non-finite parameter value");
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  CN_CHECK(prepare(m));
  CN_CHECK(ensure_capacity(m, m->step));
  std::vector<int64_t> idx;
  std::vector<int32_t> cell;
  param_targets(m, param, idx, cell);
  const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
  cn::DevModel dm = m->dm;
  if (!idx.empty()) {
    std::vector<double> val(idx.size());
    for (size_t i = 0; i < idx.size(); ++i) val[i] = values[cell[i]];
    int64_t* d_idx;
    double* d_val;
    CN_CHECK(upload(m, &d_idx, idx));
    CN_CHECK(upload(m, &d_val, val));
    double* dst = param < 2 ? const_cast<double*>(dm.hh_raw) : const_cast<double*>(dm.pas_g);
    const int64_t n = (int64_t)idx.size();
    CN_CHECK(launch_checked(m, [&] { cn::k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(dst, d_idx, d_val, n); }));
    CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
    dfree_raw(m, d_idx);
    dfree_raw(m, d_val);
  }
  if (param < 2) CN_CHECK(launch_checked(m, [&] { cn::k_hh_params<<<nb, tb, 0, m->stream>>>(dm); }));
  else {
    CN_CHECK(launch_checked(m, [&] { cn::k_pas_apply<<<nb, tb, 0, m->stream>>>(dm); }));
    CN_CHECK(launch_checked(m, [&] { cn::k_syn_consts<<<nb, tb, 0, m->stream>>>(dm); }));
  }
  CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
  return CN_OK;
}

cn_status cn_get_cell_param(cn_model* m, int32_t param, double* values) {
  if (!m || !values || param < 0 || param > 2) return m ? m->fail(CN_EINVAL, "bad parameter id") : CN_EINVAL;
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  CN_CHECK(prepare(m));
  std::vector<int64_t> idx;
  std::vector<int32_t> cell;
  param_targets(m, param, idx, cell);
  for (int c = 0; c < m->n_cells; ++c) values[c] = 0.0;
  if (idx.empty()) return CN_OK;
  int64_t* d_idx;
  double* d_out;
  CN_CHECK(upload(m, &d_idx, idx));
  CN_CHECK(zeros(m, &d_out, idx.size()));
  const double* src = param < 2 ? m->dm.hh_raw : m->dm.pas_g;
  const int64_t n = (int64_t)idx.size();
  CN_CHECK(launch_checked(m, [&] { cn::k_gather<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(src, d_idx, d_out, n); }));
  std::vector<double> h(idx.size());
  CN_TRY_CUDA(m, cudaMemcpyAsync(h.data(), d_out, h.size() * 8, cudaMemcpyDeviceToHost, m->stream));
  CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
  dfree_raw(m, d_idx);
  dfree_raw(m, d_out);
  // the value of a cell's first instance (the engine keeps them equal)
  std::vector<uint8_t> seen(m->n_cells, 0);
  for (size_t i = 0; i < idx.size(); ++i)
    if (!seen[cell[i]]++) values[cell[i]] = h[i];
  return CN_OK;
}

// ---- checkpoint / restart (Section 3.4).  The file holds the state in the
// model's input order (nodes, mechanism instances, cells), so it does not
// depend on the layout: a checkpoint taken under one mapping restores under
// another.  Pending NetCon deliveries are not stored as events: the spike
// history of the intervals that can still deliver is stored instead (one bit
// per source and step), and the pull kernel re-derives every delivery from
// it, exactly as in an uninterrupted run.

cn_status cn_checkpoint_save(cn_model* m, void* buf, size_t cap, size_t* n) {
  if (!m || !n) return CN_EINVAL;
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  CN_CHECK(prepare(m));
  if (m->step % m->D != 0) return m->fail(CN_ESTATE, "checkpoints are taken at interval boundaries");
  CN_CHECK(ensure_capacity(m, m->step));
  CkPlan P;
  ck_plan(m, P);
  const int64_t J = m->step / m->D;
  const int64_t w0 = std::max<int64_t>(0, J - (m->max_ds + m->D - 1) / m->D - 1);
  *n = ck_bytes(m, P, J - w0);
  if (!buf) return CN_OK;
  if (cap < *n) return m->fail(CN_ERANGE, "checkpoint buffer too small");
  CN_CHECK(cn_sync(m));
  char* out = static_cast<char*>(buf);
  CkHeader hd{};
  hd.magic = kCkMagic;
  hd.fingerprint = network_fingerprint(m);
  hd.step = m->step;
  hd.window0 = w0;
  hd.n_nodes = m->n_nodes;
  hd.n_hh = (int64_t)m->hh_node.size();
  hd.n_syn = (int64_t)m->syn_node.size();
  for (int t = 0; t < cn::kChanTypes; ++t) hd.n_ch[t] = (int64_t)m->ch_node[t].size();
  hd.n_cells = m->n_cells;
  hd.D = m->D;
  hd.has_cai = m->dm.cai != nullptr;
  std::memcpy(out, &hd, sizeof(hd));
  out += sizeof(hd);
  std::vector<char> h;
  for (size_t k = 0; k < P.dev.size(); ++k) {
    h.resize((size_t)std::max<int64_t>(P.dev_elems[k], 1) * P.bytes[k]);
    CN_TRY_CUDA(m, cudaMemcpy(h.data(), P.dev[k], (size_t)P.dev_elems[k] * P.bytes[k], cudaMemcpyDeviceToHost));
    for (int64_t e : *P.map[k]) {
      const double x = gate_load(h.data(), e, P.bytes[k]);
      std::memcpy(out, &x, 8);
      out += 8;
    }
  }
  std::vector<uint8_t> above(m->n_slots);
  CN_TRY_CUDA(m, cudaMemcpy(above.data(), m->dm.s_above, above.size(), cudaMemcpyDeviceToHost));
  for (int c = 0; c < m->n_cells; ++c) *out++ = (char)above[m->node_slot[m->off[c] + m->spike_node[c]]];
  const size_t hb = (size_t)(J - w0) * m->n_cells * sizeof(uint64_t);
  if (hb) CN_TRY_CUDA(m, cudaMemcpy(out, m->dm.hist + (size_t)w0 * m->n_cells, hb, cudaMemcpyDeviceToHost));
  return CN_OK;
}

cn_status cn_checkpoint_load(cn_model* m, const void* buf, size_t n) {
  if (!m || !buf) return CN_EINVAL;
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  CN_CHECK(prepare(m));
  CkHeader hd;
  if (n < sizeof(hd)) return m->fail(CN_EINVAL, "not a checkpoint");
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kCkMagic) return m->fail(CN_EINVAL, "not a checkpoint");
  if (hd.fingerprint != network_fingerprint(m) || hd.n_cells != m->n_cells || hd.D != m->D ||
      hd.n_nodes != m->n_nodes || hd.has_cai != (m->dm.cai != nullptr))
    return m->fail(CN_EINVAL, "the checkpoint belongs to another network");
  CkPlan P;
  ck_plan(m, P);
  const int64_t J = hd.step / m->D;
  if (hd.step % m->D != 0 || hd.window0 < 0 || hd.window0 > J || n != ck_bytes(m, P, J - hd.window0))
    return m->fail(CN_EINVAL, "malformed checkpoint");
  CN_CHECK(ensure_capacity(m, hd.step));
  CN_CHECK(cn_sync(m));
  const char* in = static_cast<const char*>(buf) + sizeof(hd);
  std::vector<char> h;
  for (size_t k = 0; k < P.dev.size(); ++k) {
    const size_t nb = (size_t)P.dev_elems[k] * P.bytes[k];
    h.resize(std::max<size_t>(nb, 1));
    CN_TRY_CUDA(m, cudaMemcpy(h.data(), P.dev[k], nb, cudaMemcpyDeviceToHost));
    for (int64_t e : *P.map[k]) {
      double x;
      std::memcpy(&x, in, 8);
      in += 8;
      gate_store(h.data(), e, P.bytes[k], x);
    }
    CN_TRY_CUDA(m, cudaMemcpy(P.dev[k], h.data(), nb, cudaMemcpyHostToDevice));
  }
  std::vector<uint8_t> above(m->n_slots);
  CN_TRY_CUDA(m, cudaMemcpy(above.data(), m->dm.s_above, above.size(), cudaMemcpyDeviceToHost));
  for (int c = 0; c < m->n_cells; ++c) above[m->node_slot[m->off[c] + m->spike_node[c]]] = (uint8_t)*in++;
  CN_TRY_CUDA(m, cudaMemcpy(m->dm.s_above, above.data(), above.size(), cudaMemcpyHostToDevice));
  CN_TRY_CUDA(m, cudaMemset(m->dm.hist, 0, (size_t)m->hist_cap * m->n_cells * sizeof(uint64_t)));
  const size_t hb = (size_t)(J - hd.window0) * m->n_cells * sizeof(uint64_t);
  if (hb) CN_TRY_CUDA(m, cudaMemcpy(m->dm.hist + (size_t)hd.window0 * m->n_cells, in, hb, cudaMemcpyHostToDevice));
  // this model's own external events apply from the checkpoint step on
  std::vector<int64_t> xpos(m->n_slots);
  for (int s = 0; s < m->n_slots; ++s)
    xpos[s] = std::lower_bound(m->x_step_h.begin() + m->x_off_h[s], m->x_step_h.begin() + m->x_off_h[s + 1],
                               hd.step) - m->x_step_h.begin();
  CN_TRY_CUDA(m, cudaMemcpy(m->dm.x_pos, xpos.data(), xpos.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  CN_TRY_CUDA(m, cudaMemset(m->dm.status, 0, sizeof(int32_t)));
  CN_TRY_CUDA(m, cudaMemcpy(m->dm.jdev, &J, sizeof(J), cudaMemcpyHostToDevice));
  if (m->dense) {  // channel currents (and ica) follow from the restored gates and voltages
    const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
    cn::DevModel dm = m->dm;
    switch (m->opt.precision) {
      case CN_PREC_FP64: CN_CHECK(launch_checked(m, [&] { cn::k_dense_currents<0><<<nb, tb, 0, m->stream>>>(dm); })); break;
      case CN_PREC_GATE_FP32: CN_CHECK(launch_checked(m, [&] { cn::k_dense_currents<1><<<nb, tb, 0, m->stream>>>(dm); })); break;
      default: CN_CHECK(launch_checked(m, [&] { cn::k_dense_currents<2><<<nb, tb, 0, m->stream>>>(dm); })); break;
    }
  }
  m->step = hd.step;
  m->raster_from = hd.step;
  CN_CHECK(gap_publish(m));
  if (m->dm.trace) {
    const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
    cn::DevModel dm = m->dm;
    const int64_t k = m->step;
    CN_CHECK(launch_checked(m, [&] { cn::k_record0<<<nb, tb, 0, m->stream>>>(dm, k); }));
  }
  CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
  return CN_OK;
}

cn_status cn_enable_adjoint(cn_model* m, int32_t checkpoint_steps) {
  if (!m || checkpoint_steps < 1) return m ? m->fail(CN_EINVAL, "checkpoint interval must be >= 1 step") : CN_EINVAL;
  if (m->step != 0) return m->fail(CN_ESTATE, "enable the adjoint at step 0");
  if (m->opt.precision != CN_PREC_FP64) return m->fail(CN_ESTATE, "the adjoint is defined for the FP64 path");
  if (!m->nc_src.empty() || !m->ev_syn.empty() || !m->gap_node.empty())
    return m->fail(CN_ESTATE, "the adjoint needs a model without NetCons, external events or gap junctions");
  if (m->dense) return m->fail(CN_ESTATE, "the adjoint covers HH, pas and IClamp models");
  std::vector<int> nh(m->n_cells, 0);
  for (int32_t node : m->hh_node)
    if (++nh[m->node_cell[node]] > 1) return m->fail(CN_EINVAL, "the adjoint supports one HH instance per cell");
  m->ck_steps = checkpoint_steps;
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  CN_CHECK(prepare(m));
  m->ck_bytes = snapshot_bytes(m);
  return CN_OK;
}

cn_status cn_run_adjoint(cn_model* m, const double* dj, double* grad) {
  if (!m || !dj || !grad) return CN_EINVAL;
  if (m->ck_steps <= 0) return m->fail(CN_ESTATE, "call cn_enable_adjoint before the forward run");
  const int64_t K = m->step;
  if (K < 1) return m->fail(CN_ESTATE, "run forward at least one step first");
  const int nr = m->dm.n_rec;
  if (nr == 0) return m->fail(CN_ESTATE, "the loss needs recorded nodes");
  CN_TRY_CUDA(m, cudaSetDevice(m->opt.device));
  CN_CHECK(cn_sync(m));
  const int64_t S = m->ck_steps, E = m->node_elems, H = std::max<int64_t>(m->hh_elems, 1);
  // device buffers
  std::vector<double> h_dj((size_t)(K + 1) * nr);
  for (int r = 0; r < nr; ++r)
    for (int64_t k = 0; k <= K; ++k) h_dj[(size_t)k * nr + r] = dj[(size_t)r * (K + 1) + k];
  cn::AdjView A{};
  double* p;
  CN_CHECK(upload(m, &p, h_dj)); A.dj = p;
  CN_CHECK(zeros(m, &A.lam, E));
  CN_CHECK(zeros(m, &A.ytmp, E));
  CN_CHECK(zeros(m, &A.qtmp, E));
  CN_CHECK(zeros(m, &A.xi, 3 * (size_t)m->n_slots));
  CN_CHECK(zeros(m, &A.grad, 3 * (size_t)m->n_slots));
  A.K = K;
  double *tv, *tg;
  CN_CHECK(zeros(m, &tv, (size_t)(S + 1) * E));
  CN_CHECK(zeros(m, &tg, (size_t)(S + 1) * 3 * H));
  void* fin = dalloc_raw(m, m->ck_bytes);
  if (!fin) return m->fail(CN_ENOMEM, "adjoint allocation failed");
  CN_CHECK(snapshot(m, fin, true));
  const int tb = 128, nb = (m->n_slots + tb - 1) / tb;
  {
    cn::DevModel dm = m->dm;
    CN_CHECK(launch_checked(m, [&] { cn::k_adjoint_init<<<nb, tb, 0, m->stream>>>(dm, A); }));
  }
  const size_t adj_smem = (size_t)m->dm.stack_depth * cn::kLanes * 3 * sizeof(double);
  for (int64_t seg = (K - 1) / S; seg >= 0; --seg) {
    const int64_t k0 = seg * S, k1 = std::min<int64_t>(K, k0 + S);
    CN_CHECK(snapshot(m, m->ck_buf[(size_t)seg], false));
    m->dm.traj_v = tv;
    m->dm.traj_g = tg;
    m->dm.traj_k0 = k0;
    cn::DevModel dm = m->dm;
    CN_CHECK(launch_checked(m, [&] { cn::k_traj_first<<<nb, tb, 0, m->stream>>>(dm); }));
    m->step = k0;
    CN_CHECK(advance(m, k1, true));
    CN_CHECK(launch_checked(m, [&] {
      cn::k_adjoint<<<m->n_groups, 32, adj_smem, m->stream>>>(dm, A, k0, k1);
    }));
  }
  m->dm.traj_v = nullptr;
  m->dm.traj_g = nullptr;
  CN_CHECK(snapshot(m, fin, false));
  m->step = K;
  std::vector<double> h_g(3 * (size_t)m->n_slots);
  CN_TRY_CUDA(m, cudaMemcpyAsync(h_g.data(), A.grad, h_g.size() * 8, cudaMemcpyDeviceToHost, m->stream));
  CN_TRY_CUDA(m, cudaStreamSynchronize(m->stream));
  for (size_t i = 0; i < 3 * (size_t)m->n_cells; ++i) grad[i] = 0.0;
  for (int sl = 0; sl < m->n_slots; ++sl)
    if (m->slot_cell[sl] >= 0)
      for (int q = 0; q < 3; ++q) grad[(size_t)q * m->n_cells + m->slot_cell[sl]] += h_g[(size_t)q * m->n_slots + sl];
  for (void* b : {(void*)A.dj, (void*)A.lam, (void*)A.ytmp, (void*)A.qtmp, (void*)A.xi, (void*)A.grad, (void*)tv,
                  (void*)tg, fin})
    dfree_raw(m, b);
  return CN_OK;
}

cn_status cn_fp64_peak(cn_model* m, double* tflops) {
  if (!m || !tflops) return CN_EINVAL;
  int dev = 0, nsm = 0;
  CN_TRY_CUDA(m, cudaGetDevice(&dev));
  CN_TRY_CUDA(m, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 4, threads = 128, iters = 20000;
  double* sink = static_cast<double*>(dalloc_raw(m, (size_t)blocks * threads * sizeof(double)));
  if (!sink) return m->fail(CN_ENOMEM, "device allocation failed");
  cudaEvent_t e0 = take_event(m), e1 = take_event(m);
  cn::k_dfma_stream<<<blocks, threads, 0, m->stream>>>(sink, iters / 10, 0.999999, 1e-7);  // warm-up
  CN_TRY_CUDA(m, cudaEventRecord(e0, m->stream));
  cn::k_dfma_stream<<<blocks, threads, 0, m->stream>>>(sink, iters, 0.999999, 1e-7);
  CN_TRY_CUDA(m, cudaEventRecord(e1, m->stream));
  CN_TRY_CUDA(m, cudaGetLastError());
  CN_TRY_CUDA(m, cudaEventSynchronize(e1));
  float ms = 0.f;
  CN_TRY_CUDA(m, cudaEventElapsedTime(&ms, e0, e1));
  m->ev_pool.push_back(e0);
  m->ev_pool.push_back(e1);
  dfree_raw(m, sink);
  *tflops = 2.0 * 4.0 * (double)blocks * threads * iters / (ms * 1e-3) / 1e12;
  return CN_OK;
}

cn_status cn_pivot_reciprocal(int64_t n, const double* d, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!d || !out))) return CN_EINVAL;
  if (n == 0) return CN_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int tb = 256;
  cn::k_rcp64<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(d, out, n);
  if (cudaGetLastError() != cudaSuccess) return CN_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? CN_OK : CN_ECUDA;
}

const char* cn_last_error(const cn_model* m) {
  if (!m) return g_create_error.c_str();
  return m->err.c_str();
}

void cn_model_destroy(cn_model* m) {
  if (!m) return;
  if (m->stream || m->finalized) cudaStreamSynchronize(m->stream);
  std::vector<void*> all = m->allocs;
  for (void* p : all) dfree_raw(m, p);
  for (auto& pr : m->ev_interval) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (auto& pr : m->ev_pull) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (cudaEvent_t e : m->ev_pool) cudaEventDestroy(e);
  drop_graphs(m);
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  delete m;
}

}  // extern "C"
