// cn_solve.cu -- batched tree solves (cn_solve_trees).
//
// Gaussian elimination in Hines order (Section 2, citing Hines 1984) of many
// independent tree matrices given in device memory: row i of tree t has
// diagonal d[i], coupling b[i] to its parent p and, in row p, coupling a[i]
// to i.  One thread per tree eliminates leaves to root and back-substitutes
// root to leaves.  The inputs stay untouched: the eliminated diagonal lives
// in scratch memory and the right-hand side is copied into the output first.
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "cn.h"

namespace cn {

enum : int32_t { kSolveBadParent = 1, kSolveZeroPivot = 2, kSolveBadOffset = 4 };

// Offsets are checked before any tree is touched: off[0] = 0,
// off[n_trees] = n_nodes and off[t] <= off[t+1] for every t make the trees'
// row ranges disjoint and inside [0, n_nodes).  Any violation sets
// kSolveBadOffset, and then k_solve_trees solves nothing.
__global__ void k_check_offsets(int32_t n_trees, int64_t n_nodes, const int32_t* __restrict__ off,
                                int32_t* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > n_trees) return;
  const int32_t o = off[t];
  bool bad = o < 0 || (int64_t)o > n_nodes;
  if (t == 0) bad = bad || o != 0;
  if (t == n_trees) bad = bad || (int64_t)o != n_nodes;
  else bad = bad || off[t + 1] < o;
  if (bad) atomicOr(status, kSolveBadOffset);
}

// dd: scratch of n_nodes doubles.  status: one int32, OR-ed with error bits;
// a tree with a bad parent index or a zero pivot is left unsolved, and
// nothing is solved after a bad offset.
__global__ void k_solve_trees(int32_t n_trees, const int32_t* __restrict__ off, const int32_t* __restrict__ parent,
                              const double* __restrict__ a, const double* __restrict__ b,
                              const double* __restrict__ d, const double* __restrict__ rhs, double* __restrict__ x,
                              double* __restrict__ dd, int32_t* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_trees) return;
  if (*(volatile int32_t*)status & kSolveBadOffset) return;
  const int32_t i0 = off[t], i1 = off[t + 1];
  if (i1 <= i0) return;
  if (parent[i0] != -1) {
    atomicOr(status, kSolveBadParent);
    return;
  }
  for (int32_t i = i0 + 1; i < i1; ++i) {
    const int32_t p = parent[i];
    if (p < 0 || p >= i - i0) {
      atomicOr(status, kSolveBadParent);
      return;
    }
  }
  for (int32_t i = i0; i < i1; ++i) {
    dd[i] = d[i];
    x[i] = rhs[i];
  }
  for (int32_t i = i1 - 1; i > i0; --i) {
    const int32_t p = i0 + parent[i];
    if (dd[i] == 0.0) {
      atomicOr(status, kSolveZeroPivot);
      return;
    }
    const double f = a[i] / dd[i];
    dd[p] -= f * b[i];
    x[p] -= f * x[i];
  }
  if (dd[i0] == 0.0) {
    atomicOr(status, kSolveZeroPivot);
    return;
  }
  x[i0] /= dd[i0];
  for (int32_t i = i0 + 1; i < i1; ++i) x[i] = (x[i] - b[i] * x[i0 + parent[i]]) / dd[i];
}

// The two launches of a solve on one stream: the offset check, then the
// trees (which read the check's result from the status word).
cudaError_t launch_solve(int32_t n_trees, int64_t n_nodes, const int32_t* off, const int32_t* parent,
                         const double* a, const double* b, const double* d, const double* rhs, double* x,
                         double* dd, int32_t* status, cudaStream_t st) {
  const int tb = 128;
  k_check_offsets<<<(n_trees + 1 + tb - 1) / tb, tb, 0, st>>>(n_trees, n_nodes, off, status);
  k_solve_trees<<<(n_trees + tb - 1) / tb, tb, 0, st>>>(n_trees, off, parent, a, b, d, rhs, x, dd, status);
  return cudaGetLastError();
}

cn_status solve_status(int32_t st) {
  if (st & (kSolveBadParent | kSolveBadOffset)) return CN_EINVAL;
  if (st & kSolveZeroPivot) return CN_ERANGE;
  return CN_OK;
}

}  // namespace cn

extern "C" {

cn_status cn_solve_trees(int32_t n_trees, int64_t n_nodes, const int32_t* offset, const int32_t* parent,
                         const double* a, const double* b, const double* d, const double* rhs, double* x,
                         void* stream) {
  if (n_trees < 0 || n_nodes < 0) return CN_EINVAL;
  if (n_trees == 0 || n_nodes == 0) return CN_OK;
  if (!offset || !parent || !a || !b || !d || !rhs || !x) return CN_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* dd = nullptr;
  int32_t* status = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&dd), (size_t)n_nodes * sizeof(double), st) != cudaSuccess)
    return CN_ENOMEM;
  if (cudaMallocAsync(reinterpret_cast<void**>(&status), sizeof(int32_t), st) != cudaSuccess) {
    cudaFreeAsync(dd, st);
    return CN_ENOMEM;
  }
  cn_status rc = CN_OK;
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) rc = CN_ECUDA;
  if (rc == CN_OK && cn::launch_solve(n_trees, n_nodes, offset, parent, a, b, d, rhs, x, dd, status, st) !=
                        cudaSuccess)
    rc = CN_ECUDA;
  int32_t h = 0;
  if (rc == CN_OK && cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = CN_ECUDA;
  cudaFreeAsync(dd, st);
  cudaFreeAsync(status, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = CN_ECUDA;
  if (rc == CN_OK) rc = cn::solve_status(h);
  return rc;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free variant of cn_solve_trees.
//
// Some callers cannot allocate device memory at the moment they need a
// solve: their GPU memory is already reserved in full by another allocator
// (a framework's caching pool), or an allocation would synchronize or stall
// a latency-critical loop.  For them the working diagonal and the status
// word live in the fixed arrays below, which are part of this library's
// device image: every GPU that loads the library holds them (8 MiB + 4
// bytes) until the process exits.  In host code these names are host-side
// stand-ins, never device addresses; their device addresses are looked up
// once per device with cudaGetSymbolAddress.
namespace {

constexpr int64_t kNoAllocMaxNodes = int64_t(1) << 20;  // rows across all trees of one call

static __device__ __align__(256) double g_noalloc_dd[kNoAllocMaxNodes];
static __device__ __align__(256) int32_t g_noalloc_status[1];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_dd_ptr[kMaxDevices] = {};
int32_t* g_noalloc_status_ptr[kMaxDevices] = {};

// Device addresses of the fixed scratch on the current device (set up on the
// first call per device).
cn_status noalloc_scratch(double** dd, int32_t** status) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CN_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return CN_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_dd_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_dd) != cudaSuccess) return CN_ECUDA;
    if (cudaGetSymbolAddress(&q, g_noalloc_status) != cudaSuccess) return CN_ECUDA;
    g_noalloc_dd_ptr[dev] = static_cast<double*>(p);
    g_noalloc_status_ptr[dev] = static_cast<int32_t*>(q);
  }
  *dd = g_noalloc_dd_ptr[dev];
  *status = g_noalloc_status_ptr[dev];
  return CN_OK;
}

}  // namespace

extern "C" cn_status cn_solve_trees_noalloc(int32_t n_trees, int64_t n_nodes, const int32_t* offset,
                                            const int32_t* parent, const double* a, const double* b,
                                            const double* d, const double* rhs, double* x, void* stream) {
  if (n_trees < 0 || n_nodes < 0) return CN_EINVAL;
  if (n_nodes > kNoAllocMaxNodes) return CN_ERANGE;
  if (n_trees == 0 || n_nodes == 0) return CN_OK;
  if (!offset || !parent || !a || !b || !d || !rhs || !x) return CN_EINVAL;
  double* dd = nullptr;
  int32_t* status = nullptr;
  cn_status rc = noalloc_scratch(&dd, &status);
  if (rc != CN_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The status word must start at zero; the diagonal is fully overwritten.
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return CN_ECUDA;
  if (cn::launch_solve(n_trees, n_nodes, offset, parent, a, b, d, rhs, x, dd, status, st) != cudaSuccess)
    return CN_ECUDA;
  int32_t h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CN_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CN_ECUDA;
  return cn::solve_status(h);
}
