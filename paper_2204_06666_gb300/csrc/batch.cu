// Batched EHYB SpMV: many plans (matrices of uneven size) in one persistent launch.
//
// The work units are (plan, partition) tiles, sorted by their slot count, largest first (longest-
// processing-time order).  A grid of (SMs x resident blocks) blocks pulls tiles from one atomic
// counter and runs each with the same per-partition code as the single-plan kernel
// (core::partition_spmv), so every row is summed in exactly the same order as by ehyb_spmv: the
// batch result equals the per-plan results bit for bit.  Each tile stages its slice of x straight from
// the caller's x through the plan's new_to_old (the permutation is fused into the loads, as in
// ehyb_spmv), so the batch is ONE launch.  The last block to leave resets the counter, so the launch is
// captured once into a CUDA graph and replayed; a call only rewrites the table of x / y pointers when
// they change.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ehyb_core.cuh"
#include "plan_internal.h"

namespace ehyb {
namespace {

using namespace core;

struct BatchPlan {
  KArgs a;
  const double* ell_val;
  const double* er_val;
  const double* x;  // caller's x (original numbering)
  double* y;        // caller's y (original numbering)
  int64_t n;
  int32_t kbatch;   // the plan's batch depth (6 on wide slices, else 8)
};

constexpr int kMaxThreads = 1024;  // block size: 512 when two or more blocks fit an SM, else 1024

__global__ void __launch_bounds__(kMaxThreads, 1) batch_kernel(const BatchPlan* __restrict__ plans,
                                                              const int2* __restrict__ tiles, int ntiles,
                                                              int* counters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ BlockState bs;
  __shared__ int tile_s;
  if (threadIdx.x == 0) {
    bs.bar_ready = 0;
    bs.phase = 0;
  }
  for (;;) {
    __syncthreads();  // the previous tile's reads of shared memory are complete
    if (threadIdx.x == 0) tile_s = atomicAdd(&counters[0], 1);
    __syncthreads();
    const int t = tile_s;
    if (t >= ntiles) break;
    const int2 tl = tiles[t];
    const BatchPlan& bp = plans[tl.x];
    double* xs = reinterpret_cast<double*>(smem_raw);
    const bool ok =
        bp.kbatch == 6
            ? partition_spmv<double, double, true, true, false, true, 6>(bp.a, bp.ell_val, bp.er_val, bp.x, bp.y,
                                                                         tl.y, xs, bs)
            : partition_spmv<double, double, true, true, false, true>(bp.a, bp.ell_val, bp.er_val, bp.x, bp.y, tl.y,
                                                                      xs, bs);
    if (!ok) break;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the last block out resets the queue for the next launch
    __threadfence();
    if (atomicAdd(&counters[1], 1) == (int)gridDim.x - 1) {
      counters[0] = 0;
      counters[1] = 0;
      __threadfence();
    }
  }
}

}  // namespace
}  // namespace ehyb

using namespace ehyb;

struct ehyb_batch_s {
  int32_t count = 0;
  int device = -1;
  std::vector<ehyb_plan_t> plans;
  std::vector<BatchPlan> table;
  std::vector<const double*> xs;
  std::vector<double*> ys;
  void* arena = nullptr;
  BatchPlan* d_table = nullptr;
  int2* d_tiles = nullptr;
  int* d_counters = nullptr;
  int ntiles = 0, grid = 0, threads = 512;
  size_t smem = 0;
  int64_t max_n = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
};

#define CKB(call)                                                     \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_error_status(e_, #call);       \
  } while (0)

static void batch_free(ehyb_batch_t b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->arena) cudaFree(b->arena);
  delete b;
}

extern "C" ehyb_status_t ehyb_batch_create(int32_t count, const ehyb_plan_t* plans, ehyb_batch_t* out) {
  if (!out) return EHYB_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || !plans) return EHYB_ERR_INVALID_ARG;
  ehyb_batch_s* b = new (std::nothrow) ehyb_batch_s();
  if (!b) return EHYB_ERR_OOM;
  b->count = count;
  std::vector<int2> tiles;
  std::vector<int64_t> cost;
  for (int i = 0; i < count; ++i) {
    ehyb_plan_t P = plans[i];
    if (!P) { batch_free(b); return EHYB_ERR_INVALID_ARG; }
    if (P->host_only || P->er_layout != 0) { batch_free(b); return EHYB_ERR_UNSUPPORTED; }
    if (b->device < 0) b->device = P->device;
    if (P->device != b->device) { batch_free(b); return EHYB_ERR_INVALID_ARG; }
    b->plans.push_back(P);
    BatchPlan bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.a = make_kargs(P->dev);
    bp.ell_val = P->dev.ell_val;
    bp.er_val = P->dev.er_sval;
    bp.n = P->dev.n;
    bp.kbatch = P->dev.kbatch;
    b->table.push_back(bp);
    b->max_n = std::max(b->max_n, P->dev.n);
    b->smem = std::max(b->smem, ehyb_smem_bytes(P->dev, 8));
    const HostPlan& H = P->host;
    for (int32_t p = 0; p < H.nparts; ++p) {
      const int32_t s0 = H.slice_ptr[(size_t)p], s1 = H.slice_ptr[(size_t)p + 1];
      const int64_t c = (H.slice_pos[(size_t)s1] - H.slice_pos[(size_t)s0]) +
                        (H.er_slice_pos[(size_t)s1] - H.er_slice_pos[(size_t)s0]) + 32;
      tiles.push_back(make_int2(i, p));
      cost.push_back(c);
    }
  }
  // longest tiles first (stable, so ties keep plan / partition order)
  std::vector<size_t> order(tiles.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](size_t u, size_t v) { return cost[u] > cost[v]; });
  std::vector<int2> sorted(tiles.size());
  for (size_t k = 0; k < order.size(); ++k) sorted[k] = tiles[order[k]];
  b->ntiles = (int)sorted.size();
  b->xs.assign((size_t)count, nullptr);
  b->ys.assign((size_t)count, nullptr);

  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess || cur != b->device) { batch_free(b); return EHYB_ERR_INVALID_ARG; }
  int sms = 0, per_sm = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  // 512 threads while two blocks fit an SM (one block's staging overlaps the other's slices), otherwise
  // one block of 1024 threads per SM (32 warps keep enough loads in flight)
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, 512, b->smem);
  if (e == cudaSuccess && per_sm < 2) {
    b->threads = kMaxThreads;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kMaxThreads, b->smem);
  }
  if (e != cudaSuccess) { batch_free(b); return cuda_error_status(e, "batch launch setup"); }
  b->grid = sms * std::max(per_sm, 1);

  const size_t t_bytes = ((size_t)count * sizeof(BatchPlan) + 255) & ~(size_t)255;
  const size_t l_bytes = ((size_t)std::max(b->ntiles, 1) * sizeof(int2) + 255) & ~(size_t)255;
  ehyb_status_t st = device_alloc(&b->arena, t_bytes + l_bytes + 256);
  if (st != EHYB_OK) { batch_free(b); return st; }
  b->d_table = (BatchPlan*)b->arena;
  b->d_tiles = (int2*)((char*)b->arena + t_bytes);
  b->d_counters = (int*)((char*)b->arena + t_bytes + l_bytes);
  e = cudaMemcpy(b->d_table, b->table.data(), (size_t)count * sizeof(BatchPlan), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && b->ntiles)
    e = cudaMemcpy(b->d_tiles, sorted.data(), sorted.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, 256);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) { batch_free(b); return cuda_error_status(e, "batch upload"); }
  *out = b;
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_batch_spmv(ehyb_batch_t b, const double* const* xs, double* const* ys, void* stream) {
  if (!b || !xs || !ys) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  bool changed = false;
  for (int i = 0; i < b->count; ++i) {
    if (b->table[(size_t)i].n > 0 && (!xs[i] || !ys[i] || (const void*)xs[i] == (const void*)ys[i]))
      return EHYB_ERR_INVALID_ARG;
    if (xs[i] != b->xs[(size_t)i] || ys[i] != b->ys[(size_t)i]) {
      b->xs[(size_t)i] = xs[i];
      b->ys[(size_t)i] = ys[i];
      b->table[(size_t)i].x = xs[i];
      b->table[(size_t)i].y = ys[i];
      changed = true;
    }
  }
  if (changed)
    CKB(cudaMemcpyAsync(b->d_table, b->table.data(), (size_t)b->count * sizeof(BatchPlan), cudaMemcpyHostToDevice, s));
  if (b->ntiles == 0) return EHYB_OK;
  if (!b->graph) {
    cudaGraph_t g;
    CKB(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    batch_kernel<<<b->grid, b->threads, b->smem, b->cap>>>(b->d_table, b->d_tiles, b->ntiles, b->d_counters);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    CKB(e1);
    CKB(e2);
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    CKB(e3);
  }
  CKB(cudaGraphLaunch(b->graph, s));
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_batch_info(ehyb_batch_t b, int32_t* ntiles, int32_t* grid, int32_t* threads) {
  if (!b) return EHYB_ERR_INVALID_ARG;
  if (ntiles) *ntiles = b->ntiles;
  if (grid) *grid = b->grid;
  if (threads) *threads = b->threads;
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_batch_destroy(ehyb_batch_t b) {
  if (!b) return EHYB_OK;
  cudaError_t e = cudaDeviceSynchronize();
  batch_free(b);
  return e == cudaSuccess ? EHYB_OK : cuda_error_status(e, "cudaDeviceSynchronize");
}
