// EHYB SpMV kernels for sm_103a: the per-plan launch of the fused kernel (one block per partition),
// the gather / scatter permutations and the plain vector-CSR baseline.  The fused kernel body lives
// in ehyb_core.cuh.
#include "ehyb_core.cuh"
#include "../../include/ehyb.h"

#include <cstdint>
#include <type_traits>

namespace ehyb {

namespace {

using namespace core;

// batch depth of the FP32 / BF16 kernels: a 4- or 2-byte value needs more slots in flight than an FP64 one
// (12 measured best among 8, 12, 16 and 24: tet 126^3 FP32 50.0 -> 49.0 us, BF16 52.0 -> 48.2 us).  On copies
// laid out in runs of four, whose registers hold the runs packed: 16 slots for FP32 (an FP32 run takes six
// registers; 32 spill), 32 for BF16 (four registers a run; tet 126^3 42.7 -> 41.4 us, hex 48^3 29.0 -> 26.8),
// except in the kernels with the fused dot product, where 32 spill.
constexpr int kLowBatch = 12;
template <typename V, bool DOT>
constexpr int run_batch() {
  return (sizeof(V) == 2 && !DOT) ? 32 : 16;
}
template <typename V, typename X, bool SCATTER, bool ER_SLICED, bool DOT, bool GATHER = false,
          int KB = (sizeof(V) == 8 ? kBatch : kLowBatch), bool RUNS = false>
__global__ void __launch_bounds__(1024, 1) ehyb_kernel(KArgs a, const V* __restrict__ ell_val,
                                                    const V* __restrict__ er_val, const X* __restrict__ xp,
                                                    X* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ BlockState bs;
  // Launched with programmatic stream serialization: the next kernel in the stream may be scheduled at
  // once, so its blocks become resident as this grid's blocks leave and its launch latency overlaps
  // this grid's tail.  Before its griddepcontrol.wait (inside partition_spmv) a block reads plan arrays
  // only (its slice table); the wait returns when the previous kernel in the stream has completed and
  // its writes are visible, and x, y and the skip flag are touched only after it.  (An L2 bulk prefetch
  // of each warp's first slice before the wait measured slower on the hex workload and is not done.)
  pdl_launch_dependents();
  if (threadIdx.x == 0) {
    bs.bar_ready = 0;
    bs.phase = 0;
  }
  partition_spmv<V, X, SCATTER, ER_SLICED, DOT, GATHER, KB, RUNS, true, true>(
      a, ell_val, er_val, xp, y, blockIdx.x, reinterpret_cast<X*>(smem_raw), bs);
}

template <typename X>
__global__ void permute_kernel(int64_t n, const int32_t* __restrict__ n2o, int to_new, const X* __restrict__ in,
                               X* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (to_new) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = __ldg(in + n2o[i]);
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[n2o[i]] = in[i];
  }
}

__global__ void csr_kernel(int64_t n, int tpr_log2, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = t >> tpr_log2;
  const int tpr = 1 << tpr_log2;
  const int sub = (int)(t & (tpr - 1));
  double acc = 0.0;
  if (row < n) {
    const int64_t k1 = rp[row + 1];
    for (int64_t k = rp[row] + sub; k < k1; k += tpr) acc = fma(__ldcs(val + k), __ldg(x + __ldcs(col + k)), acc);
  }
  for (int off = tpr >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
  if (sub == 0 && row < n) y[row] = acc;
}

__global__ void bounds_probe_kernel(int64_t i, int64_t lim, int32_t* status) { (void)checked(i, lim, status); }

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

size_t ehyb_smem_bytes(const DevPlan& P, int elem_bytes) {
  const int epv = 16 / elem_bytes;
  const int32_t rows = P.max_stage_rows > P.max_part_rows ? P.max_stage_rows : P.max_part_rows;
  size_t b = (size_t)(rows + epv) * (size_t)elem_bytes;
  return (b + 15) & ~(size_t)15;
}

// batch depth of the FP64 kernels for wide slices (see DevPlan::kbatch)
constexpr int kWideBatch = 6;

template <typename V, typename X>
static cudaError_t set_smem(int bytes) {
  cudaError_t e;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if constexpr (std::is_same<V, double>::value) {
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, false, true, kWideBatch>, attr, bytes))) return e;
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, true, true, kWideBatch>, attr, bytes))) return e;
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, false, true, true, false, kWideBatch>, attr, bytes))) return e;
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, false, true, false, false, kWideBatch>, attr, bytes))) return e;
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, false, false, kWideBatch>, attr, bytes))) return e;
  }
  if constexpr (!std::is_same<V, double>::value) {  // the copies laid out in runs of four (sliced ER layout)
    constexpr int R = run_batch<V, false>(), RD = run_batch<V, true>();
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, false, false, R, true>, attr, bytes))) return e;
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, false, true, false, false, R, true>, attr, bytes))) return e;
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, false, true, R, true>, attr, bytes))) return e;
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, true, true, RD, true>, attr, bytes))) return e;
    if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, false, true, true, false, RD, true>, attr, bytes))) return e;
  }
  if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, false>, attr, bytes))) return e;
  if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, false, false>, attr, bytes))) return e;
  if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, false, true, false>, attr, bytes))) return e;
  if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, false, false, false>, attr, bytes))) return e;
  if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, false, true>, attr, bytes))) return e;
  if ((e = cudaFuncSetAttribute(ehyb_kernel<V, X, true, true, true, true>, attr, bytes))) return e;
  return cudaFuncSetAttribute(ehyb_kernel<V, X, false, true, true>, attr, bytes);
}

// dynamic shared memory a fused-kernel launch may use (the attribute kernels_init sets)
static size_t g_smem_max = 0;

cudaError_t kernels_init(int smem_optin) {
  cudaError_t e;
  g_smem_max = (size_t)smem_optin;
  if ((e = set_smem<double, double>(smem_optin))) return e;
  if ((e = set_smem<float, float>(smem_optin))) return e;
  return set_smem<uint16_t, float>(smem_optin);
}

cudaError_t launch_permute_f64(const DevPlan& P, int to_new, const double* in, double* out, cudaStream_t s) {
  if (P.n == 0) return cudaSuccess;
  permute_kernel<double><<<grid_for(P.n, 256), 256, 0, s>>>(P.n, P.new_to_old, to_new, in, out);
  return cudaGetLastError();
}

cudaError_t launch_permute_f32(const DevPlan& P, int to_new, const float* in, float* out, cudaStream_t s) {
  if (P.n == 0) return cudaSuccess;
  permute_kernel<float><<<grid_for(P.n, 256), 256, 0, s>>>(P.n, P.new_to_old, to_new, in, out);
  return cudaGetLastError();
}

// every fused-kernel launch carries the programmatic-stream-serialization attribute (see ehyb_kernel)
template <typename V, typename X, bool SCATTER, bool ER_SLICED, bool DOT, bool GATHER = false>
static void launch_pdl(const DevPlan& P, size_t smem, cudaStream_t s, const KArgs& a, const V* ev, const V* erv,
                       const X* xp, X* y) {
  // FP64 kernels on plans with wide slices use the shallower batch (sliced-ER layout only); FP32 / BF16
  // copies laid out in runs of four use the run loops
  constexpr bool kWideOk = std::is_same<V, double>::value && ER_SLICED;
  constexpr bool kRunsOk = !std::is_same<V, double>::value && ER_SLICED;
  const bool wide = kWideOk && P.kbatch == kWideBatch;
  const bool runs = kRunsOk && P.lowp_group == 4;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)P.nparts);
  cfg.blockDim = dim3((unsigned)P.threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if constexpr (kWideOk) {
    if (wide) {
      cudaLaunchKernelEx(&cfg, ehyb_kernel<V, X, SCATTER, ER_SLICED, DOT, GATHER, kWideBatch>, a, ev, erv, xp, y);
      return;
    }
  }
  if constexpr (kRunsOk) {
    if (runs) {
      KArgs ar = a;  // the copies' own column arrays, in the same runs
      ar.ell_col = P.ell_col_low;
      ar.er_scol = P.er_scol_low;
      ar.er_scol_old = P.er_scol_old_low;
      cudaLaunchKernelEx(&cfg, ehyb_kernel<V, X, SCATTER, ER_SLICED, DOT, GATHER, run_batch<V, DOT>(), true>, ar, ev, erv,
                         xp, y);
      return;
    }
  }
  cudaLaunchKernelEx(&cfg, ehyb_kernel<V, X, SCATTER, ER_SLICED, DOT, GATHER>, a, ev, erv, xp, y);
}

template <typename V, typename X>
static void launch_typed(const DevPlan& P, const V* ev, const V* erv_csr, const V* erv_sl, const X* xp, X* y,
                         int scatter, size_t smem, cudaStream_t s, const DotOut* dot, const int32_t* skip) {
  KArgs a = make_kargs(P);
  a.smem_elems = (int64_t)(smem / sizeof(X));
  // the partition's slice table after the staged x, when both fit the block's shared memory
  const size_t tbytes = (size_t)P.max_part_slices * sizeof(SliceMeta);
  if (P.max_part_slices > 0 && smem + tbytes <= g_smem_max) {
    a.meta_off = (int32_t)smem;
    a.meta_cap = P.max_part_slices;
    smem += tbytes;
  }
  if (dot) {
    a.dot_part = dot->part;
    a.dot_arrive = dot->arrive;
    a.dot_result = dot->result;
    a.dot_self = dot->self;
  }
  a.skip = skip;
  const bool sl = P.er_layout != 1;  // 2: no extra-row slots of its own (zero widths), the sliced kernels run
  const V* erv = sl ? erv_sl : erv_csr;
  if (dot && scatter == 2 && sl) {  // caller's numbering with the fused dot (preconditioner SpMVs)
    launch_pdl<V, X, true, true, true, true>(P, smem, s, a, ev, erv, xp, y);
  } else if (dot) {  // the fused dot product in the plan numbering (sliced layout, solver use)
    launch_pdl<V, X, false, true, true>(P, smem, s, a, ev, erv, xp, y);
  } else if (scatter == 2 && sl) {  // x in the caller's numbering, permutation fused into the loads
    launch_pdl<V, X, true, true, false, true>(P, smem, s, a, ev, erv, xp, y);
  } else if (scatter) {
    if (sl) launch_pdl<V, X, true, true, false>(P, smem, s, a, ev, erv, xp, y);
    else launch_pdl<V, X, true, false, false>(P, smem, s, a, ev, erv, xp, y);
  } else {
    if (sl) launch_pdl<V, X, false, true, false>(P, smem, s, a, ev, erv, xp, y);
    else launch_pdl<V, X, false, false, false>(P, smem, s, a, ev, erv, xp, y);
  }
}

cudaError_t launch_ehyb_f64(const DevPlan& P, const double* xp, double* y, int scatter, cudaStream_t s,
                            const DotOut* dot, const int32_t* skip) {
  if (P.nparts == 0) return cudaSuccess;
  launch_typed<double, double>(P, P.ell_val, P.er_val, P.er_sval, xp, y, scatter, ehyb_smem_bytes(P, 8), s, dot,
                               skip);
  return cudaGetLastError();
}

cudaError_t launch_ehyb_lowp(const DevPlan& P, int lowp, const float* xp, float* y, int scatter, cudaStream_t s,
                             const DotOut* dot, const int32_t* skip) {
  if (P.nparts == 0) return cudaSuccess;
  const size_t smem = ehyb_smem_bytes(P, 4);
  if (lowp == 1)
    launch_typed<float, float>(P, P.ell_val_f32, P.er_val_f32, P.er_sval_f32, xp, y, scatter, smem, s, dot, skip);
  else
    launch_typed<uint16_t, float>(P, P.ell_val_bf16, P.er_val_bf16, P.er_sval_bf16, xp, y, scatter, smem, s, dot,
                                  skip);
  return cudaGetLastError();
}

cudaError_t launch_csr_f64(int64_t n, const int64_t* rp, const int32_t* col, const double* val, const double* x,
                           double* y, int tpr, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t total = n * (int64_t)tpr;
  const int64_t blocks = (total + threads - 1) / threads;
  csr_kernel<<<(unsigned)blocks, threads, 0, s>>>(n, ilog2(tpr), rp, col, val, x, y);
  return cudaGetLastError();
}

}  // namespace ehyb

extern "C" ehyb_status_t ehyb_test_bounds_probe(int64_t i, int64_t lim) {
  int32_t* d = nullptr;
  if (cudaMalloc(&d, sizeof(int32_t)) != cudaSuccess) return EHYB_ERR_CUDA;
  int32_t h = 0;
  cudaError_t e = cudaMemset(d, 0, sizeof(int32_t));
  if (e == cudaSuccess) {
    ehyb::bounds_probe_kernel<<<1, 1>>>(i, lim, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? (ehyb_status_t)h : EHYB_ERR_CUDA;
}
