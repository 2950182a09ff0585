// EHYB SpMM: Y = A X for k right-hand sides (X, Y row-major n x k, original numbering).
//
// FP64 SpMM on this part is bound by the FP64 FMA pipe k times over (k FMAs per 10-byte slab slot), so
// the plan's Eq. 1 partitions are kept (no re-partitioning for smaller slices, no extra ER) and the
// columns are processed in chunks of KC in {8, 4, 2, 1}: the largest KC whose KC-column slice of X fits
// one block's shared memory and divides k.  X is first gathered into a chunk-major layout
// X_p[c][i][j] = X[new_to_old[i]][c*KC + j], so every chunk's slice of a partition is one contiguous
// bulk copy; each chunk is one launch with one block per partition that stages it, walks the slab and
// the sliced ER slots of its slices exactly like the SpMV (same slot order, so column j of Y equals
// ehyb_spmv of column j bit for bit) and writes KC outputs per row into Y[new_to_old[r]][c*KC + j].
// Re-streaming the slab once per chunk costs far less time than the chunk's FMAs.
#include <cuda_runtime.h>

#include <algorithm>

#include "ehyb_core.cuh"
#include "plan_internal.h"

namespace ehyb {
namespace {

using namespace core;

// X_p (chunk-major) from X (row-major), one thread per element
__global__ void spmm_gather_kernel(int64_t n, int k, int kc, const int32_t* __restrict__ n2o,
                                   const double* __restrict__ X, double* __restrict__ Xp) {
  const int64_t total = n * (int64_t)k;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    const int c = j / kc;
    Xp[(int64_t)c * n * kc + i * kc + (j - c * kc)] = __ldg(X + (int64_t)n2o[i] * k + j);
  }
}

template <int KC>
__global__ void __launch_bounds__(512) spmm_kernel(KArgs a, const double* __restrict__ ell_val,
                                                   const double* __restrict__ er_val, const double* __restrict__ xc,
                                                   double* __restrict__ Y, int k, int c0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ BlockState bs;
  const int p = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int pb = a.part_ptr[p], pe = a.part_ptr[p + 1];
  const int s0 = a.slice_ptr[p], s1 = a.slice_ptr[p + 1];
  double* xs = reinterpret_cast<double*>(smem_raw);
  // stage doubles [pb*KC, pe*KC) of this chunk: 16-byte aligned bulk part + plain-load tail
  const int64_t e0 = (int64_t)pb * KC, e1 = (int64_t)pe * KC;
  const int64_t a0 = e0 & ~(int64_t)1, a1 = e1 & ~(int64_t)1;
  const bool aligned_src = ((reinterpret_cast<uintptr_t>(xc) & 15u) == 0);
  const uint32_t bulk_bytes = (aligned_src && a1 > a0) ? (uint32_t)((a1 - a0) * 8) : 0u;
  if (tid == 0) {
    bs.slice_counter = s0 + nwarps;
    if (bulk_bytes) {
      mbar_init(&bs.bar, 1);
      mbar_arrive_expect_tx(&bs.bar, bulk_bytes);
      if (!a.inject) bulk_g2s(xs, xc + a0, bulk_bytes, &bs.bar);
    }
  }
  {
    const int64_t lo = bulk_bytes ? (a1 > e0 ? a1 : e0) : e0;
    for (int64_t i = lo + tid; i < e1; i += blockDim.x) xs[checked(i - a0, a.smem_elems, a.status)] = xc[i];
  }
  if (tid == 0) {
    int ok = 1;
    if (bulk_bytes) {
      ok = staging_wait(&bs.bar, 0, a.timeout_ns, !a.inject, a.status) ? 1 : 0;
    }
    bs.stage_ok = ok;
  }
  __syncthreads();
  if (!bs.stage_ok) return;
  if (bulk_bytes) (void)mbar_try_wait(&bs.bar, 0);
  const double* xsl = xs + (e0 - a0);  // xsl[local_row * KC + j]
  const int tpr = 1 << a.tpr_log2;
  const int sub = lane & (tpr - 1);
  const int rows_per_slice = 32 >> a.tpr_log2;

  int s = s0 + warp;
  while (s < s1) {
    double acc[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[j] = 0.0;
    const int64_t pos = a.slice_pos[s];
    const int w = (int)((a.slice_pos[s + 1] - pos) >> 5);
    const double* vp = ell_val + pos + lane;
    const uint16_t* cp = a.ell_col + pos + lane;
    for (int kk = 0; kk < w; ++kk) {
      const double v = __ldcs(vp + 32 * (int64_t)kk);
      const int c = checked((int)__ldcs(reinterpret_cast<const unsigned short*>(cp + 32 * (int64_t)kk)), pe - pb, a.status);
      const double* xr = xsl + c * KC;
#pragma unroll
      for (int j = 0; j < KC; ++j) acc[j] = fma(v, xr[j], acc[j]);
    }
    const int64_t epos = a.er_slice_pos[s];
    const int we = (int)((a.er_slice_pos[s + 1] - epos) >> 5);
    const double* evp = er_val + epos + lane;
    const int32_t* ecp = a.er_scol + epos + lane;
    for (int kk = 0; kk < we; ++kk) {
      const double v = __ldcs(evp + 32 * (int64_t)kk);
      const double* xr = xc + (int64_t)checked(__ldcs(ecp + 32 * (int64_t)kk), a.n, a.status) * KC;
#pragma unroll
      for (int j = 0; j < KC; ++j) acc[j] = fma(v, __ldg(xr + j), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < KC; ++j)
      for (int off = tpr >> 1; off > 0; off >>= 1) acc[j] += __shfl_xor_sync(FULL, acc[j], off);
    const int row = pb + (s - s0) * rows_per_slice + (lane >> a.tpr_log2);
    if (sub == 0 && row < pe) {
      double* yr = Y + (int64_t)checked(a.new_to_old[row], a.n, a.status) * k + c0;
#pragma unroll
      for (int j = 0; j < KC; ++j) yr[j] = acc[j];
    }
    int nxt = 0;
    if (lane == 0) nxt = atomicAdd(&bs.slice_counter, 1);
    s = __shfl_sync(FULL, nxt, 0);
  }
}

template <int KC>
cudaError_t launch_chunk(const DevPlan& D, const double* xc, double* Y, int k, int c0, size_t smem, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = cudaFuncSetAttribute(spmm_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  KArgs a = make_kargs(D);
  a.smem_elems = (int64_t)(smem / sizeof(double));
  spmm_kernel<KC><<<D.nparts, 512, smem, s>>>(a, D.ell_val, D.er_sval, xc, Y, k, c0);
  return cudaGetLastError();
}

}  // namespace
}  // namespace ehyb

using namespace ehyb;

extern "C" ehyb_status_t ehyb_spmm(ehyb_plan_t P, int32_t k, const double* X, double* Y, void* stream) {
  if (!P || k < 1) return EHYB_ERR_INVALID_ARG;
  if (P->host_only || P->er_layout != 0) return EHYB_ERR_UNSUPPORTED;
  const DevPlan& D = P->dev;
  if (D.n == 0) return EHYB_OK;
  if (!X || !Y || (const void*)X == (const void*)Y) return EHYB_ERR_INVALID_ARG;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_error_status(e, "device query");
  const size_t budget = (size_t)optin - 1024;
  int kc = 0;
  for (int c : {8, 4, 2, 1}) {
    const size_t need = ((size_t)(D.max_part_rows + 1) * c + 2) * 8;
    if (k % c == 0 && need <= budget) { kc = c; break; }
  }
  if (kc == 0) return EHYB_ERR_TOO_LARGE;
  const size_t need = ((((size_t)(D.max_part_rows + 1) * kc + 2) * 8) + 15) & ~(size_t)15;
  const size_t ws_bytes = (size_t)D.n * (size_t)k * 8;
  if (P->spmm_ws_bytes < ws_bytes) {
    if (P->spmm_ws) {
      e = cudaStreamSynchronize((cudaStream_t)stream);
      if (e != cudaSuccess) return cuda_error_status(e, "cudaStreamSynchronize");
      cudaFree(P->spmm_ws);
      P->spmm_ws = nullptr;
      P->spmm_ws_bytes = 0;
    }
    ehyb_status_t st = device_alloc(&P->spmm_ws, ws_bytes);
    if (st != EHYB_OK) return st;
    P->spmm_ws_bytes = ws_bytes;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* Xp = (double*)P->spmm_ws;
  const int64_t total = D.n * (int64_t)k;
  int blocks = (int)std::min<int64_t>(152 * 16, (total + 255) / 256);
  spmm_gather_kernel<<<blocks, 256, 0, s>>>(D.n, k, kc, D.new_to_old, X, Xp);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error_status(e, "spmm gather");
  for (int c = 0; c < k / kc; ++c) {
    const double* xc = Xp + (int64_t)c * D.n * kc;
    switch (kc) {
      case 8: e = launch_chunk<8>(D, xc, Y, k, c * kc, need, s); break;
      case 4: e = launch_chunk<4>(D, xc, Y, k, c * kc, need, s); break;
      case 2: e = launch_chunk<2>(D, xc, Y, k, c * kc, need, s); break;
      default: e = launch_chunk<1>(D, xc, Y, k, c * kc, need, s); break;
    }
    if (e != cudaSuccess) return cuda_error_status(e, "spmm launch");
  }
  return EHYB_OK;
}
