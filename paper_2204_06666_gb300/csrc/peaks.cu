// Throughput probe of the FP64 FMA pipe, the unit that bounds an FP64 SpMV on this part (one DFMA per
// stored entry against at least 10 bytes of HBM traffic).  The roofline of the FP64 kernels is taken
// against the rate this probe measures on the device at hand, not against a constant.
//
// Every thread runs kChains independent FMA chains a_i <- a_i * b + c (b, c run-time values, so nothing
// folds), `iters` steps each; the grid holds 4 blocks of 512 threads per SM, enough warps that each SM
// sub-partition always has an FMA ready whatever the pipe's latency.  The chains' sums are stored, so the
// work cannot be dropped.
#include <cuda_runtime.h>

#include "../../include/ehyb.h"

namespace ehyb {
ehyb_status_t cuda_error_status(cudaError_t e, const char* what);
}  // namespace ehyb

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, double b, double c, double* out) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" ehyb_status_t ehyb_fp64_fma_peak(int32_t iters, int32_t reps, double* tflops, double* ms_best) {
  if (iters <= 0 || reps <= 0 || !tflops) return EHYB_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return ehyb::cuda_error_status(e, "fp64 probe: device query");
  const int grid = sms * kBlocksPerSm;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0.f;
  e = cudaMalloc(&out, (size_t)grid * kThreads * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int r = -1; r < reps && e == cudaSuccess; ++r) {  // r = -1: untimed warm-up launch
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      fma_probe_kernel<<<grid, kThreads>>>(iters, 0.9999999, 1e-9, out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r >= 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return ehyb::cuda_error_status(e, "fp64 probe");
  const double fmas = (double)grid * kThreads * kChains * (double)iters;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  if (ms_best) *ms_best = best;
  return EHYB_OK;
}
