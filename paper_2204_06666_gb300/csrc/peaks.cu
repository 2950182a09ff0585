// Throughput probe of the FP64 FMA pipe, the unit that bounds an FP64 SpMV on this part (one DFMA per
// stored entry against at least 10 bytes of HBM traffic).  The roofline of the FP64 kernels is taken
// against the rate this probe measures on the device at hand, not against a constant.
//
// Every thread runs C independent FMA chains acc_i <- u_i * w_i + acc_i (the accumulator as the addend, as
// in the SpMV; u_i, w_i run-time values in registers of their own, so nothing folds), `iters` steps each, on
// 4 blocks of 512 threads per SM.  The rate depends a little on how the chains' operands fall on the register
// file (measured on GB300 at 2.07 GHz: 1.82, 1.87 and 1.82 FMA/clk/SM for 2, 3 and 4 chains; 1.67 for the form
// a_i <- a_i * b + c); the probe runs C = 2, 3, 4 and reports the best.  The chains' sums are stored, so the
// work cannot be dropped.
#include <cuda_runtime.h>

#include "../../include/ehyb.h"

namespace ehyb {
ehyb_status_t cuda_error_status(cudaError_t e, const char* what);
}  // namespace ehyb

namespace {

constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;

template <int C>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, double b, double c, double* out) {
  double acc[C], u[C], w[C];
#pragma unroll
  for (int i = 0; i < C; ++i) {
    acc[i] = (double)(threadIdx.x + i) * 1e-3;
    u[i] = b + i * 1e-12;
    w[i] = c * (1.0 + i * 1e-6);
  }
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < C; ++i) acc[i] = fma(u[i], w[i], acc[i]);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < C; ++i) s += acc[i];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// best of `reps` timed launches (after one untimed) of the C-chain probe; FMAs per launch in *fmas
template <int C>
cudaError_t time_probe(int grid, int iters, int reps, double* out, cudaEvent_t e0, cudaEvent_t e1, float* best,
                       double* fmas) {
  cudaError_t e = cudaSuccess;
  *best = 0.f;
  const int it = iters * 4 / C;  // about the same FMAs per launch for every C
  for (int r = -1; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      fma_probe_kernel<C><<<grid, kThreads>>>(it, 0.9999999, 1e-9, out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r >= 0 && (*best == 0.f || ms < *best)) *best = ms;
  }
  *fmas = (double)grid * kThreads * C * (double)it;
  return e;
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
  e = cudaMalloc(&out, (size_t)grid * kThreads * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best_tf = 0.0, best_ms = 0.0;
  for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
    float ms = 0.f;
    double fmas = 0.0;
    e = v == 0 ? time_probe<2>(grid, iters, reps, out, e0, e1, &ms, &fmas)
        : v == 1 ? time_probe<3>(grid, iters, reps, out, e0, e1, &ms, &fmas)
                 : time_probe<4>(grid, iters, reps, out, e0, e1, &ms, &fmas);
    const double tf = ms > 0.f ? 2.0 * fmas / ((double)ms * 1e-3) / 1e12 : 0.0;
    if (e == cudaSuccess && tf > best_tf) {
      best_tf = tf;
      best_ms = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return ehyb::cuda_error_status(e, "fp64 probe");
  *tflops = best_tf;
  if (ms_best) *ms_best = best_ms;
  return EHYB_OK;
}
