// ehyb_spmv_noalloc: the FP64 SpMV of ehyb_spmv for callers that must not allocate device memory
// at call time.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a plug-in living inside a host
// framework that has already reserved all device memory for its own pool allocator, a latency-
// critical service loop that may not pay for (or fail on) an allocation, or a host thread that
// holds a lock the allocator also needs.  ehyb_spmv itself does not allocate either, but it gathers
// x into workspace owned by the plan; this variant gathers into a fixed array that is part of the
// library image instead, so the only device memory it touches besides the plan is that array and
// the caller's x and y.
//
// The scratch array below holds the permuted copy of x (x_p[i] = x[new_to_old[i]]) for matrices of
// at most EHYB_NOALLOC_MAX_ROWS rows: 2^20 doubles = 8 MiB, held by every GPU that loads the library
// until the process exits.  All calls share it and it keeps the last call's contents; each call
// rewrites rows [0, n) before reading them, so nothing has to be cleared, but calls that overlap in
// time on the GPU (different streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ehyb.h"
#include "device.h"

#define EHYB_NOALLOC_MAX_ROWS (1 << 20)

static __device__ __align__(256) double g_noalloc_xp[EHYB_NOALLOC_MAX_ROWS];

namespace ehyb {
// defined in api.cpp: device view of a plan (nullptr for host-only plans)
const DevPlan* plan_device_view(ehyb_plan_t plan, int* device);
// records the CUDA error text for ehyb_last_cuda_error and returns EHYB_ERR_CUDA
ehyb_status_t cuda_error_status(cudaError_t e, const char* what);
}  // namespace ehyb

namespace {

// Device address of g_noalloc_xp, looked up once per device (the name itself is only a host-side
// stand-in in host code).  The lookup happens on the first call made with that device current and is
// kept for the life of the process (a cudaDeviceReset would invalidate it, as it frees every plan).
double* scratch_address(int dev, cudaError_t* err) {
  static std::mutex mu;
  static double* addr[128] = {nullptr};
  *err = cudaSuccess;
  if (dev < 0 || dev >= 128) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_xp);
    if (e != cudaSuccess) {
      *err = e;
      return nullptr;
    }
    addr[dev] = static_cast<double*>(p);
  }
  return addr[dev];
}

}  // namespace

extern "C" ehyb_status_t ehyb_spmv_noalloc(ehyb_plan_t plan, const double* x, double* y, void* stream) {
  if (!plan) return EHYB_ERR_INVALID_ARG;
  int plan_dev = -1;
  const ehyb::DevPlan* D = ehyb::plan_device_view(plan, &plan_dev);
  if (!D) return EHYB_ERR_UNSUPPORTED;  // host-only plan
  if (D->n > EHYB_NOALLOC_MAX_ROWS) return EHYB_ERR_TOO_LARGE;
  if (D->n == 0) return EHYB_OK;
  if (!x || !y || x == y) return EHYB_ERR_INVALID_ARG;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ehyb::cuda_error_status(e, "ehyb_spmv_noalloc: cudaGetDevice");
  if (dev != plan_dev) return EHYB_ERR_INVALID_ARG;  // the plan's arrays live on another device
  double* xp = scratch_address(dev, &e);
  if (!xp) return ehyb::cuda_error_status(e, "ehyb_spmv_noalloc: cudaGetSymbolAddress");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((e = ehyb::launch_permute_f64(*D, 1, x, xp, s)) != cudaSuccess)
    return ehyb::cuda_error_status(e, "ehyb_spmv_noalloc: permute launch");
  if ((e = ehyb::launch_ehyb_f64(*D, xp, y, 1, s)) != cudaSuccess)
    return ehyb::cuda_error_status(e, "ehyb_spmv_noalloc: product launch");
  return EHYB_OK;
}
