// Conjugate gradients on an EHYB plan (the solver whose SpMV cost motivates the method, Sec. 6), and
// FP64 iterative refinement around an inner CG whose matrix values are stored in FP32 or BF16.
//
// All vectors live in the plan's numbering (b and x are permuted once in and once out).  One CG
// iteration is three kernels:
//   K1  q = A p on the EHYB kernel, with p . q accumulated in its epilogue (p_r is already in shared
//       memory): one partial per partition, reduced into one scalar by the last block to finish;
//   K2  alpha = (r.r) / (p.q) (once per block); x += alpha p; r -= alpha q; partial sums of the new r.r;
//       the last block reduces them, stores r.r(new) in the history, computes beta = r.r(new) / r.r(old),
//       advances the device iteration counter and raises `done` at convergence or at the limit;
//   K3  p = r + beta p.
// alpha and beta never leave the device.  Every reduction runs in a fixed order, so a solve is bit-
// reproducible.  Once `done` is up the remaining kernels of a chunk return at once, so the iteration
// count is exact although the host looks at the flag only once per chunk.  A chunk of kChunk
// iterations is captured once into a CUDA graph and replayed.
//
// Refinement (refine = 1: FP32 values, 2: BF16 values): outer FP64 residual r = b - A x on the FP64
// plan, inner CG on the low-precision copy of the values with FP32 vectors, FP32 SpMV accumulation and
// FP64 dot products / alpha / beta, started from d = 0 on r / ||r||; x += ||r|| d in FP64.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan_internal.h"

namespace ehyb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kVB = 608;  // vector-kernel blocks (4 per SM; 8 per SM measured slower)
constexpr int kVT = 256;
constexpr int kChunk = 16;
constexpr double kFcgInnerRtol = 0.1;  // default inner tolerance of the flexible CG's preconditioning solve

}  // namespace

struct CgState {
  int32_t it, done, converged, arrive_dot;
  int32_t arrive_rr, max_iter, breakdown, pad;
  double tol2, pq, beta, grow_limit;
};

struct CgWork {
  int64_t n = 0;
  int32_t nparts = 0, hist_cap = 0;
  void* arena = nullptr;
  double *bp = nullptr, *xp = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *xs = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
  double *part_a = nullptr, *part_b = nullptr, *pq_part = nullptr, *hist = nullptr;
  CgState* st = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g64 = nullptr, g32 = nullptr;
  int g32_lowp = 0;
};

void cg_work_free(CgWork* w) {
  if (!w) return;
  if (w->g64) cudaGraphExecDestroy(w->g64);
  if (w->g32) cudaGraphExecDestroy(w->g32);
  if (w->cap) cudaStreamDestroy(w->cap);
  if (w->arena) cudaFree(w->arena);
  delete w;
}

namespace {

// warp-level fixed-order sum of count partials (lane-strided, then an xor tree); every lane gets it
__device__ __forceinline__ double warp_sum(const double* part, int count) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < count; i += 32) v += part[i];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

// fixed-order block sum; result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
  return s;
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// r = b - q, p = r; partials of r.r (part_a) and b.b (part_b)
__global__ void init64_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ q, double* r,
                              double* p, double* part_a, double* part_b) {
  double ra = 0.0, bb = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double bi = b[i], ri = bi - q[i];
    r[i] = ri;
    p[i] = ri;
    ra = fma(ri, ri, ra);
    bb = fma(bi, bi, bb);
  }
  const double s1 = block_sum(ra);
  __syncthreads();
  const double s2 = block_sum(bb);
  if (threadIdx.x == 0) { part_a[blockIdx.x] = s1; part_b[blockIdx.x] = s2; }
}

// inner start: r32 = scale * r64 (rounded to FP32), p32 = r32, d32 = 0; partials of r32.r32
__global__ void init32_kernel(int64_t n, const double* __restrict__ r64, double scale, float* r32, float* p32,
                              float* d32, double* part_a) {
  double ra = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const float ri = (float)(r64[i] * scale);
    r32[i] = ri;
    p32[i] = ri;
    d32[i] = 0.0f;
    ra = fma((double)ri, (double)ri, ra);
  }
  const double s = block_sum(ra);
  if (threadIdx.x == 0) part_a[blockIdx.x] = s;
}

// single block: hist[0] = r.r, convergence threshold, counters
__global__ void init_finish_kernel(const double* part_a, int na, const double* part_b, int nb, double rtol2,
                                   int relative_to_r0, int max_iter, double* hist, CgState* st) {
  if (threadIdx.x >= 32) return;
  const double rr = warp_sum(part_a, na);
  const double bb = part_b ? warp_sum(part_b, nb) : 0.0;
  if (threadIdx.x == 0) {
    hist[0] = rr;
    st->tol2 = rtol2 * (relative_to_r0 ? rr : bb);
    st->grow_limit = 1e12 * rr;
    st->it = 0;
    st->arrive_dot = 0;
    st->arrive_rr = 0;
    st->breakdown = 0;
    st->max_iter = max_iter;
    st->converged = rr <= st->tol2 ? 1 : 0;
    st->done = (st->converged || max_iter <= 0) ? 1 : 0;
  }
}

template <typename T> struct Vec16;
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <typename T> __device__ __forceinline__ T& lane_of(typename Vec16<T>::type& v, int i) {
  return reinterpret_cast<T*>(&v)[i];
}

// K2: alpha = hist[it] / (p.q); x += alpha p; r -= alpha q; r.r(new) by the last block, which also
// stores it, computes beta and advances the iteration.  16-byte vector accesses (the workspace vectors
// are 256-byte aligned), scalar tail.  p.q <= 0 means the operator is not positive definite along p:
// the iteration stops with `breakdown` set and nothing updated.
template <typename T>
__global__ void update_kernel(int64_t n, T* __restrict__ x, const T* __restrict__ p, const T* __restrict__ q,
                              T* __restrict__ r,
                              double* hist, CgState* st, double* rr_part) {
  if (st->done) return;
  using V = typename Vec16<T>::type;
  constexpr int NV = Vec16<T>::N;
  __shared__ double alpha_s;
  __shared__ int last_s;
  if (threadIdx.x == 0) alpha_s = st->pq > 0.0 ? hist[st->it] / st->pq : 0.0;
  __syncthreads();
  if (!(alpha_s > 0.0) && hist[st->it] > 0.0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->breakdown = 1;
      st->done = 1;
    }
    return;
  }
  const T a = (T)alpha_s;
  double acc = 0.0;
  const int64_t nv = n / NV;
  for (int64_t j = gtid(); j < nv; j += gstride()) {
    V xv = reinterpret_cast<V*>(x)[j];
    const V pv = reinterpret_cast<const V*>(p)[j];
    const V qv = reinterpret_cast<const V*>(q)[j];
    V rv = reinterpret_cast<V*>(r)[j];
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      V& xx = xv;
      lane_of<T>(xx, u) = fma(a, lane_of<T>(const_cast<V&>(pv), u), lane_of<T>(xx, u));
      const T ri = fma(-a, lane_of<T>(const_cast<V&>(qv), u), lane_of<T>(rv, u));
      lane_of<T>(rv, u) = ri;
      acc = fma((double)ri, (double)ri, acc);
    }
    reinterpret_cast<V*>(x)[j] = xv;
    reinterpret_cast<V*>(r)[j] = rv;
  }
  for (int64_t i = nv * NV + gtid(); i < n; i += gstride()) {
    x[i] = fma(a, p[i], x[i]);
    const T ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    acc = fma((double)ri, (double)ri, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) {
    rr_part[blockIdx.x] = s;
    __threadfence();
    last_s = atomicAdd(&st->arrive_rr, 1) == (int)gridDim.x - 1;  // every block has read st->it
  }
  __syncthreads();
  if (last_s && threadIdx.x < 32) {
    __threadfence();
    const double rrn = warp_sum(rr_part, (int)gridDim.x);
    if (threadIdx.x == 0) {
      const int k = st->it;
      hist[k + 1] = rrn;
      st->beta = rrn / hist[k];
      st->arrive_rr = 0;
      st->it = k + 1;
      if (rrn <= st->tol2) {
        st->converged = 1;
        st->done = 1;
      } else if (!(rrn <= st->grow_limit)) {  // non-finite or diverging: stop this inner iteration
        st->breakdown = 1;
        st->done = 1;
      } else if (k + 1 >= st->max_iter) {
        st->done = 1;
      }
    }
  }
}

// K3: p = r + beta p (force: run although `done` is up -- the residual-replacement driver completes the
// iteration whose update raised the flag)
template <typename T>
__global__ void pupdate_kernel(int64_t n, T* __restrict__ p, const T* __restrict__ r, const CgState* st,
                               int force = 0) {
  if (st->done && !force) return;
  if (st->breakdown) return;
  using V = typename Vec16<T>::type;
  constexpr int NV = Vec16<T>::N;
  const T b = (T)st->beta;
  const int64_t nv = n / NV;
  for (int64_t j = gtid(); j < nv; j += gstride()) {
    V pv = reinterpret_cast<V*>(p)[j];
    V rv = reinterpret_cast<const V*>(r)[j];
#pragma unroll
    for (int u = 0; u < NV; ++u) lane_of<T>(pv, u) = fma(b, lane_of<T>(pv, u), lane_of<T>(rv, u));
    reinterpret_cast<V*>(p)[j] = pv;
  }
  for (int64_t i = nv * NV + gtid(); i < n; i += gstride()) p[i] = fma(b, p[i], r[i]);
}

// r = b - q (FP64) with partials of r.r
__global__ void residual_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ q, double* r,
                                double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double ri = b[i] - q[i];
    if (r) r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// partials of a.b
__global__ void dot_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) acc = fma(a[i], b[i], acc);
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// x += scale * d (FP64 update of the refinement)
__global__ void correct_kernel(int64_t n, double* x, const float* __restrict__ d, double scale) {
  for (int64_t i = gtid(); i < n; i += gstride()) x[i] = fma(scale, (double)d[i], x[i]);
}

// residual replacement: p32 *= ratio; r32 = r64 * inv_scale (FP32); d32 = 0; partials of r32.r32
__global__ void replace_kernel(int64_t n, const double* __restrict__ r64, double inv_scale, float ratio, float* r32,
                               float* p32, float* d32, double* part_a) {
  double ra = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const float ri = (float)(r64[i] * inv_scale);
    r32[i] = ri;
    p32[i] *= ratio;
    d32[i] = 0.0f;
    ra = fma((double)ri, (double)ri, ra);
  }
  const double s = block_sum(ra);
  if (threadIdx.x == 0) part_a[blockIdx.x] = s;
}

// after a replacement: hist[it] = r32.r32, new trigger delta2 * r32.r32, iterations continue
__global__ void replace_finish_kernel(const double* part_a, int na, double delta2, double* hist, CgState* st) {
  if (threadIdx.x >= 32) return;
  const double rr = warp_sum(part_a, na);
  if (threadIdx.x == 0) {
    hist[st->it] = rr;
    st->tol2 = delta2 * rr;
    st->grow_limit = 1e12 * rr;
    st->arrive_dot = 0;
    st->arrive_rr = 0;
    st->converged = 0;
    st->breakdown = 0;
    st->done = st->it >= st->max_iter ? 1 : 0;
  }
}

// ---- flexible CG (Notay's FCG with one kept direction), FP64 outer, low-precision inner CG as the variable
// preconditioner z = B_k(r)

// z = r (use_r: the inner solve gave nothing) or z = scale * d (FP32 -> FP64); partials of z.q
__global__ void fcg_z_kernel(int64_t n, int use_r, const double* __restrict__ r, const float* __restrict__ d,
                             double scale, double* __restrict__ z, const double* __restrict__ q, double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double zi = use_r ? r[i] : scale * (double)d[i];
    z[i] = zi;
    acc = fma(zi, q[i], acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// p = z + beta p; partials of p.r
__global__ void fcg_dir_kernel(int64_t n, const double* __restrict__ z, double beta, double* __restrict__ p,
                               const double* __restrict__ r, double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double pi = fma(beta, p[i], z[i]);
    p[i] = pi;
    acc = fma(pi, r[i], acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// x += alpha p; r -= alpha q; partials of r.r
__global__ void fcg_update_kernel(int64_t n, double alpha, const double* __restrict__ p, const double* __restrict__ q,
                                  double* __restrict__ x, double* __restrict__ r, double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

#define CKC(call)                                                     \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_error_status(e_, #call);       \
  } while (0)

ehyb_status_t work_get(ehyb_plan_t P, int hist_need, CgWork** out) {
  CgWork* w = P->cg;
  const int64_t n = P->dev.n;
  if (w && w->hist_cap >= hist_need) {
    *out = w;
    return EHYB_OK;
  }
  if (w) {
    CKC(cudaDeviceSynchronize());
    cg_work_free(w);
    P->cg = nullptr;
  }
  w = new CgWork();
  w->n = n;
  w->nparts = P->dev.nparts;
  w->hist_cap = hist_need < 1024 ? 1024 : hist_need;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t v64 = al((size_t)(n + 2) * 8), v32 = al((size_t)(n + 4) * 4);
  const size_t parts = al((size_t)kVB * 8), pq = al((size_t)(w->nparts + 1) * 8);
  const size_t hist = al((size_t)(w->hist_cap + 2) * 8), st = al(sizeof(CgState));
  const size_t total = 6 * v64 + 4 * v32 + 2 * parts + pq + hist + st;
  ehyb_status_t s = device_alloc(&w->arena, total);
  if (s != EHYB_OK) {
    delete w;
    return s;
  }
  char* b = (char*)w->arena;
  w->bp = (double*)b; b += v64;
  w->xp = (double*)b; b += v64;
  w->r = (double*)b; b += v64;
  w->p = (double*)b; b += v64;
  w->q = (double*)b; b += v64;
  w->xs = (double*)b; b += v64;
  w->r32 = (float*)b; b += v32;
  w->p32 = (float*)b; b += v32;
  w->q32 = (float*)b; b += v32;
  w->d32 = (float*)b; b += v32;
  w->part_a = (double*)b; b += parts;
  w->part_b = (double*)b; b += parts;
  w->pq_part = (double*)b; b += pq;
  w->hist = (double*)b; b += hist;
  w->st = (CgState*)b;
  cudaError_t e = cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cg_work_free(w);
    return cuda_error_status(e, "cudaStreamCreateWithFlags");
  }
  P->cg = w;
  *out = w;
  return EHYB_OK;
}

// FP64 iterations (lowp == 0) or inner FP32-vector iterations (lowp = 1 / 2), kChunk of them
ehyb_status_t enqueue_chunk(ehyb_plan_t P, CgWork* w, int lowp, cudaStream_t s) {
  const DevPlan& D = P->dev;
  const int64_t n = D.n;
  for (int k = 0; k < kChunk; ++k) {
    DotOut dot{w->pq_part, &w->st->arrive_dot, &w->st->pq};
    if (lowp == 0) {
      CKC(launch_ehyb_f64(D, w->p, w->q, 0, s, &dot, &w->st->done));
      update_kernel<double><<<kVB, kVT, 0, s>>>(n, w->xp, w->p, w->q, w->r, w->hist, w->st, w->part_a);
      pupdate_kernel<double><<<kVB, kVT, 0, s>>>(n, w->p, w->r, w->st);
    } else {
      CKC(launch_ehyb_lowp(D, lowp, w->p32, w->q32, 0, s, &dot, &w->st->done));
      update_kernel<float><<<kVB, kVT, 0, s>>>(n, w->d32, w->p32, w->q32, w->r32, w->hist, w->st, w->part_a);
      pupdate_kernel<float><<<kVB, kVT, 0, s>>>(n, w->p32, w->r32, w->st);
    }
    CKC(cudaGetLastError());
  }
  return EHYB_OK;
}

// one chunk through the plan's cached CUDA graph (captured on first use)
ehyb_status_t run_chunk(ehyb_plan_t P, CgWork* w, int lowp, cudaStream_t s) {
  cudaGraphExec_t* g = lowp == 0 ? &w->g64 : &w->g32;
  if (lowp && w->g32 && w->g32_lowp != lowp) {
    cudaGraphExecDestroy(w->g32);
    w->g32 = nullptr;
  }
  if (!*g) {
    cudaGraph_t graph;
    CKC(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
    ehyb_status_t st = enqueue_chunk(P, w, lowp, w->cap);
    cudaError_t e = cudaStreamEndCapture(w->cap, &graph);
    if (st != EHYB_OK) return st;
    CKC(e);
    e = cudaGraphInstantiate(g, graph, 0);
    cudaGraphDestroy(graph);
    CKC(e);
    if (lowp) w->g32_lowp = lowp;
  }
  CKC(cudaGraphLaunch(*g, s));
  return EHYB_OK;
}

ehyb_status_t read_state(CgWork* w, cudaStream_t s, CgState* out) {
  CKC(cudaMemcpyAsync(out, w->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  CKC(cudaStreamSynchronize(s));
  return EHYB_OK;
}

ehyb_status_t sum_parts(CgWork* w, cudaStream_t s, double* out) {
  double h[kVB];
  CKC(cudaMemcpyAsync(h, w->part_a, sizeof(h), cudaMemcpyDeviceToHost, s));
  CKC(cudaStreamSynchronize(s));
  double t = 0.0;
  for (int i = 0; i < kVB; ++i) t += h[i];
  *out = t;
  return EHYB_OK;
}

ehyb_status_t cg_loop(ehyb_plan_t P, CgWork* w, int lowp, cudaStream_t s, int* iters, int* converged,
                      int* breakdown);

// Flexible CG (Notay, "Flexible conjugate gradients", SIAM J. Sci. Comput. 22, 2000; truncation to one
// direction) in FP64 on the plan's FP64 values, from the x_p, r of w (r = b - A x_p, ||r||^2 = rr): each
// step applies the variable preconditioner z = B_k(r) = ||r|| d, d from an inner CG on the low-precision
// values (FP32 vectors, stopped at inner_rtol or inner_max iterations), then
//   p = z + beta p with beta = -(z . q_prev) / (p_prev . q_prev) (A-orthogonal to the previous direction),
//   q = A p, alpha = (p . r) / (p . q), x += alpha p, r -= alpha q.
// The recursive residual decides; on its convergence the true FP64 residual is recomputed and, if it is
// still too large, the iteration restarts from it.  *iters counts inner iterations, *outer the steps.
ehyb_status_t fcg_solve(ehyb_plan_t P, CgWork* w, int lowp, cudaStream_t s, double bnorm, double rtol, int max_iter,
                        double inner_rtol, double& rr, int* iters, int* outer, int* converged, double* rel_out) {
  const DevPlan& D = P->dev;
  const int64_t n = D.n;
  const int inner_max = 500;
  double* z = w->xs;
  double pq_prev = 0.0;
  bool restart = true;
  ehyb_status_t st;
  int true_checks = 0;
  for (;;) {
    const double rel = std::sqrt(rr) / bnorm;
    *rel_out = rel;
    if (rel <= rtol || rr == 0.0) {
      // confirm on the true residual (the recursive one may have drifted)
      CKC(launch_ehyb_f64(D, w->xp, w->q, 0, s));
      residual_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, w->part_a);
      if ((st = sum_parts(w, s, &rr)) != EHYB_OK) return st;
      *rel_out = std::sqrt(rr) / bnorm;
      if (*rel_out <= rtol || rr == 0.0 || ++true_checks > 3) {
        *converged = *rel_out <= rtol || rr == 0.0;
        return EHYB_OK;
      }
      restart = true;  // continue from the true residual with a fresh direction
    }
    if (*iters >= max_iter || !std::isfinite(rr)) return EHYB_OK;
    // z = B(r): inner CG on the low-precision values, from 0, on r / ||r||
    const double rn = std::sqrt(rr);
    init32_kernel<<<kVB, kVT, 0, s>>>(n, w->r, 1.0 / rn, w->r32, w->p32, w->d32, w->part_a);
    const int cap = std::min(inner_max, max_iter - *iters);
    init_finish_kernel<<<1, 32, 0, s>>>(w->part_a, kVB, nullptr, 0, inner_rtol * inner_rtol, 1, cap, w->hist, w->st);
    CKC(cudaGetLastError());
    int it_in = 0, conv_in = 0, brk = 0;
    if ((st = cg_loop(P, w, lowp, s, &it_in, &conv_in, &brk)) != EHYB_OK) return st;
    *iters += it_in;
    // a first-iteration breakdown leaves d = 0: take the unpreconditioned step z = r
    fcg_z_kernel<<<kVB, kVT, 0, s>>>(n, it_in == 0 ? 1 : 0, w->r, w->d32, rn, z, w->q, w->part_a);
    double zq = 0.0;
    if ((st = sum_parts(w, s, &zq)) != EHYB_OK) return st;
    const double beta = (restart || !(pq_prev > 0.0)) ? 0.0 : -zq / pq_prev;
    fcg_dir_kernel<<<kVB, kVT, 0, s>>>(n, z, beta, w->p, w->r, w->part_a);
    double pr = 0.0;
    if ((st = sum_parts(w, s, &pr)) != EHYB_OK) return st;
    DotOut dot{w->pq_part, &w->st->arrive_dot, &w->st->pq};
    CKC(cudaMemsetAsync(&w->st->arrive_dot, 0, sizeof(int32_t), s));
    CKC(launch_ehyb_f64(D, w->p, w->q, 0, s, &dot));
    double pq = 0.0;
    CKC(cudaMemcpyAsync(&pq, &w->st->pq, sizeof(double), cudaMemcpyDeviceToHost, s));
    CKC(cudaStreamSynchronize(s));
    ++*outer;
    if (!(pq > 0.0)) return EHYB_OK;  // A is not positive definite along p: stop (not converged)
    if (!(pr > 0.0)) {                 // not a descent direction: restart from z = B(r) alone
      if (restart) return EHYB_OK;
      restart = true;
      continue;
    }
    fcg_update_kernel<<<kVB, kVT, 0, s>>>(n, pr / pq, w->p, w->q, w->xp, w->r, w->part_a);
    if ((st = sum_parts(w, s, &rr)) != EHYB_OK) return st;
    pq_prev = pq;
    restart = false;
  }
}

// CG loop on the vectors of w (FP64 or inner FP32); returns iterations and convergence
ehyb_status_t cg_loop(ehyb_plan_t P, CgWork* w, int lowp, cudaStream_t s, int* iters, int* converged,
                      int* breakdown) {
  CgState h;
  for (;;) {
    ehyb_status_t st = run_chunk(P, w, lowp, s);
    if (st != EHYB_OK) return st;
    if ((st = read_state(w, s, &h)) != EHYB_OK) return st;
    if (h.done) break;
  }
  *iters = h.it;
  *converged = h.converged;
  if (breakdown) *breakdown = h.breakdown;
  return EHYB_OK;
}

}  // namespace

}  // namespace ehyb

using namespace ehyb;

extern "C" ehyb_status_t ehyb_cg(ehyb_plan_t P, const double* b, double* x, double rtol, int32_t max_iter,
                                 int32_t refine, double inner_rtol, ehyb_cg_info_t* info, void* stream) {
  if (!P || !info) return EHYB_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  if (P->host_only) return EHYB_ERR_UNSUPPORTED;
  if (refine < 0 || refine > 6 || !(rtol >= 0.0) || max_iter < 0) return EHYB_ERR_INVALID_ARG;
  const int lowp = refine == 0 ? 0 : (refine % 2 == 1) ? 1 : 2;
  if (refine && P->lowp != lowp) return EHYB_ERR_UNSUPPORTED;  // the plan lacks that value copy
  if (P->er_layout == 1) return EHYB_ERR_UNSUPPORTED;            // the fused dot needs every row final after its slice
  const int64_t n = P->dev.n;
  const double t0 = now_s();
  if (n == 0) {
    info->converged = 1;
    return EHYB_OK;
  }
  if (!b || !x) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CgWork* w = nullptr;
  ehyb_status_t st = work_get(P, max_iter + 2, &w);
  if (st != EHYB_OK) return st;
  const DevPlan& D = P->dev;
  CKC(launch_permute_f64(D, 1, b, w->bp, s));
  CKC(launch_permute_f64(D, 1, x, w->xp, s));
  // ||b||
  dot_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->bp, w->part_a);
  double bb = 0.0;
  if ((st = sum_parts(w, s, &bb)) != EHYB_OK) return st;
  const double bnorm = bb > 0.0 ? std::sqrt(bb) : 1.0;

  int converged = 0, iters = 0, outer = 0;
  // a stalled BF16 refinement (refine 2 / 4) hands its x and FP64 residual (w->r, rr_stall) to the flexible CG
  bool stalled = false;
  double rr_stall = 0.0;
  if (refine >= 5) {
    CKC(launch_ehyb_f64(D, w->xp, w->q, 0, s));
    residual_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, w->part_a);
    double rr = 0.0;
    if ((st = sum_parts(w, s, &rr)) != EHYB_OK) return st;
    double rel = 0.0;
    const double irtol = inner_rtol > 0.0 ? inner_rtol : kFcgInnerRtol;
    if ((st = fcg_solve(P, w, lowp, s, bnorm, rtol, max_iter, irtol, rr, &iters, &outer, &converged, &rel)) != EHYB_OK)
      return st;
    info->relres_recursive = rel;
    info->flexible = 1;
  } else if (refine == 0) {
    CKC(launch_ehyb_f64(D, w->xp, w->q, 0, s));
    init64_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, w->p, w->part_a, w->part_b);
    init_finish_kernel<<<1, 32, 0, s>>>(w->part_a, kVB, w->part_b, kVB, rtol * rtol, 0, max_iter, w->hist, w->st);
    CKC(cudaGetLastError());
    if ((st = cg_loop(P, w, 0, s, &iters, &converged, nullptr)) != EHYB_OK) return st;
    double rr_last = 0.0;
    CKC(cudaMemcpyAsync(&rr_last, w->hist + iters, sizeof(double), cudaMemcpyDeviceToHost, s));
    CKC(cudaStreamSynchronize(s));
    info->relres_recursive = std::sqrt(rr_last) / bnorm;
  } else if (refine >= 3) {
    // residual replacement: low-precision CG iterations that keep their search direction; whenever the
    // low-precision residual has dropped by `delta`, x += s d in FP64, the residual is recomputed in FP64
    // and the iteration continues on it (p rescaled, not restarted)
    const double delta = inner_rtol > 0.0 ? inner_rtol : 0.1;
    CKC(launch_ehyb_f64(D, w->xp, w->q, 0, s));
    residual_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, w->part_a);
    double rr = 0.0;
    if ((st = sum_parts(w, s, &rr)) != EHYB_OK) return st;
    double scale = std::sqrt(rr);
    if (scale / bnorm <= rtol || rr == 0.0) {
      converged = 1;
    } else {
      init32_kernel<<<kVB, kVT, 0, s>>>(n, w->r, 1.0 / scale, w->r32, w->p32, w->d32, w->part_a);
      init_finish_kernel<<<1, 32, 0, s>>>(w->part_a, kVB, nullptr, 0, delta * delta, 1, max_iter, w->hist, w->st);
      CKC(cudaGetLastError());
      double prev_rr = rr;
      int rejections = 0;
      for (;;) {
        int it_in = 0, conv_in = 0, brk = 0;
        if ((st = cg_loop(P, w, lowp, s, &it_in, &conv_in, &brk)) != EHYB_OK) return st;
        iters = it_in;
        // the direction update of the iteration that raised the trigger was skipped with it
        if (conv_in) pupdate_kernel<float><<<kVB, kVT, 0, s>>>(n, w->p32, w->r32, w->st, 1);
        CKC(cudaMemcpyAsync(w->xs, w->xp, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        correct_kernel<<<kVB, kVT, 0, s>>>(n, w->xp, w->d32, scale);
        CKC(launch_ehyb_f64(D, w->xp, w->q, 0, s));
        residual_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, w->part_a);
        if ((st = sum_parts(w, s, &rr)) != EHYB_OK) return st;
        ++outer;
        bool rejected = false;
        if (!(rr < prev_rr)) {  // the correction did not help (or is not finite): undo it
          rejected = true;
          CKC(cudaMemcpyAsync(w->xp, w->xs, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
          CKC(launch_ehyb_f64(D, w->xp, w->q, 0, s));
          residual_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, w->part_a);
          if ((st = sum_parts(w, s, &rr)) != EHYB_OK) return st;
        }
        const double rel = std::sqrt(rr) / bnorm;
        info->relres_recursive = rel;
        if (rel <= rtol) { converged = 1; break; }
        rejections = rejected ? rejections + 1 : 0;
        if (rejections >= 3 && std::isfinite(rr) && rr > 0.0) {
          stalled = true;
          rr_stall = rr;
        }
        if (iters >= max_iter || rr == 0.0 || !std::isfinite(rr) || rejections >= 3) break;
        const double ns = std::sqrt(rr);
        if (brk || rejected) {
          // lost positive definiteness along p, or no progress: restart the direction from the residual
          init32_kernel<<<kVB, kVT, 0, s>>>(n, w->r, 1.0 / ns, w->r32, w->p32, w->d32, w->part_a);
        } else {
          replace_kernel<<<kVB, kVT, 0, s>>>(n, w->r, 1.0 / ns, (float)(scale / ns), w->r32, w->p32, w->d32,
                                             w->part_a);
        }
        replace_finish_kernel<<<1, 32, 0, s>>>(w->part_a, kVB, delta * delta, w->hist, w->st);
        CKC(cudaGetLastError());
        scale = ns;
        prev_rr = rr;
      }
    }
  } else {
    // FP64 residual outside, FP32-vector CG on the low-precision values inside
    const double irtol = inner_rtol > 0.0 ? inner_rtol : (refine == 1 ? 1e-4 : 1e-2);
    const int outer_max = 60;
    double prev = 0.0;
    for (;;) {
      CKC(launch_ehyb_f64(D, w->xp, w->q, 0, s));
      residual_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, w->part_a);
      double rr = 0.0;
      if ((st = sum_parts(w, s, &rr)) != EHYB_OK) return st;
      const double rel = std::sqrt(rr) / bnorm;
      info->relres_recursive = rel;
      if (rel <= rtol) { converged = 1; break; }
      if (iters < max_iter && std::isfinite(rr) && (outer >= outer_max || (outer > 0 && !(rel < prev)))) {
        stalled = true;
        rr_stall = rr;
      }
      if (outer >= outer_max || iters >= max_iter || (outer > 0 && !(rel < prev))) break;
      prev = rel;
      ++outer;
      const double rnorm = std::sqrt(rr);
      init32_kernel<<<kVB, kVT, 0, s>>>(n, w->r, 1.0 / rnorm, w->r32, w->p32, w->d32, w->part_a);
      init_finish_kernel<<<1, 32, 0, s>>>(w->part_a, kVB, nullptr, 0, irtol * irtol, 1, max_iter - iters, w->hist,
                                          w->st);
      CKC(cudaGetLastError());
      int it_in = 0, conv_in = 0;
      if ((st = cg_loop(P, w, lowp, s, &it_in, &conv_in, nullptr)) != EHYB_OK) return st;
      iters += it_in;
      correct_kernel<<<kVB, kVT, 0, s>>>(n, w->xp, w->d32, rnorm);
      CKC(cudaGetLastError());
    }
  }
  if (stalled && lowp == 2 && !converged && iters < max_iter) {
    // BF16 values and u_bf16 kappa(A) near or above 1: the refinement stalls; the flexible CG keeps the
    // BF16 solve as a preconditioner only and lets the FP64 outer iteration carry the accuracy
    double rel = 0.0;
    if ((st = fcg_solve(P, w, lowp, s, bnorm, rtol, max_iter, kFcgInnerRtol, rr_stall, &iters, &outer, &converged,
                        &rel)) != EHYB_OK)
      return st;
    info->relres_recursive = rel;
    info->flexible = 1;
  }
  // true residual in FP64, then x back to the original numbering
  CKC(launch_ehyb_f64(D, w->xp, w->q, 0, s));
  residual_kernel<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, nullptr, w->part_a);
  double rr = 0.0;
  if ((st = sum_parts(w, s, &rr)) != EHYB_OK) return st;
  CKC(launch_permute_f64(D, 0, w->xp, x, s));
  CKC(cudaStreamSynchronize(s));
  info->iterations = iters;
  info->refinements = outer;
  info->relres = std::sqrt(rr) / bnorm;
  info->converged = converged;
  info->seconds = now_s() - t0;
  int32_t dev_status = 0;
  CKC(cudaMemcpy(&dev_status, P->dev.status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (dev_status) return (ehyb_status_t)dev_status;
  return converged ? EHYB_OK : EHYB_ERR_NOT_CONVERGED;
}

extern "C" ehyb_status_t ehyb_cg_history(ehyb_plan_t P, double* hist, int32_t cap, int32_t* count) {
  if (!P || !count || (cap > 0 && !hist)) return EHYB_ERR_INVALID_ARG;
  *count = 0;
  if (!P->cg) return EHYB_OK;
  CgState h;
  CKC(cudaDeviceSynchronize());
  CKC(cudaMemcpy(&h, P->cg->st, sizeof(h), cudaMemcpyDeviceToHost));
  const int m = h.it + 1 < cap ? h.it + 1 : cap;
  if (m > 0) CKC(cudaMemcpy(hist, P->cg->hist, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost));
  *count = m;
  return EHYB_OK;
}
