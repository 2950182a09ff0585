// Preconditioned conjugate gradients on an EHYB plan with the FSAI preconditioner M^-1 = G^T G (fsai.cpp):
// the solver the paper's Sec. 6 motivates, its preconditioner applied as two further EHYB products.
//
// All vectors live in the matrix plan's numbering (b and x are permuted once in and once out).  One
// iteration is four launches:
//   K1  q = A p on the matrix plan, p . q fused into its epilogue (last block reduces);
//   K2  alpha = (r.z) / (p.q); x += alpha p; r -= alpha q (FP32 copy of r when G is applied in FP32);
//       partials of r.r, the last block stores r.r, keeps r.z as (r.z)_old, advances the iteration and
//       raises `done` at convergence (||r|| <= rtol ||b||), at the iteration limit, or when p.q <= 0;
//   K3  t = G r on G's plan (the caller's numbering of that plan is the matrix plan's), t . t fused:
//       t . t = r . G^T G r = r . z, the new preconditioned inner product;
//   K4  z = G^T t on G^T's plan;
//   K5  p = z + beta p with beta = (r.z)_new / (r.z)_old (a coalesced pass: fusing it into K4's scattered
//       stores measured slower).
// alpha, beta and the inner products never leave the device; every reduction has a fixed order, so a
// solve is bit-reproducible.  Chunks of kChunk iterations are captured once into a CUDA graph and
// replayed; once `done` is up the remaining launches of a chunk return at once.
//
// Mixed precision (ehyb_pcg_refined): one PCG that runs on FP32 vectors -- A's FP32 / BF16 values, G's
// FP32 / BF16 values, FP32 accumulation, FP64 inner products and alpha / beta -- with FP64 residual
// replacement: the iteration works on d (A d = r / s for the residual r and scale s of the last
// replacement); whenever its residual has dropped by the factor delta, x += s d in FP64, r = b - A x is
// recomputed in FP64, the FP32 residual restarts from r / s' and the direction is kept, rescaled by s / s'
// (and (r.z)_old by (s / s')^2), so the Krylov iteration is not restarted.  Stops when ||b - A x|| <= rtol ||b||.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>

#include "plan_internal.h"

namespace ehyb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kVB = 608;  // vector-kernel blocks (4 per SM; 8 per SM measured slower)
constexpr int kVT = 256;
constexpr int kChunk = 16;

}  // namespace

struct PcgState {
  int32_t it, done, converged, breakdown;
  int32_t arrive_pq, arrive_rz, arrive_rr, pad0;
  int32_t max_iter, pad[3];
  double tol2, pq, rz_old, rz_new;
};

struct PcgWork {
  int64_t n = 0;
  int32_t hist_cap = 0, lowp = 0;
  void* arena = nullptr;
  double *bp = nullptr, *xp = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *t = nullptr;
  float *r32 = nullptr, *t32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
  double *part = nullptr, *pq_part = nullptr, *rz_part = nullptr, *hist = nullptr;
  PcgState* st = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr, graph32 = nullptr;
};

void pcg_work_free(PcgWork* w) {
  if (!w) return;
  if (w->graph) cudaGraphExecDestroy(w->graph);
  if (w->graph32) cudaGraphExecDestroy(w->graph32);
  if (w->cap) cudaStreamDestroy(w->cap);
  if (w->arena) cudaFree(w->arena);
  delete w;
}

namespace {

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

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

// fixed-order sum of count partials by one warp (lane-strided, then an xor tree); every lane gets it
__device__ __forceinline__ double warp_sum(const double* part, int count) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < count; i += 32) v += part[i];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

// r = b - q (and its FP32 copy); partials of r.r
__global__ void pcg_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ q, double* r,
                             float* r32, double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double ri = b[i] - q[i];
    r[i] = ri;
    if (r32) r32[i] = (float)ri;
    acc = fma(ri, ri, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// partials of a.a
__global__ void pcg_norm2(int64_t n, const double* __restrict__ a, double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) acc = fma(a[i], a[i], acc);
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// single block: hist[0] = r.r, stopping threshold, counters
__global__ void pcg_init_finish(const double* part, int np, double tol2, int max_iter, double* hist, PcgState* st) {
  if (threadIdx.x >= 32) return;
  const double rr = warp_sum(part, np);
  if (threadIdx.x == 0) {
    hist[0] = rr;
    st->tol2 = tol2;
    st->it = 0;
    st->arrive_pq = st->arrive_rz = st->arrive_rr = 0;
    st->breakdown = 0;
    st->max_iter = max_iter;
    st->converged = rr <= tol2 ? 1 : 0;
    st->done = (st->converged || max_iter <= 0) ? 1 : 0;
  }
}

// p = z (from FP64 z or FP32 z32)
template <typename Z>
__global__ void pcg_start(int64_t n, const Z* __restrict__ z, double* p) {
  for (int64_t i = gtid(); i < n; i += gstride()) p[i] = (double)z[i];
}

// K2 (16-byte accesses; the workspace vectors are 256-byte aligned)
__global__ void pcg_update(int64_t n, double* __restrict__ x, const double* __restrict__ p,
                           const double* __restrict__ q, double* __restrict__ r, float* __restrict__ r32, double* hist,
                           PcgState* st, double* part) {
  if (st->done) return;
  __shared__ int last_s;
  const double pq = st->pq;
  if (!(pq > 0.0)) {  // A is not positive definite along p (or p vanished): stop
    if (gtid() == 0) {
      st->breakdown = 1;
      st->done = 1;
    }
    return;
  }
  const double a = st->rz_new / pq;
  double acc = 0.0;
  const int64_t n2 = n >> 1;
  for (int64_t j = gtid(); j < n2; j += gstride()) {
    double2 xv = reinterpret_cast<double2*>(x)[j];
    const double2 pv = reinterpret_cast<const double2*>(p)[j];
    const double2 qv = reinterpret_cast<const double2*>(q)[j];
    double2 rv = reinterpret_cast<double2*>(r)[j];
    xv.x = fma(a, pv.x, xv.x);
    xv.y = fma(a, pv.y, xv.y);
    rv.x = fma(-a, qv.x, rv.x);
    rv.y = fma(-a, qv.y, rv.y);
    reinterpret_cast<double2*>(x)[j] = xv;
    reinterpret_cast<double2*>(r)[j] = rv;
    if (r32) reinterpret_cast<float2*>(r32)[j] = make_float2((float)rv.x, (float)rv.y);
    acc = fma(rv.x, rv.x, acc);
    acc = fma(rv.y, rv.y, acc);
  }
  for (int64_t i = 2 * n2 + gtid(); i < n; i += gstride()) {
    x[i] = fma(a, p[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    if (r32) r32[i] = (float)ri;
    acc = fma(ri, ri, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    last_s = atomicAdd(&st->arrive_rr, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (last_s && threadIdx.x < 32) {
    __threadfence();
    const double rr = warp_sum(part, (int)gridDim.x);
    if (threadIdx.x == 0) {
      const int k = st->it + 1;
      hist[k] = rr;
      st->it = k;
      st->arrive_rr = 0;
      st->rz_old = st->rz_new;  // every block has read it; K3 overwrites rz_new next
      if (rr <= st->tol2) {
        st->converged = 1;
        st->done = 1;
      } else if (!(rr < 1e300) || k >= st->max_iter) {
        st->done = 1;
      }
    }
  }
}

// K5: p = z + beta p (16-byte accesses)
template <typename Z>
__global__ void pcg_pupdate(int64_t n, const Z* __restrict__ z, double* __restrict__ p, const PcgState* st) {
  if (st->done) return;
  const double beta = st->rz_new / st->rz_old;
  const int64_t n2 = n >> 1;
  for (int64_t j = gtid(); j < n2; j += gstride()) {
    double2 pv = reinterpret_cast<double2*>(p)[j];
    double zx, zy;
    if (sizeof(Z) == 8) {
      const double2 zv = reinterpret_cast<const double2*>(z)[j];
      zx = zv.x;
      zy = zv.y;
    } else {
      const float2 zv = reinterpret_cast<const float2*>(z)[j];
      zx = zv.x;
      zy = zv.y;
    }
    pv.x = fma(beta, pv.x, zx);
    pv.y = fma(beta, pv.y, zy);
    reinterpret_cast<double2*>(p)[j] = pv;
  }
  for (int64_t i = 2 * n2 + gtid(); i < n; i += gstride()) p[i] = fma(beta, p[i], (double)z[i]);
}

// inner start: r32 = r * inv_scale (FP32), d32 = 0; partials of r32.r32
__global__ void pcg_inner_start(int64_t n, const double* __restrict__ r, double inv_scale, float* __restrict__ r32,
                                float* __restrict__ d32, double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const float ri = (float)(r[i] * inv_scale);
    r32[i] = ri;
    d32[i] = 0.0f;
    acc = fma((double)ri, (double)ri, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// inner K2: d += alpha p; r -= alpha q on FP32 vectors (alpha from FP64 inner products)
__global__ void pcg_update32(int64_t n, float* __restrict__ d, const float* __restrict__ p,
                             const float* __restrict__ q, float* __restrict__ r, double* hist, PcgState* st,
                             double* part) {
  if (st->done) return;
  __shared__ int last_s;
  const double pq = st->pq;
  if (!(pq > 0.0)) {
    if (gtid() == 0) {
      st->breakdown = 1;
      st->done = 1;
    }
    return;
  }
  const float a = (float)(st->rz_new / pq);
  double acc = 0.0;
  const int64_t n4 = n >> 2;
  for (int64_t j = gtid(); j < n4; j += gstride()) {
    float4 dv = reinterpret_cast<float4*>(d)[j];
    const float4 pv = reinterpret_cast<const float4*>(p)[j];
    const float4 qv = reinterpret_cast<const float4*>(q)[j];
    float4 rv = reinterpret_cast<float4*>(r)[j];
    dv.x = fmaf(a, pv.x, dv.x);
    dv.y = fmaf(a, pv.y, dv.y);
    dv.z = fmaf(a, pv.z, dv.z);
    dv.w = fmaf(a, pv.w, dv.w);
    rv.x = fmaf(-a, qv.x, rv.x);
    rv.y = fmaf(-a, qv.y, rv.y);
    rv.z = fmaf(-a, qv.z, rv.z);
    rv.w = fmaf(-a, qv.w, rv.w);
    reinterpret_cast<float4*>(d)[j] = dv;
    reinterpret_cast<float4*>(r)[j] = rv;
    acc = fma((double)rv.x, (double)rv.x, acc);
    acc = fma((double)rv.y, (double)rv.y, acc);
    acc = fma((double)rv.z, (double)rv.z, acc);
    acc = fma((double)rv.w, (double)rv.w, acc);
  }
  for (int64_t i = 4 * n4 + gtid(); i < n; i += gstride()) {
    d[i] = fmaf(a, p[i], d[i]);
    const float ri = fmaf(-a, q[i], r[i]);
    r[i] = ri;
    acc = fma((double)ri, (double)ri, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    last_s = atomicAdd(&st->arrive_rr, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (last_s && threadIdx.x < 32) {
    __threadfence();
    const double rr = warp_sum(part, (int)gridDim.x);
    if (threadIdx.x == 0) {
      const int k = st->it + 1;
      hist[k] = rr;
      st->it = k;
      st->arrive_rr = 0;
      st->rz_old = st->rz_new;
      if (rr <= st->tol2) {
        st->converged = 1;
        st->done = 1;
      } else if (!(rr < 1e30) || k >= st->max_iter) {
        st->done = 1;
      }
    }
  }
}

// inner K5: p = z + beta p (FP32)
__global__ void pcg_pupdate32(int64_t n, const float* __restrict__ z, float* __restrict__ p, const PcgState* st) {
  if (st->done) return;
  const float beta = (float)(st->rz_new / st->rz_old);
  const int64_t n4 = n >> 2;
  for (int64_t j = gtid(); j < n4; j += gstride()) {
    float4 pv = reinterpret_cast<float4*>(p)[j];
    const float4 zv = reinterpret_cast<const float4*>(z)[j];
    pv.x = fmaf(beta, pv.x, zv.x);
    pv.y = fmaf(beta, pv.y, zv.y);
    pv.z = fmaf(beta, pv.z, zv.z);
    pv.w = fmaf(beta, pv.w, zv.w);
    reinterpret_cast<float4*>(p)[j] = pv;
  }
  for (int64_t i = 4 * n4 + gtid(); i < n; i += gstride()) p[i] = fmaf(beta, p[i], z[i]);
}

// x += scale * d (the FP64 correction of an outer refinement step)
__global__ void pcg_correct(int64_t n, double* __restrict__ x, const float* __restrict__ d, double scale) {
  for (int64_t i = gtid(); i < n; i += gstride()) x[i] = fma(scale, (double)d[i], x[i]);
}

__global__ void copy_f32(int64_t n, const float* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = gtid(); i < n; i += gstride()) b[i] = a[i];
}

// residual replacement: r32 = r * inv_scale, d32 = 0, p32 *= ratio; partials of r32.r32
__global__ void pcg_replace(int64_t n, const double* __restrict__ r, double inv_scale, float ratio,
                            float* __restrict__ r32, float* __restrict__ d32, float* __restrict__ p32, double* part) {
  double acc = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const float ri = (float)(r[i] * inv_scale);
    r32[i] = ri;
    d32[i] = 0.0f;
    p32[i] *= ratio;
    acc = fma((double)ri, (double)ri, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// single block after a replacement: the next segment's threshold and counters; (r.z)_old in the new scale
__global__ void pcg_replace_finish(const double* part, int np, double delta2, double ratio2, int max_iter,
                                   double* hist, PcgState* st) {
  if (threadIdx.x >= 32) return;
  const double rr = warp_sum(part, np);
  if (threadIdx.x == 0) {
    hist[0] = rr;
    st->tol2 = delta2 * rr;
    st->it = 0;
    st->arrive_pq = st->arrive_rz = st->arrive_rr = 0;
    st->breakdown = 0;
    st->max_iter = max_iter;
    st->converged = 0;
    st->done = max_iter <= 0 ? 1 : 0;
    st->rz_old *= ratio2;
  }
}

// p32 = z32 + beta p32 once, regardless of `done` (completes the iteration a replacement interrupted)
__global__ void pcg_pupdate32_force(int64_t n, const float* __restrict__ z, float* __restrict__ p,
                                    const PcgState* st) {
  const float beta = (float)(st->rz_new / st->rz_old);
  for (int64_t i = gtid(); i < n; i += gstride()) p[i] = fmaf(beta, p[i], z[i]);
}

#define CKP(call)                                                     \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_error_status(e_, #call);       \
  } while (0)

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

ehyb_status_t work_get(ehyb_precond_t M, int hist_need, PcgWork** out) {
  PcgWork* w = M->work;
  if (w && w->hist_cap >= hist_need) {
    *out = w;
    return EHYB_OK;
  }
  if (w) {
    CKP(cudaDeviceSynchronize());
    pcg_work_free(w);
    M->work = nullptr;
  }
  const int64_t n = M->n;
  w = new PcgWork();
  w->n = n;
  w->lowp = M->lowp;
  w->hist_cap = hist_need < 1024 ? 1024 : hist_need;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const int nparts = M->plan->dev.nparts;
  const size_t v64 = al((size_t)(n + 2) * 8), v32 = al((size_t)(n + 4) * 4);
  const size_t parts = al((size_t)kVB * 8), pp = al((size_t)(nparts + 1) * 8);
  const size_t hist = al((size_t)(w->hist_cap + 2) * 8), st = al(sizeof(PcgState));
  const size_t total = 7 * v64 + 6 * v32 + parts + 2 * pp + hist + st;
  ehyb_status_t s = device_alloc(&w->arena, total);
  if (s != EHYB_OK) {
    delete w;
    return s;
  }
  char* b = (char*)w->arena;
  double** v[] = {&w->bp, &w->xp, &w->r, &w->p, &w->q, &w->z, &w->t};
  for (double** d : v) { *d = (double*)b; b += v64; }
  float** f[] = {&w->r32, &w->t32, &w->z32, &w->p32, &w->q32, &w->d32};
  for (float** d : f) { *d = (float*)b; b += v32; }
  w->part = (double*)b; b += parts;
  w->pq_part = (double*)b; b += pp;
  w->rz_part = (double*)b; b += pp;
  w->hist = (double*)b; b += hist;
  w->st = (PcgState*)b;
  cudaError_t e = cudaMemsetAsync(w->arena, 0, total, 0);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    pcg_work_free(w);
    return cuda_error_status(e, "pcg workspace");
  }
  M->work = w;
  *out = w;
  return EHYB_OK;
}

// t = G r with t.t -> rz_new, then z = G^T t (FP64, or, for an FP32 / BF16 G, on the FP32 copies)
ehyb_status_t apply_precond(ehyb_precond_t M, PcgWork* w, cudaStream_t s, const int32_t* skip) {
  DotOut dot{w->rz_part, &w->st->arrive_rz, &w->st->rz_new, 1};
  if (M->lowp == 0) {
    CKP(launch_ehyb_f64(M->g->dev, w->r, w->t, 2, s, &dot, skip));
    CKP(launch_ehyb_f64(M->gt->dev, w->t, w->z, 2, s, nullptr, skip));
  } else {
    CKP(launch_ehyb_lowp(M->g->dev, M->lowp, w->r32, w->t32, 2, s, &dot, skip));
    CKP(launch_ehyb_lowp(M->gt->dev, M->lowp, w->t32, w->z32, 2, s, nullptr, skip));
  }
  return EHYB_OK;
}

ehyb_status_t enqueue_chunk(ehyb_precond_t M, PcgWork* w, cudaStream_t s) {
  const DevPlan& D = M->plan->dev;
  const int64_t n = w->n;
  float* r32 = M->lowp ? w->r32 : nullptr;
  for (int k = 0; k < kChunk; ++k) {
    DotOut dot{w->pq_part, &w->st->arrive_pq, &w->st->pq};
    CKP(launch_ehyb_f64(D, w->p, w->q, 0, s, &dot, &w->st->done));
    pcg_update<<<kVB, kVT, 0, s>>>(n, w->xp, w->p, w->q, w->r, r32, w->hist, w->st, w->part);
    ehyb_status_t st = apply_precond(M, w, s, &w->st->done);
    if (st != EHYB_OK) return st;
    if (M->lowp == 0) pcg_pupdate<double><<<kVB, kVT, 0, s>>>(n, w->z, w->p, w->st);
    else pcg_pupdate<float><<<kVB, kVT, 0, s>>>(n, w->z32, w->p, w->st);
    CKP(cudaGetLastError());
  }
  return EHYB_OK;
}

// inner FP32 iterations: A's low-precision values, G's low-precision values, FP32 vectors
ehyb_status_t enqueue_chunk32(ehyb_precond_t M, PcgWork* w, cudaStream_t s) {
  const DevPlan& D = M->plan->dev;
  const int64_t n = w->n;
  for (int k = 0; k < kChunk; ++k) {
    DotOut dot{w->pq_part, &w->st->arrive_pq, &w->st->pq};
    CKP(launch_ehyb_lowp(D, M->plan->lowp, w->p32, w->q32, 0, s, &dot, &w->st->done));
    pcg_update32<<<kVB, kVT, 0, s>>>(n, w->d32, w->p32, w->q32, w->r32, w->hist, w->st, w->part);
    ehyb_status_t st = apply_precond(M, w, s, &w->st->done);
    if (st != EHYB_OK) return st;
    pcg_pupdate32<<<kVB, kVT, 0, s>>>(n, w->z32, w->p32, w->st);
    CKP(cudaGetLastError());
  }
  return EHYB_OK;
}

ehyb_status_t run_chunk(ehyb_precond_t M, PcgWork* w, cudaStream_t s, bool inner32 = false) {
  cudaGraphExec_t* g = inner32 ? &w->graph32 : &w->graph;
  if (!*g) {
    cudaGraph_t graph;
    CKP(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
    ehyb_status_t st = inner32 ? enqueue_chunk32(M, w, w->cap) : enqueue_chunk(M, w, w->cap);
    cudaError_t e = cudaStreamEndCapture(w->cap, &graph);
    if (st != EHYB_OK) return st;
    CKP(e);
    e = cudaGraphInstantiate(g, graph, 0);
    cudaGraphDestroy(graph);
    CKP(e);
  }
  CKP(cudaGraphLaunch(*g, s));
  return EHYB_OK;
}

ehyb_status_t sum_part(PcgWork* w, cudaStream_t s, double* out) {
  double h[kVB];
  CKP(cudaMemcpyAsync(h, w->part, sizeof(h), cudaMemcpyDeviceToHost, s));
  CKP(cudaStreamSynchronize(s));
  double t = 0.0;
  for (int i = 0; i < kVB; ++i) t += h[i];
  *out = t;
  return EHYB_OK;
}

}  // namespace
}  // namespace ehyb

using namespace ehyb;

extern "C" ehyb_status_t ehyb_pcg(ehyb_plan_t P, ehyb_precond_t M, const double* b, double* x, double rtol,
                                  int32_t max_iter, ehyb_cg_info_t* info, void* stream) {
  if (!P || !M || !info) return EHYB_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  if (M->plan != P) return EHYB_ERR_INVALID_ARG;  // the preconditioner belongs to another plan
  if (P->host_only) return EHYB_ERR_UNSUPPORTED;
  if (!(rtol >= 0.0) || max_iter < 0) return EHYB_ERR_INVALID_ARG;
  const int64_t n = P->dev.n;
  const double t0 = now_s();
  if (n == 0) {
    info->converged = 1;
    return EHYB_OK;
  }
  if (!b || !x) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PcgWork* w = nullptr;
  ehyb_status_t st = work_get(M, max_iter + 2, &w);
  if (st != EHYB_OK) return st;
  const DevPlan& D = P->dev;
  float* r32 = M->lowp ? w->r32 : nullptr;
  CKP(launch_permute_f64(D, 1, b, w->bp, s));
  CKP(launch_permute_f64(D, 1, x, w->xp, s));
  pcg_norm2<<<kVB, kVT, 0, s>>>(n, w->bp, w->part);
  double bb = 0.0;
  if ((st = sum_part(w, s, &bb)) != EHYB_OK) return st;
  const double bnorm = bb > 0.0 ? std::sqrt(bb) : 1.0;

  // r = b - A x, z = G^T G r, p = z
  CKP(launch_ehyb_f64(D, w->xp, w->q, 0, s));
  pcg_residual<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, r32, w->part);
  pcg_init_finish<<<1, 32, 0, s>>>(w->part, kVB, rtol * rtol * bnorm * bnorm, max_iter, w->hist, w->st);
  CKP(cudaGetLastError());
  if ((st = apply_precond(M, w, s, nullptr)) != EHYB_OK) return st;
  if (M->lowp == 0) pcg_start<double><<<kVB, kVT, 0, s>>>(n, w->z, w->p);
  else pcg_start<float><<<kVB, kVT, 0, s>>>(n, w->z32, w->p);
  CKP(cudaGetLastError());

  PcgState h;
  for (;;) {
    CKP(cudaMemcpyAsync(&h, w->st, sizeof(h), cudaMemcpyDeviceToHost, s));
    CKP(cudaStreamSynchronize(s));
    if (h.done) break;
    if ((st = run_chunk(M, w, s)) != EHYB_OK) return st;
  }
  // the true residual of the returned x, in FP64
  CKP(launch_ehyb_f64(D, w->xp, w->q, 0, s));
  pcg_residual<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->t, nullptr, w->part);
  double rr = 0.0;
  if ((st = sum_part(w, s, &rr)) != EHYB_OK) return st;
  double rr_rec = 0.0;
  CKP(cudaMemcpyAsync(&rr_rec, w->hist + h.it, sizeof(double), cudaMemcpyDeviceToHost, s));
  CKP(launch_permute_f64(D, 0, w->xp, x, s));
  CKP(cudaStreamSynchronize(s));
  info->iterations = h.it;
  info->converged = h.converged;
  info->relres = std::sqrt(rr) / bnorm;
  info->relres_recursive = std::sqrt(rr_rec) / bnorm;
  info->seconds = now_s() - t0;
  if (h.breakdown) return EHYB_ERR_NOT_CONVERGED;
  return h.converged ? EHYB_OK : EHYB_ERR_NOT_CONVERGED;
}

extern "C" ehyb_status_t ehyb_pcg_history(ehyb_precond_t M, double* rr, int32_t count, int32_t* n_out) {
  if (!M || !n_out || (count > 0 && !rr)) return EHYB_ERR_INVALID_ARG;
  *n_out = 0;
  PcgWork* w = M->work;
  if (!w) return EHYB_OK;
  PcgState h;
  CKP(cudaDeviceSynchronize());
  CKP(cudaMemcpy(&h, w->st, sizeof(h), cudaMemcpyDeviceToHost));
  const int32_t have = h.it + 1;
  const int32_t k = count < have ? count : have;
  if (k > 0) CKP(cudaMemcpy(rr, w->hist, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost));
  *n_out = k;
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_pcg_refined(ehyb_plan_t P, ehyb_precond_t M, const double* b, double* x, double rtol,
                                          int32_t max_iter, double inner_rtol, ehyb_cg_info_t* info, void* stream) {
  if (!P || !M || !info) return EHYB_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  if (M->plan != P) return EHYB_ERR_INVALID_ARG;
  if (P->host_only) return EHYB_ERR_UNSUPPORTED;
  if (P->lowp == 0 || M->lowp == 0) return EHYB_ERR_UNSUPPORTED;  // needs A's and G's low-precision values
  if (!(rtol >= 0.0) || max_iter < 0 || !(inner_rtol >= 0.0) || inner_rtol >= 1.0) return EHYB_ERR_INVALID_ARG;
  const double delta = inner_rtol > 0.0 ? inner_rtol : 0.01;
  const int64_t n = P->dev.n;
  const double t0 = now_s();
  if (n == 0) {
    info->converged = 1;
    return EHYB_OK;
  }
  if (!b || !x) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PcgWork* w = nullptr;
  ehyb_status_t st = work_get(M, max_iter + 2, &w);
  if (st != EHYB_OK) return st;
  const DevPlan& D = P->dev;
  CKP(launch_permute_f64(D, 1, b, w->bp, s));
  CKP(launch_permute_f64(D, 1, x, w->xp, s));
  pcg_norm2<<<kVB, kVT, 0, s>>>(n, w->bp, w->part);
  double bb = 0.0;
  if ((st = sum_part(w, s, &bb)) != EHYB_OK) return st;
  const double bnorm = bb > 0.0 ? std::sqrt(bb) : 1.0;

  // FP64 residual of x0; the first segment starts like a plain PCG on r / ||r||
  CKP(launch_ehyb_f64(D, w->xp, w->q, 0, s));
  pcg_residual<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, nullptr, w->part);
  double rr = 0.0;
  if ((st = sum_part(w, s, &rr)) != EHYB_OK) return st;
  int iters = 0, outer = 0, converged = std::sqrt(rr) <= rtol * bnorm ? 1 : 0;
  double scale = std::sqrt(rr), best_rr = rr;
  int stalls = 0;
  if (!converged && rr > 0.0) {
    pcg_inner_start<<<kVB, kVT, 0, s>>>(n, w->r, 1.0 / scale, w->r32, w->d32, w->part);
    pcg_init_finish<<<1, 32, 0, s>>>(w->part, kVB, delta * delta, max_iter, w->hist, w->st);
    CKP(cudaGetLastError());
    if ((st = apply_precond(M, w, s, nullptr)) != EHYB_OK) return st;
    copy_f32<<<kVB, kVT, 0, s>>>(n, w->z32, w->p32);
    CKP(cudaGetLastError());
    for (;;) {
      PcgState h;
      for (;;) {
        CKP(cudaMemcpyAsync(&h, w->st, sizeof(h), cudaMemcpyDeviceToHost, s));
        CKP(cudaStreamSynchronize(s));
        if (h.done) break;
        if ((st = run_chunk(M, w, s, true)) != EHYB_OK) return st;
      }
      iters += h.it;
      // replacement: x += s d, r = b - A x in FP64
      pcg_correct<<<kVB, kVT, 0, s>>>(n, w->xp, w->d32, scale);
      CKP(launch_ehyb_f64(D, w->xp, w->q, 0, s));
      pcg_residual<<<kVB, kVT, 0, s>>>(n, w->bp, w->q, w->r, nullptr, w->part);
      if ((st = sum_part(w, s, &rr)) != EHYB_OK) return st;
      ++outer;
      if (std::sqrt(rr) <= rtol * bnorm) {
        converged = 1;
        break;
      }
      if (h.breakdown || !(rr < 1e300) || iters >= max_iter) break;
      if (rr < best_rr) {
        best_rr = rr;
        stalls = 0;
      } else if (++stalls >= 3) {
        break;  // three replacements without a better FP64 residual: FP32 has nothing left to give
      }
      const double ns = std::sqrt(rr);
      const double ratio = scale / ns;
      pcg_replace<<<kVB, kVT, 0, s>>>(n, w->r, 1.0 / ns, (float)ratio, w->r32, w->d32, w->p32, w->part);
      pcg_replace_finish<<<1, 32, 0, s>>>(w->part, kVB, delta * delta, ratio * ratio, max_iter - iters, w->hist,
                                          w->st);
      CKP(cudaGetLastError());
      scale = ns;
      // finish the interrupted iteration on the replaced residual: z = M r, p = z + beta p
      if ((st = apply_precond(M, w, s, nullptr)) != EHYB_OK) return st;
      pcg_pupdate32_force<<<kVB, kVT, 0, s>>>(n, w->z32, w->p32, w->st);
      CKP(cudaGetLastError());
    }
  }
  CKP(launch_permute_f64(D, 0, w->xp, x, s));
  CKP(cudaStreamSynchronize(s));
  info->iterations = iters;
  info->refinements = outer;
  info->converged = converged;
  info->relres = std::sqrt(rr) / bnorm;
  info->relres_recursive = info->relres;
  info->seconds = now_s() - t0;
  return converged ? EHYB_OK : EHYB_ERR_NOT_CONVERGED;
}
