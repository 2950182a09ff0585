// Device code shared by the EHYB kernels (per-plan launch and persistent batch launch), sm_103a.
//
// partition_spmv: Alg. 3 re-designed for GB300.  One thread block works on one partition at a time
//   (the paper's "block = partition", Sec. 3.2):
//     1. thread 0 issues ONE bulk asynchronous copy (cp.async.bulk, completion counted on an
//        mbarrier) of the partition's slice of x into shared memory: CachedVec of Alg. 3;
//        a ragged unaligned tail (at most 15 bytes) is fetched with plain loads;
//     2. thread 0 waits on the mbarrier with a time bound (on expiry the block records
//        EHYB_ERR_TIMEOUT in the plan status word and returns);
//     3. each warp takes 32-lane slices of the partition from a shared counter (the dynamic
//        slice balancing of Alg. 3) and runs y[row] = sum_k ValELL * CachedVec[ColELL] with the
//        16-bit column offsets of Sec. 3.4, exactly one FMA per stored slot, six to 32 slots of
//        values and columns loaded ahead of their FMAs to keep enough bytes in flight; the FP32 / BF16
//        copies (sliced ER layout) keep each lane's slots in runs of four (slot_pos in plan.h), read a
//        run's values and columns with one vector load each and hold them packed until their FMAs;
//        each block keeps its partition's slice table (where each slice starts, its widths) in shared
//        memory, so claiming the next slice costs no global load;
//     4. extra-row (ER) entries, three layouts:
//        - sliced (er_layout 0, default): the ER entries of the slice's own rows are stored in
//          the same lane -> row arrangement right behind it (the paper stores its ER part as
//          stride-32 slices too, Alg. 2); the warp continues with them, gathering x from global
//          memory, and writes y once -- no block barrier, no read-modify-write, no FP64 shuffle;
//        - CSR lines (er_layout 1): after a block barrier, er_tpr lanes per ER line with a
//          shuffle reduction, y[yIdxER] += sum;
//        - halo (er_layout 2): step 1 also stages x at the partition's halo (the distinct columns
//          of its ER entries outside it) behind the slice, and a row's ER entries follow its own
//          in the slab slots with 16-bit columns into [slice | halo]: step 3 covers them.
//   In every layout the rows a block updates are its own, so the paper's second pass over ER
//   slices from a global counter is not needed: no atomics on y, deterministic results.
#pragma once
#include <cstdint>

#include "device.h"

namespace ehyb {
namespace core {


constexpr unsigned FULL = 0xffffffffu;
constexpr int kTimeoutCode = 9;  // EHYB_ERR_TIMEOUT
constexpr int kBoundsCode = 12;  // EHYB_ERR_BOUNDS
constexpr int kDrainLimits = 8;  // time limits a timed-out block waits for its own staging copy to land

// Checked build (-DEHYB_BOUNDS_CHECK=1): every index the kernels compute into shared memory, x and y is
// tested against its buffer; a violation records EHYB_ERR_BOUNDS in the plan status word and the access
// goes to index 0 instead.  The default build compiles the tests away.
#ifndef EHYB_BOUNDS_CHECK
#define EHYB_BOUNDS_CHECK 0
#endif
template <typename I>
__device__ __forceinline__ I checked(I i, int64_t lim, int32_t* status) {
  if (EHYB_BOUNDS_CHECK && ((int64_t)i < 0 || (int64_t)i >= lim)) {
    atomicCAS(status, 0, kBoundsCode);
    return I(0);
  }
  return i;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait: true when phase `parity` completed within limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// Wait (bounded) for the staging copy counted on `bar`.  On expiry record EHYB_ERR_TIMEOUT and, when the
// copy was issued, wait up to kDrainLimits more time limits for it to land before the block's shared
// memory goes away; past that the device no longer completes copies, the block leaves anyway (every wait
// is bounded) and the status word tells the host to stop using the device.  Returns false on expiry.
__device__ __forceinline__ bool staging_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns, bool issued,
                                             int32_t* status) {
  if (mbar_wait_bounded(bar, parity, limit_ns)) return true;
  atomicCAS(status, 0, kTimeoutCode);
  if (issued)
    for (int r = 0; r < kDrainLimits && !mbar_wait_bounded(bar, parity, limit_ns); ++r) {
    }
  return false;
}

// Programmatic dependent launch: let the next kernel in the stream be scheduled now / wait until the
// previous kernel in the stream has completed and its memory is visible (no-ops without the attribute).
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }

template <typename V, typename X>
__device__ __forceinline__ X load_val(const V* p);
template <>
__device__ __forceinline__ double load_val<double, double>(const double* p) {
  return __ldcs(p);
}
template <>
__device__ __forceinline__ float load_val<float, float>(const float* p) {
  return __ldcs(p);
}
template <>
__device__ __forceinline__ float load_val<uint16_t, float>(const uint16_t* p) {
  return bf16_to_f32(__ldcs(reinterpret_cast<const unsigned short*>(p)));
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

constexpr int kBatch = 8;   // slots whose loads are issued before their FMAs (default batch depth)
constexpr int kStage = 16;  // elements of x per thread in flight while a slice of x is gathered

// ---- column-major slots (Alg. 2: slot k of a lane at 32 k from its first one)

// acc += sum_{k<w} v[32k] * xs[c[32k]]: slab slots of one lane, x from shared memory.  Loads go out in
// half-batches of KB/2 slots, the next half-batch issued before the current one's FMAs (KB slots held in
// registers); the FMAs run in slot order, so the result does not depend on KB.  (A predicated last batch
// measured slower than this scalar remainder on both 3D workloads.)
template <typename V, typename X, int KB = kBatch>
__device__ __forceinline__ X slab_dot(const V* __restrict__ vp, const uint16_t* __restrict__ cp, int w,
                                      const X* xs, X acc, int lim, int32_t* status) {
  constexpr int H = KB / 2;
  int k = 0;
  if (w >= H) {
    X va[H];
    int ca[H];
#pragma unroll
    for (int u = 0; u < H; ++u) {
      va[u] = load_val<V, X>(vp + 32 * (int64_t)u);
      ca[u] = checked((int)__ldcs(reinterpret_cast<const unsigned short*>(cp + 32 * (int64_t)u)), lim, status);
    }
    for (k = H; k + H <= w; k += H) {
      X vb[H];
      int cb[H];
#pragma unroll
      for (int u = 0; u < H; ++u) {
        vb[u] = load_val<V, X>(vp + 32 * (int64_t)(k + u));
        cb[u] = checked((int)__ldcs(reinterpret_cast<const unsigned short*>(cp + 32 * (int64_t)(k + u))), lim, status);
      }
#pragma unroll
      for (int u = 0; u < H; ++u) acc = fma_t(va[u], xs[ca[u]], acc);
#pragma unroll
      for (int u = 0; u < H; ++u) {
        va[u] = vb[u];
        ca[u] = cb[u];
      }
    }
#pragma unroll
    for (int u = 0; u < H; ++u) acc = fma_t(va[u], xs[ca[u]], acc);
  }
  for (; k < w; ++k)
    acc = fma_t(load_val<V, X>(vp + 32 * (int64_t)k),
                xs[checked((int)__ldcs(reinterpret_cast<const unsigned short*>(cp + 32 * (int64_t)k)), lim, status)],
                acc);
  return acc;
}

// acc += sum_{k<w} v[32k] * xg[c[32k]]: sliced extra-row slots of one lane, x from global memory
template <typename V, typename X, int KB = kBatch>
__device__ __forceinline__ X er_dot(const V* __restrict__ vp, const int32_t* __restrict__ cp, int w,
                                    const X* __restrict__ xg, X acc, int64_t lim, int32_t* status) {
  int k = 0;
  for (; k + KB <= w; k += KB) {
    X v[KB];
    int c[KB];
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      v[u] = load_val<V, X>(vp + 32 * (int64_t)(k + u));
      c[u] = checked(__ldcs(cp + 32 * (int64_t)(k + u)), lim, status);
    }
    X xv[KB];
#pragma unroll
    for (int u = 0; u < KB; ++u) xv[u] = __ldg(xg + c[u]);
#pragma unroll
    for (int u = 0; u < KB; ++u) acc = fma_t(v[u], xv[u], acc);
  }
  for (; k < w; ++k)
    acc = fma_t(load_val<V, X>(vp + 32 * (int64_t)k), __ldg(xg + checked(__ldcs(cp + 32 * (int64_t)k), lim, status)),
                acc);
  return acc;
}

// ---- slots in runs of four per lane (the FP32 / BF16 copies of the sliced ER layout; slot_pos, group 4):
// a lane reads a run's four values with one 16-byte (FP32) or 8-byte (BF16) load and its four 16-bit columns
// with one 8-byte load; the w mod 4 slots after the runs are column-major.
constexpr int kGroup = 4;
constexpr int kErGroups = 2;  // runs per batch of the extra-row loop (8 slots, their x gathers in flight)

__device__ __forceinline__ void ld_group(const float* p, float (&o)[4]) {
  const float4 a = __ldcs(reinterpret_cast<const float4*>(p));
  o[0] = a.x;
  o[1] = a.y;
  o[2] = a.z;
  o[3] = a.w;
}
__device__ __forceinline__ void ld_group(const uint16_t* p, float (&o)[4]) {  // four BF16 values
  const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
  o[0] = __uint_as_float(v.x << 16);  // the value at the lower address is the low half (little endian)
  o[1] = __uint_as_float(v.x & 0xffff0000u);
  o[2] = __uint_as_float(v.y << 16);
  o[3] = __uint_as_float(v.y & 0xffff0000u);
}
__device__ __forceinline__ void ld_cols(const int32_t* p, int (&c)[4]) {  // four 32-bit columns
  const int4 v = __ldcs(reinterpret_cast<const int4*>(p));
  c[0] = v.x;
  c[1] = v.y;
  c[2] = v.z;
  c[3] = v.w;
}

// A run of four slots as loaded: values and 16-bit columns stay packed in registers until their FMAs (a BF16
// run takes four registers, an FP32 run six), so a lane holds twice the slots in flight for its registers.
template <typename V>
struct Run;
template <>
struct Run<float> {
  float4 v;
  uint2 c;
};
template <>
struct Run<uint16_t> {
  uint2 v;
  uint2 c;
};
__device__ __forceinline__ void ld_run(const float* vp, const uint16_t* cp, Run<float>& r) {
  r.v = __ldcs(reinterpret_cast<const float4*>(vp));
  r.c = __ldcs(reinterpret_cast<const uint2*>(cp));
}
__device__ __forceinline__ void ld_run(const uint16_t* vp, const uint16_t* cp, Run<uint16_t>& r) {
  r.v = __ldcs(reinterpret_cast<const uint2*>(vp));
  r.c = __ldcs(reinterpret_cast<const uint2*>(cp));
}
__device__ __forceinline__ void zero_run(Run<float>& r) {
  r.v = make_float4(0.f, 0.f, 0.f, 0.f);
  r.c = make_uint2(0u, 0u);
}
__device__ __forceinline__ void zero_run(Run<uint16_t>& r) {
  r.v = make_uint2(0u, 0u);
  r.c = make_uint2(0u, 0u);
}
__device__ __forceinline__ float run_val(const Run<float>& r, int t) {
  return t == 0 ? r.v.x : t == 1 ? r.v.y : t == 2 ? r.v.z : r.v.w;
}
__device__ __forceinline__ float run_val(const Run<uint16_t>& r, int t) {  // the lower address is the low half
  const uint32_t h = t < 2 ? r.v.x : r.v.y;
  return __uint_as_float((t & 1) ? (h & 0xffff0000u) : (h << 16));
}
__device__ __forceinline__ int run_col(const uint2& c, int t) {
  const uint32_t h = t < 2 ? c.x : c.y;
  return (int)((t & 1) ? (h >> 16) : (h & 0xffffu));
}
// acc += the run's four products, in slot order
template <typename V>
__device__ __forceinline__ float fma_run(const Run<V>& r, const float* xs, float acc, int lim, int32_t* status) {
#pragma unroll
  for (int t = 0; t < kGroup; ++t) acc = fmaf(run_val(r, t), xs[checked(run_col(r.c, t), lim, status)], acc);
  return acc;
}

// slab_dot on runs of four: vb, cb = the slice's first slot; half-batches of NG = KB/8 runs (KB slots in
// flight), the next half-batch's loads issued before the current one's FMAs, the last half-batch guarded by
// the run count; the w mod 4 column-major slots after the runs are loaded with the first half-batch and
// multiplied last.  Same slot order, same result as slab_dot on the column-major copy.
template <typename V, typename X, int KB>
__device__ __forceinline__ X slab_dot_runs(const V* __restrict__ vb, const uint16_t* __restrict__ cb, int lane, int w,
                                           const X* xs, X acc, int lim, int32_t* status) {
  constexpr int NG = KB / 8;
  static_assert(NG >= 1 && KB % 8 == 0, "runs: half-batches of whole runs");
  const int ng = w >> 2;
  const int nt = w & (kGroup - 1);
  const V* vp = vb + kGroup * lane;  // run g of this lane: vp + 128 g
  const uint16_t* cp = cb + kGroup * lane;
  Run<V> ra[NG];
#pragma unroll
  for (int u = 0; u < NG; ++u) {
    zero_run(ra[u]);
    if (u < ng) ld_run(vp + 128 * (int64_t)u, cp + 128 * (int64_t)u, ra[u]);
  }
  // column-major tail: slot 4 ng + t of this lane at the slice's first slot + 128 ng + 32 t + lane
  X tv[kGroup - 1];
  int tc[kGroup - 1];
#pragma unroll
  for (int t = 0; t < kGroup - 1; ++t) {
    tv[t] = X(0);
    tc[t] = 0;
    if (t < nt) {
      const int64_t o = 128 * (int64_t)ng + 32 * t + lane;
      tv[t] = load_val<V, X>(vb + o);
      tc[t] = checked((int)__ldcs(reinterpret_cast<const unsigned short*>(cb + o)), lim, status);
    }
  }
  int g = NG;  // runs [g - NG, g) are in ra
  for (; g < ng; g += NG) {
    Run<V> rb[NG];
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      zero_run(rb[u]);
      if (g + u < ng) ld_run(vp + 128 * (int64_t)(g + u), cp + 128 * (int64_t)(g + u), rb[u]);
    }
#pragma unroll
    for (int u = 0; u < NG; ++u) acc = fma_run(ra[u], xs, acc, lim, status);  // g < ng: all NG runs are stored
#pragma unroll
    for (int u = 0; u < NG; ++u) ra[u] = rb[u];
  }
  const int last = ng - (g - NG);  // 0..NG stored runs in ra
#pragma unroll
  for (int u = 0; u < NG; ++u)
    if (u < last) acc = fma_run(ra[u], xs, acc, lim, status);
#pragma unroll
  for (int t = 0; t < kGroup - 1; ++t)
    if (t < nt) acc = fma_t(tv[t], xs[tc[t]], acc);
  return acc;
}

// er_dot on runs of four: batches of kErGroups runs (values and columns loaded, then their x gathers, then
// the FMAs in slot order), then the remaining run and the column-major tail
template <typename V, typename X>
__device__ __forceinline__ X er_dot_runs(const V* __restrict__ vb, const int32_t* __restrict__ cb, int lane, int w,
                                         const X* __restrict__ xg, X acc, int64_t lim, int32_t* status) {
  constexpr int NB = kErGroups;
  const int ng = w >> 2;
  const V* vp = vb + kGroup * lane;
  const int32_t* cp = cb + kGroup * lane;
  int g = 0;
  for (; g + NB <= ng; g += NB) {
    X v[NB][kGroup];
    int c[NB][kGroup];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      ld_group(vp + 128 * (int64_t)(g + u), v[u]);
      ld_cols(cp + 128 * (int64_t)(g + u), c[u]);
    }
    X xv[NB][kGroup];
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int t = 0; t < kGroup; ++t) xv[u][t] = __ldg(xg + checked(c[u][t], lim, status));
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int t = 0; t < kGroup; ++t) acc = fma_t(v[u][t], xv[u][t], acc);
  }
  for (; g < ng; ++g) {
    X v[kGroup];
    int c[kGroup];
    ld_group(vp + 128 * (int64_t)g, v);
    ld_cols(cp + 128 * (int64_t)g, c);
    X xv[kGroup];
#pragma unroll
    for (int t = 0; t < kGroup; ++t) xv[t] = __ldg(xg + checked(c[t], lim, status));
#pragma unroll
    for (int t = 0; t < kGroup; ++t) acc = fma_t(v[t], xv[t], acc);
  }
  // the w mod 4 column-major slots: loads, then gathers, then FMAs, guarded (one round trip each)
  const int nt = w & (kGroup - 1);
  const V* tvp = vb + 128 * (int64_t)ng + lane;
  const int32_t* tcp = cb + 128 * (int64_t)ng + lane;
  X tv[kGroup - 1];
  int tc[kGroup - 1];
#pragma unroll
  for (int t = 0; t < kGroup - 1; ++t) {
    tv[t] = X(0);
    tc[t] = 0;
    if (t < nt) {
      tv[t] = load_val<V, X>(tvp + 32 * t);
      tc[t] = checked(__ldcs(tcp + 32 * t), lim, status);
    }
  }
  X tx[kGroup - 1];
#pragma unroll
  for (int t = 0; t < kGroup - 1; ++t) {
    tx[t] = X(0);
    if (t < nt) tx[t] = __ldg(xg + tc[t]);
  }
#pragma unroll
  for (int t = 0; t < kGroup - 1; ++t)
    if (t < nt) acc = fma_t(tv[t], tx[t], acc);
  return acc;
}

struct KArgs {
  int32_t tpr_log2, er_tpr_log2;
  int64_t n;              // rows of the matrix (of y)
  int64_t n_x;            // elements of x the extra-row columns index (n; a shard adds its halo)
  int64_t smem_elems;     // capacity of the staged slice of x (elements); checked build only
  const int64_t* er_slice_pos;
  const int32_t* er_scol;
  const int32_t* er_scol_old;
  const int32_t* new_to_old;
  const int32_t* part_ptr;
  const int32_t* slice_ptr;
  const int64_t* slice_pos;
  const int32_t* slice_order;
  const uint16_t* ell_col;
  const int32_t* er_part_ptr;
  const int32_t* er_row;
  const int64_t* er_ptr;
  const int32_t* er_col;
  const int64_t* halo_ptr;  // er_layout 2 (else null): partition p stages x at halo_*[halo_ptr[p] ..) after its rows
  const int32_t* halo_new;  //   plan numbering
  const int32_t* halo_old;  //   caller's numbering (GATHER)
  int32_t* status;
  uint64_t timeout_ns;
  int32_t inject;
  double* dot_part;       // optional: per-block partial of sum_r y_r * xp_r (fixed summation order)
  int32_t dot_self;       //   ... of sum_r y_r * y_r instead
  int32_t* dot_arrive;    // optional (with dot_part, one block per partition): arrival counter; the last
  double* dot_result;     //   block reduces the partials into *dot_result and resets the counter
  const int32_t* skip;    // optional: the launch does nothing while *skip != 0 (converged solver)
  int32_t meta_off;       // byte offset of the partition's slice table in dynamic shared memory (0: none)
  int32_t meta_cap;       //   ... and its capacity in entries (checked build only)
};

// One slice of a partition in its processing order, as the block keeps it in shared memory: where its slab
// and extra-row slots start and how many slots a lane has in each.  Staged once per partition, so a warp
// that claims its next slice reads it from shared memory instead of two dependent global loads
// (slice_order, then slice_pos).
struct SliceMeta {
  int64_t pos, epos;
  int32_t w, we, s, pad;
};

// warp-level fixed-order sum of count values (lane-strided, then an xor tree); every lane gets it
__device__ __forceinline__ double warp_sum_fixed(const double* part, int count) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
#pragma unroll 4
  for (int i = lane; i < count; i += 32) v += part[i];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

// Deterministic block sum (xor-tree inside warps, warps in index order); result in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v, double* ws) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
  return s;
}

// V: stored value type; X: type of x, y and of the accumulation
// Shared state of one block; a block may run several partitions one after the other.
struct BlockState {
  uint64_t bar;        // mbarrier counting the bytes of the bulk staging copy
  uint32_t phase;      // phases of bar completed so far
  int bar_ready;       // bar has been initialised
  int slice_counter;   // next slice of the current partition
  int stage_ok;
  int is_last;
  double ws[32];
};

// One partition p of a plan: stage its slice of x_p, run its slab (and ER) slices, write y.
// GATHER: x is given in the caller's numbering and the permutation into the plan numbering is fused
// into the staging (xs[r - pb] = x[new_to_old[r]], plain loads) and into the ER gathers (columns in the
// caller's numbering), so no permuted copy of x is written or read; otherwise x is x_p and the slice is
// staged by one bulk asynchronous copy.
// Returns false (uniformly across the block) when the staging wait ran
// out of time.
// TABLE: the launch may provide the partition's slice table (a.meta_off); without it only the global path is
// compiled (the persistent batch kernel, whose blocks run many partitions one after the other).
// PDL: the kernel was launched with programmatic stream serialization and has not yet waited for the previous
// grid: the slice table, which reads plan arrays only, is filled first, then griddepcontrol.wait, then every
// read of x (and of the solver's skip flag) and every write of y.
template <typename V, typename X, bool SCATTER, bool ER_SLICED, bool DOT = false, bool GATHER = false,
          int KB = kBatch, bool RUNS = false, bool TABLE = false, bool PDL = false>
__device__ __forceinline__ bool partition_spmv(const KArgs& a, const V* __restrict__ ell_val,
                                               const V* __restrict__ er_val, const X* __restrict__ xp,
                                               X* __restrict__ y, const int p, X* xs, BlockState& bs) {
  constexpr int EPV = 16 / (int)sizeof(X);  // elements per 16 bytes
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const int pb = a.part_ptr[p];
  const int pe = a.part_ptr[p + 1];
  const int s0 = a.slice_ptr[p];
  const int s1 = a.slice_ptr[p + 1];

  const int bd = blockDim.x;
  // ---- 0. the partition's slice table (a.meta_off != 0): entry t = the slice at position s0 + t of the
  // processing order, its slab / ER start and widths (plan arrays only: before the wait on the previous grid)
  SliceMeta* tbl = (TABLE && a.meta_off)
                       ? reinterpret_cast<SliceMeta*>(reinterpret_cast<unsigned char*>(xs) + a.meta_off)
                       : nullptr;
  const int ns = s1 - s0;
  if (tbl) {
    for (int t = tid; t < ns; t += bd) {
      const int sl = a.slice_order[s0 + t];
      SliceMeta m;
      m.pos = a.slice_pos[sl];
      m.w = (int)((a.slice_pos[sl + 1] - m.pos) >> 5);
      m.epos = 0;
      m.we = 0;
      if (ER_SLICED) {
        m.epos = a.er_slice_pos[sl];
        m.we = (int)((a.er_slice_pos[sl + 1] - m.epos) >> 5);
      }
      m.s = sl;
      m.pad = 0;
      tbl[checked(t, a.meta_cap, a.status)] = m;
    }
  }
  if (PDL) {
    pdl_wait();
    if (a.skip && *a.skip) return true;  // uniform across the grid (a converged solver's flag)
  }

  // ---- 1. stage x_p[pb, pe) into shared memory
  const int a0 = pb & ~(EPV - 1);  // 16-byte aligned start
  const int a1 = pe & ~(EPV - 1);  // bulk part ends at the last aligned boundary <= pe
  const bool aligned_src = ((reinterpret_cast<uintptr_t>(xp) & 15u) == 0);
  const uint32_t bulk_bytes =
      (!GATHER && aligned_src && a1 > a0) ? (uint32_t)(a1 - a0) * (uint32_t)sizeof(X) : 0u;
  if (tid == 0) {
    bs.slice_counter = s0 + nwarps;
    if (bulk_bytes) {
      if (!bs.bar_ready) {
        mbar_init(&bs.bar, 1);
        bs.bar_ready = 1;
      }
      // order this block's earlier generic-proxy use of the buffer before the async-proxy copy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(&bs.bar, bulk_bytes);
      if (!a.inject) bulk_g2s(xs, xp + a0, bulk_bytes, &bs.bar);
    }
  }
  if (GATHER) {
    // xs[r - a0] = x[new_to_old[r]]: kStage indices, then kStage values in flight per thread (one round
    // covers a partition of kStage * blockDim rows)
    for (int i0 = pb + tid; i0 < pe; i0 += kStage * bd) {
      int c[kStage];
#pragma unroll
      for (int u = 0; u < kStage; ++u)
        c[u] = (i0 + u * bd < pe) ? checked(__ldg(a.new_to_old + i0 + u * bd), a.n, a.status) : -1;
      X v[kStage];
#pragma unroll
      for (int u = 0; u < kStage; ++u) v[u] = c[u] >= 0 ? __ldg(xp + c[u]) : X(0);
#pragma unroll
      for (int u = 0; u < kStage; ++u)
        if (i0 + u * bd < pe) xs[checked(i0 + u * bd - a0, a.smem_elems, a.status)] = v[u];
    }
  } else {
    // plain loads: everything when the source is unaligned, else the ragged tail [a1, pe)
    const int lo = bulk_bytes ? (a1 > pb ? a1 : pb) : pb;
    for (int i = lo + tid; i < pe; i += blockDim.x) xs[checked(i - a0, a.smem_elems, a.status)] = xp[i];
  }
  // er_layout 2: the halo's x values right after the slice (xs[pe - a0 + j], j < nh), gathered like the
  // slice itself (plain loads; disjoint from the bulk copy's destination, which ends at a1 - a0).  A loop of
  // its own: folding it into the gather above slowed the other layouts' staging.
  int nh = 0;
  if (a.halo_ptr) {
    const int64_t h0 = a.halo_ptr[p];
    nh = (int)(a.halo_ptr[p + 1] - h0);
    const int32_t* hc = (GATHER ? a.halo_old : a.halo_new) + h0;
    for (int j0 = tid; j0 < nh; j0 += kStage * bd) {
      int c[kStage];
#pragma unroll
      for (int u = 0; u < kStage; ++u) c[u] = (j0 + u * bd < nh) ? checked(__ldg(hc + j0 + u * bd), a.n, a.status) : -1;
      X v[kStage];
#pragma unroll
      for (int u = 0; u < kStage; ++u) v[u] = c[u] >= 0 ? __ldg(xp + c[u]) : X(0);
#pragma unroll
      for (int u = 0; u < kStage; ++u)
        if (j0 + u * bd < nh) xs[checked(pe - a0 + j0 + u * bd, a.smem_elems, a.status)] = v[u];
    }
  }
  if (tid == 0) {
    int ok = 1;
    if (bulk_bytes) {
      const uint32_t par = bs.phase & 1u;
      ok = staging_wait(&bs.bar, par, a.timeout_ns, !a.inject, a.status) ? 1 : 0;
      bs.phase += 1;
    }
    bs.stage_ok = ok;
  }
  __syncthreads();
  if (!bs.stage_ok) return false;
  // every thread observes the completed phase itself (acquire of the bulk-copy writes)
  if (bulk_bytes) (void)mbar_try_wait(&bs.bar, (bs.phase - 1u) & 1u);

  const X* xsl = xs + (pb - a0);  // xsl[local column] = x_p[pb + local column]
  const int tpr = 1 << a.tpr_log2;
  const int sub = lane & (tpr - 1);
  const int rows_per_slice = 32 >> a.tpr_log2;

  // ---- 2. slab: warp per 32-lane slice, dynamic slice balancing inside the partition
  // (static round-robin when the fused dot product is requested, so its order is fixed)
  constexpr bool dot = DOT;  // a.dot_part is set
  double dacc = 0.0;
  // metadata of the slice at position j of the processing order (j < s1): from the table, else from global
  auto slice_meta = [&](int j, int& sj, int64_t& posj, int& wj, int64_t& eposj, int& wej) {
    if (tbl) {
      const SliceMeta m = tbl[checked(j - s0, a.meta_cap, a.status)];
      sj = m.s;
      posj = m.pos;
      wj = m.w;
      eposj = m.epos;
      wej = m.we;
      return;
    }
    sj = a.slice_order[j];
    posj = a.slice_pos[sj];
    wj = (int)((a.slice_pos[sj + 1] - posj) >> 5);
    if (ER_SLICED) {
      eposj = a.er_slice_pos[sj];
      wej = (int)((a.er_slice_pos[sj + 1] - eposj) >> 5);
    }
  };
  int i = s0 + warp;  // position in the partition's processing order
  int s = s1;
  int64_t pos = 0, epos = 0;
  int w = 0, we = 0;
  if (i < s1) slice_meta(i, s, pos, w, epos, we);
  while (i < s1) {
    // reserve the next slice and start its metadata loads before working on this one
    int inxt;
    if (dot) {
      inxt = i + nwarps;
    } else {
      int t = 0;
      if (lane == 0) t = atomicAdd(&bs.slice_counter, 1);
      inxt = __shfl_sync(FULL, t, 0);
    }
    int nxt = s1;
    int64_t npos = 0, nepos = 0;
    int nw = 0, nwe = 0;
    if (inxt < s1) slice_meta(inxt, nxt, npos, nw, nepos, nwe);
    X acc;
    if constexpr (RUNS) {  // the copy in runs of four slots (its own column arrays are in a.ell_col / a.er_scol*)
      acc = slab_dot_runs<V, X, KB>(ell_val + pos, a.ell_col + pos, lane, w, xsl, X(0), pe - pb + nh, a.status);
      if (ER_SLICED)
        acc = er_dot_runs<V, X>(er_val + epos, (GATHER ? a.er_scol_old : a.er_scol) + epos, lane, we, xp, acc, a.n_x,
                                a.status);
    } else {
      acc = slab_dot<V, X, KB>(ell_val + pos + lane, a.ell_col + pos + lane, w, xsl, X(0), pe - pb + nh, a.status);
      if (ER_SLICED)
        acc = er_dot<V, X, KB>(er_val + epos + lane, (GATHER ? a.er_scol_old : a.er_scol) + epos + lane, we, xp, acc,
                               a.n_x, a.status);
    }
    for (int off = tpr >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    const int row = pb + (s - s0) * rows_per_slice + (lane >> a.tpr_log2);
    if (sub == 0 && row < pe) {
      if (SCATTER) y[checked(a.new_to_old[row], a.n, a.status)] = acc;
      else y[checked(row, a.n, a.status)] = acc;
      if (dot) dacc = fma((double)acc, a.dot_self ? (double)acc : (double)xsl[row - pb], dacc);
    }
    i = inxt;
    s = nxt;
    pos = npos;
    w = nw;
    epos = nepos;
    we = nwe;
  }
  if (dot) {  // only offered for the sliced ER layout, where a slice's rows are final here
    const double t = block_sum_fixed(dacc, bs.ws);
    if (tid == 0) a.dot_part[p] = t;
    if (a.dot_arrive) {
      if (tid == 0) {
        __threadfence();
        bs.is_last = atomicAdd(a.dot_arrive, 1) == (int)gridDim.x - 1;
      }
      __syncthreads();
      if (bs.is_last && tid < 32) {
        __threadfence();
        const double sum = warp_sum_fixed(a.dot_part, (int)gridDim.x);
        if (tid == 0) {
          *a.dot_result = sum;
          *a.dot_arrive = 0;
        }
      }
    }
  }
  if (ER_SLICED) return true;
  const int e0 = a.er_part_ptr[p];
  const int e1 = a.er_part_ptr[p + 1];
  if (e0 == e1) return true;
  __syncthreads();  // slab results of this block are visible before the ER updates

  // ---- 3. ER lines of this partition: er_tpr lanes per line, shuffle reduction
  const int etpr = 1 << a.er_tpr_log2;
  const int esub = lane & (etpr - 1);
  const int lines_per_warp = 32 >> a.er_tpr_log2;
  for (int eb = e0 + warp * lines_per_warp; eb < e1; eb += nwarps * lines_per_warp) {
    const int e = eb + (lane >> a.er_tpr_log2);
    X acc = X(0);
    if (e < e1) {
      const int64_t k1 = a.er_ptr[e + 1];
      int64_t k = a.er_ptr[e] + esub;
      for (; k + 3 * etpr < k1; k += 4 * etpr) {  // four entries' loads in flight
        X v[4], xv[4];
        int c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[u] = load_val<V, X>(er_val + k + u * etpr);
          c[u] = checked(__ldcs(a.er_col + k + u * etpr), a.n, a.status);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = __ldg(xp + c[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = fma_t(v[u], xv[u], acc);
      }
      for (; k < k1; k += etpr)
        acc = fma_t(load_val<V, X>(er_val + k), __ldg(xp + checked(__ldcs(a.er_col + k), a.n, a.status)), acc);
    }
    for (int off = etpr >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    if (esub == 0 && e < e1) {
      const int row = a.er_row[e];
      if (SCATTER) y[checked(a.new_to_old[row], a.n, a.status)] += acc;
      else y[checked(row, a.n, a.status)] += acc;
    }
  }
  return true;
}

// host helpers
inline int ilog2(int v) {
  int l = 0;
  while ((1 << (l + 1)) <= v) ++l;
  return l;
}

inline KArgs make_kargs(const DevPlan& P) {
  KArgs a;
  a.tpr_log2 = ilog2(P.tpr);
  a.n = P.n;
  a.n_x = P.n_x > 0 ? P.n_x : P.n;
  // launches set the exact capacity of their shared memory
  a.smem_elems = (int64_t)(P.max_stage_rows > P.max_part_rows ? P.max_stage_rows : P.max_part_rows) + 2;
  a.er_tpr_log2 = ilog2(P.er_tpr);
  a.er_slice_pos = P.er_slice_pos;
  a.er_scol = P.er_scol;
  a.er_scol_old = P.er_scol_old;
  a.new_to_old = P.new_to_old;
  a.part_ptr = P.part_ptr;
  a.slice_ptr = P.slice_ptr;
  a.slice_pos = P.slice_pos;
  a.slice_order = P.slice_order;
  a.ell_col = P.ell_col;
  a.er_part_ptr = P.er_part_ptr;
  a.er_row = P.er_row;
  a.er_ptr = P.er_ptr;
  a.er_col = P.er_col;
  const bool halo = P.er_layout == 2;
  a.halo_ptr = halo ? P.halo_ptr : nullptr;
  a.halo_new = halo ? P.halo_new : nullptr;
  a.halo_old = halo ? P.halo_old : nullptr;
  a.status = P.status;
  a.timeout_ns = P.wait_timeout_ns;
  a.inject = P.inject_wait_fault;
  a.dot_part = nullptr;
  a.dot_self = 0;
  a.dot_arrive = nullptr;
  a.dot_result = nullptr;
  a.skip = nullptr;
  a.meta_off = 0;
  a.meta_cap = 0;
  return a;
}

}  // namespace core
}  // namespace ehyb
