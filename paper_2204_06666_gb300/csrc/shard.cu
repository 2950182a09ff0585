// Row shards of an EHYB plan for several GPUs: the halo-exchange form of the method.
//
// The paper's partitions are contiguous ranges of the reordered rows, and the slab of a partition reads
// only the partition's own slice of x (Sec. 3.1-3.2); only the extra-row (ER) entries reach outside it.
// Giving each rank a contiguous group of partitions therefore leaves one exchange per product: the x
// entries that the rank's ER columns name in other ranks' rows (its halo).  A shard holds
//   * its partitions' slab and sliced-ER slots, unchanged, with slice offsets rebased to the shard;
//   * its ER columns renumbered into x_ext = [x_local (n_local rows) | halo (n_halo)]: a column inside the
//     rank's rows becomes local, a column outside becomes n_local + its place in the halo list;
//   * the halo list (the remote plan rows it reads, ascending, so grouped by owning rank) and, for every
//     peer, the local rows it sends (the peer's halo entries that fall in this rank's rows, ascending).
// With those lists the exchange is one all-to-all: rank r packs send_buf = x_local[send_idx] in peer
// order and receives into x_ext[n_local:] in peer order (recv counts = the halo's groups).  A shard's
// product runs the same per-partition kernel as a plan, so it sums every row in the same order: the
// concatenated shard results equal the plan's result bit for bit.
//
// CG over shards (ehyb_shard_cg) keeps the data path in these kernels and hands the two communication
// steps to the caller: the halo exchange of the direction, and a sum over ranks of 1-2 host scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "plan_internal.h"

namespace ehyb {
namespace {

constexpr int kVB = 608;  // vector-kernel blocks
constexpr int kVT = 256;

}  // namespace
}  // namespace ehyb

struct ehyb_shard_s {
  int32_t nranks = 1, rank = 0;
  int32_t p0 = 0, p1 = 0;        // the plan's partitions [p0, p1)
  int64_t lo = 0, hi = 0;        // the plan's rows [lo, hi) (plan numbering)
  int64_t n_halo = 0;
  bool host_only = false;
  // host copies
  std::vector<int32_t> new_to_old;            // original row of each local row
  std::vector<int32_t> part_ptr, slice_ptr, slice_order, row_ell_count, row_er_count;
  std::vector<int64_t> slice_pos, er_slice_pos;
  std::vector<uint16_t> ell_col;
  std::vector<double> ell_val, er_sval;
  std::vector<int32_t> er_scol;               // renumbered into x_ext
  std::vector<int32_t> halo_rows;             // plan rows of the halo, ascending
  std::vector<int64_t> send_ptr, recv_ptr;    // nranks + 1 each
  std::vector<int32_t> send_idx;              // local rows, grouped by peer
  // device
  ehyb::DevPlan dev;
  void* arena = nullptr;
  const int32_t* d_send_idx = nullptr;
  double* d_dot = nullptr;                    // fused p.q: per-partition partials, result
  int32_t* d_arrive = nullptr;
  double* work = nullptr;                     // CG: r, q, partials
  size_t work_bytes = 0;
  int device = -1;
};

namespace ehyb {

ehyb_status_t cuda_error_status(cudaError_t e, const char* what);
ehyb_status_t device_alloc(void** p, size_t bytes);

namespace {

#define CKS(call)                                                     \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_error_status(e_, #call);       \
  } while (0)

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// fixed-order block sum; result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
  return s;
}

// send[i] = x[idx[i]]
__global__ void pack_kernel(int64_t count, const int32_t* __restrict__ idx, const double* __restrict__ x,
                            double* __restrict__ send) {
  for (int64_t i = gtid(); i < count; i += gstride()) send[i] = __ldg(x + idx[i]);
}

// r = b - q; p = r; partials of r.r (part) and b.b (part + gridDim)
__global__ void init_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ q, double* r,
                            double* p, double* part) {
  double rr = 0.0, bb = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double ri = b[i] - q[i];
    r[i] = ri;
    if (p) p[i] = ri;
    rr = fma(ri, ri, rr);
    bb = fma(b[i], b[i], bb);
  }
  const double s1 = block_sum(rr);
  __syncthreads();
  const double s2 = block_sum(bb);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[gridDim.x + blockIdx.x] = s2;
  }
}

// x += alpha p; r -= alpha q; partials of r.r
__global__ void update_kernel(int64_t n, double alpha, const double* __restrict__ p, const double* __restrict__ q,
                              double* x, double* r, double* part) {
  double rr = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  const double s = block_sum(rr);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// p = r + beta p
__global__ void direction_kernel(int64_t n, double beta, const double* __restrict__ r, double* p) {
  for (int64_t i = gtid(); i < n; i += gstride()) p[i] = fma(beta, p[i], r[i]);
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// partition boundaries of the ranks: contiguous groups with about equal stored slots (slab + sliced ER)
std::vector<int32_t> rank_bounds(const HostPlan& H, int nranks) {
  std::vector<int64_t> w((size_t)H.nparts + 1, 0);
  for (int32_t p = 0; p < H.nparts; ++p) {
    const int32_t s0 = H.slice_ptr[(size_t)p], s1 = H.slice_ptr[(size_t)p + 1];
    w[(size_t)p + 1] = w[(size_t)p] + (H.slice_pos[(size_t)s1] - H.slice_pos[(size_t)s0]) +
                       (H.er_slice_pos[(size_t)s1] - H.er_slice_pos[(size_t)s0]) + 1;
  }
  std::vector<int32_t> b((size_t)nranks + 1, 0);
  b[(size_t)nranks] = H.nparts;
  for (int r = 1; r < nranks; ++r) {
    const int64_t target = (w[(size_t)H.nparts] * r + nranks / 2) / nranks;
    b[(size_t)r] = (int32_t)(std::lower_bound(w.begin(), w.end(), target) - w.begin());
    b[(size_t)r] = std::max(b[(size_t)r], b[(size_t)r - 1]);
  }
  return b;
}

}  // namespace

// halo list of a rank: the distinct ER columns of its slices outside its rows, ascending
static void halo_of(const HostPlan& H, int32_t p0, int32_t p1, int64_t lo, int64_t hi, std::vector<int32_t>& out) {
  out.clear();
  const int64_t e0 = H.er_slice_pos[(size_t)H.slice_ptr[(size_t)p0]];
  const int64_t e1 = H.er_slice_pos[(size_t)H.slice_ptr[(size_t)p1]];
  for (int64_t k = e0; k < e1; ++k) {
    const int32_t c = H.er_scol[(size_t)k];
    if (c < lo || c >= hi) out.push_back(c);
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
}

}  // namespace ehyb

using namespace ehyb;

extern "C" {

ehyb_status_t ehyb_shard_create(ehyb_plan_t plan, int32_t nranks, int32_t rank, void* stream, ehyb_shard_t* out) {
  if (!out) return EHYB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!plan || nranks < 1 || rank < 0 || rank >= nranks) return EHYB_ERR_INVALID_ARG;
  if (plan->er_layout != 0) return EHYB_ERR_UNSUPPORTED;  // the halo is read by the sliced ER part
  if (!plan->host_kept) {                                  // bring the slab / ER arrays back to the host
    ehyb_plan_export_t ex;
    ehyb_status_t st = ehyb_plan_export(plan, &ex);
    if (st != EHYB_OK) return st;
  }
  const HostPlan& H = plan->host;
  std::unique_ptr<ehyb_shard_s> S;
  try {
    S.reset(new ehyb_shard_s());
    S->nranks = nranks;
    S->rank = rank;
    S->host_only = plan->host_only;
    const std::vector<int32_t> b = rank_bounds(H, nranks);
    const int32_t p0 = b[(size_t)rank], p1 = b[(size_t)rank + 1];
    S->p0 = p0;
    S->p1 = p1;
    S->lo = H.part_ptr[(size_t)p0];
    S->hi = H.part_ptr[(size_t)p1];
    const int64_t lo = S->lo, hi = S->hi, nl = hi - lo;
    const int32_t s0 = H.slice_ptr[(size_t)p0], s1 = H.slice_ptr[(size_t)p1];
    // partitions, slices and slots of the shard, rebased
    for (int32_t p = p0; p <= p1; ++p) {
      S->part_ptr.push_back((int32_t)(H.part_ptr[(size_t)p] - lo));
      S->slice_ptr.push_back(H.slice_ptr[(size_t)p] - s0);
    }
    const int64_t pos0 = H.slice_pos[(size_t)s0], epos0 = H.er_slice_pos[(size_t)s0];
    for (int32_t s = s0; s <= s1; ++s) {
      S->slice_pos.push_back(H.slice_pos[(size_t)s] - pos0);
      S->er_slice_pos.push_back(H.er_slice_pos[(size_t)s] - epos0);
    }
    for (int32_t s = s0; s < s1; ++s) S->slice_order.push_back(H.slice_order[(size_t)s] - s0);
    const int64_t pos1 = H.slice_pos[(size_t)s1], epos1 = H.er_slice_pos[(size_t)s1];
    S->ell_col.assign(H.ell_col.begin() + pos0, H.ell_col.begin() + pos1);
    S->ell_val.assign(H.ell_val.begin() + pos0, H.ell_val.begin() + pos1);
    S->er_sval.assign(H.er_sval.begin() + epos0, H.er_sval.begin() + epos1);
    S->new_to_old.assign(H.new_to_old.begin() + lo, H.new_to_old.begin() + hi);
    S->row_ell_count.assign(H.row_ell_count.begin() + lo, H.row_ell_count.begin() + hi);
    S->row_er_count.assign(H.row_er_count.begin() + lo, H.row_er_count.begin() + hi);
    // halo lists of every rank (rank q's list decides what this rank sends to q)
    std::vector<int32_t> hq;
    S->send_ptr.assign((size_t)nranks + 1, 0);
    for (int q = 0; q < nranks; ++q) {
      const int64_t qlo = H.part_ptr[(size_t)b[(size_t)q]], qhi = H.part_ptr[(size_t)b[(size_t)q + 1]];
      halo_of(H, b[(size_t)q], b[(size_t)q + 1], qlo, qhi, hq);
      if (q == rank) {
        S->halo_rows = hq;
      } else {
        auto a = std::lower_bound(hq.begin(), hq.end(), (int32_t)lo);
        auto e = std::lower_bound(hq.begin(), hq.end(), (int32_t)hi);
        for (auto it = a; it != e; ++it) S->send_idx.push_back((int32_t)(*it - lo));
      }
      S->send_ptr[(size_t)q + 1] = (int64_t)S->send_idx.size();
    }
    S->n_halo = (int64_t)S->halo_rows.size();
    S->recv_ptr.assign((size_t)nranks + 1, 0);
    for (int q = 0; q <= nranks; ++q) {
      const int64_t qlo = q < nranks ? H.part_ptr[(size_t)b[(size_t)q]] : H.n;
      S->recv_ptr[(size_t)q] =
          std::lower_bound(S->halo_rows.begin(), S->halo_rows.end(), (int32_t)qlo) - S->halo_rows.begin();
    }
    S->recv_ptr[(size_t)nranks] = S->n_halo;
    // ER columns into x_ext
    S->er_scol.resize((size_t)(epos1 - epos0));
    for (int64_t k = epos0; k < epos1; ++k) {
      const int32_t c = H.er_scol[(size_t)k];
      int64_t v;
      if (c >= lo && c < hi) {
        v = c - lo;
      } else {
        v = nl + (std::lower_bound(S->halo_rows.begin(), S->halo_rows.end(), c) - S->halo_rows.begin());
      }
      S->er_scol[(size_t)(k - epos0)] = (int32_t)v;
    }
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }
  // device view: the plan's launch shape on the shard's arrays
  DevPlan& D = S->dev;
  const DevPlan& PD = plan->dev;
  D.n = S->hi - S->lo;
  D.n_x = D.n + S->n_halo;
  D.nparts = S->p1 - S->p0;
  D.tpr = H.tpr;
  D.er_tpr = PD.er_tpr;
  D.threads = PD.threads;
  D.er_layout = 0;
  D.kbatch = PD.kbatch;
  D.wait_timeout_ns = PD.wait_timeout_ns;
  D.max_part_rows = 0;
  D.max_part_slices = 0;
  for (int32_t p = 0; p < D.nparts; ++p) {
    D.max_part_rows = std::max(D.max_part_rows, S->part_ptr[(size_t)p + 1] - S->part_ptr[(size_t)p]);
    D.max_part_slices = std::max(D.max_part_slices, S->slice_ptr[(size_t)p + 1] - S->slice_ptr[(size_t)p]);
  }
  if (!S->host_only) {
    cudaStream_t s = (cudaStream_t)stream;
    CKS(cudaGetDevice(&S->device));
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t off = 0;
    auto add = [&](size_t bytes) { const size_t o = off; off += al(bytes); return o; };
    const size_t o_n2o = add(S->new_to_old.size() * 4), o_pp = add(S->part_ptr.size() * 4),
                 o_sp = add(S->slice_ptr.size() * 4), o_pos = add(S->slice_pos.size() * 8),
                 o_so = add(S->slice_order.size() * 4), o_ec = add(S->ell_col.size() * 2),
                 o_ev = add(S->ell_val.size() * 8), o_esp = add(S->er_slice_pos.size() * 8),
                 o_esc = add(S->er_scol.size() * 4), o_esv = add(S->er_sval.size() * 8),
                 o_si = add(S->send_idx.size() * 4), o_dot = add(((size_t)D.nparts + 2) * 8), o_arr = add(16),
                 o_st = add(16);
    ehyb_status_t st = device_alloc(&S->arena, off);
    if (st != EHYB_OK) return st;
    char* base = (char*)S->arena;
    cudaError_t e = cudaSuccess;
    auto up = [&](size_t o, const void* src, size_t bytes) {
      if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s);
    };
    up(o_n2o, S->new_to_old.data(), S->new_to_old.size() * 4);
    up(o_pp, S->part_ptr.data(), S->part_ptr.size() * 4);
    up(o_sp, S->slice_ptr.data(), S->slice_ptr.size() * 4);
    up(o_pos, S->slice_pos.data(), S->slice_pos.size() * 8);
    up(o_so, S->slice_order.data(), S->slice_order.size() * 4);
    up(o_ec, S->ell_col.data(), S->ell_col.size() * 2);
    up(o_ev, S->ell_val.data(), S->ell_val.size() * 8);
    up(o_esp, S->er_slice_pos.data(), S->er_slice_pos.size() * 8);
    up(o_esc, S->er_scol.data(), S->er_scol.size() * 4);
    up(o_esv, S->er_sval.data(), S->er_sval.size() * 8);
    up(o_si, S->send_idx.data(), S->send_idx.size() * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_arr, 0, 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_st, 0, 16, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFree(S->arena);
      S->arena = nullptr;
      return cuda_error_status(e, "shard upload");
    }
    D.new_to_old = (const int32_t*)(base + o_n2o);
    D.part_ptr = (const int32_t*)(base + o_pp);
    D.slice_ptr = (const int32_t*)(base + o_sp);
    D.slice_pos = (const int64_t*)(base + o_pos);
    D.slice_order = (const int32_t*)(base + o_so);
    D.ell_col = (const uint16_t*)(base + o_ec);
    D.ell_val = (const double*)(base + o_ev);
    D.er_slice_pos = (const int64_t*)(base + o_esp);
    D.er_scol = (const int32_t*)(base + o_esc);
    D.er_scol_old = D.er_scol;
    D.er_sval = (const double*)(base + o_esv);
    D.status = (int32_t*)(base + o_st);
    S->d_send_idx = (const int32_t*)(base + o_si);
    S->d_dot = (double*)(base + o_dot);
    S->d_arrive = (int32_t*)(base + o_arr);
  }
  *out = S.release();
  return EHYB_OK;
}

ehyb_status_t ehyb_shard_info(ehyb_shard_t sh, ehyb_shard_info_t* info) {
  if (!sh || !info) return EHYB_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->nranks = sh->nranks;
  info->rank = sh->rank;
  info->part_begin = sh->p0;
  info->part_end = sh->p1;
  info->row_begin = sh->lo;
  info->row_end = sh->hi;
  info->n_local = sh->hi - sh->lo;
  info->n_halo = sh->n_halo;
  info->send_total = (int64_t)sh->send_idx.size();
  info->slab_stored = (int64_t)sh->ell_col.size();
  info->er_stored = (int64_t)sh->er_scol.size();
  if (!sh->host_only) {
    CKS(cudaDeviceSynchronize());
    CKS(cudaMemcpy(&info->device_status, sh->dev.status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  }
  return EHYB_OK;
}

ehyb_status_t ehyb_shard_lists(ehyb_shard_t sh, int64_t* send_ptr, int32_t* send_idx, int64_t* recv_ptr,
                               int32_t* halo_rows) {
  if (!sh) return EHYB_ERR_INVALID_ARG;
  const size_t np = (size_t)sh->nranks + 1;
  if (send_ptr) std::memcpy(send_ptr, sh->send_ptr.data(), np * 8);
  if (recv_ptr) std::memcpy(recv_ptr, sh->recv_ptr.data(), np * 8);
  if (send_idx && !sh->send_idx.empty()) std::memcpy(send_idx, sh->send_idx.data(), sh->send_idx.size() * 4);
  if (halo_rows && !sh->halo_rows.empty()) std::memcpy(halo_rows, sh->halo_rows.data(), sh->halo_rows.size() * 4);
  return EHYB_OK;
}

ehyb_status_t ehyb_shard_export(ehyb_shard_t sh, ehyb_plan_export_t* ex) {
  if (!sh || !ex) return EHYB_ERR_INVALID_ARG;
  std::memset(ex, 0, sizeof(*ex));
  ex->n = sh->hi - sh->lo;
  ex->nparts = sh->p1 - sh->p0;
  ex->nslices = (int32_t)sh->slice_order.size();
  ex->tpr = sh->dev.tpr;
  ex->ell_stored = (int64_t)sh->ell_col.size();
  ex->new_to_old = sh->new_to_old.data();
  ex->part_ptr = sh->part_ptr.data();
  ex->slice_ptr = sh->slice_ptr.data();
  ex->slice_pos = sh->slice_pos.data();
  ex->ell_col = sh->ell_col.data();
  ex->ell_val = sh->ell_val.data();
  ex->row_ell_count = sh->row_ell_count.data();
  ex->er_layout = 0;
  ex->er_stored = (int64_t)sh->er_scol.size();
  ex->er_slice_pos = sh->er_slice_pos.data();
  ex->er_scol = sh->er_scol.data();
  ex->er_sval = sh->er_sval.data();
  ex->row_er_count = sh->row_er_count.data();
  return EHYB_OK;
}

ehyb_status_t ehyb_shard_pack(ehyb_shard_t sh, const double* x_local, double* send_buf, void* stream) {
  if (!sh) return EHYB_ERR_INVALID_ARG;
  if (sh->host_only) return EHYB_ERR_UNSUPPORTED;
  const int64_t cnt = (int64_t)sh->send_idx.size();
  if (cnt == 0) return EHYB_OK;
  if (!x_local || !send_buf) return EHYB_ERR_INVALID_ARG;
  const int blocks = (int)std::min<int64_t>(kVB, ceil_div(cnt, kVT));
  pack_kernel<<<blocks, kVT, 0, (cudaStream_t)stream>>>(cnt, sh->d_send_idx, x_local, send_buf);
  CKS(cudaGetLastError());
  return EHYB_OK;
}

ehyb_status_t ehyb_shard_spmv(ehyb_shard_t sh, const double* x_ext, double* y_local, void* stream) {
  if (!sh) return EHYB_ERR_INVALID_ARG;
  if (sh->host_only) return EHYB_ERR_UNSUPPORTED;
  if (sh->dev.nparts == 0) return EHYB_OK;
  if (!x_ext || !y_local || x_ext == y_local) return EHYB_ERR_INVALID_ARG;
  CKS(launch_ehyb_f64(sh->dev, x_ext, y_local, 0, (cudaStream_t)stream));
  return EHYB_OK;
}

ehyb_status_t ehyb_shard_cg(ehyb_shard_t sh, const double* b, double* x, double* p_ext, double* send_buf,
                            double rtol, int32_t max_iter, ehyb_exchange_fn exchange, ehyb_allreduce_fn allreduce,
                            void* ctx, ehyb_cg_info_t* info, void* stream) {
  if (!sh || !info || !exchange || !allreduce) return EHYB_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  if (sh->host_only) return EHYB_ERR_UNSUPPORTED;
  if (!(rtol >= 0.0) || max_iter < 0) return EHYB_ERR_INVALID_ARG;
  const double t0 = now_s();
  const int64_t n = sh->hi - sh->lo, nh = sh->n_halo, ns = (int64_t)sh->send_idx.size();
  if (n > 0 && (!b || !x)) return EHYB_ERR_INVALID_ARG;
  if ((n + nh > 0 && !p_ext) || (ns > 0 && !send_buf)) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // workspace: r, q (n each), 2 x kVB partials
  const size_t need = (size_t)(2 * n + 2 * kVB + 8) * 8;
  if (sh->work_bytes < need) {
    if (sh->work) {
      CKS(cudaDeviceSynchronize());
      cudaFree(sh->work);
      sh->work = nullptr;
      sh->work_bytes = 0;
    }
    ehyb_status_t st = device_alloc((void**)&sh->work, need);
    if (st != EHYB_OK) return st;
    sh->work_bytes = need;
  }
  double* r = sh->work;
  double* q = r + n;
  double* part = q + n;
  double* pe = p_ext;                 // [p | halo of p], the caller's
  double* send = send_buf;
  const int vb = (int)std::max<int64_t>(1, std::min<int64_t>(kVB, ceil_div(n, kVT)));
  std::vector<double> hp((size_t)2 * kVB);
  auto sum_parts = [&](int count, double* out1, double* out2) -> ehyb_status_t {
    CKS(cudaMemcpyAsync(hp.data(), part, (size_t)(out2 ? 2 * count : count) * 8, cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    double a = 0.0, c = 0.0;
    for (int i = 0; i < count; ++i) a += hp[(size_t)i];
    if (out2)
      for (int i = 0; i < count; ++i) c += hp[(size_t)count + i];
    *out1 = a;
    if (out2) *out2 = c;
    return EHYB_OK;
  };
  // q = A v for v = pe[0:n] (its halo fetched first); with dot, also the local v.q
  auto product = [&](double* dot_local) -> ehyb_status_t {
    if (n > 0) {
      ehyb_status_t st = ehyb_shard_pack(sh, pe, send, s);
      if (st != EHYB_OK) return st;
    }
    CKS(cudaStreamSynchronize(s));
    if (exchange(ctx, send, pe + n, s) != 0) return EHYB_ERR_CUDA;
    if (n == 0) {
      if (dot_local) *dot_local = 0.0;
      return EHYB_OK;
    }
    if (dot_local) {
      DotOut dot{sh->d_dot, sh->d_arrive, sh->d_dot + sh->dev.nparts};
      CKS(launch_ehyb_f64(sh->dev, pe, q, 0, s, &dot));
      CKS(cudaMemcpyAsync(dot_local, sh->d_dot + sh->dev.nparts, 8, cudaMemcpyDeviceToHost, s));
      CKS(cudaStreamSynchronize(s));
    } else {
      CKS(launch_ehyb_f64(sh->dev, pe, q, 0, s));
    }
    return EHYB_OK;
  };
  ehyb_status_t st;
  // r = b - A x, p = r
  if (n > 0) CKS(cudaMemcpyAsync(pe, x, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
  if ((st = product(nullptr)) != EHYB_OK) return st;
  double sc[2] = {0.0, 0.0};
  if (n > 0) {
    init_kernel<<<vb, kVT, 0, s>>>(n, b, q, r, pe, part);
    CKS(cudaGetLastError());
    if ((st = sum_parts(vb, &sc[0], &sc[1])) != EHYB_OK) return st;
  }
  if (allreduce(ctx, sc, 2) != 0) return EHYB_ERR_CUDA;
  double rr = sc[0];
  const double bb = sc[1];
  const double bnorm = bb > 0.0 ? std::sqrt(bb) : 1.0;
  const double tol2 = rtol * rtol * bb;
  int it = 0, converged = rr <= tol2 ? 1 : 0;
  while (!converged && it < max_iter) {
    double pq = 0.0;
    if ((st = product(&pq)) != EHYB_OK) return st;
    if (allreduce(ctx, &pq, 1) != 0) return EHYB_ERR_CUDA;
    if (!(pq > 0.0)) break;  // not positive definite along p
    const double alpha = rr / pq;
    double rr_new = 0.0;
    if (n > 0) {
      update_kernel<<<vb, kVT, 0, s>>>(n, alpha, pe, q, x, r, part);
      CKS(cudaGetLastError());
      if ((st = sum_parts(vb, &rr_new, nullptr)) != EHYB_OK) return st;
    }
    if (allreduce(ctx, &rr_new, 1) != 0) return EHYB_ERR_CUDA;
    ++it;
    if (rr_new <= tol2) converged = 1;
    const double beta = rr_new / rr;
    rr = rr_new;
    if (!converged && n > 0) {
      direction_kernel<<<vb, kVT, 0, s>>>(n, beta, r, pe);
      CKS(cudaGetLastError());
    }
  }
  info->relres_recursive = std::sqrt(rr) / bnorm;
  // true residual
  if (n > 0) CKS(cudaMemcpyAsync(pe, x, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
  if ((st = product(nullptr)) != EHYB_OK) return st;
  sc[0] = sc[1] = 0.0;
  if (n > 0) {
    init_kernel<<<vb, kVT, 0, s>>>(n, b, q, r, nullptr, part);
    CKS(cudaGetLastError());
    if ((st = sum_parts(vb, &sc[0], &sc[1])) != EHYB_OK) return st;
  }
  if (allreduce(ctx, sc, 1) != 0) return EHYB_ERR_CUDA;
  info->relres = std::sqrt(sc[0]) / bnorm;
  info->iterations = it;
  info->converged = converged;
  info->seconds = now_s() - t0;
  int32_t dev_status = 0;
  CKS(cudaMemcpy(&dev_status, sh->dev.status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (dev_status) return (ehyb_status_t)dev_status;
  return converged ? EHYB_OK : EHYB_ERR_NOT_CONVERGED;
}

ehyb_status_t ehyb_shard_destroy(ehyb_shard_t sh) {
  if (!sh) return EHYB_OK;
  ehyb_status_t st = EHYB_OK;
  if (sh->arena || sh->work) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_error_status(e, "cudaDeviceSynchronize");
    if (sh->arena) cudaFree(sh->arena);
    if (sh->work) cudaFree(sh->work);
  }
  delete sh;
  return st;
}

}  // extern "C"
