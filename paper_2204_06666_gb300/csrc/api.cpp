// C ABI of the EHYB library (declared in include/ehyb.h): argument validation, option
// resolution (Eq. 1 default for VecSize), host planning, upload, kernel launches, profiling.
#include "../../include/ehyb.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "device.h"
#include "plan.h"
#include "plan_internal.h"

using namespace ehyb;

namespace {

thread_local std::string g_cuda_err;
int g_fail_allocs_after = -1;  // test hook: >= 0 makes that many successful device allocations, then fail

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

ehyb_status_t cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  g_cuda_err = buf;
  return EHYB_ERR_CUDA;
}

#define CK(call)                                                      \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);               \
  } while (0)

ehyb_status_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return EHYB_OK;
  if (g_fail_allocs_after == 0) return EHYB_ERR_OOM;
  if (g_fail_allocs_after > 0) --g_fail_allocs_after;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return EHYB_ERR_OOM;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  return EHYB_OK;
}

bool is_pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

int pow2_near(double v) {  // power of two nearest to v in [1, 32]
  int p = 1;
  while (p < 32 && (double)p * 1.41421356 < v) p <<= 1;
  return p;
}

struct DeviceInfo {
  int dev = -1, sms = 0, smem_optin = 0;
};

ehyb_status_t query_device(DeviceInfo& d) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    return EHYB_ERR_NO_DEVICE;
  }
  CK(cudaGetDevice(&d.dev));
  CK(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, d.dev));
  CK(cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d.dev));
  static int inited_dev[64] = {0};
  if (d.dev >= 0 && d.dev < 64 && !inited_dev[d.dev]) {
    CK(kernels_init(d.smem_optin - 1024));  // static shared memory and alignment slack stay outside
    inited_dev[d.dev] = 1;
  }
  return EHYB_OK;
}

// 256-byte aligned sub-allocations of one device arena
struct Arena {
  size_t size = 0;
  template <typename T>
  size_t add(size_t count) {
    size_t off = size;
    size += ((count * sizeof(T)) + 255) & ~(size_t)255;
    return off;
  }
};

ehyb_status_t validate_csr(int64_t nr, int64_t nc, int64_t nnz, const int64_t* rp, const int32_t* col,
                           const double* val) {
  if (nr < 0 || nc < 0 || nnz < 0) return EHYB_ERR_INVALID_ARG;
  if (nr != nc) return EHYB_ERR_NOT_SQUARE;
  if (nr >= (int64_t)INT32_MAX - 1) return EHYB_ERR_TOO_LARGE;
  if (!rp) return EHYB_ERR_INVALID_ARG;
  if (nnz > 0 && (!col || !val)) return EHYB_ERR_INVALID_ARG;
  if (rp[0] != 0 || rp[nr] != nnz) return EHYB_ERR_INDEX_RANGE;
  // both scans run in parallel pieces, each piece folding its violations into one flag (no early exit, so
  // the compare loops vectorise)
  std::atomic<int> bad{0};
  ehyb::parallel_for(nr, ehyb::planner_threads(0), [&](int64_t lo, int64_t hi) {
    int b = 0;
    for (int64_t i = lo; i < hi; ++i) b |= rp[i + 1] < rp[i];
    if (b) bad.store(1);
  }, 1 << 16);
  ehyb::parallel_for(nnz, ehyb::planner_threads(0), [&](int64_t lo, int64_t hi) {
    int b = 0;
    for (int64_t k = lo; k < hi; ++k) b |= (uint32_t)col[k] >= (uint64_t)nc;
    if (b) bad.store(1);
  }, 1 << 18);
  return bad.load() ? EHYB_ERR_INDEX_RANGE : EHYB_OK;
}

}  // namespace

struct ehyb_csr_s {
  int64_t n = 0, nnz = 0;
  int32_t tpr = 1;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};

namespace ehyb {
ehyb_status_t cuda_error_status(cudaError_t e, const char* what) { return cuda_fail(e, what); }
ehyb_status_t check_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* rp, const int32_t* col,
                        const double* val) {
  return validate_csr(n_rows, n_cols, nnz, rp, col, val);
}
ehyb_status_t device_query(int* dev, int* sms, int* smem_optin) {
  DeviceInfo d;
  ehyb_status_t st = query_device(d);
  if (st != EHYB_OK) return st;
  *dev = d.dev;
  *sms = d.sms;
  *smem_optin = d.smem_optin;
  return EHYB_OK;
}
ehyb_status_t device_alloc(void** p, size_t bytes) { return dev_alloc(p, bytes); }

// device view of a plan for entry points defined in other translation units
const DevPlan* plan_device_view(ehyb_plan_t plan, int* device) {
  if (!plan || plan->host_only) return nullptr;
  if (device) *device = plan->device;
  return &plan->dev;
}
}  // namespace ehyb

extern "C" {

const char* ehyb_status_string(ehyb_status_t s) {
  switch (s) {
    case EHYB_OK: return "ok";
    case EHYB_ERR_INVALID_ARG: return "invalid argument";
    case EHYB_ERR_NOT_SQUARE: return "matrix is not square";
    case EHYB_ERR_INDEX_RANGE: return "row pointer or column index out of range";
    case EHYB_ERR_TOO_LARGE: return "matrix or partition too large";
    case EHYB_ERR_OOM: return "out of memory";
    case EHYB_ERR_CUDA: return "CUDA error";
    case EHYB_ERR_UNSUPPORTED: return "unsupported for this plan";
    case EHYB_ERR_NOT_CONVERGED: return "not converged";
    case EHYB_ERR_TIMEOUT: return "device wait timed out";
    case EHYB_ERR_NO_DEVICE: return "no CUDA device";
    case EHYB_ERR_IO: return "plan file unreadable, unwritable or invalid";
    case EHYB_ERR_BOUNDS: return "device-side bounds check failed (checked build)";
  }
  return "unknown status";
}

const char* ehyb_last_cuda_error(void) { return g_cuda_err.c_str(); }

void ehyb_options_default(ehyb_options_t* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
}

// test hook (host-side fault injection): allow `count` more device allocations, then fail with
// EHYB_ERR_OOM; a negative count disables the hook.
void ehyb_test_fail_allocs_after(int32_t count) { g_fail_allocs_after = count; }

ehyb_status_t ehyb_plan_create_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                                   const int32_t* col, const double* val, const ehyb_options_t* opt_in,
                                   void* stream, ehyb_plan_t* out) {
  if (!out) return EHYB_ERR_INVALID_ARG;
  *out = nullptr;
  ehyb_status_t st = validate_csr(n_rows, n_cols, nnz, row_ptr, col, val);
  if (st != EHYB_OK) return st;
  ehyb_options_t opt;
  ehyb_options_default(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.ell_tpr == 0) opt.ell_tpr = 1;
  if (!is_pow2_in(opt.ell_tpr, 1, 32)) return EHYB_ERR_INVALID_ARG;
  if (opt.er_tpr != 0 && !is_pow2_in(opt.er_tpr, 1, 32)) return EHYB_ERR_INVALID_ARG;
  if (opt.block_threads != 0 && (opt.block_threads < 32 || opt.block_threads > 1024 || opt.block_threads % 32))
    return EHYB_ERR_INVALID_ARG;
  if (opt.er_layout < 0 || opt.er_layout > 2) return EHYB_ERR_INVALID_ARG;
  if (opt.lowp_group != 0 && opt.lowp_group != 1 && opt.lowp_group != 4) return EHYB_ERR_INVALID_ARG;
  if (opt.spmm_rhs < 0) return EHYB_ERR_INVALID_ARG;
  if (opt.slice_rows < 0 || opt.ell_width_cap < 0 || opt.lowp < 0 || opt.lowp > 2 || opt.smem_budget < 0 ||
      opt.part_nnz < 0 || opt.host_threads < 0 || opt.partitioner < 0 || opt.partitioner > 1 ||
      opt.num_sms < 0 || opt.wait_timeout_ns < 0)
    return EHYB_ERR_INVALID_ARG;
  if (opt.slice_rows > 65536) return EHYB_ERR_TOO_LARGE;
  const int64_t n = n_rows;
  if (opt.part_vec)
    for (int64_t i = 0; i < n; ++i)
      if (opt.part_vec[i] < 0 || opt.part_vec[i] >= INT32_MAX - 1) return EHYB_ERR_INVALID_ARG;

  DeviceInfo d;
  if (!opt.host_only) {
    st = query_device(d);
    if (st != EHYB_OK) return st;
  } else {
    d.sms = opt.num_sms > 0 ? opt.num_sms : 152;
    d.smem_optin = 232448;
  }
  const int64_t budget = opt.smem_budget > 0 ? opt.smem_budget : (int64_t)d.smem_optin - 1024;
  if (opt.num_sms > 0) d.sms = opt.num_sms;
  if (opt.tuner < 0 || opt.tuner > 2) return EHYB_ERR_INVALID_ARG;
  const bool knobs_free = opt.slice_rows == 0 && opt.ell_width_cap == 0 && opt.ell_tpr == 1 && !opt.part_vec &&
                          opt.part_nnz == 0 && opt.er_layout == 0;
  int32_t tuner_path = 0;
  double pred_ns = 0.0;
  if (opt.tuner && knobs_free && !opt.host_only && n > 0) {
    if (opt.tuner == 1) {
      int32_t sr = 0, cap = 0, tpr = 1;
      st = learned_choice(n, row_ptr, col, val, d.sms, d.smem_optin, &sr, &cap, &tpr, &pred_ns);
      if (st == EHYB_OK) {
        opt.slice_rows = sr;
        opt.ell_width_cap = cap;
        opt.ell_tpr = tpr;
        tuner_path = 1;
      } else if (st != EHYB_ERR_UNSUPPORTED) {
        return st;
      }
    }
    if (tuner_path == 0) {  // the sweep decides (asked for, or no model loaded)
      std::vector<ehyb_tune_entry_t> table((size_t)ehyb_tune_grid_size());
      int32_t best = -1;
      ehyb_plan_t bp = nullptr;
      ehyb_options_t base = opt;
      base.tuner = 0;
      st = sweep_impl(n, row_ptr, col, val, base, 10, table.data(), &best, &bp, stream);
      if (st != EHYB_OK) return st;
      bp->tuner_path = 2;
      bp->ell_width_cap = table[best].ell_width_cap;
      *out = bp;
      return EHYB_OK;
    }
  }

  std::unique_ptr<ehyb_plan_s> P;
  try {
    P.reset(new ehyb_plan_s());
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }
  PlanParams prm;
  prm.n = n;
  // Eq. 1 / Eq. 2 with tau = 8 (FP64 x slice), keeping 32 bytes of rounding and alignment slack
  // Eq. 1's tau: 8 bytes of x per row, or 8 KC for the KC columns of X one SpMM chunk stages per row (a row of
  // slack per chunk column kept out of the budget)
  int kc = 1;
  for (int c : {8, 4, 2})
    if (opt.spmm_rhs > 1 && opt.spmm_rhs % c == 0) { kc = c; break; }
  prm.slice_rows = opt.slice_rows > 0 ? opt.slice_rows : eq1_slice_rows(n, 8 * kc, d.sms, budget - 32 - 16 * kc);
  if (opt.slice_rows == 0 && opt.part_nnz > 0 && n > 0) {  // size partitions by work instead
    const int64_t max_rows = std::min<int64_t>(65536, (budget - 32) / 8 - 2);
    const int64_t rows = nnz > 0 ? ((int64_t)opt.part_nnz * n + nnz - 1) / nnz : n;
    prm.slice_rows = (int32_t)std::max<int64_t>(1, std::min<int64_t>(rows, max_rows));
  }
  prm.ell_width_cap = opt.ell_width_cap;
  prm.ell_tpr = opt.ell_tpr;
  prm.lowp = opt.lowp;
  prm.lowp_group = opt.lowp_group;
  prm.er_layout = opt.er_layout;
  prm.part_vec = opt.part_vec;
  prm.threads = opt.host_threads;
  prm.partitioner = opt.partitioner;
  prm.seed = opt.seed;
  HostPlan& H = P->host;
  try {
    int rc = build_plan(prm, row_ptr, col, val, H);
    if (rc != 0) return (ehyb_status_t)rc;
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }
  // every partition's slice of x (and its halo in er_layout 2; FP64, plus 16-byte alignment slack) must fit
  // one block's dynamic shared memory
  if ((int64_t)(std::max(H.max_part_rows, H.max_stage_rows) + 2) * 8 > (int64_t)d.smem_optin - 1024)
    return EHYB_ERR_TOO_LARGE;

  st = plan_finalize(P, opt, d.dev, d.sms, stream, out);
  if (st != EHYB_OK) return st;
  (*out)->tuner_path = tuner_path;
  (*out)->ell_width_cap = opt.ell_width_cap;
  if (tuner_path == 1) {  // sanity gate: the learned choice must run within 2x of its own prediction
    double ms = 0.0;
    st = measure_plan_ms(*out, 5, stream, &ms);
    if (st != EHYB_OK) return st;
    const double ns_per_nnz = nnz > 0 ? ms * 1e6 / (double)nnz : 0.0;
    if (ns_per_nnz > 2.0 * pred_ns) {
      ehyb_destroy(*out);
      *out = nullptr;
      std::vector<ehyb_tune_entry_t> table((size_t)ehyb_tune_grid_size());
      int32_t best = -1;
      ehyb_options_t base = opt;
      base.tuner = 0;
      base.slice_rows = 0;
      base.ell_width_cap = 0;
      base.ell_tpr = 1;
      st = sweep_impl(n, row_ptr, col, val, base, 10, table.data(), &best, out, stream);
      if (st != EHYB_OK) return st;
      (*out)->tuner_path = 3;
      (*out)->ell_width_cap = table[best].ell_width_cap;
    }
  }
  return EHYB_OK;
}
}  // extern "C"

namespace ehyb {

// Everything after the host build: metadata, launch defaults, device upload, dropping bulky host arrays.
ehyb_status_t plan_finalize(std::unique_ptr<ehyb_plan_s>& P, const ehyb_options_t& opt_in, int dev, int sms,
                            void* stream, ehyb_plan_t* out) {
  ehyb_options_t opt = opt_in;
  HostPlan& H = P->host;
  const int64_t n = H.n;
  struct { int dev, sms; } d{dev, sms};
  ehyb_status_t st = EHYB_OK;
  P->host_only = opt.host_only != 0;
  P->lowp = opt.lowp;
  P->num_sms = d.sms;
  P->slice_rows = H.slice_rows;
  P->ell_nnz = H.ell_nnz;
  P->ell_stored = (int64_t)H.ell_col.size();
  P->er_rows = 0;
  for (int64_t r = 0; r < n; ++r) P->er_rows += H.row_er_count[(size_t)r] > 0;
  P->er_nnz = H.er_nnz;
  P->er_stored = H.er_layout == 0 ? (int64_t)H.er_scol.size() : H.er_layout == 1 ? H.er_nnz : 0;
  P->er_layout = H.er_layout;
  P->nslices = H.nslices;
  if (opt.er_tpr) {
    P->er_tpr = opt.er_tpr;
  } else {
    double mean = P->er_rows ? (double)P->er_nnz / (double)P->er_rows : 1.0;
    P->er_tpr = pow2_near(mean / 6.0);
  }
  DevPlan& D = P->dev;
  D.n = n;
  D.nparts = H.nparts;
  D.tpr = H.tpr;
  D.er_tpr = P->er_tpr;
  if (opt.block_threads == 0) {  // enough warps for the average partition's slices
    const int64_t per_part = H.nparts ? ((int64_t)H.nslices + H.nparts - 1) / H.nparts : 1;
    opt.block_threads = (int32_t)std::min<int64_t>(1024, std::max<int64_t>(128, 32 * per_part));
  }
  D.threads = opt.block_threads;
  D.er_layout = H.er_layout;
  D.max_part_rows = H.max_part_rows;
  D.max_stage_rows = H.max_stage_rows;
  D.max_part_slices = 0;
  for (int32_t p = 0; p < H.nparts; ++p)
    D.max_part_slices = std::max(D.max_part_slices, H.slice_ptr[(size_t)p + 1] - H.slice_ptr[(size_t)p]);
  {  // batch depth: mean slab + sliced-ER slots per lane of a slice (measured: 6 is faster from about 32 up)
    const double w = mean_slice_width(H);
    D.kbatch = (H.er_layout == 0 && w >= 32.0) ? 6 : 8;
  }
  D.wait_timeout_ns = opt.wait_timeout_ns > 0 ? (uint64_t)opt.wait_timeout_ns : 1000000000ull;
  D.inject_wait_fault = opt.inject_wait_fault;

  if (!P->host_only) {
    const double t0 = now_ms();
    P->device = d.dev;
    cudaStream_t s = (cudaStream_t)stream;
    Arena A;
    const size_t o_n2o = A.add<int32_t>((size_t)n);
    const size_t o_pp = A.add<int32_t>(H.part_ptr.size());
    const size_t o_sp = A.add<int32_t>(H.slice_ptr.size());
    const size_t o_pos = A.add<int64_t>(H.slice_pos.size());
    const size_t o_ec = A.add<uint16_t>(H.ell_col.size());
    const size_t o_ev = A.add<double>(H.ell_val.size());
    const size_t o_ev32 = A.add<float>(H.ell_val_f32.size());
    const size_t o_ev16 = A.add<uint16_t>(H.ell_val_bf16.size());
    const size_t o_epp = A.add<int32_t>(H.er_part_ptr.size());
    const size_t o_er = A.add<int32_t>(H.er_row.size());
    const size_t o_erp = A.add<int64_t>(H.er_ptr.size());
    const size_t o_erc = A.add<int32_t>(H.er_col.size());
    const size_t o_erv = A.add<double>(H.er_val.size());
    const size_t o_erv32 = A.add<float>(H.er_val_f32.size());
    const size_t o_erv16 = A.add<uint16_t>(H.er_val_bf16.size());
    const size_t o_esp = A.add<int64_t>(H.er_slice_pos.size());
    const size_t o_so = A.add<int32_t>(H.slice_order.size());
    const size_t o_esc = A.add<int32_t>(H.er_scol.size());
    const size_t o_eso = A.add<int32_t>(H.er_scol_old.size());
    const size_t o_esv = A.add<double>(H.er_sval.size());
    const size_t o_esv32 = A.add<float>(H.er_sval_f32.size());
    const size_t o_esv16 = A.add<uint16_t>(H.er_sval_bf16.size());
    const size_t o_ecl = A.add<uint16_t>(H.ell_col_low.size());
    const size_t o_escl = A.add<int32_t>(H.er_scol_low.size());
    const size_t o_esol = A.add<int32_t>(H.er_scol_old_low.size());
    const size_t o_hp = A.add<int64_t>(H.halo_ptr.size());
    const size_t o_hn = A.add<int32_t>(H.halo_new.size());
    const size_t o_ho = A.add<int32_t>(H.halo_old.size());
    const size_t o_xp = A.add<double>((size_t)n + 2);
    const size_t o_xp32 = A.add<float>((size_t)n + 4);
    const size_t o_st = A.add<int32_t>(4);
    st = dev_alloc(&P->arena, A.size);
    if (st != EHYB_OK) return st;
    P->arena_bytes = A.size;
    char* base = (char*)P->arena;
    auto up = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
      if (bytes == 0) return cudaSuccess;
      return cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s);
    };
    cudaError_t e = cudaSuccess;
#define UP(off, vec)                                                                  \
  if (e == cudaSuccess) e = up(off, vec.data(), vec.size() * sizeof(vec[0]));
    UP(o_n2o, H.new_to_old) UP(o_pp, H.part_ptr) UP(o_sp, H.slice_ptr) UP(o_pos, H.slice_pos) UP(o_ec, H.ell_col)
    UP(o_ev, H.ell_val) UP(o_ev32, H.ell_val_f32) UP(o_ev16, H.ell_val_bf16) UP(o_epp, H.er_part_ptr)
    UP(o_er, H.er_row) UP(o_erp, H.er_ptr) UP(o_erc, H.er_col) UP(o_erv, H.er_val) UP(o_erv32, H.er_val_f32)
    UP(o_erv16, H.er_val_bf16) UP(o_esp, H.er_slice_pos) UP(o_so, H.slice_order) UP(o_esc, H.er_scol) UP(o_eso, H.er_scol_old) UP(o_esv, H.er_sval)
    UP(o_esv32, H.er_sval_f32) UP(o_esv16, H.er_sval_bf16) UP(o_ecl, H.ell_col_low) UP(o_escl, H.er_scol_low)
    UP(o_esol, H.er_scol_old_low) UP(o_hp, H.halo_ptr) UP(o_hn, H.halo_new) UP(o_ho, H.halo_old)
#undef UP
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_st, 0, 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_xp, 0, ((size_t)n + 2) * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFree(P->arena);
      P->arena = nullptr;
      return cuda_fail(e, "plan upload");
    }
    D.new_to_old = (const int32_t*)(base + o_n2o);
    D.part_ptr = (const int32_t*)(base + o_pp);
    D.slice_ptr = (const int32_t*)(base + o_sp);
    D.slice_pos = (const int64_t*)(base + o_pos);
    D.ell_col = (const uint16_t*)(base + o_ec);
    D.ell_val = (const double*)(base + o_ev);
    D.ell_val_f32 = (const float*)(base + o_ev32);
    D.ell_val_bf16 = (const uint16_t*)(base + o_ev16);
    D.er_part_ptr = (const int32_t*)(base + o_epp);
    D.er_row = (const int32_t*)(base + o_er);
    D.er_ptr = (const int64_t*)(base + o_erp);
    D.er_col = (const int32_t*)(base + o_erc);
    D.er_val = (const double*)(base + o_erv);
    D.er_val_f32 = (const float*)(base + o_erv32);
    D.er_val_bf16 = (const uint16_t*)(base + o_erv16);
    D.er_slice_pos = (const int64_t*)(base + o_esp);
    D.slice_order = (const int32_t*)(base + o_so);
    D.er_scol = (const int32_t*)(base + o_esc);
    D.er_scol_old = (const int32_t*)(base + o_eso);
    D.er_sval = (const double*)(base + o_esv);
    D.er_sval_f32 = (const float*)(base + o_esv32);
    D.er_sval_bf16 = (const uint16_t*)(base + o_esv16);
    D.status = (int32_t*)(base + o_st);
    D.halo_ptr = (const int64_t*)(base + o_hp);
    D.halo_new = (const int32_t*)(base + o_hn);
    D.halo_old = (const int32_t*)(base + o_ho);
    D.lowp_group = H.lowp_group;
    D.ell_col_low = H.lowp_group == 1 ? D.ell_col : (const uint16_t*)(base + o_ecl);
    D.er_scol_low = H.lowp_group == 1 ? D.er_scol : (const int32_t*)(base + o_escl);
    D.er_scol_old_low = H.lowp_group == 1 ? D.er_scol_old : (const int32_t*)(base + o_esol);
    P->xp = (double*)(base + o_xp);
    P->xp32 = (float*)(base + o_xp32);
    P->upload_ms = now_ms() - t0;
  }
  P->host_kept = P->host_only || opt.keep_host;
  if (!P->host_kept) {  // keep metadata, drop the bulky arrays
    HostPlan& h = P->host;
    auto drop = [](auto& v) { std::decay_t<decltype(v)>().swap(v); };
    drop(h.ell_col);
    drop(h.ell_val);
    drop(h.ell_val_f32);
    drop(h.ell_val_bf16);
    drop(h.er_col);
    drop(h.er_val);
    drop(h.er_val_f32);
    drop(h.er_val_bf16);
    drop(h.er_scol);
    drop(h.er_scol_old);
    drop(h.er_sval);
    drop(h.er_sval_f32);
    drop(h.er_sval_bf16);
    drop(h.ell_col_low);
    drop(h.er_scol_low);
    drop(h.er_scol_old_low);
    std::vector<int32_t>().swap(h.old_to_new);
  }
  *out = P.release();
  return EHYB_OK;
}

}  // namespace ehyb

extern "C" {

ehyb_status_t ehyb_destroy(ehyb_plan_t p) {
  if (!p) return EHYB_OK;
  ehyb_status_t st = EHYB_OK;
  if (p->arena || p->hx || p->cg || p->spmm_ws || !p->ev_pool.empty() || p->px[0] || p->s_in) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "cudaDeviceSynchronize");
    if (p->arena) cudaFree(p->arena);
    if (p->hx) cudaFree(p->hx);
    if (p->hy) cudaFree(p->hy);
    for (int b = 0; b < 2; ++b) {
      if (p->px[b]) cudaFree(p->px[b]);
      if (p->py[b]) cudaFree(p->py[b]);
      if (p->ev_in[b]) cudaEventDestroy(p->ev_in[b]);
      if (p->ev_k[b]) cudaEventDestroy(p->ev_k[b]);
      if (p->ev_out[b]) cudaEventDestroy(p->ev_out[b]);
    }
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    if (p->cg) cg_work_free(p->cg);
    if (p->spmm_ws) cudaFree(p->spmm_ws);
    for (auto& ev : p->ev_pool) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
  }
  delete p;
  return st;
}

static ehyb_status_t record_begin(ehyb_plan_t p, cudaStream_t s, std::pair<cudaEvent_t, cudaEvent_t>** slot) {
  *slot = nullptr;
  if (!p->prof) return EHYB_OK;
  if (p->ev_used == p->ev_pool.size()) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    p->ev_pool.emplace_back(a, b);
  }
  *slot = &p->ev_pool[p->ev_used++];
  CK(cudaEventRecord((*slot)->first, s));
  return EHYB_OK;
}

static ehyb_status_t record_end(std::pair<cudaEvent_t, cudaEvent_t>* slot, cudaStream_t s) {
  if (slot) CK(cudaEventRecord(slot->second, s));
  return EHYB_OK;
}

static ehyb_status_t check_run(ehyb_plan_t p) {
  if (!p) return EHYB_ERR_INVALID_ARG;
  if (p->host_only) return EHYB_ERR_UNSUPPORTED;
  return EHYB_OK;
}

ehyb_status_t ehyb_spmv_permuted(ehyb_plan_t p, const double* xp, double* yp, void* stream) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  if (p->dev.n == 0) return EHYB_OK;
  if (!xp || !yp || xp == yp) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::pair<cudaEvent_t, cudaEvent_t>* slot;
  if ((st = record_begin(p, s, &slot)) != EHYB_OK) return st;
  CK(launch_ehyb_f64(p->dev, xp, yp, 0, s));
  return record_end(slot, s);
}

ehyb_status_t ehyb_spmv(ehyb_plan_t p, const double* x, double* y, void* stream) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  if (p->dev.n == 0) return EHYB_OK;
  if (!x || !y || x == y) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::pair<cudaEvent_t, cudaEvent_t>* slot;
  if (p->dev.er_layout != 1) {  // one launch: the permutation of x is fused into the kernel's loads
    if ((st = record_begin(p, s, &slot)) != EHYB_OK) return st;
    CK(launch_ehyb_f64(p->dev, x, y, 2, s));
    return record_end(slot, s);
  }
  CK(launch_permute_f64(p->dev, 1, x, p->xp, s));
  if ((st = record_begin(p, s, &slot)) != EHYB_OK) return st;
  CK(launch_ehyb_f64(p->dev, p->xp, y, 1, s));
  return record_end(slot, s);
}

ehyb_status_t ehyb_permute(ehyb_plan_t p, int32_t to_new, const double* in, double* out, void* stream) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  if (p->dev.n == 0) return EHYB_OK;
  if (!in || !out || in == out) return EHYB_ERR_INVALID_ARG;
  CK(launch_permute_f64(p->dev, to_new ? 1 : 0, in, out, (cudaStream_t)stream));
  return EHYB_OK;
}

ehyb_status_t ehyb_spmv_host(ehyb_plan_t p, const double* xh, double* yh, void* stream) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  if (p->dev.n == 0) return EHYB_OK;
  if (!xh || !yh) return EHYB_ERR_INVALID_ARG;
  const size_t bytes = (size_t)p->dev.n * sizeof(double);
  if (!p->hx) {
    if ((st = dev_alloc((void**)&p->hx, bytes)) != EHYB_OK) return st;
    if ((st = dev_alloc((void**)&p->hy, bytes)) != EHYB_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(p->hx, xh, bytes, cudaMemcpyHostToDevice, s));
  if ((st = ehyb_spmv(p, p->hx, p->hy, stream)) != EHYB_OK) {
    (void)cudaStreamSynchronize(s);  // the copy of x has finished reading the caller's buffer
    return st;
  }
  CK(cudaMemcpyAsync(yh, p->hy, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return EHYB_OK;
}

ehyb_status_t ehyb_spmv_host_many(ehyb_plan_t p, int32_t count, const double* const* xh, double* const* yh,
                                  void* stream) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  if (count < 0 || (count > 0 && (!xh || !yh))) return EHYB_ERR_INVALID_ARG;
  for (int32_t i = 0; i < count; ++i)
    if (!xh[i] || !yh[i]) return EHYB_ERR_INVALID_ARG;
  if (p->dev.n == 0 || count == 0) return EHYB_OK;
  const size_t bytes = (size_t)p->dev.n * sizeof(double);
  if (!p->s_in) {  // first use: two buffer pairs, two copy streams, six events
    for (int b = 0; b < 2; ++b) {
      if ((st = dev_alloc((void**)&p->px[b], bytes)) != EHYB_OK) return st;
      if ((st = dev_alloc((void**)&p->py[b], bytes)) != EHYB_OK) return st;
      CK(cudaEventCreateWithFlags(&p->ev_in[b], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&p->ev_k[b], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&p->ev_out[b], cudaEventDisableTiming));
    }
    CK(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
  }
  cudaStream_t s = (cudaStream_t)stream;
  // one step's enqueues; on a failure every stream is drained before returning, so no copy is still in
  // flight to or from the caller's host buffers
  auto step = [&](int32_t i) -> ehyb_status_t {
    const int b = i & 1;
    if (i >= 2) CK(cudaStreamWaitEvent(p->s_in, p->ev_k[b], 0));  // product i-2 has read px[b]
    CK(cudaMemcpyAsync(p->px[b], xh[i], bytes, cudaMemcpyHostToDevice, p->s_in));
    CK(cudaEventRecord(p->ev_in[b], p->s_in));
    CK(cudaStreamWaitEvent(s, p->ev_in[b], 0));
    if (i >= 2) CK(cudaStreamWaitEvent(s, p->ev_out[b], 0));  // y of step i-2 has left py[b]
    const ehyb_status_t r = ehyb_spmv(p, p->px[b], p->py[b], stream);
    if (r != EHYB_OK) return r;
    CK(cudaEventRecord(p->ev_k[b], s));
    CK(cudaStreamWaitEvent(p->s_out, p->ev_k[b], 0));
    CK(cudaMemcpyAsync(yh[i], p->py[b], bytes, cudaMemcpyDeviceToHost, p->s_out));
    CK(cudaEventRecord(p->ev_out[b], p->s_out));
    return EHYB_OK;
  };
  for (int32_t i = 0; i < count && st == EHYB_OK; ++i) st = step(i);
  const cudaError_t e1 = cudaStreamSynchronize(p->s_in);
  const cudaError_t e2 = cudaStreamSynchronize(p->s_out);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (st != EHYB_OK) return st;
  if (e1 != cudaSuccess) return cuda_fail(e1, "cudaStreamSynchronize");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize");
  if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamSynchronize");
  return EHYB_OK;
}

ehyb_status_t ehyb_spmv_lowp(ehyb_plan_t p, const float* x, float* y, void* stream) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  if (p->lowp == 0) return EHYB_ERR_UNSUPPORTED;
  if (p->dev.n == 0) return EHYB_OK;
  if (!x || !y || x == y) return EHYB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::pair<cudaEvent_t, cudaEvent_t>* slot;
  if (p->dev.er_layout != 1) {
    if ((st = record_begin(p, s, &slot)) != EHYB_OK) return st;
    CK(launch_ehyb_lowp(p->dev, p->lowp, x, y, 2, s));
    return record_end(slot, s);
  }
  CK(launch_permute_f32(p->dev, 1, x, p->xp32, s));
  if ((st = record_begin(p, s, &slot)) != EHYB_OK) return st;
  CK(launch_ehyb_lowp(p->dev, p->lowp, p->xp32, y, 1, s));
  return record_end(slot, s);
}

ehyb_status_t ehyb_plan_check(ehyb_plan_t p) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  CK(cudaDeviceSynchronize());
  int32_t w = 0;
  CK(cudaMemcpy(&w, p->dev.status, sizeof(w), cudaMemcpyDeviceToHost));
  if (w) CK(cudaMemset(p->dev.status, 0, sizeof(int32_t)));
  return (ehyb_status_t)w;
}

ehyb_status_t ehyb_plan_info(ehyb_plan_t p, ehyb_plan_info_t* info) {
  if (!p || !info) return EHYB_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  const HostPlan& H = p->host;
  info->n = H.n;
  info->nnz = H.nnz;
  info->nparts = H.nparts;
  info->nslices = p->nslices;
  info->slice_rows = p->slice_rows;
  info->ell_tpr = H.tpr;
  info->er_tpr = p->er_tpr;
  info->block_threads = p->dev.threads;
  info->smem_bytes = (int32_t)ehyb_smem_bytes(p->dev, 8);
  info->lowp = p->lowp;
  info->ell_nnz = p->ell_nnz;
  info->ell_stored = p->ell_stored;
  info->er_rows = p->er_rows;
  info->er_nnz = p->er_nnz;
  // values + column indices + x + y; the CSR layout also reads yIdxER and a line offset per ER line; the
  // halo layout reads 16-bit columns for the ER entries and a column and an x value per halo entry
  const int64_t n_halo = H.halo_ptr.empty() ? 0 : H.halo_ptr.back();
  info->bytes_effective = p->er_layout == 2
                              ? p->ell_nnz * 10 + p->er_nnz * 10 + n_halo * 12 + H.n * 16
                              : p->ell_nnz * 10 + p->er_nnz * 12 + (p->er_layout == 1 ? p->er_rows * 8 : 0) + H.n * 16;
  info->max_stage_rows = std::max(H.max_part_rows, H.max_stage_rows);
  info->n_halo = n_halo;
  info->er_layout = p->er_layout;
  info->er_stored = p->er_stored;
  info->tuner_path = p->tuner_path;
  info->ell_width_cap = p->ell_width_cap;
  info->lowp_group = H.lowp_group;
  info->bytes_device = (int64_t)p->arena_bytes;
  info->partition_ms = H.partition_ms;
  info->reorder_ms = H.reorder_ms;
  info->upload_ms = p->upload_ms;
  info->num_sms = p->num_sms;
  if (!p->host_only) {
    CK(cudaDeviceSynchronize());
    int32_t w = 0;
    CK(cudaMemcpy(&w, p->dev.status, sizeof(w), cudaMemcpyDeviceToHost));
    info->device_status = w;
  }
  return EHYB_OK;
}

ehyb_status_t ehyb_plan_export(ehyb_plan_t p, ehyb_plan_export_t* ex) {
  if (!p || !ex) return EHYB_ERR_INVALID_ARG;
  HostPlan& H = p->host;
  if (!p->host_kept && !p->exported) {  // copy the bulky arrays back from the device
    CK(cudaDeviceSynchronize());
    const bool sl = p->er_layout == 0, csr = p->er_layout == 1;
    try {
      H.ell_col.resize((size_t)p->ell_stored);
      H.ell_val.resize((size_t)p->ell_stored);
      H.er_col.resize(csr ? (size_t)p->er_nnz : 0);
      H.er_val.resize(csr ? (size_t)p->er_nnz : 0);
      H.er_scol.resize(sl ? (size_t)p->er_stored : 0);
      H.er_sval.resize(sl ? (size_t)p->er_stored : 0);
    } catch (const std::bad_alloc&) {
      return EHYB_ERR_OOM;
    }
    const DevPlan& D = p->dev;
    if (!H.ell_col.empty()) {
      CK(cudaMemcpy(H.ell_col.data(), D.ell_col, H.ell_col.size() * 2, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(H.ell_val.data(), D.ell_val, H.ell_val.size() * 8, cudaMemcpyDeviceToHost));
    }
    if (!H.er_col.empty()) {
      CK(cudaMemcpy(H.er_col.data(), D.er_col, H.er_col.size() * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(H.er_val.data(), D.er_val, H.er_val.size() * 8, cudaMemcpyDeviceToHost));
    }
    if (!H.er_scol.empty()) {
      CK(cudaMemcpy(H.er_scol.data(), D.er_scol, H.er_scol.size() * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(H.er_sval.data(), D.er_sval, H.er_sval.size() * 8, cudaMemcpyDeviceToHost));
    }
    p->exported = true;
  }
  ex->n = H.n;
  ex->nparts = H.nparts;
  ex->nslices = H.nslices;
  ex->tpr = H.tpr;
  ex->ell_stored = p->ell_stored;
  ex->er_rows = (int64_t)H.er_row.size();
  ex->er_nnz = p->er_layout == 1 ? p->er_nnz : 0;
  ex->new_to_old = H.new_to_old.data();
  ex->part_ptr = H.part_ptr.data();
  ex->slice_ptr = H.slice_ptr.data();
  ex->slice_pos = H.slice_pos.data();
  ex->ell_col = H.ell_col.data();
  ex->ell_val = H.ell_val.data();
  ex->row_ell_count = H.row_ell_count.data();
  ex->er_part_ptr = H.er_part_ptr.data();
  ex->er_row = H.er_row.data();
  ex->er_ptr = H.er_ptr.data();
  ex->er_col = H.er_col.data();
  ex->er_val = H.er_val.data();
  ex->er_layout = p->er_layout;
  ex->er_stored = p->er_stored;
  ex->er_slice_pos = H.er_slice_pos.data();
  ex->er_scol = H.er_scol.data();
  ex->er_sval = H.er_sval.data();
  ex->row_er_count = H.row_er_count.data();
  ex->n_halo = H.halo_ptr.empty() ? 0 : H.halo_ptr.back();
  ex->halo_ptr = H.halo_ptr.data();
  ex->halo_new = H.halo_new.data();
  ex->lowp = p->lowp;
  ex->lowp_group = H.lowp_group;
  if (p->host_kept && p->lowp) {
    const bool g1 = H.lowp_group == 1;
    ex->ell_val_low = p->lowp == 1 ? (const void*)H.ell_val_f32.data() : (const void*)H.ell_val_bf16.data();
    ex->er_sval_low = p->lowp == 1 ? (const void*)H.er_sval_f32.data() : (const void*)H.er_sval_bf16.data();
    ex->ell_col_low = g1 ? H.ell_col.data() : H.ell_col_low.data();
    ex->er_scol_low = g1 ? H.er_scol.data() : H.er_scol_low.data();
  }
  return EHYB_OK;
}

ehyb_status_t ehyb_profile_enable(ehyb_plan_t p, int32_t enable) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  p->prof = enable != 0;
  p->ev_used = 0;
  return EHYB_OK;
}

ehyb_status_t ehyb_profile_read(ehyb_plan_t p, double* total_ms, int64_t* launches) {
  ehyb_status_t st = check_run(p);
  if (st != EHYB_OK) return st;
  if (!total_ms || !launches) return EHYB_ERR_INVALID_ARG;
  double t = 0;
  for (size_t i = 0; i < p->ev_used; ++i) {
    CK(cudaEventSynchronize(p->ev_pool[i].second));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, p->ev_pool[i].first, p->ev_pool[i].second));
    t += ms;
  }
  *total_ms = t;
  *launches = (int64_t)p->ev_used;
  return EHYB_OK;
}

// ---------------------------------------------------------------- CSR baseline

ehyb_status_t ehyb_csr_create(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* col, const double* val,
                              int32_t tpr, void* stream, ehyb_csr_t* out) {
  if (!out) return EHYB_ERR_INVALID_ARG;
  *out = nullptr;
  ehyb_status_t st = validate_csr(n, n, nnz, rp, col, val);
  if (st != EHYB_OK) return st;
  if (tpr != 0 && !is_pow2_in(tpr, 1, 32)) return EHYB_ERR_INVALID_ARG;
  DeviceInfo d;
  if ((st = query_device(d)) != EHYB_OK) return st;
  std::unique_ptr<ehyb_csr_s> m(new ehyb_csr_s());
  m->n = n;
  m->nnz = nnz;
  m->tpr = tpr ? tpr : pow2_near(n ? std::sqrt((double)nnz / (double)n) : 1.0);
  if ((st = dev_alloc((void**)&m->rp, (size_t)(n + 1) * 8)) != EHYB_OK) return st;
  if ((st = dev_alloc((void**)&m->col, (size_t)nnz * 4)) != EHYB_OK) { cudaFree(m->rp); return st; }
  if ((st = dev_alloc((void**)&m->val, (size_t)nnz * 8)) != EHYB_OK) { cudaFree(m->rp); cudaFree(m->col); return st; }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(m->rp, rp, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(m->col, col, (size_t)nnz * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(m->val, val, (size_t)nnz * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(m->rp); cudaFree(m->col); cudaFree(m->val);
    return cuda_fail(e, "csr upload");
  }
  *out = m.release();
  return EHYB_OK;
}

ehyb_status_t ehyb_csr_spmv(ehyb_csr_t m, const double* x, double* y, void* stream) {
  if (!m) return EHYB_ERR_INVALID_ARG;
  if (m->n == 0) return EHYB_OK;
  if (!x || !y || x == y) return EHYB_ERR_INVALID_ARG;
  CK(launch_csr_f64(m->n, m->rp, m->col, m->val, x, y, m->tpr, (cudaStream_t)stream));
  return EHYB_OK;
}

ehyb_status_t ehyb_csr_set_tpr(ehyb_csr_t m, int32_t tpr) {
  if (!m || !is_pow2_in(tpr, 1, 32)) return EHYB_ERR_INVALID_ARG;
  m->tpr = tpr;
  return EHYB_OK;
}

ehyb_status_t ehyb_csr_destroy(ehyb_csr_t m) {
  if (!m) return EHYB_OK;
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(m->rp);
  cudaFree(m->col);
  cudaFree(m->val);
  delete m;
  return e == cudaSuccess ? EHYB_OK : cuda_fail(e, "cudaDeviceSynchronize");
}

}  // extern "C"
