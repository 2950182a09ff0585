// Internal definition of a plan (shared by the translation units of the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <utility>
#include <vector>

#include "device.h"
#include "plan.h"

#include "../../include/ehyb.h"

namespace ehyb {
struct CgWork;  // solver workspace, defined in cg.cu
void cg_work_free(CgWork* w);
struct PcgWork;  // preconditioned-solver workspace, defined in pcg.cu
void pcg_work_free(PcgWork* w);
// the CSR checks of ehyb_plan_create_csr (square, monotone row pointers, columns in range)
ehyb_status_t check_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* rp, const int32_t* col,
                        const double* val);
// records the CUDA error text for ehyb_last_cuda_error and returns EHYB_ERR_CUDA
ehyb_status_t cuda_error_status(cudaError_t e, const char* what);
// device allocation through the library's allocation hook (EHYB_ERR_OOM on failure)
ehyb_status_t device_alloc(void** p, size_t bytes);
}  // namespace ehyb

struct ehyb_plan_s {
  ehyb::HostPlan host;        // arrays kept only when requested (or host-only); metadata always
  bool host_kept = false;
  bool host_only = false;
  ehyb::DevPlan dev;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  double* xp = nullptr;     // FP64 workspace (plan numbering), n + 2
  float* xp32 = nullptr;    // FP32 workspace
  double* hx = nullptr;     // device staging for ehyb_spmv_host
  double* hy = nullptr;
  // pipelined host entry (ehyb_spmv_host_many): two device x / y pairs, copy-in and copy-out streams,
  // and per buffer the events "x copied in", "product done", "y copied out"
  double* px[2] = {nullptr, nullptr};
  double* py[2] = {nullptr, nullptr};
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_k[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  int32_t lowp = 0;
  int32_t er_tpr = 1;
  int32_t er_layout = 0;
  int64_t ell_nnz = 0, ell_stored = 0, er_rows = 0, er_nnz = 0, er_stored = 0;
  int32_t nslices = 0, slice_rows = 0, num_sms = 0;
  double upload_ms = 0;
  int device = -1;
  // profiling
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  // export copies (host)
  bool exported = false;
  // solver workspace (allocated by the first ehyb_cg call)
  ehyb::CgWork* cg = nullptr;
  // SpMM workspace: X gathered into the chunk-major plan numbering (allocated by ehyb_spmm)
  void* spmm_ws = nullptr;
  size_t spmm_ws_bytes = 0;
  int32_t tuner_path = 0;
  int32_t ell_width_cap = 0;
};


namespace ehyb {
// Metadata, launch defaults, device upload (unless host-only) of a plan whose host part P->host is built;
// on success *out owns the plan.
ehyb_status_t plan_finalize(std::unique_ptr<ehyb_plan_s>& P, const ehyb_options_t& opt, int dev, int sms,
                            void* stream, ehyb_plan_t* out);
// SM count, opt-in shared memory per block and current device; initialises the kernels' attributes once
ehyb_status_t device_query(int* dev, int* sms, int* smem_optin);
// tuner.cpp: the exhaustive sweep (best plan kept when best_plan is not NULL) and the learned choice
ehyb_status_t sweep_impl(int64_t n, const int64_t* rp, const int32_t* col, const double* val,
                         const ehyb_options_t& base, int reps, ehyb_tune_entry_t* table, int32_t* best_idx,
                         ehyb_plan_t* best_plan, void* stream);
ehyb_status_t learned_choice(int64_t n, const int64_t* rp, const int32_t* col, const double* val, int sms,
                             int smem_optin, int32_t* slice_rows, int32_t* cap, int32_t* tpr, double* pred_ns);
// mean time of reps ehyb_spmv calls on the plan (allocates its own x and y)
ehyb_status_t measure_plan_ms(ehyb_plan_t P, int reps, void* stream, double* ms);
}  // namespace ehyb

// FSAI preconditioner of a plan's matrix (fsai.cpp): G lower triangular in the plan's numbering, applied
// as M^-1 = G^T G through two EHYB plans whose partitions are the matrix plan's.
struct ehyb_precond_s {
  ehyb_plan_t plan = nullptr;  // the matrix plan it belongs to (its numbering)
  ehyb_plan_t g = nullptr, gt = nullptr;
  int32_t lowp = 0;
  int64_t n = 0;
  std::vector<int64_t> rp;  // G on the host (kept for export)
  std::vector<int32_t> col;
  std::vector<double> val;
  double setup_ms = 0, factor_ms = 0;
  ehyb::PcgWork* work = nullptr;
};
