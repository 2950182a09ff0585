// Knob selection for EHYB plans.  Not in the paper (which fixes VecSize by Eq. 1): the learned-tuning
// subsystem built around the method.
//
//   features : 16 numbers describing a CSR matrix (size, row-length distribution, bandwidth, diagonal
//              dominance, pattern symmetry, locality of a contiguous-block split).
//   grid     : the knob configurations the tuner chooses among -- partition rows (VecSize) in {Eq. 1
//              default, 1024, 2048, 4096, 8192, 16384, the shared-memory maximum} x slab width cap in
//              {none, p99, p90, p75 of the row lengths} x lanes per row in {1, 2, 4, 8}: 112 configurations.
//   sweep    : builds every configuration (host encodings in parallel threads, one partitioning per
//              distinct partition size), uploads and times each one's ehyb_spmv on the GPU; the
//              exhaustive answer, used as training data, as the fallback and as the yardstick of the
//              learned choice.
//   learned  : the MLP of mlp.cu (weights loaded with ehyb_tuner_set_model) maps normalised features to
//              (log2 VecSize, cap index, log2 lanes, log time per entry); outputs snap to the grid.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "plan_internal.h"

namespace ehyb {
namespace {

constexpr int kSlices = 7, kCaps = 4, kTprs = 4, kGrid = kSlices * kCaps * kTprs;
const int kTprVal[kTprs] = {1, 2, 4, 8};

double pct(const std::vector<int64_t>& sorted, double q) {
  if (sorted.empty()) return 0.0;
  return (double)sorted[(size_t)std::floor(q * (double)(sorted.size() - 1))];
}

void features16(int64_t n, const int64_t* rp, const int32_t* col, const double* val, int sms, float* f) {
  std::memset(f, 0, 16 * sizeof(float));
  const int64_t nnz = n > 0 ? rp[n] : 0;
  f[0] = (float)std::log2((double)n + 1.0);
  f[1] = (float)std::log2((double)nnz + 1.0);
  if (n == 0) return;
  std::vector<int64_t> len((size_t)n);
  double sum = 0.0, sum2 = 0.0;
  int64_t over32 = 0;
  for (int64_t i = 0; i < n; ++i) {
    len[(size_t)i] = rp[i + 1] - rp[i];
    sum += (double)len[(size_t)i];
    sum2 += (double)len[(size_t)i] * (double)len[(size_t)i];
    over32 += len[(size_t)i] > 32;
  }
  const double mean = sum / (double)n;
  f[2] = (float)mean;
  f[3] = (float)std::sqrt(std::max(0.0, sum2 / (double)n - mean * mean));
  std::vector<int64_t> s = len;
  std::sort(s.begin(), s.end());
  f[4] = (float)std::log2((double)s.back() + 1.0);
  f[5] = (float)s.front();
  f[6] = (float)pct(s, 0.50);
  f[7] = (float)pct(s, 0.90);
  f[8] = (float)pct(s, 0.99);
  f[9] = (float)((double)over32 / (double)n);
  // Gini coefficient of the row lengths (ascending order, 1-based ranks)
  double g = 0.0;
  for (int64_t i = 0; i < n; ++i) g += (double)(2 * (i + 1) - n - 1) * (double)s[(size_t)i];
  f[10] = sum > 0.0 ? (float)(g / ((double)n * sum)) : 0.0f;
  // bandwidth and locality
  const int64_t band = (n + sms - 1) / std::max(sms, 1);
  const int64_t blk = band;
  double dist = 0.0;
  int64_t near = 0, same_block = 0, dominant = 0;
  for (int64_t i = 0; i < n; ++i) {
    double diag = 0.0, off = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t j = col[k];
      const int64_t d = j > i ? j - i : i - j;
      dist += (double)d;
      near += d <= band;
      same_block += (j / blk) == (i / blk);
      if (j == i) diag += std::fabs(val[k]);
      else off += std::fabs(val[k]);
    }
    dominant += diag >= off && (rp[i + 1] > rp[i]);
  }
  f[11] = nnz ? (float)(dist / (double)nnz / (double)n) : 0.0f;
  f[12] = nnz ? (float)((double)near / (double)nnz) : 0.0f;
  f[13] = (float)((double)dominant / (double)n);
  // pattern symmetry on up to 1000 evenly spaced rows: share of entries (i, j) with an entry (j, i)
  int64_t checked = 0, mirrored = 0;
  const int64_t stride = std::max<int64_t>(1, n / 1000);
  for (int64_t i = 0; i < n; i += stride) {
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t j = col[k];
      bool found = false;
      for (int64_t t = rp[j]; t < rp[j + 1] && !found; ++t) found = col[t] == i;
      ++checked;
      mirrored += found;
    }
  }
  f[14] = checked ? (float)((double)mirrored / (double)checked) : 1.0f;
  f[15] = nnz ? (float)((double)same_block / (double)nnz) : 0.0f;
}

int32_t max_slice_rows(int smem_optin) {
  return (int32_t)std::min<int64_t>(65536, ((int64_t)smem_optin - 1024 - 32) / 8 - 2);
}

void grid_values(int64_t n, const int64_t* rp, int sms, int smem_optin, int32_t slices[kSlices],
                 int32_t caps[kCaps]) {
  const int32_t fixed[5] = {1024, 2048, 4096, 8192, 16384};
  slices[0] = eq1_slice_rows(n, 8, sms, (int64_t)smem_optin - 1024 - 32);
  for (int k = 0; k < 5; ++k) slices[k + 1] = fixed[k];
  slices[6] = max_slice_rows(smem_optin);
  std::vector<int64_t> len((size_t)std::max<int64_t>(n, 0));
  for (int64_t i = 0; i < n; ++i) len[(size_t)i] = rp[i + 1] - rp[i];
  std::sort(len.begin(), len.end());
  caps[0] = 0;
  caps[1] = (int32_t)std::max(1.0, pct(len, 0.99));
  caps[2] = (int32_t)std::max(1.0, pct(len, 0.90));
  caps[3] = (int32_t)std::max(1.0, pct(len, 0.75));
}

struct TunerModel {
  bool loaded = false;
  int device = -1;
  float* d_params = nullptr;
  float* d_io = nullptr;  // 16 inputs, 4 outputs
  void* d_ws = nullptr;
  float feat_mean[16], feat_std[16], out_mean[4], out_std[4];
};
TunerModel g_model;
std::mutex g_model_mu;

}  // namespace

// time of one ehyb_spmv on a plan, ms (mean of reps after two warm-up calls)
static ehyb_status_t time_plan(ehyb_plan_t P, const double* x, double* y, int reps, cudaStream_t s, double* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return cuda_error_status(e, "cudaEventCreate");
  cudaEventCreate(&e1);
  ehyb_status_t st = EHYB_OK;
  for (int i = 0; i < 2 && st == EHYB_OK; ++i) st = ehyb_spmv(P, x, y, s);
  cudaEventRecord(e0, s);
  for (int i = 0; i < reps && st == EHYB_OK; ++i) st = ehyb_spmv(P, x, y, s);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != EHYB_OK) return st;
  if (e != cudaSuccess) return cuda_error_status(e, "sweep timing");
  *ms = (double)t / (double)std::max(reps, 1);
  return EHYB_OK;
}

ehyb_status_t measure_plan_ms(ehyb_plan_t P, int reps, void* stream, double* ms) {
  const int64_t n = std::max<int64_t>(P->dev.n, 1);
  double *x = nullptr, *y = nullptr;
  ehyb_status_t st = device_alloc((void**)&x, (size_t)n * 8);
  if (st != EHYB_OK) return st;
  if ((st = device_alloc((void**)&y, (size_t)n * 8)) != EHYB_OK) {
    cudaFree(x);
    return st;
  }
  cudaMemset(x, 0, (size_t)n * 8);
  st = time_plan(P, x, y, reps, (cudaStream_t)stream, ms);
  cudaFree(x);
  cudaFree(y);
  return st;
}

// The exhaustive sweep; when keep_best, *best_plan receives the fastest plan (others are destroyed).
ehyb_status_t sweep_impl(int64_t n, const int64_t* rp, const int32_t* col, const double* val,
                         const ehyb_options_t& base, int reps, ehyb_tune_entry_t* table, int32_t* best_idx,
                         ehyb_plan_t* best_plan, void* stream) {
  int dev = 0, sms = 0, optin = 0;
  ehyb_status_t st = device_query(&dev, &sms, &optin);
  if (st != EHYB_OK) return st;
  if (base.num_sms > 0) sms = base.num_sms;
  int32_t slices[kSlices], caps[kCaps];
  grid_values(n, rp, sms, optin, slices, caps);
  // one partitioning per distinct partition size, in parallel
  std::vector<std::vector<int32_t>> parts(kSlices);
  {
    std::vector<std::thread> th;
    for (int si = 0; si < kSlices; ++si) {
      bool dup = false;
      for (int sj = 0; sj < si; ++sj) dup |= slices[sj] == slices[si];
      if (!dup)
        th.emplace_back([&, si]() {
          partition_graph(n, rp, col, slices[si], parts[(size_t)si], std::max(1, planner_threads(0) / kSlices));
        });
    }
    for (auto& t : th) t.join();
    for (int si = 0; si < kSlices; ++si)
      if (parts[(size_t)si].empty() && n > 0)
        for (int sj = 0; sj < si; ++sj)
          if (slices[sj] == slices[si]) { parts[(size_t)si] = parts[(size_t)sj]; break; }
  }
  double *x = nullptr, *y = nullptr;
  if ((st = device_alloc((void**)&x, (size_t)std::max<int64_t>(n, 1) * 8)) != EHYB_OK) return st;
  if ((st = device_alloc((void**)&y, (size_t)std::max<int64_t>(n, 1) * 8)) != EHYB_OK) { cudaFree(x); return st; }
  {
    std::vector<double> ones((size_t)std::max<int64_t>(n, 1), 0.5);
    cudaMemcpy(x, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice);
  }
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  double best_ms = 1e300;
  int best = -1;
  ehyb_plan_t keep = nullptr;
  for (int g0 = 0; g0 < kGrid && st == EHYB_OK; g0 += (int)hw) {
    const int g1 = std::min(kGrid, g0 + (int)hw);
    std::vector<std::unique_ptr<ehyb_plan_s>> built((size_t)(g1 - g0));
    std::vector<int> rc((size_t)(g1 - g0), 0);
    std::vector<std::thread> th;
    for (int g = g0; g < g1; ++g) {
      th.emplace_back([&, g]() {
        const int si = g / (kCaps * kTprs), ci = (g / kTprs) % kCaps, ti = g % kTprs;
        std::unique_ptr<ehyb_plan_s> P(new ehyb_plan_s());
        PlanParams prm;
        prm.n = n;
        prm.slice_rows = slices[si];
        prm.ell_width_cap = caps[ci];
        prm.ell_tpr = kTprVal[ti];
        prm.part_vec = n > 0 ? parts[(size_t)si].data() : nullptr;
        prm.threads = 1;  // the configurations themselves are built in parallel
        try {
          rc[(size_t)(g - g0)] = build_plan(prm, rp, col, val, P->host);
        } catch (...) {
          rc[(size_t)(g - g0)] = EHYB_ERR_OOM;
        }
        P->host.slice_rows = slices[si];
        built[(size_t)(g - g0)] = std::move(P);
      });
    }
    for (auto& t : th) t.join();
    for (int g = g0; g < g1 && st == EHYB_OK; ++g) {
      const int si = g / (kCaps * kTprs), ci = (g / kTprs) % kCaps, ti = g % kTprs;
      ehyb_tune_entry_t& e = table[g];
      e.slice_rows = slices[si];
      e.ell_width_cap = caps[ci];
      e.ell_tpr = kTprVal[ti];
      e.valid = 0;
      e.ms = 0.0;
      if (rc[(size_t)(g - g0)] != 0) continue;
      ehyb_options_t opt = base;
      opt.slice_rows = slices[si];
      opt.ell_width_cap = caps[ci];
      opt.ell_tpr = kTprVal[ti];
      opt.part_vec = nullptr;
      opt.host_only = 0;
      opt.tuner = 0;
      ehyb_plan_t P = nullptr;
      if ((int64_t)(built[(size_t)(g - g0)]->host.max_part_rows + 2) * 8 > (int64_t)optin - 1024) continue;
      ehyb_status_t s2 = plan_finalize(built[(size_t)(g - g0)], opt, dev, sms, stream, &P);
      if (s2 == EHYB_ERR_OOM) continue;
      if (s2 != EHYB_OK) { st = s2; break; }
      double ms = 0.0;
      s2 = time_plan(P, x, y, reps, (cudaStream_t)stream, &ms);
      if (s2 != EHYB_OK) { ehyb_destroy(P); st = s2; break; }
      e.valid = 1;
      e.ms = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best = g;
        if (best_plan) {
          if (keep) ehyb_destroy(keep);
          keep = P;
          P = nullptr;
        }
      }
      if (P) ehyb_destroy(P);
    }
  }
  cudaFree(x);
  cudaFree(y);
  if (st != EHYB_OK) {
    if (keep) ehyb_destroy(keep);
    return st;
  }
  if (best_idx) *best_idx = best;
  if (best_plan) *best_plan = keep;
  return best >= 0 ? EHYB_OK : EHYB_ERR_UNSUPPORTED;
}

// Learned choice: features -> MLP (GPU) -> snapped knobs and the predicted ns per entry
ehyb_status_t learned_choice(int64_t n, const int64_t* rp, const int32_t* col, const double* val, int sms,
                             int smem_optin, int32_t* slice_rows, int32_t* cap, int32_t* tpr, double* pred_ns) {
  std::lock_guard<std::mutex> lock(g_model_mu);
  if (!g_model.loaded) return EHYB_ERR_UNSUPPORTED;
  float f[16], xin[16], out[4];
  features16(n, rp, col, val, sms, f);
  for (int i = 0; i < 16; ++i) xin[i] = (f[i] - g_model.feat_mean[i]) / g_model.feat_std[i];
  cudaError_t e = cudaMemcpy(g_model.d_io, xin, sizeof(xin), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error_status(e, "tuner input");
  ehyb_status_t st = ehyb_mlp_forward(g_model.d_params, g_model.d_io, 1, g_model.d_io + 16, g_model.d_ws, nullptr);
  if (st != EHYB_OK) return st;
  e = cudaMemcpy(out, g_model.d_io + 16, sizeof(out), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error_status(e, "tuner output");
  for (int i = 0; i < 4; ++i) out[i] = out[i] * g_model.out_std[i] + g_model.out_mean[i];
  int32_t slices[kSlices], caps[kCaps];
  grid_values(n, rp, sms, smem_optin, slices, caps);
  int bs = 0;
  double bd = 1e300;
  for (int si = 0; si < kSlices; ++si) {
    const double d = std::fabs(std::log2((double)slices[si]) - (double)out[0]);
    if (d < bd) { bd = d; bs = si; }
  }
  const int ci = (int)std::min((float)(kCaps - 1), std::max(0.0f, std::round(out[1])));
  const int ti = (int)std::min((float)(kTprs - 1), std::max(0.0f, std::round(out[2])));
  *slice_rows = slices[bs];
  *cap = caps[ci];
  *tpr = kTprVal[ti];
  *pred_ns = std::exp((double)out[3]);
  return EHYB_OK;
}

}  // namespace ehyb

using namespace ehyb;

extern "C" ehyb_status_t ehyb_features(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                                       int32_t num_sms, float* out16) {
  if (!out16 || n < 0 || (n > 0 && (!row_ptr || !col || !val))) return EHYB_ERR_INVALID_ARG;
  features16(n, row_ptr, col, val, num_sms > 0 ? num_sms : 152, out16);
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_tune_grid(int64_t n, const int64_t* row_ptr, int32_t num_sms, int32_t smem_optin,
                                        ehyb_tune_entry_t* table) {
  if (!table || n < 0 || (n > 0 && !row_ptr)) return EHYB_ERR_INVALID_ARG;
  int32_t slices[kSlices], caps[kCaps];
  grid_values(n, row_ptr, num_sms > 0 ? num_sms : 152, smem_optin > 0 ? smem_optin : 232448, slices, caps);
  for (int g = 0; g < kGrid; ++g) {
    table[g].slice_rows = slices[g / (kCaps * kTprs)];
    table[g].ell_width_cap = caps[(g / kTprs) % kCaps];
    table[g].ell_tpr = kTprVal[g % kTprs];
    table[g].valid = 0;
    table[g].ms = 0.0;
  }
  return EHYB_OK;
}

extern "C" int32_t ehyb_tune_grid_size(void) { return kGrid; }

extern "C" ehyb_status_t ehyb_tune_sweep(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                         const double* val, int32_t reps, ehyb_tune_entry_t* table, int32_t* best,
                                         void* stream) {
  if (!table) return EHYB_ERR_INVALID_ARG;
  if (n < 0 || nnz < 0 || !row_ptr || (nnz > 0 && (!col || !val)) || row_ptr[n] != nnz) return EHYB_ERR_INVALID_ARG;
  ehyb_options_t base;
  ehyb_options_default(&base);
  return sweep_impl(n, row_ptr, col, val, base, reps > 0 ? reps : 10, table, best, nullptr, stream);
}

extern "C" ehyb_status_t ehyb_tuner_set_model(const float* params, const float* feat_mean, const float* feat_std,
                                              const float* out_mean, const float* out_std) {
  std::lock_guard<std::mutex> lock(g_model_mu);
  if (!params) {  // unload
    g_model.loaded = false;
    return EHYB_OK;
  }
  if (!feat_mean || !feat_std || !out_mean || !out_std) return EHYB_ERR_INVALID_ARG;
  for (int i = 0; i < 16; ++i)
    if (!(feat_std[i] > 0.0f)) return EHYB_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (!(out_std[i] > 0.0f)) return EHYB_ERR_INVALID_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return EHYB_ERR_NO_DEVICE;
  if (!g_model.d_params || g_model.device != dev) {
    ehyb_status_t st = device_alloc((void**)&g_model.d_params, (size_t)ehyb_mlp_param_count() * sizeof(float));
    if (st != EHYB_OK) return st;
    if ((st = device_alloc((void**)&g_model.d_io, 32 * sizeof(float))) != EHYB_OK) return st;
    if ((st = device_alloc(&g_model.d_ws, (size_t)ehyb_mlp_workspace_bytes(1) + 256)) != EHYB_OK) return st;
    g_model.device = dev;
  }
  e = cudaMemcpy(g_model.d_params, params, (size_t)ehyb_mlp_param_count() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error_status(e, "tuner weights");
  std::memcpy(g_model.feat_mean, feat_mean, sizeof(g_model.feat_mean));
  std::memcpy(g_model.feat_std, feat_std, sizeof(g_model.feat_std));
  std::memcpy(g_model.out_mean, out_mean, sizeof(g_model.out_mean));
  std::memcpy(g_model.out_std, out_std, sizeof(g_model.out_std));
  g_model.loaded = true;
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_tuner_predict(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                            const double* val, int32_t* slice_rows, int32_t* ell_width_cap,
                                            int32_t* ell_tpr, double* pred_ns_per_nnz) {
  if (!slice_rows || !ell_width_cap || !ell_tpr || !pred_ns_per_nnz || n < 0 || !row_ptr) return EHYB_ERR_INVALID_ARG;
  if (row_ptr[n] != nnz || (nnz > 0 && (!col || !val))) return EHYB_ERR_INVALID_ARG;
  int dev = 0, sms = 0, optin = 0;
  ehyb_status_t st = device_query(&dev, &sms, &optin);
  if (st != EHYB_OK) return st;
  return learned_choice(n, row_ptr, col, val, sms, optin, slice_rows, ell_width_cap, ell_tpr, pred_ns_per_nnz);
}
