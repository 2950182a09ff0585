// FSAI preconditioner for the solver built on a plan.  The paper's motivating use is a Krylov solver whose
// preconditioner is a further sparse product (Sec. 6); this builds the factorized sparse approximate
// inverse of an SPD matrix (Kolotilina and Yeremin): a lower-triangular G on the pattern of the lower
// triangle of B = P A P^T (B in the matrix plan's numbering), row r restricted to the column set J_r
// (the pattern's columns c <= r, r itself included) and defined by
//
//     B[J_r, J_r] = L L^T (Cholesky),   L^T g_r = e_last,   G[r, J_r] = g_r,
//
// which is A[J,J]^{-1} e_r scaled so that (G B G^T)_rr = 1.  M^{-1} = G^T G is applied by two EHYB plans
// (G and G^T) built with the matrix plan's partition, so every vector stays in the plan's numbering.
// Rows are independent: they are computed on host threads.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "plan_internal.h"

namespace ehyb {
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr int64_t kMaxBlock = 1024;  // largest |J_r| accepted (the dense block is |J_r|^2 doubles)

}  // namespace
}  // namespace ehyb

using namespace ehyb;

extern "C" ehyb_status_t ehyb_fsai_create(ehyb_plan_t plan, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                          const int32_t* col, const double* val, int32_t lowp, void* stream,
                                          ehyb_precond_t* out) {
  if (!out) return EHYB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!plan || lowp < 0 || lowp > 2) return EHYB_ERR_INVALID_ARG;
  if (plan->er_layout != 0) return EHYB_ERR_UNSUPPORTED;
  if (n != plan->dev.n) return EHYB_ERR_INVALID_ARG;
  ehyb_status_t st = check_csr(n, n, nnz, row_ptr, col, val);
  if (st != EHYB_OK) return st;
  const double t0 = now_ms();
  const HostPlan& H = plan->host;
  const int T = planner_threads(0);
  std::vector<int32_t> o2n((size_t)n);
  for (int64_t r = 0; r < n; ++r) o2n[(size_t)H.new_to_old[(size_t)r]] = (int32_t)r;

  // B = P A P^T by rows (plan numbering): columns sorted, duplicates summed
  std::vector<int64_t> brp((size_t)n + 1, 0);
  std::vector<int32_t> bcol;
  std::vector<double> bval;
  try {
    std::vector<std::pair<int32_t, double>> tmp((size_t)nnz);
    std::vector<int64_t> len((size_t)n, 0), off((size_t)n + 1, 0);
    for (int64_t r = 0; r < n; ++r) {
      const int32_t i = H.new_to_old[(size_t)r];
      off[(size_t)r + 1] = off[(size_t)r] + (row_ptr[i + 1] - row_ptr[i]);
    }
    parallel_for(n, T, [&](int64_t lo, int64_t hi) {
      for (int64_t r = lo; r < hi; ++r) {
        const int32_t i = H.new_to_old[(size_t)r];
        auto* t = tmp.data() + off[(size_t)r];
        int64_t m = 0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) t[m++] = {o2n[(size_t)col[k]], val[k]};
        std::sort(t, t + m, [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
          return a.first < b.first;
        });
        int64_t u = 0;
        for (int64_t k = 0; k < m; ++k) {
          if (u > 0 && t[u - 1].first == t[k].first) t[u - 1].second += t[k].second;
          else t[u++] = t[k];
        }
        len[(size_t)r] = u;
      }
    });
    for (int64_t r = 0; r < n; ++r) brp[(size_t)r + 1] = brp[(size_t)r] + len[(size_t)r];
    bcol.resize((size_t)brp[(size_t)n]);
    bval.resize((size_t)brp[(size_t)n]);
    parallel_for(n, T, [&](int64_t lo, int64_t hi) {
      for (int64_t r = lo; r < hi; ++r)
        for (int64_t k = 0; k < len[(size_t)r]; ++k) {
          bcol[(size_t)(brp[(size_t)r] + k)] = tmp[(size_t)(off[(size_t)r] + k)].first;
          bval[(size_t)(brp[(size_t)r] + k)] = tmp[(size_t)(off[(size_t)r] + k)].second;
        }
    });
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }

  // pattern of G: row r takes B's columns c <= r and r itself
  std::unique_ptr<ehyb_precond_s> M;
  try {
    M.reset(new ehyb_precond_s());
    M->rp.assign((size_t)n + 1, 0);
    std::atomic<int> too_large{0};
    parallel_for(n, T, [&](int64_t lo, int64_t hi) {
      for (int64_t r = lo; r < hi; ++r) {
        int64_t m = 0;
        bool diag = false;
        for (int64_t k = brp[(size_t)r]; k < brp[(size_t)r + 1] && bcol[(size_t)k] <= r; ++k) {
          ++m;
          diag = diag || bcol[(size_t)k] == r;
        }
        if (!diag) ++m;
        if (m > kMaxBlock) too_large.store(1, std::memory_order_relaxed);
        M->rp[(size_t)r + 1] = m;
      }
    });
    if (too_large.load()) return EHYB_ERR_TOO_LARGE;
    for (int64_t r = 0; r < n; ++r) M->rp[(size_t)r + 1] += M->rp[(size_t)r];
    M->col.resize((size_t)M->rp[(size_t)n]);
    M->val.resize((size_t)M->rp[(size_t)n]);
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }
  const double t1 = now_ms();

  // rows of G: Cholesky of the dense block B[J, J], then L^T g = e_last
  std::atomic<int> not_spd{0};
  parallel_for(n, T, [&](int64_t lo, int64_t hi) {
    std::vector<double> L;
    for (int64_t r = lo; r < hi && !not_spd.load(std::memory_order_relaxed); ++r) {
      int32_t* J = M->col.data() + M->rp[(size_t)r];
      const int64_t m = M->rp[(size_t)r + 1] - M->rp[(size_t)r];
      int64_t q = 0;
      for (int64_t k = brp[(size_t)r]; k < brp[(size_t)r + 1] && bcol[(size_t)k] < r; ++k) J[q++] = bcol[(size_t)k];
      J[q++] = (int32_t)r;  // the largest index of J
      L.assign((size_t)(m * m), 0.0);
      for (int64_t a = 0; a < m; ++a) {  // row J[a] of B merged with J (both sorted)
        const int32_t ja = J[a];
        int64_t k = brp[(size_t)ja], e = brp[(size_t)ja + 1], b = 0;
        while (k < e && b < m) {
          if (bcol[(size_t)k] < J[b]) ++k;
          else if (bcol[(size_t)k] > J[b]) ++b;
          else { L[(size_t)(a * m + b)] = bval[(size_t)k]; ++k; ++b; }
        }
      }
      // in-place Cholesky, lower triangle: L[a][b] for b <= a
      bool ok = true;
      for (int64_t j = 0; j < m && ok; ++j) {
        double d = L[(size_t)(j * m + j)];
        for (int64_t k = 0; k < j; ++k) d -= L[(size_t)(j * m + k)] * L[(size_t)(j * m + k)];
        if (!(d > 0.0) || !std::isfinite(d)) { ok = false; break; }
        const double ljj = std::sqrt(d);
        L[(size_t)(j * m + j)] = ljj;
        for (int64_t a = j + 1; a < m; ++a) {
          double s = L[(size_t)(a * m + j)];
          for (int64_t k = 0; k < j; ++k) s -= L[(size_t)(a * m + k)] * L[(size_t)(j * m + k)];
          L[(size_t)(a * m + j)] = s / ljj;
        }
      }
      if (!ok) {
        not_spd.store(1);
        break;
      }
      // L^T g = e_last by back substitution
      double* g = M->val.data() + M->rp[(size_t)r];
      for (int64_t a = m - 1; a >= 0; --a) {
        double s = a == m - 1 ? 1.0 : 0.0;
        for (int64_t k = a + 1; k < m; ++k) s -= L[(size_t)(k * m + a)] * g[k];
        g[a] = s / L[(size_t)(a * m + a)];
      }
    }
  });
  if (not_spd.load()) return EHYB_ERR_INVALID_ARG;  // a principal block is not positive definite
  const double t2 = now_ms();

  // G^T (rows = columns of G), then the two plans on the matrix plan's partition
  // counting transpose on T row blocks: each block counts its columns, the offsets of column c are laid
  // out block after block, so every row of G^T lists its entries in increasing row of G (the serial order)
  std::vector<int64_t> trp;
  std::vector<int32_t> tcol;
  std::vector<double> tval;
  try {
    trp.assign((size_t)n + 1, 0);
    tcol.resize(M->col.size());
    tval.resize(M->val.size());
    const int64_t TB = std::max<int64_t>(1, std::min<int64_t>(std::min(T, 8), n / 65536 + 1));  // <= 8 count arrays
    std::vector<std::vector<int64_t>> cnt((size_t)TB);
    parallel_for(TB, (int)TB, [&](int64_t b0, int64_t b1) {
      for (int64_t b = b0; b < b1; ++b) {
        std::vector<int64_t>& c = cnt[(size_t)b];
        c.assign((size_t)n, 0);
        for (int64_t r = n * b / TB; r < n * (b + 1) / TB; ++r)
          for (int64_t k = M->rp[(size_t)r]; k < M->rp[(size_t)r + 1]; ++k) ++c[(size_t)M->col[(size_t)k]];
      }
    }, 1);
    // cnt[b][c] becomes block b's first position in row c of G^T
    parallel_for(n, T, [&](int64_t lo, int64_t hi) {
      for (int64_t c = lo; c < hi; ++c) {
        int64_t tot = 0;
        for (int64_t b = 0; b < TB; ++b) tot += cnt[(size_t)b][(size_t)c];
        trp[(size_t)c + 1] = tot;
      }
    });
    for (int64_t r = 0; r < n; ++r) trp[(size_t)r + 1] += trp[(size_t)r];
    parallel_for(n, T, [&](int64_t lo, int64_t hi) {
      for (int64_t c = lo; c < hi; ++c) {
        int64_t at = trp[(size_t)c];
        for (int64_t b = 0; b < TB; ++b) {
          const int64_t k = cnt[(size_t)b][(size_t)c];
          cnt[(size_t)b][(size_t)c] = at;
          at += k;
        }
      }
    });
    parallel_for(TB, (int)TB, [&](int64_t b0, int64_t b1) {
      for (int64_t b = b0; b < b1; ++b) {
        std::vector<int64_t>& fill = cnt[(size_t)b];
        for (int64_t r = n * b / TB; r < n * (b + 1) / TB; ++r)
          for (int64_t k = M->rp[(size_t)r]; k < M->rp[(size_t)r + 1]; ++k) {
            const int64_t pos = fill[(size_t)M->col[(size_t)k]]++;
            tcol[(size_t)pos] = (int32_t)r;
            tval[(size_t)pos] = M->val[(size_t)k];
          }
      }
    }, 1);
  } catch (const std::bad_alloc&) {
    return EHYB_ERR_OOM;
  }
  std::vector<int32_t> pv((size_t)n);
  for (int32_t p = 0; p < H.nparts; ++p)
    for (int32_t r = H.part_ptr[(size_t)p]; r < H.part_ptr[(size_t)p + 1]; ++r) pv[(size_t)r] = p;
  ehyb_options_t opt;
  ehyb_options_default(&opt);
  opt.part_vec = pv.data();
  opt.lowp = lowp;
  opt.host_only = plan->host_only ? 1 : 0;  // a host-only matrix plan gets host-only G plans (inspection)
  opt.num_sms = plan->num_sms;
  st = ehyb_plan_create_csr(n, n, M->rp[(size_t)n], M->rp.data(), M->col.data(), M->val.data(), &opt, stream, &M->g);
  if (st != EHYB_OK) return st;
  st = ehyb_plan_create_csr(n, n, trp[(size_t)n], trp.data(), tcol.data(), tval.data(), &opt, stream, &M->gt);
  if (st != EHYB_OK) {
    ehyb_destroy(M->g);
    return st;
  }
  M->plan = plan;
  M->lowp = lowp;
  M->n = n;
  M->factor_ms = t2 - t1;
  M->setup_ms = now_ms() - t0;
  *out = M.release();
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_precond_info(ehyb_precond_t M, int64_t* nnz_g, double* setup_ms) {
  if (!M) return EHYB_ERR_INVALID_ARG;
  if (nnz_g) *nnz_g = M->rp.empty() ? 0 : M->rp.back();
  if (setup_ms) *setup_ms = M->setup_ms;
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_precond_export(ehyb_precond_t M, int64_t* n, const int64_t** row_ptr, const int32_t** col,
                                             const double** val) {
  if (!M || !n || !row_ptr || !col || !val) return EHYB_ERR_INVALID_ARG;
  *n = M->n;
  *row_ptr = M->rp.data();
  *col = M->col.data();
  *val = M->val.data();
  return EHYB_OK;
}

extern "C" ehyb_status_t ehyb_precond_destroy(ehyb_precond_t M) {
  if (!M) return EHYB_OK;
  // a preconditioner of a host-only plan holds no device memory: nothing to wait for
  cudaError_t e = cudaSuccess;
  if (M->work) {
    e = cudaDeviceSynchronize();
    pcg_work_free(M->work);
  }
  ehyb_status_t st = ehyb_destroy(M->g);
  const ehyb_status_t st2 = ehyb_destroy(M->gt);
  delete M;  // freed whatever the status: the handle is invalid after this call
  if (e != cudaSuccess) return cuda_error_status(e, "cudaDeviceSynchronize");
  return st != EHYB_OK ? st : st2;
}
