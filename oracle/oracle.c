/*
 * CPU oracle for the EHYB SpMV library -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this file's library.  It shares no code with the CUDA path: it computes what the
 * path must compute from the plain definitions, slowly and obviously.
 *
 *   oracle_spmv_csr   y = A x (Sec. 1: y = A * x with A sparse, x and y dense),
 *                     y_i = sum over the stored entries k of row i of val_k * x[col_k],
 *                     summed in storage order, FP64, no FMA contraction.
 *   oracle_spmm_csr   Y = A X for k right-hand sides stored row-major (n x k):
 *                     column j of Y is oracle_spmv_csr of column j of X.
 *   oracle_cg         textbook conjugate gradients (Hestenes-Stiefel), the solver
 *                     whose SpMV cost motivates the method (Sec. 6), FP64.
 *   oracle_cg_refined iterative refinement: outer FP64 residual r = b - A x, inner
 *                     CG on A with its values rounded to FP32 or BF16, vectors,
 *                     SpMV accumulation and vector updates in FP32, dot products
 *                     and the step scalars in FP64; x += d in FP64.  (Not in the
 *                     paper: the precision subsystem built around the method.)
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add anywhere).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

void oracle_spmv_csr(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                     const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = s + val[k] * x[col[k]];
    y[i] = s;
  }
}

/* rows [r0, r1) only: the bounded CPU-baseline sample uses this */
void oracle_spmv_csr_rows(int64_t r0, int64_t r1, const int64_t* row_ptr, const int32_t* col,
                          const double* val, const double* x, double* y) {
  for (int64_t i = r0; i < r1; ++i) {
    double s = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = s + val[k] * x[col[k]];
    y[i] = s;
  }
}

void oracle_spmm_csr(int64_t n, int32_t nrhs, const int64_t* row_ptr, const int32_t* col, const double* val,
                     const double* X, double* Y) {
  for (int64_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < nrhs; ++j) {
      double s = 0.0;
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = s + val[k] * X[(int64_t)col[k] * nrhs + j];
      Y[i * nrhs + j] = s;
    }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
  return s;
}

/*
 * Conjugate gradients for SPD A.  x holds x0 on entry and the iterate on exit.
 *   r = b - A x;  p = r;  rr = r.r
 *   repeat: q = A p; alpha = rr / (p.q); x += alpha p; r -= alpha q;
 *           rr' = r.r; stop if sqrt(rr') <= rtol ||b||; beta = rr'/rr; p = r + beta p
 * hist (optional, max_iter+1 entries) receives ||r_k|| / ||b|| for k = 0..iters.
 * Returns 0 when converged, 1 when max_iter was reached.
 */
int oracle_cg(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
              const double* b, double* x, double rtol, int32_t max_iter,
              int32_t* iters_out, double* relres_out, double* hist) {
  double* r = (double*)malloc((size_t)n * sizeof(double));
  double* p = (double*)malloc((size_t)n * sizeof(double));
  double* q = (double*)malloc((size_t)n * sizeof(double));
  oracle_spmv_csr(n, row_ptr, col, val, x, q);
  for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
  double bnorm = sqrt(dot(n, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
  double rr = dot(n, r, r);
  int32_t it = 0;
  int status = 1;
  if (hist) hist[0] = sqrt(rr) / bnorm;
  if (sqrt(rr) <= rtol * bnorm) status = 0;
  while (status != 0 && it < max_iter) {
    oracle_spmv_csr(n, row_ptr, col, val, p, q);
    double pq = dot(n, p, q);
    double alpha = rr / pq;
    for (int64_t i = 0; i < n; ++i) { x[i] = x[i] + alpha * p[i]; r[i] = r[i] - alpha * q[i]; }
    double rr_new = dot(n, r, r);
    ++it;
    if (hist) hist[it] = sqrt(rr_new) / bnorm;
    if (sqrt(rr_new) <= rtol * bnorm) { rr = rr_new; status = 0; break; }
    double beta = rr_new / rr;
    rr = rr_new;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
  }
  /* true residual */
  oracle_spmv_csr(n, row_ptr, col, val, x, q);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  if (relres_out) *relres_out = sqrt(dot(n, r, r)) / bnorm;
  if (iters_out) *iters_out = it;
  free(r); free(p); free(q);
  return status;
}

/* round a double to bfloat16 (round to nearest even on the float32 value), returned as float */
static float to_bf16(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {       /* finite: RNE on the low 16 bits */
    uint32_t lsb = (u >> 16) & 1u;
    u = u + 0x7fffu + lsb;
  }
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return f;
}

/* y = A_low x in float: values rounded to the storage precision, float products and sums */
static void spmv_low(int64_t n, const int64_t* row_ptr, const int32_t* col, const float* val_low,
                     const float* x, float* y) {
  for (int64_t i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = s + val_low[k] * x[col[k]];
    y[i] = s;
  }
}

static double dotf(int64_t n, const float* a, const float* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = s + (double)a[i] * (double)b[i];
  return s;
}

/* y = A_low x with the product in float but x given in double (rounded to float first) */
void oracle_spmv_low(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                     int32_t bf16, const double* x, double* y) {
  float* vl = (float*)malloc((size_t)row_ptr[n] * sizeof(float) + 4);
  float* xf = (float*)malloc((size_t)n * sizeof(float) + 4);
  float* yf = (float*)malloc((size_t)n * sizeof(float) + 4);
  for (int64_t k = 0; k < row_ptr[n]; ++k) vl[k] = bf16 ? to_bf16(val[k]) : (float)val[k];
  for (int64_t i = 0; i < n; ++i) xf[i] = (float)x[i];
  spmv_low(n, row_ptr, col, vl, xf, yf);
  for (int64_t i = 0; i < n; ++i) y[i] = yf[i];
  free(vl); free(xf); free(yf);
}

/*
 * Mixed-precision iterative refinement.
 * outer: r = b - A x (FP64); stop when ||r|| <= rtol ||b||; solve A_low d ~= r by inner CG
 * (float vectors, float SpMV, FP64 dots/alpha/beta, relative tolerance inner_rtol, at most
 * inner_max iterations); x += d.  Returns 0 when converged.
 * outer_out / inner_total_out: number of refinement steps and of inner CG iterations.
 */
int oracle_cg_refined(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                      int32_t bf16, const double* b, double* x, double rtol, double inner_rtol,
                      int32_t inner_max, int32_t outer_max, int32_t* outer_out, int32_t* inner_total_out,
                      double* relres_out) {
  int64_t nnz = row_ptr[n];
  float* vl = (float*)malloc((size_t)nnz * sizeof(float) + 4);
  for (int64_t k = 0; k < nnz; ++k) vl[k] = bf16 ? to_bf16(val[k]) : (float)val[k];
  double* r = (double*)malloc((size_t)n * sizeof(double) + 8);
  double* ax = (double*)malloc((size_t)n * sizeof(double) + 8);
  float* rf = (float*)malloc((size_t)n * sizeof(float) + 4);
  float* pf = (float*)malloc((size_t)n * sizeof(float) + 4);
  float* qf = (float*)malloc((size_t)n * sizeof(float) + 4);
  float* df = (float*)malloc((size_t)n * sizeof(float) + 4);
  double bnorm = sqrt(dot(n, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
  int status = 1, outer = 0, inner_total = 0;
  double relres = 0.0;
  for (;;) {
    oracle_spmv_csr(n, row_ptr, col, val, x, ax);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - ax[i];
    relres = sqrt(dot(n, r, r)) / bnorm;
    if (relres <= rtol) { status = 0; break; }
    if (outer >= outer_max) break;
    ++outer;
    /* inner CG on A_low d = r, d0 = 0 */
    for (int64_t i = 0; i < n; ++i) { rf[i] = (float)r[i]; pf[i] = rf[i]; df[i] = 0.0f; }
    double rr = dotf(n, rf, rf);
    double r0 = sqrt(rr);
    for (int32_t it = 0; it < inner_max; ++it) {
      spmv_low(n, row_ptr, col, vl, pf, qf);
      double pq = dotf(n, pf, qf);
      double alpha = rr / pq;
      float af = (float)alpha;
      for (int64_t i = 0; i < n; ++i) {
        df[i] = df[i] + af * pf[i];
        rf[i] = rf[i] - af * qf[i];
      }
      double rr_new = dotf(n, rf, rf);
      ++inner_total;
      if (sqrt(rr_new) <= inner_rtol * r0) break;
      double beta = rr_new / rr;
      rr = rr_new;
      float bf = (float)beta;
      for (int64_t i = 0; i < n; ++i) pf[i] = rf[i] + bf * pf[i];
    }
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + (double)df[i];
  }
  if (outer_out) *outer_out = outer;
  if (inner_total_out) *inner_total_out = inner_total;
  if (relres_out) *relres_out = relres;
  free(vl); free(r); free(ax); free(rf); free(pf); free(qf); free(df);
  return status;
}
