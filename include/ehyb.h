/*
 * ehyb.h -- C ABI of the GB300 EHYB ("explicit caching hybrid") sparse matrix-vector
 * library: y = A x with A sparse and square, x and y dense (Sec. 1).
 *
 * Method (Sec. 3, Sec. 4):
 *   1. The rows of A are partitioned as an undirected graph so that most entries have
 *      row and column in the same partition (Sec. 3.1; greedy graph growing or a multilevel
 *      scheme here, METIS in the paper), with at most VecSize rows per partition chosen by
 *      Eq. 1 / Eq. 2 (Sec. 3.3).
 *   2. Rows are renumbered partition by partition, each partition sorted by its number
 *      of in-partition entries, descending (Alg. 1).
 *   3. In-partition entries go to a sliced ELL slab (32-lane slices stored column-major)
 *      with 16-bit column offsets into the partition's slice of x (Sec. 3.2, Sec. 3.4,
 *      Alg. 2); the others go to the extra-rows (ER) part, each ER line mapped back to
 *      its row by yIdxER (Sec. 3.2).
 *   4. On the GPU one thread block per partition stages its slice of x into shared memory
 *      (gathered through the permutation, or with a bulk asynchronous copy in the plan's
 *      numbering), runs the slab from shared memory, and adds the ER entries of its rows
 *      with global gathers (Alg. 3).
 *
 * Conventions for every call:
 *   - Every function returns an ehyb_status_t and never aborts the process.
 *   - Host pointers are only read during the call (borrowed); device pointers named
 *     *_dev / x / y below are caller-owned device memory (cudaMalloc or torch), 8-byte
 *     aligned for doubles; 16-byte alignment lets the staging use bulk copies.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - SpMV-type calls are asynchronous on `stream`; plan creation, ehyb_cg, ehyb_plan_info,
 *     ehyb_plan_check and ehyb_plan_export synchronise.
 *   - A plan owns device workspace: calls that use the same plan must not overlap in time
 *     (issue them on one stream).  x and y must not alias.
 *   - Device-detected faults (a staging wait that ran out of time) are recorded in a
 *     per-plan status word and returned by the next ehyb_plan_check / ehyb_plan_info.
 *     After a timed-out wait the block waits up to eight more time limits for the copy it
 *     issued to land before it leaves.  A copy still outstanding after that means the device
 *     no longer completes copies: it may yet write into shared memory a later block owns, so
 *     after EHYB_ERR_TIMEOUT discard every result since the last check and launch nothing
 *     more on that device.
 *   - Accepted matrices: square, 0 <= n < 2^31 - 1, nnz < 2^63; unsorted columns,
 *     duplicate entries (summed like separate terms) and explicit zeros are kept; empty
 *     rows give y_i = 0; n = 0 is a valid no-op.
 *   - Non-finite entries of x: padding entries of the slab hold value 0 and column 0 of
 *     their partition, so an Inf/NaN at that position of x can reach other rows of the
 *     same slice as NaN.
 */
#ifndef EHYB_H
#define EHYB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EHYB_OK = 0,
  EHYB_ERR_INVALID_ARG = 1,   /* NULL where a pointer is required, bad option value */
  EHYB_ERR_NOT_SQUARE = 2,    /* n_rows != n_cols */
  EHYB_ERR_INDEX_RANGE = 3,   /* row_ptr not monotone / inconsistent, column out of [0, n) */
  EHYB_ERR_TOO_LARGE = 4,     /* n >= 2^31 - 1, or a partition does not fit the shared-memory slice */
  EHYB_ERR_OOM = 5,           /* host or device allocation failed */
  EHYB_ERR_CUDA = 6,          /* a CUDA runtime call failed (see ehyb_last_cuda_error) */
  EHYB_ERR_UNSUPPORTED = 7,   /* operation not available for this plan (e.g. host-only plan) */
  EHYB_ERR_NOT_CONVERGED = 8, /* iterative solver stopped at max_iter */
  EHYB_ERR_TIMEOUT = 9,       /* a bounded device-side wait ran out; results of that call are invalid */
  EHYB_ERR_NO_DEVICE = 10,    /* no CUDA device */
  EHYB_ERR_IO = 11,           /* a plan file cannot be written or read, or fails its checksum / structure checks */
  EHYB_ERR_BOUNDS = 12        /* bounds-checked build only: a kernel computed an index outside its buffer (the access
                                 was skipped); reported by ehyb_plan_check like EHYB_ERR_TIMEOUT */
} ehyb_status_t;

typedef enum { EHYB_F64 = 0, EHYB_F32 = 1, EHYB_BF16 = 2 } ehyb_dtype_t;

typedef struct {
  int32_t slice_rows;        /* VecSize: max rows per partition; 0 = Eq. 1 / Eq. 2 default */
  int32_t ell_width_cap;     /* max in-partition entries per row kept in the slab (rest -> ER); 0 = no cap */
  int32_t ell_tpr;           /* lanes per row inside a 32-lane slab slice: 1,2,4,8,16,32; 0 = 1 */
  int32_t er_tpr;            /* lanes per ER line (shuffle-reduced): 1,2,4,8,16,32; 0 = auto */
  int32_t block_threads;     /* threads per block (multiple of 32, <= 1024); 0 = auto (enough warps for the
                                average partition's slices, 128..1024) */
  int32_t lowp;              /* also store values as EHYB_F32 (1) or EHYB_BF16 (2) for the FP32 kernels; 0 = no */
  int32_t host_only;         /* 1: build the format on the host only (inspection, no GPU use) */
  int32_t num_sms;           /* P of Eq. 1 for host-only plans; 0 = query the current device */
  int32_t smem_budget;       /* SHM^max of Eq. 1 in bytes per block; 0 = device opt-in maximum - 1024 */
  const int32_t* part_vec;   /* optional PartVec (one partition id >= 0 per row); NULL = in-house partitioner */
  int64_t wait_timeout_ns;   /* bound on each device-side wait; 0 = 1e9 (one second) */
  int32_t inject_wait_fault; /* test hook: the staging wait waits for a copy that is never issued */
  int32_t keep_host;         /* keep host copies of the plan arrays (ehyb_plan_export without device reads) */
  uint64_t seed;             /* seed of the multilevel partitioner's matching order (partitioner 1); the plan is a
                                deterministic function of the matrix, the options and this seed */
  int32_t er_layout;         /* extra rows: 0 = sliced with the slab's own slices (one pass per slice, default),
                                1 = CSR lines, er_tpr lanes each with a shuffle reduction, after a block barrier,
                                2 = in the slab slices after each row's own entries (slice width = the longest
                                row of the slice), with 16-bit columns into [the partition's rows | its halo]:
                                the block stages x at the halo (the distinct columns of its extra entries outside
                                the partition) after its own slice, so no entry reads x from global memory in the
                                multiply.  Same results, bit for bit, as layout 0.  EHYB_ERR_TOO_LARGE when a
                                partition's rows plus halo exceed the shared-memory budget or 65,536; plan files,
                                ehyb_spmm, batches, FSAI and shards take layout 0 only (EHYB_ERR_UNSUPPORTED) */
  int32_t part_nnz;          /* when slice_rows is 0: size partitions for about this many entries each (capped by
                                shared memory) instead of Eq. 1's one-per-SM split; for plans run in a batch */
  int32_t tuner;             /* knob choice when slice_rows, ell_width_cap and ell_tpr are 0: 0 = Eq. 1 default,
                                1 = learned model (ehyb_tuner_set_model) with the sweep as fallback when the plan
                                runs over 2x the model's predicted time, 2 = exhaustive sweep (ehyb_tune_sweep) */
  int32_t host_threads;      /* host threads of the planner's parallel phases (0 = the machine's, at most 32); the
                                plan does not depend on it */
  int32_t partitioner;       /* PartVec when part_vec is NULL (Sec. 3.1): 0 = greedy graph growing (default),
                                1 = multilevel recursive bisection (heavy-edge coarsening, greedy-growing initial
                                bisection, Fiduccia-Mattheyses refinement; ceil(n / slice_rows) parts of equal
                                size; more than 16,384 parts fall back to greedy growing); other values give
                                EHYB_ERR_INVALID_ARG.  The exhaustive sweep (tuner 2) times greedy-growing
                                partitions only */
  int32_t lowp_group;        /* slot layout of the lowp value copies: 1 = column-major like the FP64 arrays,
                                4 = each lane's slots in runs of four (one vector load per run; the copies get
                                their own column arrays in that layout), 0 = 4 (1 when er_layout is 1).
                                Results do not depend on it. */
  int32_t spmm_rhs;          /* right-hand sides the plan is built for (ehyb_spmm): when slice_rows is 0 and this is
                                above 1, Eq. 1 sizes the partitions for a KC-column slice of X per block (KC the
                                largest of 8, 4, 2, 1 dividing it: tau = 8 KC bytes per row), so one chunk covers KC
                                columns; 0 or 1 = the SpMV's tau of 8 bytes.  Results do not depend on it. */
} ehyb_options_t;

typedef struct ehyb_plan_s* ehyb_plan_t;
typedef struct ehyb_precond_s* ehyb_precond_t;
typedef struct ehyb_csr_s* ehyb_csr_t;

typedef struct {
  int64_t n, nnz;
  int32_t nparts, nslices, slice_rows, ell_tpr, er_tpr, block_threads, smem_bytes, lowp;
  int64_t ell_nnz;           /* entries in the slab (without padding) */
  int64_t ell_stored;        /* slab slots including padding */
  int64_t er_rows, er_nnz;   /* ER lines and their entries */
  int64_t bytes_effective;   /* algorithmic bytes of one FP64 SpMV (see ehyb_spmv) */
  int64_t bytes_device;      /* device memory held by the plan */
  double partition_ms, reorder_ms, upload_ms;
  int32_t device_status;     /* EHYB_OK or the first fault recorded by a kernel */
  int32_t num_sms;
  int32_t er_layout;         /* as ehyb_options_t.er_layout */
  int64_t er_stored;         /* sliced layout: ER slots including padding (CSR layout: er_nnz) */
  int32_t tuner_path;        /* 0 options as given, 1 learned choice kept, 2 sweep, 3 learned choice failed its
                                sanity check and the sweep decided */
  int32_t ell_width_cap;     /* slab width cap in force (0 = none) */
  int32_t lowp_group;        /* slot layout of the lowp copies in force (1 or 4; see ehyb_options_t) */
  int32_t max_stage_rows;    /* largest rows + halo of a partition (er_layout 2; the largest partition otherwise) */
  int64_t n_halo;            /* er_layout 2: halo entries over all partitions (0 otherwise) */
} ehyb_plan_info_t;

/* Pointers into arrays owned by the plan (valid until ehyb_destroy); see ehyb_plan_export. */
typedef struct {
  int64_t n;
  int32_t nparts, nslices, tpr;
  int64_t ell_stored, er_rows, er_nnz;
  const int32_t* new_to_old;     /* [n]: original index of new row i (inverse of ReorderTable) */
  const int32_t* part_ptr;       /* [nparts+1]: partBoundary, partition p = new rows [part_ptr[p], part_ptr[p+1]) */
  const int32_t* slice_ptr;      /* [nparts+1]: slices of partition p */
  const int64_t* slice_pos;      /* [nslices+1]: PositionELL; slice width = (slice_pos[s+1]-slice_pos[s])/32 */
  const uint16_t* ell_col;       /* [ell_stored]: ColELL, column - part_ptr[p] (16-bit offset into the slice) */
  const double* ell_val;         /* [ell_stored]: ValELL; slot of (lane, k) = slice_pos[s] + 32 k + lane */
  const int32_t* row_ell_count;  /* [n]: slab entries of each new row (slots k*tpr+sub < count are real) */
  const int32_t* er_part_ptr;    /* [nparts+1]: ER lines owned by partition p */
  const int32_t* er_row;         /* [er_rows]: yIdxER, the new row of each ER line */
  const int64_t* er_ptr;         /* [er_rows+1]: CSR offsets of the ER lines */
  const int32_t* er_col;         /* [er_nnz]: new-numbering column */
  const double* er_val;          /* [er_nnz] */
  /* er_layout 0 (the CSR arrays above are then empty): ER slots of slab slice s at
   * er_slice_pos[s] + 32 k + lane, same lane -> row map as the slab, new-numbering columns */
  int32_t er_layout;
  int64_t er_stored;
  const int64_t* er_slice_pos;   /* [nslices+1] */
  const int32_t* er_scol;        /* [er_stored] (padding: first row of the partition, value 0) */
  const double* er_sval;         /* [er_stored] */
  const int32_t* row_er_count;   /* [n]: extra entries of each new row */
  /* the lowp value copies (plans that keep host arrays only: host_only or keep_host; NULL otherwise):
   * FP32 (lowp 1) or BF16 bits (lowp 2) in the slot layout lowp_group (options.lowp_group), with their own
   * slab / sliced-ER columns when lowp_group is 4 (the FP64 arrays' columns when it is 1) */
  int32_t lowp, lowp_group;
  const void* ell_val_low;       /* [ell_stored] */
  const uint16_t* ell_col_low;   /* [ell_stored] */
  const void* er_sval_low;       /* [er_stored] */
  const int32_t* er_scol_low;    /* [er_stored] */
  /* er_layout 2: partition p's halo is halo_new[halo_ptr[p] .. halo_ptr[p+1]) (plan numbering, ascending); a
   * slab column c >= part_ptr[p+1] - part_ptr[p] of partition p stands for halo_new[halo_ptr[p] + c - rows] */
  int64_t n_halo;
  const int64_t* halo_ptr;       /* [nparts+1] (er_layout 2; all zero otherwise) */
  const int32_t* halo_new;       /* [n_halo] */
} ehyb_plan_export_t;

const char* ehyb_status_string(ehyb_status_t s);
/* Text of the last CUDA error seen by this library in this thread ("" if none). */
const char* ehyb_last_cuda_error(void);
void ehyb_options_default(ehyb_options_t* opt);

/*
 * Build a plan from a host CSR matrix (Alg. 1 and Alg. 2, Sec. 4.1) and upload it.
 * row_ptr: int64[n_rows+1], col: int32[nnz], val: double[nnz], all host memory.
 * opt: NULL for defaults.  Synchronous.  On success *out owns host and device memory.
 */
ehyb_status_t ehyb_plan_create_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                                   const int32_t* col, const double* val, const ehyb_options_t* opt,
                                   void* stream, ehyb_plan_t* out);

/* Release a plan (NULL is accepted).  Synchronises the device before freeing. */
ehyb_status_t ehyb_destroy(ehyb_plan_t plan);

/*
 * y = A x in FP64 (Alg. 3, Sec. 3.2), x and y device arrays of n doubles in the ORIGINAL numbering.
 * With the default sliced ER layout (and with er_layout 2) this is ONE launch, one block per partition: the
 * block gathers its slice of x through new_to_old into shared memory (CachedVec), multiplies the slab from
 * shared memory, adds the ER entries of the same slices with x read from global memory through columns in
 * the original numbering (er_layout 2: from the halo staged beside the slice), and writes y[new_to_old[r]]
 * directly.  With er_layout 1 a gather kernel first writes
 * x_p = x[new_to_old] to plan workspace and the ER lines run after the slab.  Effective bytes per call
 * (ehyb_plan_info): 10 per slab entry (value + 16-bit column), 12 per ER entry, 8 n each for x and y,
 * plus 8 per ER line (yIdxER and its CSR offset) with er_layout 1.  With er_layout 2 the ER entries cost 10
 * bytes like the slab's and each halo entry 12 (its column and its x value, read once per partition).
 */
ehyb_status_t ehyb_spmv(ehyb_plan_t plan, const double* x, double* y, void* stream);

/* y_p = A_p x_p in the plan's numbering (x_p[i] = x[new_to_old[i]]): one kernel, no gathers. */
ehyb_status_t ehyb_spmv_permuted(ehyb_plan_t plan, const double* xp, double* yp, void* stream);

/* out = in reordered: to_new != 0 gives out[i] = in[new_to_old[i]], else out[new_to_old[i]] = in[i]. */
ehyb_status_t ehyb_permute(ehyb_plan_t plan, int32_t to_new, const double* in, double* out, void* stream);

/*
 * y = A x (the product of ehyb_spmv, Alg. 3) with HOST x and y (n doubles each): copies x in, runs
 * ehyb_spmv, copies y out, on `stream`, and waits for the stream.  Pinned host memory makes the copies
 * asynchronous DMA.  On an error the stream is drained before the call returns.
 */
ehyb_status_t ehyb_spmv_host(ehyb_plan_t plan, const double* x_host, double* y_host, void* stream);

/*
 * y_i = A x_i (the product of ehyb_spmv, Alg. 3; the paper's use is many products with one plan, Sec. 6)
 * for `count` pairs of HOST vectors (x_host[i], y_host[i]: n doubles each), pipelined: the copy
 * of x_{i+1} into the device and the copy of y_{i-1} out of it overlap the product of step i (two device
 * buffer pairs; the copies run on two streams of the plan's own, the products on `stream`).  Every y_i is
 * on the host when the call returns; each equals ehyb_spmv's result bit for bit.  Host memory should be
 * pinned (pageable memory works, without the overlap).  NULL arrays or entries give EHYB_ERR_INVALID_ARG;
 * count 0 does nothing.  On an error every stream is drained before the call returns.
 */
ehyb_status_t ehyb_spmv_host_many(ehyb_plan_t plan, int32_t count, const double* const* x_host,
                                  double* const* y_host, void* stream);

/*
 * y = A x exactly as ehyb_spmv computes it, for callers that cannot allocate device memory when
 * they call (a plug-in whose host framework owns all device memory, a latency-critical loop, a
 * thread holding a lock the allocator needs).  The paper has no counterpart: this is a library
 * convenience.  Instead of the plan's workspace, the gathered copy of x goes to a fixed 8 MiB
 * array compiled into the library (present on every GPU that loads it, until exit), so the plan
 * may have at most 2^20 rows (EHYB_ERR_TOO_LARGE otherwise).  The call allocates nothing.  The
 * first call on a device looks the array's device address up once, with that device current;
 * make that first call before any stream capture.  The address is kept for the life of the
 * process: do not use the library across cudaDeviceReset (which also frees every plan's device
 * arrays).  All calls share the array: calls that overlap in time on the GPU (other streams,
 * other threads) race on it; each call rewrites what it reads.  A failed CUDA step returns
 * EHYB_ERR_CUDA with its text in ehyb_last_cuda_error, like every other entry point.
 */
ehyb_status_t ehyb_spmv_noalloc(ehyb_plan_t plan, const double* x, double* y, void* stream);

/* y = A_low x in FP32 arithmetic with values stored as opt.lowp (FP32 or BF16), x and y float
 * device arrays in the original numbering.  EHYB_ERR_UNSUPPORTED if the plan has no lowp copy. */
ehyb_status_t ehyb_spmv_lowp(ehyb_plan_t plan, const float* x, float* y, void* stream);

/*
 * Y = A X for k right-hand sides in FP64: X and Y are row-major n x k device arrays (original
 * numbering).  The columns run in chunks of KC in {8, 4, 2, 1} (the largest that divides k and whose
 * KC-wide slice of X fits a block's shared memory), one launch per chunk, after one gather of X into a
 * chunk-major workspace (n x k doubles, allocated by the first call).  Column j of Y equals ehyb_spmv of
 * column j of X bit for bit.  Requires the sliced ER layout.  Asynchronous on `stream`.  A plan built with
 * opt.spmm_rhs = k has partitions small enough for whole 8-column chunks (one pass over A per 8 columns).
 */
ehyb_status_t ehyb_spmm(ehyb_plan_t plan, int32_t k, const double* X, double* Y, void* stream);

/* ---- conjugate gradients on a plan (Sec. 6: SpMV-dominated iterative solvers) ---- */

typedef struct {
  int32_t iterations;        /* CG iterations (refinement: inner iterations summed over the outer steps) */
  int32_t refinements;       /* FP64 residual corrections (refine != 0) */
  int32_t converged;         /* 1 when the stopping test was met */
  int32_t flexible;          /* 1 when the flexible FP64 CG with the low-precision solve as preconditioner ran
                                (refine 5 / 6, or taking over a stalled BF16 refinement, refine 2 / 4) */
  double relres;             /* ||b - A x||_2 / ||b||_2 of the returned x, recomputed in FP64 */
  double relres_recursive;   /* FP64 CG: sqrt(r.r)/||b|| of the recursion at exit; refinement: last outer residual */
  double seconds;            /* host wall time of the call */
} ehyb_cg_info_t;

/*
 * Solve A x = b for symmetric positive definite A.  b, x: device arrays of n doubles in the ORIGINAL
 * numbering; x holds the initial guess on entry and the solution on return.  Synchronous.
 *   refine = 0: FP64 CG (Hestenes-Stiefel), stop when ||r_k|| <= rtol ||b|| (recursive residual)
 *               or after max_iter iterations.
 *   refine = 1 / 2: FP64 iterative refinement: r = b - A x in FP64, an inner CG on the values stored in
 *               FP32 (1) / BF16 (2) with FP32 vectors and FP32 SpMV accumulation, FP64 dot products and
 *               alpha/beta, to a relative residual inner_rtol (0 = 1e-4 for FP32, 1e-2 for BF16), then
 *               x += d in FP64; stop when the FP64 residual <= rtol ||b||, when it stops decreasing, or
 *               when max_iter inner iterations are spent.  The plan must hold that value copy
 *               (opt.lowp == refine), else EHYB_ERR_UNSUPPORTED.
 *   refine = 3 / 4: FP64 residual replacement around one low-precision CG (values FP32 (3) / BF16 (4),
 *               plan with opt.lowp = 1 / 2): the inner iteration keeps its search direction; each time
 *               its residual has dropped by the factor inner_rtol (0 = 0.1), x += s d in FP64, the
 *               residual is recomputed in FP64 and the iteration continues on it (direction rescaled,
 *               not restarted).  Stops on the FP64 residual <= rtol ||b|| or max_iter iterations.
 *   refine = 5 / 6: flexible CG (Notay's FCG keeping one direction) in FP64 whose preconditioner is an
 *               inner CG on the FP32 (5) / BF16 (6) values (plan with opt.lowp = 1 / 2), from 0 on
 *               r / ||r||, to the relative residual inner_rtol (0 = 0.1) or 500 iterations; each outer
 *               step is one FP64 product q = A p with p A-orthogonal to the previous direction.  The FP64
 *               outer iteration carries the accuracy, so it converges where u_bf16 kappa(A) >= 1 makes
 *               refine 2 / 4 stall; those two hand a stalled solve over to it (info->flexible = 1).
 *               iterations counts inner iterations, refinements the outer steps.
 * Requires er_layout 0 or 2 (every row final after its slice).  Returns EHYB_ERR_NOT_CONVERGED (info
 * filled) when the test was not met.  The solver workspace (5 FP64 + 4 FP32 vectors) is allocated on the first call.
 */
ehyb_status_t ehyb_cg(ehyb_plan_t plan, const double* b, double* x, double rtol, int32_t max_iter, int32_t refine,
                      double inner_rtol, ehyb_cg_info_t* info, void* stream);

/* r.r of the recursion for iterations 0..count-1 of the last FP64 CG solve (or of the last inner solve). */
ehyb_status_t ehyb_cg_history(ehyb_plan_t plan, double* hist, int32_t cap, int32_t* count);

/* ---- row shards for several GPUs: the halo-exchange form of the method ---- */

/*
 * The partitions of a plan are contiguous ranges of the reordered rows, and a partition's slab reads only
 * its own slice of x (Sec. 3.1-3.2): only the extra-row (ER) entries reach other rows.  A shard is one
 * rank's contiguous group of partitions (about 1/nranks of the stored slots each).  Its ER columns are
 * renumbered into x_ext = [x_local | halo]: x_local = the rank's rows [row_begin, row_end) of x in the
 * plan's numbering, halo = the other ranks' rows its ER entries read (halo_rows, ascending, hence grouped
 * by owning rank).  One product on every rank is then
 *     ehyb_shard_pack(x_local -> send_buf);  all-to-all: send_buf -> x_ext + n_local;  ehyb_shard_spmv
 * where rank r sends send_buf[send_ptr[q] : send_ptr[q+1]] to every q and receives from q into halo
 * positions [recv_ptr[q], recv_ptr[q+1]) (counts match pairwise by construction).  Every row is summed in
 * the plan's order, so the shards' y_local concatenated equal ehyb_spmv_permuted's result bit for bit.
 * The library itself never communicates: the caller moves the halo (NCCL, MPI, peer copies).
 */
typedef struct ehyb_shard_s* ehyb_shard_t;

typedef struct {
  int32_t nranks, rank;
  int32_t part_begin, part_end;   /* the plan's partitions of this rank */
  int64_t row_begin, row_end;     /* its rows, plan numbering */
  int64_t n_local;                /* row_end - row_begin */
  int64_t n_halo;                 /* remote x entries read by its ER entries */
  int64_t send_total;             /* entries it sends per exchange (all peers) */
  int64_t slab_stored, er_stored; /* its slab and sliced-ER slots */
  int32_t device_status;          /* its device status word (as ehyb_plan_check, not cleared) */
  int32_t pad;
} ehyb_shard_info_t;

/*
 * Shard `rank` of `nranks` of a plan built with the sliced ER layout (EHYB_ERR_UNSUPPORTED otherwise).
 * Every rank builds the same plan and takes its own shard; the plan may be destroyed afterwards.  A shard
 * of a host-only plan is host-only (lists and arrays for inspection, no device calls).  Uploads its arrays
 * to the current device on `stream` and synchronises.  With more ranks than partitions some shards are empty.
 */
ehyb_status_t ehyb_shard_create(ehyb_plan_t plan, int32_t nranks, int32_t rank, void* stream, ehyb_shard_t* out);
ehyb_status_t ehyb_shard_info(ehyb_shard_t shard, ehyb_shard_info_t* info);

/*
 * Host copies of the exchange lists (each pointer may be NULL): send_ptr, recv_ptr (nranks + 1 each),
 * send_idx (send_total local rows, grouped by destination rank), halo_rows (n_halo plan rows).
 */
ehyb_status_t ehyb_shard_lists(ehyb_shard_t shard, int64_t* send_ptr, int32_t* send_idx, int64_t* recv_ptr,
                               int32_t* halo_rows);

/* The shard's arrays (host copies, valid until ehyb_shard_destroy) in the layout of ehyb_plan_export: n =
 * n_local, ER columns index x_ext, new_to_old = the original row of each local row. */
ehyb_status_t ehyb_shard_export(ehyb_shard_t shard, ehyb_plan_export_t* ex);

/* send_buf[i] = x_local[send_idx[i]] (device arrays), asynchronous on `stream`. */
ehyb_status_t ehyb_shard_pack(ehyb_shard_t shard, const double* x_local, double* send_buf, void* stream);

/* y_local = A_shard x_ext (device arrays: x_ext of n_local + n_halo, y_local of n_local), asynchronous. */
ehyb_status_t ehyb_shard_spmv(ehyb_shard_t shard, const double* x_ext, double* y_local, void* stream);

/*
 * The caller's communication for ehyb_shard_cg; each returns 0 on success.  exchange: called with `stream`
 * idle and send_dev (the caller's send_buf) packed; must leave the halo in halo_dev (p_ext + n_local, n_halo
 * doubles on the device) before it returns.  allreduce: sums `count` host doubles over all ranks in place;
 * every rank must get the same sums.
 */
typedef int32_t (*ehyb_exchange_fn)(void* ctx, const double* send_dev, double* halo_dev, void* stream);
typedef int32_t (*ehyb_allreduce_fn)(void* ctx, double* values, int32_t count);

/*
 * FP64 CG (Hestenes-Stiefel, the solver Sec. 6 motivates) over the shards of all ranks, called by every rank
 * with its rows of b and x (device, plan numbering; x = initial guess in, solution out) and two device
 * buffers of the caller's: p_ext (n_local + n_halo doubles: the direction and its halo) and send_buf
 * (send_total doubles).  Per iteration: one halo exchange of the direction and two scalar sums over ranks
 * (p.q, then r.r); every rank takes the same decisions from the same sums.  Stops when ||r|| <= rtol ||b||
 * or after max_iter iterations; info as for ehyb_cg (relres recomputed after the loop).  Synchronous;
 * allocates its r and q workspace on the first call.
 */
ehyb_status_t ehyb_shard_cg(ehyb_shard_t shard, const double* b, double* x, double* p_ext, double* send_buf,
                            double rtol, int32_t max_iter, ehyb_exchange_fn exchange, ehyb_allreduce_fn allreduce,
                            void* ctx, ehyb_cg_info_t* info, void* stream);
ehyb_status_t ehyb_shard_destroy(ehyb_shard_t shard);

/* ---- preconditioned CG (the solver of Sec. 6 with its preconditioner as further EHYB products) ---- */

/*
 * FSAI preconditioner (factorized sparse approximate inverse of an SPD matrix, Kolotilina and Yeremin) for
 * the matrix of `plan`: G lower triangular on the pattern of the lower triangle of P A P^T (the plan's
 * numbering), row r from the dense principal block B[J_r, J_r] = L L^T of its pattern J_r as the solution
 * of L^T g = e_last, so that (G B G^T)_rr = 1; M^-1 = G^T G.  The CSR arrays (host, caller's numbering,
 * borrowed for the call) must be the matrix the plan was built from.  G and G^T become two EHYB plans on
 * the plan's own partition (lowp 1 / 2: their values also stored FP32 / BF16 and applied in FP32).
 * Synchronous.  Needs a plan with the sliced ER layout (EHYB_ERR_UNSUPPORTED otherwise); for a host-only
 * plan G is built for inspection (ehyb_precond_export) and cannot be used by ehyb_pcg;
 * EHYB_ERR_INVALID_ARG when a principal block is not positive definite (A not SPD); EHYB_ERR_TOO_LARGE
 * when a row of G would have more than 1024 entries.
 */
ehyb_status_t ehyb_fsai_create(ehyb_plan_t plan, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                               const double* val, int32_t lowp, void* stream, ehyb_precond_t* out);
/* entries of G and the host time the setup took (ms) */
ehyb_status_t ehyb_precond_info(ehyb_precond_t M, int64_t* nnz_g, double* setup_ms);
/* G in the plan's numbering (host CSR, rows sorted; valid until ehyb_precond_destroy) */
ehyb_status_t ehyb_precond_export(ehyb_precond_t M, int64_t* n, const int64_t** row_ptr, const int32_t** col,
                                  const double** val);
ehyb_status_t ehyb_precond_destroy(ehyb_precond_t M); /* NULL is fine; synchronises the device when M holds
                                                         device memory; M is freed whatever the status */

/*
 * Preconditioned CG on `plan` with M (built for this plan): x (device, caller's numbering) holds x0 on
 * entry and the solution on return; b likewise.  Stops when the recursive residual ||r_k|| <= rtol ||b||
 * or after max_iter iterations; info->relres is the true FP64 residual ||b - A x|| / ||b|| of the returned
 * x.  Five launches per iteration (A p with p.q, the update, G r with r.z, G^T t, the direction), replayed
 * from CUDA graphs of 16 iterations; alpha and beta stay on the device.  Synchronous.
 * EHYB_ERR_NOT_CONVERGED at the iteration limit or when p.A p <= 0; EHYB_ERR_INVALID_ARG when M belongs
 * to another plan.
 */
ehyb_status_t ehyb_pcg(ehyb_plan_t plan, ehyb_precond_t M, const double* b, double* x, double rtol, int32_t max_iter,
                       ehyb_cg_info_t* info, void* stream);
/*
 * Mixed-precision preconditioned CG: one PCG on FP32 vectors that uses A's FP32 / BF16 values (plan built with
 * opt.lowp = 1 / 2), G's FP32 / BF16 values (M built with lowp = 1 / 2), FP32 accumulation and FP64 inner
 * products, with FP64 residual replacement: each time the FP32 residual has dropped by inner_rtol (0 = 0.01)
 * x += s d and r = b - A x are computed in FP64 and the iteration continues on r (direction kept, rescaled).
 * Stops when ||b - A x|| <= rtol ||b|| (FP64, recomputed at every replacement), after three replacements
 * without a smaller FP64 residual, or when the iterations reach max_iter.  info->refinements counts the
 * replacements.  Synchronous.  EHYB_ERR_UNSUPPORTED when the plan or M lacks its low-precision values.
 */
ehyb_status_t ehyb_pcg_refined(ehyb_plan_t plan, ehyb_precond_t M, const double* b, double* x, double rtol,
                               int32_t max_iter, double inner_rtol, ehyb_cg_info_t* info, void* stream);
/* r.r of iterations 0..count-1 of the last ehyb_pcg solve with M (of the last inner solve for
 * ehyb_pcg_refined) */
ehyb_status_t ehyb_pcg_history(ehyb_precond_t M, double* rr, int32_t cap, int32_t* count);

/* ---- batching: many plans in one persistent launch ---- */

typedef struct ehyb_batch_s* ehyb_batch_t;

/*
 * Group `count` plans (FP64, sliced ER layout, all on the current device) for ehyb_batch_spmv.  The
 * batch keeps pointers to the plans: destroy the batch before any of its plans.  Its work list is the
 * (plan, partition) pairs ordered by stored slots, largest first.
 */
ehyb_status_t ehyb_batch_create(int32_t count, const ehyb_plan_t* plans, ehyb_batch_t* out);

/*
 * ys[i] = A_i xs[i] for every plan of the batch (device arrays, original numbering), asynchronously on
 * `stream`: ONE persistent launch whose blocks pull (plan, partition) tiles from a shared queue, each
 * tile gathering its slice of x through its plan's permutation as it stages it, replayed from a CUDA
 * graph captured on the first call.  Results equal
 * ehyb_spmv on each plan bit for bit.  Uses the plans' workspaces: do not overlap with other calls on
 * the same plans.  xs / ys are host arrays of `count` device pointers.
 */
ehyb_status_t ehyb_batch_spmv(ehyb_batch_t batch, const double* const* xs, double* const* ys, void* stream);

/* Work list length, persistent grid size and threads per block of the batch launch. */
ehyb_status_t ehyb_batch_info(ehyb_batch_t batch, int32_t* ntiles, int32_t* grid, int32_t* threads);

ehyb_status_t ehyb_batch_destroy(ehyb_batch_t batch);  /* NULL is accepted */

/* Plan statistics; synchronises and reads the device status word. */
ehyb_status_t ehyb_plan_info(ehyb_plan_t plan, ehyb_plan_info_t* info);

/* Synchronise the device and return the plan's device status word (then clear it). */
ehyb_status_t ehyb_plan_check(ehyb_plan_t plan);

/* Fill *ex with pointers to host copies of the plan arrays (copied back from the device
 * on first use when the plan did not keep them).  Valid until ehyb_destroy. */
ehyb_status_t ehyb_plan_export(ehyb_plan_t plan, ehyb_plan_export_t* ex);

/*
 * Plan files (the preprocessing of Sec. 3.1-3.3 -- partition, reorder, encode -- done once and reused;
 * the paper weighs its cost against the SpMVs of a solver, Sec. 6).
 *
 * ehyb_plan_save writes the plan's partition, permutation and FP64 slab / ER arrays to `path` (read back
 * from the device when the plan did not keep host copies; synchronises the device).  The file is in the
 * machine's native byte order with a checksum.  EHYB_ERR_IO when the file cannot be written.
 *
 * ehyb_plan_load reads such a file, verifies its checksum and every structural invariant the kernels
 * index by (permutation, monotone pointers, slice widths, column ranges), then uploads it like
 * ehyb_plan_create_csr (synchronous).  From `opt` (NULL = defaults) it takes the run-time choices only:
 * lowp (FP32 / BF16 value copies are made from the stored FP64 values), er_tpr, block_threads, host_only,
 * num_sms, wait_timeout_ns, keep_host; the partition and encoding come from the file.  A loaded plan
 * computes bit-identical results to the plan that was saved.  EHYB_ERR_IO when the file is missing,
 * truncated, of another format version, fails its checksum or its structure checks; EHYB_ERR_TOO_LARGE
 * when a partition does not fit this device's shared memory.
 */
ehyb_status_t ehyb_plan_save(ehyb_plan_t plan, const char* path);
ehyb_status_t ehyb_plan_load(const char* path, const ehyb_options_t* opt, void* stream, ehyb_plan_t* out);

/*
 * Kernel timing: while enabled, every SpMV call on the plan records a CUDA event pair around
 * its main (slab + ER) kernel on the launch stream; ehyb_profile_read synchronises and returns
 * the summed milliseconds and the number of timed launches since the last enable.
 */
ehyb_status_t ehyb_profile_enable(ehyb_plan_t plan, int32_t enable);
ehyb_status_t ehyb_profile_read(ehyb_plan_t plan, double* total_ms, int64_t* launches);

/* ---- plain CSR baseline (vector CSR: tpr lanes per row, shuffle reduction; Sec. 2.2) ---- */

/* Upload a CSR matrix (host arrays as for ehyb_plan_create_csr).  tpr: 1..32 power of two, 0 = auto. */
ehyb_status_t ehyb_csr_create(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col, const double* val,
                              int32_t tpr, void* stream, ehyb_csr_t* out);
ehyb_status_t ehyb_csr_spmv(ehyb_csr_t m, const double* x, double* y, void* stream);
ehyb_status_t ehyb_csr_set_tpr(ehyb_csr_t m, int32_t tpr);
ehyb_status_t ehyb_csr_destroy(ehyb_csr_t m);

/*
 * Measure the FP64 FMA throughput of the current device: every thread of a grid of 4 x 512-thread blocks per
 * SM runs C independent chains acc <- u * w + acc (C = 2, 3 and 4, about 4 x `iters` FMAs per thread each);
 * the best of `reps` timed launches per C (CUDA events, after one untimed launch) gives *tflops = 2 x FMAs /
 * time for the fastest C, and its launch time *ms_best.  An FP64 SpMV spends one FMA per stored entry
 * (Alg. 3), so this rate, not HBM, bounds it on a part whose FP64 pipe is narrow; the roofline of the FP64
 * kernels is taken against it.  Synchronous; allocates and frees its output array.  iters = 2048 takes about
 * 9 ms per launch on a 152-SM part at 2.07 GHz.
 */
ehyb_status_t ehyb_fp64_fma_peak(int32_t iters, int32_t reps, double* tflops, double* ms_best);

/* ---- knob tuning (not in the paper: Eq. 1 fixes VecSize; this chooses VecSize, the slab width cap and
 *      the lanes per row per matrix) ---- */

typedef struct {
  int32_t slice_rows, ell_width_cap, ell_tpr, valid;
  double ms;                 /* measured ehyb_spmv time (sweep), 0 when not timed */
} ehyb_tune_entry_t;

/* Number of knob configurations in the tuning grid (112): VecSize in {Eq. 1 default, 1024, 2048, 4096,
 * 8192, 16384, shared-memory maximum} x slab width cap in {none, p99, p90, p75 row length} x lanes per row in
 * {1, 2, 4, 8}; entry g has VecSize index g / 16, cap index (g / 4) % 4, lanes index g % 4. */
int32_t ehyb_tune_grid_size(void);

/* The grid's knob values for this matrix (no GPU use).  table: ehyb_tune_grid_size() entries. */
ehyb_status_t ehyb_tune_grid(int64_t n, const int64_t* row_ptr, int32_t num_sms, int32_t smem_optin,
                             ehyb_tune_entry_t* table);

/* 16 features of a host CSR matrix (the tuner's input): log2 n, log2 nnz, mean / std / log2 max / min /
 * p50 / p90 / p99 row length, share of rows longer than 32, Gini of the row lengths, mean |i-j|/n, share of
 * entries within n/P of the diagonal, share of diagonally dominant rows, pattern symmetry on up to 1000
 * sampled rows, share of entries inside contiguous blocks of n/P rows (P = num_sms, 0 = 152). */
ehyb_status_t ehyb_features(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                            int32_t num_sms, float* out16);

/* Exhaustive sweep: build every grid configuration (host encodings in parallel threads), time its
 * ehyb_spmv on the current device (two warm-up calls, then the mean of reps, 0 = 10), fill table and
 * *best (index of the fastest).  Synchronous. */
ehyb_status_t ehyb_tune_sweep(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col, const double* val,
                              int32_t reps, ehyb_tune_entry_t* table, int32_t* best, void* stream);

/* Load the tuner network (host arrays): params = ehyb_mlp_param_count() floats; feature and output
 * normalisation (x_norm = (x - mean) / std; outputs = net * out_std + out_mean).  params NULL unloads. */
ehyb_status_t ehyb_tuner_set_model(const float* params, const float* feat_mean, const float* feat_std,
                                   const float* out_mean, const float* out_std);

/* The loaded model's knob choice for a matrix and its predicted ehyb_spmv time per entry (ns). */
ehyb_status_t ehyb_tuner_predict(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                 const double* val, int32_t* slice_rows, int32_t* ell_width_cap, int32_t* ell_tpr,
                                 double* pred_ns_per_nnz);

/* ---- the tuner network's kernels: MLP 16 -> 64 -> 64 -> 4, ReLU, FP32, MSE loss, Adam ---- */

int32_t ehyb_mlp_param_count(void);                /* 5508 */
int64_t ehyb_mlp_workspace_bytes(int32_t batch);   /* device workspace for a batch */

/* out (batch x 4) = net(X (batch x 16)); all device arrays, row-major.  Asynchronous on `stream`. */
ehyb_status_t ehyb_mlp_forward(const float* params, const float* X, int32_t batch, float* out, void* workspace,
                               void* stream);

/* loss = mean((net(X) - T)^2) over batch x 4 outputs, grad = dloss/dparams (device arrays). */
ehyb_status_t ehyb_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t batch, float* grad,
                                 float* loss, void* workspace, void* stream);

/* One Adam step (Kingma & Ba) with bias correction for step number `step` >= 1, on device arrays. */
ehyb_status_t ehyb_mlp_adam(float* params, float* m, float* v, const float* grad, int32_t step, float lr,
                            float beta1, float beta2, float eps, void* stream);

/* ---- test hook (host-side fault injection) ---- */

/* Allow `count` more device allocations by this library, then fail them with EHYB_ERR_OOM;
 * a negative count switches the hook off.  Used to test the out-of-memory paths. */
void ehyb_test_fail_allocs_after(int32_t count);
/* Test hook: runs the kernels' index check on index i against limit lim in a one-thread kernel with its own
 * status word and returns that word (EHYB_ERR_BOUNDS for an index outside [0, lim) in the bounds-checked
 * build, always EHYB_OK in the default build); synchronous.  Nothing is read or written at i. */
ehyb_status_t ehyb_test_bounds_probe(int64_t i, int64_t lim);

#ifdef __cplusplus
}
#endif
#endif /* EHYB_H */
