// Device-side view of a plan and the launch entry points of the SpMV kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ehyb {

// Plan arrays on the device (names after the paper: part_ptr = partBoundary, slice_pos =
// PositionELL, ell_col = ColELL, ell_val = ValELL, er_row = yIdxER).
struct DevPlan {
  int64_t n = 0;
  int64_t n_x = 0;  // elements of x the extra-row columns index; 0 = n (a shard's x holds its halo too)
  int32_t nparts = 0, tpr = 1, er_tpr = 1, threads = 512;
  int32_t max_part_rows = 0;
  int32_t max_stage_rows = 0;  // largest rows + halo of a partition: the staged x elements (er_layout 2)
  int32_t max_part_slices = 0;  // most slices of one partition (entries of the fused kernel's slice table)
  int32_t kbatch = 8;  // FP64 batch depth (two pipelined half-batches): 6 on wide slices (>= 32 slots a lane), else 8;
                       // the FP32 / BF16 kernels hold 12 (column-major copies) or 16 / 32 (copies in runs of four)
  const int32_t* new_to_old = nullptr;
  const int32_t* part_ptr = nullptr;
  const int32_t* slice_ptr = nullptr;
  const int64_t* slice_pos = nullptr;
  const int32_t* slice_order = nullptr;  // per partition, slices in processing order (longest first)
  const uint16_t* ell_col = nullptr;
  const double* ell_val = nullptr;
  const float* ell_val_f32 = nullptr;
  const uint16_t* ell_val_bf16 = nullptr;
  const int32_t* er_part_ptr = nullptr;
  const int32_t* er_row = nullptr;
  const int64_t* er_ptr = nullptr;
  const int32_t* er_col = nullptr;
  const double* er_val = nullptr;
  const float* er_val_f32 = nullptr;
  const uint16_t* er_val_bf16 = nullptr;
  int32_t er_layout = 0;  // 0: sliced with the slab slices; 1: CSR lines; 2: in the slab slices, x staged at a halo
  const int64_t* halo_ptr = nullptr;  // er_layout 2: partition p's halo is halo_new / halo_old[halo_ptr[p] ..)
  const int32_t* halo_new = nullptr;
  const int32_t* halo_old = nullptr;
  const int64_t* er_slice_pos = nullptr;
  const int32_t* er_scol = nullptr;
  const int32_t* er_scol_old = nullptr;  // er_scol in the caller's numbering (x read in place)
  const double* er_sval = nullptr;
  const float* er_sval_f32 = nullptr;
  const uint16_t* er_sval_bf16 = nullptr;
  // slot layout of the FP32 / BF16 copies (1: column-major like the FP64 arrays; 4: runs of four slots per
  // lane, with these column arrays in the same layout; for group 1 they alias the FP64 layout's columns)
  int32_t lowp_group = 1;
  const uint16_t* ell_col_low = nullptr;
  const int32_t* er_scol_low = nullptr;
  const int32_t* er_scol_old_low = nullptr;
  int32_t* status = nullptr;  // device status word (first fault wins)
  uint64_t wait_timeout_ns = 1000000000ull;
  int32_t inject_wait_fault = 0;
};

// dynamic shared memory of the fused kernel for an x element of `elem_bytes`
size_t ehyb_smem_bytes(const DevPlan& P, int elem_bytes);

// x_p[i] = x[new_to_old[i]] (to_new) or y[new_to_old[i]] = y_p[i] (!to_new)
cudaError_t launch_permute_f64(const DevPlan& P, int to_new, const double* in, double* out, cudaStream_t s);
cudaError_t launch_permute_f32(const DevPlan& P, int to_new, const float* in, float* out, cudaStream_t s);

// Fused slab + ER kernel.  scatter 0: x and y in the plan numbering; 1: x in the plan numbering, y
// written at new_to_old[r]; 2 (ER layouts 0 and 2, else as 1): x and y both in the caller's numbering,
// x read through new_to_old while it is staged.  The fused dot product is offered with scatter 0 and 2.
// Fused dot product sum_r y_r * xp_r in FP64 (sliced ER layout only): one partial per partition in
// part[nparts]; the last block reduces them in a fixed order into *result and resets *arrive (zero).
struct DotOut {
  double* part;
  int32_t* arrive;
  double* result;
  int32_t self = 0;  // 1: sum_r y_r * y_r instead of y . xp
};
// skip (optional): device flag; the launch returns at once while it is non-zero.
cudaError_t launch_ehyb_f64(const DevPlan& P, const double* xp, double* y, int scatter, cudaStream_t s,
                            const DotOut* dot = nullptr, const int32_t* skip = nullptr);
// values stored FP32 (lowp = 1) or BF16 (lowp = 2); x, y and the accumulation in FP32
cudaError_t launch_ehyb_lowp(const DevPlan& P, int lowp, const float* xp, float* y, int scatter, cudaStream_t s,
                             const DotOut* dot = nullptr, const int32_t* skip = nullptr);

// plain vector-CSR baseline: tpr lanes per row
cudaError_t launch_csr_f64(int64_t n, const int64_t* rp, const int32_t* col, const double* val, const double* x,
                           double* y, int tpr, cudaStream_t s);

// one-time per-device kernel attribute setup (opt-in shared memory)
cudaError_t kernels_init(int smem_optin);

}  // namespace ehyb
