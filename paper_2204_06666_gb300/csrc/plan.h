// Host-side EHYB planner: graph partitioning (Sec. 3.1), the cache-size rule (Eq. 1, Eq. 2),
// the post-partition reordering (Alg. 1) and the slab / extra-rows encoding (Alg. 2).
#pragma once
#include <algorithm>
#include <cstdint>
#include <new>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

namespace ehyb {

// Slot layouts of a slice (slab: Alg. 2's ValELL / ColELL; the sliced ER part alike).  A slice of width w
// (slots per lane) stores its 32 x w slots from `base` on (a multiple of 32).
//   group 1 (Alg. 2, the FP64 arrays): slot k of lane L at base + 32 k + L (column-major);
//   group 4 (the FP32 / BF16 copies of plans with wide slices): the first wg = 4 floor(w / 4) slots of each
//     lane in runs of four, slot k < wg of lane L at base + 128 (k / 4) + 4 L + k % 4, so a lane reads four
//     values with one vector load (16 bytes of FP32, 8 of BF16; four 16-bit columns in 8 bytes); the last
//     w - wg slots column-major as in group 1.  Every run is aligned to its own size.
constexpr int kSlotGroup = 4;
inline int64_t slot_pos(int64_t base, int32_t w, int32_t k, int32_t lane, int32_t group) {
  const int32_t wg = group == kSlotGroup ? (w & ~(kSlotGroup - 1)) : 0;
  return k < wg ? base + 32 * kSlotGroup * (int64_t)(k / kSlotGroup) + kSlotGroup * lane + (k % kSlotGroup)
                : base + 32 * (int64_t)k + lane;
}

// Allocator of the planner's large host arrays (graph adjacency, slab and extra-row slots and their copies):
// resize() leaves the new elements uninitialised, so that the planner can zero or fill them in parallel
// (first touch by many threads instead of one serial value-initialisation of hundreds of megabytes).  Every
// array of this kind is written in full after each resize.
template <class T>
struct UninitAlloc : std::allocator<T> {
  using value_type = T;
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U>&) noexcept {}
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  template <class U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new ((void*)p) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new ((void*)p) U(std::forward<A>(a)...);
  }
};
template <class T>
using UninitVec = std::vector<T, UninitAlloc<T>>;

struct PlanParams {
  int64_t n = 0;
  int32_t slice_rows = 0;     // hard cap on rows per partition (VecSize), resolved before build
  int32_t ell_width_cap = 0;  // 0 = unlimited
  int32_t ell_tpr = 1;        // lanes per row in a slab slice
  int32_t lowp = 0;           // 0 none, 1 fp32, 2 bf16 value copies
  int32_t lowp_group = 0;     // slot layout of the value copies: 1, 4, or 0 = 4 (make_lowp_copies)
  int32_t er_layout = 0;      // 0: ER entries sliced with the slab slices; 1: ER lines in CSR; 2: in the slab
                              //    slices after each row's own entries, x staged at the partition's halo
  const int32_t* part_vec = nullptr;
  int32_t threads = 0;        // host threads for the parallel phases (0 = the machine's); results do not depend on it
  int32_t partitioner = 0;    // 0 greedy graph growing, 1 multilevel recursive bisection
  uint64_t seed = 0;          // matching-order seed of the multilevel partitioner
};

struct HostPlan {
  int64_t n = 0, nnz = 0;
  int32_t nparts = 0, nslices = 0, tpr = 1, slice_rows = 0;
  std::vector<int32_t> new_to_old, old_to_new;
  std::vector<int32_t> part_ptr, slice_ptr;
  std::vector<int64_t> slice_pos;
  // processing order: per partition, its slice ids by decreasing estimated work (slab width + 2 x sliced
  // ER width, ties by id), so the warps of a block take the long slices first and the block's tail
  // consists of short ones
  std::vector<int32_t> slice_order;
  UninitVec<uint16_t> ell_col;
  UninitVec<double> ell_val;
  UninitVec<float> ell_val_f32;
  UninitVec<uint16_t> ell_val_bf16;
  std::vector<int32_t> row_ell_count;
  std::vector<int32_t> er_part_ptr, er_row;
  std::vector<int64_t> er_ptr;
  UninitVec<int32_t> er_col;
  UninitVec<double> er_val;
  UninitVec<float> er_val_f32;
  UninitVec<uint16_t> er_val_bf16;
  // er_layout 0: the ER entries of slab slice s, column-major like the slab, 32-bit new-numbering
  // columns; slice width = (er_slice_pos[s+1] - er_slice_pos[s]) / 32
  int32_t er_layout = 0;
  std::vector<int64_t> er_slice_pos;
  UninitVec<int32_t> er_scol;
  UninitVec<int32_t> er_scol_old;  // the same columns in the caller's (original) numbering
  UninitVec<double> er_sval;
  UninitVec<float> er_sval_f32;
  UninitVec<uint16_t> er_sval_bf16;
  std::vector<int32_t> row_er_count;
  // er_layout 2: no separate extra-row arrays; a row's extra-row entries take the slab slots after its own
  // (slice width = the longest row of the slice, slab + extra), their 16-bit columns pointing into
  // [the partition's rows | its halo].  halo_new[halo_ptr[p] .. halo_ptr[p+1]) is partition p's halo in the
  // plan numbering (ascending), halo_old the same columns in the caller's numbering.
  std::vector<int64_t> halo_ptr;
  std::vector<int32_t> halo_new, halo_old;
  int32_t max_stage_rows = 0;  // largest rows + halo of a partition (= max_part_rows without a halo)
  // slot layout of the FP32 / BF16 copies (slot_pos group); with group 4 they come with their own slab and
  // sliced-ER column arrays in that layout (the FP64 arrays stay column-major)
  int32_t lowp_group = 1;
  UninitVec<uint16_t> ell_col_low;
  UninitVec<int32_t> er_scol_low, er_scol_old_low;
  int64_t er_nnz = 0;
  int64_t ell_nnz = 0;
  int32_t max_part_rows = 0;
  double partition_ms = 0, reorder_ms = 0;
};

// FP32 (lowp 1) or BF16 (lowp 2) copies of the FP64 slab and ER values (FP64 -> FP32 -> BF16, round to
// nearest even at each step); lowp 0 does nothing.  group: their slot layout (1 or 4; 0 = 4 when a slice
// holds 32 or more slab + sliced-ER slots per lane on average, else 1); with 4 the columns are copied into
// that layout too.  threads: host threads of the copy loops (0 = the machine's); the copies do not depend on it.
void make_lowp_copies(HostPlan& P, int lowp, int group = 0, int threads = 0);

// mean slab + sliced-ER slots per lane of a slice
double mean_slice_width(const HostPlan& P);

// Eq. 1 and Eq. 2: smallest K >= 1 with n*tau/(K*P) < budget (and at most 2^16 rows so the
// 16-bit column offset holds); returns VecSize = ceil(n / (K*P)).
int32_t eq1_slice_rows(int64_t n, int tau, int P, int64_t budget_bytes);

// Partition the symmetrised graph of A (pattern of A + A^T, no self loops) into parts of at most
// `cap` vertices by greedy graph growing; returns the number of parts.  threads: host threads for the
// parallel phases (0 = the machine's, capped at 32); the result does not depend on it.
int32_t partition_graph(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t cap,
                        std::vector<int32_t>& part, int threads = 0);

// above this many parts the planner uses greedy growing even when the multilevel partitioner is asked for
constexpr int64_t kMaxMultilevelParts = 16384;

// Partition the same graph by multilevel recursive bisection into ceil(n / cap) parts of at most `cap`
// vertices each; `seed` fixes the matching order of the coarsening.  Returns the number of parts; the
// result does not depend on `threads`.
int32_t partition_multilevel(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t cap, uint64_t seed,
                             std::vector<int32_t>& part, int threads = 0);

// host threads the planner uses for `requested` (0 = the machine's, at most 32)
int planner_threads(int requested);

// splitmix64 finaliser: a well-mixed 64-bit hash of x
inline uint64_t mix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// pattern of A + A^T without the diagonal, each list sorted and duplicate-free
void sym_adjacency(int64_t n, const int64_t* rp, const int32_t* col, int threads, std::vector<int64_t>& xadj,
                   UninitVec<int32_t>& adj);

// supervariables of the graph (xadj, adj): maximal runs of consecutive rows with equal closed
// neighbourhoods; run v is rows first[v] .. first[v+1]-1, sv_of maps a row to its run
int64_t supervariables(int64_t n, const std::vector<int64_t>& xadj, const UninitVec<int32_t>& adj, int threads,
                       std::vector<int32_t>& sv_of, std::vector<int64_t>& first);

// breadth-first order of every component of (xadj, adj), the first component from `s`; returns the size
// of the first component
int64_t bfs_order(int64_t n, const int64_t* xadj, const int32_t* adj, int32_t s, std::vector<int32_t>& order);

// the supervariable graph: vertex v = run v of `first`, an edge wherever two runs' rows are adjacent
int64_t supervariable_graph(int64_t n, const int64_t* rp, const int32_t* col, int threads, std::vector<int64_t>& first,
                            std::vector<int64_t>& gx, UninitVec<int32_t>& ga);

// f(lo, hi) on `threads` contiguous pieces of [0, count), in parallel (in the caller when threads <= 1)
template <typename F>
inline void parallel_for(int64_t count, int threads, F&& f, int64_t grain = 4096) {
  const int64_t t = std::min<int64_t>(threads, (count + grain - 1) / grain);
  if (t <= 1) {
    f((int64_t)0, count);
    return;
  }
  std::vector<std::thread> th;
  th.reserve((size_t)t);
  for (int64_t k = 0; k < t; ++k) th.emplace_back([&, k]() { f(count * k / t, count * (k + 1) / t); });
  for (auto& x : th) x.join();
}


// 0 on success, else an ehyb_status_t code (validation is done by the caller).
int build_plan(const PlanParams& prm, const int64_t* row_ptr, const int32_t* col, const double* val,
               HostPlan& out);

uint16_t f32_to_bf16_rne(float f);

}  // namespace ehyb
