// Host-side EHYB planner.
//
//   partition_graph : Sec. 3.1 -- rows/columns are vertices, entries are edges; the graph is cut
//                     into parts of at most VecSize vertices.  The paper calls ParMETIS; this is an
//                     in-house greedy graph-growing partitioner (gain = edges into the growing part,
//                     FIFO among equal gains, the next part seeded next to the previous one at the
//                     most enclosed free vertex, a breadth-first sweep order as the fallback).
//   eq1_slice_rows  : Eq. 1 and Eq. 2 (Sec. 3.3).
//   build_plan      : Alg. 1 (per-row in-partition / extra-row counts, sort of each partition's rows
//                     by in-partition count descending, ReorderTable, yIdxER, PositionELL) and
//                     Alg. 2 (placement of every entry in the slab or in the ER part).
#include "plan.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>

namespace ehyb {

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int32_t eq1_slice_rows(int64_t n, int tau, int P, int64_t budget) {
  if (n <= 0) return 1;
  if (P < 1) P = 1;
  for (int64_t K = 1;; ++K) {
    int64_t parts = K * (int64_t)P;
    int64_t vec = (n + parts - 1) / parts;
    // n * tau / (K * P) < SHM^max, compared exactly in integers
    if ((__int128)n * tau < (__int128)budget * parts && vec <= 65536) return (int32_t)vec;
  }
}

uint16_t f32_to_bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) {  // Inf / NaN: keep the class, quiet NaNs
    uint16_t h = (uint16_t)(u >> 16);
    if (u & 0x007fffffu) h |= 0x0040u;
    return h;
  }
  uint32_t bias = 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)((u + bias) >> 16);
}

void make_lowp_copies(HostPlan& P, int lowp) {
  const size_t stored = P.ell_val.size(), er_nnz = P.er_val.size(), er_stored = P.er_sval.size();
  if (lowp == 1) {
    P.ell_val_f32.resize(stored);
    P.er_val_f32.resize(er_nnz);
    P.er_sval_f32.resize(er_stored);
    for (size_t k = 0; k < stored; ++k) P.ell_val_f32[k] = (float)P.ell_val[k];
    for (size_t k = 0; k < er_nnz; ++k) P.er_val_f32[k] = (float)P.er_val[k];
    for (size_t k = 0; k < er_stored; ++k) P.er_sval_f32[k] = (float)P.er_sval[k];
  } else if (lowp == 2) {
    P.ell_val_bf16.resize(stored);
    P.er_val_bf16.resize(er_nnz);
    P.er_sval_bf16.resize(er_stored);
    for (size_t k = 0; k < stored; ++k) P.ell_val_bf16[k] = f32_to_bf16_rne((float)P.ell_val[k]);
    for (size_t k = 0; k < er_nnz; ++k) P.er_val_bf16[k] = f32_to_bf16_rne((float)P.er_val[k]);
    for (size_t k = 0; k < er_stored; ++k) P.er_sval_bf16[k] = f32_to_bf16_rne((float)P.er_sval[k]);
  }
}


// ---------------------------------------------------------------- graph

// pattern of A + A^T without the diagonal, each list sorted and duplicate-free
static void sym_adjacency(int64_t n, const int64_t* rp, const int32_t* col, std::vector<int64_t>& xadj,
                          std::vector<int32_t>& adj) {
  std::vector<int64_t> start(n + 1, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      int32_t c = col[k];
      if (c != i) { ++start[i + 1]; ++start[(int64_t)c + 1]; }
    }
  for (int64_t i = 0; i < n; ++i) start[i + 1] += start[i];
  adj.resize((size_t)start[n]);
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      int32_t c = col[k];
      if (c != i) { adj[(size_t)fill[i]++] = c; adj[(size_t)fill[c]++] = (int32_t)i; }
    }
  xadj.assign((size_t)n + 1, 0);
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t* b = adj.data() + start[i];
    int32_t* e = adj.data() + start[i + 1];
    std::sort(b, e);
    int64_t len = std::unique(b, e) - b;
    if (w != start[i]) std::memmove(adj.data() + w, b, (size_t)len * sizeof(int32_t));
    w += len;
    xadj[(size_t)i + 1] = w;
  }
  adj.resize((size_t)w);
}

// breadth-first order over every component; the first component starts at `s`
static int64_t bfs_order(int64_t n, const std::vector<int64_t>& xadj, const std::vector<int32_t>& adj, int32_t s,
                         std::vector<int32_t>& order) {
  std::vector<char> seen((size_t)n, 0);
  order.clear();
  order.reserve((size_t)n);
  int64_t first_size = -1;
  auto run = [&](int32_t r) {
    size_t h = order.size();
    order.push_back(r);
    seen[(size_t)r] = 1;
    while (h < order.size()) {
      int32_t v = order[h++];
      for (int64_t e = xadj[(size_t)v]; e < xadj[(size_t)v + 1]; ++e) {
        int32_t u = adj[(size_t)e];
        if (!seen[(size_t)u]) { seen[(size_t)u] = 1; order.push_back(u); }
      }
    }
  };
  run(s);
  first_size = (int64_t)order.size();
  for (int64_t i = 0; i < n; ++i)
    if (!seen[(size_t)i]) run((int32_t)i);
  return first_size;
}

// max-priority bucket queue with FIFO order inside a bucket and lazy deletion
struct BucketQueue {
  std::vector<std::vector<int32_t>> b;
  std::vector<size_t> head;
  int top = -1, used = -1;
  explicit BucketQueue(int nkeys) : b((size_t)nkeys), head((size_t)nkeys, 0) {}
  void push(int32_t v, int key) {
    b[(size_t)key].push_back(v);
    if (key > top) top = key;
    if (key > used) used = key;
  }
  bool pop(int32_t& v, int& key) {
    while (top >= 0) {
      size_t t = (size_t)top;
      if (head[t] < b[t].size()) { v = b[t][head[t]++]; key = top; return true; }
      --top;
    }
    return false;
  }
  void clear() {
    for (int k = 0; k <= used; ++k) { b[(size_t)k].clear(); head[(size_t)k] = 0; }
    top = used = -1;
  }
};

int32_t partition_graph(int64_t n, const int64_t* rp, const int32_t* col, int32_t cap, std::vector<int32_t>& part) {
  part.assign((size_t)n, -1);
  if (n == 0) return 0;
  if (cap < 1) cap = 1;
  std::vector<int64_t> xadj;
  std::vector<int32_t> adj;
  sym_adjacency(n, rp, col, xadj, adj);
  // pseudo-peripheral start: the last vertex reached by a breadth-first search from vertex 0
  std::vector<int32_t> order;
  int64_t comp0 = bfs_order(n, xadj, adj, 0, order);
  int32_t start = order[(size_t)comp0 - 1];
  bfs_order(n, xadj, adj, start, order);

  int64_t maxdeg = 0;
  for (int64_t i = 0; i < n; ++i) maxdeg = std::max(maxdeg, xadj[(size_t)i + 1] - xadj[(size_t)i]);
  BucketQueue q((int)maxdeg + 2);
  std::vector<int32_t> conn((size_t)n, 0), touched, members, stamp((size_t)n, -1);
  int64_t cursor = 0, assigned = 0;
  auto next_free = [&]() -> int32_t {
    while (cursor < n && part[(size_t)order[(size_t)cursor]] != -1) ++cursor;
    return cursor < n ? order[(size_t)cursor] : -1;
  };
  int32_t p = 0, seed = start;
  while (assigned < n) {
    if (seed < 0 || part[(size_t)seed] != -1) seed = next_free();
    members.clear();
    int32_t size = 0;
    auto add = [&](int32_t v) {
      part[(size_t)v] = p;
      ++size;
      ++assigned;
      members.push_back(v);
      for (int64_t e = xadj[(size_t)v]; e < xadj[(size_t)v + 1]; ++e) {
        int32_t u = adj[(size_t)e];
        if (part[(size_t)u] != -1) continue;
        if (conn[(size_t)u] == 0) touched.push_back(u);
        q.push(u, ++conn[(size_t)u]);
      }
    };
    add(seed);
    while (size < cap && assigned < n) {
      int32_t v = -1;
      int key = 0;
      bool got = false;
      while (q.pop(v, key))
        if (part[(size_t)v] == -1 && conn[(size_t)v] == key) { got = true; break; }
      if (!got) v = next_free();  // frontier exhausted: continue this part elsewhere in sweep order
      if (v < 0) break;
      add(v);
    }
    for (int32_t u : touched) conn[(size_t)u] = 0;
    touched.clear();
    q.clear();
    // next seed: the free neighbour of this part with the most already-assigned neighbours
    seed = -1;
    int64_t best = -1;
    for (int32_t v : members)
      for (int64_t e = xadj[(size_t)v]; e < xadj[(size_t)v + 1]; ++e) {
        int32_t u = adj[(size_t)e];
        if (part[(size_t)u] != -1 || stamp[(size_t)u] == p) continue;
        stamp[(size_t)u] = p;
        int64_t a = 0;
        for (int64_t f = xadj[(size_t)u]; f < xadj[(size_t)u + 1]; ++f) a += part[(size_t)adj[(size_t)f]] != -1;
        if (a > best) { best = a; seed = u; }
      }
    ++p;
  }
  return p;
}

// ---------------------------------------------------------------- Alg. 1 + Alg. 2

int build_plan(const PlanParams& prm, const int64_t* rp, const int32_t* col, const double* val, HostPlan& P) {
  const double t0 = now_ms();
  const int64_t n = prm.n;
  const int64_t nnz = n > 0 ? rp[n] : 0;
  const int tpr = prm.ell_tpr;
  const int rps = 32 / tpr;  // rows per 32-lane slice
  P.n = n;
  P.nnz = nnz;
  P.tpr = tpr;
  P.slice_rows = prm.slice_rows;

  // PartVec
  std::vector<int32_t> part;
  int32_t nparts = 0;
  if (prm.part_vec) {
    part.assign(prm.part_vec, prm.part_vec + n);
    for (int64_t i = 0; i < n; ++i) nparts = std::max(nparts, part[(size_t)i] + 1);
  } else {
    nparts = partition_graph(n, rp, col, prm.slice_rows, part);
  }
  P.nparts = nparts;
  const double t1 = now_ms();
  P.partition_ms = t1 - t0;

  // S_array1 / S_array2: in-partition (slab) and extra-row entry counts of every row
  const int64_t cap = prm.ell_width_cap > 0 ? prm.ell_width_cap : INT64_MAX;
  std::vector<int32_t> cin((size_t)n), cer((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t a = 0, b = 0;
    const int32_t pi = part[(size_t)i];
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (part[(size_t)col[k]] == pi && a < cap) ++a;
      else ++b;
    }
    cin[(size_t)i] = (int32_t)a;
    cer[(size_t)i] = (int32_t)b;
  }

  // partition boundaries and the per-partition sort (descending in-partition count, stable)
  P.part_ptr.assign((size_t)nparts + 1, 0);
  for (int64_t i = 0; i < n; ++i) ++P.part_ptr[(size_t)part[(size_t)i] + 1];
  for (int32_t p = 0; p < nparts; ++p) P.part_ptr[(size_t)p + 1] += P.part_ptr[(size_t)p];
  P.new_to_old.resize((size_t)n);
  {
    std::vector<int32_t> fill(P.part_ptr.begin(), P.part_ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) P.new_to_old[(size_t)fill[(size_t)part[(size_t)i]]++] = (int32_t)i;
  }
  P.max_part_rows = 0;
  for (int32_t p = 0; p < nparts; ++p) {
    auto b = P.new_to_old.begin() + P.part_ptr[(size_t)p], e = P.new_to_old.begin() + P.part_ptr[(size_t)p + 1];
    // Alg. 1 sorts by in-partition count, descending; ties go to the larger extra-row count first,
    // which keeps the extra-row widths of a 32-row slice close together (less slice padding)
    std::stable_sort(b, e, [&](int32_t a, int32_t c) {
      if (cin[(size_t)a] != cin[(size_t)c]) return cin[(size_t)a] > cin[(size_t)c];
      return cer[(size_t)a] > cer[(size_t)c];
    });
    P.max_part_rows = std::max(P.max_part_rows, P.part_ptr[(size_t)p + 1] - P.part_ptr[(size_t)p]);
  }
  if (P.max_part_rows > 65536) return 4;  // the 16-bit column offset would overflow
  P.old_to_new.resize((size_t)n);
  for (int64_t r = 0; r < n; ++r) P.old_to_new[(size_t)P.new_to_old[(size_t)r]] = (int32_t)r;

  // slices (rps rows each, never straddling partitions) and PositionELL
  P.slice_ptr.assign((size_t)nparts + 1, 0);
  for (int32_t p = 0; p < nparts; ++p) {
    int32_t m = P.part_ptr[(size_t)p + 1] - P.part_ptr[(size_t)p];
    P.slice_ptr[(size_t)p + 1] = P.slice_ptr[(size_t)p] + (m + rps - 1) / rps;
  }
  P.nslices = P.slice_ptr[(size_t)nparts];
  P.slice_pos.assign((size_t)P.nslices + 1, 0);
  for (int32_t p = 0; p < nparts; ++p) {
    const int32_t pb = P.part_ptr[(size_t)p], pe = P.part_ptr[(size_t)p + 1];
    for (int32_t s = P.slice_ptr[(size_t)p]; s < P.slice_ptr[(size_t)p + 1]; ++s) {
      int32_t r0 = pb + (s - P.slice_ptr[(size_t)p]) * rps;
      int32_t r1 = std::min(pe, r0 + rps);
      int32_t w = 0;
      for (int32_t r = r0; r < r1; ++r) w = std::max(w, cin[(size_t)P.new_to_old[(size_t)r]]);
      w = (w + tpr - 1) / tpr;
      P.slice_pos[(size_t)s + 1] = P.slice_pos[(size_t)s] + 32 * (int64_t)w;
    }
  }
  const int64_t stored = P.slice_pos[(size_t)P.nslices];

  P.er_layout = prm.er_layout;
  P.row_er_count.resize((size_t)n);
  for (int64_t r = 0; r < n; ++r) P.row_er_count[(size_t)r] = cer[(size_t)P.new_to_old[(size_t)r]];
  P.er_nnz = 0;
  for (int64_t i = 0; i < n; ++i) P.er_nnz += cer[(size_t)i];

  // er_layout 0: ER entries in the slab's own 32-lane slices (same lane -> row map, column-major)
  P.er_slice_pos.assign((size_t)P.nslices + 1, 0);
  if (P.er_layout == 0) {
    for (int32_t p = 0; p < nparts; ++p) {
      const int32_t pb = P.part_ptr[(size_t)p], pe = P.part_ptr[(size_t)p + 1];
      for (int32_t s = P.slice_ptr[(size_t)p]; s < P.slice_ptr[(size_t)p + 1]; ++s) {
        int32_t r0 = pb + (s - P.slice_ptr[(size_t)p]) * rps;
        int32_t r1 = std::min(pe, r0 + rps);
        int32_t w = 0;
        for (int32_t r = r0; r < r1; ++r) w = std::max(w, P.row_er_count[(size_t)r]);
        w = (w + tpr - 1) / tpr;
        P.er_slice_pos[(size_t)s + 1] = P.er_slice_pos[(size_t)s] + 32 * (int64_t)w;
      }
    }
  }
  const int64_t er_stored = P.er_slice_pos[(size_t)P.nslices];

  // processing order of the slices inside each partition: longest estimated work first (an ER slot
  // gathers x from global memory and is counted twice)
  P.slice_order.resize((size_t)P.nslices);
  for (int32_t p = 0; p < nparts; ++p) {
    const int32_t s0 = P.slice_ptr[(size_t)p], s1 = P.slice_ptr[(size_t)p + 1];
    auto work = [&](int32_t s) {
      return (P.slice_pos[(size_t)s + 1] - P.slice_pos[(size_t)s]) +
             2 * (P.er_slice_pos[(size_t)s + 1] - P.er_slice_pos[(size_t)s]);
    };
    for (int32_t s = s0; s < s1; ++s) P.slice_order[(size_t)s] = s;
    std::stable_sort(P.slice_order.begin() + s0, P.slice_order.begin() + s1,
                     [&](int32_t u, int32_t v) { return work(u) > work(v); });
  }

  // er_layout 1: ER lines (rows with extra entries), per partition, sorted by ER count descending
  P.er_part_ptr.assign((size_t)nparts + 1, 0);
  P.er_row.clear();
  for (int32_t p = 0; p < nparts && P.er_layout == 1; ++p) {
    size_t b = P.er_row.size();
    for (int32_t r = P.part_ptr[(size_t)p]; r < P.part_ptr[(size_t)p + 1]; ++r)
      if (cer[(size_t)P.new_to_old[(size_t)r]] > 0) P.er_row.push_back(r);
    std::stable_sort(P.er_row.begin() + (long)b, P.er_row.end(), [&](int32_t a, int32_t c) {
      return cer[(size_t)P.new_to_old[(size_t)a]] > cer[(size_t)P.new_to_old[(size_t)c]];
    });
    P.er_part_ptr[(size_t)p + 1] = (int32_t)P.er_row.size();
  }
  const int64_t ner = (int64_t)P.er_row.size();
  P.er_ptr.assign((size_t)ner + 1, 0);
  std::vector<int64_t> line_of((size_t)n, -1);
  for (int64_t e = 0; e < ner; ++e) {
    const int32_t r = P.er_row[(size_t)e];
    P.er_ptr[(size_t)e + 1] = P.er_ptr[(size_t)e] + cer[(size_t)P.new_to_old[(size_t)r]];
    line_of[(size_t)r] = e;
  }
  const int64_t er_nnz = P.er_ptr[(size_t)ner];

  // Alg. 2: place each entry
  P.ell_col.assign((size_t)stored, 0);
  P.ell_val.assign((size_t)stored, 0.0);
  P.er_col.assign((size_t)er_nnz, 0);
  P.er_val.assign((size_t)er_nnz, 0.0);
  P.er_scol.assign((size_t)er_stored, 0);
  P.er_scol_old.assign((size_t)er_stored, 0);
  P.er_sval.assign((size_t)er_stored, 0.0);
  // padding slots of the sliced ER part point at the first row of their partition (value 0)
  for (int32_t p = 0; p < nparts && P.er_layout == 0; ++p)
    for (int64_t k = P.er_slice_pos[(size_t)P.slice_ptr[(size_t)p]];
         k < P.er_slice_pos[(size_t)P.slice_ptr[(size_t)p + 1]]; ++k)
    {
      P.er_scol[(size_t)k] = P.part_ptr[(size_t)p];
      P.er_scol_old[(size_t)k] = P.new_to_old[(size_t)P.part_ptr[(size_t)p]];
    }
  P.row_ell_count.resize((size_t)n);
  P.ell_nnz = 0;
  std::vector<int32_t> part_of_new((size_t)nparts > 0 ? (size_t)n : 0);
  for (int32_t p = 0; p < nparts; ++p)
    for (int32_t r = P.part_ptr[(size_t)p]; r < P.part_ptr[(size_t)p + 1]; ++r) part_of_new[(size_t)r] = p;
  for (int64_t r = 0; r < n; ++r) {
    const int32_t i = P.new_to_old[(size_t)r];
    const int32_t p = part_of_new[(size_t)r];
    const int32_t pb = P.part_ptr[(size_t)p];
    const int32_t l = (int32_t)r - pb;
    const int32_t sl = P.slice_ptr[(size_t)p] + l / rps;
    const int64_t base = P.slice_pos[(size_t)sl];
    const int64_t ebase = P.er_slice_pos[(size_t)sl];
    const int32_t lane0 = (l % rps) * tpr;
    int64_t j = 0, je = 0;
    int64_t eo = line_of[(size_t)r] >= 0 ? P.er_ptr[(size_t)line_of[(size_t)r]] : -1;
    for (int64_t k = rp[i]; k < rp[(int64_t)i + 1]; ++k) {
      const int32_t c = col[k];
      if (part[(size_t)c] == part[(size_t)i] && j < cap) {
        const int64_t pos = base + 32 * (j / tpr) + lane0 + (int32_t)(j % tpr);
        P.ell_col[(size_t)pos] = (uint16_t)(P.old_to_new[(size_t)c] - pb);
        P.ell_val[(size_t)pos] = val[k];
        ++j;
      } else if (P.er_layout == 0) {
        const int64_t pos = ebase + 32 * (je / tpr) + lane0 + (int32_t)(je % tpr);
        P.er_scol[(size_t)pos] = P.old_to_new[(size_t)c];
        P.er_scol_old[(size_t)pos] = c;
        P.er_sval[(size_t)pos] = val[k];
        ++je;
      } else {
        P.er_col[(size_t)eo] = P.old_to_new[(size_t)c];
        P.er_val[(size_t)eo] = val[k];
        ++eo;
      }
    }
    P.row_ell_count[(size_t)r] = (int32_t)j;
    P.ell_nnz += j;
  }
  make_lowp_copies(P, prm.lowp);
  P.reorder_ms = now_ms() - t1;
  return 0;
}

}  // namespace ehyb
