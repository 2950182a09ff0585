// Host-side EHYB planner.
//
//   partition_graph : Sec. 3.1 -- rows/columns are vertices, entries are edges; the graph is cut
//                     into parts of at most VecSize vertices.  The paper calls ParMETIS; this is an
//                     in-house greedy graph-growing partitioner (gain = edges into the growing part,
//                     FIFO among equal gains, the next part seeded next to the previous one at the
//                     most enclosed free vertex, a breadth-first sweep order as the fallback), run on
//                     the supervariable graph (runs of consecutive rows with equal closed
//                     neighbourhoods merged, weighted by their row count, split only where a part
//                     fills up).
//   eq1_slice_rows  : Eq. 1 and Eq. 2 (Sec. 3.3).
//   build_plan      : Alg. 1 (per-row in-partition / extra-row counts, sort of each partition's rows
//                     by in-partition count descending, ReorderTable, yIdxER, PositionELL) and
//                     Alg. 2 (placement of every entry in the slab or in the ER part).
#include "plan.h"

#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <chrono>
#include <climits>
#include <cstring>
#include <thread>

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

double mean_slice_width(const HostPlan& P) {
  const double slots = (double)(P.slice_pos.empty() ? 0 : P.slice_pos.back()) +
                       (double)(P.er_slice_pos.empty() ? 0 : P.er_slice_pos.back());
  return P.nslices ? slots / (32.0 * (double)P.nslices) : 0.0;
}

void make_lowp_copies(HostPlan& P, int lowp, int group, int threads) {
  if (lowp == 0) return;
  if (group == 0) group = kSlotGroup;  // runs measured faster than column-major copies on every workload
  if (P.er_layout == 1) group = 1;  // the run loops read the sliced extra-row slots (none in the halo layout)
  P.lowp_group = group;
  const int T = planner_threads(threads);
  const size_t stored = P.ell_val.size(), er_nnz = P.er_val.size(), er_stored = P.er_sval.size();
  // destination of every column-major slot (identity in group 1); each slice's slots map into its own range
  auto regroup = [&](const std::vector<int64_t>& pos, size_t total, std::vector<int64_t>& dst) {
    dst.resize(total);
    parallel_for(P.nslices, T, [&](int64_t lo, int64_t hi) {
      for (int64_t s = lo; s < hi; ++s) {
        const int64_t base = pos[(size_t)s];
        const int32_t w = (int32_t)((pos[(size_t)s + 1] - base) / 32);
        for (int32_t k = 0; k < w; ++k)
          for (int32_t lane = 0; lane < 32; ++lane)
            dst[(size_t)(base + 32 * (int64_t)k + lane)] = slot_pos(base, w, k, lane, group);
      }
    }, 256);
  };
  // every destination is written once: each loop below runs in parallel pieces
  auto each = [&](size_t count, auto&& f) {
    parallel_for((int64_t)count, T, [&](int64_t lo, int64_t hi) {
      for (int64_t k = lo; k < hi; ++k) f((size_t)k);
    }, 1 << 15);
  };
  std::vector<int64_t> sd, ed;
  if (group != 1) {
    regroup(P.slice_pos, stored, sd);
    if (P.er_layout == 0) regroup(P.er_slice_pos, er_stored, ed);
    P.ell_col_low.resize(stored);
    each(stored, [&](size_t k) { P.ell_col_low[(size_t)sd[k]] = P.ell_col[k]; });
    P.er_scol_low.resize(er_stored);
    P.er_scol_old_low.resize(er_stored);
    each(er_stored, [&](size_t k) {
      P.er_scol_low[(size_t)ed[k]] = P.er_scol[k];
      P.er_scol_old_low[(size_t)ed[k]] = P.er_scol_old[k];
    });
  }
  auto at = [&](const std::vector<int64_t>& d, size_t k) { return d.empty() ? k : (size_t)d[k]; };
  if (lowp == 1) {
    P.ell_val_f32.resize(stored);
    P.er_val_f32.resize(er_nnz);
    P.er_sval_f32.resize(er_stored);
    each(stored, [&](size_t k) { P.ell_val_f32[at(sd, k)] = (float)P.ell_val[k]; });
    each(er_nnz, [&](size_t k) { P.er_val_f32[k] = (float)P.er_val[k]; });
    each(er_stored, [&](size_t k) { P.er_sval_f32[at(ed, k)] = (float)P.er_sval[k]; });
  } else if (lowp == 2) {
    P.ell_val_bf16.resize(stored);
    P.er_val_bf16.resize(er_nnz);
    P.er_sval_bf16.resize(er_stored);
    each(stored, [&](size_t k) { P.ell_val_bf16[at(sd, k)] = f32_to_bf16_rne((float)P.ell_val[k]); });
    each(er_nnz, [&](size_t k) { P.er_val_bf16[k] = f32_to_bf16_rne((float)P.er_val[k]); });
    each(er_stored, [&](size_t k) { P.er_sval_bf16[at(ed, k)] = f32_to_bf16_rne((float)P.er_sval[k]); });
  }
}


// ---------------------------------------------------------------- graph

int planner_threads(int requested) {
  if (requested > 0) return requested;
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(32u, hw));
}

// Graph of A for the partitioner: pattern of A + A^T without the diagonal, each list sorted and
// duplicate-free.  The rows' own sorted lists are built in parallel; when the pattern is symmetric
// (every FEM matrix) they already are the answer, otherwise the transpose is merged in.
void sym_adjacency(int64_t n, const int64_t* rp, const int32_t* col, int threads, std::vector<int64_t>& xadj,
                   UninitVec<int32_t>& adj) {
  std::vector<int64_t> len((size_t)n + 1, 0);
  std::unique_ptr<int32_t[]> tmp(new int32_t[(size_t)(n > 0 ? rp[n] : 0) + 1]);  // every used slot is written
  parallel_for(n, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      int32_t* b = tmp.get() + rp[i];
      int64_t m = 0;
      bool increasing = true;  // rows stored with strictly increasing columns need no sort
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
        if (col[k] != i) {
          increasing = increasing && (m == 0 || col[k] > b[m - 1]);
          b[m++] = col[k];
        }
      if (!increasing) {
        std::sort(b, b + m);
        m = std::unique(b, b + m) - b;
      }
      len[(size_t)i + 1] = m;
    }
  });
  // the pattern is symmetric when the multiset of its edges (i, c) equals that of (c, i): compared
  // through two order-independent 64-bit hash sums (a mismatch proves asymmetry; a false match is a
  // 2^-64 event and would only leave out some edges of the partitioner's heuristic graph)
  uint64_t fwd = 0, bwd = 0;
  {
    std::mutex mu;
    parallel_for(n, threads, [&](int64_t lo, int64_t hi) {
      uint64_t f = 0, b = 0;
      for (int64_t i = lo; i < hi; ++i)
        for (int64_t k = 0; k < len[(size_t)i + 1]; ++k) {
          const uint64_t c = (uint64_t)tmp[(size_t)(rp[i] + k)];
          f += mix64(((uint64_t)i << 32) | c);
          b += mix64((c << 32) | (uint64_t)i);
        }
      std::lock_guard<std::mutex> g(mu);
      fwd += f;
      bwd += b;
    });
  }
  const bool symmetric = fwd == bwd;
  if (symmetric) {
    xadj.assign((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) xadj[(size_t)i + 1] = xadj[(size_t)i] + len[(size_t)i + 1];
    adj.resize((size_t)xadj[(size_t)n]);
    parallel_for(n, threads, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i)
        std::copy(tmp.get() + rp[i], tmp.get() + rp[i] + len[(size_t)i + 1], adj.data() + xadj[(size_t)i]);
    });
    return;
  }
  // general pattern: every edge in both directions, then sort and deduplicate each list
  std::vector<int64_t> start((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = 0; k < len[(size_t)i + 1]; ++k) {
      ++start[(size_t)i + 1];
      ++start[(size_t)tmp[(size_t)(rp[i] + k)] + 1];
    }
  for (int64_t i = 0; i < n; ++i) start[(size_t)i + 1] += start[(size_t)i];
  adj.resize((size_t)start[(size_t)n]);
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = 0; k < len[(size_t)i + 1]; ++k) {
      const int32_t c = tmp[(size_t)(rp[i] + k)];
      adj[(size_t)fill[(size_t)i]++] = c;
      adj[(size_t)fill[(size_t)c]++] = (int32_t)i;
    }
  std::vector<int64_t> ulen((size_t)n + 1, 0);
  parallel_for(n, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      int32_t* b = adj.data() + start[(size_t)i];
      int32_t* e = adj.data() + start[(size_t)i + 1];
      std::sort(b, e);
      ulen[(size_t)i + 1] = std::unique(b, e) - b;
    }
  });
  xadj.assign((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i) xadj[(size_t)i + 1] = xadj[(size_t)i] + ulen[(size_t)i + 1];
  UninitVec<int32_t> out((size_t)xadj[(size_t)n]);
  parallel_for(n, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      std::copy(adj.data() + start[(size_t)i], adj.data() + start[(size_t)i] + ulen[(size_t)i + 1],
                out.data() + xadj[(size_t)i]);
  });
  adj.swap(out);
}

// Supervariables: maximal runs of consecutive rows whose closed neighbourhoods (the row itself plus its
// neighbours) coincide -- the dofs of one node of a vector-valued FEM matrix, which are numbered
// together.  sv_of[i] numbers the runs in row order; run v is rows first[v] .. first[v+1]-1.  Returns
// the count (n when no two consecutive rows match).
int64_t supervariables(int64_t n, const std::vector<int64_t>& xadj, const UninitVec<int32_t>& adj, int threads,
                              std::vector<int32_t>& sv_of, std::vector<int64_t>& first) {
  std::vector<uint64_t> key((size_t)n);
  parallel_for(n, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      uint64_t h = mix64((uint64_t)i);  // order-independent hash of the closed neighbourhood
      for (int64_t e = xadj[(size_t)i]; e < xadj[(size_t)i + 1]; ++e) h += mix64((uint64_t)adj[(size_t)e]);
      key[(size_t)i] = h;
    }
  });
  // closed neighbourhoods of a and b are equal: same degree, b in N(a), and N(a) \ {b} == N(b) \ {a}
  auto same = [&](int32_t a, int32_t b) {
    const int64_t da = xadj[(size_t)a + 1] - xadj[(size_t)a], db = xadj[(size_t)b + 1] - xadj[(size_t)b];
    if (da != db) return false;
    const int32_t* pa = adj.data() + xadj[(size_t)a];
    const int32_t* pb = adj.data() + xadj[(size_t)b];
    if (!std::binary_search(pa, pa + da, b)) return false;
    int64_t i = 0, j = 0;
    while (i < da || j < db) {
      if (i < da && pa[i] == b) { ++i; continue; }
      if (j < db && pb[j] == a) { ++j; continue; }
      if (i >= da || j >= db || pa[i] != pb[j]) return false;
      ++i;
      ++j;
    }
    return true;
  };
  // a run breaks before row i unless rows i-1 and i have equal closed neighbourhoods (an equivalence, so
  // comparing neighbours in row order finds the same runs as comparing with each run's first row); the
  // comparisons are independent and run in parallel
  std::vector<uint8_t> brk((size_t)n);
  parallel_for(n, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      brk[(size_t)i] = i == 0 || key[(size_t)i] != key[(size_t)i - 1] || !same((int32_t)(i - 1), (int32_t)i);
  });
  sv_of.assign((size_t)n, 0);
  first.clear();
  first.reserve((size_t)n + 1);
  int64_t nsv = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (brk[(size_t)i]) {
      first.push_back(i);
      ++nsv;
    }
    sv_of[(size_t)i] = (int32_t)(nsv - 1);
  }
  first.push_back(n);
  return nsv;
}

// The graph the partitioners cut: one vertex per supervariable (its weight is first[v+1] - first[v]
// rows), an edge wherever two supervariables' rows are adjacent in the pattern of A + A^T; lists sorted.
// Returns the vertex count.
int64_t supervariable_graph(int64_t n, const int64_t* rp, const int32_t* col, int threads, std::vector<int64_t>& first,
                            std::vector<int64_t>& gx, UninitVec<int32_t>& ga) {
  std::vector<int64_t> xadj;
  UninitVec<int32_t> adj;
  sym_adjacency(n, rp, col, threads, xadj, adj);
  std::vector<int32_t> sv_of;
  const int64_t nv = supervariables(n, xadj, adj, threads, sv_of, first);
  if (nv < n) {
    // sv_of does not decrease along the rows and every row's list is sorted, so a list mapped through sv_of
    // is sorted too: its distinct supervariables are found by comparing neighbours, counted in a first pass
    // and written in a second
    auto each_neighbour = [&](int64_t v, auto&& f) {
      const int64_t r = first[(size_t)v];  // the rows of a supervariable share their closed neighbourhood
      int32_t prev = -1;
      for (int64_t e = xadj[(size_t)r]; e < xadj[(size_t)r + 1]; ++e) {
        const int32_t u = sv_of[(size_t)adj[(size_t)e]];
        if (u != v && u != prev) {
          f(u);
          prev = u;
        }
      }
    };
    gx.assign((size_t)nv + 1, 0);
    parallel_for(nv, threads, [&](int64_t lo, int64_t hi) {
      for (int64_t v = lo; v < hi; ++v) {
        int64_t m = 0;
        each_neighbour(v, [&](int32_t) { ++m; });
        gx[(size_t)v + 1] = m;
      }
    });
    for (int64_t v = 0; v < nv; ++v) gx[(size_t)v + 1] += gx[(size_t)v];
    ga.resize((size_t)gx[(size_t)nv]);
    parallel_for(nv, threads, [&](int64_t lo, int64_t hi) {
      for (int64_t v = lo; v < hi; ++v) {
        int32_t* d = ga.data() + gx[(size_t)v];
        each_neighbour(v, [&](int32_t u) { *d++ = u; });
      }
    });
    std::vector<int64_t>().swap(xadj);
    UninitVec<int32_t>().swap(adj);
  } else {
    gx.swap(xadj);
    ga.swap(adj);
  }
  return nv;
}

// breadth-first order over every component; the first component starts at `s`
int64_t bfs_order(int64_t n, const int64_t* xadj, const int32_t* adj, int32_t s, std::vector<int32_t>& order) {
  // visited flags as bits: 2M vertices take 256 KB, which stays in a core's L2
  std::vector<uint64_t> seen((size_t)(n + 63) / 64, 0);
  auto test_set = [&](int32_t u) {
    uint64_t& w = seen[(size_t)u >> 6];
    const uint64_t b = 1ull << (u & 63);
    const bool was = (w & b) != 0;
    w |= b;
    return was;
  };
  order.resize((size_t)n);
  int32_t* q = order.data();
  int64_t tail = 0, first_size = -1;
  // the queue is known a few vertices ahead: their offsets, lists and neighbours' flags are prefetched in
  // three stages (on a randomly numbered graph every one of them is a cache miss otherwise)
  auto run = [&](int32_t r) {
    int64_t h = tail;
    q[tail++] = r;
    test_set(r);
    while (h < tail) {
      if (h + 12 < tail) __builtin_prefetch(&xadj[(size_t)q[h + 12]]);
      if (h + 6 < tail) __builtin_prefetch(&adj[(size_t)xadj[(size_t)q[h + 6]]]);
      if (h + 3 < tail) {
        const int32_t w = q[h + 3];
        for (int64_t e = xadj[(size_t)w]; e < xadj[(size_t)w + 1]; ++e)
          __builtin_prefetch(&seen[(size_t)adj[(size_t)e] >> 6]);
      }
      const int32_t v = q[h++];
      for (int64_t e = xadj[(size_t)v]; e < xadj[(size_t)v + 1]; ++e) {
        const int32_t u = adj[(size_t)e];
        if (!test_set(u)) q[tail++] = u;
      }
    }
  };
  if (n > 0) run(s);
  first_size = tail;
  for (int64_t i = 0; i < n; ++i)
    if (!(seen[(size_t)i >> 6] >> (i & 63) & 1)) run((int32_t)i);
  return first_size;
}

// Per-vertex state of the greedy growth, packed so that visiting a vertex touches one cache line (the
// growth is bound by the latency of these visits, not by arithmetic).
struct GrowState {
  int32_t conn;      // its edges into the part being grown (its gain)
  int32_t done_nb;   // its neighbours already done
  int32_t left;      // its rows not yet assigned; 0 once it is done
  int32_t next_row;  // its first row not yet assigned (row counts stay below 2^31)
};

// rows [row, row + count) go to part p (recorded during the growth, written to `part` afterwards)
struct RowRun {
  int64_t row;
  int32_t count, p;
};

// Max-gain queue of free vertices.  Bucket k lists, in the order they reached it, the vertices whose gain
// became k while the current part grew; a vertex whose gain rises is appended to the higher bucket and its
// entry in the lower one goes stale (an entry is live while its vertex is free and its gain still equals
// the bucket's).  So the queue pops the free vertex of highest gain and, among equal gains, the one that
// reached that gain first; stale entries are skipped when the read position passes them.  Gains only rise
// during a part, so a skipped entry never becomes live again.
struct GainQueue {
  std::vector<std::vector<int32_t>> bucket;  // per gain, appended in arrival order
  std::vector<size_t> rd;                    // per gain, the next entry to read
  const std::vector<GrowState>& st;
  int top = -1, used = -1;  // highest bucket that may hold live entries; highest bucket written
  GainQueue(const std::vector<GrowState>& state, int nkeys) : bucket((size_t)nkeys), rd((size_t)nkeys, 0), st(state) {}
  // v's gain has just become k
  void raise(int32_t v, int k) {
    bucket[(size_t)k].push_back(v);
    if (k > top) top = k;
    if (k > used) used = k;
  }
  bool pop(int32_t& v) {
    for (; top >= 0; --top) {
      const std::vector<int32_t>& b = bucket[(size_t)top];
      size_t& r = rd[(size_t)top];
      while (r < b.size()) {
        const int32_t u = b[r++];
        const GrowState& s = st[(size_t)u];
        if (s.left > 0 && s.conn == top) {
          v = u;
          return true;
        }
      }
    }
    return false;
  }
  // the k-th entry after the read position of the top bucket (-1 if none): likely among the next pops
  int32_t peek(size_t k) const {
    if (top < 0) return -1;
    const std::vector<int32_t>& b = bucket[(size_t)top];
    const size_t i = rd[(size_t)top] + k;
    return i < b.size() ? b[i] : -1;
  }
  void clear() {
    for (int k = 0; k <= used; ++k) {
      bucket[(size_t)k].clear();
      rd[(size_t)k] = 0;
    }
    top = used = -1;
  }
};

int32_t partition_graph(int64_t n, const int64_t* rp, const int32_t* col, int32_t cap, std::vector<int32_t>& part,
                        int threads) {
  part.assign((size_t)n, -1);
  if (n == 0) return 0;
  if (cap < 1) cap = 1;
  threads = planner_threads(threads);
  // grow on the supervariable graph: vertex weight = rows of the supervariable
  std::vector<int64_t> first, gx;
  UninitVec<int32_t> ga;
  const int64_t nv = supervariable_graph(n, rp, col, threads, first, gx, ga);

  // pseudo-peripheral start: the last vertex reached by a breadth-first search from vertex 0.  The graph
  // is then renumbered in that search's order (neighbours get nearby numbers), so the second search and
  // the growth below walk memory locally; `label` maps the new numbers back.
  std::vector<int32_t> order;
  int64_t comp0 = bfs_order(nv, gx.data(), ga.data(), 0, order);
  std::vector<int32_t> label(order);  // new vertex -> old vertex
  std::unique_ptr<int32_t[]> adjr;
  {
    std::vector<int32_t> inv((size_t)nv);
    std::vector<int64_t> rx((size_t)nv + 1, 0);
    parallel_for(nv, threads, [&](int64_t lo, int64_t hi) {
      for (int64_t k = lo; k < hi; ++k) {
        const int32_t o = label[(size_t)k];
        inv[(size_t)o] = (int32_t)k;
        rx[(size_t)k + 1] = gx[(size_t)o + 1] - gx[(size_t)o];
      }
    });
    for (int64_t k = 0; k < nv; ++k) rx[(size_t)k + 1] += rx[(size_t)k];
    // the renumbered lists go to an uninitialised buffer, first touched by the threads that fill it
    adjr.reset(new int32_t[(size_t)rx[(size_t)nv] + 1]);
    int32_t* ra = adjr.get();
    parallel_for(nv, threads, [&](int64_t lo, int64_t hi) {  // in the old order: the old lists stream
      for (int64_t o = lo; o < hi; ++o) {
        int32_t* d = ra + rx[(size_t)inv[(size_t)o]];
        int64_t m = 0;
        for (int64_t e = gx[(size_t)o]; e < gx[(size_t)o + 1]; ++e) d[m++] = inv[(size_t)ga[(size_t)e]];
        std::sort(d, d + m);
      }
    });
    gx.swap(rx);
    UninitVec<int32_t>().swap(ga);
  }
  const int32_t* G = adjr.get();  // adjacency lists of the renumbered graph (offsets gx)
  const int32_t start = (int32_t)(comp0 - 1);  // the search's last vertex of the first component
  bfs_order(nv, gx.data(), G, start, order);

  int64_t maxdeg = 0;
  for (int64_t v = 0; v < nv; ++v) maxdeg = std::max(maxdeg, gx[(size_t)v + 1] - gx[(size_t)v]);
  std::vector<GrowState> gs((size_t)nv);
  parallel_for(nv, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t v = lo; v < hi; ++v) {
      const int32_t o = label[(size_t)v];
      gs[(size_t)v] = GrowState{0, 0, (int32_t)(first[(size_t)o + 1] - first[(size_t)o]), (int32_t)first[(size_t)o]};
    }
  });
  GainQueue q(gs, (int)maxdeg + 2);
  std::vector<int32_t> touched;  // vertices whose gain left 0 in the current part, in that order
  std::vector<RowRun> runs;      // the assignments in the order they are made
  runs.reserve((size_t)nv);
  int64_t cursor = 0, assigned = 0;
  auto next_free = [&]() -> int32_t {
    while (cursor < nv && gs[(size_t)order[(size_t)cursor]].left == 0) ++cursor;
    return cursor < nv ? order[(size_t)cursor] : -1;
  };
  int32_t p = 0, seed = start;
  while (assigned < n) {
    if (seed < 0 || gs[(size_t)seed].left == 0) seed = next_free();
    int32_t size = 0;
    // take as many of v's remaining rows as the part holds
    auto add = [&](int32_t v) {
      GrowState& sv = gs[(size_t)v];
      const int32_t take = std::min(sv.left, cap - size);
      runs.push_back(RowRun{sv.next_row, take, p});
      sv.next_row += take;
      sv.left -= take;
      size += take;
      assigned += take;
      if (sv.left > 0) return;
      for (int64_t e = gx[(size_t)v]; e < gx[(size_t)v + 1]; ++e) {
        const int32_t u = G[(size_t)e];
        GrowState& su = gs[(size_t)u];
        ++su.done_nb;
        if (su.left == 0) continue;
        if (su.conn == 0) touched.push_back(u);
        q.raise(u, ++su.conn);
      }
    };
    add(seed);
    while (size < cap && assigned < n) {
      int32_t v = -1;
      if (!q.pop(v)) v = next_free();  // frontier exhausted: continue this part elsewhere in sweep order
      if (v < 0) break;
      {  // prefetch for the likely next pops: offsets and state three ahead, the list one ahead, and the
         // states of the next one's neighbours (hints only; the order of the growth does not depend on them)
        const int32_t c1 = q.peek(0), c2 = q.peek(1), c3 = q.peek(3);
        if (c3 >= 0) {
          __builtin_prefetch(&gx[(size_t)c3]);
          __builtin_prefetch(&gs[(size_t)c3]);
        }
        if (c2 >= 0) __builtin_prefetch(&G[(size_t)gx[(size_t)c2]]);
        if (c1 >= 0)
          for (int64_t e = gx[(size_t)c1]; e < gx[(size_t)c1 + 1]; ++e) __builtin_prefetch(&gs[(size_t)G[(size_t)e]]);
      }
      add(v);
    }
    // next seed: the free neighbour of this part with the most already-assigned neighbours (a vertex
    // split by the full part stays free and joins whichever part reaches it).  The free neighbours are the
    // touched vertices still free, listed in the order a scan of the part's vertices and their lists first
    // meets them; the first of the best wins.
    seed = -1;
    int32_t best = -1;
    for (int32_t u : touched) {
      GrowState& su = gs[(size_t)u];
      su.conn = 0;
      if (su.left > 0 && su.done_nb > best) {
        best = su.done_nb;
        seed = u;
      }
    }
    touched.clear();
    q.clear();
    ++p;
  }
  parallel_for((int64_t)runs.size(), threads, [&](int64_t lo, int64_t hi) {  // the runs' rows are disjoint
    for (int64_t k = lo; k < hi; ++k) {
      const RowRun& r = runs[(size_t)k];
      std::fill(part.data() + r.row, part.data() + r.row + r.count, r.p);
    }
  });
  return p;
}

// ---------------------------------------------------------------- Alg. 1 + Alg. 2

// sets every element of v to zero, in contiguous pieces on `threads` threads
template <class V>
static void zero_parallel(V& v, int threads) {
  using T = typename V::value_type;
  if (v.empty()) return;
  T* d = v.data();
  parallel_for((int64_t)v.size(), threads, [d](int64_t lo, int64_t hi) {
    std::memset((void*)(d + lo), 0, (size_t)(hi - lo) * sizeof(T));
  }, 1 << 16);
}

int build_plan(const PlanParams& prm, const int64_t* rp, const int32_t* col, const double* val, HostPlan& P) {
  const double t0 = now_ms();
  const int64_t n = prm.n;
  const int64_t nnz = n > 0 ? rp[n] : 0;
  const int T = planner_threads(prm.threads);
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
    // the multilevel scheme is meant for parts on the order of the SM count; for very many tiny parts
    // (more than kMaxMultilevelParts) greedy growing is used instead
    const int64_t want = prm.slice_rows > 0 ? (n + prm.slice_rows - 1) / prm.slice_rows : n;
    nparts = prm.partitioner == 1 && want <= kMaxMultilevelParts
                 ? partition_multilevel(n, rp, col, prm.slice_rows, prm.seed, part, prm.threads)
                 : partition_graph(n, rp, col, prm.slice_rows, part, prm.threads);
  }
  P.nparts = nparts;
  const double t1 = now_ms();
  P.partition_ms = t1 - t0;

  // S_array1 / S_array2: in-partition (slab) and extra-row entry counts of every row
  const int64_t cap = prm.ell_width_cap > 0 ? prm.ell_width_cap : INT64_MAX;
  std::vector<int32_t> cin((size_t)n), cer((size_t)n);
  parallel_for(n, T, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      int64_t a = 0, b = 0;
      const int32_t pi = part[(size_t)i];
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        if (part[(size_t)col[k]] == pi && a < cap) ++a;
        else ++b;
      }
      cin[(size_t)i] = (int32_t)a;
      cer[(size_t)i] = (int32_t)b;
    }
  });

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
  for (int32_t p = 0; p < nparts; ++p)
    P.max_part_rows = std::max(P.max_part_rows, P.part_ptr[(size_t)p + 1] - P.part_ptr[(size_t)p]);
  if (P.max_part_rows > 65536) return 4;  // the 16-bit column offset would overflow
  parallel_for(nparts, T, [&](int64_t lo, int64_t hi) {
    for (int64_t p = lo; p < hi; ++p) {
      auto b = P.new_to_old.begin() + P.part_ptr[(size_t)p], e = P.new_to_old.begin() + P.part_ptr[(size_t)p + 1];
      // Alg. 1 sorts by in-partition count, descending; ties go to the larger extra-row count first,
      // which keeps the extra-row widths of a 32-row slice close together (less slice padding)
      std::stable_sort(b, e, [&](int32_t a, int32_t c) {
        if (cin[(size_t)a] != cin[(size_t)c]) return cin[(size_t)a] > cin[(size_t)c];
        return cer[(size_t)a] > cer[(size_t)c];
      });
    }
  }, 1);
  P.old_to_new.resize((size_t)n);
  parallel_for(n, T, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi; ++r) P.old_to_new[(size_t)P.new_to_old[(size_t)r]] = (int32_t)r;
  });

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
      int32_t w = 0;  // er_layout 2: a row's extra-row slots follow its slab slots in the same slice
      for (int32_t r = r0; r < r1; ++r) {
        const int32_t i = P.new_to_old[(size_t)r];
        w = std::max(w, cin[(size_t)i] + (prm.er_layout == 2 ? cer[(size_t)i] : 0));
      }
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

  // er_layout 2: each partition's halo, the distinct plan-numbering columns of its rows' extra-row entries
  // that lie outside the partition, ascending; the kernel stages x at them after the partition's own slice
  P.halo_ptr.assign((size_t)nparts + 1, 0);
  P.halo_new.clear();
  P.halo_old.clear();
  P.max_stage_rows = P.max_part_rows;
  if (P.er_layout == 2) {
    std::vector<std::vector<int32_t>> halo((size_t)nparts);
    parallel_for(nparts, T, [&](int64_t lo, int64_t hi) {
      for (int64_t q = lo; q < hi; ++q) {
        std::vector<int32_t>& h = halo[(size_t)q];
        for (int32_t r = P.part_ptr[(size_t)q]; r < P.part_ptr[(size_t)q + 1]; ++r) {
          const int32_t i = P.new_to_old[(size_t)r];
          for (int64_t k = rp[i]; k < rp[(int64_t)i + 1]; ++k)
            if (part[(size_t)col[k]] != (int32_t)q) h.push_back(P.old_to_new[(size_t)col[k]]);
        }
        std::sort(h.begin(), h.end());
        h.erase(std::unique(h.begin(), h.end()), h.end());
      }
    }, 1);
    int64_t stage = P.max_part_rows;
    for (int32_t q = 0; q < nparts; ++q) {
      P.halo_ptr[(size_t)q + 1] = P.halo_ptr[(size_t)q] + (int64_t)halo[(size_t)q].size();
      stage = std::max<int64_t>(stage, (int64_t)(P.part_ptr[(size_t)q + 1] - P.part_ptr[(size_t)q]) +
                                           (int64_t)halo[(size_t)q].size());
    }
    if (stage > 65536) return 4;  // the 16-bit local column would overflow
    P.max_stage_rows = (int32_t)stage;
    P.halo_new.resize((size_t)P.halo_ptr[(size_t)nparts]);
    P.halo_old.resize(P.halo_new.size());
    parallel_for(nparts, T, [&](int64_t lo, int64_t hi) {
      for (int64_t q = lo; q < hi; ++q) {
        const std::vector<int32_t>& h = halo[(size_t)q];
        const int64_t o = P.halo_ptr[(size_t)q];
        for (size_t t = 0; t < h.size(); ++t) {
          P.halo_new[(size_t)o + t] = h[t];
          P.halo_old[(size_t)o + t] = P.new_to_old[(size_t)h[t]];
        }
      }
    }, 1);
  }

  // processing order of the slices inside each partition: longest estimated work first (an ER slot
  // gathers x from global memory and is counted twice).  er_layout 2 takes the estimate of layout 0 (slab
  // and extra widths of the slice taken apart), so both layouts process the slices in the same order and
  // the solvers' fused dot products, summed in that order, agree bit for bit.
  std::vector<int64_t> er_work;
  if (P.er_layout == 2) {
    er_work.assign((size_t)P.nslices, 0);
    for (int32_t p = 0; p < nparts; ++p) {
      const int32_t pb = P.part_ptr[(size_t)p], pe = P.part_ptr[(size_t)p + 1];
      for (int32_t s = P.slice_ptr[(size_t)p]; s < P.slice_ptr[(size_t)p + 1]; ++s) {
        const int32_t r0 = pb + (s - P.slice_ptr[(size_t)p]) * rps, r1 = std::min(pe, r0 + rps);
        int32_t wi = 0, we = 0;
        for (int32_t r = r0; r < r1; ++r) {
          wi = std::max(wi, cin[(size_t)P.new_to_old[(size_t)r]]);
          we = std::max(we, P.row_er_count[(size_t)r]);
        }
        er_work[(size_t)s] = 32 * (int64_t)((wi + tpr - 1) / tpr) + 2 * 32 * (int64_t)((we + tpr - 1) / tpr);
      }
    }
  }
  P.slice_order.resize((size_t)P.nslices);
  for (int32_t p = 0; p < nparts; ++p) {
    const int32_t s0 = P.slice_ptr[(size_t)p], s1 = P.slice_ptr[(size_t)p + 1];
    auto work = [&](int32_t s) {
      if (!er_work.empty()) return er_work[(size_t)s];
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
  // every slot starts at zero (padding slots keep value 0); the arrays are zeroed in parallel pieces
  P.ell_col.resize((size_t)stored);
  P.ell_val.resize((size_t)stored);
  P.er_col.resize((size_t)er_nnz);
  P.er_val.resize((size_t)er_nnz);
  P.er_scol.resize((size_t)er_stored);
  P.er_scol_old.resize((size_t)er_stored);
  P.er_sval.resize((size_t)er_stored);
  zero_parallel(P.ell_col, T);
  zero_parallel(P.ell_val, T);
  zero_parallel(P.er_col, T);
  zero_parallel(P.er_val, T);
  zero_parallel(P.er_scol, T);
  zero_parallel(P.er_scol_old, T);
  zero_parallel(P.er_sval, T);
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
  std::vector<int64_t> ell_part((size_t)T + 1, 0);
  std::atomic<int> piece{0};
  parallel_for(n, T, [&](int64_t lo, int64_t hi) {
    int64_t ell_sum = 0;
    for (int64_t r = lo; r < hi; ++r) {
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
        } else if (P.er_layout == 2) {  // after the row's slab slots; column into [own slice | halo]
          const int32_t cn = P.old_to_new[(size_t)c];
          int32_t local = cn - pb;
          if (part[(size_t)c] != p) {
            const int32_t* h0 = P.halo_new.data() + P.halo_ptr[(size_t)p];
            const int32_t* h1 = P.halo_new.data() + P.halo_ptr[(size_t)p + 1];
            local = (P.part_ptr[(size_t)p + 1] - pb) + (int32_t)(std::lower_bound(h0, h1, cn) - h0);
          }
          const int64_t jj = cin[(size_t)i] + je;
          const int64_t pos = base + 32 * (jj / tpr) + lane0 + (int32_t)(jj % tpr);
          P.ell_col[(size_t)pos] = (uint16_t)local;
          P.ell_val[(size_t)pos] = val[k];
          ++je;
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
      ell_sum += j;
    }
    ell_part[(size_t)piece.fetch_add(1)] = ell_sum;
  });
  for (int64_t v : ell_part) P.ell_nnz += v;
  make_lowp_copies(P, prm.lowp, prm.lowp_group, prm.threads);
  P.reorder_ms = now_ms() - t1;
  return 0;
}

}  // namespace ehyb
