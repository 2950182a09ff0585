// Multilevel partitioner for the planner's PartVec (Sec. 3.1 cuts the graph of A with METIS's multilevel
// scheme; this is the Karypis-Kumar scheme written from its published description):
//
//   * the graph: one vertex per supervariable (weight = its rows), an edge wherever two supervariables'
//     rows are adjacent in A + A^T, weighted by the entries it stands for (the product of the two row
//     counts), so the cut weight is the count of entries that leave their partition (the ER entries); it
//     is renumbered breadth-first so that every later pass walks memory locally;
//   * coarsening, once for the whole graph: heavy-edge matching (vertices visited in seeded-shuffled blocks
//     of the numbering, each paired with the free neighbour across its heaviest edge), until about 20
//     vertices per part remain;
//   * initial partition of the coarsest graph into k = ceil(n / cap) parts by recursive bisection, each
//     bisection itself multilevel: heavy-edge coarsening, greedy graph growing from several seeds, and
//     Fiduccia-Mattheyses passes (boundary vertices moved by largest cut reduction, the best prefix of each
//     pass kept) on the way back up; the two halves run in parallel;
//   * uncoarsening with greedy k-way refinement: boundary vertices move to the adjacent part that gains the
//     most cut weight while parts stay within 3 % of the mean;
//   * exact part sizes, top-down over the bisection tree of part ids: at each node the heavy half gives its
//     best-gain boundary vertices to the light half until the left half holds exactly its share of the rows,
//     the last vertex split when it is heavier than what is left (a supervariable can straddle two parts,
//     as in the greedy partitioner), so every part ends with at most `cap` rows.
// Every step depends only on its input and the seed, so the result does not depend on the thread count.
#include <algorithm>
#include <cstdlib>
#include <thread>

#include "plan.h"

namespace ehyb {
namespace {

struct Graph {
  int64_t nv = 0;
  std::vector<int64_t> xadj;
  UninitVec<int32_t> adj;
  std::vector<int64_t> ew;    // edge weights, parallel to adj
  std::vector<int64_t> vw;    // vertex weights (rows)
  std::vector<int32_t> orig;  // top-level supervariable of each vertex (finest level of a bisection only)
  int64_t total() const {
    int64_t s = 0;
    for (int64_t w : vw) s += w;
    return s;
  }
};

// deterministic generator of the matching order and the growing seeds (splitmix64 stream)
struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(seed) {}
  uint64_t next() { return mix64(s++); }
  int64_t below(int64_t m) { return (int64_t)(next() % (uint64_t)m); }
};

void random_order(int64_t nv, Rng& r, std::vector<int32_t>& ord) {
  ord.resize((size_t)nv);
  for (int64_t i = 0; i < nv; ++i) ord[(size_t)i] = (int32_t)i;
  for (int64_t i = nv - 1; i > 0; --i) std::swap(ord[(size_t)i], ord[(size_t)r.below(i + 1)]);
}

// the matching order: blocks of kBlock consecutive vertices in index order, each block shuffled.  The
// graph is numbered breadth-first, so this keeps the walk local while the seed still varies the pairs.
constexpr int64_t kBlock = 256;
void blocked_order(int64_t nv, Rng& r, std::vector<int32_t>& ord) {
  ord.resize((size_t)nv);
  for (int64_t i = 0; i < nv; ++i) ord[(size_t)i] = (int32_t)i;
  for (int64_t b = 0; b < nv; b += kBlock) {
    const int64_t m = std::min(kBlock, nv - b);
    for (int64_t i = m - 1; i > 0; --i) std::swap(ord[(size_t)(b + i)], ord[(size_t)(b + r.below(i + 1))]);
  }
}

// adjacency built in parallel: worker k emits vertex i's list by fill(i, k, adj, ew) into its own buffers,
// which are then concatenated in vertex order, so the result does not depend on the thread count
template <typename F>
void build_lists(int64_t nv, int threads, Graph& out, F&& fill) {
  const int64_t t = std::max<int64_t>(1, std::min<int64_t>(threads, (nv + 16383) / 16384));
  std::vector<std::vector<int32_t>> adj((size_t)t);
  std::vector<std::vector<int64_t>> ew((size_t)t);
  out.xadj.assign((size_t)nv + 1, 0);
  auto run = [&](int64_t k) {
    const int64_t lo = nv * k / t, hi = nv * (k + 1) / t;
    std::vector<int32_t> a;  // worker-local until done (no shared cache lines while filling)
    std::vector<int64_t> w;
    for (int64_t i = lo; i < hi; ++i) {
      const size_t before = a.size();
      fill(i, k, a, w);
      out.xadj[(size_t)i + 1] = (int64_t)(a.size() - before);
    }
    adj[(size_t)k].swap(a);
    ew[(size_t)k].swap(w);
  };
  if (t == 1) {
    run(0);
  } else {
    std::vector<std::thread> th;
    for (int64_t k = 0; k < t; ++k) th.emplace_back(run, k);
    for (auto& x : th) x.join();
  }
  for (int64_t i = 0; i < nv; ++i) out.xadj[(size_t)i + 1] += out.xadj[(size_t)i];
  out.adj.resize((size_t)out.xadj[(size_t)nv]);
  out.ew.resize((size_t)out.xadj[(size_t)nv]);
  parallel_for(t, (int)t, [&](int64_t lo, int64_t hi) {
    for (int64_t k = lo; k < hi; ++k) {
      const int64_t at = out.xadj[(size_t)(nv * k / t)];
      std::copy(adj[(size_t)k].begin(), adj[(size_t)k].end(), out.adj.begin() + at);
      std::copy(ew[(size_t)k].begin(), ew[(size_t)k].end(), out.ew.begin() + at);
    }
  }, 1);
}

// max-heap of vertices keyed by gain (ties: smaller vertex first), with position index for updates
struct Heap {
  std::vector<int64_t> key;
  std::vector<int32_t> pos, h;
  explicit Heap(int64_t nv) : key((size_t)nv, 0), pos((size_t)nv, -1) {}
  bool better(int32_t a, int32_t b) const { return key[(size_t)a] > key[(size_t)b] || (key[(size_t)a] == key[(size_t)b] && a < b); }
  void place(size_t i, int32_t v) {
    h[i] = v;
    pos[(size_t)v] = (int32_t)i;
  }
  void up(size_t i) {
    const int32_t v = h[i];
    while (i > 0) {
      const size_t p = (i - 1) / 2;
      if (!better(v, h[p])) break;
      place(i, h[p]);
      i = p;
    }
    place(i, v);
  }
  void down(size_t i) {
    const int32_t v = h[i];
    for (;;) {
      size_t c = 2 * i + 1;
      if (c >= h.size()) break;
      if (c + 1 < h.size() && better(h[c + 1], h[c])) ++c;
      if (!better(h[c], v)) break;
      place(i, h[c]);
      i = c;
    }
    place(i, v);
  }
  bool has(int32_t v) const { return pos[(size_t)v] >= 0; }
  bool empty() const { return h.empty(); }
  int32_t top() const { return h[0]; }
  void set(int32_t v, int64_t k) {
    if (!has(v)) {
      key[(size_t)v] = k;
      h.push_back(v);
      up(h.size() - 1);
      return;
    }
    const int64_t old = key[(size_t)v];
    key[(size_t)v] = k;
    if (k > old) up((size_t)pos[(size_t)v]);
    else down((size_t)pos[(size_t)v]);
  }
  void remove(int32_t v) {
    const size_t i = (size_t)pos[(size_t)v];
    pos[(size_t)v] = -1;
    const int32_t last = h.back();
    h.pop_back();
    if (i < h.size()) {
      place(i, last);
      up(i);
      down((size_t)pos[(size_t)last]);
    }
  }
  int32_t pop() {
    const int32_t v = h[0];
    remove(v);
    return v;
  }
  void clear() {
    for (int32_t v : h) pos[(size_t)v] = -1;
    h.clear();
  }
};

// Two-way partition state: side[v] in {0, 1}, internal (id) and external (ed) edge weight of every
// vertex, the side weights and the cut.  The gain of moving v is ed[v] - id[v].
struct Bisection {
  const Graph& g;
  std::vector<uint8_t> side;
  std::vector<int64_t> id, ed;
  int64_t w[2] = {0, 0};
  int64_t cut = 0;
  explicit Bisection(const Graph& gr) : g(gr) {}
  void compute() {
    id.assign((size_t)g.nv, 0);
    ed.assign((size_t)g.nv, 0);
    w[0] = w[1] = 0;
    cut = 0;
    for (int64_t v = 0; v < g.nv; ++v) {
      w[side[(size_t)v]] += g.vw[(size_t)v];
      for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e) {
        if (side[(size_t)g.adj[(size_t)e]] == side[(size_t)v]) id[(size_t)v] += g.ew[(size_t)e];
        else ed[(size_t)v] += g.ew[(size_t)e];
      }
      cut += ed[(size_t)v];
    }
    cut /= 2;
  }
  int64_t gain(int32_t v) const { return ed[(size_t)v] - id[(size_t)v]; }
  // move v to the other side; `touch(u)` is called for every neighbour after its id/ed change
  template <typename F>
  void move(int32_t v, F&& touch) {
    const uint8_t from = side[(size_t)v], to = (uint8_t)(1 - from);
    cut -= gain(v);
    std::swap(id[(size_t)v], ed[(size_t)v]);
    side[(size_t)v] = to;
    w[from] -= g.vw[(size_t)v];
    w[to] += g.vw[(size_t)v];
    for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e) {
      const int32_t u = g.adj[(size_t)e];
      const int64_t we = g.ew[(size_t)e];
      if (side[(size_t)u] == to) {
        id[(size_t)u] += we;
        ed[(size_t)u] -= we;
      } else {
        id[(size_t)u] -= we;
        ed[(size_t)u] += we;
      }
      touch(u);
    }
  }
};

// is state (cut a, imbalance ia) better than (cut b, imbalance ib) under tolerance tol?
bool better_state(int64_t a, int64_t ia, int64_t b, int64_t ib, int64_t tol) {
  const bool oka = ia <= tol, okb = ib <= tol;
  if (oka != okb) return oka;
  if (!oka) return ia < ib || (ia == ib && a < b);
  return a < b || (a == b && ia < ib);
}

// Fiduccia-Mattheyses refinement of a bisection toward side-0 weight t0 within tol
void fm_refine(Bisection& B, int64_t t0, int64_t tol, int max_passes) {
  const Graph& g = B.g;
  const int64_t limit = std::min<int64_t>(std::max<int64_t>(g.nv / 100, 15), 100);
  Heap q0(g.nv), q1(g.nv);
  Heap* q[2] = {&q0, &q1};
  std::vector<uint8_t> locked((size_t)g.nv, 0);
  std::vector<int32_t> moved;
  for (int pass = 0; pass < max_passes; ++pass) {
    for (int64_t v = 0; v < g.nv; ++v)
      if (B.ed[(size_t)v] > 0) q[B.side[(size_t)v]]->set((int32_t)v, B.gain((int32_t)v));
    moved.clear();
    int64_t best_cut = B.cut, best_imb = std::llabs(B.w[0] - t0);
    size_t best_n = 0;
    int64_t bad = 0;
    auto touch = [&](int32_t u) {
      if (locked[(size_t)u]) return;
      Heap* hq = q[B.side[(size_t)u]];
      if (B.ed[(size_t)u] > 0) hq->set(u, B.gain(u));
      else if (hq->has(u)) hq->remove(u);
    };
    for (;;) {
      int from = B.w[0] > t0 ? 0 : 1;
      if (q[from]->empty()) {
        // the heavy side has no boundary vertex: the light side may still give one within tolerance
        if (q[1 - from]->empty()) break;
        const int32_t c = q[1 - from]->top();
        const int64_t nw0 = B.w[0] + (from == 0 ? g.vw[(size_t)c] : -g.vw[(size_t)c]);
        if (std::llabs(nw0 - t0) > tol) break;
        from = 1 - from;
      }
      const int32_t v = q[from]->top();
      const int64_t nw0 = B.w[0] + (from == 0 ? -g.vw[(size_t)v] : g.vw[(size_t)v]);
      const int64_t imb = std::llabs(B.w[0] - t0), nimb = std::llabs(nw0 - t0);
      if (nimb > tol && nimb > imb) break;  // the move would break the balance
      q[from]->pop();
      locked[(size_t)v] = 1;
      B.move(v, touch);
      moved.push_back(v);
      if (better_state(B.cut, nimb, best_cut, best_imb, tol)) {
        best_cut = B.cut;
        best_imb = nimb;
        best_n = moved.size();
        bad = 0;
      } else if (++bad > limit) {
        break;
      }
    }
    auto none = [](int32_t) {};
    for (size_t i = moved.size(); i > best_n; --i) B.move(moved[i - 1], none);
    for (int32_t v : moved) locked[(size_t)v] = 0;
    q0.clear();
    q1.clear();
    if (best_n == 0) break;
  }
}

// greedy graph growing from seed s: side 0 grows by largest gain until it holds about t0
void grow(Bisection& B, int32_t s, int64_t t0, const std::vector<int32_t>& ord) {
  const Graph& g = B.g;
  B.side.assign((size_t)g.nv, 1);
  B.compute();
  Heap q(g.nv);
  auto touch = [&](int32_t u) {
    if (B.side[(size_t)u] == 1) q.set(u, B.gain(u));
  };
  size_t cursor = 0;
  int32_t v = s;
  while (true) {
    if (q.has(v)) q.remove(v);
    B.move(v, touch);
    if (B.w[0] >= t0) break;
    if (!q.empty()) {
      v = q.top();
    } else {
      while (cursor < ord.size() && B.side[(size_t)ord[cursor]] == 0) ++cursor;
      if (cursor == ord.size()) break;
      v = ord[cursor];
    }
    // stop where taking v would overshoot the target by more than stopping undershoots it
    if (B.w[0] + g.vw[(size_t)v] - t0 > t0 - B.w[0]) break;
  }
}

// heavy-edge matching: returns the coarse graph and cmap (fine vertex -> coarse vertex)
void coarsen(const Graph& g, int64_t maxvw, Rng& r, int threads, Graph& c, std::vector<int32_t>& cmap) {
  std::vector<int32_t> ord, match((size_t)g.nv, -1);
  blocked_order(g.nv, r, ord);
  for (int32_t v : ord) {
    if (match[(size_t)v] >= 0) continue;
    int32_t best = v;
    int64_t bw = -1;
    for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e) {
      const int32_t u = g.adj[(size_t)e];
      if (match[(size_t)u] >= 0 || g.vw[(size_t)v] + g.vw[(size_t)u] > maxvw) continue;
      if (g.ew[(size_t)e] > bw) {
        bw = g.ew[(size_t)e];
        best = u;
      }
    }
    match[(size_t)v] = best;
    match[(size_t)best] = v;
  }
  // the smaller vertex of a pair (or a single vertex) numbers the coarse vertex
  cmap.assign((size_t)g.nv, -1);
  std::vector<int32_t> rep;
  rep.reserve((size_t)g.nv / 2 + 1);
  for (int64_t v = 0; v < g.nv; ++v)
    if (match[(size_t)v] >= v) {
      cmap[(size_t)v] = (int32_t)rep.size();
      cmap[(size_t)match[(size_t)v]] = (int32_t)rep.size();
      rep.push_back((int32_t)v);
    }
  const int64_t nc = (int64_t)rep.size();
  c.nv = nc;
  c.vw.resize((size_t)nc);
  for (int64_t cv = 0; cv < nc; ++cv) {
    const int32_t v = rep[(size_t)cv], u = match[(size_t)v];
    c.vw[(size_t)cv] = g.vw[(size_t)v] + (u != v ? g.vw[(size_t)u] : 0);
  }
  // coarse lists: the union of the pair's lists, weights of parallel edges summed, self edges dropped
  const int64_t t = std::max<int64_t>(1, std::min<int64_t>(threads, (nc + 16383) / 16384));
  std::vector<std::vector<int64_t>> slots((size_t)t);  // per worker: position of a coarse neighbour in its list
  build_lists(nc, (int)t, c, [&](int64_t cv, int64_t worker, std::vector<int32_t>& a, std::vector<int64_t>& w) {
    std::vector<int64_t>& slot = slots[(size_t)worker];
    if (slot.empty()) slot.assign((size_t)nc, -1);
    const int64_t begin = (int64_t)a.size();
    const int32_t pair[2] = {rep[(size_t)cv], match[(size_t)rep[(size_t)cv]]};
    for (int h = 0; h < (pair[1] == pair[0] ? 1 : 2); ++h) {
      const int32_t f = pair[h];
      for (int64_t e = g.xadj[(size_t)f]; e < g.xadj[(size_t)f + 1]; ++e) {
        const int32_t cu = cmap[(size_t)g.adj[(size_t)e]];
        if (cu == cv) continue;
        int64_t& sl = slot[(size_t)cu];
        if (sl >= begin) {  // already in this list (positions only grow within a worker's buffer)
          w[(size_t)sl] += g.ew[(size_t)e];
        } else {
          sl = (int64_t)a.size();
          a.push_back(cu);
          w.push_back(g.ew[(size_t)e]);
        }
      }
    }
  });
}

constexpr int64_t kCoarsest = 120;  // a bisection coarsens its graph to about this many vertices
constexpr int kTrials = 6;          // growing seeds tried on the coarsest graph of a bisection
constexpr int64_t kPerPart = 20;    // the global hierarchy stops at about this many vertices per part

int64_t max_weight(const Graph& h) {
  int64_t m = 1;
  for (int64_t w : h.vw) m = std::max(m, w);
  return m;
}

// Multilevel bisection of a (small) graph: side 0 gets about t0 of the weight
void bisect(const Graph& g, int64_t t0, uint64_t seed, std::vector<uint8_t>& side) {
  const int64_t W = g.total();
  Rng r(seed);
  std::vector<Graph> lv;
  lv.reserve(48);
  std::vector<std::vector<int32_t>> cmaps;
  const Graph* cur = &g;
  const int64_t maxvw = std::max<int64_t>(1, (3 * W) / (2 * kCoarsest));
  while (cur->nv > kCoarsest && lv.size() < 48) {
    Graph c;
    std::vector<int32_t> cm;
    coarsen(*cur, maxvw, r, 1, c, cm);
    if (c.nv > (cur->nv * 9) / 10) break;  // matching no longer shrinks the graph
    lv.push_back(std::move(c));
    cmaps.push_back(std::move(cm));
    cur = &lv.back();
  }
  // initial bisection: greedy growing from several seeds, each refined; the best kept
  std::vector<uint8_t> best;
  {
    const Graph& c = *cur;
    const int64_t tol = std::max<int64_t>(max_weight(c), W / 100);
    int64_t best_cut = 0, best_imb = 0;
    std::vector<int32_t> ord;
    random_order(c.nv, r, ord);
    for (int t = 0; t < kTrials && t < c.nv; ++t) {
      Bisection B(c);
      grow(B, ord[(size_t)t], t0, ord);
      fm_refine(B, t0, tol, 8);
      const int64_t imb = std::llabs(B.w[0] - t0);
      if (best.empty() || better_state(B.cut, imb, best_cut, best_imb, tol)) {
        best_cut = B.cut;
        best_imb = imb;
        best = B.side;
      }
    }
  }
  // uncoarsening: project and refine at every level
  for (size_t l = lv.size(); l-- > 0;) {
    const Graph& fine = l == 0 ? g : lv[l - 1];
    std::vector<uint8_t> s((size_t)fine.nv);
    for (int64_t v = 0; v < fine.nv; ++v) s[(size_t)v] = best[(size_t)cmaps[l][(size_t)v]];
    Bisection B(fine);
    B.side.swap(s);
    B.compute();
    fm_refine(B, t0, std::max<int64_t>(max_weight(fine), W / 200), 4);
    best.swap(B.side);
  }
  side.swap(best);
}

// subgraph of the vertices with side == s; orig carries over
void extract(const Graph& g, const std::vector<uint8_t>& side, uint8_t s, Graph& out) {
  std::vector<int32_t> idx((size_t)g.nv, -1), keep;
  for (int64_t v = 0; v < g.nv; ++v)
    if (side[(size_t)v] == s) {
      idx[(size_t)v] = (int32_t)keep.size();
      keep.push_back((int32_t)v);
    }
  const int64_t m = (int64_t)keep.size();
  out.nv = m;
  out.vw.resize((size_t)m);
  out.orig.resize((size_t)m);
  for (int64_t i = 0; i < m; ++i) {
    out.vw[(size_t)i] = g.vw[(size_t)keep[(size_t)i]];
    out.orig[(size_t)i] = g.orig[(size_t)keep[(size_t)i]];
  }
  build_lists(m, 1, out, [&](int64_t i, int64_t, std::vector<int32_t>& a, std::vector<int64_t>& w) {
    const int32_t v = keep[(size_t)i];
    for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e)
      if (idx[(size_t)g.adj[(size_t)e]] >= 0) {
        a.push_back(idx[(size_t)g.adj[(size_t)e]]);
        w.push_back(g.ew[(size_t)e]);
      }
  });
}

// the side-0 share of a node of the bisection tree with weight W and k = kl + kr parts of at most cap
int64_t left_target(int64_t W, int32_t k, int64_t cap) {
  const int32_t kl = k / 2, kr = k - kl;
  const int64_t t = (W * kl + k / 2) / k;
  return std::min<int64_t>(std::max<int64_t>(t, W - (int64_t)kr * cap), (int64_t)kl * cap);
}

// initial k-way partition of the coarsest graph by recursive bisection: part[orig[v]] for its vertices
void rb(const Graph& g, int32_t k, int32_t p0, uint64_t seed, int threads, std::vector<int32_t>& part) {
  if (k == 1 || g.nv == 0) {
    for (int64_t v = 0; v < g.nv; ++v) part[(size_t)g.orig[(size_t)v]] = p0;
    return;
  }
  const int32_t kl = k / 2, kr = k - kl;
  std::vector<uint8_t> side;
  const int64_t W = g.total();
  bisect(g, (W * kl + k / 2) / k, mix64(seed ^ ((uint64_t)p0 << 32) ^ (uint64_t)k), side);
  Graph L, R;
  extract(g, side, 0, L);
  extract(g, side, 1, R);
  if (threads > 1) {  // the halves write disjoint entries of part
    const int tr = threads / 2;
    std::thread th([&]() { rb(R, kr, p0 + kl, seed, tr, part); });
    rb(L, kl, p0, seed, threads - tr, part);
    th.join();
  } else {
    rb(L, kl, p0, seed, 1, part);
    rb(R, kr, p0 + kl, seed, 1, part);
  }
}

// Greedy k-way refinement: boundary vertices move to the adjacent part that gains the most cut weight
// while that part stays under maxw; a vertex of a part above maxw moves even at a loss.  Only vertices that
// touch another part are visited (the list grows by the neighbours of every moved vertex).
void kway_refine(const Graph& g, int32_t k, std::vector<int32_t>& part, std::vector<int64_t>& pw, int64_t maxw,
                 int passes, int threads) {
  std::vector<uint8_t> in((size_t)g.nv, 0);
  parallel_for(g.nv, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t v = lo; v < hi; ++v)
      for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e)
        if (part[(size_t)g.adj[(size_t)e]] != part[(size_t)v]) {
          in[(size_t)v] = 1;
          break;
        }
  });
  std::vector<int32_t> list;
  for (int64_t v = 0; v < g.nv; ++v)
    if (in[(size_t)v]) list.push_back((int32_t)v);
  std::vector<int64_t> conn((size_t)k, 0);
  std::vector<int32_t> touched;
  for (int pass = 0; pass < passes; ++pass) {
    int64_t moves = 0;
    for (size_t i = 0; i < list.size(); ++i) {
      const int32_t v = list[i];
      const int32_t a = part[(size_t)v];
      touched.clear();
      for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e) {
        const int32_t q = part[(size_t)g.adj[(size_t)e]];
        if (conn[(size_t)q] == 0) touched.push_back(q);
        conn[(size_t)q] += g.ew[(size_t)e];
      }
      int32_t best = -1;
      int64_t bg = 0;
      const int64_t wv = g.vw[(size_t)v];
      for (int32_t q : touched) {
        if (q == a || pw[(size_t)q] + wv > maxw) continue;
        const int64_t gain = conn[(size_t)q] - conn[(size_t)a];
        if (best < 0 || gain > bg || (gain == bg && pw[(size_t)q] < pw[(size_t)best])) {
          best = q;
          bg = gain;
        }
      }
      for (int32_t q : touched) conn[(size_t)q] = 0;
      if (best < 0) continue;
      const bool over = pw[(size_t)a] > maxw;
      const bool evens = bg == 0 && pw[(size_t)best] + wv < pw[(size_t)a];
      if (bg > 0 || evens || over) {
        part[(size_t)v] = best;
        pw[(size_t)a] -= wv;
        pw[(size_t)best] += wv;
        ++moves;
        for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e) {
          const int32_t u = g.adj[(size_t)e];
          if (!in[(size_t)u]) {
            in[(size_t)u] = 1;
            list.push_back(u);
          }
        }
      }
    }
    if (moves * 1000 < (int64_t)list.size()) break;  // under 0.1 % of the boundary moved
  }
}

// A piece of a vertex's rows that was split off into another part by the exact balancing
struct Piece {
  int32_t v, part;
  int64_t w;
};

// Exact part weights, top-down over the bisection tree of part ids: at node [lo, hi) the parts
// [lo, lo + k/2) must hold exactly left_target of the node's weight.  Vertices of the heavy half that touch
// the light half move there by largest gain (to their best-connected light part); a vertex heavier than
// what is left to move is split, its excess becoming a Piece.  Without a boundary between the halves,
// vertices (then pieces) of the heavy half move to the lightest part of the light half.
struct Balancer {
  const Graph& g;
  int32_t k;
  int64_t cap;
  std::vector<int32_t>& part;
  std::vector<int64_t>& vw;  // the graph's vertex weights, reduced by splits
  std::vector<int64_t>& pw;
  std::vector<Piece>& pieces;
  std::vector<std::vector<int32_t>> bl;  // per part: vertices that touch (or touched) another part; an entry
  std::vector<uint8_t> inbl;             // whose vertex has since left the part is skipped
  std::vector<int64_t> conn;
  std::vector<int32_t> touched;
  Heap q;
  Balancer(const Graph& gr, int32_t kk, int64_t c, std::vector<int32_t>& p, std::vector<int64_t>& w,
           std::vector<int64_t>& parts_w, std::vector<Piece>& pc, int threads)
      : g(gr), k(kk), cap(c), part(p), vw(w), pw(parts_w), pieces(pc), bl((size_t)kk), inbl((size_t)gr.nv, 0),
        conn((size_t)kk, 0), q(gr.nv) {
    parallel_for(g.nv, threads, [&](int64_t lo, int64_t hi) {
      for (int64_t v = lo; v < hi; ++v)
        for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e)
          if (part[(size_t)g.adj[(size_t)e]] != part[(size_t)v]) {
            inbl[(size_t)v] = 1;
            break;
          }
    });
    for (int64_t v = 0; v < g.nv; ++v)
      if (inbl[(size_t)v]) bl[(size_t)part[(size_t)v]].push_back((int32_t)v);
  }
  // best light part [l0, l1) adjacent to v and the gain of moving v there (-1 part when none)
  int32_t best_light(int32_t v, int32_t l0, int32_t l1, int64_t& gain) {
    touched.clear();
    for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e) {
      const int32_t p = part[(size_t)g.adj[(size_t)e]];
      if (conn[(size_t)p] == 0) touched.push_back(p);
      conn[(size_t)p] += g.ew[(size_t)e];
    }
    int32_t b = -1;
    for (int32_t p : touched)
      if (p >= l0 && p < l1 && (b < 0 || conn[(size_t)p] > conn[(size_t)b] ||
                                (conn[(size_t)p] == conn[(size_t)b] && pw[(size_t)p] < pw[(size_t)b])))
        b = p;
    gain = b >= 0 ? conn[(size_t)b] - conn[(size_t)part[(size_t)v]] : 0;
    for (int32_t p : touched) conn[(size_t)p] = 0;
    return b;
  }
  int32_t lightest(int32_t l0, int32_t l1) const {
    int32_t b = l0;
    for (int32_t p = l0 + 1; p < l1; ++p)
      if (pw[(size_t)p] < pw[(size_t)b]) b = p;
    return b;
  }
  // move `amount` (<= the owner's weight) of vertex v or of piece i from part a to part b
  void shift(int32_t v, int32_t b, int64_t amount) {
    const int32_t a = part[(size_t)v];
    pw[(size_t)a] -= amount;
    pw[(size_t)b] += amount;
    if (amount == vw[(size_t)v]) {
      part[(size_t)v] = b;
      if (inbl[(size_t)v]) bl[(size_t)b].push_back(v);
    } else {
      vw[(size_t)v] -= amount;
      pieces.push_back({v, b, amount});
    }
  }
  void settle(int32_t lo, int32_t hi) {
    if (hi - lo < 2) return;
    const int32_t kk = hi - lo, mid = lo + kk / 2;
    int64_t W = 0, wl = 0;
    for (int32_t p = lo; p < hi; ++p) W += pw[(size_t)p];
    for (int32_t p = lo; p < mid; ++p) wl += pw[(size_t)p];
    const int64_t t0 = left_target(W, kk, cap);
    int64_t excess = std::llabs(wl - t0);
    const bool left_heavy = wl > t0;
    const int32_t h0 = left_heavy ? lo : mid, h1 = left_heavy ? mid : hi;
    const int32_t l0 = left_heavy ? mid : lo, l1 = left_heavy ? hi : mid;
    auto heavy = [&](int32_t v) { return part[(size_t)v] >= h0 && part[(size_t)v] < h1; };
    if (excess > 0) {
      q.clear();
      for (int32_t p = h0; p < h1; ++p)
        for (int32_t v : bl[(size_t)p]) {
          if (part[(size_t)v] != p || q.has(v) || vw[(size_t)v] == 0) continue;
          int64_t gain;
          if (best_light(v, l0, l1, gain) >= 0) q.set(v, gain);
        }
      while (excess > 0 && !q.empty()) {
        const int32_t v = q.top();
        int64_t gain;
        const int32_t b = best_light(v, l0, l1, gain);
        if (b < 0 || gain != q.key[(size_t)v]) {  // stale entry: requeue with the current gain
          if (b < 0) q.remove(v);
          else q.set(v, gain);
          continue;
        }
        q.remove(v);
        const int64_t amount = std::min(excess, vw[(size_t)v]);
        shift(v, b, amount);
        excess -= amount;
        if (part[(size_t)v] != b) continue;  // split: the rest of v stays in the heavy half
        for (int64_t e = g.xadj[(size_t)v]; e < g.xadj[(size_t)v + 1]; ++e) {
          const int32_t u = g.adj[(size_t)e];
          if (!inbl[(size_t)u]) {
            inbl[(size_t)u] = 1;
            bl[(size_t)part[(size_t)u]].push_back(u);
          }
          if (!heavy(u) || vw[(size_t)u] == 0) continue;
          int64_t gu;
          if (best_light(u, l0, l1, gu) >= 0) q.set(u, gu);
        }
      }
      for (int64_t v = 0; v < g.nv && excess > 0; ++v)
        if (heavy((int32_t)v) && vw[(size_t)v] > 0) {
          const int64_t amount = std::min(excess, vw[(size_t)v]);
          shift((int32_t)v, lightest(l0, l1), amount);
          excess -= amount;
        }
      for (size_t i = 0; i < pieces.size() && excess > 0; ++i)
        if (pieces[i].part >= h0 && pieces[i].part < h1) {
          const int64_t amount = std::min(excess, pieces[i].w);
          const int32_t b = lightest(l0, l1);
          pw[(size_t)pieces[i].part] -= amount;
          pw[(size_t)b] += amount;
          if (amount == pieces[i].w) {
            pieces[i].part = b;
          } else {
            pieces[i].w -= amount;
            pieces.push_back({pieces[i].v, b, amount});
          }
          excess -= amount;
        }
    }
    settle(lo, mid);
    settle(mid, hi);
  }
};

}  // namespace

int32_t partition_multilevel(int64_t n, const int64_t* rp, const int32_t* col, int32_t cap, uint64_t seed,
                             std::vector<int32_t>& part, int threads) {
  part.assign((size_t)n, -1);
  if (n == 0) return 0;
  if (cap < 1) cap = 1;
  threads = planner_threads(threads);
  const int32_t k = (int32_t)((n + cap - 1) / cap);
  Graph g;
  std::vector<int64_t> first;
  {
    Graph s;
    s.nv = supervariable_graph(n, rp, col, threads, first, s.xadj, s.adj);
    // renumber in breadth-first order so that neighbours have nearby numbers: every level then walks
    // memory locally (the caller's numbering may be a random permutation)
    std::vector<int32_t> order, inv((size_t)s.nv);
    bfs_order(s.nv, s.xadj.data(), s.adj.data(), 0, order);
    for (int64_t i = 0; i < s.nv; ++i) inv[(size_t)order[(size_t)i]] = (int32_t)i;
    g.nv = s.nv;
    g.xadj.assign((size_t)g.nv + 1, 0);
    for (int64_t i = 0; i < g.nv; ++i) {
      const int32_t o = order[(size_t)i];
      g.xadj[(size_t)i + 1] = g.xadj[(size_t)i] + (s.xadj[(size_t)o + 1] - s.xadj[(size_t)o]);
    }
    g.adj.resize(s.adj.size());
    g.ew.resize(s.adj.size());
    g.vw.resize((size_t)g.nv);
    g.orig.resize((size_t)g.nv);
    parallel_for(g.nv, threads, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        const int32_t o = order[(size_t)i];
        const int64_t wo = first[(size_t)o + 1] - first[(size_t)o];
        g.vw[(size_t)i] = wo;
        g.orig[(size_t)i] = o;
        int64_t d = g.xadj[(size_t)i];
        for (int64_t e = s.xadj[(size_t)o]; e < s.xadj[(size_t)o + 1]; ++e, ++d) {
          const int32_t u = s.adj[(size_t)e];
          g.adj[(size_t)d] = inv[(size_t)u];
          g.ew[(size_t)d] = wo * (first[(size_t)u + 1] - first[(size_t)u]);  // entries the edge stands for
        }
      }
    });
  }
  // the global hierarchy
  Rng r(seed);
  std::vector<Graph> lv;
  lv.reserve(64);
  std::vector<std::vector<int32_t>> cmaps;
  const Graph* cur = &g;
  const int64_t W = n;
  const int64_t stop = std::max<int64_t>(kPerPart * k, kCoarsest);
  const int64_t maxvw = std::max<int64_t>(1, (3 * W) / (2 * stop));
  while (cur->nv > stop && lv.size() < 64) {
    Graph c;
    std::vector<int32_t> cm;
    coarsen(*cur, maxvw, r, threads, c, cm);
    if (c.nv > (cur->nv * 9) / 10) break;
    lv.push_back(std::move(c));
    cmaps.push_back(std::move(cm));
    cur = &lv.back();
  }
  // initial partition of the coarsest graph
  std::vector<int32_t> cp((size_t)cur->nv, 0);
  {
    Graph c = *cur;
    c.orig.resize((size_t)c.nv);
    for (int64_t v = 0; v < c.nv; ++v) c.orig[(size_t)v] = (int32_t)v;
    rb(c, k, 0, seed, threads, cp);
  }
  // uncoarsening with k-way refinement (parts within 3 % of the mean)
  const int64_t maxw = (W * 103 + 100 * (int64_t)k - 1) / (100 * (int64_t)k);
  for (size_t l = lv.size() + 1; l-- > 0;) {
    const Graph& h = l == 0 ? g : lv[l - 1];
    if (l < lv.size()) {
      std::vector<int32_t> fp((size_t)h.nv);
      for (int64_t v = 0; v < h.nv; ++v) fp[(size_t)v] = cp[(size_t)cmaps[l][(size_t)v]];
      cp.swap(fp);
    }
    std::vector<int64_t> pw((size_t)k, 0);
    for (int64_t v = 0; v < h.nv; ++v) pw[(size_t)cp[(size_t)v]] += h.vw[(size_t)v];
    kway_refine(h, k, cp, pw, maxw, l == 0 ? 4 : 3, threads);
  }
  // exact weights: every part ends with its share of the rows, at most cap
  std::vector<int64_t> vw(g.vw), pw((size_t)k, 0);
  for (int64_t v = 0; v < g.nv; ++v) pw[(size_t)cp[(size_t)v]] += vw[(size_t)v];
  std::vector<Piece> pieces;
  Balancer(g, k, cap, cp, vw, pw, pieces, threads).settle(0, k);
  // rows of each supervariable go to its parts in part order: whole vertices in parallel, then the few
  // vertices with split-off pieces
  std::vector<uint8_t> split((size_t)g.nv, 0);
  for (const Piece& pc : pieces) split[(size_t)pc.v] = 1;
  parallel_for(g.nv, threads, [&](int64_t lo, int64_t hi) {
    for (int64_t v = lo; v < hi; ++v) {
      if (split[(size_t)v]) continue;
      const int32_t o = g.orig[(size_t)v];
      for (int64_t row = first[(size_t)o]; row < first[(size_t)o + 1]; ++row) part[(size_t)row] = cp[(size_t)v];
    }
  });
  for (int64_t v = 0; v < g.nv; ++v)
    if (split[(size_t)v] && vw[(size_t)v] > 0) pieces.push_back({(int32_t)v, cp[(size_t)v], vw[(size_t)v]});
  std::sort(pieces.begin(), pieces.end(), [](const Piece& a, const Piece& b) {
    return a.v < b.v || (a.v == b.v && a.part < b.part);
  });
  for (size_t i = 0; i < pieces.size();) {
    const int32_t v = pieces[i].v;
    int64_t row = first[(size_t)g.orig[(size_t)v]];
    for (; i < pieces.size() && pieces[i].v == v; ++i)
      for (int64_t j = 0; j < pieces[i].w; ++j) part[(size_t)row++] = pieces[i].part;
  }
  return k;
}

}  // namespace ehyb
