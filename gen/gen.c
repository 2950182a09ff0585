/*
 * Seeded synthetic inputs: finite-element stiffness matrices on jittered
 * structured meshes, delivered in CSR after a seeded symmetric node relabelling,
 * plus seeded uniform vectors.  These stand in for the unstructured-mesh FEM
 * matrices (structural, CFD, electromagnetic problems) on which the EHYB paper
 * measures its SpMV (Sec. 5).  Nothing here knows about the EHYB format: the
 * generators only produce A (and x), in the same way for the CUDA path and the
 * CPU oracle.
 *
 * Families (all symmetric; the row order is randomised by a node relabelling):
 *   - 2D P1 Laplacian on a triangulated N x N node grid (SW-NE diagonal split):
 *     7-point pattern, nnz = N^2 + 2(2N(N-1) + (N-1)^2).
 *   - 3D trilinear (Q1) hexahedral isotropic elasticity, 3 dof per node,
 *     2x2x2 Gauss quadrature: 27 neighbour nodes x 9, nnz = 9 (3N-2)^3.
 *   - 3D Q1 hexahedral scalar Laplacian: nnz = (3N-2)^3.
 *   - 3D P1 tetrahedral Laplacian on the Freudenthal (Kuhn) 6-tet split of each
 *     cube: 15-point pattern, nnz = N^3 + 2(3N^2(N-1) + 3N(N-1)^2 + (N-1)^3).
 *
 * Determinism: pure integer hashing for random numbers (splitmix64 finaliser
 * applied to a counter), a single thread, fixed loop orders, and only +,-,*,/
 * and sqrt (all correctly rounded).  Compile with -ffp-contract=off so that the
 * results are bit-identical on x86-64 and aarch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ RNG */

/* splitmix64 output function (Steele, Lea & Flood, 2014), used as a hash. */
static uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Counter-based stream: value number `ctr` of stream (`seed`, `stream`). */
static uint64_t rng64(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return mix64(mix64(seed ^ 0xD1B54A32D192ED03ULL) ^ mix64(stream * 0x9E3779B97F4A7C15ULL + ctr));
}

/* Uniform double in [0, 1) with 53 random bits. */
static double u01(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return (double)(rng64(seed, stream, ctr) >> 11) * (1.0 / 9007199254740992.0);
}

/* Uniform integer in [0, m) by multiply-high (Lemire's reduction, no rejection). */
static uint64_t below(uint64_t r, uint64_t m) {
  return (uint64_t)(((unsigned __int128)r * (unsigned __int128)m) >> 64);
}

void gen_uniform(int64_t n, uint64_t seed, double lo, double hi, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * u01(seed, 0x5EEDULL, (uint64_t)i);
}

/* Fisher-Yates shuffle: perm[old] = new label.  Returns 0. */
int gen_permutation(int64_t n, uint64_t seed, int32_t* perm) {
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    int64_t j = (int64_t)below(rng64(seed, 0x9E7ULL, (uint64_t)i), (uint64_t)(i + 1));
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  return 0;
}

/* ------------------------------------------------------------ meshes */

/* Structured node grid with jittered coordinates.  Nodes (i,j,k), i fastest. */
typedef struct {
  int dim, N;
  int64_t nn;           /* nodes */
  double h, jitter;     /* spacing, jitter amplitude as a fraction of h */
  uint64_t seed;
  int32_t* attempt;     /* per-node redraw counter; -1 = unjittered */
  double* xyz;          /* nn x 3 */
} grid_t;

static void grid_node_coord(const grid_t* g, int64_t node, double* p) {
  int64_t i = node % g->N, j = (node / g->N) % g->N, k = node / ((int64_t)g->N * g->N);
  double base[3] = { i * g->h, j * g->h, g->dim == 3 ? k * g->h : 0.0 };
  for (int d = 0; d < 3; ++d) {
    double off = 0.0;
    if (d < g->dim && g->attempt[node] >= 0) {
      double u = u01(g->seed, (uint64_t)node * 4u + (uint64_t)d, (uint64_t)g->attempt[node]);
      off = g->jitter * g->h * (2.0 * u - 1.0);
    }
    p[d] = base[d] + off;
  }
}

static int grid_init(grid_t* g, int dim, int N, double jitter, uint64_t seed) {
  g->dim = dim; g->N = N; g->jitter = jitter; g->seed = seed;
  g->nn = (int64_t)N * N * (dim == 3 ? N : 1);
  g->h = 1.0 / (double)(N - 1);
  g->attempt = (int32_t*)calloc((size_t)g->nn, sizeof(int32_t));
  g->xyz = (double*)malloc((size_t)g->nn * 3 * sizeof(double));
  if (!g->attempt || !g->xyz) return -1;
  for (int64_t v = 0; v < g->nn; ++v) grid_node_coord(g, v, g->xyz + 3 * v);
  return 0;
}

static void grid_free(grid_t* g) { free(g->attempt); free(g->xyz); }

static int64_t node_id(const grid_t* g, int i, int j, int k) {
  return (int64_t)i + (int64_t)g->N * ((int64_t)j + (int64_t)g->N * (int64_t)k);
}

/* ---- element geometry ---- */

/* 2D triangles of cell (i,j): T0 = (SW,SE,NE), T1 = (SW,NE,NW). Local corner offsets. */
static const int TRI_OFF[2][3][2] = { { {0, 0}, {1, 0}, {1, 1} }, { {0, 0}, {1, 1}, {0, 1} } };

/* 3D Freudenthal split: tet t uses axis order PERM3[t]; vertices v0=0, v1=e_a, v2=e_a+e_b, v3=(1,1,1). */
static const int PERM3[6][3] = { {0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0} };

static void tet_vertices(int t, int off[4][3]) {
  memset(off, 0, sizeof(int) * 12);
  off[1][PERM3[t][0]] = 1;
  off[2][PERM3[t][0]] = 1; off[2][PERM3[t][1]] = 1;
  off[3][0] = off[3][1] = off[3][2] = 1;
}

static double det3(const double m[3][3]) {
  return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
       - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
       + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

/* inverse of a 3x3 matrix by cofactors; returns the determinant */
static double inv3(const double m[3][3], double r[3][3]) {
  double d = det3(m);
  double id = 1.0 / d;
  r[0][0] = (m[1][1] * m[2][2] - m[1][2] * m[2][1]) * id;
  r[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) * id;
  r[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) * id;
  r[1][0] = (m[1][2] * m[2][0] - m[1][0] * m[2][2]) * id;
  r[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) * id;
  r[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) * id;
  r[2][0] = (m[1][0] * m[2][1] - m[1][1] * m[2][0]) * id;
  r[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) * id;
  r[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) * id;
  return d;
}

/* Hex (Q1) reference derivatives at a Gauss point: dN[a][r], a = local node (ai + 2aj + 4ak). */
static void hex_dshape(const double xi[3], double dN[8][3]) {
  for (int a = 0; a < 8; ++a) {
    double s[3] = { (a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0 };
    double f[3] = { 1.0 + s[0] * xi[0], 1.0 + s[1] * xi[1], 1.0 + s[2] * xi[2] };
    dN[a][0] = 0.125 * s[0] * f[1] * f[2];
    dN[a][1] = 0.125 * s[1] * f[0] * f[2];
    dN[a][2] = 0.125 * s[2] * f[0] * f[1];
  }
}

static void hex_corner_nodes(const grid_t* g, int i, int j, int k, int64_t v[8]) {
  for (int a = 0; a < 8; ++a) v[a] = node_id(g, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
}

/* physical gradients of the 8 shape functions at one Gauss point; returns det J */
static double hex_grad(const grid_t* g, const int64_t v[8], const double xi[3], double G[8][3]) {
  double dN[8][3], J[3][3] = { {0} }, Ji[3][3];
  hex_dshape(xi, dN);
  for (int a = 0; a < 8; ++a)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) J[r][c] += g->xyz[3 * v[a] + r] * dN[a][c];
  double d = inv3(J, Ji);
  /* grad_x N = J^{-T} grad_xi N */
  for (int a = 0; a < 8; ++a)
    for (int r = 0; r < 3; ++r) G[a][r] = Ji[0][r] * dN[a][0] + Ji[1][r] * dN[a][1] + Ji[2][r] * dN[a][2];
  return d;
}

static double gauss_pt(int q, int axis) {
  static double gp = 0.0;
  if (gp == 0.0) gp = 1.0 / sqrt(3.0);
  return ((q >> axis) & 1) ? gp : -gp;
}

/* ---- validity: each element's measure must be at least 10% of its nominal value ---- */

static int tri_ok(const grid_t* g, int i, int j, int t) {
  double p[3][2];
  for (int a = 0; a < 3; ++a) {
    int64_t v = node_id(g, i + TRI_OFF[t][a][0], j + TRI_OFF[t][a][1], 0);
    p[a][0] = g->xyz[3 * v]; p[a][1] = g->xyz[3 * v + 1];
  }
  double twice_area = (p[1][0] - p[0][0]) * (p[2][1] - p[0][1]) - (p[2][0] - p[0][0]) * (p[1][1] - p[0][1]);
  return twice_area >= 0.1 * g->h * g->h;
}

static int tet_sign(int t) { return (t == 0 || t == 3 || t == 4) ? 1 : -1; }

static int tet_ok(const grid_t* g, int i, int j, int k, int t) {
  int off[4][3];
  tet_vertices(t, off);
  double p[4][3];
  for (int a = 0; a < 4; ++a) {
    int64_t v = node_id(g, i + off[a][0], j + off[a][1], k + off[a][2]);
    for (int d = 0; d < 3; ++d) p[a][d] = g->xyz[3 * v + d];
  }
  double E[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) E[r][c] = p[c + 1][r] - p[0][r];
  double d = det3(E) * (double)tet_sign(t);
  return d >= 0.1 * g->h * g->h * g->h;
}

static int hex_ok(const grid_t* g, int i, int j, int k) {
  int64_t v[8];
  hex_corner_nodes(g, i, j, k, v);
  double G[8][3];
  for (int q = 0; q < 8; ++q) {
    double xi[3] = { gauss_pt(q, 0), gauss_pt(q, 1), gauss_pt(q, 2) };
    double d = hex_grad(g, v, xi, G);
    if (!(d >= 0.1 * 0.125 * g->h * g->h * g->h)) return 0;
  }
  return 1;
}

/* Re-draw the jitter of every node of an invalid element until all are valid.
 * After 32 redraws a node falls back to its unjittered position, so the loop ends. */
static void grid_make_valid(grid_t* g, int kind /*0 tri, 1 tet, 2 hex*/) {
  int N = g->N, nz = (g->dim == 3) ? N - 1 : 1;
  char* mark = (char*)malloc((size_t)g->nn);
  for (int round = 0; round < 64; ++round) {
    memset(mark, 0, (size_t)g->nn);
    int64_t bad = 0;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < N - 1; ++j)
        for (int i = 0; i < N - 1; ++i) {
          int nel = kind == 0 ? 2 : kind == 1 ? 6 : 1;
          for (int t = 0; t < nel; ++t) {
            int ok = kind == 0 ? tri_ok(g, i, j, t) : kind == 1 ? tet_ok(g, i, j, k, t) : hex_ok(g, i, j, k);
            if (ok) continue;
            ++bad;
            int kk = (g->dim == 3) ? 1 : 0;
            for (int c = 0; c < (kk ? 8 : 4); ++c)
              mark[node_id(g, i + (c & 1), j + ((c >> 1) & 1), kk ? k + ((c >> 2) & 1) : 0)] = 1;
          }
        }
    if (bad == 0) break;
    for (int64_t v = 0; v < g->nn; ++v) {
      if (!mark[v]) continue;
      if (g->attempt[v] >= 0 && g->attempt[v] < 32) g->attempt[v] += 1;
      else g->attempt[v] = -1;
      grid_node_coord(g, v, g->xyz + 3 * v);
    }
  }
  free(mark);
}

/* ------------------------------------------------------------ stencil assembly */

/* Node-level stencil store: for node v and neighbour offset slot s (27 slots,
 * s = (dx+1) + 3(dy+1) + 9(dz+1)), an ncomp x ncomp block. */
typedef struct {
  const grid_t* g;
  int ncomp;
  double* blk;           /* nn * 27 * ncomp * ncomp */
  unsigned mask;         /* structural offsets present (bit s) */
} stencil_t;

static int slot_of(int dx, int dy, int dz) { return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1); }

static double* st_block(stencil_t* st, int64_t v, int s) {
  return st->blk + ((size_t)v * 27 + (size_t)s) * (size_t)(st->ncomp * st->ncomp);
}

static void node_ijk(const grid_t* g, int64_t v, int* i, int* j, int* k) {
  *i = (int)(v % g->N); *j = (int)((v / g->N) % g->N); *k = (int)(v / ((int64_t)g->N * g->N));
}

/* number of structural neighbours (including itself) of node v */
static int node_degree(const stencil_t* st, int64_t v) {
  int i, j, k, deg = 0;
  node_ijk(st->g, v, &i, &j, &k);
  for (int s = 0; s < 27; ++s) {
    if (!((st->mask >> s) & 1u)) continue;
    int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
    int a = i + dx, b = j + dy, c = k + dz;
    int N = st->g->N;
    if (a < 0 || a >= N || b < 0 || b >= N) continue;
    if (st->g->dim == 3 ? (c < 0 || c >= N) : (c != 0)) continue;
    ++deg;
  }
  return deg;
}

/* Build CSR of the relabelled matrix: new node label = perm[old], dof = node*ncomp + comp.
 * `fixed` (optional, per old node) marks Dirichlet nodes: their rows and columns are
 * zeroed (entries kept as explicit zeros) and the diagonal set to 1. */
static void stencil_to_csr(stencil_t* st, const int32_t* perm, const char* fixed,
                           int64_t* row_ptr, int32_t* col, double* val) {
  const grid_t* g = st->g;
  int nc = st->ncomp;
  int64_t nn = g->nn;
  int32_t* inv = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
  for (int64_t v = 0; v < nn; ++v) inv[perm[v]] = (int32_t)v;
  /* row pointers in the new order */
  row_ptr[0] = 0;
  for (int64_t q = 0; q < nn; ++q) {
    int deg = node_degree(st, inv[q]);
    for (int c = 0; c < nc; ++c) row_ptr[q * nc + c + 1] = row_ptr[q * nc + c] + (int64_t)deg * nc;
  }
  for (int64_t q = 0; q < nn; ++q) {
    int64_t v = inv[q];
    int i, j, k;
    node_ijk(g, v, &i, &j, &k);
    int32_t nb_lab[27]; int nb_slot[27]; int64_t nb_node[27]; int cnt = 0;
    for (int s = 0; s < 27; ++s) {
      if (!((st->mask >> s) & 1u)) continue;
      int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
      int a = i + dx, b = j + dy, c = k + dz;
      if (a < 0 || a >= g->N || b < 0 || b >= g->N) continue;
      if (g->dim == 3 ? (c < 0 || c >= g->N) : (c != 0)) continue;
      int64_t w = node_id(g, a, b, g->dim == 3 ? c : 0);
      /* insertion by new label (ascending columns) */
      int p = cnt++;
      while (p > 0 && nb_lab[p - 1] > perm[w]) { nb_lab[p] = nb_lab[p - 1]; nb_slot[p] = nb_slot[p - 1]; nb_node[p] = nb_node[p - 1]; --p; }
      nb_lab[p] = perm[w]; nb_slot[p] = s; nb_node[p] = w;
    }
    for (int c1 = 0; c1 < nc; ++c1) {
      int64_t pos = row_ptr[q * nc + c1];
      for (int e = 0; e < cnt; ++e) {
        const double* B = st_block(st, v, nb_slot[e]);
        for (int c2 = 0; c2 < nc; ++c2) {
          double a = B[c1 * nc + c2];
          if (fixed && (fixed[v] || fixed[nb_node[e]])) a = (nb_node[e] == v && c1 == c2) ? 1.0 : 0.0;
          col[pos] = nb_lab[e] * nc + c2;
          val[pos] = a;
          ++pos;
        }
      }
    }
  }
  free(inv);
}

/* ------------------------------------------------------------ public generators */

int64_t gen_fem2d_p1_nnz(int N) {
  int64_t n = (int64_t)N * N, m = N - 1;
  return n + 2 * (2 * (int64_t)N * m + m * m);
}

int64_t gen_hex_nnz(int N, int ncomp) {
  int64_t s = 3 * (int64_t)N - 2;
  return (int64_t)ncomp * ncomp * s * s * s;
}

int64_t gen_tet_lap3d_nnz(int N) {
  int64_t n = (int64_t)N * N * N, m = N - 1;
  return n + 2 * (3 * (int64_t)N * N * m + 3 * (int64_t)N * m * m + m * m * m);
}

/* Jittered node coordinates indexed by the NEW node label (for null-space checks). */
int gen_coords(int dim, int N, double jitter, uint64_t seed_mesh, uint64_t seed_perm, int kind, double* xyz_new) {
  grid_t g;
  if (grid_init(&g, dim, N, jitter, seed_mesh)) return -1;
  grid_make_valid(&g, kind);
  int32_t* perm = (int32_t*)malloc((size_t)g.nn * sizeof(int32_t));
  gen_permutation(g.nn, seed_perm, perm);
  for (int64_t v = 0; v < g.nn; ++v)
    for (int d = 0; d < 3; ++d) xyz_new[3 * (int64_t)perm[v] + d] = g.xyz[3 * v + d];
  free(perm);
  grid_free(&g);
  return 0;
}

/* 2D P1 Laplacian, N x N nodes on [0,1]^2, jitter in units of h. */
int gen_fem2d_p1(int N, double jitter, uint64_t seed_mesh, uint64_t seed_perm,
                 int64_t* row_ptr, int32_t* col, double* val) {
  grid_t g;
  if (N < 2 || grid_init(&g, 2, N, jitter, seed_mesh)) return -1;
  grid_make_valid(&g, 0);
  stencil_t st = { &g, 1, NULL, 0u };
  st.mask = (1u << slot_of(0, 0, 0)) | (1u << slot_of(1, 0, 0)) | (1u << slot_of(-1, 0, 0)) |
            (1u << slot_of(0, 1, 0)) | (1u << slot_of(0, -1, 0)) | (1u << slot_of(1, 1, 0)) |
            (1u << slot_of(-1, -1, 0));
  st.blk = (double*)calloc((size_t)g.nn * 27, sizeof(double));
  if (!st.blk) { grid_free(&g); return -1; }
  for (int j = 0; j < N - 1; ++j)
    for (int i = 0; i < N - 1; ++i)
      for (int t = 0; t < 2; ++t) {
        int64_t v[3]; double x[3], y[3];
        for (int a = 0; a < 3; ++a) {
          v[a] = node_id(&g, i + TRI_OFF[t][a][0], j + TRI_OFF[t][a][1], 0);
          x[a] = g.xyz[3 * v[a]]; y[a] = g.xyz[3 * v[a] + 1];
        }
        double twice_area = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
        double bb[3], cc[3];
        for (int a = 0; a < 3; ++a) {
          bb[a] = y[(a + 1) % 3] - y[(a + 2) % 3];
          cc[a] = x[(a + 2) % 3] - x[(a + 1) % 3];
        }
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            int dx = TRI_OFF[t][b][0] - TRI_OFF[t][a][0], dy = TRI_OFF[t][b][1] - TRI_OFF[t][a][1];
            double kab = (bb[a] * bb[b] + cc[a] * cc[b]) / (2.0 * twice_area);
            st_block(&st, v[a], slot_of(dx, dy, 0))[0] += kab;
          }
      }
  int32_t* perm = (int32_t*)malloc((size_t)g.nn * sizeof(int32_t));
  gen_permutation(g.nn, seed_perm, perm);
  stencil_to_csr(&st, perm, NULL, row_ptr, col, val);
  free(perm); free(st.blk); grid_free(&g);
  return 0;
}

/* 3D Q1 hexahedra: ncomp = 3 isotropic elasticity (E, nu); ncomp = 1 scalar Laplacian.
 * clamp_minz: Dirichlet on all nodes of the k = 0 face. */
int gen_hex3d(int N, int ncomp, double jitter, double E, double nu, uint64_t seed_mesh, uint64_t seed_perm,
              int clamp_minz, int64_t* row_ptr, int32_t* col, double* val) {
  grid_t g;
  if (N < 2 || (ncomp != 1 && ncomp != 3) || grid_init(&g, 3, N, jitter, seed_mesh)) return -1;
  grid_make_valid(&g, 2);
  stencil_t st = { &g, ncomp, NULL, (1u << 27) - 1u };
  st.blk = (double*)calloc((size_t)g.nn * 27 * ncomp * ncomp, sizeof(double));
  if (!st.blk) { grid_free(&g); return -1; }
  double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double mu = E / (2.0 * (1.0 + nu));
  double Ke[24][24];
  for (int k = 0; k < N - 1; ++k)
    for (int j = 0; j < N - 1; ++j)
      for (int i = 0; i < N - 1; ++i) {
        int64_t v[8];
        hex_corner_nodes(&g, i, j, k, v);
        memset(Ke, 0, sizeof(Ke));
        for (int q = 0; q < 8; ++q) {
          double xi[3] = { gauss_pt(q, 0), gauss_pt(q, 1), gauss_pt(q, 2) };
          double G[8][3];
          double w = hex_grad(&g, v, xi, G); /* unit Gauss weights */
          for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b) {
              double gg = G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2];
              if (ncomp == 1) { Ke[a][b] += w * gg; continue; }
              /* K[(a,r),(b,c)] = lam d_r N_a d_c N_b + mu d_c N_a d_r N_b + mu delta_rc grad N_a . grad N_b */
              for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                  double kk = lam * G[a][r] * G[b][c] + mu * G[a][c] * G[b][r];
                  if (r == c) kk += mu * gg;
                  Ke[3 * a + r][3 * b + c] += w * kk;
                }
            }
        }
        /* mirror the upper triangle so that the element (and assembled) matrix is exactly symmetric */
        for (int r = 0; r < 8 * ncomp; ++r)
          for (int c = 0; c < r; ++c) Ke[r][c] = Ke[c][r];
        for (int a = 0; a < 8; ++a)
          for (int b = 0; b < 8; ++b) {
            int dx = (b & 1) - (a & 1), dy = ((b >> 1) & 1) - ((a >> 1) & 1), dz = ((b >> 2) & 1) - ((a >> 2) & 1);
            double* B = st_block(&st, v[a], slot_of(dx, dy, dz));
            for (int r = 0; r < ncomp; ++r)
              for (int c = 0; c < ncomp; ++c) B[r * ncomp + c] += Ke[ncomp * a + r][ncomp * b + c];
          }
      }
  char* fixed = NULL;
  if (clamp_minz) {
    fixed = (char*)calloc((size_t)g.nn, 1);
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) fixed[node_id(&g, i, j, 0)] = 1;
  }
  int32_t* perm = (int32_t*)malloc((size_t)g.nn * sizeof(int32_t));
  gen_permutation(g.nn, seed_perm, perm);
  stencil_to_csr(&st, perm, fixed, row_ptr, col, val);
  free(perm); free(fixed); free(st.blk); grid_free(&g);
  return 0;
}

/* 3D P1 Laplacian on the Freudenthal split; dirichlet: all boundary nodes fixed. */
int gen_tet_lap3d(int N, double jitter, uint64_t seed_mesh, uint64_t seed_perm, int dirichlet,
                  int64_t* row_ptr, int32_t* col, double* val) {
  grid_t g;
  if (N < 2 || grid_init(&g, 3, N, jitter, seed_mesh)) return -1;
  grid_make_valid(&g, 1);
  stencil_t st = { &g, 1, NULL, 0u };
  static const int OFF15[15][3] = { {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
                                    {1, 1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1},
                                    {1, 1, 1}, {-1, -1, -1} };
  for (int s = 0; s < 15; ++s) st.mask |= 1u << slot_of(OFF15[s][0], OFF15[s][1], OFF15[s][2]);
  st.blk = (double*)calloc((size_t)g.nn * 27, sizeof(double));
  if (!st.blk) { grid_free(&g); return -1; }
  for (int k = 0; k < N - 1; ++k)
    for (int j = 0; j < N - 1; ++j)
      for (int i = 0; i < N - 1; ++i)
        for (int t = 0; t < 6; ++t) {
          int off[4][3];
          tet_vertices(t, off);
          int64_t v[4]; double p[4][3];
          for (int a = 0; a < 4; ++a) {
            v[a] = node_id(&g, i + off[a][0], j + off[a][1], k + off[a][2]);
            for (int d = 0; d < 3; ++d) p[a][d] = g.xyz[3 * v[a] + d];
          }
          double Em[3][3], Ei[3][3];
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Em[r][c] = p[c + 1][r] - p[0][r];
          double d = inv3(Em, Ei);
          double vol = fabs(d) / 6.0;
          double G[4][3];
          for (int c = 0; c < 3; ++c) {
            G[1][c] = Ei[0][c]; G[2][c] = Ei[1][c]; G[3][c] = Ei[2][c];
            G[0][c] = -(Ei[0][c] + Ei[1][c] + Ei[2][c]);
          }
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
              double kab = vol * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
              int s = slot_of(off[b][0] - off[a][0], off[b][1] - off[a][1], off[b][2] - off[a][2]);
              st_block(&st, v[a], s)[0] += kab;
            }
        }
  char* fixed = NULL;
  if (dirichlet) {
    fixed = (char*)calloc((size_t)g.nn, 1);
    for (int64_t v = 0; v < g.nn; ++v) {
      int i, j, k;
      node_ijk(&g, v, &i, &j, &k);
      if (i == 0 || j == 0 || k == 0 || i == N - 1 || j == N - 1 || k == N - 1) fixed[v] = 1;
    }
  }
  int32_t* perm = (int32_t*)malloc((size_t)g.nn * sizeof(int32_t));
  gen_permutation(g.nn, seed_perm, perm);
  stencil_to_csr(&st, perm, fixed, row_ptr, col, val);
  free(perm); free(fixed); free(st.blk); grid_free(&g);
  return 0;
}
