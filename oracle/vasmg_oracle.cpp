// V-ASMG-PCG oracle (arXiv 2505.09064) -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow FP64 CPU implementation of what the solve path computes,
// single-threaded as built by default.  Only the test-suite, the smoke check
// and the CPU-baseline leg of the benchmark may load it; the library never
// does.  It shares no code with
// the CUDA path: every step is written here from the paper's description, in
// the paper's order, with no blocking, fusion or reordering.  Build flags keep
// IEEE semantics (-O2 -ffp-contract=off) so the geometric steps round exactly
// as written.  A second build of this same file with -fopenmp (the parallel
// CPU line of the benchmark) runs three kinds of independent row loops on
// all host cores: the rows of one colour in a sweep, the rows of y = A x, and
// the fine rows of the prolongation.  No reduction is split, and every row
// keeps its own order of additions, so both builds give the same bits.
//
// Steps (paper section / equation / algorithm):
//   assembly            Sec. 2, the 2x2 block form of A and F (P1 elements),
//                       written for d = 2, 3 as K_ij[a][b] = |K|(lam g_ia g_jb
//                       + mu g_ib g_ja + mu delta_ab g_i.g_j)
//   Dirichlet rows      not discussed in the paper: identity rows/columns
//   bounding square     Sec. 3.1.1 Step 1
//   region tree         Sec. 3.1.1 Step 2 (sequential insertion, split at > T)
//   empty-leaf removal  Sec. 3.1.1 Step 3, coarse vertices = leaf corners
//   fine<->coarse map   Sec. 3.1.1 Step 4
//   coarser grids       Sec. 3.1.2 (merge deepest cells into their parents)
//   weights             Sec. 3.2, eq. (wkl), (wkl_xy) read as bilinear weights
//   Galerkin            eq. (R), eq. (Ac)
//   smoother            Sec. 2.1 / Alg. 1 as multicolour point-block GS
//   coarsest solve      Sec. 3, Step 2.3 (Cholesky)
//   V-cycle             Alg. 3 applied recursively, zero initial guess;
//                       W-cycle (Fig. 2) and the additive form
//                       B_h = S_h + Pi B_0 Pi^T (Sec. 4) as comparators
//   PCG                 Alg. 2, stop rule of Sec. 5 item (3)
//
// Parity status: every function here is pinned by the CPU test-suite
// (patch test, rigid-body null space, exact symmetry, insertion-order
// invariance of the tree, bilinear reproduction, Theorem 3.2, dense direct
// solves, V-cycle symmetry).  Iteration counts of the paper's own meshes are
// "parity unpinned": those meshes are not available.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef int64_t i64;
typedef uint64_t u64;

// ---------------------------------------------------------------- utilities

// splitmix64 output function (Steele, Lea, Flood 2014; Vigna's constants).
u64 splitmix64(u64 x) {
  u64 z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Interleave: bit b of axis a goes to bit b*d + a.
u64 interleave(const u64* c, int d, int bits) {
  u64 k = 0;
  for (int b = 0; b < bits; ++b)
    for (int a = 0; a < d; ++a) k |= ((c[a] >> b) & 1ull) << (b * d + a);
  return k;
}
void deinterleave(u64 k, int d, int bits, u64* c) {
  for (int a = 0; a < d; ++a) c[a] = 0;
  for (int b = 0; b < bits; ++b)
    for (int a = 0; a < d; ++a) c[a] |= ((k >> (b * d + a)) & 1ull) << b;
}

// Block-sparse matrix with d x d blocks, columns sorted, diagonal present.
struct BSR {
  int d = 0;
  i64 n = 0;
  std::vector<i64> rp;
  std::vector<int32_t> ci;
  std::vector<double> v;  // nnz * d * d, row-major blocks
  i64 nnz() const { return (i64)ci.size(); }
  i64 find(i64 i, int32_t j) const {
    auto b = ci.begin() + rp[i], e = ci.begin() + rp[i + 1];
    auto it = std::lower_bound(b, e, j);
    if (it == e || *it != j) return -1;
    return (i64)(it - ci.begin());
  }
  double* blk(i64 k) { return &v[(size_t)k * d * d]; }
  const double* blk(i64 k) const { return &v[(size_t)k * d * d]; }
};

// Build a BSR pattern from a list of (row, col) pairs (duplicates allowed).
BSR pattern_from_pairs(int d, i64 n, std::vector<std::pair<int32_t, int32_t>>& pairs) {
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  BSR A;
  A.d = d;
  A.n = n;
  A.rp.assign(n + 1, 0);
  for (auto& p : pairs) A.rp[p.first + 1]++;
  for (i64 i = 0; i < n; ++i) A.rp[i + 1] += A.rp[i];
  A.ci.resize(pairs.size());
  for (size_t k = 0; k < pairs.size(); ++k) A.ci[k] = pairs[k].second;
  A.v.assign(pairs.size() * d * d, 0.0);
  return A;
}

// y = A x (full vector, dof = vertex*d + component).
// The rows are independent; the parallel build of this file splits them over
// threads (each row's sum keeps its order, so the result is the same).
void bsr_apply(const BSR& A, const double* x, double* y) {
  const int d = A.d;
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < A.n; ++i) {
    for (int a = 0; a < d; ++a) y[i * d + a] = 0.0;
    for (i64 k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const double* B = A.blk(k);
      i64 j = A.ci[k];
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) y[i * d + a] += B[a * d + b] * x[j * d + b];
    }
  }
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// Inverse of a small dense d x d matrix by Gauss-Jordan with partial pivoting.
bool small_inverse(int d, const double* A, double* Ainv) {
  double M[3][6];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < 2 * d; ++j) M[i][j] = j < d ? A[i * d + j] : (j - d == i ? 1.0 : 0.0);
  for (int c = 0; c < d; ++c) {
    int p = c;
    for (int r = c + 1; r < d; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[p][c])) p = r;
    if (M[p][c] == 0.0) return false;
    for (int j = 0; j < 2 * d; ++j) std::swap(M[c][j], M[p][j]);
    double piv = M[c][c];
    for (int j = 0; j < 2 * d; ++j) M[c][j] /= piv;
    for (int r = 0; r < d; ++r) {
      if (r == c) continue;
      double f = M[r][c];
      for (int j = 0; j < 2 * d; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Ainv[i * d + j] = M[i][j + d];
  return true;
}

// ---------------------------------------------------------------- hierarchy data

struct Cell {
  int depth;
  u64 c[3];  // cell index per axis at resolution 2^depth
};
struct CellKey {
  int depth;
  u64 key;  // interleaved cell index
  bool operator<(const CellKey& o) const { return depth != o.depth ? depth < o.depth : key < o.key; }
  bool operator==(const CellKey& o) const { return depth == o.depth && key == o.key; }
};

// Scalar interpolation weights P_s (rows: vertices of the finer level, columns:
// vertices of the coarser level); the dof-level operator is P_s (x) I_d with
// rows of dead dofs masked.
struct Prolong {
  std::vector<i64> rp;
  std::vector<int32_t> ci;
  std::vector<double> w;
};

struct Level {
  i64 nv = 0;
  std::vector<u64> lat;           // level >= 1: Morton key of the lattice corner (K+1 bits/axis)
  std::vector<CellKey> cells;     // level >= 1: the cells whose corners these vertices are
  BSR A;                          // operator, identity rows/cols at dead dofs
  std::vector<uint8_t> dead;      // per dof
  std::vector<int32_t> colour;    // per vertex
  int ncol = 0;
  std::vector<std::vector<int32_t>> by_colour;
  std::vector<double> dinv;       // per vertex, d*d
  Prolong P;                      // to the next coarser level (absent on the coarsest)
};

struct Oracle {
  int dim = 2, K = 31, T = 4;
  int smoother = 0;               // 0: multicolour point-block GS, 1: scalar lexicographic GS
  int gamma = 1;                  // coarse corrections per level: 1 = V-cycle, 2 = W-cycle (Fig. 2)
  int additive = 0;               // 1: B_h = S_h + Pi B_0 Pi^T at the fine level (Sec. 4)
  i64 nv = 0, ne = 0, coarse_max_dofs = 0;
  std::vector<double> X;
  std::vector<int32_t> E;
  std::vector<double> lam, mu, vol;
  std::vector<uint8_t> is_dir;    // per dof
  std::vector<double> udir;       // per dof (0 where free)
  std::vector<double> lift;       // A_full * udir
  double m = 0, Mx = 0;           // bounding square [m, Mx]^d
  std::vector<u64> q;             // quantised coordinates, nv*dim
  std::vector<u64> mkey;          // Morton keys of the quantised coordinates
  std::vector<CellKey> leaf_of;   // insertion leaf of every fine vertex
  std::vector<Level> L;
  // coarsest factor
  i64 nc = 0;
  std::vector<double> chol;
  std::vector<uint8_t> chol_drop;
  int status = 0;
};

int dim_K(int d) { return d == 2 ? 31 : 20; }

// ---------------------------------------------------------------- assembly (Sec. 2)

// Barycentric gradients g[k][a] of the P1 basis on simplex e and its measure.
bool p1_gradients(const Oracle& o, i64 e, double g[4][3], double* measure) {
  const int d = o.dim;
  const int32_t* v = &o.E[e * (d + 1)];
  double J[3][3];  // J[a][k] = x_{k+1,a} - x_{0,a}
  for (int k = 0; k < d; ++k)
    for (int a = 0; a < d; ++a) J[a][k] = o.X[(i64)v[k + 1] * d + a] - o.X[(i64)v[0] * d + a];
  double det, inv[3][3];
  if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (!(det != 0.0) || !std::isfinite(det)) return false;
    inv[0][0] = J[1][1] / det;
    inv[0][1] = -J[0][1] / det;
    inv[1][0] = -J[1][0] / det;
    inv[1][1] = J[0][0] / det;
    *measure = std::fabs(det) / 2.0;
  } else {
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det != 0.0) || !std::isfinite(det)) return false;
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    *measure = std::fabs(det) / 6.0;
  }
  // basis k (k >= 1) has gradient = row k-1 of J^{-1}; basis 0 = minus their sum
  for (int k = 1; k <= d; ++k)
    for (int a = 0; a < d; ++a) g[k][a] = inv[k - 1][a];
  for (int a = 0; a < d; ++a) {
    double s = 0.0;
    for (int k = 1; k <= d; ++k) s += g[k][a];
    g[0][a] = -s;
  }
  return true;
}

int assemble(Oracle& o, BSR& A) {
  const int d = o.dim, nl = d + 1;
  std::vector<std::pair<int32_t, int32_t>> pairs;
  pairs.reserve((size_t)o.ne * nl * nl + o.nv);
  for (i64 i = 0; i < o.nv; ++i) pairs.push_back({(int32_t)i, (int32_t)i});
  for (i64 e = 0; e < o.ne; ++e)
    for (int r = 0; r < nl; ++r)
      for (int c = 0; c < nl; ++c) pairs.push_back({o.E[e * nl + r], o.E[e * nl + c]});
  A = pattern_from_pairs(d, o.nv, pairs);
  o.vol.assign(o.ne, 0.0);
  for (i64 e = 0; e < o.ne; ++e) {
    double g[4][3], meas;
    if (!p1_gradients(o, e, g, &meas)) return -2;
    o.vol[e] = meas;
    const double la = o.lam[e], m = o.mu[e];
    for (int r = 0; r < nl; ++r)
      for (int c = 0; c < nl; ++c) {
        i64 k = A.find(o.E[e * nl + r], o.E[e * nl + c]);
        double* B = A.blk(k);
        double gg = 0.0;
        for (int x = 0; x < d; ++x) gg += g[r][x] * g[c][x];
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b)
            // products of the two gradients are formed first so that the mirrored
            // entry (c, r, b, a) rounds identically: A is exactly symmetric
            B[a * d + b] += meas * (la * (g[r][a] * g[c][b]) + m * (g[r][b] * g[c][a]) + (a == b ? m * gg : 0.0));
      }
  }
  return 0;
}

// Load vector for a constant body force: F_i += f |K| / (d+1) (Sec. 2, F_1, F_2).
void assemble_load(const Oracle& o, const double* f, double* F) {
  const int d = o.dim, nl = d + 1;
  for (i64 i = 0; i < o.nv * d; ++i) F[i] = 0.0;
  for (i64 e = 0; e < o.ne; ++e)
    for (int r = 0; r < nl; ++r)
      for (int a = 0; a < d; ++a) F[(i64)o.E[e * nl + r] * d + a] += f[a] * o.vol[e] / (double)nl;
}

// Dirichlet dofs become identity rows and columns; lift = A u_d is kept so the
// solve can form the reduced right-hand side F_f - A_fd u_d.
void apply_dirichlet(Oracle& o, BSR& A) {
  const int d = o.dim;
  o.lift.assign(o.nv * d, 0.0);
  bsr_apply(A, o.udir.data(), o.lift.data());
  for (i64 i = 0; i < o.nv; ++i)
    for (i64 k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      i64 j = A.ci[k];
      double* B = A.blk(k);
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b)
          if (o.is_dir[i * d + a] || o.is_dir[j * d + b]) B[a * d + b] = (i == j && a == b) ? 1.0 : 0.0;
    }
}

// ---------------------------------------------------------------- region tree (Sec. 3.1.1)

// Step 1: the square [m, M]^d with m the smallest and M the largest coordinate
// over all axes; quantisation to the 2^K lattice with half-open cells.
void bounding_square_and_keys(Oracle& o) {
  const int d = o.dim;
  o.m = o.X[0];
  o.Mx = o.X[0];
  for (i64 i = 0; i < o.nv * d; ++i) {
    o.m = std::min(o.m, o.X[i]);
    o.Mx = std::max(o.Mx, o.X[i]);
  }
  const double span = o.Mx - o.m;
  const u64 top = (1ull << o.K) - 1;
  o.q.assign(o.nv * d, 0);
  o.mkey.assign(o.nv, 0);
  for (i64 v = 0; v < o.nv; ++v) {
    for (int a = 0; a < d; ++a) {
      double t = span > 0.0 ? (o.X[v * d + a] - o.m) / span : 0.0;
      double s = std::floor(std::ldexp(t, o.K));
      u64 qa = s <= 0.0 ? 0 : (s >= (double)top ? top : (u64)s);
      o.q[v * d + a] = qa;
    }
    o.mkey[v] = interleave(&o.q[v * d], d, o.K);
  }
}

// Normalised coordinate t_a in [0,1] of a fine vertex (same arithmetic as the
// quantisation above).
double norm_coord(const Oracle& o, i64 v, int a) {
  const double span = o.Mx - o.m;
  return span > 0.0 ? (o.X[v * o.dim + a] - o.m) / span : 0.0;
}

// Step 2: literal sequential insertion into a point-region tree.  A node whose
// vertex set exceeds T is split into 2^d children and its members are inserted
// again (recursively, so a child that receives more than T splits as well).
struct TreeNode {
  int depth;
  u64 c[3];
  bool leaf;
  std::vector<int32_t> verts;
  int32_t child[8];
};

struct Tree {
  const Oracle* o;
  std::vector<TreeNode> nodes;
  int child_index(int node, int32_t v) const {
    int idx = 0, sh = o->K - nodes[node].depth - 1;
    for (int a = 0; a < o->dim; ++a) idx |= (int)((o->q[(i64)v * o->dim + a] >> sh) & 1ull) << a;
    return idx;
  }
  void split(int node) {
    nodes[node].leaf = false;
    const int nch = 1 << o->dim;
    for (int ch = 0; ch < nch; ++ch) {
      TreeNode t;
      t.depth = nodes[node].depth + 1;
      for (int a = 0; a < 3; ++a) t.c[a] = a < o->dim ? 2 * nodes[node].c[a] + ((ch >> a) & 1) : 0;
      t.leaf = true;
      for (int k = 0; k < 8; ++k) t.child[k] = -1;
      nodes.push_back(t);
      nodes[node].child[ch] = (int32_t)nodes.size() - 1;
    }
    std::vector<int32_t> members;
    members.swap(nodes[node].verts);
    for (int32_t v : members) insert(node, v);
  }
  void insert(int node, int32_t v) {
    while (!nodes[node].leaf) node = nodes[node].child[child_index(node, v)];
    nodes[node].verts.push_back(v);
    if ((int)nodes[node].verts.size() > o->T && nodes[node].depth < o->K) split(node);
  }
};

CellKey cell_key(const Cell& c, int d) { return CellKey{c.depth, interleave(c.c, d, std::max(c.depth, 1))}; }

void build_tree_insertion(Oracle& o, const i64* order) {
  Tree t;
  t.o = &o;
  TreeNode root;
  root.depth = 0;
  root.c[0] = root.c[1] = root.c[2] = 0;
  root.leaf = true;
  for (int k = 0; k < 8; ++k) root.child[k] = -1;
  t.nodes.push_back(root);
  for (i64 i = 0; i < o.nv; ++i) t.insert(0, (int32_t)(order ? order[i] : i));
  // Step 3: keep the non-empty leaves; each fine vertex remembers its leaf.
  o.leaf_of.assign(o.nv, CellKey{0, 0});
  for (auto& n : t.nodes) {
    if (!n.leaf || n.verts.empty()) continue;
    Cell c{n.depth, {n.c[0], n.c[1], n.c[2]}};
    for (int32_t v : n.verts) o.leaf_of[v] = cell_key(c, o.dim);
  }
}

// Independent cross-check: the same tree from the sorted keys.  A cell is split
// iff it holds more than T vertices, so a vertex's leaf is the shallowest cell
// on its path holding at most T vertices (or the depth-K cell).
void build_tree_sorted(const Oracle& o, std::vector<CellKey>& leaf) {
  std::vector<u64> sk(o.mkey);
  std::sort(sk.begin(), sk.end());
  const int d = o.dim;
  leaf.assign(o.nv, CellKey{0, 0});
  for (i64 v = 0; v < o.nv; ++v) {
    for (int depth = 0; depth <= o.K; ++depth) {
      int rest = d * (o.K - depth);
      u64 lo = rest >= 64 ? 0 : (o.mkey[v] >> rest) << rest;
      u64 cnt;
      if (rest >= 64) {
        cnt = (u64)o.nv;
      } else {
        u64 hi_excl = lo + (1ull << rest);  // may wrap to 0 for the last cell
        auto b = std::lower_bound(sk.begin(), sk.end(), lo);
        auto e = hi_excl == 0 ? sk.end() : std::lower_bound(sk.begin(), sk.end(), hi_excl);
        cnt = (u64)(e - b);
      }
      if ((i64)cnt <= o.T || depth == o.K) {
        leaf[v] = CellKey{depth, rest >= 64 ? 0 : o.mkey[v] >> rest};
        break;
      }
    }
  }
}

// ---------------------------------------------------------------- coarse grids and weights

// Lattice corner of a cell at full resolution (K+1 bits per axis).
void cell_corner(const Oracle& o, const CellKey& ck, int delta, u64* p) {
  u64 c[3];
  deinterleave(ck.key, o.dim, std::max(ck.depth, 1), c);
  for (int a = 0; a < o.dim; ++a) p[a] = (c[a] + ((delta >> a) & 1)) << (o.K - ck.depth);
}

// Vertices of a level = the deduplicated corners of its cells (Step 3 of
// Sec. 3.1.1 and Sec. 3.1.2), in ascending Morton order of the lattice corner.
void level_vertices(const Oracle& o, Level& lv) {
  std::vector<u64> keys;
  const int nch = 1 << o.dim;
  for (auto& ck : lv.cells)
    for (int dl = 0; dl < nch; ++dl) {
      u64 p[3];
      cell_corner(o, ck, dl, p);
      keys.push_back(interleave(p, o.dim, o.K + 1));
    }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  lv.lat = keys;
  lv.nv = (i64)keys.size();
}

i64 vertex_index(const Level& lv, u64 key) {
  auto it = std::lower_bound(lv.lat.begin(), lv.lat.end(), key);
  if (it == lv.lat.end() || *it != key) return -1;
  return (i64)(it - lv.lat.begin());
}

// Bilinear / trilinear weights of the 2^d corners from local coordinates
// s_a in [0,1] (eq. (wkl): w = w^x * w^y [* w^z]; the printed per-axis
// factors are read as the standard 1 - |x_k - x_l| / (R - L)).
void corner_weights(int d, const double* s, double* w) {
  for (int dl = 0; dl < (1 << d); ++dl) {
    double acc = 1.0;
    for (int a = 0; a < d; ++a) {
      double f = ((dl >> a) & 1) ? s[a] : 1.0 - s[a];
      acc = acc * f;
    }
    w[dl] = acc;
  }
}

// P_0: each fine vertex interpolates from the corners of its insertion leaf
// (Step 4 of Sec. 3.1.1 and Sec. 3.2).
void build_P0(const Oracle& o, Level& fine, const Level& coarse) {
  const int d = o.dim, nch = 1 << d;
  fine.P.rp.assign(o.nv + 1, 0);
  fine.P.ci.clear();
  fine.P.w.clear();
  for (i64 v = 0; v < o.nv; ++v) {
    const CellKey& ck = o.leaf_of[v];
    u64 c[3];
    deinterleave(ck.key, d, std::max(ck.depth, 1), c);
    double s[3];
    for (int a = 0; a < d; ++a) s[a] = std::ldexp(norm_coord(o, v, a), ck.depth) - (double)c[a];
    double w[8];
    corner_weights(d, s, w);
    std::vector<std::pair<int32_t, double>> row;
    for (int dl = 0; dl < nch; ++dl) {
      if (w[dl] == 0.0) continue;
      u64 p[3];
      cell_corner(o, ck, dl, p);
      row.push_back({(int32_t)vertex_index(coarse, interleave(p, d, o.K + 1)), w[dl]});
    }
    std::sort(row.begin(), row.end());
    for (auto& e : row) {
      fine.P.ci.push_back(e.first);
      fine.P.w.push_back(e.second);
    }
    fine.P.rp[v + 1] = (i64)fine.P.ci.size();
  }
}

// Cell of a coarser level that interpolates a lattice point p: the cell whose
// half-open box contains p; on the outer edge of the covered region, the cell
// of smallest (depth, key) among those whose closed box contains p.
bool locate_half_open(const Oracle& o, const std::set<CellKey>& cells, const u64* p, CellKey* out) {
  const u64 lim = 1ull << o.K;
  for (int a = 0; a < o.dim; ++a)
    if (p[a] >= lim) return false;
  for (int depth = 0; depth <= o.K; ++depth) {
    u64 c[3];
    for (int a = 0; a < o.dim; ++a) c[a] = p[a] >> (o.K - depth);
    CellKey ck{depth, interleave(c, o.dim, std::max(depth, 1))};
    if (cells.count(ck)) {
      *out = ck;
      return true;
    }
  }
  return false;
}

bool locate_cell(const Oracle& o, const std::set<CellKey>& cells, const u64* p, CellKey* out) {
  if (locate_half_open(o, cells, p, out)) return true;
  bool found = false;
  for (int dl = 1; dl < (1 << o.dim); ++dl) {
    u64 pp[3];
    bool ok = true;
    for (int a = 0; a < o.dim; ++a) {
      u64 da = (dl >> a) & 1;
      if (p[a] < da) ok = false;
      pp[a] = p[a] - da;
    }
    CellKey ck;
    if (!ok || !locate_half_open(o, cells, pp, &ck)) continue;
    if (!found || ck < *out) *out = ck;
    found = true;
  }
  return found;
}

void build_Pl(const Oracle& o, Level& fine, const Level& coarse) {
  const int d = o.dim, nch = 1 << d;
  std::set<CellKey> cells(coarse.cells.begin(), coarse.cells.end());
  fine.P.rp.assign(fine.nv + 1, 0);
  fine.P.ci.clear();
  fine.P.w.clear();
  for (i64 v = 0; v < fine.nv; ++v) {
    u64 p[3];
    deinterleave(fine.lat[v], d, o.K + 1, p);
    CellKey ck;
    locate_cell(o, cells, p, &ck);
    u64 c[3];
    deinterleave(ck.key, d, std::max(ck.depth, 1), c);
    const int sh = o.K - ck.depth;
    double s[3];
    for (int a = 0; a < d; ++a) s[a] = std::ldexp((double)(p[a] - (c[a] << sh)), -sh);
    double w[8];
    corner_weights(d, s, w);
    std::vector<std::pair<int32_t, double>> row;
    for (int dl = 0; dl < nch; ++dl) {
      if (w[dl] == 0.0) continue;
      u64 pc[3];
      cell_corner(o, ck, dl, pc);
      row.push_back({(int32_t)vertex_index(coarse, interleave(pc, d, o.K + 1)), w[dl]});
    }
    std::sort(row.begin(), row.end());
    for (auto& e : row) {
      fine.P.ci.push_back(e.first);
      fine.P.w.push_back(e.second);
    }
    fine.P.rp[v + 1] = (i64)fine.P.ci.size();
  }
}

// Sec. 3.1.2: replace every cell at the current maximum depth by its parent.
std::vector<CellKey> merge_deepest(const Oracle& o, const std::vector<CellKey>& cells) {
  int D = 0;
  for (auto& c : cells) D = std::max(D, c.depth);
  std::set<CellKey> out;
  for (auto& c : cells) {
    if (c.depth < D) {
      out.insert(c);
    } else {
      u64 cc[3];
      deinterleave(c.key, o.dim, std::max(c.depth, 1), cc);
      for (int a = 0; a < o.dim; ++a) cc[a] >>= 1;
      out.insert(CellKey{D - 1, interleave(cc, o.dim, std::max(D - 1, 1))});
    }
  }
  return std::vector<CellKey>(out.begin(), out.end());
}

// ---------------------------------------------------------------- Galerkin (eq. (R), (Ac))

// A_c = P^T A P with P = P_s (x) I_d and rows of dead fine dofs masked.  The
// block pattern is the structural product pattern plus the diagonal; coarse
// dofs whose masked column of P is empty are dead and get identity rows.
void galerkin(const Oracle& o, const Level& fine, Level& coarse) {
  const int d = o.dim;
  const Prolong& P = fine.P;
  const BSR& A = fine.A;
  std::vector<std::pair<int32_t, int32_t>> pairs;
  for (i64 I = 0; I < coarse.nv; ++I) pairs.push_back({(int32_t)I, (int32_t)I});
  for (i64 i = 0; i < fine.nv; ++i)
    for (i64 a = P.rp[i]; a < P.rp[i + 1]; ++a)
      for (i64 k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        i64 j = A.ci[k];
        for (i64 b = P.rp[j]; b < P.rp[j + 1]; ++b) pairs.push_back({P.ci[a], P.ci[b]});
      }
  coarse.A = pattern_from_pairs(d, coarse.nv, pairs);
  // dead coarse dofs
  coarse.dead.assign(coarse.nv * d, 1);
  for (i64 i = 0; i < fine.nv; ++i)
    for (i64 a = P.rp[i]; a < P.rp[i + 1]; ++a)
      for (int c = 0; c < d; ++c)
        if (!fine.dead[i * d + c]) coarse.dead[(i64)P.ci[a] * d + c] = 0;
  // values: sum over i, j of P_iI (M A M)_ij P_jJ
  for (i64 i = 0; i < fine.nv; ++i)
    for (i64 a = P.rp[i]; a < P.rp[i + 1]; ++a) {
      const int32_t I = P.ci[a];
      const double wI = P.w[a];
      for (i64 k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const i64 j = A.ci[k];
        const double* B = A.blk(k);
        for (i64 b = P.rp[j]; b < P.rp[j + 1]; ++b) {
          const int32_t J = P.ci[b];
          const double wJ = P.w[b];
          double* C = coarse.A.blk(coarse.A.find(I, J));
          for (int r = 0; r < d; ++r) {
            if (fine.dead[i * d + r]) continue;
            for (int s = 0; s < d; ++s) {
              if (fine.dead[j * d + s]) continue;
              C[r * d + s] += wI * B[r * d + s] * wJ;
            }
          }
        }
      }
    }
  for (i64 I = 0; I < coarse.nv; ++I)
    for (int r = 0; r < d; ++r)
      if (coarse.dead[I * d + r]) coarse.A.blk(coarse.A.find(I, I))[r * d + r] = 1.0;
}

// ---------------------------------------------------------------- colouring

// Colouring priority.  Fine level: splitmix64(vertex).  Coarser levels (the
// vertices are lattice points): lattice class first, then splitmix64 -- the
// class of a vertex is sum_a ((p_a / u) mod 3) 3^a with u the side of the
// level's smallest cell, and class 0 ranks highest.  On a uniform level the
// Galerkin stencil has radius 2 cells, so vertices of one class are never
// neighbours and the greedy colouring uses 3^d colours there.
u64 colour_priority(const Oracle& o, const Level& lv, size_t l, i64 v) {
  if (l == 0) return splitmix64((u64)v);
  int D = 0;
  for (auto& c : lv.cells) D = std::max(D, c.depth);
  const int sh = o.K - D;
  u64 p[3];
  deinterleave(lv.lat[v], o.dim, o.K + 1, p);
  u64 cls = 0, w = 1;
  for (int a = 0; a < o.dim; ++a) {
    cls += ((p[a] >> sh) % 3) * w;
    w *= 3;
  }
  const u64 ncls = w;  // 9 or 27
  return ((ncls - 1 - cls) << 58) | (splitmix64((u64)v) >> 6);
}

// Greedy colouring in decreasing priority (ties: smaller vertex first): each
// vertex takes the smallest colour unused by its already-coloured neighbours.
// (Jones-Plassmann with the same priorities yields exactly this colouring.)
void colour_level(const Oracle& o, Level& lv, size_t l) {
  const BSR& A = lv.A;
  std::vector<std::pair<u64, int32_t>> order;
  for (i64 v = 0; v < lv.nv; ++v) order.push_back({colour_priority(o, lv, l, v), (int32_t)v});
  std::sort(order.begin(), order.end(), [](const std::pair<u64, int32_t>& a, const std::pair<u64, int32_t>& b) {
    return a.first != b.first ? a.first > b.first : a.second < b.second;
  });
  lv.colour.assign(lv.nv, -1);
  lv.ncol = 0;
  for (auto& pr : order) {
    i64 v = pr.second;
    std::vector<char> used(lv.ncol + 1, 0);
    for (i64 k = A.rp[v]; k < A.rp[v + 1]; ++k) {
      i64 j = A.ci[k];
      if (j != v && lv.colour[j] >= 0) used[lv.colour[j]] = 1;
    }
    int c = 0;
    while (used[c]) ++c;
    lv.colour[v] = c;
    lv.ncol = std::max(lv.ncol, c + 1);
  }
  lv.by_colour.assign(lv.ncol, {});
  for (i64 v = 0; v < lv.nv; ++v) lv.by_colour[lv.colour[v]].push_back((int32_t)v);
}

void diag_inverses(const Oracle& o, Level& lv) {
  const int d = o.dim;
  lv.dinv.assign(lv.nv * d * d, 0.0);
  for (i64 i = 0; i < lv.nv; ++i) small_inverse(d, lv.A.blk(lv.A.find(i, (int32_t)i)), &lv.dinv[i * d * d]);
}

// ---------------------------------------------------------------- coarsest solve (Cholesky)

void factor_coarsest(Oracle& o) {
  const Level& lv = o.L.back();
  const int d = o.dim;
  const i64 n = lv.nv * d;
  o.nc = n;
  std::vector<double> M(n * n, 0.0);
  for (i64 i = 0; i < lv.nv; ++i)
    for (i64 k = lv.A.rp[i]; k < lv.A.rp[i + 1]; ++k)
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) M[(i * d + a) * n + (i64)lv.A.ci[k] * d + b] = lv.A.blk(k)[a * d + b];
  double maxdiag = 0.0;
  for (i64 i = 0; i < n; ++i) maxdiag = std::max(maxdiag, M[i * n + i]);
  o.chol.assign(n * n, 0.0);
  o.chol_drop.assign(n, 0);
  for (i64 j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (i64 k = 0; k < j; ++k) s -= o.chol[j * n + k] * o.chol[j * n + k];
    if (s <= 1e-14 * maxdiag) {
      o.chol_drop[j] = 1;
      continue;
    }
    double ljj = std::sqrt(s);
    o.chol[j * n + j] = ljj;
    for (i64 i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (i64 k = 0; k < j; ++k) t -= o.chol[i * n + k] * o.chol[j * n + k];
      o.chol[i * n + j] = t / ljj;
    }
  }
}

void solve_coarsest(const Oracle& o, const double* b, double* x) {
  const i64 n = o.nc;
  std::vector<double> y(n, 0.0);
  for (i64 i = 0; i < n; ++i) {
    if (o.chol_drop[i]) continue;
    double t = b[i];
    for (i64 k = 0; k < i; ++k) t -= o.chol[i * n + k] * y[k];
    y[i] = t / o.chol[i * n + i];
  }
  for (i64 i = n - 1; i >= 0; --i) {
    if (o.chol_drop[i]) {
      x[i] = 0.0;
      continue;
    }
    double t = y[i];
    for (i64 k = i + 1; k < n; ++k) t -= o.chol[k * n + i] * x[k];
    x[i] = t / o.chol[i * n + i];
  }
}

// ---------------------------------------------------------------- smoother and V-cycle (Alg. 1, Alg. 3)

// One multicolour block Gauss-Seidel sweep: for each colour in turn, every
// vertex i of that colour sets x_i = D_ii^{-1} (b_i - sum_{j != i} A_ij x_j).
// The vertices of one colour are never neighbours, so within a colour the
// updates are independent (the parallel build splits them over threads).
void gs_sweep(const Oracle& o, const Level& lv, const double* b, double* x, bool forward) {
  const int d = o.dim;
  for (int cc = 0; cc < lv.ncol; ++cc) {
    const int c = forward ? cc : lv.ncol - 1 - cc;
    const std::vector<int32_t>& vs = lv.by_colour[c];
#pragma omp parallel for schedule(static)
    for (i64 t = 0; t < (i64)vs.size(); ++t) {
      const int32_t i = vs[t];
      double r[3];
      for (int a = 0; a < d; ++a) r[a] = b[(i64)i * d + a];
      for (i64 k = lv.A.rp[i]; k < lv.A.rp[i + 1]; ++k) {
        i64 j = lv.A.ci[k];
        if (j == i) continue;
        const double* B = lv.A.blk(k);
        for (int a = 0; a < d; ++a)
          for (int bb = 0; bb < d; ++bb) r[a] -= B[a * d + bb] * x[j * d + bb];
      }
      const double* Di = &lv.dinv[(i64)i * d * d];
      for (int a = 0; a < d; ++a) {
        double s = 0.0;
        for (int bb = 0; bb < d; ++bb) s += Di[a * d + bb] * r[bb];
        x[(i64)i * d + a] = s;
      }
    }
  }
}

// The paper's own smoother (Sec. 2.1, Alg. 1): scalar Gauss-Seidel over the
// unknowns in component-major order U = (u^1_1 .. u^1_N, u^2_1 .. u^2_N, ..),
// vertices in the level's own numbering; the backward sweep visits them in
// reverse order.  Unknown (i, a) is set to
// (b_ia - sum over (j, b) != (i, a) of A_ij[a][b] x_jb) / A_ii[a][a].
void gs_lex_sweep(const Oracle& o, const Level& lv, const double* b, double* x, bool forward) {
  const int d = o.dim;
  const i64 n = lv.nv * d;
  for (i64 step = 0; step < n; ++step) {
    const i64 u = forward ? step : n - 1 - step;
    const int a = (int)(u / lv.nv);
    const i64 i = u - (i64)a * lv.nv;
    double r = b[i * d + a], diag = 0.0;
    for (i64 k = lv.A.rp[i]; k < lv.A.rp[i + 1]; ++k) {
      const i64 j = lv.A.ci[k];
      const double* B = lv.A.blk(k);
      for (int bb = 0; bb < d; ++bb) {
        if (j == i && bb == a) {
          diag = B[a * d + bb];
          continue;
        }
        r -= B[a * d + bb] * x[j * d + bb];
      }
    }
    x[i * d + a] = r / diag;
  }
}

void smooth(const Oracle& o, const Level& lv, const double* b, double* x, bool forward) {
  if (o.smoother == 1)
    gs_lex_sweep(o, lv, b, x, forward);
  else
    gs_sweep(o, lv, b, x, forward);
}

void restrict_to(const Oracle& o, const Level& fine, const Level& coarse, const double* r, double* bc) {
  const int d = o.dim;
  for (i64 i = 0; i < coarse.nv * d; ++i) bc[i] = 0.0;
  for (i64 i = 0; i < fine.nv; ++i)
    for (i64 a = fine.P.rp[i]; a < fine.P.rp[i + 1]; ++a)
      for (int c = 0; c < d; ++c)
        if (!fine.dead[i * d + c]) bc[(i64)fine.P.ci[a] * d + c] += fine.P.w[a] * r[i * d + c];
}

void prolong_add(const Oracle& o, const Level& fine, const double* ec, double* x) {
  const int d = o.dim;
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < fine.nv; ++i)
    for (i64 a = fine.P.rp[i]; a < fine.P.rp[i + 1]; ++a)
      for (int c = 0; c < d; ++c)
        if (!fine.dead[i * d + c]) x[i * d + c] += fine.P.w[a] * ec[(i64)fine.P.ci[a] * d + c];
}

// Alg. 3 (two-level V-cycle) used recursively, as the preconditioner:
// zero initial guess, n1 pre-smoothing and n2 post-smoothing sweeps with the
// post-smoothing sweeps in reverse order, direct solve on the coarsest level.
// With o.gamma = 2 it is the W-cycle of Fig. 2: the coarse problem
// A_{l+1} e = R r is approximated by gamma cycles from e = 0, each on the
// current coarse residual (the coarsest level is solved once, exactly).
void vcycle(const Oracle& o, size_t l, const double* b, double* x, int n1, int n2) {
  const Level& lv = o.L[l];
  const int d = o.dim;
  const i64 n = lv.nv * d;
  if (l + 1 == o.L.size()) {
    solve_coarsest(o, b, x);
    return;
  }
  for (i64 i = 0; i < n; ++i) x[i] = 0.0;
  for (int s = 0; s < n1; ++s) smooth(o, lv, b, x, true);
  std::vector<double> r(n);
  bsr_apply(lv.A, x, r.data());
  for (i64 i = 0; i < n; ++i) r[i] = b[i] - r[i];
  const Level& cv = o.L[l + 1];
  const i64 nc = cv.nv * d;
  std::vector<double> bc(nc), ec(nc);
  restrict_to(o, lv, cv, r.data(), bc.data());
  vcycle(o, l + 1, bc.data(), ec.data(), n1, n2);
  const int reps = l + 2 == o.L.size() ? 1 : o.gamma;
  for (int rep = 1; rep < reps; ++rep) {
    std::vector<double> rc(nc), dc(nc);
    bsr_apply(cv.A, ec.data(), rc.data());
    for (i64 i = 0; i < nc; ++i) rc[i] = bc[i] - rc[i];
    vcycle(o, l + 1, rc.data(), dc.data(), n1, n2);
    for (i64 i = 0; i < nc; ++i) ec[i] += dc[i];
  }
  prolong_add(o, lv, ec.data(), x);
  for (int s = 0; s < n2; ++s) smooth(o, lv, b, x, false);
}

// The additive form of Sec. 4, B_h = S_h + Pi B_0 Pi^T, at the fine level:
// S_h is the symmetric Gauss-Seidel smoother (n1 forward then n2 backward
// sweeps from zero), Pi = P_0, and B_0 is the cycle above on level 1 (the
// exact inverse when level 1 is the coarsest).  The two terms are summed.
void additive_precond(const Oracle& o, const double* r, double* z, int n1, int n2) {
  const Level& lv = o.L[0];
  const int d = o.dim;
  const i64 n = lv.nv * d;
  if (o.L.size() == 1) {
    solve_coarsest(o, r, z);
    return;
  }
  for (i64 i = 0; i < n; ++i) z[i] = 0.0;
  for (int s = 0; s < n1; ++s) smooth(o, lv, r, z, true);
  for (int s = 0; s < n2; ++s) smooth(o, lv, r, z, false);
  const Level& cv = o.L[1];
  std::vector<double> bc(cv.nv * d), ec(cv.nv * d);
  restrict_to(o, lv, cv, r, bc.data());
  vcycle(o, 1, bc.data(), ec.data(), n1, n2);
  prolong_add(o, lv, ec.data(), z);
}

// The preconditioner PCG applies: the cycle from the fine level, or the
// additive form.
void apply_preconditioner(const Oracle& o, const double* r, double* z) {
  if (o.additive)
    additive_precond(o, r, z, 1, 1);
  else
    vcycle(o, 0, r, z, 1, 1);
}

// ---------------------------------------------------------------- setup driver

int setup(Oracle& o, const i64* order) {
  const int d = o.dim;
  o.K = dim_K(d);
  BSR A;
  int rc = assemble(o, A);
  if (rc) return rc;
  apply_dirichlet(o, A);
  bounding_square_and_keys(o);
  build_tree_insertion(o, order);
  o.L.clear();
  o.L.emplace_back();
  Level& L0 = o.L[0];
  L0.nv = o.nv;
  L0.A = std::move(A);
  L0.dead.assign(o.is_dir.begin(), o.is_dir.end());
  if (o.coarse_max_dofs > 0 && o.nv * d <= o.coarse_max_dofs) {
    colour_level(o, o.L[0], 0);
    diag_inverses(o, o.L[0]);
    factor_coarsest(o);
    return 0;
  }
  // level 1: the non-empty leaves
  std::set<CellKey> leaves(o.leaf_of.begin(), o.leaf_of.end());
  Level L1;
  L1.cells.assign(leaves.begin(), leaves.end());
  level_vertices(o, L1);
  o.L.push_back(std::move(L1));
  build_P0(o, o.L[0], o.L[1]);
  galerkin(o, o.L[0], o.L[1]);
  // coarser levels until the root (or until the level is small enough)
  while (true) {
    Level& cur = o.L.back();
    bool at_root = cur.cells.size() == 1 && cur.cells[0].depth == 0;
    if (at_root) break;
    if (o.coarse_max_dofs > 0 && cur.nv * d <= o.coarse_max_dofs) break;
    Level nx;
    nx.cells = merge_deepest(o, cur.cells);
    level_vertices(o, nx);
    o.L.push_back(std::move(nx));
    Level& f = o.L[o.L.size() - 2];
    build_Pl(o, f, o.L.back());
    galerkin(o, f, o.L.back());
  }
  for (size_t l = 0; l < o.L.size(); ++l) {
    colour_level(o, o.L[l], l);
    diag_inverses(o, o.L[l]);
  }
  factor_coarsest(o);
  return 0;
}

// Alg. 2 (PCG) with U0 = 0; rel_res = ||r|| / ||F|| (Sec. 5 item (3)).  The
// iteration count is the number of products A p.  M is applied only while
// not converged (same iterates as Alg. 2).
int pcg(const Oracle& o, const double* Fin, double* U, double tol, int max_iters, int* iters, double* relres,
        double* hist, int hist_cap, int precondition) {
  const int d = o.dim;
  const i64 n = o.nv * d;
  std::vector<double> F(n), r(n), z(n), p(n), q(n), x(n, 0.0);
  for (i64 i = 0; i < n; ++i) F[i] = o.is_dir[i] ? 0.0 : Fin[i] - o.lift[i];
  const Level& L0 = o.L[0];
  r = F;
  double res0 = std::sqrt(dot(r, r));
  *iters = 0;
  *relres = 0.0;
  int status = 0;
  if (res0 == 0.0) {
    for (i64 i = 0; i < n; ++i) U[i] = o.udir[i];
    return 0;
  }
  auto applyM = [&](const std::vector<double>& rr, std::vector<double>& zz) {
    if (precondition)
      apply_preconditioner(o, rr.data(), zz.data());
    else
      zz = rr;
  };
  applyM(r, z);
  p = z;
  double rho = dot(r, z);
  int k = 0;
  status = 1;  // not converged unless the loop breaks
  while (k < max_iters) {
    bsr_apply(L0.A, p.data(), q.data());
    double pq = dot(p, q);
    if (!(pq > 0.0)) {
      status = -5;
      break;
    }
    double alpha = rho / pq;
    for (i64 i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    ++k;
    double rel = std::sqrt(dot(r, r)) / res0;
    if (hist && k - 1 < hist_cap) hist[k - 1] = rel;
    *relres = rel;
    if (rel < tol) {
      status = 0;
      break;
    }
    applyM(r, z);
    double rho_new = dot(r, z);
    double beta = rho_new / rho;
    for (i64 i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
  *iters = k;
  for (i64 i = 0; i < n; ++i) U[i] = x[i] + o.udir[i];
  return status;
}

}  // namespace

// ---------------------------------------------------------------- C interface for the tests

extern "C" {

typedef struct Oracle oracle_t;

// Export selectors.
enum {
  OR_MORTON = 0,      // u64[nv]            Morton keys of the quantised fine coordinates
  OR_LEAF = 1,        // i64[2*nv]          (depth, cell key) of every fine vertex's leaf (insertion)
  OR_LEAF_SORTED = 2, // i64[2*nv]          same, from the sort/count cross-check
  OR_CELLS = 3,       // i64[2*ncells]      (depth, key) of the cells of a level >= 1
  OR_LATTICE = 4,     // u64[nv_l]          lattice corner keys of a level >= 1
  OR_P_RP = 5,        // i64[nv_l+1]        P_s row pointers (level -> level+1)
  OR_P_CI = 6,        // i32[nnz]
  OR_P_W = 7,         // f64[nnz]
  OR_A_RP = 8,        // i64[nv_l+1]        operator block pattern
  OR_A_CI = 9,        // i32[nnzb]
  OR_A_V = 10,        // f64[nnzb*d*d]
  OR_DEAD = 11,       // u8[nv_l*d]
  OR_COLOUR = 12,     // i32[nv_l]
  OR_DINV = 13,       // f64[nv_l*d*d]
  OR_BOX = 14,        // f64[2]             (m, M)
  OR_LIFT = 15,       // f64[n]
  OR_VOL = 16,        // f64[ne]
};

int or_setup(int dim, int64_t nv, const double* X, int64_t ne, const int32_t* E, const double* lam,
             const double* mu, int64_t ndir, const int64_t* dir_dofs, const double* dir_vals, int threshold,
             int64_t coarse_max_dofs, const int64_t* insertion_order, oracle_t** out) {
  if ((dim != 2 && dim != 3) || nv <= 0 || ne <= 0 || !X || !E || !lam || !mu || !out) return -1;
  Oracle* o = new Oracle();
  o->dim = dim;
  o->nv = nv;
  o->ne = ne;
  o->T = threshold > 0 ? threshold : (dim == 2 ? 4 : 8);
  o->coarse_max_dofs = coarse_max_dofs;
  o->X.assign(X, X + nv * dim);
  o->E.assign(E, E + ne * (dim + 1));
  for (auto v : o->E)
    if (v < 0 || v >= nv) {
      delete o;
      return -1;
    }
  o->lam.assign(lam, lam + ne);
  o->mu.assign(mu, mu + ne);
  o->is_dir.assign(nv * dim, 0);
  o->udir.assign(nv * dim, 0.0);
  for (int64_t k = 0; k < ndir; ++k) {
    if (dir_dofs[k] < 0 || dir_dofs[k] >= nv * dim) {
      delete o;
      return -1;
    }
    o->is_dir[dir_dofs[k]] = 1;
    o->udir[dir_dofs[k]] = dir_vals ? dir_vals[k] : 0.0;
  }
  int rc = setup(*o, insertion_order);
  if (rc) {
    delete o;
    return rc;
  }
  *out = o;
  return 0;
}

// Fine level only: assembly (Sec. 2), Dirichlet rows, bounding square and
// Morton keys (Sec. 3.1.1 Step 1).  No tree insertion, hierarchy or colouring:
// enough for A u, the load vector, the keys and the sorted-key leaves of a
// mesh too large for the full setup.
int or_setup_fine(int dim, int64_t nv, const double* X, int64_t ne, const int32_t* E, const double* lam,
                  const double* mu, int64_t ndir, const int64_t* dir_dofs, const double* dir_vals, int threshold,
                  oracle_t** out) {
  if ((dim != 2 && dim != 3) || nv <= 0 || ne <= 0 || !X || !E || !lam || !mu || !out) return -1;
  Oracle* o = new Oracle();
  o->dim = dim;
  o->nv = nv;
  o->ne = ne;
  o->T = threshold > 0 ? threshold : (dim == 2 ? 4 : 8);
  o->X.assign(X, X + nv * dim);
  o->E.assign(E, E + ne * (dim + 1));
  for (auto v : o->E)
    if (v < 0 || v >= nv) {
      delete o;
      return -1;
    }
  o->lam.assign(lam, lam + ne);
  o->mu.assign(mu, mu + ne);
  o->is_dir.assign(nv * dim, 0);
  o->udir.assign(nv * dim, 0.0);
  for (int64_t k = 0; k < ndir; ++k) {
    if (dir_dofs[k] < 0 || dir_dofs[k] >= nv * dim) {
      delete o;
      return -1;
    }
    o->is_dir[dir_dofs[k]] = 1;
    o->udir[dir_dofs[k]] = dir_vals ? dir_vals[k] : 0.0;
  }
  o->K = dim_K(dim);
  BSR A;
  int rc = assemble(*o, A);
  if (rc) {
    delete o;
    return rc;
  }
  apply_dirichlet(*o, A);
  bounding_square_and_keys(*o);
  o->L.clear();
  o->L.emplace_back();
  o->L[0].nv = nv;
  o->L[0].A = std::move(A);
  o->L[0].dead.assign(o->is_dir.begin(), o->is_dir.end());
  *out = o;
  return 0;
}

void or_destroy(oracle_t* o) { delete o; }

int or_num_levels(const oracle_t* o) { return (int)o->L.size(); }

int or_level_info(const oracle_t* o, int l, int64_t* nv, int64_t* nnzb, int32_t* ncol) {
  if (l < 0 || l >= (int)o->L.size()) return -1;
  *nv = o->L[l].nv;
  *nnzb = o->L[l].A.nnz();
  *ncol = o->L[l].ncol;
  return 0;
}

int64_t or_export(const oracle_t* o, int what, int l, void* buf) {
  const int d = o->dim;
  auto put = [&](const void* src, int64_t bytes) -> int64_t {
    if (buf) std::memcpy(buf, src, (size_t)bytes);
    return bytes;
  };
  if (what == OR_MORTON) return put(o->mkey.data(), o->nv * 8);
  if (what == OR_LEAF || what == OR_LEAF_SORTED) {
    std::vector<CellKey> lf;
    if (what == OR_LEAF)
      lf = o->leaf_of;
    else
      build_tree_sorted(*o, lf);
    std::vector<int64_t> out(2 * o->nv);
    for (int64_t v = 0; v < o->nv; ++v) {
      out[2 * v] = lf[v].depth;
      out[2 * v + 1] = (int64_t)lf[v].key;
    }
    return put(out.data(), (int64_t)out.size() * 8);
  }
  if (what == OR_BOX) {
    double b[2] = {o->m, o->Mx};
    return put(b, 16);
  }
  if (what == OR_LIFT) return put(o->lift.data(), (int64_t)o->lift.size() * 8);
  if (what == OR_VOL) return put(o->vol.data(), (int64_t)o->vol.size() * 8);
  if (l < 0 || l >= (int)o->L.size()) return -1;
  const Level& lv = o->L[l];
  switch (what) {
    case OR_CELLS: {
      std::vector<int64_t> out;
      for (auto& c : lv.cells) {
        out.push_back(c.depth);
        out.push_back((int64_t)c.key);
      }
      return put(out.data(), (int64_t)out.size() * 8);
    }
    case OR_LATTICE: return put(lv.lat.data(), (int64_t)lv.lat.size() * 8);
    case OR_P_RP: return put(lv.P.rp.data(), (int64_t)lv.P.rp.size() * 8);
    case OR_P_CI: return put(lv.P.ci.data(), (int64_t)lv.P.ci.size() * 4);
    case OR_P_W: return put(lv.P.w.data(), (int64_t)lv.P.w.size() * 8);
    case OR_A_RP: return put(lv.A.rp.data(), (int64_t)lv.A.rp.size() * 8);
    case OR_A_CI: return put(lv.A.ci.data(), (int64_t)lv.A.ci.size() * 4);
    case OR_A_V: return put(lv.A.v.data(), (int64_t)lv.A.v.size() * 8);
    case OR_DEAD: return put(lv.dead.data(), (int64_t)lv.dead.size());
    case OR_COLOUR: return put(lv.colour.data(), (int64_t)lv.colour.size() * 4);
    case OR_DINV: return put(lv.dinv.data(), (int64_t)lv.dinv.size() * 8);
    default: return -1;
  }
  (void)d;
}

int or_assemble_load(const oracle_t* o, const double* f, double* F) {
  assemble_load(*o, f, F);
  return 0;
}

// y = A_l x on level l (identity rows at dead dofs).
int or_apply_A(const oracle_t* o, int l, const double* x, double* y) {
  if (l < 0 || l >= (int)o->L.size()) return -1;
  bsr_apply(o->L[l].A, x, y);
  return 0;
}

// One multicolour GS sweep on level l, in place on x.
// Select the smoother of the V-cycle and of or_gs_sweep: 0 multicolour
// point-block GS (the GPU path's), 1 scalar lexicographic GS (the paper's).
// Threads of the parallel build (returns the count in use); the default
// build runs on one thread and returns 1.
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int or_set_smoother(oracle_t* o, int smoother) {
  if (!o || smoother < 0 || smoother > 1) return -1;
  o->smoother = smoother;
  return 0;
}

int or_gs_sweep(const oracle_t* o, int l, const double* b, double* x, int forward) {
  if (l < 0 || l >= (int)o->L.size()) return -1;
  smooth(*o, o->L[l], b, x, forward != 0);
  return 0;
}

// x = M b on level l (the V-cycle from level l down).
int or_vcycle(const oracle_t* o, int l, const double* b, double* x) {
  if (l < 0 || l >= (int)o->L.size()) return -1;
  vcycle(*o, (size_t)l, b, x, 1, 1);
  return 0;
}

// Cycle variant: gamma >= 1 coarse corrections per level (1 = V, 2 = W);
// additive = 1 makes the preconditioner B_h = S_h + Pi B_0 Pi^T.
int or_set_cycle(oracle_t* o, int gamma, int additive) {
  if (!o || gamma < 1 || gamma > 8 || additive < 0 || additive > 1) return -1;
  o->gamma = gamma;
  o->additive = additive;
  return 0;
}

// z = B r with the preconditioner PCG uses (cycle variant included).
int or_precondition(const oracle_t* o, const double* r, double* z) {
  if (!o) return -1;
  apply_preconditioner(*o, r, z);
  return 0;
}

int or_restrict(const oracle_t* o, int l, const double* r, double* bc) {
  if (l < 0 || l + 1 >= (int)o->L.size()) return -1;
  restrict_to(*o, o->L[l], o->L[l + 1], r, bc);
  return 0;
}

int or_prolong_add(const oracle_t* o, int l, const double* ec, double* x) {
  if (l < 0 || l + 1 >= (int)o->L.size()) return -1;
  prolong_add(*o, o->L[l], ec, x);
  return 0;
}

int or_coarse_solve(const oracle_t* o, const double* b, double* x) {
  solve_coarsest(*o, b, x);
  return 0;
}

int or_solve(const oracle_t* o, const double* F, double* U, double tol, int max_iters, int* iters, double* relres,
             double* hist, int hist_cap, int precondition) {
  return pcg(*o, F, U, tol, max_iters, iters, relres, hist, hist_cap, precondition);
}

uint64_t or_splitmix64(uint64_t x) { return splitmix64(x); }

}  // extern "C"
