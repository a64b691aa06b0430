// ASMG oracle: TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded FP64 restatement of the auxiliary-space
// multigrid preconditioned CG of Grasedyck, Wang and Xu ("A Nearly Optimal
// Multigrid Method for General Unstructured Grids").  Only the test suite,
// the smoke check and the CPU-baseline leg of the benchmark may load it.  It
// shares no code, header or table with the CUDA library and imports nothing
// from it.  Compile with -O2 -ffp-contract=off (no FMA contraction) so that
// the cluster-tree quantisation rounds exactly like the device code.
//
// Each function names the passage of the paper it follows.  Where the paper
// is silent or garbled, the reading taken is stated beside the code:
//   R1  root box = vertex bounding box widened to a square at its min corner
//   R2  quantised Morton keys with D = 31 (2D) / 21 (3D) bits per coordinate
//   R3  closure = unique minimal edge-2:1-balanced refinement of the box tree
//   R4  box triangulation: SW-NE diagonal, or a centre fan when an edge
//       carries a hanging midpoint (the Fig. "closure2" templates)
//   R5  Scott-Zhang support sigma_i = lowest-index element at node i;
//       psi_i = (12 lambda_i - 3)/|sigma_i| (2D dual basis); exact clipping
//   R6  finest auxiliary coefficient = area-weighted mean of the fine ones;
//       coarser auxiliary operators are Galerkin (I^T A I)
//   R7  smoother R_l = multicolour Gauss-Seidel on the set N~_l of new or
//       changed nodes (local smoothing, eq. "decomposition"); "full" mode
//       smooths every node of the level instead
//   R8  Algorithm 1 with "+" corrections applied from zero as a preconditioner
//   R9  flexible (Polak-Ribiere) beta in PCG, stop at ||r|| <= rtol ||b||
//   R10 colouring = Jones-Plassmann with splitmix64 priorities, smallest
//       free colour, on the non-vanishing couplings, then three rounds of
//       iterated greedy recolouring; the same definition is implemented
//       independently on the device, so no colouring is ever passed from one
//       side to the other.  Option colouring = 2 colours an auxiliary level
//       by lattice parity when that parity 2-colours its couplings (uniform
//       levels are bipartite: couplings across hypotenuses vanish) and by
//       the default otherwise
//   R18 mixed Dirichlet/Neumann boundaries (2D and 3D): contact of a simplex with
//       Omega or Gamma_D means contact of its interior; Dirichlet auxiliary
//       nodes lie on Gamma_D or on a triangle removed for Gamma_D
//   R19 near-boundary correction: after the coarse correction of every level
//       above the coarsest, the free nodes of the j-th layer around the
//       level's boundary are solved exactly (dense Cholesky)
//
// 3D: the same steps on an octree with tetrahedral auxiliary grids (R4-3D
// below); fine assembly, mass matrix and the tree are dimension-generic.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

typedef __int128 i128;

struct CSR {
  int64_t nr = 0, nc = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  double get(int64_t i, int32_t j) const {
    for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p)
      if (col[p] == j) return val[p];
    return 0.0;
  }
};

// Build a CSR matrix from per-row (column, value) lists: sort each row by
// column and add duplicates.
CSR csr_from_rows(int64_t nr, int64_t nc, std::vector<std::vector<std::pair<int32_t, double>>>& rows) {
  CSR M;
  M.nr = nr;
  M.nc = nc;
  M.ptr.assign(nr + 1, 0);
  for (int64_t i = 0; i < nr; ++i) {
    auto& r = rows[i];
    std::stable_sort(r.begin(), r.end(),
                     [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) { return a.first < b.first; });
    int64_t cnt = 0;
    for (size_t k = 0; k < r.size(); ++k)
      if (k == 0 || r[k].first != r[k - 1].first) ++cnt;
    M.ptr[i + 1] = M.ptr[i] + cnt;
  }
  M.col.resize(M.ptr[nr]);
  M.val.resize(M.ptr[nr]);
  for (int64_t i = 0; i < nr; ++i) {
    auto& r = rows[i];
    int64_t p = M.ptr[i] - 1;
    for (size_t k = 0; k < r.size(); ++k) {
      if (k == 0 || r[k].first != r[k - 1].first) {
        ++p;
        M.col[p] = r[k].first;
        M.val[p] = 0.0;
      }
      M.val[p] += r[k].second;
    }
    std::vector<std::pair<int32_t, double>>().swap(r);
  }
  return M;
}

void spmv(const CSR& A, const double* x, double* y) {
  for (int64_t i = 0; i < A.nr; ++i) {
    double s = 0.0;
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) s += A.val[p] * x[A.col[p]];
    y[i] = s;
  }
}

CSR transpose(const CSR& A) {
  std::vector<std::vector<std::pair<int32_t, double>>> rows(A.nc);
  for (int64_t i = 0; i < A.nr; ++i)
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) rows[A.col[p]].push_back({(int32_t)i, A.val[p]});
  return csr_from_rows(A.nc, A.nr, rows);
}

// C = A * B (plain row-by-row sparse product).
CSR matmul(const CSR& A, const CSR& B) {
  std::vector<std::vector<std::pair<int32_t, double>>> rows(A.nr);
  for (int64_t i = 0; i < A.nr; ++i)
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
      for (int64_t q = B.ptr[A.col[p]]; q < B.ptr[A.col[p] + 1]; ++q)
        rows[i].push_back({B.col[q], A.val[p] * B.val[q]});
  return csr_from_rows(A.nr, B.nc, rows);
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// splitmix64 (Steele, Lea, Flood 2014; Vigna's published constants): a
// counter-based 64-bit mixer used for colouring priorities.
uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

struct Params {
  int n_min = 3, nu_pre = 2, nu_post = 2, coarse_max = 512, smoothing = 0, max_iter = 500, colouring = 0, stage = 2;
  int smoother = 0;     // fine smoother S: 0 Gauss-Seidel (D - L)^{-1}, 1 Jacobi D^{-1} (Sec. 4.1)
  int additive = 0;     // 0: multiplicative (Algorithm 1); 1: additive B = S + Pi Btilde Pi^t (eq. fasp)
  int fine_sweeps = 1;  // smoothing steps per application of S (and of S^t)
  int iteration = 0;    // 0: PCG (Sec. 5.2); 1: the ASMG iteration u <- u + B (b - A u)
  int nb_layers = 2;    // mixed boundaries: layers j of the near-boundary correction (Algorithm 3); < 0: none
};

struct Seg {
  uint64_t prefix;
  int64_t begin, end;
  int split;
};

struct Level {
  std::vector<uint64_t> key;                 // free nodes, ascending lattice Morton key
  std::vector<uint64_t> allkey;              // all nodes incl. boundary, ascending
  std::vector<std::array<uint64_t, 3>> tri;  // level triangles (lattice Morton keys, CCW)
  std::vector<std::array<uint64_t, 4>> tet;  // level tetrahedra (3D, positively oriented)
  CSR A;                                     // level operator on free nodes
  CSR I;                                     // nodal interpolation from level l-1
  std::vector<int32_t> smooth;               // smoothing set sorted by (colour, index)
  std::vector<int32_t> colour;               // colour per free node, -1 outside the set
  std::vector<int32_t> cstart;               // colour class starts in `smooth`
  std::vector<int32_t> nbset;                // near-boundary free nodes J_{l,j} (Algorithm 3)
  std::vector<double> nbchol;                // Cholesky factor of A restricted to nbset
};

struct Oracle {
  int dim = 2;
  int64_t nv = 0, ne = 0;
  std::vector<double> X;
  std::vector<int32_t> E;
  std::vector<uint8_t> bflag;
  std::vector<double> coeff;
  Params prm;
  std::string err;

  // fine problem (Sec. 2)
  std::vector<int32_t> free_of_vertex, vertex_of_free;
  CSR A;
  std::vector<int32_t> fine_colour, fine_smooth, fine_cstart;

  // cluster tree (Sec. 3.1)
  int D = 31;
  double amin[3] = {0, 0, 0}, L = 0;
  std::vector<uint64_t> keys;   // per element, in element order
  std::vector<int32_t> perm;    // elements sorted by key (stable)
  std::vector<std::vector<Seg>> tree;

  // closed box tree (Sec. 3.2): per depth, packed box coordinates -> split
  std::vector<std::unordered_map<uint64_t, uint8_t>> boxes;
  int J = 0;  // finest auxiliary level (depth)
  int LB = 0; // 3D: lattice bits of the auxiliary nodes (J + 1)
  int c = 0;  // coarsest level used by the V-cycle
  bool boxdomain = true;  // the fine elements fill the root box (else Dirichlet auxiliary grids, R17)
  bool neumann = false;   // some vertex is Neumann: mixed auxiliary grids (R18) and Algorithm 3
  std::vector<Level> lv;
  std::vector<double> finest_coef;  // per triangle of level J
  CSR P, Pfull;                     // Scott-Zhang transfer (free / all aux columns)
  std::vector<double> chol;         // dense Cholesky factor of A_c (row-major lower)
  int64_t nc_dense = 0;
};

// --------------------------------------------------------------------------
// Sec. 2: P1 stiffness a_ij = int a grad phi_i . grad phi_j and mass matrix.
// --------------------------------------------------------------------------

// Barycentric gradients G (rows) and measure of a simplex.
void simplex_geometry(const Oracle& o, int64_t e, double G[4][3], double& vol) {
  const int d = o.dim;
  const int32_t* v = &o.E[e * (d + 1)];
  const double* p0 = &o.X[(int64_t)v[0] * d];
  if (d == 2) {
    const double* p1 = &o.X[(int64_t)v[1] * 2];
    const double* p2 = &o.X[(int64_t)v[2] * 2];
    double x10 = p1[0] - p0[0], y10 = p1[1] - p0[1], x20 = p2[0] - p0[0], y20 = p2[1] - p0[1];
    double det = x10 * y20 - x20 * y10;
    vol = 0.5 * det;
    G[1][0] = y20 / det;
    G[1][1] = -x20 / det;
    G[2][0] = -y10 / det;
    G[2][1] = x10 / det;
    G[0][0] = -(G[1][0] + G[2][0]);
    G[0][1] = -(G[1][1] + G[2][1]);
  } else {
    double Jm[3][3];
    for (int k = 1; k <= 3; ++k)
      for (int r = 0; r < 3; ++r) Jm[r][k - 1] = o.X[(int64_t)v[k] * 3 + r] - p0[r];
    double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                 Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                 Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
    vol = det / 6.0;
    // rows of J^{-1} are the gradients of lambda_1..lambda_3
    double inv[3][3];
    inv[0][0] = (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) / det;
    inv[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) / det;
    inv[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) / det;
    inv[1][0] = (Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2]) / det;
    inv[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) / det;
    inv[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) / det;
    inv[2][0] = (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]) / det;
    inv[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) / det;
    inv[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) / det;
    for (int k = 0; k < 3; ++k)
      for (int r = 0; r < 3; ++r) G[k + 1][r] = inv[k][r];
    for (int r = 0; r < 3; ++r) G[0][r] = -(G[1][r] + G[2][r] + G[3][r]);
  }
}

void assemble_fine(Oracle& o) {
  const int d = o.dim, nvert = d + 1;
  o.free_of_vertex.assign(o.nv, -1);
  o.vertex_of_free.clear();
  for (int64_t v = 0; v < o.nv; ++v)
    if (o.bflag[v] != 1) {
      o.free_of_vertex[v] = (int32_t)o.vertex_of_free.size();
      o.vertex_of_free.push_back((int32_t)v);
    }
  int64_t n = o.vertex_of_free.size();
  std::vector<std::vector<std::pair<int32_t, double>>> rows(n);
  for (int64_t e = 0; e < o.ne; ++e) {
    double G[4][3], vol;
    simplex_geometry(o, e, G, vol);
    double a = o.coeff.empty() ? 1.0 : o.coeff[e];
    const int32_t* v = &o.E[e * nvert];
    for (int i = 0; i < nvert; ++i) {
      int32_t fi = o.free_of_vertex[v[i]];
      if (fi < 0) continue;
      for (int j = 0; j < nvert; ++j) {
        int32_t fj = o.free_of_vertex[v[j]];
        if (fj < 0) continue;
        double g = 0.0;
        for (int r = 0; r < d; ++r) g += G[i][r] * G[j][r];
        rows[fi].push_back({fj, a * vol * g});
      }
    }
  }
  o.A = csr_from_rows(n, n, rows);
}

// b = M f_h restricted to free rows; M_e = |tau| (1 + delta_ij) / ((d+1)(d+2)).
void mass_apply(const Oracle& o, const double* f, double* b) {
  const int d = o.dim, nvert = d + 1;
  const double den = (d == 2) ? 12.0 : 20.0;
  std::vector<double> full(o.nv, 0.0);
  for (int64_t e = 0; e < o.ne; ++e) {
    double G[4][3], vol;
    simplex_geometry(o, e, G, vol);
    const int32_t* v = &o.E[e * nvert];
    for (int i = 0; i < nvert; ++i) {
      double s = 0.0;
      for (int j = 0; j < nvert; ++j) s += (i == j ? 2.0 : 1.0) * f[v[j]];
      full[v[i]] += vol / den * s;
    }
  }
  for (size_t k = 0; k < o.vertex_of_free.size(); ++k) b[k] = full[o.vertex_of_free[k]];
}

// --------------------------------------------------------------------------
// Sec. 3.1: box tree over element barycenters (R1, R2).
// --------------------------------------------------------------------------

uint64_t interleave(const uint64_t* q, int dim, int bits) {
  uint64_t key = 0;
  for (int j = 0; j < bits; ++j)
    for (int k = 0; k < dim; ++k)
      if ((q[k] >> j) & 1ULL) key |= 1ULL << (dim * j + k);
  return key;
}

void deinterleave(uint64_t key, int dim, int bits, uint64_t* q) {
  for (int k = 0; k < dim; ++k) q[k] = 0;
  for (int j = 0; j < bits; ++j)
    for (int k = 0; k < dim; ++k)
      if ((key >> (dim * j + k)) & 1ULL) q[k] |= 1ULL << j;
}

uint64_t pack_box(const uint64_t* q, int dim) {
  return dim == 2 ? (q[0] | (q[1] << 32)) : (q[0] | (q[1] << 21) | (q[2] << 42));
}

void unpack_box(uint64_t p, int dim, uint64_t* q) {
  if (dim == 2) {
    q[0] = p & 0xffffffffULL;
    q[1] = p >> 32;
  } else {
    q[0] = p & 0x1fffffULL;
    q[1] = (p >> 21) & 0x1fffffULL;
    q[2] = p >> 42;
  }
}

void build_tree(Oracle& o) {
  const int d = o.dim, nvert = d + 1;
  o.D = (d == 2) ? 31 : 21;
  double mx[3];
  for (int k = 0; k < d; ++k) {
    o.amin[k] = INFINITY;
    mx[k] = -INFINITY;
  }
  for (int64_t v = 0; v < o.nv; ++v)
    for (int k = 0; k < d; ++k) {
      o.amin[k] = std::min(o.amin[k], o.X[v * d + k]);
      mx[k] = std::max(mx[k], o.X[v * d + k]);
    }
  o.L = 0.0;
  for (int k = 0; k < d; ++k) o.L = std::max(o.L, mx[k] - o.amin[k]);
  // Quantisation: q = floor((sum_v p_v - (d+1) a) * 2^D / ((d+1) L)), clamped.
  const double S = std::ldexp(1.0, o.D) / (double)(d + 1) / o.L;
  double Ak[3];
  for (int k = 0; k < d; ++k) Ak[k] = (double)(d + 1) * o.amin[k];
  const uint64_t qmax = (1ULL << o.D) - 1;
  o.keys.resize(o.ne);
  for (int64_t e = 0; e < o.ne; ++e) {
    uint64_t q[3];
    for (int k = 0; k < d; ++k) {
      double s = o.X[(int64_t)o.E[e * nvert] * d + k];
      for (int j = 1; j < nvert; ++j) s = s + o.X[(int64_t)o.E[e * nvert + j] * d + k];
      double t = (s - Ak[k]) * S;
      double f = std::floor(t);
      if (!(f > 0.0)) f = 0.0;
      q[k] = (f >= (double)qmax) ? qmax : (uint64_t)f;
    }
    o.keys[e] = interleave(q, d, o.D);
  }
  o.perm.resize(o.ne);
  for (int64_t e = 0; e < o.ne; ++e) o.perm[e] = (int32_t)e;
  std::stable_sort(o.perm.begin(), o.perm.end(), [&](int32_t a, int32_t b) { return o.keys[a] < o.keys[b]; });
  // Level-by-level subdivision; a node with more than n_min barycenters is
  // split into all 2^d children, including empty ones (Sec. 3.1).
  o.tree.clear();
  o.tree.push_back({Seg{0, 0, o.ne, 0}});
  for (int lvl = 0;; ++lvl) {
    std::vector<Seg> next;
    for (auto& s : o.tree[lvl]) {
      if (s.end - s.begin <= o.prm.n_min || lvl >= o.D) continue;
      s.split = 1;
      const int shift = d * (o.D - lvl - 1);
      int64_t p = s.begin;
      for (uint64_t ch = 0; ch < (1ULL << d); ++ch) {
        int64_t b = p;
        while (p < s.end && ((o.keys[o.perm[p]] >> shift) & ((1ULL << d) - 1)) == ch) ++p;
        next.push_back(Seg{(s.prefix << d) | ch, b, p, 0});
      }
    }
    if (next.empty()) break;
    o.tree.push_back(next);
  }
}

// --------------------------------------------------------------------------
// Sec. 3.2: closure (R3).  A leaf must be split when an edge-adjacent leaf
// (face- or edge-adjacent in 3D) is two or more levels finer.
// --------------------------------------------------------------------------

bool box_exists(const Oracle& o, int depth, const uint64_t* q, uint8_t* split) {
  if (depth >= (int)o.boxes.size()) return false;
  auto it = o.boxes[depth].find(pack_box(q, o.dim));
  if (it == o.boxes[depth].end()) return false;
  if (split) *split = it->second;
  return true;
}

// The neighbour offsets whose shared boundary with a box can carry hanging
// nodes: edges in 2D; faces and edges in 3D.
std::vector<std::array<int, 3>> neighbour_offsets(int dim) {
  std::vector<std::array<int, 3>> offs;
  for (int z = (dim == 3 ? -1 : 0); z <= (dim == 3 ? 1 : 0); ++z)
    for (int y = -1; y <= 1; ++y)
      for (int x = -1; x <= 1; ++x) {
        int nz = (x != 0) + (y != 0) + (z != 0);
        if (nz >= 1 && nz <= dim - 1) offs.push_back({x, y, z});
      }
  return offs;
}

bool must_split(const Oracle& o, int depth, const uint64_t* q, const std::vector<std::array<int, 3>>& offs) {
  const int d = o.dim;
  const int64_t nb = 1LL << depth;
  for (auto& off : offs) {
    uint64_t n[3];
    bool inside = true;
    for (int k = 0; k < d; ++k) {
      int64_t v = (int64_t)q[k] + off[k];
      if (v < 0 || v >= nb) inside = false;
      n[k] = (uint64_t)v;
    }
    if (!inside) continue;
    uint8_t sp = 0;
    if (!box_exists(o, depth, n, &sp) || !sp) continue;
    for (int ch = 0; ch < (1 << d); ++ch) {
      bool touches = true;
      uint64_t cq[3];
      for (int k = 0; k < d; ++k) {
        int bit = (ch >> k) & 1;
        if (off[k] == 1 && bit != 0) touches = false;
        if (off[k] == -1 && bit != 1) touches = false;
        cq[k] = 2 * n[k] + bit;
      }
      if (!touches) continue;
      uint8_t csp = 0;
      if (box_exists(o, depth + 1, cq, &csp) && csp) return true;
    }
  }
  return false;
}

void build_closure(Oracle& o) {
  const int d = o.dim;
  o.boxes.assign(o.tree.size(), {});
  for (size_t lvl = 0; lvl < o.tree.size(); ++lvl)
    for (auto& s : o.tree[lvl]) {
      uint64_t q[3];
      deinterleave(s.prefix, d, (int)lvl, q);
      o.boxes[lvl][pack_box(q, d)] = (uint8_t)s.split;
    }
  auto offs = neighbour_offsets(d);
  for (;;) {
    std::vector<std::pair<int, uint64_t>> todo;
    for (size_t lvl = 0; lvl < o.boxes.size(); ++lvl)
      for (auto& kv : o.boxes[lvl]) {
        if (kv.second) continue;
        uint64_t q[3];
        unpack_box(kv.first, d, q);
        if (must_split(o, (int)lvl, q, offs)) todo.push_back({(int)lvl, kv.first});
      }
    if (todo.empty()) break;
    for (auto& t : todo) {
      o.boxes[t.first][t.second] = 1;
      if ((int)o.boxes.size() <= t.first + 1) o.boxes.resize(t.first + 2);
      uint64_t q[3];
      unpack_box(t.second, d, q);
      for (int ch = 0; ch < (1 << d); ++ch) {
        uint64_t cq[3];
        for (int k = 0; k < d; ++k) cq[k] = 2 * q[k] + ((ch >> k) & 1);
        o.boxes[t.first + 1][pack_box(cq, d)] = 0;
      }
    }
  }
  while (!o.boxes.empty() && o.boxes.back().empty()) o.boxes.pop_back();
  o.J = (int)o.boxes.size() - 1;
}

// --------------------------------------------------------------------------
// Sec. 3.3: conforming nested auxiliary triangulations sigma^(l) (R4), 2D.
// Lattice coordinates are integers on the 2^D grid of the root box.
// --------------------------------------------------------------------------

uint64_t node_key2(uint64_t x, uint64_t y) {
  uint64_t q[2] = {x, y};
  return interleave(q, 2, 32);
}

void node_xy(uint64_t key, uint64_t& x, uint64_t& y) {
  uint64_t q[2];
  deinterleave(key, 2, 32, q);
  x = q[0];
  y = q[1];
}

// Triangles of box (depth, ix, iy) as seen at level `lvl`: the SW-NE diagonal
// split, or a fan about the centre when a same-depth edge neighbour is split
// (then the shared edge carries a hanging midpoint).
void box_triangles(const Oracle& o, int depth, uint64_t ix, uint64_t iy, int lvl,
                   std::vector<std::array<uint64_t, 3>>& out) {
  const uint64_t s = 1ULL << (o.D - depth);
  const uint64_t x0 = ix * s, y0 = iy * s;
  bool hang[4] = {false, false, false, false};  // S, E, N, W
  if (depth < lvl) {
    const int dx[4] = {0, 1, 0, -1}, dy[4] = {-1, 0, 1, 0};
    const int64_t nb = 1LL << depth;
    for (int e = 0; e < 4; ++e) {
      int64_t nx = (int64_t)ix + dx[e], ny = (int64_t)iy + dy[e];
      if (nx < 0 || ny < 0 || nx >= nb || ny >= nb) continue;
      uint64_t q[2] = {(uint64_t)nx, (uint64_t)ny};
      uint8_t sp = 0;
      if (box_exists(o, depth, q, &sp) && sp) hang[e] = true;
    }
  }
  uint64_t SW = node_key2(x0, y0), SE = node_key2(x0 + s, y0), NE = node_key2(x0 + s, y0 + s),
           NW = node_key2(x0, y0 + s);
  if (!(hang[0] || hang[1] || hang[2] || hang[3])) {
    out.push_back({SW, SE, NE});
    out.push_back({SW, NE, NW});
    return;
  }
  const uint64_t h = s / 2;
  uint64_t C = node_key2(x0 + h, y0 + h);
  std::vector<uint64_t> ring;
  ring.push_back(SW);
  if (hang[0]) ring.push_back(node_key2(x0 + h, y0));
  ring.push_back(SE);
  if (hang[1]) ring.push_back(node_key2(x0 + s, y0 + h));
  ring.push_back(NE);
  if (hang[2]) ring.push_back(node_key2(x0 + h, y0 + s));
  ring.push_back(NW);
  if (hang[3]) ring.push_back(node_key2(x0, y0 + h));
  for (size_t i = 0; i < ring.size(); ++i) out.push_back({ring[i], ring[(i + 1) % ring.size()], C});
}

bool on_boundary(const Oracle& o, uint64_t key) {
  uint64_t x, y;
  node_xy(key, x, y);
  const uint64_t top = 1ULL << o.D;
  return x == 0 || y == 0 || x == top || y == top;
}

void level_triangles(const Oracle& o, int lvl, std::vector<std::array<uint64_t, 3>>& tri) {
  tri.clear();
  for (int depth = 0; depth <= lvl && depth < (int)o.boxes.size(); ++depth) {
    // deterministic order: sort the boxes of this depth by packed coordinate
    std::vector<std::pair<uint64_t, uint8_t>> bx(o.boxes[depth].begin(), o.boxes[depth].end());
    std::sort(bx.begin(), bx.end());
    for (auto& kv : bx) {
      if (depth < lvl && kv.second) continue;  // interior box of the truncated tree
      uint64_t q[2];
      unpack_box(kv.first, 2, q);
      box_triangles(o, depth, q[0], q[1], lvl, tri);
    }
  }
}

int32_t find_index(const std::vector<uint64_t>& sorted, uint64_t k) {
  auto it = std::lower_bound(sorted.begin(), sorted.end(), k);
  if (it == sorted.end() || *it != k) return -1;
  return (int32_t)(it - sorted.begin());
}

void physical(const Oracle& o, uint64_t key, double* p) {
  uint64_t x, y;
  node_xy(key, x, y);
  p[0] = o.amin[0] + std::ldexp((double)x, -o.D) * o.L;
  p[1] = o.amin[1] + std::ldexp((double)y, -o.D) * o.L;
}

// P1 stiffness of a triangle given in physical coordinates.
void tri_stiffness(const double* p0, const double* p1, const double* p2, double K[3][3]) {
  double x10 = p1[0] - p0[0], y10 = p1[1] - p0[1], x20 = p2[0] - p0[0], y20 = p2[1] - p0[1];
  double det = x10 * y20 - x20 * y10;
  double G[3][2];
  G[1][0] = y20 / det;
  G[1][1] = -x20 / det;
  G[2][0] = -y10 / det;
  G[2][1] = x10 / det;
  G[0][0] = -(G[1][0] + G[2][0]);
  G[0][1] = -(G[1][1] + G[2][1]);
  double area = 0.5 * det;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K[i][j] = area * (G[i][0] * G[j][0] + G[i][1] * G[j][1]);
}

// --------------------------------------------------------------------------
// Clipping and exact integration (R5, R6).
// --------------------------------------------------------------------------

struct Pt {
  double x, y;
};

// Sutherland-Hodgman clipping of a convex polygon by a CCW triangle.
std::vector<Pt> clip(const std::vector<Pt>& poly0, const Pt* K) {
  std::vector<Pt> poly = poly0;
  for (int e = 0; e < 3 && !poly.empty(); ++e) {
    Pt a = K[e], b = K[(e + 1) % 3];
    std::vector<Pt> out;
    size_t n = poly.size();
    for (size_t i = 0; i < n; ++i) {
      Pt P = poly[i], Q = poly[(i + 1) % n];
      double dP = (b.x - a.x) * (P.y - a.y) - (b.y - a.y) * (P.x - a.x);
      double dQ = (b.x - a.x) * (Q.y - a.y) - (b.y - a.y) * (Q.x - a.x);
      bool inP = dP >= 0.0, inQ = dQ >= 0.0;
      if (inP) out.push_back(P);
      if (inP != inQ) {
        double t = dP / (dP - dQ);
        out.push_back(Pt{P.x + t * (Q.x - P.x), P.y + t * (Q.y - P.y)});
      }
    }
    poly.swap(out);
  }
  return poly;
}

// barycentric coordinates of x in triangle T
void bary(const Pt* T, Pt x, double* lam) {
  double det = (T[1].x - T[0].x) * (T[2].y - T[0].y) - (T[2].x - T[0].x) * (T[1].y - T[0].y);
  lam[1] = ((x.x - T[0].x) * (T[2].y - T[0].y) - (T[2].x - T[0].x) * (x.y - T[0].y)) / det;
  lam[2] = ((T[1].x - T[0].x) * (x.y - T[0].y) - (x.x - T[0].x) * (T[1].y - T[0].y)) / det;
  lam[0] = 1.0 - lam[1] - lam[2];
}

double poly_area(const std::vector<Pt>& p) {
  double a = 0.0;
  for (size_t i = 1; i + 1 < p.size(); ++i)
    a += 0.5 * ((p[i].x - p[0].x) * (p[i + 1].y - p[0].y) - (p[i + 1].x - p[0].x) * (p[i].y - p[0].y));
  return a;
}

// Leaf boxes of the closed tree whose closed extent meets [lo, hi].
void leaves_overlapping(const Oracle& o, double lox, double loy, double hix, double hiy,
                        std::vector<std::array<uint64_t, 3>>& out) {
  std::vector<std::array<uint64_t, 3>> stack;  // (depth, ix, iy)
  stack.push_back({0, 0, 0});
  while (!stack.empty()) {
    auto b = stack.back();
    stack.pop_back();
    int depth = (int)b[0];
    double w = std::ldexp(o.L, -depth);
    double x0 = o.amin[0] + (double)b[1] * w, y0 = o.amin[1] + (double)b[2] * w;
    if (x0 > hix || y0 > hiy || x0 + w < lox || y0 + w < loy) continue;
    uint64_t q[2] = {b[1], b[2]};
    uint8_t sp = 0;
    if (!box_exists(o, depth, q, &sp)) continue;
    if (!sp) {
      out.push_back(b);
      continue;
    }
    for (int ch = 0; ch < 4; ++ch) stack.push_back({(uint64_t)depth + 1, 2 * b[1] + (ch & 1), 2 * b[2] + (ch >> 1)});
  }
}

// The triangle of sigma^(l) containing the point (X3/3, Y3/3) (lattice
// units): descend the truncated tree to the level-l box holding it, then test
// its triangles with integer barycentric coordinates.  The point must lie
// strictly inside a triangle (a centroid of a finer nested triangle).
bool locate_level_triangle(const Oracle& o, int l, uint64_t X3, uint64_t Y3, std::array<uint64_t, 3>& out) {
  int depth = 0;
  uint64_t bx = 0, by = 0;
  for (;;) {
    uint64_t q[2] = {bx, by};
    uint8_t sp = 0;
    box_exists(o, depth, q, &sp);
    if (depth == l || !sp) break;
    const uint64_t half3 = 3 * (1ULL << (o.D - depth - 1));
    const uint64_t cx = (X3 - bx * 2 * half3) >= half3 ? 1 : 0;
    const uint64_t cy = (Y3 - by * 2 * half3) >= half3 ? 1 : 0;
    bx = 2 * bx + cx;
    by = 2 * by + cy;
    ++depth;
  }
  std::vector<std::array<uint64_t, 3>> ktri;
  box_triangles(o, depth, bx, by, l, ktri);
  for (auto& kt : ktri) {
    i128 P[3][2];
    for (int v = 0; v < 3; ++v) {
      uint64_t vx, vy;
      node_xy(kt[v], vx, vy);
      P[v][0] = 3 * (i128)vx;
      P[v][1] = 3 * (i128)vy;
    }
    const i128 x = (i128)X3, y = (i128)Y3;
    const i128 det = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]);
    const i128 n1 = (x - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (y - P[0][1]);
    const i128 n2 = (P[1][0] - P[0][0]) * (y - P[0][1]) - (x - P[0][0]) * (P[1][1] - P[0][1]);
    if (n1 > 0 && n2 > 0 && det - n1 - n2 > 0) {
      out = kt;
      return true;
    }
  }
  return false;
}

// R17: Dirichlet auxiliary grids (Sec. 3.4, Def. "Dirichlet auxiliary grids")
// for a domain that does not fill the root box.  T^D_l keeps the triangles of
// sigma^(l) inside Omega: the fine elements cover at least (1 - 1e-9) of their
// area.  Coverage of the level-J triangles is clipped exactly; a coarser
// triangle's coverage is the sum over the level-J triangles nested in it (found
// by their centroids).  Returns, per level, the inside triangles.
void dirichlet_triangles(Oracle& o, std::vector<std::vector<std::array<uint64_t, 3>>>& inside) {
  const int J = o.J;
  std::vector<std::array<uint64_t, 3>> tJ;
  level_triangles(o, J, tJ);
  std::map<std::array<uint64_t, 3>, int64_t> idx;
  for (size_t t = 0; t < tJ.size(); ++t) idx[tJ[t]] = (int64_t)t;
  std::vector<double> cov(tJ.size(), 0.0);
  std::vector<std::array<uint64_t, 3>> leaves, ktri;
  for (int64_t e = 0; e < o.ne; ++e) {
    Pt T[3];
    for (int k = 0; k < 3; ++k) T[k] = Pt{o.X[(int64_t)o.E[3 * e + k] * 2], o.X[(int64_t)o.E[3 * e + k] * 2 + 1]};
    double lox = std::min({T[0].x, T[1].x, T[2].x}), hix = std::max({T[0].x, T[1].x, T[2].x});
    double loy = std::min({T[0].y, T[1].y, T[2].y}), hiy = std::max({T[0].y, T[1].y, T[2].y});
    leaves.clear();
    leaves_overlapping(o, lox, loy, hix, hiy, leaves);
    std::vector<Pt> poly(T, T + 3);
    for (auto& b : leaves) {
      ktri.clear();
      box_triangles(o, (int)b[0], b[1], b[2], J, ktri);
      for (auto& kt : ktri) {
        Pt K[3];
        for (int k = 0; k < 3; ++k) {
          double p[2];
          physical(o, kt[k], p);
          K[k] = Pt{p[0], p[1]};
        }
        auto cp = clip(poly, K);
        if (cp.size() < 3) continue;
        cov[idx.at(kt)] += poly_area(cp);
      }
    }
  }
  auto area_of = [&](const std::array<uint64_t, 3>& t) {
    double p0[2], p1[2], p2[2];
    physical(o, t[0], p0);
    physical(o, t[1], p1);
    physical(o, t[2], p2);
    return 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]));
  };
  inside.assign(J + 1, {});
  for (int l = 0; l <= J; ++l) {
    std::vector<std::array<uint64_t, 3>> tl;
    level_triangles(o, l, tl);
    std::map<std::array<uint64_t, 3>, double> cl;
    if (l == J) {
      for (size_t t = 0; t < tJ.size(); ++t) cl[tJ[t]] = cov[t];
    } else {
      for (size_t t = 0; t < tJ.size(); ++t) {
        uint64_t X3 = 0, Y3 = 0;
        for (int v = 0; v < 3; ++v) {
          uint64_t x, y;
          node_xy(tJ[t][v], x, y);
          X3 += x;
          Y3 += y;
        }
        std::array<uint64_t, 3> anc;
        if (!locate_level_triangle(o, l, X3, Y3, anc)) {
          o.err = "oracle: nested triangle not located";
          return;
        }
        cl[anc] += cov[t];
      }
    }
    for (auto& t : tl)
      if (cl[t] >= (1.0 - 1e-9) * area_of(t)) inside[l].push_back(t);
  }
}

bool cholesky(std::vector<double>& M, int64_t n);
void chol_solve(const std::vector<double>& Lm, int64_t n, const double* b, double* x);

// Orientation of r against the directed line p -> q (twice the signed area).
double orient2(const Pt& p, const Pt& q, const Pt& r) {
  return (q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - p.x);
}

// r on the closed segment [p, q] (orientation zero and inside the bounding box)
bool on_segment(const Pt& p, const Pt& q, const Pt& r) {
  return orient2(p, q, r) == 0 && std::min(p.x, q.x) <= r.x && r.x <= std::max(p.x, q.x) &&
         std::min(p.y, q.y) <= r.y && r.y <= std::max(p.y, q.y);
}

// The closed segment [a, b] meets the interior of the CCW triangle K.  By
// orientation signs: a segment on an edge's line cannot; an endpoint strictly
// inside does; two endpoints in the closed triangle do when their midpoint is
// strictly inside; otherwise the segment must cross an edge at an interior
// point of both, or pass through a vertex between the other two.
bool seg_meets_open_triangle(const Pt& a, const Pt& b, const Pt* K) {
  double oa[3], ob[3];
  for (int e = 0; e < 3; ++e) {
    oa[e] = orient2(K[e], K[(e + 1) % 3], a);
    ob[e] = orient2(K[e], K[(e + 1) % 3], b);
    if (oa[e] == 0 && ob[e] == 0) return false;
  }
  const bool ina = oa[0] >= 0 && oa[1] >= 0 && oa[2] >= 0, inb = ob[0] >= 0 && ob[1] >= 0 && ob[2] >= 0;
  if ((oa[0] > 0 && oa[1] > 0 && oa[2] > 0) || (ob[0] > 0 && ob[1] > 0 && ob[2] > 0)) return true;
  if (ina && inb) return oa[0] + ob[0] > 0 && oa[1] + ob[1] > 0 && oa[2] + ob[2] > 0;
  for (int e = 0; e < 3; ++e) {
    const Pt &p = K[e], &q = K[(e + 1) % 3];
    const double dp = orient2(a, b, p), dq = orient2(a, b, q);
    if (((oa[e] > 0 && ob[e] < 0) || (oa[e] < 0 && ob[e] > 0)) && ((dp > 0 && dq < 0) || (dp < 0 && dq > 0)))
      return true;
  }
  for (int v = 0; v < 3; ++v) {
    const Pt &r = K[v], &p = K[(v + 1) % 3], &q = K[(v + 2) % 3];
    if (!on_segment(a, b, r) || (r.x == a.x && r.y == a.y) || (r.x == b.x && r.y == b.y)) continue;
    const double dp = orient2(a, b, p), dq = orient2(a, b, q);
    if ((dp > 0 && dq < 0) || (dp < 0 && dq > 0)) return true;
  }
  return false;
}

// R18: mixed Dirichlet / Neumann boundaries (Sec. 3.4, the remark on mixed
// boundary conditions), 2D.  Gamma_D is the union of the fine boundary edges
// (edges of one element) whose two endpoints are Dirichlet.  T^M_l keeps the
// triangles of sigma^(l) whose interior meets Omega (positive covered area)
// and does not meet Gamma_D.  The Dirichlet nodes of level l are the nodes of
// kept triangles that lie on Gamma_D or belong to a triangle removed for
// Gamma_D; every other node of T^M_l is free (natural conditions on the rest
// of the boundary of Omega^M_l).  The grids are not nested, so every level is
// its own P1 discretisation with the mean of a over tau n Omega; the transfer
// between levels is nodal interpolation (zero where the coarse function has no
// kept triangle), every level is smoothed as a whole, and Algorithm 3 adds the
// near-boundary correction (R19).
void build_aux_mixed(Oracle& o) {
  const int J = o.J;
  o.lv.assign(J + 1, Level());
  std::vector<std::array<uint64_t, 3>> tJ;
  level_triangles(o, J, tJ);
  std::map<std::array<uint64_t, 3>, int64_t> idx;
  for (size_t t = 0; t < tJ.size(); ++t) idx[tJ[t]] = (int64_t)t;
  // covered area and integral of a over tau n Omega (exact clipping)
  std::vector<double> cov(tJ.size(), 0.0), num(tJ.size(), 0.0);
  std::vector<std::array<uint64_t, 3>> leaves, ktri;
  auto tri_pts = [&](const std::array<uint64_t, 3>& kt, Pt* K) {
    for (int k = 0; k < 3; ++k) {
      double p[2];
      physical(o, kt[k], p);
      K[k] = Pt{p[0], p[1]};
    }
  };
  for (int64_t e = 0; e < o.ne; ++e) {
    Pt T[3];
    for (int k = 0; k < 3; ++k) T[k] = Pt{o.X[(int64_t)o.E[3 * e + k] * 2], o.X[(int64_t)o.E[3 * e + k] * 2 + 1]};
    const double lox = std::min({T[0].x, T[1].x, T[2].x}), hix = std::max({T[0].x, T[1].x, T[2].x});
    const double loy = std::min({T[0].y, T[1].y, T[2].y}), hiy = std::max({T[0].y, T[1].y, T[2].y});
    leaves.clear();
    leaves_overlapping(o, lox, loy, hix, hiy, leaves);
    const double a = o.coeff.empty() ? 1.0 : o.coeff[e];
    std::vector<Pt> poly(T, T + 3);
    for (auto& b : leaves) {
      ktri.clear();
      box_triangles(o, (int)b[0], b[1], b[2], J, ktri);
      for (auto& kt : ktri) {
        Pt K[3];
        tri_pts(kt, K);
        auto cp = clip(poly, K);
        if (cp.size() < 3) continue;
        const double ar = poly_area(cp);
        cov[idx.at(kt)] += ar;
        num[idx.at(kt)] += a * ar;
      }
    }
  }
  // Gamma_D: fine boundary edges (of one element only) with Dirichlet endpoints
  std::map<std::pair<int32_t, int32_t>, int> ecount;
  for (int64_t e = 0; e < o.ne; ++e)
    for (int k = 0; k < 3; ++k) {
      int32_t a = o.E[3 * e + k], b = o.E[3 * e + (k + 1) % 3];
      ecount[{std::min(a, b), std::max(a, b)}] += 1;
    }
  std::vector<std::array<Pt, 2>> gamma_d;
  for (auto& kv : ecount)
    if (kv.second == 1 && o.bflag[kv.first.first] == 1 && o.bflag[kv.first.second] == 1)
      gamma_d.push_back({Pt{o.X[2 * (int64_t)kv.first.first], o.X[2 * (int64_t)kv.first.first + 1]},
                         Pt{o.X[2 * (int64_t)kv.first.second], o.X[2 * (int64_t)kv.first.second + 1]}});
  auto area_of = [&](const std::array<uint64_t, 3>& t) {
    Pt K[3];
    tri_pts(t, K);
    return 0.5 * ((K[1].x - K[0].x) * (K[2].y - K[0].y) - (K[2].x - K[0].x) * (K[1].y - K[0].y));
  };
  // every level: kept triangles, their coefficients, free nodes
  std::vector<std::vector<double>> coef(J + 1);
  for (int l = 0; l <= J; ++l) {
    std::vector<std::array<uint64_t, 3>> tl;
    level_triangles(o, l, tl);
    std::map<std::array<uint64_t, 3>, double> cl, nl;
    for (size_t t = 0; t < tJ.size(); ++t) {
      std::array<uint64_t, 3> anc = tJ[t];
      if (l < J) {
        uint64_t X3 = 0, Y3 = 0;
        for (int v = 0; v < 3; ++v) {
          uint64_t x, y;
          node_xy(tJ[t][v], x, y);
          X3 += x;
          Y3 += y;
        }
        if (!locate_level_triangle(o, l, X3, Y3, anc)) {
          o.err = "oracle: nested triangle not located";
          return;
        }
      }
      cl[anc] += cov[t];
      nl[anc] += num[t];
    }
    Level& L = o.lv[l];
    // Dirichlet nodes: those of triangles whose interior meets Gamma_D, and
    // those lying on Gamma_D
    std::set<uint64_t> dirn;
    for (auto& t : tl) {
      Pt K[3];
      tri_pts(t, K);
      bool hit = false;
      for (auto& sg : gamma_d) hit = hit || seg_meets_open_triangle(sg[0], sg[1], K);
      if (hit) {
        for (int v = 0; v < 3; ++v) dirn.insert(t[v]);
        continue;
      }
      if (!(cl[t] > 1e-12 * area_of(t))) continue;  // outside Omega
      L.tri.push_back(t);
      coef[l].push_back(nl[t] / cl[t]);
    }
    for (auto& t : L.tri)
      for (int k = 0; k < 3; ++k) L.allkey.push_back(t[k]);
    std::sort(L.allkey.begin(), L.allkey.end());
    L.allkey.erase(std::unique(L.allkey.begin(), L.allkey.end()), L.allkey.end());
    for (auto k : L.allkey) {
      double p[2];
      physical(o, k, p);
      bool ond = false;
      for (auto& sg : gamma_d) ond = ond || on_segment(sg[0], sg[1], Pt{p[0], p[1]});
      if (!dirn.count(k) && !ond) L.key.push_back(k);
    }
  }
  o.c = 0;
  for (int l = 0; l <= J; ++l)
    if ((int64_t)o.lv[l].key.size() <= o.prm.coarse_max) o.c = l;
  o.finest_coef = coef[J];
  // every level's own P1 stiffness
  for (int l = o.c; l <= J; ++l) {
    Level& L = o.lv[l];
    std::vector<std::vector<std::pair<int32_t, double>>> rows(L.key.size());
    for (size_t t = 0; t < L.tri.size(); ++t) {
      double p[3][2];
      int32_t id[3];
      for (int k = 0; k < 3; ++k) {
        physical(o, L.tri[t][k], p[k]);
        id[k] = find_index(L.key, L.tri[t][k]);
      }
      double K[3][3];
      tri_stiffness(p[0], p[1], p[2], K);
      for (int i = 0; i < 3; ++i)
        if (id[i] >= 0)
          for (int j = 0; j < 3; ++j)
            if (id[j] >= 0) rows[id[i]].push_back({id[j], coef[l][t] * K[i][j]});
    }
    L.A = csr_from_rows(L.key.size(), L.key.size(), rows);
  }
  // nodal interpolation from level l-1: the coarse function on its kept
  // triangles, zero outside them and at its Dirichlet nodes
  for (int l = std::max(1, o.c + 1); l <= J; ++l) {
    Level& Lf = o.lv[l];
    Level& Lc = o.lv[l - 1];
    std::set<std::array<uint64_t, 3>> kept(Lc.tri.begin(), Lc.tri.end());
    std::vector<std::vector<std::pair<int32_t, double>>> rows(Lf.key.size());
    for (size_t k = 0; k < Lf.key.size(); ++k) {
      const int32_t j = find_index(Lc.key, Lf.key[k]);
      if (j >= 0) {
        rows[k].push_back({j, 1.0});
        continue;
      }
      uint64_t x, y;
      node_xy(Lf.key[k], x, y);
      // every box shown at level l-1 whose closed square holds the point; the
      // first kept triangle containing it gives the coarse function's value
      // (the same in every kept triangle that contains it)
      std::vector<std::array<uint64_t, 3>> hold, stack;
      stack.push_back({0, 0, 0});
      while (!stack.empty()) {
        const auto b = stack.back();
        stack.pop_back();
        const int depth = (int)b[0];
        const uint64_t s = 1ULL << (o.D - depth);
        if (x < b[1] * s || x > (b[1] + 1) * s || y < b[2] * s || y > (b[2] + 1) * s) continue;
        uint64_t q[2] = {b[1], b[2]};
        uint8_t sp = 0;
        if (!box_exists(o, depth, q, &sp)) continue;
        if (depth == l - 1 || !sp) {
          hold.push_back(b);
          continue;
        }
        for (uint64_t ch = 0; ch < 4; ++ch)
          stack.push_back({(uint64_t)depth + 1, 2 * b[1] + (ch & 1), 2 * b[2] + (ch >> 1)});
      }
      bool found = false;
      for (const auto& b : hold) {
        if (found) break;
        std::vector<std::array<uint64_t, 3>> ct;
        box_triangles(o, (int)b[0], b[1], b[2], l - 1, ct);
        for (auto& kt : ct) {
          if (!kept.count(kt)) continue;
          i128 P[3][2];
          for (int v = 0; v < 3; ++v) {
            uint64_t vx, vy;
            node_xy(kt[v], vx, vy);
            P[v][0] = (i128)vx;
            P[v][1] = (i128)vy;
          }
          const i128 det = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]);
          const i128 n1 = ((i128)x - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * ((i128)y - P[0][1]);
          const i128 n2 = (P[1][0] - P[0][0]) * ((i128)y - P[0][1]) - ((i128)x - P[0][0]) * (P[1][1] - P[0][1]);
          const i128 n0 = det - n1 - n2;
          if (n0 < 0 || n1 < 0 || n2 < 0) continue;
          const i128 nn[3] = {n0, n1, n2};
          for (int v = 0; v < 3; ++v) {
            if (nn[v] == 0) continue;
            const int32_t jj = find_index(Lc.key, kt[v]);
            if (jj >= 0) rows[k].push_back({jj, (double)((long double)nn[v] / (long double)det)});
          }
          found = true;
          break;
        }
      }
    }
    Lf.I = csr_from_rows(Lf.key.size(), Lc.key.size(), rows);
  }
  // every level smoothed as a whole; near-boundary sets of Algorithm 3
  for (int l = o.c + 1; l <= J; ++l) {
    Level& L = o.lv[l];
    L.smooth.resize(L.key.size());
    for (size_t k = 0; k < L.key.size(); ++k) L.smooth[k] = (int32_t)k;
    if (o.prm.nb_layers < 0) continue;
    // Gamma_l: endpoints of edges of one kept triangle only; layer 0 = kept
    // triangles with a vertex on Gamma_l, layer i = those with a vertex in layer i-1
    std::map<std::pair<uint64_t, uint64_t>, int> edges;
    for (auto& t : L.tri)
      for (int k = 0; k < 3; ++k) edges[{std::min(t[k], t[(k + 1) % 3]), std::max(t[k], t[(k + 1) % 3])}] += 1;
    std::set<uint64_t> verts;
    for (auto& kv : edges)
      if (kv.second == 1) {
        verts.insert(kv.first.first);
        verts.insert(kv.first.second);
      }
    std::set<uint64_t> layer;
    for (int i = 0; i <= o.prm.nb_layers; ++i) {
      layer.clear();
      for (auto& t : L.tri)
        if (verts.count(t[0]) || verts.count(t[1]) || verts.count(t[2]))
          for (int k = 0; k < 3; ++k) layer.insert(t[k]);
      if (layer == verts) break;
      verts = layer;
    }
    for (auto k : verts) {
      const int32_t id = find_index(L.key, k);
      if (id >= 0) L.nbset.push_back(id);
    }
    std::sort(L.nbset.begin(), L.nbset.end());
    const int64_t m = (int64_t)L.nbset.size();
    L.nbchol.assign(m * m, 0.0);
    for (int64_t a = 0; a < m; ++a)
      for (int64_t b = 0; b < m; ++b) L.nbchol[a * m + b] = L.A.get(L.nbset[a], L.nbset[b]);
    if (m && !cholesky(L.nbchol, m)) {
      o.err = "oracle: near-boundary block not positive definite";
      return;
    }
  }
}

void build_aux(Oracle& o) {
  for (int64_t v = 0; v < o.nv; ++v) o.neumann = o.neumann || o.bflag[v] == 2;
  if (o.neumann) {
    build_aux_mixed(o);
    return;
  }
  const int J = o.J;
  o.lv.assign(J + 1, Level());
  // does the domain fill the root box?
  {
    double area = 0.0;
    for (int64_t e = 0; e < o.ne; ++e) {
      const double* p0 = &o.X[(int64_t)o.E[3 * e] * 2];
      const double* p1 = &o.X[(int64_t)o.E[3 * e + 1] * 2];
      const double* p2 = &o.X[(int64_t)o.E[3 * e + 2] * 2];
      area += 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]));
    }
    o.boxdomain = std::fabs(area - o.L * o.L) <= 1e-12 * o.L * o.L;
  }
  std::vector<std::vector<std::array<uint64_t, 3>>> inside;
  if (!o.boxdomain) {
    dirichlet_triangles(o, inside);
    if (!o.err.empty()) return;
  }
  for (int l = 0; l <= J; ++l) {
    Level& L = o.lv[l];
    if (o.boxdomain)
      level_triangles(o, l, L.tri);
    else
      L.tri = inside[l];
    for (auto& t : L.tri)
      for (int k = 0; k < 3; ++k) L.allkey.push_back(t[k]);
    std::sort(L.allkey.begin(), L.allkey.end());
    L.allkey.erase(std::unique(L.allkey.begin(), L.allkey.end()), L.allkey.end());
    if (o.boxdomain) {
      for (auto k : L.allkey)
        if (!on_boundary(o, k)) L.key.push_back(k);
    } else {
      // Gamma_l = boundary of the union of T^D_l: endpoints of edges that
      // belong to one triangle only
      std::map<std::pair<uint64_t, uint64_t>, int> edges;
      for (auto& t : L.tri)
        for (int k = 0; k < 3; ++k) {
          uint64_t a = t[k], b = t[(k + 1) % 3];
          edges[{std::min(a, b), std::max(a, b)}] += 1;
        }
      std::set<uint64_t> gamma;
      for (auto& kv : edges)
        if (kv.second == 1) {
          gamma.insert(kv.first.first);
          gamma.insert(kv.first.second);
        }
      for (auto k : L.allkey)
        if (!gamma.count(k)) L.key.push_back(k);
    }
  }
  // coarsest level used: the finest level with at most coarse_max free nodes
  o.c = 0;
  for (int l = 0; l <= J; ++l)
    if ((int64_t)o.lv[l].key.size() <= o.prm.coarse_max) o.c = l;

  // Finest auxiliary coefficient (R6) by exact clipping of every fine element
  // against the level-J triangles of the leaf boxes it meets.
  Level& LJ = o.lv[J];
  std::map<std::array<uint64_t, 3>, int64_t> tri_index;
  for (size_t t = 0; t < LJ.tri.size(); ++t) tri_index[LJ.tri[t]] = (int64_t)t;
  std::vector<double> num(LJ.tri.size(), 0.0);
  std::vector<std::array<uint64_t, 3>> leaves, ktri;
  for (int64_t e = 0; e < o.ne; ++e) {
    Pt T[3];
    for (int k = 0; k < 3; ++k) T[k] = Pt{o.X[(int64_t)o.E[3 * e + k] * 2], o.X[(int64_t)o.E[3 * e + k] * 2 + 1]};
    double lox = std::min({T[0].x, T[1].x, T[2].x}), hix = std::max({T[0].x, T[1].x, T[2].x});
    double loy = std::min({T[0].y, T[1].y, T[2].y}), hiy = std::max({T[0].y, T[1].y, T[2].y});
    leaves.clear();
    leaves_overlapping(o, lox, loy, hix, hiy, leaves);
    double a = o.coeff.empty() ? 1.0 : o.coeff[e];
    std::vector<Pt> poly(T, T + 3);
    for (auto& b : leaves) {
      ktri.clear();
      box_triangles(o, (int)b[0], b[1], b[2], J, ktri);
      for (auto& kt : ktri) {
        Pt K[3];
        for (int k = 0; k < 3; ++k) {
          double p[2];
          physical(o, kt[k], p);
          K[k] = Pt{p[0], p[1]};
        }
        auto cp = clip(poly, K);
        if (cp.size() < 3) continue;
        auto it = tri_index.find(kt);
        if (it == tri_index.end()) continue;  // outside Omega (not in T^D_J)
        num[it->second] += a * poly_area(cp);
      }
    }
  }
  o.finest_coef.resize(LJ.tri.size());
  for (size_t t = 0; t < LJ.tri.size(); ++t) {
    double p0[2], p1[2], p2[2];
    physical(o, LJ.tri[t][0], p0);
    physical(o, LJ.tri[t][1], p1);
    physical(o, LJ.tri[t][2], p2);
    double area = 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]));
    o.finest_coef[t] = num[t] / area;
  }

  // A_J: P1 stiffness of T_J with the averaged coefficient (Sec. 4.1: the
  // auxiliary operator comes from the bilinear form).
  {
    std::vector<std::vector<std::pair<int32_t, double>>> rows(LJ.key.size());
    for (size_t t = 0; t < LJ.tri.size(); ++t) {
      double p[3][2];
      int32_t id[3];
      for (int k = 0; k < 3; ++k) {
        physical(o, LJ.tri[t][k], p[k]);
        id[k] = find_index(LJ.key, LJ.tri[t][k]);
      }
      double K[3][3];
      tri_stiffness(p[0], p[1], p[2], K);
      for (int i = 0; i < 3; ++i)
        if (id[i] >= 0)
          for (int j = 0; j < 3; ++j)
            if (id[j] >= 0) rows[id[i]].push_back({id[j], o.finest_coef[t] * K[i][j]});
    }
    LJ.A = csr_from_rows(LJ.key.size(), LJ.key.size(), rows);
  }

  // Interpolation I_l: nodal interpolation of the level l-1 P1 function at
  // the level-l nodes (nested spaces, Sec. 3.3).
  for (int l = std::max(1, o.c + 1); l <= J; ++l) {
    Level& Lf = o.lv[l];
    Level& Lc = o.lv[l - 1];
    std::vector<std::vector<std::pair<int32_t, double>>> rows(Lf.key.size());
    for (size_t k = 0; k < Lf.key.size(); ++k) {
      int32_t j = find_index(Lc.key, Lf.key[k]);
      if (j >= 0) {
        rows[k].push_back({j, 1.0});
        continue;
      }
      uint64_t x, y;
      node_xy(Lf.key[k], x, y);
      // descend the truncated tree to the level-(l-1) leaf box containing the node
      int depth = 0;
      uint64_t bx = 0, by = 0;
      for (;;) {
        uint64_t q[2] = {bx, by};
        uint8_t sp = 0;
        box_exists(o, depth, q, &sp);
        if (depth == l - 1 || !sp) break;
        uint64_t half = 1ULL << (o.D - depth - 1);
        uint64_t cx = (x - bx * (2 * half)) >= half ? 1 : 0;
        uint64_t cy = (y - by * (2 * half)) >= half ? 1 : 0;
        // points on the far edge of the root box stay in the last child
        if (x == (bx + 1) * 2 * half) cx = 1;
        if (y == (by + 1) * 2 * half) cy = 1;
        bx = 2 * bx + cx;
        by = 2 * by + cy;
        ++depth;
      }
      std::vector<std::array<uint64_t, 3>> ktri;
      box_triangles(o, depth, bx, by, l - 1, ktri);
      bool found = false;
      for (auto& kt : ktri) {
        i128 P[3][2];
        for (int v = 0; v < 3; ++v) {
          uint64_t vx, vy;
          node_xy(kt[v], vx, vy);
          P[v][0] = (i128)vx;
          P[v][1] = (i128)vy;
        }
        i128 det = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]);
        i128 n1 = ((i128)x - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * ((i128)y - P[0][1]);
        i128 n2 = (P[1][0] - P[0][0]) * ((i128)y - P[0][1]) - ((i128)x - P[0][0]) * (P[1][1] - P[0][1]);
        i128 n0 = det - n1 - n2;
        if (n0 < 0 || n1 < 0 || n2 < 0) continue;
        i128 nn[3] = {n0, n1, n2};
        for (int v = 0; v < 3; ++v) {
          if (nn[v] == 0) continue;
          int32_t jj = find_index(Lc.key, kt[v]);
          if (jj < 0) continue;  // Dirichlet vertex: value 0
          rows[k].push_back({jj, (double)((long double)nn[v] / (long double)det)});
        }
        found = true;
        break;
      }
      if (!found) {
        o.err = "oracle: interpolation point not located";
        return;
      }
    }
    Lf.I = csr_from_rows(Lf.key.size(), Lc.key.size(), rows);
  }

  // Galerkin coarse operators A_{l-1} = I_l^T A_l I_l (Sec. 2.3: A_i is the
  // restriction of A to V_i).
  for (int l = J; l > o.c; --l) {
    CSR It = transpose(o.lv[l].I);
    CSR AI = matmul(o.lv[l].A, o.lv[l].I);
    o.lv[l - 1].A = matmul(It, AI);
  }

  // Smoothing sets (R7): free vertices of level-l triangles that are not
  // level-(l-1) triangles, i.e. new nodes and nodes whose hat changed.
  for (int l = o.c + 1; l <= J; ++l) {
    Level& Lf = o.lv[l];
    std::vector<int32_t> set;
    if (o.prm.smoothing == 1) {
      for (size_t k = 0; k < Lf.key.size(); ++k) set.push_back((int32_t)k);
    } else {
      std::set<std::array<uint64_t, 3>> prev;
      for (auto t : o.lv[l - 1].tri) {
        std::sort(t.begin(), t.end());
        prev.insert(t);
      }
      std::vector<uint8_t> mark(Lf.key.size(), 0);
      for (auto t : Lf.tri) {
        auto ts = t;
        std::sort(ts.begin(), ts.end());
        if (prev.count(ts)) continue;
        for (int v = 0; v < 3; ++v) {
          int32_t id = find_index(Lf.key, t[v]);
          if (id >= 0) mark[id] = 1;
        }
      }
      for (size_t k = 0; k < Lf.key.size(); ++k)
        if (mark[k]) set.push_back((int32_t)k);
    }
    Lf.smooth = set;
  }
}

// --------------------------------------------------------------------------
// Scott-Zhang transfer (Sec. 4.1, R5): P_ik = int_{sigma_i} psi_i phi^J_k.
// --------------------------------------------------------------------------

void build_transfer(Oracle& o) {
  const Level& LJ = o.lv[o.J];
  const int64_t n = o.vertex_of_free.size();
  std::vector<int32_t> sigma(o.nv, -1);
  for (int64_t e = 0; e < o.ne; ++e)
    for (int k = 0; k < 3; ++k) {
      int32_t v = o.E[3 * e + k];
      if (sigma[v] < 0) sigma[v] = (int32_t)e;  // elements visited in index order
    }
  std::vector<std::vector<std::pair<int32_t, double>>> rows(n), rows_full(n);
  std::vector<std::array<uint64_t, 3>> leaves, ktri;
  std::set<std::array<uint64_t, 3>> tri_in(LJ.tri.begin(), LJ.tri.end());
  for (int64_t i = 0; i < n; ++i) {
    int32_t v = o.vertex_of_free[i];
    int32_t e = sigma[v];
    Pt T[3];
    int loc = -1;
    for (int k = 0; k < 3; ++k) {
      int32_t vk = o.E[3 * (int64_t)e + k];
      T[k] = Pt{o.X[(int64_t)vk * 2], o.X[(int64_t)vk * 2 + 1]};
      if (vk == v) loc = k;
    }
    double area = 0.5 * ((T[1].x - T[0].x) * (T[2].y - T[0].y) - (T[2].x - T[0].x) * (T[1].y - T[0].y));
    double lox = std::min({T[0].x, T[1].x, T[2].x}), hix = std::max({T[0].x, T[1].x, T[2].x});
    double loy = std::min({T[0].y, T[1].y, T[2].y}), hiy = std::max({T[0].y, T[1].y, T[2].y});
    leaves.clear();
    leaves_overlapping(o, lox, loy, hix, hiy, leaves);
    std::vector<Pt> poly(T, T + 3);
    for (auto& b : leaves) {
      ktri.clear();
      box_triangles(o, (int)b[0], b[1], b[2], o.J, ktri);
      for (auto& kt : ktri) {
        if ((!o.boxdomain || o.neumann) && !tri_in.count(kt)) continue;  // hats only on the kept triangles
        Pt K[3];
        for (int k = 0; k < 3; ++k) {
          double p[2];
          physical(o, kt[k], p);
          K[k] = Pt{p[0], p[1]};
        }
        auto cp = clip(poly, K);
        if (cp.size() < 3) continue;
        for (size_t s = 1; s + 1 < cp.size(); ++s) {
          Pt q[3] = {cp[0], cp[s], cp[s + 1]};
          double ta = 0.5 * ((q[1].x - q[0].x) * (q[2].y - q[0].y) - (q[2].x - q[0].x) * (q[1].y - q[0].y));
          // edge-midpoint rule: exact for the quadratic psi_i * phi_k
          double acc[3] = {0, 0, 0};
          for (int m = 0; m < 3; ++m) {
            Pt mid{0.5 * (q[m].x + q[(m + 1) % 3].x), 0.5 * (q[m].y + q[(m + 1) % 3].y)};
            double ls[3], lk[3];
            bary(T, mid, ls);
            bary(K, mid, lk);
            double psi = (12.0 * ls[loc] - 3.0) / area;
            for (int k = 0; k < 3; ++k) acc[k] += psi * lk[k];
          }
          for (int k = 0; k < 3; ++k) {
            double val = ta * acc[k] / 3.0;
            int32_t jf = find_index(LJ.allkey, kt[k]);
            rows_full[i].push_back({jf, val});
            int32_t jj = find_index(LJ.key, kt[k]);
            if (jj >= 0) rows[i].push_back({jj, val});
          }
        }
      }
    }
  }
  o.P = csr_from_rows(n, LJ.key.size(), rows);
  o.Pfull = csr_from_rows(n, LJ.allkey.size(), rows_full);
}

// --------------------------------------------------------------------------
// 3D (Sec. 1: the octree version "without intrinsic difficulties"): nested
// conforming tetrahedral auxiliary grids.  Reading R4-3D: a box without edge
// midpoints or subdivided faces is split into the 6 Kuhn tetrahedra of its
// (0,0,0)-(1,1,1) diagonal; otherwise every face is triangulated -- a face
// whose neighbour is split by its 4 sub-squares, each along its
// min-to-max diagonal; a face with an edge midpoint by a fan about its
// centre; other faces by their min-to-max diagonal -- and each face triangle
// is coned to the box centre.  Nodes lie on the 2^(J+1) lattice of the root
// cube and are named by their 63-bit Morton key.
// --------------------------------------------------------------------------

uint64_t key3(uint64_t x, uint64_t y, uint64_t z) {
  uint64_t q[3] = {x, y, z};
  return interleave(q, 3, 21);
}

void xyz3(uint64_t key, uint64_t* q) { deinterleave(key, 3, 21, q); }

bool on_boundary3(const Oracle& o, uint64_t key) {
  uint64_t q[3];
  xyz3(key, q);
  const uint64_t top = 1ULL << o.LB;
  for (int k = 0; k < 3; ++k)
    if (q[k] == 0 || q[k] == top) return true;
  return false;
}

void physical3(const Oracle& o, uint64_t key, double* p) {
  uint64_t q[3];
  xyz3(key, q);
  for (int k = 0; k < 3; ++k) p[k] = o.amin[k] + std::ldexp((double)q[k], -o.LB) * o.L;
}

i128 det3(const i128* a, const i128* b, const i128* c) {
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

i128 orient3(const std::array<uint64_t, 4>& t) {
  i128 P[4][3];
  for (int v = 0; v < 4; ++v) {
    uint64_t q[3];
    xyz3(t[v], q);
    for (int k = 0; k < 3; ++k) P[v][k] = (i128)q[k];
  }
  i128 a[3], b[3], c[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = P[1][k] - P[0][k];
    b[k] = P[2][k] - P[0][k];
    c[k] = P[3][k] - P[0][k];
  }
  return det3(a, b, c);
}

bool split3(const Oracle& o, int depth, const int64_t* q) {
  const int64_t nb = 1LL << depth;
  uint64_t u[3];
  for (int k = 0; k < 3; ++k) {
    if (q[k] < 0 || q[k] >= nb) return false;
    u[k] = (uint64_t)q[k];
  }
  uint8_t sp = 0;
  return box_exists(o, depth, u, &sp) && sp;
}

// Tetrahedra of box (depth, q) as seen at level lvl.
void box_tets(const Oracle& o, int depth, const uint64_t* q, int lvl, std::vector<std::array<uint64_t, 4>>& out) {
  const uint64_t s = 1ULL << (o.LB - depth), h = s / 2;
  const int64_t qi[3] = {(int64_t)q[0], (int64_t)q[1], (int64_t)q[2]};
  auto pt = [&](int u0, int u1, int u2) {  // local coordinates in units of h (0..2)
    return key3(q[0] * s + u0 * h, q[1] * s + u1 * h, q[2] * s + u2 * h);
  };
  bool facesub[3][2] = {{false, false}, {false, false}, {false, false}};
  bool anyhang = false;
  // edge midpoint of the cube edge along axis e at sides (sf, sg) of the other axes
  auto edgemid = [&](int e, int f, int sf, int g, int sg) {
    if (depth >= lvl) return false;
    int64_t n1[3] = {qi[0], qi[1], qi[2]}, n2[3] = {qi[0], qi[1], qi[2]}, n3[3] = {qi[0], qi[1], qi[2]};
    (void)e;
    n1[f] += sf ? 1 : -1;
    n2[g] += sg ? 1 : -1;
    n3[f] += sf ? 1 : -1;
    n3[g] += sg ? 1 : -1;
    return split3(o, depth, n1) || split3(o, depth, n2) || split3(o, depth, n3);
  };
  if (depth < lvl) {
    for (int a = 0; a < 3; ++a)
      for (int sd = 0; sd < 2; ++sd) {
        int64_t n[3] = {qi[0], qi[1], qi[2]};
        n[a] += sd ? 1 : -1;
        facesub[a][sd] = split3(o, depth, n);
      }
    for (int e = 0; e < 3 && !anyhang; ++e) {
      int f = (e + 1) % 3, g = (e + 2) % 3;
      for (int sf = 0; sf < 2 && !anyhang; ++sf)
        for (int sg = 0; sg < 2 && !anyhang; ++sg)
          if (edgemid(e, f, sf, g, sg)) anyhang = true;
    }
  }
  auto push = [&](std::array<uint64_t, 4> t) {
    if (orient3(t) < 0) std::swap(t[2], t[3]);
    out.push_back(t);
  };
  if (!anyhang) {  // Kuhn: (0, e_a, e_a + e_b, 1)
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (auto& pm : perm) {
      int u1[3] = {0, 0, 0}, u2[3] = {0, 0, 0};
      u1[pm[0]] = 2;
      u2[pm[0]] = 2;
      u2[pm[1]] = 2;
      push({pt(0, 0, 0), pt(u1[0], u1[1], u1[2]), pt(u2[0], u2[1], u2[2]), pt(2, 2, 2)});
    }
    return;
  }
  const uint64_t C = pt(1, 1, 1);
  for (int a = 0; a < 3; ++a) {
    const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;  // in-plane axes, b < c
    for (int sd = 0; sd < 2; ++sd) {
      auto fp = [&](int ub, int uc) {
        int u[3];
        u[a] = 2 * sd;
        u[b] = ub;
        u[c] = uc;
        return pt(u[0], u[1], u[2]);
      };
      std::vector<std::array<uint64_t, 3>> tris;
      if (facesub[a][sd]) {
        for (int sb = 0; sb < 2; ++sb)
          for (int sc = 0; sc < 2; ++sc) {
            tris.push_back({fp(sb, sc), fp(sb + 1, sc), fp(sb + 1, sc + 1)});
            tris.push_back({fp(sb, sc), fp(sb + 1, sc + 1), fp(sb, sc + 1)});
          }
      } else {
        // edges of this face: along b at c = 0 / 2, along c at b = 0 / 2
        bool m_c0 = edgemid(b, a, sd, c, 0), m_c2 = edgemid(b, a, sd, c, 1);
        bool m_b0 = edgemid(c, a, sd, b, 0), m_b2 = edgemid(c, a, sd, b, 1);
        if (m_c0 || m_c2 || m_b0 || m_b2) {
          std::vector<uint64_t> ring;
          ring.push_back(fp(0, 0));
          if (m_c0) ring.push_back(fp(1, 0));
          ring.push_back(fp(2, 0));
          if (m_b2) ring.push_back(fp(2, 1));
          ring.push_back(fp(2, 2));
          if (m_c2) ring.push_back(fp(1, 2));
          ring.push_back(fp(0, 2));
          if (m_b0) ring.push_back(fp(0, 1));
          for (size_t i = 0; i < ring.size(); ++i) tris.push_back({ring[i], ring[(i + 1) % ring.size()], fp(1, 1)});
        } else {
          tris.push_back({fp(0, 0), fp(2, 0), fp(2, 2)});
          tris.push_back({fp(0, 0), fp(2, 2), fp(0, 2)});
        }
      }
      for (auto& t : tris) push({t[0], t[1], t[2], C});
    }
  }
}

void level_tets(const Oracle& o, int lvl, std::vector<std::array<uint64_t, 4>>& tet) {
  tet.clear();
  for (int depth = 0; depth <= lvl && depth < (int)o.boxes.size(); ++depth) {
    std::vector<std::pair<uint64_t, uint8_t>> bx(o.boxes[depth].begin(), o.boxes[depth].end());
    std::sort(bx.begin(), bx.end());
    for (auto& kv : bx) {
      if (depth < lvl && kv.second) continue;
      uint64_t q[3];
      unpack_box(kv.first, 3, q);
      box_tets(o, depth, q, lvl, tet);
    }
  }
}

typedef std::array<double, 3> P3;

// barycentric coordinates of x in tetrahedron T (Cramer's rule)
void bary3(const P3* T, const P3& x, double* lam) {
  double e1[3], e2[3], e3[3], r[3];
  for (int k = 0; k < 3; ++k) {
    e1[k] = T[1][k] - T[0][k];
    e2[k] = T[2][k] - T[0][k];
    e3[k] = T[3][k] - T[0][k];
    r[k] = x[k] - T[0][k];
  }
  auto det = [](const double* a, const double* b, const double* c) {
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
  };
  const double d = det(e1, e2, e3);
  lam[1] = det(r, e2, e3) / d;
  lam[2] = det(e1, r, e3) / d;
  lam[3] = det(e1, e2, r) / d;
  lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

double tet_volume(const P3& a, const P3& b, const P3& c, const P3& d) {
  double e1[3], e2[3], e3[3];
  for (int k = 0; k < 3; ++k) {
    e1[k] = b[k] - a[k];
    e2[k] = c[k] - a[k];
    e3[k] = d[k] - a[k];
  }
  return (e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
          e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) / 6.0;
}

// P1 stiffness of a tetrahedron: |T| grad lambda_i . grad lambda_j
void tet_stiffness(const P3* T, double K[4][4]) {
  double Jm[3][3];
  for (int k = 1; k <= 3; ++k)
    for (int r = 0; r < 3; ++r) Jm[r][k - 1] = T[k][r] - T[0][r];
  double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) - Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
               Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
  double inv[3][3];
  inv[0][0] = (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) / det;
  inv[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) / det;
  inv[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) / det;
  inv[1][0] = (Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2]) / det;
  inv[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) / det;
  inv[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) / det;
  inv[2][0] = (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]) / det;
  inv[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) / det;
  inv[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) / det;
  double G[4][3];
  for (int k = 0; k < 3; ++k)
    for (int r = 0; r < 3; ++r) G[k + 1][r] = inv[k][r];
  for (int r = 0; r < 3; ++r) G[0][r] = -(G[1][r] + G[2][r] + G[3][r]);
  const double vol = det / 6.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) K[i][j] = vol * (G[i][0] * G[j][0] + G[i][1] * G[j][1] + G[i][2] * G[j][2]);
}

// K cut by the four half-spaces of S, kept as a list of tetrahedra with
// signs +1 / -1 whose signed sum is the intersection.  A plane cut of one
// tetrahedron keeps (by the exact sign of each vertex's distance):
//   1 vertex inside   the corner tetrahedron at that vertex
//   3 vertices inside the tetrahedron minus the corner at the outside vertex
//   2 vertices inside the wedge between the two inside vertices, as three
//                     tetrahedra
// Every cut point lies on its edge (parameter in [0, 1]), so no tolerance is
// needed; pieces of zero volume are harmless.
struct SignedTet {
  P3 v[4];
  double sign;
};

P3 edge_point(const P3& a, const P3& b, double da, double db) {
  const double t = da / (da - db);
  return {a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1]), a[2] + t * (b[2] - a[2])};
}

void halfspace_cut(std::vector<SignedTet>& pieces, const P3& n, double c) {
  std::vector<SignedTet> kept;
  for (const SignedTet& T : pieces) {
    double d[4];
    int in[4], out[4], ni = 0, no = 0;
    for (int k = 0; k < 4; ++k) {
      d[k] = n[0] * T.v[k][0] + n[1] * T.v[k][1] + n[2] * T.v[k][2] - c;
      if (d[k] <= 0) in[ni++] = k; else out[no++] = k;
    }
    if (no == 0) {
      kept.push_back(T);
    } else if (ni == 1) {
      const int a = in[0];
      SignedTet C;
      C.v[0] = T.v[a];
      for (int k = 0; k < 3; ++k) C.v[k + 1] = edge_point(T.v[a], T.v[out[k]], d[a], d[out[k]]);
      C.sign = T.sign;
      kept.push_back(C);
    } else if (ni == 3) {
      const int o = out[0];
      SignedTet C;
      C.v[0] = T.v[o];
      for (int k = 0; k < 3; ++k) C.v[k + 1] = edge_point(T.v[o], T.v[in[k]], d[o], d[in[k]]);
      C.sign = -T.sign;
      kept.push_back(T);
      kept.push_back(C);
    } else if (ni == 2) {
      const P3 &i0 = T.v[in[0]], &i1 = T.v[in[1]];
      const P3 x00 = edge_point(i0, T.v[out[0]], d[in[0]], d[out[0]]);
      const P3 x01 = edge_point(i0, T.v[out[1]], d[in[0]], d[out[1]]);
      const P3 x10 = edge_point(i1, T.v[out[0]], d[in[1]], d[out[0]]);
      const P3 x11 = edge_point(i1, T.v[out[1]], d[in[1]], d[out[1]]);
      kept.push_back({{i0, i1, x00, x01}, T.sign});
      kept.push_back({{i1, x00, x01, x11}, T.sign});
      kept.push_back({{i1, x00, x11, x10}, T.sign});
    }
  }
  pieces.swap(kept);
}

// sigma (S) intersected with the auxiliary tetrahedron K
std::vector<SignedTet> intersect_tets(const P3* S, const P3* K) {
  std::vector<SignedTet> pieces(1);
  for (int k = 0; k < 4; ++k) pieces[0].v[k] = K[k];
  pieces[0].sign = 1.0;
  const int fc[4][4] = {{1, 2, 3, 0}, {0, 2, 3, 1}, {0, 1, 3, 2}, {0, 1, 2, 3}};  // face + opposite vertex
  for (auto& f : fc) {
    const P3 &a = S[f[0]], &b = S[f[1]], &c = S[f[2]], &d = S[f[3]];
    P3 e1 = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2 = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    P3 n = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double cc = n[0] * a[0] + n[1] * a[1] + n[2] * a[2];
    if (n[0] * d[0] + n[1] * d[1] + n[2] * d[2] > cc) {  // inside is the side of the opposite vertex
      for (int k = 0; k < 3; ++k) n[k] = -n[k];
      cc = -cc;
    }
    halfspace_cut(pieces, n, cc);
    if (pieces.empty()) break;
  }
  return pieces;
}

// int over the signed pieces of f * g for affine f, g given as evaluators;
// on a tetrahedron int f g = |T|/20 (sum_i f_i g_i + sum_i f_i sum_i g_i).
template <class F, class G>
double pieces_integral(const std::vector<SignedTet>& pieces, F f, G g) {
  double sum = 0.0;
  for (const SignedTet& T : pieces) {
    const double vol = std::fabs(tet_volume(T.v[0], T.v[1], T.v[2], T.v[3]));
    double sf = 0, sg = 0, sfg = 0;
    for (int k = 0; k < 4; ++k) {
      const double fv = f(T.v[k]), gv = g(T.v[k]);
      sf += fv;
      sg += gv;
      sfg += fv * gv;
    }
    sum += T.sign * vol / 20.0 * (sfg + sf * sg);
  }
  return sum;
}

void leaves_overlapping3(const Oracle& o, const double* lo, const double* hi, std::vector<std::array<uint64_t, 4>>& out) {
  std::vector<std::array<uint64_t, 4>> st;
  st.push_back({0, 0, 0, 0});
  while (!st.empty()) {
    auto b = st.back();
    st.pop_back();
    int depth = (int)b[0];
    double w = std::ldexp(o.L, -depth);
    bool meet = true;
    for (int k = 0; k < 3; ++k) {
      double x0 = o.amin[k] + (double)b[1 + k] * w;
      if (x0 > hi[k] || x0 + w < lo[k]) meet = false;
    }
    if (!meet) continue;
    uint64_t q[3] = {b[1], b[2], b[3]};
    uint8_t sp = 0;
    if (!box_exists(o, depth, q, &sp)) continue;
    if (!sp) {
      out.push_back(b);
      continue;
    }
    for (int ch = 0; ch < 8; ++ch)
      st.push_back({(uint64_t)depth + 1, 2 * b[1] + (ch & 1), 2 * b[2] + ((ch >> 1) & 1), 2 * b[3] + (ch >> 2)});
  }
}

void tet_points(const Oracle& o, const std::array<uint64_t, 4>& t, P3* K) {
  for (int v = 0; v < 4; ++v) {
    double p[3];
    physical3(o, t[v], p);
    K[v] = {p[0], p[1], p[2]};
  }
}

// The tetrahedron of sigma^(l) containing the point (X4/4) (lattice units,
// per axis): descend the truncated octree to the level-l box holding it,
// then test its tetrahedra with integer barycentric coordinates.  The point
// must lie strictly inside a tetrahedron (a centroid of a finer nested one).
bool locate_level_tet(const Oracle& o, int l, const uint64_t* X4, std::array<uint64_t, 4>& out) {
  int depth = 0;
  uint64_t bq[3] = {0, 0, 0};
  for (;;) {
    uint8_t sp = 0;
    box_exists(o, depth, bq, &sp);
    if (depth == l || !sp) break;
    const uint64_t half4 = 4 * (1ULL << (o.LB - depth - 1));
    for (int d = 0; d < 3; ++d) bq[d] = 2 * bq[d] + ((X4[d] - bq[d] * 2 * half4) >= half4 ? 1 : 0);
    ++depth;
  }
  std::vector<std::array<uint64_t, 4>> tets;
  box_tets(o, depth, bq, l, tets);
  for (auto& t : tets) {
    i128 P[4][3];
    for (int v = 0; v < 4; ++v) {
      uint64_t q[3];
      xyz3(t[v], q);
      for (int d = 0; d < 3; ++d) P[v][d] = 4 * (i128)q[d];
    }
    i128 e1[3], e2[3], e3[3], r[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = P[1][d] - P[0][d];
      e2[d] = P[2][d] - P[0][d];
      e3[d] = P[3][d] - P[0][d];
      r[d] = (i128)X4[d] - P[0][d];
    }
    const i128 det = det3(e1, e2, e3);
    const i128 n1 = det3(r, e2, e3), n2 = det3(e1, r, e3), n3 = det3(e1, e2, r);
    const i128 n0 = det - n1 - n2 - n3;
    // same sign as det for all four: strictly inside
    if ((det > 0 && n0 > 0 && n1 > 0 && n2 > 0 && n3 > 0) || (det < 0 && n0 < 0 && n1 < 0 && n2 < 0 && n3 < 0)) {
      out = t;
      return true;
    }
  }
  return false;
}

// R17 in 3D: T^D_l keeps the tetrahedra of sigma^(l) that the fine elements
// cover to at least (1 - 1e-9) of their volume.  The coverage of the level-J
// tetrahedra is the exact intersection volume with the fine elements; a
// coarser tetrahedron's coverage is the sum over the level-J tetrahedra
// nested in it (found by their centroids).
void dirichlet_tets(Oracle& o, std::vector<std::vector<std::array<uint64_t, 4>>>& inside) {
  const int J = o.J;
  std::vector<std::array<uint64_t, 4>> tJ;
  level_tets(o, J, tJ);
  std::map<std::array<uint64_t, 4>, int64_t> idx;
  for (size_t t = 0; t < tJ.size(); ++t) idx[tJ[t]] = (int64_t)t;
  std::vector<double> cov(tJ.size(), 0.0);
  std::vector<std::array<uint64_t, 4>> leaves, kt;
  for (int64_t e = 0; e < o.ne; ++e) {
    P3 T[4];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < 4; ++v)
      for (int k = 0; k < 3; ++k) {
        T[v][k] = o.X[(int64_t)o.E[4 * e + v] * 3 + k];
        lo[k] = std::min(lo[k], T[v][k]);
        hi[k] = std::max(hi[k], T[v][k]);
      }
    leaves.clear();
    leaves_overlapping3(o, lo, hi, leaves);
    for (auto& b : leaves) {
      kt.clear();
      uint64_t q[3] = {b[1], b[2], b[3]};
      box_tets(o, (int)b[0], q, J, kt);
      for (auto& k4 : kt) {
        P3 K[4];
        tet_points(o, k4, K);
        std::vector<SignedTet> P = intersect_tets(T, K);
        if (P.empty()) continue;
        cov[idx.at(k4)] += pieces_integral(P, [](const P3&) { return 1.0; }, [](const P3&) { return 1.0; });
      }
    }
  }
  inside.assign(J + 1, {});
  for (int l = 0; l <= J; ++l) {
    std::vector<std::array<uint64_t, 4>> tl;
    level_tets(o, l, tl);
    std::map<std::array<uint64_t, 4>, double> cl;
    if (l == J) {
      for (size_t t = 0; t < tJ.size(); ++t) cl[tJ[t]] = cov[t];
    } else {
      for (size_t t = 0; t < tJ.size(); ++t) {
        uint64_t X4[3] = {0, 0, 0};
        for (int v = 0; v < 4; ++v) {
          uint64_t q[3];
          xyz3(tJ[t][v], q);
          for (int d = 0; d < 3; ++d) X4[d] += q[d];
        }
        std::array<uint64_t, 4> anc;
        if (!locate_level_tet(o, l, X4, anc)) {
          o.err = "oracle: nested tetrahedron not located";
          return;
        }
        cl[anc] += cov[t];
      }
    }
    for (auto& t : tl) {
      P3 K[4];
      tet_points(o, t, K);
      if (cl[t] >= (1.0 - 1e-9) * tet_volume(K[0], K[1], K[2], K[3])) inside[l].push_back(t);
    }
  }
}

// R18 in 3D.  Gamma_D is the union of the fine boundary faces (faces of one
// element) whose three vertices are Dirichlet.  T^M_l keeps the tetrahedra of
// sigma^(l) whose interior meets Omega (positive covered volume) and no Gamma_D
// triangle; the Dirichlet nodes are the kept-tetrahedron nodes on Gamma_D or on
// a tetrahedron removed for Gamma_D.  Each level is its own P1 discretisation
// with the mean of a over tau n Omega; nodal interpolation between levels; the
// near-boundary sets J_{l,j} of Algorithm 3 are built from the faces of one
// kept tetrahedron only.

P3 sub3(const P3& a, const P3& b) { return P3{a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
P3 cross3(const P3& a, const P3& b) {
  return P3{a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
double dot3(const P3& a, const P3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// The closed triangle T meets the interior of the tetrahedron K exactly when
// no separating direction exists with touching allowed; the candidate
// directions are K's face normals, T's normal and the cross products of an
// edge of K with an edge of T (the facet normals of K - T).  Projections are
// computed in FP64, so an overlap below 1e-12 |a| L along direction a (L the
// root box side) counts as touching: a lattice node on the edge of a jittered
// Gamma_D triangle touches it, and rounding must not turn that into a cut.
bool tri_meets_open_tet(const P3* T, const P3* K, double L) {
  std::vector<P3> axes;
  const int fv[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  for (auto& f : fv) axes.push_back(cross3(sub3(K[f[1]], K[f[0]]), sub3(K[f[2]], K[f[0]])));
  axes.push_back(cross3(sub3(T[1], T[0]), sub3(T[2], T[0])));
  const int ke[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  for (auto& e : ke)
    for (int t = 0; t < 3; ++t) axes.push_back(cross3(sub3(K[e[1]], K[e[0]]), sub3(T[(t + 1) % 3], T[t])));
  for (auto& a : axes) {
    if (a[0] == 0 && a[1] == 0 && a[2] == 0) continue;
    const double tol = 1e-12 * std::sqrt(dot3(a, a)) * L;
    double kmin = INFINITY, kmax = -INFINITY, tmin = INFINITY, tmax = -INFINITY;
    for (int v = 0; v < 4; ++v) {
      const double d = dot3(a, K[v]);
      kmin = std::min(kmin, d);
      kmax = std::max(kmax, d);
    }
    for (int v = 0; v < 3; ++v) {
      const double d = dot3(a, T[v]);
      tmin = std::min(tmin, d);
      tmax = std::max(tmax, d);
    }
    if (tmax <= kmin + tol || tmin >= kmax - tol) return false;
  }
  return true;
}

// The point p lies in the closed triangle T (coplanar, then inside in the
// projection that drops the largest normal component), both within the same
// relative 1e-12 as above.
bool point_in_tri3(const P3* T, const P3& p, double L) {
  const P3 n = cross3(sub3(T[1], T[0]), sub3(T[2], T[0]));
  const double nn = std::sqrt(dot3(n, n));
  if (std::fabs(dot3(n, sub3(p, T[0]))) > 1e-12 * nn * L) return false;
  int ax = 0;
  for (int k = 1; k < 3; ++k)
    if (std::fabs(n[k]) > std::fabs(n[ax])) ax = k;
  const int u = (ax + 1) % 3, v = (ax + 2) % 3;
  auto o2 = [&](const P3& a, const P3& b, const P3& c) {
    return (b[u] - a[u]) * (c[v] - a[v]) - (b[v] - a[v]) * (c[u] - a[u]);
  };
  const double tol = 1e-12 * nn * L;
  const double s0 = o2(T[0], T[1], p), s1 = o2(T[1], T[2], p), s2 = o2(T[2], T[0], p);
  return (s0 >= -tol && s1 >= -tol && s2 >= -tol) || (s0 <= tol && s1 <= tol && s2 <= tol);
}

void build_aux_mixed3(Oracle& o) {
  const int J = o.J;
  o.lv.assign(J + 1, Level());
  std::vector<std::array<uint64_t, 4>> tJ;
  level_tets(o, J, tJ);
  std::map<std::array<uint64_t, 4>, int64_t> idx;
  for (size_t t = 0; t < tJ.size(); ++t) idx[tJ[t]] = (int64_t)t;
  // covered volume and integral of a over tau n Omega (exact intersection)
  std::vector<double> cov(tJ.size(), 0.0), num(tJ.size(), 0.0);
  std::vector<std::array<uint64_t, 4>> leaves, kt;
  for (int64_t e = 0; e < o.ne; ++e) {
    P3 T[4];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < 4; ++v)
      for (int k = 0; k < 3; ++k) {
        T[v][k] = o.X[(int64_t)o.E[4 * e + v] * 3 + k];
        lo[k] = std::min(lo[k], T[v][k]);
        hi[k] = std::max(hi[k], T[v][k]);
      }
    leaves.clear();
    leaves_overlapping3(o, lo, hi, leaves);
    const double a = o.coeff.empty() ? 1.0 : o.coeff[e];
    for (auto& b : leaves) {
      kt.clear();
      uint64_t q[3] = {b[1], b[2], b[3]};
      box_tets(o, (int)b[0], q, J, kt);
      for (auto& k4 : kt) {
        P3 K[4];
        tet_points(o, k4, K);
        std::vector<SignedTet> P = intersect_tets(T, K);
        if (P.empty()) continue;
        const double vol = pieces_integral(P, [](const P3&) { return 1.0; }, [](const P3&) { return 1.0; });
        cov[idx.at(k4)] += vol;
        num[idx.at(k4)] += a * vol;
      }
    }
  }
  // Gamma_D: faces of one element whose three vertices are Dirichlet
  std::map<std::array<int32_t, 3>, int> fcount;
  for (int64_t e = 0; e < o.ne; ++e)
    for (int k = 0; k < 4; ++k) {
      std::array<int32_t, 3> f = {o.E[4 * e + (k + 1) % 4], o.E[4 * e + (k + 2) % 4], o.E[4 * e + (k + 3) % 4]};
      std::sort(f.begin(), f.end());
      fcount[f] += 1;
    }
  std::vector<std::array<P3, 3>> gamma_d;
  for (auto& kv : fcount) {
    if (kv.second != 1) continue;
    bool dir = true;
    for (int k = 0; k < 3; ++k) dir = dir && o.bflag[kv.first[k]] == 1;
    if (!dir) continue;
    std::array<P3, 3> tr;
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) tr[k][d] = o.X[(int64_t)kv.first[k] * 3 + d];
    gamma_d.push_back(tr);
  }
  auto vol_of = [&](const std::array<uint64_t, 4>& t) {
    P3 K[4];
    tet_points(o, t, K);
    return std::fabs(tet_volume(K[0], K[1], K[2], K[3]));
  };
  std::vector<std::vector<double>> coef(J + 1);
  for (int l = 0; l <= J; ++l) {
    std::vector<std::array<uint64_t, 4>> tl;
    level_tets(o, l, tl);
    std::map<std::array<uint64_t, 4>, double> cl, nl;
    for (size_t t = 0; t < tJ.size(); ++t) {
      std::array<uint64_t, 4> anc = tJ[t];
      if (l < J) {
        uint64_t X4[3] = {0, 0, 0};
        for (int v = 0; v < 4; ++v) {
          uint64_t q[3];
          xyz3(tJ[t][v], q);
          for (int d = 0; d < 3; ++d) X4[d] += q[d];
        }
        if (!locate_level_tet(o, l, X4, anc)) {
          o.err = "oracle: nested tetrahedron not located";
          return;
        }
      }
      cl[anc] += cov[t];
      nl[anc] += num[t];
    }
    Level& L = o.lv[l];
    std::set<uint64_t> dirn;
    for (auto& t : tl) {
      P3 K[4];
      tet_points(o, t, K);
      double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int v = 0; v < 4; ++v)
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::min(lo[d], K[v][d]);
          hi[d] = std::max(hi[d], K[v][d]);
        }
      bool hit = false;
      for (auto& g : gamma_d) {
        bool apart = false;
        for (int d = 0; d < 3; ++d)
          apart = apart || std::max({g[0][d], g[1][d], g[2][d]}) < lo[d] || std::min({g[0][d], g[1][d], g[2][d]}) > hi[d];
        if (!apart && tri_meets_open_tet(g.data(), K, o.L)) {
          hit = true;
          break;
        }
      }
      if (hit) {
        for (int v = 0; v < 4; ++v) dirn.insert(t[v]);
        continue;
      }
      if (!(cl[t] > 1e-12 * vol_of(t))) continue;  // outside Omega
      L.tet.push_back(t);
      coef[l].push_back(nl[t] / cl[t]);
    }
    for (auto& t : L.tet)
      for (int k = 0; k < 4; ++k) L.allkey.push_back(t[k]);
    std::sort(L.allkey.begin(), L.allkey.end());
    L.allkey.erase(std::unique(L.allkey.begin(), L.allkey.end()), L.allkey.end());
    for (auto k : L.allkey) {
      if (dirn.count(k)) continue;
      double pp[3];
      physical3(o, k, pp);
      const P3 p = {pp[0], pp[1], pp[2]};
      bool ond = false;
      for (auto& g : gamma_d) ond = ond || point_in_tri3(g.data(), p, o.L);
      if (!ond) L.key.push_back(k);
    }
  }
  o.c = 0;
  for (int l = 0; l <= J; ++l)
    if ((int64_t)o.lv[l].key.size() <= o.prm.coarse_max) o.c = l;
  o.finest_coef = coef[J];
  for (int l = o.c; l <= J; ++l) {
    Level& L = o.lv[l];
    std::vector<std::vector<std::pair<int32_t, double>>> rows(L.key.size());
    for (size_t t = 0; t < L.tet.size(); ++t) {
      P3 K[4];
      tet_points(o, L.tet[t], K);
      int32_t id[4];
      for (int k = 0; k < 4; ++k) id[k] = find_index(L.key, L.tet[t][k]);
      double Ke[4][4];
      tet_stiffness(K, Ke);
      for (int i = 0; i < 4; ++i)
        if (id[i] >= 0)
          for (int j = 0; j < 4; ++j)
            if (id[j] >= 0) rows[id[i]].push_back({id[j], coef[l][t] * Ke[i][j]});
    }
    L.A = csr_from_rows(L.key.size(), L.key.size(), rows);
  }
  // nodal interpolation from level l-1: the coarse function on its kept
  // tetrahedra (every box shown at level l-1 whose closed cube holds the
  // point is searched), zero outside them and at its Dirichlet nodes
  for (int l = std::max(1, o.c + 1); l <= J; ++l) {
    Level& Lf = o.lv[l];
    Level& Lc = o.lv[l - 1];
    std::set<std::array<uint64_t, 4>> kept(Lc.tet.begin(), Lc.tet.end());
    std::vector<std::vector<std::pair<int32_t, double>>> rows(Lf.key.size());
    for (size_t k = 0; k < Lf.key.size(); ++k) {
      const int32_t j = find_index(Lc.key, Lf.key[k]);
      if (j >= 0) {
        rows[k].push_back({j, 1.0});
        continue;
      }
      uint64_t x[3];
      xyz3(Lf.key[k], x);
      std::vector<std::array<uint64_t, 4>> hold, stack;  // (depth, qx, qy, qz)
      stack.push_back({0, 0, 0, 0});
      while (!stack.empty()) {
        const auto b = stack.back();
        stack.pop_back();
        const int depth = (int)b[0];
        const uint64_t sz = 1ULL << (o.LB - depth);
        bool in = true;
        for (int d = 0; d < 3; ++d) in = in && x[d] >= b[1 + d] * sz && x[d] <= (b[1 + d] + 1) * sz;
        if (!in) continue;
        uint64_t q[3] = {b[1], b[2], b[3]};
        uint8_t sp = 0;
        if (!box_exists(o, depth, q, &sp)) continue;
        if (depth == l - 1 || !sp) {
          hold.push_back(b);
          continue;
        }
        for (uint64_t ch = 0; ch < 8; ++ch)
          stack.push_back({(uint64_t)depth + 1, 2 * b[1] + (ch & 1), 2 * b[2] + ((ch >> 1) & 1), 2 * b[3] + (ch >> 2)});
      }
      bool found = false;
      for (const auto& b : hold) {
        if (found) break;
        std::vector<std::array<uint64_t, 4>> ct;
        uint64_t q[3] = {b[1], b[2], b[3]};
        box_tets(o, (int)b[0], q, l - 1, ct);
        for (auto& t : ct) {
          if (!kept.count(t)) continue;
          i128 P[4][3];
          for (int v = 0; v < 4; ++v) {
            uint64_t qq[3];
            xyz3(t[v], qq);
            for (int d = 0; d < 3; ++d) P[v][d] = (i128)qq[d];
          }
          i128 e1[3], e2[3], e3[3], r[3];
          for (int d = 0; d < 3; ++d) {
            e1[d] = P[1][d] - P[0][d];
            e2[d] = P[2][d] - P[0][d];
            e3[d] = P[3][d] - P[0][d];
            r[d] = (i128)x[d] - P[0][d];
          }
          const i128 det = det3(e1, e2, e3);
          const i128 n1 = det3(r, e2, e3), n2 = det3(e1, r, e3), n3 = det3(e1, e2, r);
          const i128 n0 = det - n1 - n2 - n3;
          const i128 nn[4] = {n0, n1, n2, n3};
          bool inside = true;
          for (int v = 0; v < 4; ++v) inside = inside && (det > 0 ? nn[v] >= 0 : nn[v] <= 0);
          if (!inside) continue;
          for (int v = 0; v < 4; ++v) {
            if (nn[v] == 0) continue;
            const int32_t jj = find_index(Lc.key, t[v]);
            if (jj >= 0) rows[k].push_back({jj, (double)((long double)nn[v] / (long double)det)});
          }
          found = true;
          break;
        }
      }
    }
    Lf.I = csr_from_rows(Lf.key.size(), Lc.key.size(), rows);
  }
  // every level smoothed as a whole; near-boundary sets of Algorithm 3
  for (int l = o.c + 1; l <= J; ++l) {
    Level& L = o.lv[l];
    L.smooth.resize(L.key.size());
    for (size_t k = 0; k < L.key.size(); ++k) L.smooth[k] = (int32_t)k;
    if (o.prm.nb_layers < 0) continue;
    // Gamma_l: vertices of faces of one kept tetrahedron only; layer 0 = kept
    // tetrahedra with a vertex on Gamma_l, layer i = those with a vertex in layer i-1
    std::map<std::array<uint64_t, 3>, int> faces;
    for (auto& t : L.tet)
      for (int k = 0; k < 4; ++k) {
        std::array<uint64_t, 3> f = {t[(k + 1) % 4], t[(k + 2) % 4], t[(k + 3) % 4]};
        std::sort(f.begin(), f.end());
        faces[f] += 1;
      }
    std::set<uint64_t> verts;
    for (auto& kv : faces)
      if (kv.second == 1)
        for (int k = 0; k < 3; ++k) verts.insert(kv.first[k]);
    std::set<uint64_t> layer;
    for (int i = 0; i <= o.prm.nb_layers; ++i) {
      layer.clear();
      for (auto& t : L.tet)
        if (verts.count(t[0]) || verts.count(t[1]) || verts.count(t[2]) || verts.count(t[3]))
          for (int k = 0; k < 4; ++k) layer.insert(t[k]);
      if (layer == verts) break;
      verts = layer;
    }
    for (auto k : verts) {
      const int32_t id = find_index(L.key, k);
      if (id >= 0) L.nbset.push_back(id);
    }
    std::sort(L.nbset.begin(), L.nbset.end());
    const int64_t m = (int64_t)L.nbset.size();
    L.nbchol.assign(m * m, 0.0);
    for (int64_t a = 0; a < m; ++a)
      for (int64_t b = 0; b < m; ++b) L.nbchol[a * m + b] = L.A.get(L.nbset[a], L.nbset[b]);
    if (m && !cholesky(L.nbchol, m)) {
      o.err = "oracle: near-boundary block not positive definite";
      return;
    }
  }
}

void build_aux3(Oracle& o) {
  const int J = o.J;
  o.LB = J + 1;
  if (o.LB > 21) {
    o.err = "oracle: 3D auxiliary hierarchy deeper than 20 levels";
    return;
  }
  o.lv.assign(J + 1, Level());
  // does the domain fill the root cube?
  {
    double vol = 0.0;
    for (int64_t e = 0; e < o.ne; ++e) {
      P3 T[4];
      for (int v = 0; v < 4; ++v)
        for (int k = 0; k < 3; ++k) T[v][k] = o.X[(int64_t)o.E[4 * e + v] * 3 + k];
      vol += tet_volume(T[0], T[1], T[2], T[3]);
    }
    o.boxdomain = std::fabs(vol - o.L * o.L * o.L) <= 1e-12 * o.L * o.L * o.L;
  }
  for (int64_t v = 0; v < o.nv; ++v) o.neumann = o.neumann || o.bflag[v] == 2;
  if (o.neumann) {
    build_aux_mixed3(o);
    return;
  }
  std::vector<std::vector<std::array<uint64_t, 4>>> inside;
  if (!o.boxdomain) {
    dirichlet_tets(o, inside);
    if (!o.err.empty()) return;
  }
  for (int l = 0; l <= J; ++l) {
    Level& L = o.lv[l];
    if (o.boxdomain)
      level_tets(o, l, L.tet);
    else
      L.tet = inside[l];
    for (auto& t : L.tet)
      for (int k = 0; k < 4; ++k) L.allkey.push_back(t[k]);
    std::sort(L.allkey.begin(), L.allkey.end());
    L.allkey.erase(std::unique(L.allkey.begin(), L.allkey.end()), L.allkey.end());
    if (o.boxdomain) {
      for (auto k : L.allkey)
        if (!on_boundary3(o, k)) L.key.push_back(k);
    } else {
      // Gamma_l = boundary of the union of T^D_l: vertices of faces that
      // belong to one tetrahedron only
      std::map<std::array<uint64_t, 3>, int> faces;
      for (auto& t : L.tet)
        for (int k = 0; k < 4; ++k) {
          std::array<uint64_t, 3> f = {t[(k + 1) % 4], t[(k + 2) % 4], t[(k + 3) % 4]};
          std::sort(f.begin(), f.end());
          faces[f] += 1;
        }
      std::set<uint64_t> gamma;
      for (auto& kv : faces)
        if (kv.second == 1)
          for (int k = 0; k < 3; ++k) gamma.insert(kv.first[k]);
      for (auto k : L.allkey)
        if (!gamma.count(k)) L.key.push_back(k);
    }
  }
  o.c = 0;
  for (int l = 0; l <= J; ++l)
    if ((int64_t)o.lv[l].key.size() <= o.prm.coarse_max) o.c = l;
  // finest coefficient: volume-weighted mean of the fine coefficients (clipping)
  Level& LJ = o.lv[J];
  std::map<std::array<uint64_t, 4>, int64_t> tet_index;
  for (size_t t = 0; t < LJ.tet.size(); ++t) tet_index[LJ.tet[t]] = (int64_t)t;
  std::vector<double> num(LJ.tet.size(), 0.0);
  std::vector<std::array<uint64_t, 4>> leaves, kt;
  for (int64_t e = 0; e < o.ne; ++e) {
    P3 T[4];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < 4; ++v)
      for (int k = 0; k < 3; ++k) {
        T[v][k] = o.X[(int64_t)o.E[4 * e + v] * 3 + k];
        lo[k] = std::min(lo[k], T[v][k]);
        hi[k] = std::max(hi[k], T[v][k]);
      }
    leaves.clear();
    leaves_overlapping3(o, lo, hi, leaves);
    const double a = o.coeff.empty() ? 1.0 : o.coeff[e];
    for (auto& b : leaves) {
      kt.clear();
      uint64_t q[3] = {b[1], b[2], b[3]};
      box_tets(o, (int)b[0], q, J, kt);
      for (auto& k4 : kt) {
        P3 K[4];
        tet_points(o, k4, K);
        auto it = tet_index.find(k4);
        if (it == tet_index.end()) continue;  // outside Omega (not in T^D_J)
        std::vector<SignedTet> P = intersect_tets(T, K);
        if (P.empty()) continue;
        double vol = pieces_integral(P, [](const P3&) { return 1.0; }, [](const P3&) { return 1.0; });
        num[it->second] += a * vol;
      }
    }
  }
  o.finest_coef.resize(LJ.tet.size());
  for (size_t t = 0; t < LJ.tet.size(); ++t) {
    P3 K[4];
    tet_points(o, LJ.tet[t], K);
    o.finest_coef[t] = num[t] / tet_volume(K[0], K[1], K[2], K[3]);
  }
  {
    std::vector<std::vector<std::pair<int32_t, double>>> rows(LJ.key.size());
    for (size_t t = 0; t < LJ.tet.size(); ++t) {
      P3 K[4];
      tet_points(o, LJ.tet[t], K);
      int32_t id[4];
      for (int k = 0; k < 4; ++k) id[k] = find_index(LJ.key, LJ.tet[t][k]);
      double Ke[4][4];
      tet_stiffness(K, Ke);
      for (int i = 0; i < 4; ++i)
        if (id[i] >= 0)
          for (int j = 0; j < 4; ++j)
            if (id[j] >= 0) rows[id[i]].push_back({id[j], o.finest_coef[t] * Ke[i][j]});
    }
    LJ.A = csr_from_rows(LJ.key.size(), LJ.key.size(), rows);
  }
  // nodal interpolation from level l-1
  for (int l = std::max(1, o.c + 1); l <= J; ++l) {
    Level& Lf = o.lv[l];
    Level& Lc = o.lv[l - 1];
    std::vector<std::vector<std::pair<int32_t, double>>> rows(Lf.key.size());
    for (size_t k = 0; k < Lf.key.size(); ++k) {
      int32_t j = find_index(Lc.key, Lf.key[k]);
      if (j >= 0) {
        rows[k].push_back({j, 1.0});
        continue;
      }
      uint64_t x[3];
      xyz3(Lf.key[k], x);
      int depth = 0;
      uint64_t bq[3] = {0, 0, 0};
      for (;;) {
        uint8_t sp = 0;
        box_exists(o, depth, bq, &sp);
        if (depth == l - 1 || !sp) break;
        uint64_t half = 1ULL << (o.LB - depth - 1);
        for (int d = 0; d < 3; ++d) bq[d] = 2 * bq[d] + ((x[d] - bq[d] * 2 * half) >= half ? 1 : 0);
        ++depth;
      }
      std::vector<std::array<uint64_t, 4>> tets;
      box_tets(o, depth, bq, l - 1, tets);
      bool found = false;
      for (auto& t : tets) {
        i128 P[4][3];
        for (int v = 0; v < 4; ++v) {
          uint64_t q[3];
          xyz3(t[v], q);
          for (int d = 0; d < 3; ++d) P[v][d] = (i128)q[d];
        }
        i128 e1[3], e2[3], e3[3], r[3];
        for (int d = 0; d < 3; ++d) {
          e1[d] = P[1][d] - P[0][d];
          e2[d] = P[2][d] - P[0][d];
          e3[d] = P[3][d] - P[0][d];
          r[d] = (i128)x[d] - P[0][d];
        }
        i128 det = det3(e1, e2, e3);
        i128 n1 = det3(r, e2, e3), n2 = det3(e1, r, e3), n3 = det3(e1, e2, r);
        i128 n0 = det - n1 - n2 - n3;
        if (n0 < 0 || n1 < 0 || n2 < 0 || n3 < 0) continue;
        i128 nn[4] = {n0, n1, n2, n3};
        for (int v = 0; v < 4; ++v) {
          if (nn[v] == 0) continue;
          int32_t jj = find_index(Lc.key, t[v]);
          if (jj < 0) continue;
          rows[k].push_back({jj, (double)((long double)nn[v] / (long double)det)});
        }
        found = true;
        break;
      }
      if (!found) {
        o.err = "oracle: 3D interpolation point not located";
        return;
      }
    }
    Lf.I = csr_from_rows(Lf.key.size(), Lc.key.size(), rows);
  }
  for (int l = J; l > o.c; --l) {
    CSR It = transpose(o.lv[l].I);
    CSR AI = matmul(o.lv[l].A, o.lv[l].I);
    o.lv[l - 1].A = matmul(It, AI);
  }
  for (int l = o.c + 1; l <= J; ++l) {
    Level& Lf = o.lv[l];
    std::vector<int32_t> set;
    if (o.prm.smoothing == 1) {
      for (size_t k = 0; k < Lf.key.size(); ++k) set.push_back((int32_t)k);
    } else {
      std::set<std::array<uint64_t, 4>> prev;
      for (auto t : o.lv[l - 1].tet) {
        std::sort(t.begin(), t.end());
        prev.insert(t);
      }
      std::vector<uint8_t> mark(Lf.key.size(), 0);
      for (auto t : Lf.tet) {
        auto ts = t;
        std::sort(ts.begin(), ts.end());
        if (prev.count(ts)) continue;
        for (int v = 0; v < 4; ++v) {
          int32_t id = find_index(Lf.key, t[v]);
          if (id >= 0) mark[id] = 1;
        }
      }
      for (size_t k = 0; k < Lf.key.size(); ++k)
        if (mark[k]) set.push_back((int32_t)k);
    }
    Lf.smooth = set;
  }
}

// Scott-Zhang in 3D: psi_i = (20 lambda_i - 4)/|sigma_i| on the lowest-index
// tetrahedron at node i; P_ik = int_{sigma_i} psi_i phi_k by exact clipping.
void build_transfer3(Oracle& o) {
  const Level& LJ = o.lv[o.J];
  const int64_t n = o.vertex_of_free.size();
  std::vector<int32_t> sigma(o.nv, -1);
  for (int64_t e = 0; e < o.ne; ++e)
    for (int k = 0; k < 4; ++k) {
      int32_t v = o.E[4 * e + k];
      if (sigma[v] < 0) sigma[v] = (int32_t)e;
    }
  std::vector<std::vector<std::pair<int32_t, double>>> rows(n), rows_full(n);
  std::vector<std::array<uint64_t, 4>> leaves, kt;
  std::set<std::array<uint64_t, 4>> tet_in(LJ.tet.begin(), LJ.tet.end());
  for (int64_t i = 0; i < n; ++i) {
    int32_t v = o.vertex_of_free[i];
    int32_t e = sigma[v];
    P3 T[4];
    int loc = -1;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < 4; ++k) {
      int32_t vk = o.E[4 * (int64_t)e + k];
      for (int d = 0; d < 3; ++d) {
        T[k][d] = o.X[(int64_t)vk * 3 + d];
        lo[d] = std::min(lo[d], T[k][d]);
        hi[d] = std::max(hi[d], T[k][d]);
      }
      if (vk == v) loc = k;
    }
    const double vol = tet_volume(T[0], T[1], T[2], T[3]);
    auto psi = [&](const P3& x) {
      double l4[4];
      bary3(T, x, l4);
      return (20.0 * l4[loc] - 4.0) / vol;
    };
    leaves.clear();
    leaves_overlapping3(o, lo, hi, leaves);
    for (auto& b : leaves) {
      kt.clear();
      uint64_t q[3] = {b[1], b[2], b[3]};
      box_tets(o, (int)b[0], q, o.J, kt);
      for (auto& k4 : kt) {
        if ((!o.boxdomain || o.neumann) && !tet_in.count(k4)) continue;  // hats only on the kept tetrahedra
        P3 K[4];
        tet_points(o, k4, K);
        std::vector<SignedTet> P = intersect_tets(T, K);
        if (P.empty()) continue;
        for (int k = 0; k < 4; ++k) {
          auto phi = [&](const P3& x) {
            double l4[4];
            bary3(K, x, l4);
            return l4[k];
          };
          double val = pieces_integral(P, psi, phi);
          rows_full[i].push_back({find_index(LJ.allkey, k4[k]), val});
          int32_t jj = find_index(LJ.key, k4[k]);
          if (jj >= 0) rows[i].push_back({jj, val});
        }
      }
    }
  }
  o.P = csr_from_rows(n, LJ.key.size(), rows);
  o.Pfull = csr_from_rows(n, LJ.allkey.size(), rows_full);
}

// --------------------------------------------------------------------------
// Colouring (R10): Jones-Plassmann with splitmix64 priorities on the graph of
// couplings |a_vw| > 1e-12 sqrt(a_vv a_ww) (entries that vanish by symmetry,
// e.g. across the hypotenuse of a right isosceles triangle, are not
// couplings), then `ig_rounds` rounds of iterated greedy recolouring (classes
// visited in descending order; each node takes the smallest colour unused by
// the neighbours already visited in that round).
// --------------------------------------------------------------------------

bool coupled(const CSR& A, int64_t p, int32_t v, const std::vector<double>& diag) {
  int32_t w = A.col[p];
  if (w == v) return false;
  return std::fabs(A.val[p]) > 1e-12 * std::sqrt(diag[v] * diag[w]);
}

void jp_colour(const CSR& A, const std::vector<int32_t>& set, const std::vector<uint64_t>& prio_key,
               std::vector<int32_t>& colour, int mode, int ig_rounds) {
  colour.assign(A.nr, -1);
  std::vector<uint8_t> in(A.nr, 0);
  for (auto v : set) in[v] = 1;
  if (mode == 1) {  // one colour per node, in index order: lexicographic GS
    std::vector<int32_t> s = set;
    std::sort(s.begin(), s.end());
    for (size_t k = 0; k < s.size(); ++k) colour[s[k]] = (int32_t)k;
    return;
  }
  std::vector<double> diag(A.nr, 0.0);
  for (int64_t i = 0; i < A.nr; ++i) diag[i] = A.get(i, (int32_t)i);
  auto prio = [&](int32_t v) { return std::make_pair(splitmix64(prio_key[v]), prio_key[v]); };
  std::vector<int32_t> todo = set;
  while (!todo.empty()) {
    std::vector<int32_t> winners, rest;
    for (auto v : todo) {
      bool win = true;
      auto pv = prio(v);
      for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
        int32_t w = A.col[p];
        if (!in[w] || colour[w] >= 0 || !coupled(A, p, v, diag)) continue;
        if (prio(w) > pv) {
          win = false;
          break;
        }
      }
      (win ? winners : rest).push_back(v);
    }
    for (auto v : winners) {
      std::vector<uint8_t> used;
      for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
        int32_t w = A.col[p];
        if (!in[w] || colour[w] < 0 || !coupled(A, p, v, diag)) continue;
        if ((size_t)colour[w] >= used.size()) used.resize(colour[w] + 1, 0);
        used[colour[w]] = 1;
      }
      int32_t cc = 0;
      while ((size_t)cc < used.size() && used[cc]) ++cc;
      colour[v] = cc;
    }
    todo.swap(rest);
  }
  for (int round = 0; round < ig_rounds; ++round) {
    int32_t ncol = 0;
    for (auto v : set) ncol = std::max(ncol, colour[v] + 1);
    std::vector<int32_t> next(A.nr, -1);
    for (int32_t c = ncol - 1; c >= 0; --c)
      for (auto v : set) {
        if (colour[v] != c) continue;
        std::vector<uint8_t> used;
        for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
          int32_t w = A.col[p];
          if (!in[w] || colour[w] <= c || !coupled(A, p, v, diag)) continue;  // visited earlier this round
          if ((size_t)next[w] >= used.size()) used.resize(next[w] + 1, 0);
          used[next[w]] = 1;
        }
        int32_t cc = 0;
        while ((size_t)cc < used.size() && used[cc]) ++cc;
        next[v] = cc;
      }
    for (auto v : set) colour[v] = next[v];
  }
}

void order_by_colour(const std::vector<int32_t>& set, const std::vector<int32_t>& colour,
                     std::vector<int32_t>& smooth, std::vector<int32_t>& cstart) {
  smooth = set;
  std::stable_sort(smooth.begin(), smooth.end(), [&](int32_t a, int32_t b) {
    return colour[a] != colour[b] ? colour[a] < colour[b] : a < b;
  });
  cstart.clear();
  for (size_t k = 0; k < smooth.size(); ++k)
    if (k == 0 || colour[smooth[k]] != colour[smooth[k - 1]]) cstart.push_back((int32_t)k);
  cstart.push_back((int32_t)smooth.size());
}

// Colouring mode 2 on an auxiliary level: the lattice parity of each node of
// the smoothing set, (X + Y [+ Z]) / h_l mod 2 with h_l the lattice spacing of
// level l, when no two coupled nodes of the set share it (the level's
// coupling graph is bipartite: two colour classes).  Returns false, leaving
// `colour` untouched, when some coupled pair shares a parity.
bool parity_colour(const Oracle& o, int l, const CSR& A, const std::vector<int32_t>& set,
                   const std::vector<uint64_t>& key, std::vector<int32_t>& colour) {
  const int bits = o.dim == 2 ? o.D : o.LB;
  const uint64_t h = 1ULL << (bits - l);
  std::vector<int32_t> par(A.nr, -1);
  for (int32_t v : set) {
    uint64_t q[3] = {0, 0, 0};
    if (o.dim == 2) node_xy(key[v], q[0], q[1]);
    else xyz3(key[v], q);
    par[v] = (int32_t)(((q[0] + q[1] + q[2]) / h) & 1);
  }
  std::vector<double> diag(A.nr, 0.0);
  for (int64_t i = 0; i < A.nr; ++i) diag[i] = A.get(i, (int32_t)i);
  for (int32_t v : set)
    for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
      const int32_t w = A.col[p];
      if (par[w] >= 0 && par[w] == par[v] && coupled(A, p, v, diag)) return false;
    }
  colour.assign(A.nr, -1);
  for (int32_t v : set) colour[v] = par[v];
  return true;
}

void build_colourings(Oracle& o) {
  std::vector<int32_t> all(o.A.nr);
  std::vector<uint64_t> pk(o.A.nr);
  for (int64_t i = 0; i < o.A.nr; ++i) {
    all[i] = (int32_t)i;
    pk[i] = (uint64_t)o.vertex_of_free[i];
  }
  const int mode = o.prm.colouring == 2 ? 0 : o.prm.colouring;  // mode 2: JP on the fine grid
  jp_colour(o.A, all, pk, o.fine_colour, mode, 3);
  order_by_colour(all, o.fine_colour, o.fine_smooth, o.fine_cstart);
  for (int l = o.c + 1; l <= o.J; ++l) {
    Level& L = o.lv[l];
    if (!(o.prm.colouring == 2 && parity_colour(o, l, L.A, L.smooth, L.key, L.colour)))
      jp_colour(L.A, L.smooth, L.key, L.colour, mode, 3);
    std::vector<int32_t> set = L.smooth;
    order_by_colour(set, L.colour, L.smooth, L.cstart);
  }
}

// --------------------------------------------------------------------------
// Coarsest level: B_0 = A_0^{-1} by dense Cholesky (Algorithm 2).
// --------------------------------------------------------------------------

bool cholesky(std::vector<double>& M, int64_t n) {
  for (int64_t j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= M[j * n + k] * M[j * n + k];
    if (!(s > 0.0)) return false;
    double d = std::sqrt(s);
    M[j * n + j] = d;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (int64_t k = 0; k < j; ++k) t -= M[i * n + k] * M[j * n + k];
      M[i * n + j] = t / d;
    }
    for (int64_t i = 0; i < j; ++i) M[i * n + j] = 0.0;
  }
  return true;
}

void chol_solve(const std::vector<double>& Lm, int64_t n, const double* b, double* x) {
  std::vector<double> y(n);
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= Lm[i * n + k] * y[k];
    y[i] = s / Lm[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int64_t k = i + 1; k < n; ++k) s -= Lm[k * n + i] * x[k];
    x[i] = s / Lm[i * n + i];
  }
}

void build_coarse(Oracle& o) {
  const CSR& Ac = o.lv[o.c].A;
  int64_t n = Ac.nr;
  o.nc_dense = n;
  o.chol.assign(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = Ac.ptr[i]; p < Ac.ptr[i + 1]; ++p) o.chol[i * n + Ac.col[p]] = Ac.val[p];
  if (!cholesky(o.chol, n)) o.err = "oracle: coarse matrix not positive definite";
}

// --------------------------------------------------------------------------
// Smoother, V-cycle (Algorithm 2) and the multiplicative preconditioner
// (Algorithm 1, R8).
// --------------------------------------------------------------------------

// One Gauss-Seidel sweep over `smooth` in colour order (forward) or reverse
// colour order (backward): u_i += (f_i - (A u)_i) / a_ii.  Nodes of one
// colour are not coupled, so their order inside the class is immaterial.
void gs_sweep(const CSR& A, const std::vector<int32_t>& smooth, const std::vector<int32_t>& cstart,
              const double* f, double* u, bool forward) {
  int ncol = (int)cstart.size() - 1;
  for (int cc = 0; cc < ncol; ++cc) {
    int col = forward ? cc : ncol - 1 - cc;
    for (int32_t k = cstart[col]; k < cstart[col + 1]; ++k) {
      int32_t i = smooth[k];
      double s = f[i], dia = 0.0;
      for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
        s -= A.val[p] * u[A.col[p]];
        if (A.col[p] == i) dia = A.val[p];
      }
      u[i] += s / dia;
    }
  }
}

void vcycle(const Oracle& o, int l, const std::vector<double>& f, std::vector<double>& u) {
  const Level& L = o.lv[l];
  u.assign(L.key.size(), 0.0);
  if (l == o.c) {
    if (o.nc_dense > 0) chol_solve(o.chol, o.nc_dense, f.data(), u.data());
    return;
  }
  for (int s = 0; s < o.prm.nu_pre; ++s) gs_sweep(L.A, L.smooth, L.cstart, f.data(), u.data(), true);
  std::vector<double> Au(L.key.size()), r(L.key.size());
  spmv(L.A, u.data(), Au.data());
  for (size_t i = 0; i < r.size(); ++i) r[i] = f[i] - Au[i];
  const CSR& I = L.I;
  std::vector<double> fc(o.lv[l - 1].key.size(), 0.0);
  for (int64_t i = 0; i < I.nr; ++i)
    for (int64_t p = I.ptr[i]; p < I.ptr[i + 1]; ++p) fc[I.col[p]] += I.val[p] * r[i];
  std::vector<double> ec;
  vcycle(o, l - 1, fc, ec);
  for (int64_t i = 0; i < I.nr; ++i)
    for (int64_t p = I.ptr[i]; p < I.ptr[i + 1]; ++p) u[i] += I.val[p] * ec[I.col[p]];
  if (!L.nbset.empty()) {
    // Algorithm 3: near-boundary correction, u_J += (A_JJ)^{-1} (f - A u)_J
    spmv(L.A, u.data(), Au.data());
    const int64_t m = (int64_t)L.nbset.size();
    std::vector<double> rj(m), dj(m);
    for (int64_t a = 0; a < m; ++a) rj[a] = f[L.nbset[a]] - Au[L.nbset[a]];
    chol_solve(L.nbchol, m, rj.data(), dj.data());
    for (int64_t a = 0; a < m; ++a) u[L.nbset[a]] += dj[a];
  }
  for (int s = 0; s < o.prm.nu_post; ++s) gs_sweep(L.A, L.smooth, L.cstart, f.data(), u.data(), false);
}

// u <- u + S (r - A u), fine_sweeps times: Gauss-Seidel is one multicolour
// sweep in place (forward for S, backward for S^t); Jacobi takes the whole
// residual first and adds D^{-1} of it (S = S^t = D^{-1}).
void fine_smooth(const Oracle& o, const double* r, double* u, bool forward) {
  const int64_t n = o.A.nr;
  std::vector<double> Au(n);
  for (int m = 0; m < o.prm.fine_sweeps; ++m) {
    if (o.prm.smoother == 0) {
      gs_sweep(o.A, o.fine_smooth, o.fine_cstart, r, u, forward);
    } else {
      spmv(o.A, u, Au.data());
      for (int64_t i = 0; i < n; ++i) u[i] += (r[i] - Au[i]) / o.A.get(i, (int32_t)i);
    }
  }
}

// One application z = B r.
//   multiplicative (Algorithm 1):  u1 = S r;  u2 = u1 + Pi Btilde Pi^t (r - A u1);
//                                  z = u2 + S^t (r - A u2)
//   additive (eq. fasp):           z = S r + Pi Btilde Pi^t r
// with Btilde the V-cycle of Algorithm 2 on the auxiliary hierarchy.
void precond(const Oracle& o, const double* r, double* z) {
  const int64_t n = o.A.nr;
  std::vector<double> u(n, 0.0), Au(n), rho(n);
  fine_smooth(o, r, u.data(), true);
  if (o.prm.additive) {
    for (int64_t i = 0; i < n; ++i) rho[i] = r[i];
  } else {
    spmv(o.A, u.data(), Au.data());
    for (int64_t i = 0; i < n; ++i) rho[i] = r[i] - Au[i];
  }
  const int64_t nJ = o.lv[o.J].key.size();
  if (nJ > 0) {
    std::vector<double> fJ(nJ, 0.0), eJ;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = o.P.ptr[i]; p < o.P.ptr[i + 1]; ++p) fJ[o.P.col[p]] += o.P.val[p] * rho[i];
    vcycle(o, o.J, fJ, eJ);
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t p = o.P.ptr[i]; p < o.P.ptr[i + 1]; ++p) s += o.P.val[p] * eJ[o.P.col[p]];
      u[i] += s;
    }
  }
  if (!o.prm.additive) fine_smooth(o, r, u.data(), false);
  for (int64_t i = 0; i < n; ++i) z[i] = u[i];
}

// The ASMG iteration as a solver (Sec. 5.1, "convergence rates for the ASMG
// iteration"): u <- u + B (b - A u) until ||b - A u|| <= rtol ||b||.
// Returns 0 converged, 1 not converged, -4 on a non-finite residual.
int asmg_iteration(const Oracle& o, const double* b, double* u, double rtol, int* iters, double* hist) {
  const int64_t n = o.A.nr;
  std::vector<double> bb(b, b + n), x(u, u + n), r(n), z(n), Ax(n);
  const double nb = std::sqrt(dot(bb, bb));
  int status = 1;
  *iters = 0;
  for (int k = 0;; ++k) {
    spmv(o.A, x.data(), Ax.data());
    for (int64_t i = 0; i < n; ++i) r[i] = bb[i] - Ax[i];
    const double nr = std::sqrt(dot(r, r));
    hist[k] = nr;
    *iters = k;
    if (!std::isfinite(nr)) {
      status = -4;
      break;
    }
    if (nr <= rtol * nb) {
      status = 0;
      break;
    }
    if (k == o.prm.max_iter) break;
    precond(o, r.data(), z.data());
    for (int64_t i = 0; i < n; ++i) x[i] += z[i];
  }
  for (int64_t i = 0; i < n; ++i) u[i] = x[i];
  return status;
}

// PCG with the flexible beta (R9); returns 0 converged, 1 not converged,
// -4 breakdown.
int pcg(const Oracle& o, const double* b, double* u, double rtol, int* iters, double* hist) {
  const int64_t n = o.A.nr;
  std::vector<double> bb(b, b + n), x(u, u + n), r(n), z(n), p(n), q(n), rold(n);
  spmv(o.A, x.data(), q.data());
  for (int64_t i = 0; i < n; ++i) r[i] = bb[i] - q[i];
  double nb = std::sqrt(dot(bb, bb));
  double nr = std::sqrt(dot(r, r));
  hist[0] = nr;
  *iters = 0;
  if (nr <= rtol * nb) {
    for (int64_t i = 0; i < n; ++i) u[i] = x[i];
    return 0;
  }
  precond(o, r.data(), z.data());
  p = z;
  double rz = dot(r, z);
  int status = 1;
  for (int k = 0; k < o.prm.max_iter; ++k) {
    spmv(o.A, p.data(), q.data());
    double pq = dot(p, q);
    if (!(pq > 0.0) || !(rz > 0.0)) {
      status = -4;
      break;
    }
    double alpha = rz / pq;
    rold = r;
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    nr = std::sqrt(dot(r, r));
    hist[k + 1] = nr;
    *iters = k + 1;
    if (nr <= rtol * nb) {
      status = 0;
      break;
    }
    precond(o, r.data(), z.data());
    double num = 0.0;
    for (int64_t i = 0; i < n; ++i) num += z[i] * (r[i] - rold[i]);
    double beta = num / rz;
    rz = dot(r, z);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  for (int64_t i = 0; i < n; ++i) u[i] = x[i];
  return status;
}

}  // namespace

// ==========================================================================
// C interface (ctypes)
// ==========================================================================

extern "C" {

void* orc_create(int dim, int64_t nv, const double* X, int64_t ne, const int32_t* E, const uint8_t* bflag,
                 const double* coeff, const int32_t* params, char* err, int errlen) {
  Oracle* o = new Oracle();
  o->dim = dim;
  o->nv = nv;
  o->ne = ne;
  o->X.assign(X, X + nv * dim);
  o->E.assign(E, E + ne * (dim + 1));
  o->bflag.assign(bflag, bflag + nv);
  if (coeff) o->coeff.assign(coeff, coeff + ne);
  if (params) {
    o->prm.n_min = params[0];
    o->prm.nu_pre = params[1];
    o->prm.nu_post = params[2];
    o->prm.coarse_max = params[3];
    o->prm.smoothing = params[4];
    o->prm.max_iter = params[5];
    o->prm.colouring = params[6];
    o->prm.stage = params[7];
    o->prm.smoother = params[8];
    o->prm.additive = params[9];
    o->prm.fine_sweeps = params[10];
    o->prm.iteration = params[11];
    o->prm.nb_layers = params[12];
  }
  if (o->prm.stage >= 0) assemble_fine(*o);  // stage -1: cluster tree only
  build_tree(*o);
  if (o->prm.stage >= 1) build_closure(*o);
  if (o->prm.stage >= 2) {
    if (dim == 2) {
      build_aux(*o);
      if (o->err.empty()) build_transfer(*o);
    } else {
      build_aux3(*o);
      if (o->err.empty()) build_transfer3(*o);
    }
    if (o->err.empty()) build_colourings(*o);
    if (o->err.empty()) build_coarse(*o);
  }
  if (!o->err.empty()) {
    if (err) snprintf(err, errlen, "%s", o->err.c_str());
    delete o;
    return nullptr;
  }
  return o;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

// Integer information.  `what`: nfree, J, c, D, ntree_levels, nseg(l),
// nlevel(l) [free nodes], nall(l), ntri(l), nnzA(l) [l=-1: fine A], nI(l),
// nsmooth(l), ncolours(l) [l=-1 fine], nP, nPfull, nbox(l).
int64_t orc_info(void* h, const char* what, int l) {
  Oracle& o = *(Oracle*)h;
  std::string w(what);
  if (w == "nfree") return o.A.nr;
  if (w == "J") return o.J;
  if (w == "c") return o.c;
  if (w == "D") return o.D;
  if (w == "ntree_levels") return (int64_t)o.tree.size();
  if (w == "nseg") return (int64_t)o.tree.at(l).size();
  if (w == "nbox_levels") return (int64_t)o.boxes.size();
  if (w == "nbox") return (int64_t)o.boxes.at(l).size();
  if (w == "nlevel") return (int64_t)o.lv.at(l).key.size();
  if (w == "nall") return (int64_t)o.lv.at(l).allkey.size();
  if (w == "ntri") return (int64_t)o.lv.at(l).tri.size();
  if (w == "nalltri") {
    std::vector<std::array<uint64_t, 3>> t;
    level_triangles(o, l, t);
    return (int64_t)t.size();
  }
  if (w == "ntet") return (int64_t)o.lv.at(l).tet.size();
  if (w == "nalltet") {
    std::vector<std::array<uint64_t, 4>> t;
    level_tets(o, l, t);
    return (int64_t)t.size();
  }
  if (w == "LB") return o.LB;
  if (w == "nnzA") return l < 0 ? (int64_t)o.A.col.size() : (int64_t)o.lv.at(l).A.col.size();
  if (w == "nI") return (int64_t)o.lv.at(l).I.col.size();
  if (w == "nsmooth") return l < 0 ? (int64_t)o.fine_smooth.size() : (int64_t)o.lv.at(l).smooth.size();
  if (w == "ncolours") return l < 0 ? (int64_t)o.fine_cstart.size() - 1 : (int64_t)o.lv.at(l).cstart.size() - 1;
  if (w == "nnb") return (int64_t)o.lv.at(l).nbset.size();
  if (w == "nP") return (int64_t)o.P.col.size();
  if (w == "nPfull") return (int64_t)o.Pfull.col.size();
  return -1;
}

static void put_csr(const CSR& M, void* out, int part) {
  if (part == 0) memcpy(out, M.ptr.data(), M.ptr.size() * 8);
  if (part == 1) memcpy(out, M.col.data(), M.col.size() * 4);
  if (part == 2) memcpy(out, M.val.data(), M.val.size() * 8);
}

// Array export; the caller sizes `out` from orc_info.
int orc_get(void* h, const char* what, int l, void* out) {
  Oracle& o = *(Oracle*)h;
  std::string w(what);
  if (w == "keys") { memcpy(out, o.keys.data(), o.keys.size() * 8); return 0; }
  if (w == "perm") { memcpy(out, o.perm.data(), o.perm.size() * 4); return 0; }
  if (w == "root") { double* d = (double*)out; d[0] = o.amin[0]; d[1] = o.amin[1]; d[2] = o.dim == 3 ? o.amin[2] : 0; d[3] = o.L; return 0; }
  if (w == "seg") {  // int64 [nseg, 4]: prefix, begin, end, split
    int64_t* d = (int64_t*)out;
    for (size_t k = 0; k < o.tree.at(l).size(); ++k) {
      auto& s = o.tree[l][k];
      d[4 * k] = (int64_t)s.prefix; d[4 * k + 1] = s.begin; d[4 * k + 2] = s.end; d[4 * k + 3] = s.split;
    }
    return 0;
  }
  if (w == "box") {  // uint64 [nbox, 2]: packed coords, split; sorted
    std::vector<std::pair<uint64_t, uint8_t>> bx(o.boxes.at(l).begin(), o.boxes.at(l).end());
    std::sort(bx.begin(), bx.end());
    uint64_t* d = (uint64_t*)out;
    for (size_t k = 0; k < bx.size(); ++k) { d[2 * k] = bx[k].first; d[2 * k + 1] = bx[k].second; }
    return 0;
  }
  if (w == "level_key") { memcpy(out, o.lv.at(l).key.data(), o.lv[l].key.size() * 8); return 0; }
  if (w == "level_allkey") { memcpy(out, o.lv.at(l).allkey.data(), o.lv[l].allkey.size() * 8); return 0; }
  if (w == "level_tri") { memcpy(out, o.lv.at(l).tri.data(), o.lv[l].tri.size() * 24); return 0; }
  if (w == "level_alltri") {  // every triangle of sigma^(l), inside Omega or not
    std::vector<std::array<uint64_t, 3>> t;
    level_triangles(o, l, t);
    memcpy(out, t.data(), t.size() * 24);
    return 0;
  }
  if (w == "level_tet") { memcpy(out, o.lv.at(l).tet.data(), o.lv[l].tet.size() * 32); return 0; }
  if (w == "level_alltet") {  // every tetrahedron of sigma^(l), inside Omega or not
    std::vector<std::array<uint64_t, 4>> t;
    level_tets(o, l, t);
    memcpy(out, t.data(), t.size() * 32);
    return 0;
  }
  if (w == "finest_coef") { memcpy(out, o.finest_coef.data(), o.finest_coef.size() * 8); return 0; }
  if (w == "nbset") { memcpy(out, o.lv.at(l).nbset.data(), o.lv[l].nbset.size() * 4); return 0; }
  if (w == "smooth") {
    if (l < 0) memcpy(out, o.fine_smooth.data(), o.fine_smooth.size() * 4);
    else memcpy(out, o.lv.at(l).smooth.data(), o.lv[l].smooth.size() * 4);
    return 0;
  }
  if (w == "cstart") {
    if (l < 0) memcpy(out, o.fine_cstart.data(), o.fine_cstart.size() * 4);
    else memcpy(out, o.lv.at(l).cstart.data(), o.lv[l].cstart.size() * 4);
    return 0;
  }
  if (w == "colour") {
    if (l < 0) memcpy(out, o.fine_colour.data(), o.fine_colour.size() * 4);
    else memcpy(out, o.lv.at(l).colour.data(), o.lv[l].colour.size() * 4);
    return 0;
  }
  if (w == "vertex_of_free") { memcpy(out, o.vertex_of_free.data(), o.vertex_of_free.size() * 4); return 0; }
  const CSR* M = nullptr;
  std::string base;
  if (w.rfind("A_", 0) == 0) { M = l < 0 ? &o.A : &o.lv.at(l).A; base = w.substr(2); }
  else if (w.rfind("I_", 0) == 0) { M = &o.lv.at(l).I; base = w.substr(2); }
  else if (w.rfind("Pfull_", 0) == 0) { M = &o.Pfull; base = w.substr(6); }
  else if (w.rfind("P_", 0) == 0) { M = &o.P; base = w.substr(2); }
  if (M) {
    put_csr(*M, out, base == "ptr" ? 0 : base == "col" ? 1 : 2);
    return 0;
  }
  return -1;
}

void orc_mass_apply(void* h, const double* f, double* b) { mass_apply(*(Oracle*)h, f, b); }

void orc_spmv(void* h, int l, const double* x, double* y) {
  Oracle& o = *(Oracle*)h;
  spmv(l < 0 ? o.A : o.lv.at(l).A, x, y);
}

void orc_precond(void* h, const double* r, double* z) { precond(*(Oracle*)h, r, z); }

void orc_vcycle(void* h, const double* f, double* e) {
  Oracle& o = *(Oracle*)h;
  std::vector<double> fv(f, f + o.lv[o.J].key.size()), ev;
  vcycle(o, o.J, fv, ev);
  std::copy(ev.begin(), ev.end(), e);
}

void orc_gs_sweep(void* h, const double* f, double* u, int forward) {
  Oracle& o = *(Oracle*)h;
  gs_sweep(o.A, o.fine_smooth, o.fine_cstart, f, u, forward != 0);
}

int orc_solve(void* h, const double* b, double* u, double rtol, int* iters, double* hist) {
  Oracle& o = *(Oracle*)h;
  return o.prm.iteration ? asmg_iteration(o, b, u, rtol, iters, hist) : pcg(o, b, u, rtol, iters, hist);
}

// dL/da_e = -lambda_e^T K_e^(1) u_e, with u, lambda given on free nodes
// (zero on Dirichlet vertices) and K_e^(1) the element stiffness for a = 1.
void orc_elem_grad(void* h, const double* u, const double* lam, double* g) {
  Oracle& o = *(Oracle*)h;
  const int d = o.dim, nvert = d + 1;
  for (int64_t e = 0; e < o.ne; ++e) {
    double G[4][3], vol;
    simplex_geometry(o, e, G, vol);
    double ue[4], le[4];
    for (int k = 0; k < nvert; ++k) {
      int32_t f = o.free_of_vertex[o.E[e * nvert + k]];
      ue[k] = f >= 0 ? u[f] : 0.0;
      le[k] = f >= 0 ? lam[f] : 0.0;
    }
    double s = 0.0;
    for (int i = 0; i < nvert; ++i)
      for (int j = 0; j < nvert; ++j) {
        double gg = 0.0;
        for (int r = 0; r < d; ++r) gg += G[i][r] * G[j][r];
        s += le[i] * vol * gg * ue[j];
      }
    g[e] = -s;
  }
}

}  // extern "C"
