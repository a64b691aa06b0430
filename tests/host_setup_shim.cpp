// Test shim: runs the library's host part of the setup (closure, auxiliary
// grids, node sets, smoothing sets, level simplices, new nodes, transfer
// table) on a given cluster tree, then computes the Scott-Zhang rows with
// the library's own row routine on the host, and exposes the results to the
// CPU tests, which compare them with the oracle.  Built by the tests with g++
// from the library sources; no GPU is involved.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>

#include "../paper_1410_2153_gb300/csrc/internal.h"
#include "../paper_1410_2153_gb300/csrc/keyindex.h"
#include "../paper_1410_2153_gb300/csrc/nbsolve.h"
#include "../paper_1410_2153_gb300/csrc/sz_row.h"

using namespace asmg;

namespace {

struct Shim {
  AuxHost aux;
  std::string err;
};

// the transfer rows through the library's row routine, run on the host
void transfer_rows(const MeshHost& m, const std::vector<int32_t>& vof, const SZTable& tab, Triplets& P) {
  using namespace szrow;
  const int nvpe = tab.dim + 1;
  std::vector<int32_t> sigma(m.nv, INT_MAX);
  for (int64_t e = 0; e < m.ne; ++e)
    for (int k = 0; k < nvpe; ++k) sigma[m.E[nvpe * e + k]] = std::min(sigma[m.E[nvpe * e + k]], (int32_t)e);
  SZDev t;
  t.dim = tab.dim;
  t.D = tab.D;
  for (int a = 0; a < 3; ++a) t.amin[a] = tab.amin[a];
  t.L = tab.L;
  t.sc = std::ldexp(1.0, tab.D) / tab.L;
  t.node_key = tab.node_key.data();
  t.node_pay = tab.node_pay.data();
  t.leaf_first = tab.leaf_first.data();
  t.simp_key = tab.simp_key.data();
  t.simp_col = tab.simp_col.data();
  t.X = m.X.data();
  t.E = m.E.data();
  t.sigma = sigma.data();
  t.vof = vof.data();
  t.n = (int64_t)vof.size();
  t.nnode = (int64_t)tab.node_key.size();
  t.nleaf = (int64_t)tab.leaf_first.size() - 1;
  t.nsimp = (int64_t)tab.simp_col.size() / nvpe;
  t.nv = m.nv;
  t.ne = m.ne;
  P = Triplets();
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t i = 0; i < t.n; ++i) {
    row.clear();
    auto emit = [&](int32_t c, double v) { row.push_back({c, v}); };
    const bool ok = tab.dim == 2 ? sz_row<2>(t, i, true, emit) : sz_row<3>(t, i, true, emit);
    if (!ok) throw Error{ASMG_ERR_CUDA, "transfer row: index out of range"};
    std::stable_sort(row.begin(), row.end(), [](const std::pair<int32_t, double>& a,
                                                const std::pair<int32_t, double>& b) { return a.first < b.first; });
    for (size_t k = 0; k < row.size();) {
      size_t j = k;
      double s = 0;
      while (j < row.size() && row[j].first == row[k].first) s += row[j++].second;
      P.r.push_back((int32_t)i);
      P.c.push_back(row[k].first);
      P.v.push_back(s);
      k = j;
    }
  }
}

}  // namespace

extern "C" {

// BF16 bits of FP32 values as the library stores auxiliary-level values
// (asmg_params::level_bf16)
void shim_bf16(const float* x, uint16_t* y, int64_t n) {
  for (int64_t k = 0; k < n; ++k) y[k] = asmg::bf16_bits(x[k]);
}


// dim 2 or 3; the tree as split prefixes per depth (cnt[d] of them in flat);
// root box: amin[dim], side L; returns a handle (errors: see shim_error)
void* shim_build(int dim, int64_t nv, const double* X, int64_t ne, const int32_t* E, const uint8_t* bflag,
                 const double* coeff, int nlev, const int64_t* cnt, const uint64_t* flat, const double* amin, double L,
                 int n_min, int coarse_max, int smoothing, int nb_layers) {
  Shim* h = new Shim();
  try {
    const int nvpe = dim + 1;
    MeshHost m;
    m.dim = dim;
    m.nv = nv;
    m.ne = ne;
    m.X.assign(X, X + dim * nv);
    m.E.assign(E, E + nvpe * ne);
    m.bflag.assign(bflag, bflag + nv);
    if (coeff) m.coeff.assign(coeff, coeff + ne);
    double meas = 0;
    for (int64_t e = 0; e < ne; ++e) {
      const int32_t* v = &E[nvpe * e];
      if (dim == 2) {
        meas += 0.5 * ((X[2 * v[1]] - X[2 * v[0]]) * (X[2 * v[2] + 1] - X[2 * v[0] + 1]) -
                       (X[2 * v[2]] - X[2 * v[0]]) * (X[2 * v[1] + 1] - X[2 * v[0] + 1]));
      } else {
        double a[3], b[3], c[3];
        for (int k = 0; k < 3; ++k) {
          a[k] = X[3 * v[1] + k] - X[3 * v[0] + k];
          b[k] = X[3 * v[2] + k] - X[3 * v[0] + k];
          c[k] = X[3 * v[3] + k] - X[3 * v[0] + k];
        }
        meas += (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                 a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
      }
    }
    const double box = std::pow(L, dim);
    m.boxdomain = std::fabs(meas - box) <= 1e-12 * box;
    m.mixed = std::find(bflag, bflag + nv, (uint8_t)2) != bflag + nv;
    m.nb_layers = nb_layers;
    TreeResult tree;
    for (int k = 0; k < dim; ++k) tree.amin[k] = amin[k];
    tree.L = L;
    tree.D = dim == 2 ? 31 : 21;
    int64_t o = 0;
    for (int d = 0; d < nlev; ++d) {
      tree.split.push_back(std::vector<uint64_t>(flat + o, flat + o + cnt[d]));
      o += cnt[d];
    }
    asmg_params p;
    std::memset(&p, 0, sizeof p);
    p.n_min = n_min;
    p.nu_pre = 2;
    p.nu_post = 2;
    p.coarse_max_dofs = coarse_max;
    p.smoothing = smoothing;
    p.max_iter = 500;
    p.fine_sweeps = 1;
    std::vector<int32_t> vof;
    for (int64_t v = 0; v < nv; ++v)
      if (bflag[v] != 1) vof.push_back((int32_t)v);  // Neumann vertices are unknowns too
    if (dim == 2)
      build_aux_host(m, tree, p, h->aux);
    else
      build_aux_host3(m, tree, p, h->aux);
    transfer_rows(m, vof, h->aux.sz, h->aux.P);
  } catch (const Error& e) {
    h->err = e.msg;
  }
  return h;
}

const char* shim_error(void* hp) { return ((Shim*)hp)->err.c_str(); }

void shim_free(void* hp) { delete (Shim*)hp; }

// number of elements of array `what` at level l; copied to out when out != NULL
int64_t shim_get(void* hp, const char* what, int l, void* out) {
  AuxHost& a = ((Shim*)hp)->aux;
  const std::string w(what);
  auto put = [&](const void* src, int64_t n, size_t el) {
    if (out && n) memcpy(out, src, n * el);
    return n;
  };
  if (w == "J") return a.J;
  if (w == "c") return a.c;
  if (w == "nlevel") return put(a.nlevel.data(), (int64_t)a.nlevel.size(), 8);
  if (w == "split") return l < (int)a.split.size() ? put(a.split[l].data(), (int64_t)a.split[l].size(), 8) : 0;
  if (w == "aux_key") return put(a.aux_key.data(), (int64_t)a.aux_key.size(), 8);
  if (w == "coarse_id") return put(a.coarse_id.data(), (int64_t)a.coarse_id.size(), 4);
  if (w == "P_r") return put(a.P.r.data(), (int64_t)a.P.r.size(), 4);
  if (w == "P_c") return put(a.P.c.data(), (int64_t)a.P.c.size(), 4);
  if (w == "P_v") return put(a.P.v.data(), (int64_t)a.P.v.size(), 8);
  if (w == "phi") return put(a.phi.data(), (int64_t)a.phi.size(), 4);
  if (w == "psi") return put(a.psi.data(), (int64_t)a.psi.size(), 4);
  const int k = l - (a.c + 1);
  if (k < 0 || k >= (int)a.levels.size()) return -1;
  AuxLevelHost& L = a.levels[k];
  if (w == "smooth") return put(L.smooth.data(), (int64_t)L.smooth.size(), 4);
  if (w == "new_id") return put(L.new_id.data(), (int64_t)L.new_id.size(), 4);
  if (w == "new_p0") return put(L.new_p0.data(), (int64_t)L.new_p0.size(), 4);
  if (w == "new_p1") return put(L.new_p1.data(), (int64_t)L.new_p1.size(), 4);
  if (w == "tri_key") return put(L.tri_key.data(), (int64_t)L.tri_key.size(), 8);
  if (w == "tri_id") return put(L.tri_id.data(), (int64_t)L.tri_id.size(), 4);
  if (w == "tri_coef") return put(L.tri_coef.data(), (int64_t)L.tri_coef.size(), 8);
  if (w == "nb_id") return put(L.nb_id.data(), (int64_t)L.nb_id.size(), 4);
  if (w == "nb_ptr") return put(L.nb_ptr.data(), (int64_t)L.nb_ptr.size(), 8);
  if (w == "nb_col") return put(L.nb_col.data(), (int64_t)L.nb_col.size(), 4);
  if (w == "nb_val") return put(L.nb_val.data(), (int64_t)L.nb_val.size(), 8);
  return -1;
}

// x = A_l[J,J]^{-1} b with the factor the host setup stored for level l
// (b, x over the positions in nb_id); -1 if the level has none
int64_t shim_level_nbsolve(void* hp, int l, const double* b, double* x) {
  AuxHost& a = ((Shim*)hp)->aux;
  const int k = l - (a.c + 1);
  if (k < 0 || k >= (int)a.levels.size()) return -1;
  const AuxLevelHost& L = a.levels[k];
  nb::solve(L.nb_fac, b, x);
  return (int64_t)L.nb_id.size();
}

// x = A^{-1} b through the near-boundary block cyclic reduction (A: CSR, m
// rows); returns the number of level-set blocks, or -1 if the factorisation
// failed
int64_t shim_nbsolve(int64_t m, const int64_t* ptr, const int32_t* col, const double* val, const double* b,
                     double* x) {
  nb::Factor F;
  if (!nb::factor(m, ptr, col, val, F)) return -1;
  nb::solve(F, b, x);
  return m ? (int64_t)F.bstart.size() - 1 : 0;
}

// positions of the queries in the sorted keys through the host setup's
// bucket index (-1: absent)
void shim_keyindex(const uint64_t* keys, int64_t n, int bits, const uint64_t* q, int64_t m, int32_t* out) {
  std::vector<uint64_t> k(keys, keys + n);
  KeyIndex idx;
  idx.build(k, bits);
  for (int64_t i = 0; i < m; ++i) out[i] = idx.find(q[i]);
}

}  // extern "C"
