// Device assembly of P1 stiffness matrices (Sec. 2: a_ij = int a grad phi_i .
// grad phi_j) for the fine grid and the auxiliary levels, the consistent mass
// matrix, Jones-Plassmann colouring and the SELL-32 layout of the operators.
#include <cub/cub.cuh>

#include <cmath>
#include <thread>

#include "internal.h"

namespace asmg {

namespace {

int nblk(int64_t n, int t = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 1 << 20)); }

// Element stiffness of a triangle: K_ij = a (b_i b_j + c_i c_j) / (4 |T|),
// b_i = y_{i+1} - y_{i+2}, c_i = x_{i+2} - x_{i+1} (indices mod 3).
__device__ __forceinline__ void tri_K(const double x[3], const double y[3], double a, double K[3][3]) {
  double b[3], c[3];
  for (int i = 0; i < 3; ++i) {
    b[i] = y[(i + 1) % 3] - y[(i + 2) % 3];
    c[i] = x[(i + 2) % 3] - x[(i + 1) % 3];
  }
  double twoA = c[2] * b[1] - c[1] * b[2];  // (x1-x0)(y2-y0) - (x2-x0)(y1-y0)
  double s = a / (2.0 * twoA);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K[i][j] = s * (b[i] * b[j] + c[i] * c[j]);
}

__device__ __forceinline__ void emit9(int64_t t, const int32_t id[3], const double K[3][3], const uint8_t* keep,
                                      uint64_t* key, double* val) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      bool ok = id[i] >= 0 && id[j] >= 0 && (keep == nullptr || keep[id[i]] || keep[id[j]]);
      key[9 * t + 3 * i + j] = ok ? (((uint64_t)(uint32_t)id[i] << 32) | (uint32_t)id[j]) : ~0ULL;
      val[9 * t + 3 * i + j] = ok ? K[i][j] : 0.0;
    }
}

// triangles given by coordinates and row ids
__global__ void k_tri_coo(int64_t ntri, const double* __restrict__ XY, const int32_t* __restrict__ ID,
                          const double* __restrict__ coef, const uint8_t* __restrict__ keep, uint64_t* key,
                          double* val) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  double x[3], y[3];
  int32_t id[3];
  for (int k = 0; k < 3; ++k) {
    x[k] = XY[6 * t + 2 * k];
    y[k] = XY[6 * t + 2 * k + 1];
    id[k] = ID[3 * t + k];
  }
  double K[3][3];
  tri_K(x, y, coef ? coef[t] : 1.0, K);
  emit9(t, id, K, keep, key, val);
}

// triangles of the fine mesh: rows are free-dof numbers
__global__ void k_mesh_coo(int64_t ne, const double* __restrict__ X, const int32_t* __restrict__ E,
                           const int32_t* __restrict__ fv, const double* __restrict__ coef, uint64_t* key,
                           double* val) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne) return;
  double x[3], y[3];
  int32_t id[3];
  for (int k = 0; k < 3; ++k) {
    int32_t v = E[3 * t + k];
    x[k] = X[2 * v];
    y[k] = X[2 * v + 1];
    id[k] = fv[v];
  }
  double K[3][3];
  tri_K(x, y, coef ? coef[t] : 1.0, K);
  emit9(t, id, K, nullptr, key, val);
}

// Element stiffness of a tetrahedron: with edge vectors e_k = p_k - p_0 and
// c_1 = e_2 x e_3, c_2 = e_3 x e_1, c_3 = e_1 x e_2, c_0 = -(c_1 + c_2 + c_3),
// grad lambda_k = c_k / det (det = e_1 . c_1 = 6 |T|), so
// K_ij = a |T| grad lambda_i . grad lambda_j = a (c_i . c_j) / (6 det).
__device__ __forceinline__ void tet_K(const double P[4][3], double a, double K[4][4]) {
  double e[3][3], c[4][3];
  for (int k = 0; k < 3; ++k)
    for (int r = 0; r < 3; ++r) e[k][r] = P[k + 1][r] - P[0][r];
  for (int k = 0; k < 3; ++k) {
    const double* u = e[(k + 1) % 3];
    const double* w = e[(k + 2) % 3];
    c[k + 1][0] = u[1] * w[2] - u[2] * w[1];
    c[k + 1][1] = u[2] * w[0] - u[0] * w[2];
    c[k + 1][2] = u[0] * w[1] - u[1] * w[0];
  }
  for (int r = 0; r < 3; ++r) c[0][r] = -(c[1][r] + c[2][r] + c[3][r]);
  const double det = e[0][0] * c[1][0] + e[0][1] * c[1][1] + e[0][2] * c[1][2];
  const double sc = a / (6.0 * det);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) K[i][j] = sc * (c[i][0] * c[j][0] + c[i][1] * c[j][1] + c[i][2] * c[j][2]);
}

__device__ __forceinline__ void emit16(int64_t t, const int32_t id[4], const double K[4][4], const uint8_t* keep,
                                       uint64_t* key, double* val) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      bool ok = id[i] >= 0 && id[j] >= 0 && (keep == nullptr || keep[id[i]] || keep[id[j]]);
      key[16 * t + 4 * i + j] = ok ? (((uint64_t)(uint32_t)id[i] << 32) | (uint32_t)id[j]) : ~0ULL;
      val[16 * t + 4 * i + j] = ok ? K[i][j] : 0.0;
    }
}

// tetrahedra given by coordinates and row ids
__global__ void k_tet_coo(int64_t ntet, const double* __restrict__ XYZ, const int32_t* __restrict__ ID,
                          const double* __restrict__ coef, const uint8_t* __restrict__ keep, uint64_t* key,
                          double* val) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ntet) return;
  double P[4][3];
  int32_t id[4];
  for (int k = 0; k < 4; ++k) {
    for (int r = 0; r < 3; ++r) P[k][r] = XYZ[12 * t + 3 * k + r];
    id[k] = ID[4 * t + k];
  }
  double K[4][4];
  tet_K(P, coef ? coef[t] : 1.0, K);
  emit16(t, id, K, keep, key, val);
}

// tetrahedra of the fine mesh: rows are free-dof numbers
__global__ void k_mesh_coo3(int64_t ne, const double* __restrict__ X, const int32_t* __restrict__ E,
                            const int32_t* __restrict__ fv, const double* __restrict__ coef, uint64_t* key,
                            double* val) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne) return;
  double P[4][3];
  int32_t id[4];
  for (int k = 0; k < 4; ++k) {
    int32_t v = E[4 * t + k];
    for (int r = 0; r < 3; ++r) P[k][r] = X[3 * (int64_t)v + r];
    id[k] = fv[v];
  }
  double K[4][4];
  tet_K(P, coef ? coef[t] : 1.0, K);
  emit16(t, id, K, nullptr, key, val);
}

HostCSR coo_to_csr(int64_t m, DBuf<uint64_t>& key, DBuf<double>& val, int64_t nrows, cudaStream_t s) {
  DBuf<uint64_t> skey;
  DBuf<double> sval;
  skey.alloc(m);
  sval.alloc(m);
  size_t tmp = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp, key.p, skey.p, val.p, sval.p, m, 0, 64, s);
  DBuf<char> tb;
  tb.alloc((int64_t)tmp);
  ASMG_CUDA(cub::DeviceRadixSort::SortPairs(tb.p, tmp, key.p, skey.p, val.p, sval.p, m, 0, 64, s));
  key.release();
  val.release();
  DBuf<uint64_t> ukey;
  DBuf<double> uval;
  DBuf<int64_t> nu;
  ukey.alloc(m);
  uval.alloc(m);
  nu.alloc(1);
  size_t tmp2 = 0;
  cub::DeviceReduce::ReduceByKey(nullptr, tmp2, skey.p, ukey.p, sval.p, uval.p, nu.p, ::cuda::std::plus<double>(), m, s);
  DBuf<char> tb2;
  tb2.alloc((int64_t)tmp2);
  ASMG_CUDA(cub::DeviceReduce::ReduceByKey(tb2.p, tmp2, skey.p, ukey.p, sval.p, uval.p, nu.p, ::cuda::std::plus<double>(), m, s));
  auto hn = nu.download(s);
  int64_t u = hn[0];
  std::vector<uint64_t> hk(u);
  std::vector<double> hv(u);
  if (u) {
    ASMG_CUDA(cudaMemcpyAsync(hk.data(), ukey.p, 8 * u, cudaMemcpyDeviceToHost, s));
    ASMG_CUDA(cudaMemcpyAsync(hv.data(), uval.p, 8 * u, cudaMemcpyDeviceToHost, s));
    ASMG_CUDA(cudaStreamSynchronize(s));
  }
  if (u && hk[u - 1] == ~0ULL) --u;  // dropped entries sort last
  HostCSR A;
  A.nr = nrows;
  A.nc = nrows;
  A.ptr.assign(nrows + 1, 0);
  A.col.resize(u);
  A.val.resize(u);
  for (int64_t k = 0; k < u; ++k) {
    A.ptr[(hk[k] >> 32) + 1]++;
    A.col[k] = (int32_t)(hk[k] & 0xffffffffULL);
    A.val[k] = hv[k];
  }
  for (int64_t i = 0; i < nrows; ++i) A.ptr[i + 1] += A.ptr[i];
  return A;
}

// consistent P1 mass matrix applied to nodal values, gathered per vertex:
// b_v = sum over the elements T around v (ascending element index) of
// |T|/12 (f_v + sum_j f_j) in 2D, |T|/20 (f_v + sum_j f_j) in 3D.  Each sum
// runs in a fixed order, so the result is the same bit for bit on every run
// (no atomics).  v2e: element indices around each vertex (CSR by vertex).
__global__ void k_mass_gather(int64_t nv, const int64_t* __restrict__ v2e_ptr, const int32_t* __restrict__ v2e,
                              const double* __restrict__ X, const int32_t* __restrict__ E,
                              const double* __restrict__ f, double* __restrict__ b) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double acc = 0;
  const double fv = f[v];
  for (int64_t p = v2e_ptr[v]; p < v2e_ptr[v + 1]; ++p) {
    const int64_t t = v2e[p];
    const int32_t v0 = E[3 * t], v1 = E[3 * t + 1], v2 = E[3 * t + 2];
    const double area = 0.5 * ((X[2 * v1] - X[2 * v0]) * (X[2 * v2 + 1] - X[2 * v0 + 1]) -
                               (X[2 * v2] - X[2 * v0]) * (X[2 * v1 + 1] - X[2 * v0 + 1]));
    const double sum = f[v0] + f[v1] + f[v2];
    acc += area / 12.0 * (sum + fv);
  }
  b[v] = acc;
}

__global__ void k_mass_gather3(int64_t nv, const int64_t* __restrict__ v2e_ptr, const int32_t* __restrict__ v2e,
                               const double* __restrict__ X, const int32_t* __restrict__ E,
                               const double* __restrict__ f, double* __restrict__ b) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double acc = 0;
  const double fv = f[v];
  for (int64_t p = v2e_ptr[v]; p < v2e_ptr[v + 1]; ++p) {
    const int64_t t = v2e[p];
    int32_t w[4];
    double P[4][3];
    for (int k = 0; k < 4; ++k) {
      w[k] = E[4 * t + k];
      for (int r = 0; r < 3; ++r) P[k][r] = X[3 * (int64_t)w[k] + r];
    }
    double e[3][3];
    for (int k = 0; k < 3; ++k)
      for (int r = 0; r < 3; ++r) e[k][r] = P[k + 1][r] - P[0][r];
    const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) +
                       e[0][1] * (e[1][2] * e[2][0] - e[1][0] * e[2][2]) +
                       e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    const double sum = f[w[0]] + f[w[1]] + f[w[2]] + f[w[3]];
    acc += det / 120.0 * (sum + fv);  // |T| / 20
  }
  b[v] = acc;
}

// dL/da_e = -lambda_e^T K_e^(1) u_e, times scale[e] when scale is given
// (scale = a: the derivative with respect to g_e for a = exp(g))
__global__ void k_elem_grad3(int64_t ne, const double* __restrict__ X, const int32_t* __restrict__ E,
                             const double* __restrict__ u, const double* __restrict__ lam,
                             const double* __restrict__ scale, double* __restrict__ g) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne) return;
  double P[4][3], ue[4], le[4];
  for (int k = 0; k < 4; ++k) {
    int32_t v = E[4 * t + k];
    for (int r = 0; r < 3; ++r) P[k][r] = X[3 * (int64_t)v + r];
    ue[k] = u[v];
    le[k] = lam[v];
  }
  double K[4][4];
  tet_K(P, 1.0, K);
  double s = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) s += le[i] * K[i][j] * ue[j];
  g[t] = scale ? -(scale[t] * s) : -s;
}

// dL/da_e = -lambda_e^T K_e^(1) u_e (times scale[e] when given), triangles
__global__ void k_elem_grad(int64_t ne, const double* __restrict__ X, const int32_t* __restrict__ E,
                            const double* __restrict__ u, const double* __restrict__ lam,
                            const double* __restrict__ scale, double* __restrict__ g) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne) return;
  double x[3], y[3], ue[3], le[3];
  for (int k = 0; k < 3; ++k) {
    int32_t v = E[3 * t + k];
    x[k] = X[2 * v];
    y[k] = X[2 * v + 1];
    ue[k] = u[v];
    le[k] = lam[v];
  }
  double K[3][3];
  tri_K(x, y, 1.0, K);
  double s = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) s += le[i] * K[i][j] * ue[j];
  g[t] = scale ? -(scale[t] * s) : -s;
}

// splitmix64 (published constants of Steele, Lea and Flood / Vigna).
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

// a coupling of the colouring graph: |a_vw| > 1e-12 sqrt(a_vv a_ww), w != v
__device__ __forceinline__ bool coupled(int32_t v, int32_t w, double a, const double* __restrict__ diag) {
  return w != v && fabs(a) > 1e-12 * sqrt(diag[v] * diag[w]);
}

__global__ void k_jp_cand(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const double* __restrict__ diag,
                          const uint8_t* __restrict__ inset, const uint64_t* __restrict__ pk,
                          const int32_t* __restrict__ colour, uint8_t* __restrict__ cand) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n) return;
  cand[v] = 0;
  if (!inset[v] || colour[v] >= 0) return;
  const uint64_t hv = mix64(pk[v]), kv = pk[v];
  for (int64_t p = ptr[v]; p < ptr[v + 1]; ++p) {
    int32_t w = col[p];
    if (!inset[w] || colour[w] >= 0 || !coupled((int32_t)v, w, val[p], diag)) continue;
    uint64_t hw = mix64(pk[w]);
    if (hw > hv || (hw == hv && pk[w] > kv)) return;
  }
  cand[v] = 1;
}

__global__ void k_jp_assign(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const double* __restrict__ diag,
                            const uint8_t* __restrict__ inset, const uint8_t* __restrict__ cand,
                            int32_t* __restrict__ colour, unsigned long long* __restrict__ ncol, int* bad) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n || !cand[v]) return;
  uint64_t used[2] = {0, 0};
  for (int64_t p = ptr[v]; p < ptr[v + 1]; ++p) {
    int32_t w = col[p];
    if (!inset[w] || !coupled((int32_t)v, w, val[p], diag)) continue;
    int32_t c = colour[w];
    if (c >= 0 && c < 128) used[c >> 6] |= 1ULL << (c & 63);
  }
  int c = 0;
  while (c < 128 && ((used[c >> 6] >> (c & 63)) & 1)) ++c;
  if (c >= 128) atomicOr(bad, 1);
  colour[v] = c;
  atomicAdd(ncol, 1ULL);
}

// one class of an iterated-greedy round: nodes of class c take the smallest
// colour unused by their neighbours of the classes already visited (> c)
__global__ void k_ig_class(int64_t n, int32_t c, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ diag,
                           const uint8_t* __restrict__ inset, const int32_t* __restrict__ colour,
                           int32_t* __restrict__ next, int* bad) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n || !inset[v] || colour[v] != c) return;
  uint64_t used[2] = {0, 0};
  for (int64_t p = ptr[v]; p < ptr[v + 1]; ++p) {
    int32_t w = col[p];
    if (!inset[w] || colour[w] <= c || !coupled((int32_t)v, w, val[p], diag)) continue;
    int32_t k = next[w];
    if (k >= 0 && k < 128) used[k >> 6] |= 1ULL << (k & 63);
  }
  int k = 0;
  while (k < 128 && ((used[k >> 6] >> (k & 63)) & 1)) ++k;
  if (k >= 128) atomicOr(bad, 1);
  next[v] = k;
}

}  // namespace

HostCSR assemble_simplices(int dim, int64_t n, const double* dP, const int32_t* dID, const double* dCoef,
                           const uint8_t* dKeep, int64_t nrows, cudaStream_t s) {
  if (n == 0) {
    HostCSR A;
    A.nr = A.nc = nrows;
    A.ptr.assign(nrows + 1, 0);
    return A;
  }
  const int64_t m = (int64_t)(dim + 1) * (dim + 1) * n;
  DBuf<uint64_t> key;
  DBuf<double> val;
  key.alloc(m);
  val.alloc(m);
  if (dim == 2)
    k_tri_coo<<<nblk(n), 256, 0, s>>>(n, dP, dID, dCoef, dKeep, key.p, val.p);
  else
    k_tet_coo<<<nblk(n), 256, 0, s>>>(n, dP, dID, dCoef, dKeep, key.p, val.p);
  ASMG_CUDA(cudaGetLastError());
  return coo_to_csr(m, key, val, nrows, s);
}

HostCSR assemble_mesh(int dim, int64_t ne, const double* dX, const int32_t* dE, const int32_t* dFree,
                      const double* dCoef, int64_t nfree, cudaStream_t s) {
  const int64_t m = (int64_t)(dim + 1) * (dim + 1) * ne;
  DBuf<uint64_t> key;
  DBuf<double> val;
  key.alloc(m);
  val.alloc(m);
  if (dim == 2)
    k_mesh_coo<<<nblk(ne), 256, 0, s>>>(ne, dX, dE, dFree, dCoef, key.p, val.p);
  else
    k_mesh_coo3<<<nblk(ne), 256, 0, s>>>(ne, dX, dE, dFree, dCoef, key.p, val.p);
  ASMG_CUDA(cudaGetLastError());
  return coo_to_csr(m, key, val, nfree, s);
}

void mass_apply_gpu(int dim, int64_t nv, const int64_t* v2e_ptr, const int32_t* v2e, const double* dX,
                    const int32_t* dE, const double* df, double* db, cudaStream_t s) {
  if (dim == 2)
    k_mass_gather<<<nblk(nv), 256, 0, s>>>(nv, v2e_ptr, v2e, dX, dE, df, db);
  else
    k_mass_gather3<<<nblk(nv), 256, 0, s>>>(nv, v2e_ptr, v2e, dX, dE, df, db);
  ASMG_CUDA(cudaGetLastError());
}

void element_grad_gpu(int dim, int64_t ne, const double* dX, const int32_t* dE, const double* du, const double* dl,
                      const double* dscale, double* dg, cudaStream_t s) {
  if (dim == 2)
    k_elem_grad<<<nblk(ne), 256, 0, s>>>(ne, dX, dE, du, dl, dscale, dg);
  else
    k_elem_grad3<<<nblk(ne), 256, 0, s>>>(ne, dX, dE, du, dl, dscale, dg);
  ASMG_CUDA(cudaGetLastError());
}

std::vector<int32_t> jp_colour_gpu(const HostCSR& A, const std::vector<uint8_t>& inset,
                                   const std::vector<uint64_t>& prio_key, cudaStream_t s) {
  const int64_t n = A.nr;
  std::vector<int32_t> out(n, -1);
  int64_t todo = 0;
  for (auto f : inset) todo += f;
  if (n == 0 || todo == 0) return out;
  std::vector<double> diag(n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
      if (A.col[p] == i) diag[i] = A.val[p];
  DBuf<int64_t> ptr;
  DBuf<int32_t> col, colour, next;
  DBuf<double> val, dg;
  DBuf<uint8_t> ins, cand;
  DBuf<uint64_t> pk;
  DBuf<unsigned long long> cnt;
  DBuf<int> bad;
  ptr.upload(A.ptr, s);
  col.upload(A.col, s);
  val.upload(A.val, s);
  dg.upload(diag, s);
  ins.upload(inset, s);
  pk.upload(prio_key, s);
  colour.upload(out, s);
  cand.alloc(n);
  cnt.alloc(1);
  cnt.zero(s);
  bad.alloc(1);
  bad.zero(s);
  unsigned long long done = 0;
  for (int round = 0; round < 100000 && (int64_t)done < todo; ++round) {
    k_jp_cand<<<nblk(n), 256, 0, s>>>(n, ptr.p, col.p, val.p, dg.p, ins.p, pk.p, colour.p, cand.p);
    k_jp_assign<<<nblk(n), 256, 0, s>>>(n, ptr.p, col.p, val.p, dg.p, ins.p, cand.p, colour.p, cnt.p, bad.p);
    ASMG_CUDA(cudaGetLastError());
    ASMG_CUDA(cudaMemcpyAsync(&done, cnt.p, 8, cudaMemcpyDeviceToHost, s));
    ASMG_CUDA(cudaStreamSynchronize(s));
  }
  if ((int64_t)done != todo) ASMG_FAIL(ASMG_ERR_CUDA, "colouring did not finish");
  // three rounds of iterated greedy recolouring, classes in descending order
  next.alloc(n);
  for (int round = 0; round < 3; ++round) {
    std::vector<int32_t> hc = colour.download(s);
    int32_t ncol = 0;
    for (int64_t v = 0; v < n; ++v)
      if (inset[v]) ncol = std::max(ncol, hc[v] + 1);
    ASMG_CUDA(cudaMemsetAsync(next.p, 0xff, 4 * n, s));
    for (int32_t c = ncol - 1; c >= 0; --c)
      k_ig_class<<<nblk(n), 256, 0, s>>>(n, c, ptr.p, col.p, val.p, dg.p, ins.p, colour.p, next.p, bad.p);
    ASMG_CUDA(cudaGetLastError());
    ASMG_CUDA(cudaMemcpyAsync(colour.p, next.p, 4 * n, cudaMemcpyDeviceToDevice, s));
  }
  auto hb = bad.download(s);
  if (hb[0]) ASMG_FAIL(ASMG_ERR_UNSUPPORTED, "more than 128 colours needed");
  return colour.download(s);
}

// Host-side packing, parallel over slices (slice widths, then the column-
// major fill of each slice).
template <class T>
void sell_build(Sell<T>& S, const HostCSR& rows, int32_t pad_col, cudaStream_t s) {
  const int64_t nr = rows.nr;
  S.nslices = (nr + SELL_C - 1) / SELL_C;
  S.nrows = S.nslices * SELL_C;
  const unsigned nt = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), S.nslices / 4096));
  auto par = [&](auto body) {
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
      th.emplace_back([&, t] { body(S.nslices * t / nt, S.nslices * (t + 1) / nt); });
    for (auto& x : th) x.join();
  };
  std::vector<int64_t> off(S.nslices + 1, 0);
  par([&](int64_t s0, int64_t s1) {
    for (int64_t sl = s0; sl < s1; ++sl) {
      int64_t w = 0;
      for (int64_t r = sl * SELL_C; r < std::min(nr, (sl + 1) * SELL_C); ++r)
        w = std::max(w, rows.ptr[r + 1] - rows.ptr[r]);
      off[sl + 1] = w * SELL_C;
    }
  });
  for (int64_t sl = 0; sl < S.nslices; ++sl) off[sl + 1] += off[sl];
  S.nnz = off[S.nslices];
  S.nnz_real = rows.ptr[nr];
  std::vector<int32_t> col(S.nnz, pad_col);
  std::vector<T> val(S.nnz, (T)0);
  par([&](int64_t s0, int64_t s1) {
    for (int64_t r = s0 * SELL_C; r < std::min(nr, s1 * SELL_C); ++r) {
      const int64_t sl = r / SELL_C, t = r % SELL_C;
      int64_t k = 0;
      for (int64_t p = rows.ptr[r]; p < rows.ptr[r + 1]; ++p, ++k) {
        col[off[sl] + k * SELL_C + t] = rows.col[p];
        val[off[sl] + k * SELL_C + t] = (T)rows.val[p];
      }
    }
  });
  S.off.upload(off, s);
  S.col.upload(col, s);
  S.val.upload(val, s);
  ASMG_CUDA(cudaStreamSynchronize(s));
}

template void sell_build<float>(Sell<float>&, const HostCSR&, int32_t, cudaStream_t);
template void sell_build<double>(Sell<double>&, const HostCSR&, int32_t, cudaStream_t);

__global__ void k_to_bf16(int64_t n, const float* __restrict__ x, bf16v* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i].bits = bf16_bits(x[i]);
}

void sell_bf16(Sell<float>& S, cudaStream_t s) {
  S.v16.alloc(std::max<int64_t>(S.nnz, 1));
  if (S.nnz > 0) {
    k_to_bf16<<<(unsigned)((S.nnz + 255) / 256), 256, 0, s>>>(S.nnz, S.val.p, S.v16.p);
    ASMG_CUDA(cudaGetLastError());
  }
  ASMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace asmg
