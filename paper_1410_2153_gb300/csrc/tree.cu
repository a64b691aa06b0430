// Cluster tree over element barycenters (Sec. 3.1) on the device:
// barycenter keys, a stable radix sort and level-by-level bisection.
//
// Keys: with the root box [a, a + L)^d (the vertex bounding box widened to a
// square at its min corner) the quantised coordinate of an element is
//   q_k = floor((sum_v p_vk - (d+1) a_k) * 2^D / ((d+1) L)),  clamped to [0, 2^D),
// formed with IEEE round-to-nearest add/sub/mul only (no FMA, no division),
// and the key interleaves the bits of q (bit d*j + k = bit j of q_k).  The
// top d*l bits of a key name the depth-l box holding the barycenter.
#include <cub/cub.cuh>

#include <cmath>

#include "internal.h"

namespace asmg {

namespace {

__device__ __forceinline__ uint64_t spread2(uint64_t v) {  // 32 bits -> even bits of 64
  v &= 0xffffffffULL;
  v = (v | (v << 16)) & 0x0000FFFF0000FFFFULL;
  v = (v | (v << 8)) & 0x00FF00FF00FF00FFULL;
  v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0FULL;
  v = (v | (v << 2)) & 0x3333333333333333ULL;
  v = (v | (v << 1)) & 0x5555555555555555ULL;
  return v;
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

// K1: barycenter sums, quantisation and Morton interleave; also the mesh
// checks that need the elements (index range, orientation).
__global__ void k_keys(int dim, int64_t nv, const double* __restrict__ X, int64_t ne,
                       const int32_t* __restrict__ E, double A0, double A1, double A2, double S, int D,
                       uint64_t* __restrict__ keys, int32_t* __restrict__ ids, int* __restrict__ bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint64_t qmax = (1ULL << D) - 1;
  const double Ak[3] = {A0, A1, A2};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += stride) {
    const int nvert = dim + 1;
    int32_t v[4];
    bool ok = true;
    for (int j = 0; j < nvert; ++j) {
      v[j] = E[e * nvert + j];
      if (v[j] < 0 || v[j] >= nv) ok = false;
    }
    if (!ok) {
      atomicOr(bad, 1);
      keys[e] = 0;
      ids[e] = (int32_t)e;
      continue;
    }
    // orientation
    double det;
    if (dim == 2) {
      double x10 = X[2 * v[1]] - X[2 * v[0]], y10 = X[2 * v[1] + 1] - X[2 * v[0] + 1];
      double x20 = X[2 * v[2]] - X[2 * v[0]], y20 = X[2 * v[2] + 1] - X[2 * v[0] + 1];
      det = x10 * y20 - x20 * y10;
    } else {
      double a[3], b[3], c[3];
      for (int r = 0; r < 3; ++r) {
        a[r] = X[3 * v[1] + r] - X[3 * v[0] + r];
        b[r] = X[3 * v[2] + r] - X[3 * v[0] + r];
        c[r] = X[3 * v[3] + r] - X[3 * v[0] + r];
      }
      det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    if (!(det > 0.0)) atomicOr(bad, 2);
    uint64_t key = 0;
    for (int k = 0; k < dim; ++k) {
      double s = X[(int64_t)v[0] * dim + k];
      for (int j = 1; j < nvert; ++j) s = __dadd_rn(s, X[(int64_t)v[j] * dim + k]);
      double t = __dmul_rn(__dsub_rn(s, Ak[k]), S);
      double f = floor(t);
      if (!(f > 0.0)) f = 0.0;
      uint64_t q = (f >= (double)qmax) ? qmax : (uint64_t)f;
      key |= (dim == 2 ? spread2(q) : spread3(q)) << k;
    }
    keys[e] = key;
    ids[e] = (int32_t)e;
  }
}

// Per-block min/max of each coordinate and finiteness check.
__global__ void k_bbox(int dim, int64_t nv, const double* __restrict__ X, double* __restrict__ part,
                       int* __restrict__ bad) {
  __shared__ double smin[3][256], smax[3][256];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += stride)
    for (int k = 0; k < dim; ++k) {
      double x = X[v * dim + k];
      if (!isfinite(x)) atomicOr(bad, 4);
      mn[k] = fmin(mn[k], x);
      mx[k] = fmax(mx[k], x);
    }
  for (int k = 0; k < 3; ++k) {
    smin[k][threadIdx.x] = mn[k];
    smax[k][threadIdx.x] = mx[k];
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 3; ++k) {
        smin[k][threadIdx.x] = fmin(smin[k][threadIdx.x], smin[k][threadIdx.x + w]);
        smax[k][threadIdx.x] = fmax(smax[k][threadIdx.x], smax[k][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) {
      part[blockIdx.x * 6 + k] = smin[k][0];
      part[blockIdx.x * 6 + 3 + k] = smax[k][0];
    }
}

// Split decision of the nodes at one depth.
__global__ void k_split(int64_t n, const int64_t* __restrict__ b, const int64_t* __restrict__ e, int n_min,
                        int can_split, int32_t* __restrict__ flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (can_split && e[i] - b[i] > n_min) ? 1 : 0;
}

// Children of every split node: boundaries by binary search in the sorted keys.
__global__ void k_children(int64_t n, int dim, int shift, const uint64_t* __restrict__ skeys,
                           const uint64_t* __restrict__ prefix, const int64_t* __restrict__ b,
                           const int64_t* __restrict__ e, const int32_t* __restrict__ flag,
                           const int32_t* __restrict__ pos, uint64_t* __restrict__ cprefix,
                           int64_t* __restrict__ cb, int64_t* __restrict__ ce) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  const int nch = 1 << dim;
  const int64_t base = (int64_t)pos[i] * nch;
  int64_t lo = b[i];
  for (int c = 0; c < nch; ++c) {
    uint64_t cp = (prefix[i] << dim) | (uint64_t)c;
    int64_t hi;
    if (c == nch - 1) {
      hi = e[i];
    } else {
      uint64_t target = (cp + 1) << shift;  // first key of the next child
      int64_t l = lo, r = e[i];
      while (l < r) {
        int64_t m = (l + r) >> 1;
        if (skeys[m] < target) l = m + 1; else r = m;
      }
      hi = l;
    }
    cprefix[base + c] = cp;
    cb[base + c] = lo;
    ce[base + c] = hi;
    lo = hi;
  }
}

int nblocks(int64_t n, int t = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 1 << 20)); }

}  // namespace

void build_tree_gpu(int dim, int64_t nv, const double* dX, int64_t ne, const int32_t* dE, int n_min,
                    cudaStream_t s, TreeResult& out) {
  out.D = dim == 2 ? 31 : 21;
  // root box (Sec. 3.1): minimal square anchored at the vertex minimum
  const int nb = 304;
  DBuf<double> part;
  part.alloc(nb * 6);
  DBuf<int> bad;
  bad.alloc(1);
  bad.zero(s);
  k_bbox<<<nb, 256, 0, s>>>(dim, nv, dX, part.p, bad.p);
  ASMG_CUDA(cudaGetLastError());
  auto hp = part.download(s);
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < dim; ++k) {
      mn[k] = std::min(mn[k], hp[b * 6 + k]);
      mx[k] = std::max(mx[k], hp[b * 6 + 3 + k]);
    }
  out.L = 0;
  for (int k = 0; k < dim; ++k) {
    out.amin[k] = mn[k];
    out.L = std::max(out.L, mx[k] - mn[k]);
  }
  if (!(out.L > 0)) ASMG_FAIL(ASMG_ERR_BAD_MESH, "degenerate vertex bounding box");
  const double S = std::ldexp(1.0, out.D) / (double)(dim + 1) / out.L;
  double Ak[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) Ak[k] = (double)(dim + 1) * out.amin[k];

  DBuf<uint64_t> keys_in;
  DBuf<int32_t> ids_in;
  keys_in.alloc(ne);
  ids_in.alloc(ne);
  k_keys<<<nblocks(ne), 256, 0, s>>>(dim, nv, dX, ne, dE, Ak[0], Ak[1], Ak[2], S, out.D, keys_in.p, ids_in.p, bad.p);
  ASMG_CUDA(cudaGetLastError());
  int hbad = 0;
  ASMG_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
  if (hbad & 1) ASMG_FAIL(ASMG_ERR_BAD_MESH, "element vertex index out of range");
  if (hbad & 2) ASMG_FAIL(ASMG_ERR_BAD_MESH, "element with non-positive orientation");
  if (hbad & 4) ASMG_FAIL(ASMG_ERR_BAD_MESH, "non-finite vertex coordinate");

  // K2: stable LSD radix sort of (key, element id)
  out.keys = std::move(keys_in);
  DBuf<uint64_t> skeys;
  skeys.alloc(ne);
  out.perm.alloc(ne);
  size_t tmp = 0;
  const int end_bit = dim * out.D;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp, out.keys.p, skeys.p, ids_in.p, out.perm.p, ne, 0, end_bit, s);
  DBuf<char> tmpb;
  tmpb.alloc((int64_t)tmp);
  ASMG_CUDA(cub::DeviceRadixSort::SortPairs(tmpb.p, tmp, out.keys.p, skeys.p, ids_in.p, out.perm.p, ne, 0, end_bit, s));

  // K3: level-by-level bisection
  DBuf<uint64_t> pre;
  DBuf<int64_t> b, e;
  pre.alloc(1);
  b.alloc(1);
  e.alloc(1);
  {
    uint64_t z = 0;
    int64_t zb = 0;
    ASMG_CUDA(cudaMemcpyAsync(pre.p, &z, 8, cudaMemcpyHostToDevice, s));
    ASMG_CUDA(cudaMemcpyAsync(b.p, &zb, 8, cudaMemcpyHostToDevice, s));
    ASMG_CUDA(cudaMemcpyAsync(e.p, &ne, 8, cudaMemcpyHostToDevice, s));
  }
  int64_t n = 1;
  out.seg.clear();
  out.split.clear();
  for (int d = 0;; ++d) {
    DBuf<int32_t> flag, pos;
    flag.alloc(n);
    pos.alloc(n + 1);
    k_split<<<nblocks(n), 256, 0, s>>>(n, b.p, e.p, n_min, d < out.D ? 1 : 0, flag.p);
    ASMG_CUDA(cudaGetLastError());
    size_t t2 = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, t2, flag.p, pos.p, n + 1, s);
    // pos has n+1 entries; flag has n: scan n entries and add the last flag for the total
    DBuf<char> tb;
    tb.alloc((int64_t)t2);
    ASMG_CUDA(cub::DeviceScan::ExclusiveSum(tb.p, t2, flag.p, pos.p, n, s));
    auto hpre = pre.download(s);
    auto hb = b.download(s);
    auto he = e.download(s);
    auto hflag = flag.download(s);
    std::vector<int64_t> seg(4 * n);
    std::vector<uint64_t> sp;
    int64_t nsplit = 0;
    for (int64_t i = 0; i < n; ++i) {
      seg[4 * i] = (int64_t)hpre[i];
      seg[4 * i + 1] = hb[i];
      seg[4 * i + 2] = he[i];
      seg[4 * i + 3] = hflag[i];
      if (hflag[i]) {
        sp.push_back(hpre[i]);
        ++nsplit;
      }
    }
    out.seg.push_back(std::move(seg));
    out.split.push_back(std::move(sp));  // prefixes are ascending (Morton order)
    if (nsplit == 0) break;
    const int64_t nn = nsplit << dim;
    DBuf<uint64_t> npre;
    DBuf<int64_t> nbeg, nend;
    npre.alloc(nn);
    nbeg.alloc(nn);
    nend.alloc(nn);
    k_children<<<nblocks(n), 256, 0, s>>>(n, dim, dim * (out.D - d - 1), skeys.p, pre.p, b.p, e.p, flag.p, pos.p,
                                         npre.p, nbeg.p, nend.p);
    ASMG_CUDA(cudaGetLastError());
    pre = std::move(npre);
    b = std::move(nbeg);
    e = std::move(nend);
    n = nn;
  }
  out.split.pop_back();  // the deepest level has no split nodes
}

}  // namespace asmg
