// Scott-Zhang transfer (Sec. 4.1), one row per free fine vertex (sz_row.h):
// 2D rows on the device, one thread per row; 3D rows on host threads.
//
// Rows have no fixed length, so the rows are computed twice: the first pass
// counts the (simplex, vertex) contributions of each row, the second writes
// them into the scanned slots; each row is then sorted by column (stable:
// duplicates are added in traversal order) and merged, and the merged rows
// are compacted.
#include <algorithm>
#include <atomic>
#include <thread>

#include <cub/cub.cuh>

#include "internal.h"
#include "sz_row.h"

namespace asmg {

namespace {

using namespace szrow;

__global__ void k_sigma(int64_t ne, int64_t nv, int nvpe, const int32_t* __restrict__ E, int32_t* __restrict__ sigma) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  for (int k = 0; k < nvpe; ++k) {
    const int32_t v = E[nvpe * e + k];
    if (v >= 0 && v < nv) atomicMin(&sigma[v], (int32_t)e);
  }
}

// mode 0: count the contributions of every row; mode 1: write them (err 2
// if a row's count changed between the passes)
template <int DIM>
__global__ void k_sz_pass(SZDev t, int mode, const int64_t* __restrict__ off, int64_t* __restrict__ cnt,
                          int32_t* __restrict__ col, double* __restrict__ val, int* __restrict__ err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= t.n) return;
  bool stack_ok = true;
  if (!sz_pass<DIM>(t, i, mode, off, cnt, col, val, &stack_ok)) atomicExch(err, 2);
  if (!stack_ok) atomicExch(err, 1);
}

__global__ void k_sz_merge(int64_t n, const int64_t* __restrict__ off, int32_t* __restrict__ col,
                           double* __restrict__ val, int64_t* __restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  cnt[i] = sz_merge(i, off, cnt, col, val);
}

__global__ void k_sz_compact(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const int64_t* __restrict__ foff,
                             int32_t* __restrict__ row_o, int32_t* __restrict__ col_o, double* __restrict__ val_o) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = off[i];
  for (int64_t p = foff[i]; p < foff[i + 1]; ++p) {
    row_o[p] = (int32_t)i;
    col_o[p] = col[b + p - foff[i]];
    val_o[p] = val[b + p - foff[i]];
  }
}

void exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  size_t tmp = 0;
  ASMG_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, in, out, n, s));
  DBuf<uint8_t> tb;
  tb.alloc((int64_t)tmp);
  ASMG_CUDA(cub::DeviceScan::ExclusiveSum(tb.p, tmp, in, out, n, s));
}

// 3D rows on host threads: each row in one pass (a local list), rows in
// contiguous ranges per thread, parts appended in thread order
void transfer_host3(const MeshHost& mesh, const std::vector<int32_t>& vertex_of_free, const SZTable& tab,
                    Triplets& P) {
  const int64_t n = (int64_t)vertex_of_free.size();
  std::vector<int32_t> sigma((size_t)mesh.nv, INT32_MAX);
  for (int64_t e = 0; e < mesh.ne; ++e)
    for (int k = 0; k < 4; ++k) {
      const int32_t v = mesh.E[4 * e + k];
      sigma[v] = std::min(sigma[v], (int32_t)e);
    }
  SZDev t;
  t.dim = 3;
  t.D = tab.D;
  for (int a = 0; a < 3; ++a) t.amin[a] = tab.amin[a];
  t.L = tab.L;
  t.sc = std::ldexp(1.0, tab.D) / tab.L;
  t.node_key = tab.node_key.data();
  t.node_pay = tab.node_pay.data();
  t.leaf_first = tab.leaf_first.data();
  t.simp_key = tab.simp_key.data();
  t.simp_col = tab.simp_col.data();
  t.X = mesh.X.data();
  t.E = mesh.E.data();
  t.sigma = sigma.data();
  t.vof = vertex_of_free.data();
  t.n = n;
  t.nnode = (int64_t)tab.node_key.size();
  t.nleaf = (int64_t)tab.leaf_first.size() - 1;
  t.nsimp = (int64_t)tab.simp_col.size() / 4;
  t.nv = mesh.nv;
  t.ne = mesh.ne;
  unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  if (n < 2048) nt = 1;
  std::vector<Triplets> parts(nt);
  std::atomic<int> bad(0);
  std::vector<std::thread> th;
  for (unsigned w = 0; w < nt; ++w)
    th.emplace_back([&, w] {
      Triplets& mine = parts[w];
      std::vector<std::pair<int32_t, double>> row;
      for (int64_t i = n * w / nt; i < n * (w + 1) / nt; ++i) {
        row.clear();
        if (!sz_row<3>(t, i, true, [&](int32_t c, double v) { row.push_back({c, v}); })) bad = 1;
        std::stable_sort(row.begin(), row.end(), [](const std::pair<int32_t, double>& a,
                                                    const std::pair<int32_t, double>& b) { return a.first < b.first; });
        for (size_t k = 0; k < row.size();) {
          size_t j = k;
          double sum = 0;
          while (j < row.size() && row[j].first == row[k].first) sum += row[j++].second;
          mine.r.push_back((int32_t)i);
          mine.c.push_back(row[k].first);
          mine.v.push_back(sum);
          k = j;
        }
      }
    });
  for (auto& x : th) x.join();
  if (bad) ASMG_FAIL(ASMG_ERR_CUDA, "transfer: tree traversal stack exceeded or index out of range");
  for (auto& p : parts) {
    P.r.insert(P.r.end(), p.r.begin(), p.r.end());
    P.c.insert(P.c.end(), p.c.begin(), p.c.end());
    P.v.insert(P.v.end(), p.v.begin(), p.v.end());
  }
}

}  // namespace

void build_transfer(const MeshHost& mesh, const double* dX, const int32_t* dE,
                        const std::vector<int32_t>& vertex_of_free, const SZTable& tab, Triplets& P, cudaStream_t s) {
  const int64_t n = (int64_t)vertex_of_free.size();
  P = Triplets();
  if (n == 0) return;
  if (tab.node_key.size() >= (size_t)INT32_MAX) ASMG_FAIL(ASMG_ERR_UNSUPPORTED, "closed tree too large");
  if (tab.D > STACK) ASMG_FAIL(ASMG_ERR_UNSUPPORTED, "tree too deep for the transfer kernel");
  if (tab.dim == 3) {
    // tetrahedron clipping is FP64 work whose piece count varies from pair to
    // pair: on this part the host threads beat the device (measured at 129^3:
    // 4.4 s against 10.3 s), so 3D rows run the same row code on the host
    transfer_host3(mesh, vertex_of_free, tab, P);
    return;
  }
  DBuf<uint64_t> nkey, skey;
  DBuf<int64_t> npay, lfirst;
  DBuf<int32_t> scol, sigma, vof;
  nkey.upload(tab.node_key, s);
  npay.upload(tab.node_pay, s);
  lfirst.upload(tab.leaf_first, s);
  skey.upload(tab.simp_key, s);
  scol.upload(tab.simp_col, s);
  vof.upload(vertex_of_free, s);
  std::vector<int32_t> big((size_t)mesh.nv, INT32_MAX);
  sigma.upload(big, s);
  const int nvpe = tab.dim + 1;
  const int TB = 128;
  k_sigma<<<(unsigned)((mesh.ne + 255) / 256), 256, 0, s>>>(mesh.ne, mesh.nv, nvpe, dE, sigma.p);
  ASMG_CUDA(cudaGetLastError());
  SZDev t;
  t.dim = tab.dim;
  t.D = tab.D;
  for (int a = 0; a < 3; ++a) t.amin[a] = tab.amin[a];
  t.L = tab.L;
  t.sc = std::ldexp(1.0, tab.D) / tab.L;
  t.node_key = nkey.p;
  t.node_pay = npay.p;
  t.leaf_first = lfirst.p;
  t.simp_key = skey.p;
  t.simp_col = scol.p;
  t.X = dX;
  t.E = dE;
  t.sigma = sigma.p;
  t.vof = vof.p;
  t.n = n;
  t.nnode = (int64_t)tab.node_key.size();
  t.nleaf = (int64_t)tab.leaf_first.size() - 1;
  t.nsimp = (int64_t)tab.simp_col.size() / nvpe;
  t.nv = mesh.nv;
  t.ne = mesh.ne;
  if (t.nleaf < 1 || tab.node_pay.size() != tab.node_key.size() || tab.simp_key.size() != tab.simp_col.size())
    ASMG_FAIL(ASMG_ERR_CUDA, "transfer: inconsistent tree table");
  const unsigned nb = (unsigned)((n + TB - 1) / TB);
  DBuf<int64_t> cnt, off;
  DBuf<int> err;
  cnt.alloc(n + 1);
  off.alloc(n + 1);
  err.alloc(1);
  err.zero(s);
  ASMG_CUDA(cudaMemsetAsync(cnt.p + n, 0, sizeof(int64_t), s));
  k_sz_pass<2><<<nb, TB, 0, s>>>(t, 0, nullptr, cnt.p, nullptr, nullptr, err.p);
  ASMG_CUDA(cudaGetLastError());
  if (err.download(s)[0]) ASMG_FAIL(ASMG_ERR_CUDA, "transfer: tree traversal stack exceeded or index out of range");
  exclusive_scan(cnt.p, off.p, n + 1, s);
  int64_t nraw = 0;
  ASMG_CUDA(cudaMemcpyAsync(&nraw, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
  DBuf<int32_t> col;
  DBuf<double> val;
  col.alloc(nraw);
  val.alloc(nraw);
  k_sz_pass<2><<<nb, TB, 0, s>>>(t, 1, off.p, cnt.p, col.p, val.p, err.p);
  ASMG_CUDA(cudaGetLastError());
  if (const int e = err.download(s)[0])
    ASMG_FAIL(ASMG_ERR_CUDA, "transfer: %s", e == 1 ? "tree traversal stack exceeded or index out of range" : "row count changed between passes");
  k_sz_merge<<<nb, TB, 0, s>>>(n, off.p, col.p, val.p, cnt.p);
  ASMG_CUDA(cudaGetLastError());
  DBuf<int64_t> foff;
  foff.alloc(n + 1);
  exclusive_scan(cnt.p, foff.p, n + 1, s);
  int64_t nnz = 0;
  ASMG_CUDA(cudaMemcpyAsync(&nnz, foff.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
  DBuf<int32_t> ro, co;
  DBuf<double> vo;
  ro.alloc(nnz);
  co.alloc(nnz);
  vo.alloc(nnz);
  k_sz_compact<<<nb, TB, 0, s>>>(n, off.p, col.p, val.p, foff.p, ro.p, co.p, vo.p);
  ASMG_CUDA(cudaGetLastError());
  P.r = ro.download(s);
  P.c = co.download(s);
  P.v = vo.download(s);
  // every entry must name a free row and a finest aux node
  int64_t ncol = 0;
  for (int32_t c : tab.simp_col) ncol = std::max<int64_t>(ncol, (int64_t)c + 1);
  for (size_t k = 0; k < P.r.size(); ++k)
    if (P.r[k] < 0 || P.r[k] >= n || P.c[k] < 0 || P.c[k] >= ncol || !std::isfinite(P.v[k]))
      ASMG_FAIL(ASMG_ERR_CUDA, "transfer: entry %lld (row %d, column %d) out of range", (long long)k, P.r[k], P.c[k]);
}

}  // namespace asmg
