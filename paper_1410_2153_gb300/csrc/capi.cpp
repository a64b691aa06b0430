// C ABI entry points (include/asmg.h) and the setup pipeline.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstring>
#include <exception>
#include <numeric>
#include <thread>
#include <unordered_map>

#include "handle.h"

using namespace asmg;

namespace {

thread_local std::string g_err;

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

bool is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
std::vector<T> to_host(const T* p, int64_t n, cudaStream_t s) {
  std::vector<T> h((size_t)n);
  if (n == 0) return h;
  if (is_device(p)) {
    ASMG_CUDA(cudaMemcpyAsync(h.data(), p, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
    ASMG_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(h.data(), p, sizeof(T) * n);
  }
  return h;
}

void copy_in(double* dst, const double* src, int64_t n, cudaStream_t s) {
  ASMG_CUDA(cudaMemcpyAsync(dst, src, 8 * n, is_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

void copy_out(double* dst, const double* src, int64_t n, cudaStream_t s) {
  ASMG_CUDA(cudaMemcpyAsync(dst, src, 8 * n, is_device(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

int64_t pad32(int64_t n) { return (n + 31) / 32 * 32; }

// Temporally blocked sweeps (asmg_params::tile_rows = 0): tile sizes tried in
// order (own rows per tile) on levels of two colour classes and on levels of
// more (whose longer dependency chains make deeper halos, which larger tiles
// amortise: measured on graded 2049^2, 512-row tiles run the 5-class levels
// 10-35% faster than 256-row ones, the 2-class levels no faster), the shared
// memory a tile may use (two thread blocks per SM), and the largest halo
// accepted, as a multiple of the own rows.
constexpr int TILE_SIZES_2COL[] = {256};
constexpr int TILE_SIZES_MULTI[] = {512, 256};
constexpr size_t TILE_SMEM = 110 * 1024;
constexpr size_t TILE_SMEM_MAX = TILE_SMEM_LIMIT;  // one thread block per SM
constexpr double TILE_MAX_HALO = 1.5;

// f(begin, end) over contiguous ranges of [0, n) on host threads
template <class F>
void host_for(int64_t n, F f) {
  unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < (1 << 15)) nt = 1;
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) th.emplace_back([&, t] { f(n * t / nt, n * (t + 1) / nt); });
  for (auto& x : th) x.join();
}

// rows of a host CSR selected and renumbered: out row k = A row sel[k] (or
// empty when sel[k] < 0), columns mapped by cmap (dropped when < 0); rows
// counted, then filled, in parallel
HostCSR select_rows(const HostCSR& A, const std::vector<int64_t>& sel, const std::vector<int32_t>* cmap,
                    const std::vector<uint8_t>* colkeep) {
  HostCSR B;
  B.nr = (int64_t)sel.size();
  B.nc = A.nc;
  B.ptr.assign(B.nr + 1, 0);
  auto keep = [&](int64_t p) {
    // couplings that vanish by symmetry are not stored
    return !(colkeep && !(*colkeep)[A.col[p]]) && A.val[p] != 0.0;
  };
  host_for(B.nr, [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; ++k) {
      int64_t c = 0;
      if (sel[k] >= 0)
        for (int64_t p = A.ptr[sel[k]]; p < A.ptr[sel[k] + 1]; ++p) c += keep(p);
      B.ptr[k + 1] = c;
    }
  });
  for (int64_t k = 0; k < B.nr; ++k) B.ptr[k + 1] += B.ptr[k];
  B.col.resize(B.ptr[B.nr]);
  B.val.resize(B.ptr[B.nr]);
  host_for(B.nr, [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; ++k) {
      if (sel[k] < 0) continue;
      int64_t q = B.ptr[k];
      for (int64_t p = A.ptr[sel[k]]; p < A.ptr[sel[k] + 1]; ++p)
        if (keep(p)) {
          B.col[q] = cmap ? (*cmap)[A.col[p]] : A.col[p];
          B.val[q] = A.val[p];
          ++q;
        }
    }
  });
  return B;
}

// Shared-memory form of a small level: local numbering (smoothing nodes in
// colour order first, then the other rows of E_l), 16-bit local columns.
template <class T>
void build_small(const AuxLevelHost& L, const HostCSR& Arows, const std::vector<uint8_t>& inset,
                 const std::vector<int64_t>& sel, const std::vector<int64_t>& rsel, const std::vector<T>& dinv_pad,
                 const std::vector<int32_t>& pid, const std::vector<int32_t>& pptr, const std::vector<int32_t>& child,
                 bool bf16, AuxLevelDev<T>& D, cudaStream_t s) {
  SmallLevelDev<T>& S = D.small;
  S.ok = false;
  std::vector<int32_t> gid;
  std::vector<T> dinv;
  std::vector<int> cs(1, 0);
  for (int c = 0; c < D.ncolours; ++c) {
    for (int64_t k = D.cstart[c]; k < D.cstart[c + 1]; ++k)
      if (sel[k] >= 0) {
        gid.push_back((int32_t)sel[k]);
        dinv.push_back(dinv_pad[k]);
      }
    cs.push_back((int)gid.size());
  }
  const int mS = (int)gid.size();
  for (int64_t r : rsel)
    if (r >= 0 && !inset[r]) gid.push_back((int32_t)r);
  const int mE = (int)gid.size();
  if (mE > SMALL_LMAX || D.ncolours > SMALL_MAXC) return;
  std::unordered_map<int32_t, int32_t> loc;
  loc.reserve(mE * 2);
  for (int k = 0; k < mE; ++k) loc[gid[k]] = k;
  auto L_ = [&](int32_t g) -> int32_t {
    auto it = loc.find(g);
    return it == loc.end() ? -1 : it->second;
  };
  std::vector<int32_t> sm_ptr(1, 0), rs_ptr(1, 0);
  std::vector<uint16_t> sm_col, rs_col;
  std::vector<T> sm_val, rs_val;
  for (int k = 0; k < mE; ++k) {
    const int32_t r = gid[k];
    for (int64_t p = Arows.ptr[r]; p < Arows.ptr[r + 1]; ++p) {
      if (Arows.val[p] == 0.0) continue;
      const int32_t c = Arows.col[p];
      if (k < mS) {
        const int32_t lc = L_(c);
        if (lc < 0) return;  // a neighbour outside E_l: keep the level on the general path
        sm_col.push_back((uint16_t)lc);
        sm_val.push_back((T)Arows.val[p]);
      }
      if (inset[c]) {
        const int32_t lc = L_(c);
        if (lc < 0) return;
        rs_col.push_back((uint16_t)lc);
        rs_val.push_back((T)Arows.val[p]);
      }
    }
    if (k < mS) sm_ptr.push_back((int32_t)sm_col.size());
    rs_ptr.push_back((int32_t)rs_col.size());
  }
  std::vector<uint16_t> nn_id, rp_id, rp_child;
  std::vector<int32_t> nn_p0, nn_p1, rp_ptr(1, 0);
  for (size_t t = 0; t < L.new_id.size(); ++t) {
    const int32_t a = L_(L.new_id[t]);
    const int32_t b0 = L.new_p0[t] >= 0 ? L_(L.new_p0[t]) : -1;
    const int32_t b1 = L.new_p1[t] >= 0 ? L_(L.new_p1[t]) : -1;
    if (a < 0 || (L.new_p0[t] >= 0 && b0 < 0) || (L.new_p1[t] >= 0 && b1 < 0)) return;
    nn_id.push_back((uint16_t)a);
    nn_p0.push_back(b0);
    nn_p1.push_back(b1);
  }
  for (size_t t = 0; t < pid.size(); ++t) {
    const int32_t a = L_(pid[t]);
    if (a < 0) return;
    rp_id.push_back((uint16_t)a);
    for (int32_t p = pptr[t]; p < pptr[t + 1]; ++p) {
      const int32_t b = L_(child[p]);
      if (b < 0) return;
      rp_child.push_back((uint16_t)b);
    }
    rp_ptr.push_back((int32_t)rp_child.size());
  }
  S.mS = mS;
  S.mE = mE;
  S.ncol = D.ncolours;
  S.nnew = (int)nn_id.size();
  S.npar = (int)rp_id.size();
  S.nnz_sm = (int64_t)sm_col.size();
  S.nnz_rs = (int64_t)rs_col.size();
  S.nchild = (int64_t)rp_child.size();
  S.cs = cs;
  S.gid.upload(gid, s);
  S.sm_ptr.upload(sm_ptr, s);
  S.sm_col.upload(sm_col, s);
  S.sm_val.upload(sm_val, s);
  S.dinv.upload(dinv, s);
  S.rs_ptr.upload(rs_ptr, s);
  S.rs_col.upload(rs_col, s);
  S.rs_val.upload(rs_val, s);
  if (bf16) {
    std::vector<bf16v> a(sm_val.size()), b(rs_val.size());
    for (size_t k = 0; k < a.size(); ++k) a[k].bits = bf16_bits((float)sm_val[k]);
    for (size_t k = 0; k < b.size(); ++k) b[k].bits = bf16_bits((float)rs_val[k]);
    S.sm_v16.upload(a, s);
    S.rs_v16.upload(b, s);
  }
  S.nn_id.upload(nn_id, s);
  S.nn_p0.upload(nn_p0, s);
  S.nn_p1.upload(nn_p1, s);
  S.rp_id.upload(rp_id, s);
  S.rp_ptr.upload(rp_ptr, s);
  S.rp_child.upload(rp_child, s);
  S.ok = true;
}

// Tiles of one sweep direction of a level (TileSweeps).  The own rows of a
// tile are tile_rows consecutive smoothing rows in aux-ID order.  Its rows
// are the closure of the pairs (row, sweep) that the own rows' final values
// depend on: a row's value after sweep s reads its own value after sweep
// s - 1 and each coupled row j of N~_l either after sweep s (j's class is
// swept before the row's in this direction) or after sweep s - 1 (j's class
// comes later).  Before the first sweep the values are the start values:
// zero on the way down (such reads need no row), read from us on the way up
// (the row is kept, with its start value).  Every entry of a kept row that
// points to a row of N~_l outside the tile is left out: no pair of the
// closure reads it.  Entries of the post-sweeps' rows whose column lies
// outside N~_l become the tile's outside values.  SMd: SM-order rows with
// their N~_l columns as SM rows; SM: the same rows with all columns as aux
// IDs; pos: aux ID -> SM row.  Returns false (and builds nothing) when a tile
// needs more than smem_max bytes of shared memory or more than 65,535 local
// values, or when the halo exceeds max_halo times the own rows.
template <class T>
bool build_tiles(bool up, int nu, int tile_rows, const std::vector<int64_t>& sel, const std::vector<int64_t>& cstart,
                 const std::vector<T>& dinv, const HostCSR& SMd, const HostCSR& SM, const std::vector<int32_t>& pos,
                 size_t smem_max, double max_halo, unsigned max_threads, bool bf16, TileSweeps<T>& TS,
                 cudaStream_t s) {
  const int64_t nsm = (int64_t)sel.size();
  const int ncol = (int)cstart.size() - 1;
  std::vector<int32_t> colr(nsm);
  for (int c = 0; c < ncol; ++c)
    for (int64_t k = cstart[c]; k < cstart[c + 1]; ++k) colr[k] = c;
  std::vector<int32_t> own;
  for (int64_t k = 0; k < nsm; ++k)
    if (sel[k] >= 0) own.push_back((int32_t)k);
  std::sort(own.begin(), own.end(), [&](int32_t a, int32_t b) { return sel[a] < sel[b]; });
  const int64_t ntiles = ((int64_t)own.size() + tile_rows - 1) / tile_rows;
  struct Out {
    std::vector<int32_t> lrow, phase, ext;
    std::vector<unsigned char> blob;
    int64_t interior = 0, halo = 0, nnz = 0, nnz_real = 0;
    bool ok = true;
  };
  std::vector<Out> out(ntiles);
  const unsigned nt = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)max_threads, ntiles));
  std::vector<std::thread> th;
  for (unsigned w = 0; w < nt; ++w)
    th.emplace_back([&, w] {
      // stamps: mark[sw * nsm + k] == tile: pair (k, sw) needed; inx[k] == tile: k kept
      std::vector<int32_t> mark((size_t)nu * nsm, -1), inx(nsm, -1), loc(nsm, 0), ownm(nsm, -1);
      std::vector<std::pair<int32_t, int32_t>> stack;
      std::vector<int32_t> X;
      std::unordered_map<int32_t, int32_t> extpos;
      std::vector<int64_t> rptr;
      std::vector<int32_t> rcol;
      std::vector<double> rval;
      std::vector<std::pair<int64_t, int32_t>> rlen;
      for (int64_t t = ntiles * w / nt; t < ntiles * (w + 1) / nt; ++t) {
        const int32_t tag = (int32_t)t;
        stack.clear();
        X.clear();
        auto keep = [&](int32_t k) {
          if (inx[k] != tag) {
            inx[k] = tag;
            X.push_back(k);
          }
        };
        auto need = [&](int32_t k, int sw) {
          int32_t& m = mark[(size_t)sw * nsm + k];
          if (m != tag) {
            m = tag;
            stack.push_back({k, sw});
          }
        };
        const int64_t o0 = t * tile_rows, o1 = std::min<int64_t>((int64_t)own.size(), o0 + tile_rows);
        for (int64_t q = o0; q < o1; ++q) {
          ownm[own[q]] = tag;
          need(own[q], nu - 1);
        }
        while (!stack.empty()) {
          const auto [k, sw] = stack.back();
          stack.pop_back();
          keep(k);
          if (sw >= 1) need(k, sw - 1);
          for (int64_t p = SMd.ptr[k]; p < SMd.ptr[k + 1]; ++p) {
            const int32_t j = SMd.col[p];
            if (j == k) continue;
            const int cj = colr[j], ck = colr[k];
            const bool before = up ? cj > ck : cj < ck;
            if (before || cj == ck) need(j, sw);
            if (!before) {
              if (sw >= 1) need(j, sw - 1);
              else if (up) keep(j);
            }
          }
        }
        // local rows: grouped by colour class (SM order); within a class,
        // where order does not matter, longest rows first so that the slices
        // carry little padding
        auto row_len = [&](int32_t k) {
          int64_t n = 0;
          if (!up) {
            for (int64_t p = SMd.ptr[k]; p < SMd.ptr[k + 1]; ++p) n += inx[SMd.col[p]] == tag;
          } else {
            for (int64_t p = SM.ptr[k]; p < SM.ptr[k + 1]; ++p) {
              const int32_t j = pos[SM.col[p]];
              n += j < 0 || inx[j] == tag;
            }
          }
          return n;
        };
        std::sort(X.begin(), X.end());
        rlen.resize(X.size());
        for (size_t q = 0; q < X.size(); ++q) rlen[q] = {-row_len(X[q]), X[q]};
        Out& O = out[t];
        O.phase.assign(ncol + 1, 0);
        size_t x = 0;
        for (int c = 0; c < ncol; ++c) {
          O.phase[c] = (int32_t)O.lrow.size();
          const size_t x0 = x;
          while (x < X.size() && X[x] < cstart[c + 1]) ++x;
          std::sort(rlen.begin() + x0, rlen.begin() + x);
          for (size_t q = x0; q < x; ++q) {
            const int32_t k = rlen[q].second;
            loc[k] = (int32_t)O.lrow.size();
            const bool mine = ownm[k] == tag;
            O.lrow.push_back(mine ? k : -2 - k);
            if (mine) ++O.interior;
            else ++O.halo;
          }
          while (O.lrow.size() % 32) O.lrow.push_back(-1);
        }
        O.phase[ncol] = (int32_t)O.lrow.size();
        const int nl = (int)O.lrow.size();
        // rows with local columns (outside values numbered after the rows)
        extpos.clear();
        rptr.assign(1, 0);
        rcol.clear();
        rval.clear();
        for (int32_t g : O.lrow) {
          if (g != -1) {
            const int32_t k = g >= 0 ? g : -2 - g;
            if (!up) {
              for (int64_t p = SMd.ptr[k]; p < SMd.ptr[k + 1]; ++p) {
                const int32_t j = SMd.col[p];
                if (inx[j] != tag) continue;
                rcol.push_back(loc[j]);
                rval.push_back(SMd.val[p]);
              }
            } else {
              for (int64_t p = SM.ptr[k]; p < SM.ptr[k + 1]; ++p) {
                const int32_t a = SM.col[p];
                const int32_t j = pos[a];
                if (j >= 0) {
                  if (inx[j] != tag) continue;
                  rcol.push_back(loc[j]);
                } else {
                  auto it = extpos.find(a);
                  int32_t e;
                  if (it == extpos.end()) {
                    e = (int32_t)O.ext.size();
                    extpos.emplace(a, e);
                    O.ext.push_back(a);
                  } else {
                    e = it->second;
                  }
                  rcol.push_back(nl + e);
                }
                rval.push_back(SM.val[p]);
              }
            }
          }
          rptr.push_back((int64_t)rcol.size());
        }
        if (nl + (int64_t)O.ext.size() > 65535) {
          O.ok = false;
          continue;
        }
        // the tile's block: SELL-32 slice offsets, uint16 columns, values, then
        // per local row the diagonal inverse, the SM row (own: k, halo:
        // -2 - k, padding: -1) and the aux ID, then the outside values' aux
        // IDs; each part padded to 16 bytes
        const int nsl = nl / 32;
        std::vector<int32_t> soff(nsl + 1, 0);
        for (int sl = 0; sl < nsl; ++sl) {
          int64_t wmax = 0;
          for (int r = sl * 32; r < sl * 32 + 32; ++r) wmax = std::max(wmax, rptr[r + 1] - rptr[r]);
          soff[sl + 1] = soff[sl] + (int32_t)(wmax * 32);
        }
        const int64_t ne_ = soff[nsl], nx = (int64_t)O.ext.size();
        O.nnz = ne_;
        O.nnz_real = rptr[nl];
        const TileLayout lay =
            tile_layout((int64_t)nl, ne_, nx, (int64_t)sizeof(T), bf16 ? (int64_t)sizeof(bf16v) : (int64_t)sizeof(T));
        O.blob.assign(lay.end, 0);
        std::memcpy(O.blob.data(), soff.data(), 4 * (size_t)(nsl + 1));
        uint16_t* cc = reinterpret_cast<uint16_t*>(O.blob.data() + lay.col);
        T* vv = reinterpret_cast<T*>(O.blob.data() + lay.val);
        bf16v* vb = reinterpret_cast<bf16v*>(O.blob.data() + lay.val);
        for (int r = 0; r < nl; ++r) {
          const int sl = r / 32, lane = r % 32;
          int64_t e = 0;
          for (int64_t p = rptr[r]; p < rptr[r + 1]; ++p, ++e) {
            cc[soff[sl] + e * 32 + lane] = (uint16_t)rcol[p];
            if (bf16)
              vb[soff[sl] + e * 32 + lane].bits = bf16_bits((float)rval[p]);
            else
              vv[soff[sl] + e * 32 + lane] = (T)rval[p];
          }
        }
        T* dd = reinterpret_cast<T*>(O.blob.data() + lay.dinv);
        int32_t* ls = reinterpret_cast<int32_t*>(O.blob.data() + lay.lsm);
        int32_t* la = reinterpret_cast<int32_t*>(O.blob.data() + lay.laux);
        for (int r = 0; r < nl; ++r) {
          const int32_t g = O.lrow[r];
          ls[r] = g;
          if (g == -1) {
            dd[r] = (T)0;
            la[r] = -1;
          } else {
            const int32_t k = g >= 0 ? g : -2 - g;
            dd[r] = dinv[k];
            la[r] = (int32_t)sel[k];
          }
        }
        if (nx) std::memcpy(O.blob.data() + lay.ext, O.ext.data(), 4 * (size_t)nx);
      }
    });
  for (auto& x : th) x.join();
  int64_t maxloc = 0, maxext = 0, maxblob = 0, interior = 0, halo = 0;
  for (auto& O : out) {
    if (!O.ok) return false;
    maxloc = std::max<int64_t>(maxloc, (int64_t)O.lrow.size());
    maxext = std::max<int64_t>(maxext, (int64_t)O.ext.size());
    maxblob = std::max<int64_t>(maxblob, (int64_t)O.blob.size());
    interior += O.interior;
    halo += O.halo;
  }
  const size_t smem = (size_t)maxblob + (size_t)(maxloc + (maxext + 3) / 4 * 4) * sizeof(T) + (size_t)maxloc * sizeof(T);
  if (smem > smem_max || (double)halo > max_halo * (double)interior) return false;
  std::vector<int64_t> loc_off(1, 0), blob_off(1, 0), ext_off(1, 0);
  std::vector<int32_t> phase;
  std::vector<unsigned char> blob;
  for (auto& O : out) {
    loc_off.push_back(loc_off.back() + (int64_t)O.lrow.size());
    blob_off.push_back(blob_off.back() + (int64_t)O.blob.size());
    ext_off.push_back(ext_off.back() + (int64_t)O.ext.size());
    phase.insert(phase.end(), O.phase.begin(), O.phase.end());
    blob.insert(blob.end(), O.blob.begin(), O.blob.end());
    TS.nnz += O.nnz;
    TS.nnz_real += O.nnz_real;
  }
  if (up) {
    // where each SM row sits in tile order (own and halo copies)
    std::vector<int64_t> pptr(nsm + 1, 0);
    for (auto& O : out)
      for (int32_t g : O.lrow)
        if (g != -1) ++pptr[(g >= 0 ? g : -2 - g) + 1];
    for (int64_t k = 0; k < nsm; ++k) pptr[k + 1] += pptr[k];
    std::vector<int32_t> pos(pptr[nsm]);
    std::vector<int64_t> fill(pptr.begin(), pptr.end() - 1);
    for (int64_t t = 0; t < ntiles; ++t)
      for (size_t k = 0; k < out[t].lrow.size(); ++k) {
        const int32_t g = out[t].lrow[k];
        if (g != -1) pos[fill[g >= 0 ? g : -2 - g]++] = (int32_t)(loc_off[t] + (int64_t)k);
      }
    TS.pos_ptr.upload(pptr, s);
    TS.pos.upload(pos, s);
  }
  TS.ntiles = ntiles;
  TS.nloc = loc_off.back();
  TS.maxloc = (int)maxloc;
  TS.maxext = (int)((maxext + 3) / 4 * 4);  // F follows U in shared memory, 16-byte aligned
  TS.maxblob = maxblob;
  TS.interior = interior;
  TS.halo = halo;
  TS.loc_off.upload(loc_off, s);
  TS.blob_off.upload(blob_off, s);
  TS.ext_off.upload(ext_off, s);
  TS.phase.upload(phase, s);
  TS.blob.upload(blob, s);
  ASMG_CUDA(cudaStreamSynchronize(s));
  return true;
}

// The near-boundary solve of a level (mixed boundaries, Algorithm 3) for the
// device: the rows of A_l on J_{l,j} in the factor's order (all columns) and
// the block cyclic reduction flattened into NbDev.
template <class T>
void build_nb_dev(const AuxLevelHost& L, const HostCSR& Arows, const std::vector<int32_t>& pos, AuxLevelDev<T>& D,
                  cudaStream_t s) {
  const nb::Factor& Fz = L.nb_fac;
  NbDev& N = D.nb;
  N.m = (int64_t)L.nb_id.size();
  if (N.m == 0) return;
  if (!Fz.ok || Fz.m != N.m) ASMG_FAIL(ASMG_ERR_BAD_MESH, "auxiliary level %d: no near-boundary factor", L.level);
  std::vector<int32_t> aux(N.m), sm(N.m);
  std::vector<int64_t> sel(N.m);
  for (int64_t q = 0; q < N.m; ++q) {
    const int32_t a = L.nb_id[Fz.order[q]];
    aux[q] = a;
    sm[q] = pos[a];
    sel[q] = a;
    if (sm[q] < 0) ASMG_FAIL(ASMG_ERR_BAD_MESH, "auxiliary level %d: near-boundary node outside the level", L.level);
  }
  HostCSR rows = select_rows(Arows, sel, nullptr, nullptr);
  sell_build<T>(D.NB, rows, 0, s);
  // block sizes of round 0, then the even blocks of each round form the next
  std::vector<int> sz0;
  for (size_t b = 0; b + 1 < Fz.bstart.size(); ++b) sz0.push_back((int)(Fz.bstart[b + 1] - Fz.bstart[b]));
  N.R = (int)Fz.rounds.size();
  std::vector<int32_t> nblk, boff;
  std::vector<int64_t> btab, voff(1, 0);
  std::vector<double> mats;
  auto put = [&](const nb::Blk& B) -> int64_t {
    if (B.empty()) return -1;
    const int64_t o = (int64_t)mats.size();
    mats.insert(mats.end(), B.a.begin(), B.a.end());
    return o;
  };
  std::vector<int> sz = sz0;
  for (int r = 0; r < N.R; ++r) {
    const nb::Round& Rd = Fz.rounds[r];
    if (Rd.n != (int)sz.size()) ASMG_FAIL(ASMG_ERR_CUDA, "near-boundary factor: inconsistent rounds");
    nblk.push_back(Rd.n);
    boff.push_back((int32_t)(btab.size() / 5));
    int64_t off = 0;
    for (int k = 0; k < Rd.n; ++k) {
      btab.push_back(sz[k]);
      btab.push_back(off);
      btab.push_back((k & 1) ? put(Rd.F[k]) : -1);
      btab.push_back(k > 0 ? put(Rd.Lo[k]) : -1);
      btab.push_back(k + 1 < Rd.n ? put(Rd.Up[k]) : -1);
      off += sz[k];
    }
    voff.push_back(voff.back() + off);
    std::vector<int> nx;
    for (int k = 0; k < Rd.n; k += 2) nx.push_back(sz[k]);
    sz.swap(nx);
  }
  if (sz.size() != 1 || Fz.last.r != sz[0]) ASMG_FAIL(ASMG_ERR_CUDA, "near-boundary factor: inconsistent last block");
  N.last_size = sz[0];
  N.last_off = put(Fz.last);
  voff.push_back(voff.back() + sz[0]);  // the last block's vector, then the pool size
  N.nblk_h = nblk;
  N.nblk.upload(nblk, s);
  N.boff.upload(boff, s);
  N.btab.upload(btab, s);
  N.voff.upload(voff, s);
  N.mats.upload(mats, s);
  N.aux.upload(aux, s);
  N.sm.upload(sm, s);
}

template <class T>
void build_level_dev(const AuxLevelHost& L, const HostCSR& Arows, const std::vector<int32_t>& colour,
                     const std::vector<uint8_t>& inset, const asmg_params& prm, AuxLevelDev<T>& D, cudaStream_t s) {
  D.level = L.level;
  // the mixed form may read the level matrices in BF16 (asmg_params::level_bf16)
  const bool bf16 = std::is_same<T, float>::value && prm.level_bf16 == 1;
  // smoothing rows ordered by (colour, id), colour blocks padded to 32
  int ncol = 0;
  for (int32_t id : L.smooth) ncol = std::max(ncol, colour[id] + 1);
  D.ncolours = ncol;
  std::vector<std::vector<int32_t>> byc(ncol);
  for (int32_t id : L.smooth) byc[colour[id]].push_back(id);
  std::vector<int64_t> sel;
  D.cstart.assign(1, 0);
  for (int c = 0; c < ncol; ++c) {
    for (int32_t id : byc[c]) sel.push_back(id);
    while (sel.size() % 32) sel.push_back(-1);
    D.cstart.push_back((int64_t)sel.size());
  }
  D.nsm = (int64_t)sel.size();
  D.nsm_real = (int64_t)L.smooth.size();
  std::vector<int32_t> rows(sel.size());
  std::vector<T> dinv(sel.size(), (T)0);
  for (size_t k = 0; k < sel.size(); ++k) {
    rows[k] = (int32_t)sel[k];
    if (sel[k] >= 0) {
      double dg = 0;
      for (int64_t p = Arows.ptr[sel[k]]; p < Arows.ptr[sel[k] + 1]; ++p)
        if (Arows.col[p] == sel[k]) dg = Arows.val[p];
      if (!(dg > 0)) ASMG_FAIL(ASMG_ERR_CUDA, "auxiliary level %d: non-positive diagonal", L.level);
      dinv[k] = (T)(1.0 / dg);
    }
  }
  HostCSR SM = select_rows(Arows, sel, nullptr, nullptr);
  // SM row index of every node of N~_l: the down sweeps and the residual work
  // on the level's own correction us (SM order), where every other node is 0
  std::vector<int32_t> pos(Arows.nr, -1);
  for (size_t k = 0; k < sel.size(); ++k)
    if (sel[k] >= 0) pos[sel[k]] = (int32_t)k;
  HostCSR SMd = select_rows(Arows, sel, &pos, &inset);
  D.cnnz.assign(ncol, 0);
  D.cnnz_d.assign(ncol, 0);
  D.crows.assign(ncol, 0);
  for (int c = 0; c < ncol; ++c)
    for (int64_t k = D.cstart[c]; k < D.cstart[c + 1]; ++k)
      if (sel[k] >= 0) {
        D.crows[c] += 1;
        D.cnnz[c] += SM.ptr[k + 1] - SM.ptr[k];
        D.cnnz_d[c] += SMd.ptr[k + 1] - SMd.ptr[k];
      }
  sell_build<T>(D.SM, SM, 0, s);
  sell_build<T>(D.SMd, SMd, 0, s);
  if constexpr (std::is_same<T, float>::value)
    if (bf16) {
      sell_bf16(D.SM, s);
      sell_bf16(D.SMd, s);
    }
  D.sm_rows.upload(rows, s);
  D.sm_dinv.upload(dinv, s);
  // temporal blocking of the level's sweeps (TileSweeps): the first tile size
  // of TILE_SIZES_2COL / TILE_SIZES_MULTI (or the requested size) whose tiles
  // fit the shared-memory budget with a halo of at most TILE_MAX_HALO times the
  // own rows; the level needs at least two tiles and every new node must be a
  // smoothing row (k_up_init prolongs through the smoothing rows)
  D.tiled = false;
  if (prm.tile_rows >= 0 && prm.nu_post >= 1) {
    bool ok = true;
    for (int32_t id : L.new_id)
      if (pos[id] < 0) ok = false;
    std::vector<int> sizes;
    if (prm.tile_rows > 0) sizes.push_back(prm.tile_rows);
    else if (ncol <= 2) sizes.assign(std::begin(TILE_SIZES_2COL), std::end(TILE_SIZES_2COL));
    else sizes.assign(std::begin(TILE_SIZES_MULTI), std::end(TILE_SIZES_MULTI));
    // a requested size takes any halo and up to TILE_SMEM_MAX of shared memory
    const double max_halo = prm.tile_rows > 0 ? 1e30 : TILE_MAX_HALO;
    const size_t smem_max = prm.tile_rows > 0 ? TILE_SMEM_MAX : TILE_SMEM;
    for (int trows : sizes) {
      if (!ok || D.nsm_real < 2 * (int64_t)trows) continue;
      // the two directions are built at the same time, each on half the host threads
      TileSweeps<T> td, tu;
      const unsigned half = std::max(1u, std::thread::hardware_concurrency() / 2);
      bool okd = false, oku = false;
      std::exception_ptr eu, ed;
      std::thread up_th([&] {
        try {
          oku = build_tiles<T>(true, prm.nu_post, trows, sel, D.cstart, dinv, SMd, SM, pos, smem_max, max_halo, half,
                               bf16, tu, s);
        } catch (...) {
          eu = std::current_exception();
        }
      });
      try {
        okd = build_tiles<T>(false, prm.nu_pre, trows, sel, D.cstart, dinv, SMd, SM, pos, smem_max, max_halo, half,
                             bf16, td, s);
      } catch (...) {
        ed = std::current_exception();
      }
      up_th.join();
      if (ed) std::rethrow_exception(ed);
      if (eu) std::rethrow_exception(eu);
      if (!okd || !oku) continue;
      std::vector<int32_t> p0(sel.size(), -3), p1(sel.size(), -3);
      for (size_t t = 0; t < L.new_id.size(); ++t) {
        p0[pos[L.new_id[t]]] = L.new_p0[t];
        p1[pos[L.new_id[t]]] = L.new_p1[t];
      }
      D.sm_par0.upload(p0, s);
      D.sm_par1.upload(p1, s);
      D.tdown = std::move(td);
      D.tup = std::move(tu);
      D.tiled = D.tiled_down = D.tiled_up = true;
      D.tile_rows = trows;
      break;
    }
  }
  // residual rows: every row with an entry in a smoothing column
  std::vector<uint8_t> touched(Arows.nr, 0);
  host_for(Arows.nr, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i)
      for (int64_t p = Arows.ptr[i]; p < Arows.ptr[i + 1]; ++p)
        if (inset[Arows.col[p]]) {
          touched[i] = 1;
          break;
        }
  });
  std::vector<int64_t> rsel;
  for (int64_t i = 0; i < Arows.nr; ++i)
    if (touched[i]) rsel.push_back(i);
  D.nrs_real = (int64_t)rsel.size();
  while (rsel.size() % 32) rsel.push_back(-1);
  D.nrs = (int64_t)rsel.size();
  HostCSR RS = select_rows(Arows, rsel, &pos, &inset);
  sell_build<T>(D.RS, RS, 0, s);
  if constexpr (std::is_same<T, float>::value)
    if (bf16) sell_bf16(D.RS, s);
  std::vector<int32_t> rsrows(rsel.begin(), rsel.end());
  D.rs_rows.upload(rsrows, s);
  // prolongation and restriction of the new nodes
  D.nnew = (int64_t)L.new_id.size();
  D.nn_id.upload(L.new_id, s);
  D.nn_p0.upload(L.new_p0, s);
  D.nn_p1.upload(L.new_p1, s);
  std::vector<std::pair<int32_t, int32_t>> pc;  // (parent, child)
  for (size_t k = 0; k < L.new_id.size(); ++k) {
    if (L.new_p0[k] >= 0) pc.push_back({L.new_p0[k], L.new_id[k]});
    if (L.new_p1[k] >= 0) pc.push_back({L.new_p1[k], L.new_id[k]});
  }
  std::sort(pc.begin(), pc.end());
  std::vector<int32_t> pid, pptr(1, 0), child;
  for (size_t k = 0; k < pc.size(); ++k) {
    if (k == 0 || pc[k].first != pc[k - 1].first) {
      if (k) pptr.push_back((int32_t)child.size());
      pid.push_back(pc[k].first);
    }
    child.push_back(pc[k].second);
  }
  if (!pid.empty()) pptr.push_back((int32_t)child.size());
  D.npar = (int64_t)pid.size();
  D.nchild = (int64_t)child.size();
  D.rp_id.upload(pid, s);
  D.rp_ptr.upload(pptr, s);
  D.rp_child.upload(child, s);
  build_nb_dev<T>(L, Arows, pos, D, s);
  // a level with a near-boundary solve keeps its own launches (the solve sits
  // between the coarse correction and the post-smoothing)
  if (D.nb.m == 0) build_small<T>(L, Arows, inset, sel, rsel, dinv, pid, pptr, child, bf16, D, s);
  else D.small.ok = false;
}

// triangles given by lattice keys -> device coordinates, ids, coefficients
struct TriDev {
  DBuf<double> xy, coef;
  DBuf<int32_t> id;
};

void upload_tris(const asmg_s& h, const std::vector<uint64_t>& keys, const std::vector<int32_t>& ids,
                 const std::vector<double>& coef, TriDev& T, cudaStream_t s) {
  const int dim = h.mesh.dim;
  std::vector<double> xy(keys.size() * dim);
  for (size_t k = 0; k < keys.size(); ++k) {
    if (dim == 2)
      lattice_point(h.tree, keys[k], &xy[2 * k]);
    else
      lattice_point3(h.tree, h.aux.LB, keys[k], &xy[3 * k]);
  }
  T.xy.upload(xy, s);
  T.id.upload(ids, s);
  T.coef.upload(coef, s);
}

template <class T>
void build_prec(asmg_s& h, Prec<T>& P, const HostCSR& Aperm, const std::vector<double>& dinv_perm, cudaStream_t s) {
  if (std::is_same<T, float>::value) {
    sell_build<T>(P.Af, Aperm, 0, s);
    std::vector<T> d(dinv_perm.begin(), dinv_perm.end());
    P.dinv_f.upload(d, s);
  }
  // transfer P (rows: permuted fine rows) and P^T (rows: aux nodes), built
  // by counting sort into flat CSR arrays; each row sorted by column
  const Triplets& Tp = h.aux.P;
  const int64_t m = (int64_t)Tp.r.size();
  auto to_csr = [&](int64_t nr, int64_t nc, bool transpose) {
    HostCSR A;
    A.nr = nr;
    A.nc = nc;
    A.ptr.assign(nr + 1, 0);
    for (int64_t k = 0; k < m; ++k) ++A.ptr[1 + (transpose ? Tp.c[k] : h.row_of_free[Tp.r[k]])];
    for (int64_t i = 0; i < nr; ++i) A.ptr[i + 1] += A.ptr[i];
    A.col.resize(m);
    A.val.resize(m);
    std::vector<int64_t> fill(A.ptr.begin(), A.ptr.end() - 1);
    for (int64_t k = 0; k < m; ++k) {
      const int32_t pr = h.row_of_free[Tp.r[k]];
      const int64_t row = transpose ? Tp.c[k] : pr;
      const int64_t q = fill[row]++;
      A.col[q] = transpose ? pr : Tp.c[k];
      A.val[q] = Tp.v[k];
    }
    std::vector<std::pair<int32_t, double>> tmp;
    for (int64_t i = 0; i < nr; ++i) {
      const int64_t b = A.ptr[i], e = A.ptr[i + 1];
      bool sorted = true;
      for (int64_t q = b + 1; q < e && sorted; ++q) sorted = A.col[q - 1] < A.col[q];
      if (sorted) continue;
      tmp.clear();
      for (int64_t q = b; q < e; ++q) tmp.push_back({A.col[q], A.val[q]});
      std::sort(tmp.begin(), tmp.end());
      for (int64_t q = b; q < e; ++q) {
        A.col[q] = tmp[q - b].first;
        A.val[q] = tmp[q - b].second;
      }
    }
    return A;
  };
  HostCSR Pc = to_csr(h.npad, h.nJpad, false), Ptc = to_csr(h.nJpad, h.npad, true);
  sell_build<T>(P.P, Pc, 0, s);
  sell_build<T>(P.PT, Ptc, 0, s);
}

// Colouring option 2 on an auxiliary level: the lattice parity of each node
// of the smoothing set, (X + Y [+ Z]) / h_l mod 2 with h_l the lattice
// spacing of level l (2^(bits - l) on the lattice of the node keys), used when
// no two coupled nodes of the set share it (couplings as for the Jones-
// Plassmann colouring: |a_vw| > 1e-12 sqrt(a_vv a_ww), w != v).  Uniform
// levels are bipartite this way (couplings across hypotenuses vanish), so
// they take two colour classes.  Returns false, leaving `colour` as it is,
// when some coupled pair shares a parity.
bool parity_colour(const asmg_s& h, int l, const HostCSR& A, const std::vector<int32_t>& smooth,
                   const std::vector<uint8_t>& inset, std::vector<int32_t>& colour) {
  const int dim = h.mesh.dim;
  const int bits = dim == 2 ? h.tree.D : h.aux.LB;
  const uint64_t step = 1ULL << (bits - l);
  std::vector<int8_t> par(A.nr, -1);
  for (int32_t v : smooth) {
    const uint64_t k = h.aux.aux_key[v];
    uint64_t q[3] = {0, 0, 0};
    for (int j = 0; j < 64 / dim; ++j)
      for (int c = 0; c < dim; ++c)
        if ((k >> (dim * j + c)) & 1ULL) q[c] |= 1ULL << j;
    par[v] = (int8_t)(((q[0] + q[1] + q[2]) / step) & 1);
  }
  std::vector<double> diag(A.nr, 0.0);
  host_for(A.nr, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i)
      for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p)
        if (A.col[p] == i) diag[i] = A.val[p];
  });
  std::atomic<bool> ok(true);
  host_for((int64_t)smooth.size(), [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1 && ok.load(std::memory_order_relaxed); ++k) {
      const int32_t v = smooth[k];
      for (int64_t p = A.ptr[v]; p < A.ptr[v + 1]; ++p) {
        const int32_t w = A.col[p];
        if (w == v || !inset[w] || par[w] != par[v]) continue;
        if (std::fabs(A.val[p]) > 1e-12 * std::sqrt(diag[v] * diag[w])) {
          ok.store(false, std::memory_order_relaxed);
          break;
        }
      }
    }
  });
  if (!ok.load()) return false;
  for (int32_t v : smooth) colour[v] = par[v];
  return true;
}

void build_all(asmg_s& h, cudaStream_t s) {
  double t0 = now();
  MeshHost& m = h.mesh;
  const int64_t nv = m.nv, ne = m.ne;
  // ---- fine problem: free dofs, assembly, colouring, permutation
  h.free_of_vertex.assign(nv, -1);
  h.vertex_of_free.clear();
  for (int64_t v = 0; v < nv; ++v)
    if (m.bflag[v] != 1) {  // free and Neumann vertices are unknowns
      h.free_of_vertex[v] = (int32_t)h.vertex_of_free.size();
      h.vertex_of_free.push_back((int32_t)v);
    }
  h.n = (int64_t)h.vertex_of_free.size();
  if (h.n == 0) ASMG_FAIL(ASMG_ERR_BAD_MESH, "no free vertices");
  h.d_free_of_vertex.upload(h.free_of_vertex, s);
  h.A_host = assemble_mesh(m.dim, ne, h.dX.p, h.dE.p, h.d_free_of_vertex.p, h.dCoeff.p, h.n, s);
  {
    std::vector<uint8_t> all(h.n, 1);
    std::vector<uint64_t> pk(h.vertex_of_free.begin(), h.vertex_of_free.end());
    h.fine_colour = jp_colour_gpu(h.A_host, all, pk, s);
  }
  int ncol = 0;
  for (auto c : h.fine_colour) ncol = std::max(ncol, c + 1);
  std::vector<int64_t> sel;
  h.fine_cstart.assign(1, 0);
  {
    std::vector<std::vector<int32_t>> byc(ncol);
    for (int64_t i = 0; i < h.n; ++i) byc[h.fine_colour[i]].push_back((int32_t)i);
    for (int c = 0; c < ncol; ++c) {
      for (auto i : byc[c]) sel.push_back(i);
      while (sel.size() % 32) sel.push_back(-1);
      h.fine_cstart.push_back((int64_t)sel.size());
    }
  }
  h.npad = (int64_t)sel.size();
  h.row_of_free.assign(h.n, -1);
  std::vector<int32_t> vrow(h.npad, -1), rowv(nv, -1);
  for (int64_t k = 0; k < h.npad; ++k)
    if (sel[k] >= 0) {
      h.row_of_free[sel[k]] = (int32_t)k;
      vrow[k] = h.vertex_of_free[sel[k]];
      rowv[vrow[k]] = (int32_t)k;
    }
  h.d_vertex_of_row.upload(vrow, s);
  h.d_row_of_vertex.upload(rowv, s);
  HostCSR Aperm = select_rows(h.A_host, sel, &h.row_of_free, nullptr);
  std::vector<double> dinv(h.npad, 0.0);
  for (int64_t k = 0; k < h.npad; ++k)
    for (int64_t p = Aperm.ptr[k]; p < Aperm.ptr[k + 1]; ++p)
      if (Aperm.col[p] == k) dinv[k] = 1.0 / Aperm.val[p];
  sell_build<double>(h.A64, Aperm, 0, s);
  h.dinv64.upload(dinv, s);
  h.fine_cnnz.assign(ncol, 0);
  h.fine_crows.assign(ncol, 0);
  for (int c = 0; c < ncol; ++c)
    for (int64_t k = h.fine_cstart[c]; k < h.fine_cstart[c + 1]; ++k)
      if (sel[k] >= 0) {
        h.fine_crows[c] += 1;
        h.fine_cnnz[c] += Aperm.ptr[k + 1] - Aperm.ptr[k];
      }
  h.stats.t_fine = now() - t0;

  // ---- auxiliary hierarchy (host), transfer
  double t1 = now();
  h.aux = AuxHost();
  if (m.dim == 2)
    build_aux_host(m, h.tree, h.prm, h.aux);
  else
    build_aux_host3(m, h.tree, h.prm, h.aux);
  h.stats.t_aux = now() - t1;
  t1 = now();
  build_transfer(m, h.dX.p, h.dE.p, h.vertex_of_free, h.aux.sz, h.aux.P, s);
  h.aux.sz = SZTable();
  h.stats.t_sz = now() - t1;
  double t2 = now();
  h.nJ = (int64_t)h.aux.aux_key.size();
  h.nJpad = pad32(h.nJ);

  // ---- auxiliary levels: device assembly, colouring, SELL
  h.level_smooth_keys.clear();
  h.level_smooth_colour.clear();
  h.level_rows.clear();
  h.p64.lev.clear();
  h.p32.lev.clear();
  h.stats.t_lv_assemble = h.stats.t_lv_colour = h.stats.t_lv_pack = h.stats.t_lv_export = 0;
  for (const AuxLevelHost& L : h.aux.levels) {
    double ta = now();
    std::vector<uint8_t> inset(h.nJ, 0);
    for (int32_t id : L.smooth) inset[id] = 1;
    TriDev T;
    upload_tris(h, L.tri_key, L.tri_id, L.tri_coef, T, s);
    DBuf<uint8_t> dkeep;
    dkeep.upload(inset, s);
    HostCSR Arows = assemble_simplices(m.dim, (int64_t)L.tri_coef.size(), T.xy.p, T.id.p, T.coef.p, dkeep.p, h.nJ, s);
    double tb = now();
    h.stats.t_lv_assemble += tb - ta;
    std::vector<int32_t> colour = jp_colour_gpu(Arows, inset, h.aux.aux_key, s);
    if (h.prm.colouring == 2) parity_colour(h, L.level, Arows, L.smooth, inset, colour);
    double tc = now();
    h.stats.t_lv_colour += tc - tb;
    // export copies
    std::vector<uint64_t> sk;
    std::vector<int32_t> sc;
    for (int32_t id : L.smooth) {
      sk.push_back(h.aux.aux_key[id]);
      sc.push_back(colour[id]);
    }
    h.level_smooth_keys.push_back(sk);
    h.level_smooth_colour.push_back(sc);
    Triplets tr;
    const int64_t nz = Arows.ptr[Arows.nr];
    tr.r.resize(nz);
    tr.c.assign(Arows.col.begin(), Arows.col.begin() + nz);
    tr.v.assign(Arows.val.begin(), Arows.val.begin() + nz);
    host_for(Arows.nr, [&](int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i)
        for (int64_t p = Arows.ptr[i]; p < Arows.ptr[i + 1]; ++p) tr.r[p] = (int32_t)i;
    });
    h.level_rows.push_back(std::move(tr));
    double td = now();
    h.stats.t_lv_export += td - tc;
    if (h.prm.precision == ASMG_MIXED) {
      h.p32.lev.emplace_back();
      build_level_dev<float>(L, Arows, colour, inset, h.prm, h.p32.lev.back(), s);
    } else {
      h.p64.lev.emplace_back();
      build_level_dev<double>(L, Arows, colour, inset, h.prm, h.p64.lev.back(), s);
    }
    h.stats.t_lv_pack += now() - td;
  }
  double te = now();
  // ---- coarsest level: explicit inverse of A_c (B_0 = A_0^{-1})
  h.nc = (int64_t)h.aux.coarse_id.size();
  if (h.nc > 0) {
    std::vector<int32_t> loc(h.aux.coarse_tri_id.size());
    for (size_t k = 0; k < loc.size(); ++k) {
      int32_t id = h.aux.coarse_tri_id[k];
      loc[k] = id < 0 ? -1
                      : (int32_t)(std::lower_bound(h.aux.coarse_id.begin(), h.aux.coarse_id.end(), id) -
                                  h.aux.coarse_id.begin());
    }
    TriDev T;
    upload_tris(h, h.aux.coarse_tri_key, loc, h.aux.coarse_tri_coef, T, s);
    HostCSR Ac = assemble_simplices(m.dim, (int64_t)h.aux.coarse_tri_coef.size(), T.xy.p, T.id.p, T.coef.p, nullptr,
                                    h.nc, s);
    const int64_t n = h.nc;
    std::vector<double> M(n * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = Ac.ptr[i]; p < Ac.ptr[i + 1]; ++p) M[i * n + Ac.col[p]] = Ac.val[p];
    // Cholesky M = L L^T (lower, in place)
    for (int64_t j = 0; j < n; ++j) {
      double d = M[j * n + j];
      for (int64_t k = 0; k < j; ++k) d -= M[j * n + k] * M[j * n + k];
      if (!(d > 0)) ASMG_FAIL(ASMG_ERR_CUDA, "coarsest auxiliary matrix is not positive definite");
      d = std::sqrt(d);
      M[j * n + j] = d;
      for (int64_t i = j + 1; i < n; ++i) {
        double t = M[i * n + j];
        for (int64_t k = 0; k < j; ++k) t -= M[i * n + k] * M[j * n + k];
        M[i * n + j] = t / d;
      }
    }
    // inverse column by column: solve L L^T x = e_c
    std::vector<double> inv(n * n), y(n);
    for (int64_t c = 0; c < n; ++c) {
      for (int64_t i = 0; i < n; ++i) {
        double t = (i == c) ? 1.0 : 0.0;
        for (int64_t k = 0; k < i; ++k) t -= M[i * n + k] * y[k];
        y[i] = t / M[i * n + i];
      }
      for (int64_t i = n - 1; i >= 0; --i) {
        double t = y[i];
        for (int64_t k = i + 1; k < n; ++k) t -= M[k * n + i] * inv[k * n + c];
        inv[i * n + c] = t / M[i * n + i];
      }
    }
    h.d_cinv.upload(inv, s);
    h.d_cid.upload(h.aux.coarse_id, s);
  }
  double tf = now();
  h.stats.t_coarse = tf - te;
  // ---- transfer and fine smoother copy
  if (h.prm.precision == ASMG_MIXED)
    build_prec<float>(h, h.p32, Aperm, dinv, s);
  else
    build_prec<double>(h, h.p64, Aperm, dinv, s);
  ASMG_CUDA(cudaStreamSynchronize(s));
  double tg = now();
  h.stats.t_transfer = tg - tf;
  setup_solve(h, s);
  ASMG_CUDA(cudaStreamSynchronize(s));
  h.stats.t_slots = now() - tg;
  h.stats.t_levels = now() - t2;
}

// algorithmic bytes of one PCG iteration (compulsory traffic, real non-zeros)
template <class T>
int64_t iteration_bytes(const asmg_s& h, const Prec<T>& P) {
  const int64_t s = sizeof(T), n = h.n, nJ = h.nJ;
  const int64_t nnzA = h.A64.nnz_real;
  int64_t b = 0;
  b += nnzA * 12 + 16 * n;                  // q = A p, <p, q>
  b += 48 * n;                              // x += a p, r -= a q, ||r||
  b += (s + 16) * n;                        // <z, r>, <z, q>
  b += (s + 16) * n;                        // p = z + beta p
  b += 2 * (nnzA * (s + 4) + 8 * n + 2 * s * n);  // two fine sweeps
  if (nJ > 0) {
    b += nnzA * (s + 4) + 8 * n + 2 * s * n;  // fine residual
    b += (P.PT.nnz_real) * (s + 4) + s * n + 2 * s * nJ;  // P^T
    b += (P.P.nnz_real) * (s + 4) + s * nJ + 2 * s * n;   // P
    for (auto& L : P.lev) {
      const int64_t m = L.nsm_real;
      b += (h.prm.nu_pre + h.prm.nu_post) * (L.SM.nnz_real * (s + 4) + m * (4 + 3 * s));
      b += L.RS.nnz_real * (s + 4) + L.nrs * (4 + 2 * s);
      b += 2 * m * (4 + 2 * s) + L.nnew * (12 + 3 * s);
    }
    b += h.nc * h.nc * 8 + h.nc * (4 + 2 * s);
  }
  return b;
}

int finish(int rc) { return rc; }

}  // namespace

namespace asmg {
void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
}  // namespace asmg

#define API_BEGIN \
  g_err.clear();  \
  try {
#define API_END                                   \
  }                                               \
  catch (const asmg::Error& e) {                  \
    g_err = e.msg;                                \
    return e.code;                                \
  }                                               \
  catch (const std::exception& e) {               \
    g_err = std::string("internal error: ") + e.what(); \
    return ASMG_ERR_CUDA;                         \
  }

extern "C" {

const char* amg_last_error(void) { return g_err.c_str(); }

int asmg_default_params(asmg_params* p) {
  if (!p) return ASMG_ERR_INVALID_ARG;
  p->n_min = 3;
  p->nu_pre = 2;
  p->nu_post = 2;
  p->coarse_max_dofs = 512;
  p->precision = ASMG_FP64;
  p->max_iter = 500;
  p->smoothing = 0;
  p->use_graph = 1;
  p->use_pdl = 1;
  p->smoother = 0;
  p->additive = 0;
  p->fine_sweeps = 1;
  p->iteration = 0;
  p->tile_rows = 0;
  p->inject_timeout = 0;
  p->nb_layers = 2;
  p->colouring = 2;
  p->level_bf16 = 0;
  return ASMG_OK;
}

int amg_setup(int dim, int64_t nv, const double* vertices, int64_t ne, const int32_t* elements, const uint8_t* boundary,
              const double* coeff, const asmg_params* params, void* stream, asmg_handle* out) {
  API_BEGIN
  if (!out) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!vertices || !elements || !boundary) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null input array");
  if (nv <= 0 || ne <= 0) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "nv and ne must be positive");
  if (dim != 2 && dim != 3) ASMG_FAIL(ASMG_ERR_UNSUPPORTED, "dim %d not supported (2 or 3)", dim);
  if (ne > (1LL << 31) / ((dim + 1) * (dim + 1)) || nv > (1LL << 31) - 1)
    ASMG_FAIL(ASMG_ERR_INVALID_ARG, "mesh too large");
  asmg_params prm;
  asmg_default_params(&prm);
  if (params) prm = *params;
  if (prm.n_min < 1 || prm.nu_pre < 1 || prm.nu_post < 0 || prm.coarse_max_dofs < 1 || prm.max_iter < 1 ||
      (prm.precision != ASMG_FP64 && prm.precision != ASMG_MIXED) || (prm.smoothing != 0 && prm.smoothing != 1) ||
      prm.coarse_max_dofs > 8192 || (prm.use_pdl != 0 && prm.use_pdl != 1) || (prm.use_graph != 0 && prm.use_graph != 1) ||
      (prm.smoother != 0 && prm.smoother != 1) || (prm.additive != 0 && prm.additive != 1) || prm.fine_sweeps < 1 ||
      prm.fine_sweeps > 8 || (prm.iteration != 0 && prm.iteration != 1) ||
      (prm.tile_rows != -1 && prm.tile_rows != 0 && (prm.tile_rows < 32 || prm.tile_rows > 65536)) ||
      (prm.inject_timeout != 0 && prm.inject_timeout != 1) || prm.nb_layers < -1 || prm.nb_layers > 16 ||
      (prm.colouring != 0 && prm.colouring != 2) || (prm.level_bf16 != 0 && prm.level_bf16 != 1) ||
      (prm.level_bf16 == 1 && prm.precision != ASMG_MIXED))
    ASMG_FAIL(ASMG_ERR_INVALID_ARG, "invalid parameter");
  cudaStream_t s = (cudaStream_t)stream;
  double t0 = now();
  std::unique_ptr<asmg_s> h(new asmg_s());
  h->prm = prm;
  MeshHost& m = h->mesh;
  m.dim = dim;
  m.nv = nv;
  m.ne = ne;
  m.X = to_host(vertices, nv * dim, s);
  m.E = to_host(elements, ne * (dim + 1), s);
  m.bflag = to_host(boundary, nv, s);
  if (coeff) m.coeff = to_host(coeff, ne, s);
  for (int64_t v = 0; v < nv; ++v) {
    if (m.bflag[v] > 2) ASMG_FAIL(ASMG_ERR_BAD_MESH, "boundary flag %d at vertex %lld", (int)m.bflag[v], (long long)v);
    if (m.bflag[v] == 2) m.mixed = true;
  }
  m.nb_layers = prm.nb_layers;
  if (m.mixed) {
    // the mixed grids are not nested and every level is smoothed as a whole;
    // the near-boundary solve runs between the coarse correction and the
    // post-smoothing, so those levels take the per-class launches
    h->prm.tile_rows = -1;
  }
  for (int64_t e = 0; e < (int64_t)m.coeff.size(); ++e)
    if (!(m.coeff[e] > 0) || !std::isfinite(m.coeff[e]))
      ASMG_FAIL(ASMG_ERR_BAD_MESH, "coefficient of element %lld is not positive and finite", (long long)e);
  h->dX.upload(m.X, s);
  h->dE.upload(m.E, s);
  if (!m.coeff.empty()) h->dCoeff.upload(m.coeff, s);
  // cluster tree (also checks index range and orientation)
  double tt = now();
  build_tree_gpu(dim, nv, h->dX.p, ne, h->dE.p, prm.n_min, s, h->tree);
  h->stats.t_tree = now() - tt;
  // does the domain fill the root box (the element measures add up to
  // L^dim)?  A domain that does not uses the Dirichlet auxiliary grids
  // (Sec. 3.4)
  {
    double meas = 0;
    for (int64_t e = 0; e < ne; ++e) {
      const int32_t* v = &m.E[(dim + 1) * e];
      if (dim == 2) {
        meas += 0.5 * ((m.X[2 * v[1]] - m.X[2 * v[0]]) * (m.X[2 * v[2] + 1] - m.X[2 * v[0] + 1]) -
                       (m.X[2 * v[2]] - m.X[2 * v[0]]) * (m.X[2 * v[1] + 1] - m.X[2 * v[0] + 1]));
      } else {
        double e3[3][3];
        for (int k = 0; k < 3; ++k)
          for (int r = 0; r < 3; ++r) e3[k][r] = m.X[3 * (int64_t)v[k + 1] + r] - m.X[3 * (int64_t)v[0] + r];
        meas += (e3[0][0] * (e3[1][1] * e3[2][2] - e3[1][2] * e3[2][1]) -
                 e3[0][1] * (e3[1][0] * e3[2][2] - e3[1][2] * e3[2][0]) +
                 e3[0][2] * (e3[1][0] * e3[2][1] - e3[1][1] * e3[2][0])) /
                6.0;
      }
    }
    const double box = std::pow(h->tree.L, dim);
    m.boxdomain = std::fabs(meas - box) <= 1e-12 * box;
  }
  build_all(*h, s);
  h->bytes_iter = prm.precision == ASMG_MIXED ? iteration_bytes(*h, h->p32) : iteration_bytes(*h, h->p64);
  // load the allocation-free entry point's module (and so its fixed scratch
  // array) on this device now, so that its calls never create memory
  noalloc_scratch_for_current_device();
  h->stats.t_total = now() - t0;
  *out = h.release();
  return ASMG_OK;
  API_END
}

void amg_destroy(asmg_handle h) { delete h; }

int amg_cluster_tree(int dim, int64_t nv, const double* vertices, int64_t ne, const int32_t* elements, uint64_t* keys,
                     int32_t* perm, void* stream) {
  API_BEGIN
  if (!vertices || !elements || !keys || !perm) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  if (dim != 2 && dim != 3) ASMG_FAIL(ASMG_ERR_UNSUPPORTED, "dim %d not supported", dim);
  if (nv <= 0 || ne <= 0) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "nv and ne must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<double> dX;
  DBuf<int32_t> dE;
  dX.upload(to_host(vertices, nv * dim, s), s);
  dE.upload(to_host(elements, ne * (dim + 1), s), s);
  TreeResult t;
  build_tree_gpu(dim, nv, dX.p, ne, dE.p, 3, s, t);
  ASMG_CUDA(cudaMemcpyAsync(keys, t.keys.p, 8 * ne, cudaMemcpyDefault, s));
  ASMG_CUDA(cudaMemcpyAsync(perm, t.perm.p, 4 * ne, cudaMemcpyDefault, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
  return ASMG_OK;
  API_END
}

}  // extern "C"

struct asmg_batch_s {
  std::vector<asmg_handle> H;
  int nrhs = 0;
  double rtol = 0;
  bool multi = false;  // right-hand sides in groups of KRHS columns (SpMM form), one graph branch per group
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~asmg_batch_s() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  Slot& slot(int p, int j) { return *H[p]->slots.at(1 + j); }
  MultiSlot& mslot(int p, int g) { return *H[p]->mslots.at(1 + g); }
};

extern "C" {

int amg_batch_create(int nprob, const asmg_handle* handles, int nrhs, double rtol, void* stream, asmg_batch* out) {
  API_BEGIN
  if (!handles || !out || nprob <= 0 || nrhs <= 0) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "invalid batch arguments");
  if (!(rtol >= 0) || !std::isfinite(rtol)) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "rtol must be finite and >= 0");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<asmg_batch_s> B(new asmg_batch_s());
  B->H.assign(handles, handles + nprob);
  B->nrhs = nrhs;
  B->rtol = rtol;
  B->multi = nrhs > 1;
  for (auto h : B->H) {
    if (!h) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null handle in batch");
    if (!multi_supported(*h)) B->multi = false;
  }
  const int ngroups = (nrhs + KRHS - 1) / KRHS;
  for (auto h : B->H) {
    if (B->multi) {
      if (h->mslots.empty()) add_multi_slot(*h, s);
      while ((int)h->mslots.size() < 1 + ngroups) add_multi_slot(*h, s);
    } else {
      while ((int)h->slots.size() < 1 + nrhs) add_slot(*h, s);
    }
  }
  ASMG_CUDA(cudaGraphCreate(&B->graph, 0));
  cudaStream_t cs;
  ASMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  if (B->multi) {
    // one branch per (problem, group of KRHS right-hand sides): gather, the
    // multiple solve's graph, scatter
    for (int p = 0; p < nprob; ++p)
      for (int g = 0; g < ngroups; ++g) {
        asmg_s& h = *B->H[p];
        MultiSlot& S = B->mslot(p, g);
        ASMG_CUDA(cudaStreamBeginCaptureToGraph(cs, B->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        gather_multi(h, S.vb.p, S.b.p, cs);
        gather_multi(h, S.vu.p, S.x.p, cs);
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* leaf = nullptr;
        size_t nleaf = 0;
        ASMG_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &leaf, nullptr, &nleaf));
        std::vector<cudaGraphNode_t> leaves(leaf, leaf + nleaf);
        cudaGraph_t gg;
        ASMG_CUDA(cudaStreamEndCapture(cs, &gg));
        cudaGraphNode_t wnode = capture_solve_multi(h, S, rtol, B->graph, leaves.data(), leaves.size());
        ASMG_CUDA(cudaStreamBeginCaptureToGraph(cs, B->graph, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
        scatter_multi(h, S.x.p, S.vu.p, cs);
        ASMG_CUDA(cudaStreamEndCapture(cs, &gg));
      }
  }
  for (int p = 0; p < (B->multi ? 0 : nprob); ++p)
    for (int j = 0; j < nrhs; ++j) {
      asmg_s& h = *B->H[p];
      Slot& S = B->slot(p, j);
      // gather the staged rhs / initial guess (a root of its own branch)
      ASMG_CUDA(cudaStreamBeginCaptureToGraph(cs, B->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      gather_rows(h, S.vb.p, S.b.p, cs);
      gather_rows(h, S.vu.p, S.x.p, cs);
      cudaStreamCaptureStatus st;
      const cudaGraphNode_t* leaf = nullptr;
      size_t nleaf = 0;
      ASMG_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &leaf, nullptr, &nleaf));
      std::vector<cudaGraphNode_t> leaves(leaf, leaf + nleaf);
      cudaGraph_t gg;
      ASMG_CUDA(cudaStreamEndCapture(cs, &gg));
      cudaGraphNode_t wnode = capture_solve(h, S, rtol, B->graph, leaves.data(), leaves.size());
      ASMG_CUDA(cudaStreamBeginCaptureToGraph(cs, B->graph, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
      scatter_rows(h, S.x.p, false, S.vu.p, cs);
      ASMG_CUDA(cudaStreamEndCapture(cs, &gg));
    }
  ASMG_CUDA(cudaStreamDestroy(cs));
  ASMG_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
  *out = B.release();
  return ASMG_OK;
  API_END
}

int amg_batch_solve(asmg_batch B, const double* const* bs, double* const* us, int* iterations, int* status,
                    void* stream) {
  API_BEGIN
  if (!B || !bs || !us || !iterations) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int np = (int)B->H.size(), nr = B->nrhs;
  for (int k = 0; k < np * nr; ++k)
    if (!bs[k] || !us[k]) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null array in batch");
  if (B->multi) {
    const int ngroups = (nr + KRHS - 1) / KRHS;
    for (int p = 0; p < np; ++p)
      for (int g = 0; g < ngroups; ++g) {
        MultiSlot& S = B->mslot(p, g);
        const int64_t nv = B->H[p]->mesh.nv;
        for (int c = 0; c < KRHS; ++c) {
          const int j = g * KRHS + c;
          if (j < nr) {
            copy_in(S.vb.p + c * nv, bs[p * nr + j], nv, s);
            copy_in(S.vu.p + c * nv, us[p * nr + j], nv, s);
          } else {
            // unused column: zero right-hand side, converged from the start
            ASMG_CUDA(cudaMemsetAsync(S.vb.p + c * nv, 0, 8 * nv, s));
            ASMG_CUDA(cudaMemsetAsync(S.vu.p + c * nv, 0, 8 * nv, s));
          }
        }
      }
    ASMG_CUDA(cudaGraphLaunch(B->exec, s));
    std::vector<MultiScalars> sc((size_t)np * ngroups);
    for (int p = 0; p < np; ++p)
      for (int g = 0; g < ngroups; ++g) {
        MultiSlot& S = B->mslot(p, g);
        const int64_t nv = B->H[p]->mesh.nv;
        for (int c = 0; c < KRHS && g * KRHS + c < nr; ++c) copy_out(us[p * nr + g * KRHS + c], S.vu.p + c * nv, nv, s);
        ASMG_CUDA(cudaMemcpyAsync(&sc[p * ngroups + g], S.scal.p, sizeof(MultiScalars), cudaMemcpyDeviceToHost, s));
      }
    ASMG_CUDA(cudaStreamSynchronize(s));
    int worst = ASMG_OK;
    for (int p = 0; p < np; ++p)
      for (int j = 0; j < nr; ++j) {
        const MultiScalars& m = sc[p * ngroups + j / KRHS];
        const int c = j % KRHS;
        iterations[p * nr + j] = m.k[c];
        const int st = m.status[c] == 0                    ? ASMG_OK
                       : m.status[c] == ASMG_ERR_BREAKDOWN ? ASMG_ERR_BREAKDOWN
                       : m.status[c] == ASMG_ERR_TIMEOUT   ? ASMG_ERR_TIMEOUT
                                                           : ASMG_NOT_CONVERGED;
        if (status) status[p * nr + j] = st;
        if (st < 0 || (worst == ASMG_OK && st != ASMG_OK)) worst = st;
      }
    if (worst == ASMG_ERR_BREAKDOWN) g_err = "PCG breakdown in a batched solve";
    return worst;
  }
  for (int p = 0; p < np; ++p)
    for (int j = 0; j < nr; ++j) {
      Slot& S = B->slot(p, j);
      const int64_t nv = B->H[p]->mesh.nv;
      copy_in(S.vb.p, bs[p * nr + j], nv, s);
      copy_in(S.vu.p, us[p * nr + j], nv, s);
    }
  ASMG_CUDA(cudaGraphLaunch(B->exec, s));
  std::vector<PcgScalars> sc((size_t)np * nr);
  for (int p = 0; p < np; ++p)
    for (int j = 0; j < nr; ++j) {
      Slot& S = B->slot(p, j);
      copy_out(us[p * nr + j], S.vu.p, B->H[p]->mesh.nv, s);
      ASMG_CUDA(cudaMemcpyAsync(&sc[p * nr + j], S.scal.p, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    }
  ASMG_CUDA(cudaStreamSynchronize(s));
  int worst = ASMG_OK;
  for (size_t k = 0; k < sc.size(); ++k) {
    iterations[k] = sc[k].k;
    const int st = sc[k].status == 0                    ? ASMG_OK
                   : sc[k].status == ASMG_ERR_BREAKDOWN ? ASMG_ERR_BREAKDOWN
                   : sc[k].status == ASMG_ERR_TIMEOUT   ? ASMG_ERR_TIMEOUT
                                                        : ASMG_NOT_CONVERGED;
    if (status) status[k] = st;
    if (st < 0 || (worst == ASMG_OK && st != ASMG_OK)) worst = st;
  }
  if (worst == ASMG_ERR_BREAKDOWN) g_err = "PCG breakdown in a batched solve";
  if (worst == ASMG_ERR_TIMEOUT) g_err = "a bounded device wait expired in a batched solve";
  return worst;
  API_END
}

void amg_batch_destroy(asmg_batch B) { delete B; }

int amg_residual_norm_noalloc(asmg_handle h, const double* b, const double* u, double* out, void* stream) {
  API_BEGIN
  if (!h || !b || !u || !out) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  residual_norm_noalloc(*h, b, u, out, (cudaStream_t)stream);
  return ASMG_OK;
  API_END
}

int amg_profile(asmg_handle h, const double* b, double rtol, double* out, int* iterations, void* stream) {
  API_BEGIN
  if (!h || !b || !out || !iterations) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  Slot& S0 = h->slot0();
  const int64_t nv = h->mesh.nv;
  copy_in(S0.vb.p, b, nv, s);
  gather_rows(*h, S0.vb.p, S0.b.p, s);
  S0.x.zero(s);
  *iterations = profile_solve(*h, rtol, s, out);
  return ASMG_OK;
  API_END
}

int amg_profile_levels(asmg_handle h, const double* b, double rtol, double* out, double* out_levels, int nlev,
                       int* iterations, void* stream) {
  API_BEGIN
  if (!h || !b || !out || !out_levels || !iterations || nlev < 0)
    ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  Slot& S0 = h->slot0();
  const int64_t nv = h->mesh.nv;
  copy_in(S0.vb.p, b, nv, s);
  gather_rows(*h, S0.vb.p, S0.b.p, s);
  S0.x.zero(s);
  *iterations = profile_solve(*h, rtol, s, out, out_levels, nlev);
  return ASMG_OK;
  API_END
}

int amg_solve(asmg_handle h, const double* b, double* u, double rtol, int* iterations, double* res_history,
              void* stream) {
  API_BEGIN
  if (!h || !b || !u || !iterations) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  if (!(rtol >= 0) || !std::isfinite(rtol)) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "rtol must be finite and >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  Slot& S0 = h->slot0();
  const int64_t nv = h->mesh.nv;
  copy_in(S0.vb.p, b, nv, s);
  copy_in(S0.vu.p, u, nv, s);
  gather_rows(*h, S0.vb.p, S0.b.p, s);
  gather_rows(*h, S0.vu.p, S0.x.p, s);
  run_solve(*h, S0, rtol, s);
  scatter_rows(*h, S0.x.p, false, S0.vu.p, s);
  copy_out(u, S0.vu.p, nv, s);
  PcgScalars sc;
  ASMG_CUDA(cudaMemcpyAsync(&sc, S0.scal.p, sizeof sc, cudaMemcpyDeviceToHost, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
  *iterations = sc.k;
  if (res_history) {
    ASMG_CUDA(cudaMemcpyAsync(res_history, S0.hist.p, 8 * (size_t)(sc.k + 1), cudaMemcpyDeviceToHost, s));
    ASMG_CUDA(cudaStreamSynchronize(s));
  }
  if (sc.status == ASMG_ERR_BREAKDOWN) {
    g_err = "PCG breakdown: <p, A p> or <r, z> not positive";
    return ASMG_ERR_BREAKDOWN;
  }
  if (sc.status == ASMG_ERR_TIMEOUT) {
    g_err = "a bounded device wait expired (a tile's shared-memory copy did not complete); u holds the last iterate";
    return ASMG_ERR_TIMEOUT;
  }
  return sc.status == 0 ? ASMG_OK : ASMG_NOT_CONVERGED;
  API_END
}

int amg_solve_multi(asmg_handle h, int k, const double* b, double* u, double rtol, int* iterations, int* status,
                    double* res_history, void* stream) {
  API_BEGIN
  if (!h || !b || !u || !iterations) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  if (k < 1 || k > KRHS) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "k = %d right-hand sides (1..%d)", k, KRHS);
  if (!(rtol >= 0) || !std::isfinite(rtol)) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "rtol must be finite and >= 0");
  if (!multi_supported(*h))
    ASMG_FAIL(ASMG_ERR_UNSUPPORTED, "multiple right-hand sides need the multiplicative Gauss-Seidel PCG without "
                                    "Neumann vertices");
  cudaStream_t s = (cudaStream_t)stream;
  if (h->mslots.empty()) add_multi_slot(*h, s);
  MultiSlot& S = *h->mslots[0];
  const int64_t nv = h->mesh.nv;
  for (int c = 0; c < KRHS; ++c) {
    if (c < k) {
      copy_in(S.vb.p + c * nv, b + c * nv, nv, s);
      copy_in(S.vu.p + c * nv, u + c * nv, nv, s);
    } else {
      ASMG_CUDA(cudaMemsetAsync(S.vb.p + c * nv, 0, 8 * nv, s));
      ASMG_CUDA(cudaMemsetAsync(S.vu.p + c * nv, 0, 8 * nv, s));
    }
  }
  gather_multi(*h, S.vb.p, S.b.p, s);
  gather_multi(*h, S.vu.p, S.x.p, s);
  run_solve_multi(*h, S, rtol, s);
  scatter_multi(*h, S.x.p, S.vu.p, s);
  for (int c = 0; c < k; ++c) copy_out(u + c * nv, S.vu.p + c * nv, nv, s);
  MultiScalars sc;
  ASMG_CUDA(cudaMemcpyAsync(&sc, S.scal.p, sizeof sc, cudaMemcpyDeviceToHost, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
  const int64_t hl = h->prm.max_iter + 1;
  int worst = ASMG_OK;
  for (int c = 0; c < k; ++c) {
    iterations[c] = sc.k[c];
    const int st = sc.status[c] == 0                    ? ASMG_OK
                   : sc.status[c] == ASMG_ERR_BREAKDOWN ? ASMG_ERR_BREAKDOWN
                   : sc.status[c] == ASMG_ERR_TIMEOUT   ? ASMG_ERR_TIMEOUT
                                                        : ASMG_NOT_CONVERGED;
    if (status) status[c] = st;
    if (st < 0 || (worst == ASMG_OK && st != ASMG_OK)) worst = st;
    if (res_history)
      ASMG_CUDA(cudaMemcpyAsync(res_history + c * hl, S.hist.p + c * hl, 8 * (size_t)(sc.k[c] + 1),
                                cudaMemcpyDeviceToHost, s));
  }
  ASMG_CUDA(cudaStreamSynchronize(s));
  if (worst == ASMG_ERR_BREAKDOWN) g_err = "PCG breakdown in a column of a multiple solve";
  return worst;
  API_END
}

int amg_mass_apply(asmg_handle h, const double* f, double* bout, void* stream) {
  API_BEGIN
  if (!h || !f || !bout) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  Slot& S0 = h->slot0();
  const int64_t nv = h->mesh.nv;
  if (!h->d_v2e_ptr.p) {
    // elements around each vertex, ascending element index (counting sort)
    const MeshHost& m = h->mesh;
    const int nvert = m.dim + 1;
    std::vector<int64_t> ptr(nv + 1, 0);
    for (int64_t k = 0; k < m.ne * nvert; ++k) ++ptr[m.E[k] + 1];
    for (int64_t v = 0; v < nv; ++v) ptr[v + 1] += ptr[v];
    std::vector<int32_t> el(m.ne * nvert);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < m.ne; ++e)
      for (int k = 0; k < nvert; ++k) el[fill[m.E[e * nvert + k]]++] = (int32_t)e;
    h->d_v2e_ptr.upload(ptr, s);
    h->d_v2e.upload(el, s);
  }
  copy_in(S0.vb.p, f, nv, s);
  mass_apply_gpu(h->mesh.dim, nv, h->d_v2e_ptr.p, h->d_v2e.p, h->dX.p, h->dE.p, S0.vb.p, S0.vu.p, s);
  gather_rows(*h, S0.vu.p, S0.q.p, s);
  scatter_rows(*h, S0.q.p, false, S0.vu.p, s);  // zero at Dirichlet vertices
  copy_out(bout, S0.vu.p, nv, s);
  ASMG_CUDA(cudaStreamSynchronize(s));
  return ASMG_OK;
  API_END
}

int amg_precond_apply(asmg_handle h, const double* r, double* z, void* stream) {
  API_BEGIN
  if (!h || !r || !z) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  Slot& S0 = h->slot0();
  const int64_t nv = h->mesh.nv;
  copy_in(S0.vb.p, r, nv, s);
  gather_rows(*h, S0.vb.p, S0.r.p, s);
  int* tflag = reinterpret_cast<int*>(reinterpret_cast<char*>(S0.scal.p) + offsetof(PcgScalars, timeout));
  ASMG_CUDA(cudaMemsetAsync(tflag, 0, sizeof(int), s));
  precond_apply(*h, S0.r.p, s);
  if (h->prm.precision == ASMG_MIXED)
    scatter_rows(*h, S0.s32.uf.p, true, S0.vu.p, s);
  else
    scatter_rows(*h, S0.s64.uf.p, false, S0.vu.p, s);
  copy_out(z, S0.vu.p, nv, s);
  int tout = 0;
  ASMG_CUDA(cudaMemcpyAsync(&tout, tflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
  if (tout) ASMG_FAIL(ASMG_ERR_TIMEOUT, "a bounded device wait expired (a tile's shared-memory copy did not complete)");
  return ASMG_OK;
  API_END
}

int amg_spmv(asmg_handle h, const double* x, double* y, void* stream) {
  API_BEGIN
  if (!h || !x || !y) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  Slot& S0 = h->slot0();
  const int64_t nv = h->mesh.nv;
  copy_in(S0.vb.p, x, nv, s);
  gather_rows(*h, S0.vb.p, S0.p.p, s);
  spmv64(*h, S0.p.p, S0.q.p, s);
  scatter_rows(*h, S0.q.p, false, S0.vu.p, s);
  copy_out(y, S0.vu.p, nv, s);
  ASMG_CUDA(cudaStreamSynchronize(s));
  return ASMG_OK;
  API_END
}

}  // extern "C"

namespace {
// dL/da (scale = NULL) or dL/dg = a dL/da for a = exp(g) (scale = the coefficients)
void element_grad_common(asmg_handle h, const double* u, const double* lambda, double* g, bool log_coeff,
                         cudaStream_t s) {
  Slot& S0 = h->slot0();
  const int64_t nv = h->mesh.nv, ne = h->mesh.ne;
  // Dirichlet entries are treated as 0: gather/scatter through the free rows
  copy_in(S0.vb.p, u, nv, s);
  gather_rows(*h, S0.vb.p, S0.p.p, s);
  scatter_rows(*h, S0.p.p, false, S0.vb.p, s);
  copy_in(S0.vu.p, lambda, nv, s);
  gather_rows(*h, S0.vu.p, S0.q.p, s);
  scatter_rows(*h, S0.q.p, false, S0.vu.p, s);
  DBuf<double> dg;
  const bool dev = is_device(g);
  double* out = g;
  if (!dev) {
    dg.alloc(ne);
    out = dg.p;
  }
  element_grad_gpu(h->mesh.dim, ne, h->dX.p, h->dE.p, S0.vb.p, S0.vu.p, log_coeff ? h->dCoeff.p : nullptr, out, s);
  if (!dev) ASMG_CUDA(cudaMemcpyAsync(g, dg.p, 8 * ne, cudaMemcpyDeviceToHost, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
}

void set_coefficients(asmg_handle h, std::vector<double> c, cudaStream_t s) {
  for (int64_t e = 0; e < h->mesh.ne; ++e)
    if (!(c[e] > 0) || !std::isfinite(c[e]))
      ASMG_FAIL(ASMG_ERR_BAD_MESH, "coefficient of element %lld is not positive and finite", (long long)e);
  h->mesh.coeff = std::move(c);
  h->dCoeff.upload(h->mesh.coeff, s);
  build_all(*h, s);
  h->bytes_iter = h->prm.precision == ASMG_MIXED ? iteration_bytes(*h, h->p32) : iteration_bytes(*h, h->p64);
}
}  // namespace

extern "C" {

int amg_element_grad(asmg_handle h, const double* u, const double* lambda, double* g, void* stream) {
  API_BEGIN
  if (!h || !u || !lambda || !g) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  element_grad_common(h, u, lambda, g, false, (cudaStream_t)stream);
  return ASMG_OK;
  API_END
}

int amg_element_grad_log(asmg_handle h, const double* u, const double* lambda, double* g, void* stream) {
  API_BEGIN
  if (!h || !u || !lambda || !g) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  element_grad_common(h, u, lambda, g, !h->mesh.coeff.empty(), (cudaStream_t)stream);
  return ASMG_OK;
  API_END
}

int amg_set_log_coefficients(asmg_handle h, const double* gl, void* stream) {
  API_BEGIN
  if (!h || !gl) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<double> c = to_host(gl, h->mesh.ne, s);
  for (auto& x : c) {
    if (!std::isfinite(x)) ASMG_FAIL(ASMG_ERR_BAD_MESH, "log-coefficient is not finite");
    x = std::exp(x);
  }
  set_coefficients(h, std::move(c), s);
  return ASMG_OK;
  API_END
}

int amg_update_coefficients(asmg_handle h, const double* coeff, void* stream) {
  API_BEGIN
  if (!h || !coeff) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  set_coefficients(h, to_host(coeff, h->mesh.ne, s), s);
  return ASMG_OK;
  API_END
}

int amg_info(asmg_handle h, int what, int level, int64_t* value) {
  API_BEGIN
  if (!h || !value) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  auto lev_index = [&](int l) -> int {
    int k = l - (h->aux.c + 1);
    if (k < 0 || k >= (int)h->aux.levels.size()) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "level %d has no smoothing data", l);
    return k;
  };
  auto nsm = [&](int k) -> int64_t {
    return h->prm.precision == ASMG_MIXED ? h->p32.lev[k].nsm_real : h->p64.lev[k].nsm_real;
  };
  switch (what) {
    case ASMG_INFO_NFREE: *value = h->n; break;
    case ASMG_INFO_J: *value = h->aux.J; break;
    case ASMG_INFO_COARSE: *value = h->aux.c; break;
    case ASMG_INFO_NAUX:
      if (level < 0 || level > h->aux.J) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "bad level");
      if (!h->aux.phi.empty()) {
        // mixed grids: the nodes free on this level (phi <= l < psi)
        int64_t c = 0;
        for (size_t q = 0; q < h->aux.phi.size(); ++q) c += h->aux.phi[q] <= level && level < h->aux.psi[q];
        *value = c;
      } else {
        *value = h->aux.nlevel[level];
      }
      break;
    case ASMG_INFO_NSMOOTH: *value = level < 0 ? h->n : nsm(lev_index(level)); break;
    case ASMG_INFO_NCOLOURS:
      if (level < 0) {
        *value = (int64_t)h->fine_cstart.size() - 1;
      } else {
        int k = lev_index(level);
        *value = h->prm.precision == ASMG_MIXED ? h->p32.lev[k].ncolours : h->p64.lev[k].ncolours;
      }
      break;
    case ASMG_INFO_NTREE_LEVELS: *value = (int64_t)h->tree.seg.size(); break;
    case ASMG_INFO_NSEG:
      if (level < 0 || level >= (int)h->tree.seg.size()) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "bad level");
      *value = (int64_t)h->tree.seg[level].size() / 4;
      break;
    case ASMG_INFO_NSPLIT:
      if (level < 0 || level >= (int)h->aux.split.size()) *value = 0;
      else *value = (int64_t)h->aux.split[level].size();
      break;
    case ASMG_INFO_NNZ_A: *value = h->A64.nnz_real; break;
    case ASMG_INFO_NNZ_P: *value = (int64_t)h->aux.P.r.size(); break;
    case ASMG_INFO_NROWS_E: {
      int k = lev_index(level);
      *value = h->prm.precision == ASMG_MIXED ? h->p32.lev[k].nrs : h->p64.lev[k].nrs;
      break;
    }
    case ASMG_INFO_BYTES_ITER: *value = h->bytes_iter; break;
    case ASMG_INFO_NNZ_LEVEL: {
      int k = lev_index(level);
      *value = h->prm.precision == ASMG_MIXED ? h->p32.lev[k].SM.nnz_real + h->p32.lev[k].RS.nnz_real
                                              : h->p64.lev[k].SM.nnz_real + h->p64.lev[k].RS.nnz_real;
      break;
    }
    case ASMG_INFO_NTILES: {
      int k = lev_index(level);
      *value = h->prm.precision == ASMG_MIXED ? (h->p32.lev[k].tiled_down ? h->p32.lev[k].tdown.ntiles : 0)
                                              : (h->p64.lev[k].tiled_down ? h->p64.lev[k].tdown.ntiles : 0);
      break;
    }
    case ASMG_INFO_NTILES_UP: {
      int k = lev_index(level);
      *value = h->prm.precision == ASMG_MIXED ? (h->p32.lev[k].tiled_up ? h->p32.lev[k].tup.ntiles : 0)
                                              : (h->p64.lev[k].tiled_up ? h->p64.lev[k].tup.ntiles : 0);
      break;
    }
    case ASMG_INFO_HALO_ROWS: {
      int k = lev_index(level);
      *value = h->prm.precision == ASMG_MIXED ? h->p32.lev[k].tdown.halo : h->p64.lev[k].tdown.halo;
      break;
    }
    case 100: *value = h->gpu_launches_per_iter; break;
    case 101: *value = (int64_t)(h->stats.t_total * 1e6); break;
    case 102: *value = (int64_t)(h->stats.t_tree * 1e6); break;
    case 103: *value = (int64_t)(h->stats.t_aux * 1e6); break;
    case 104: *value = (int64_t)(h->stats.t_fine * 1e6); break;
    case 105: *value = (int64_t)(h->stats.t_levels * 1e6); break;
    case 108: *value = (int64_t)(h->stats.t_lv_assemble * 1e6); break;
    case 109: *value = (int64_t)(h->stats.t_lv_colour * 1e6); break;
    case 110: *value = (int64_t)(h->stats.t_lv_pack * 1e6); break;
    case 111: *value = (int64_t)(h->stats.t_lv_export * 1e6); break;
    case 112: *value = (int64_t)(h->stats.t_coarse * 1e6); break;
    case 113: *value = (int64_t)(h->stats.t_transfer * 1e6); break;
    case 114: *value = (int64_t)(h->stats.t_slots * 1e6); break;
    case 115: *value = (int64_t)(h->stats.t_sz * 1e6); break;
    default: ASMG_FAIL(ASMG_ERR_INVALID_ARG, "unknown info %d", what);
  }
  return ASMG_OK;
  API_END
}

int amg_export(asmg_handle h, int what, int level, void* buf, int64_t* count) {
  API_BEGIN
  if (!h || !count) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = 0;
  auto put = [&](const void* src, int64_t n, size_t elem) {
    *count = n;
    if (buf && n) std::memcpy(buf, src, elem * n);
  };
  auto trip = [&](const std::vector<uint64_t>& a, const std::vector<uint64_t>& b2, const std::vector<double>& v) {
    *count = (int64_t)v.size();
    if (!buf) return;
    char* o = (char*)buf;
    for (size_t k = 0; k < v.size(); ++k) {
      std::memcpy(o + 24 * k, &a[k], 8);
      std::memcpy(o + 24 * k + 8, &b2[k], 8);
      std::memcpy(o + 24 * k + 16, &v[k], 8);
    }
  };
  switch (what) {
    case ASMG_EXPORT_KEYS: {
      auto k = h->tree.keys.download(s);
      put(k.data(), (int64_t)k.size(), 8);
      break;
    }
    case ASMG_EXPORT_PERM: {
      auto k = h->tree.perm.download(s);
      put(k.data(), (int64_t)k.size(), 4);
      break;
    }
    case ASMG_EXPORT_SEG:
      if (level < 0 || level >= (int)h->tree.seg.size()) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "bad level");
      put(h->tree.seg[level].data(), (int64_t)h->tree.seg[level].size(), 8);
      break;
    case ASMG_EXPORT_SPLIT:
      if (level < 0 || level >= (int)h->aux.split.size()) {
        *count = 0;
      } else {
        put(h->aux.split[level].data(), (int64_t)h->aux.split[level].size(), 8);
      }
      break;
    case ASMG_EXPORT_AUX_KEYS: put(h->aux.aux_key.data(), (int64_t)h->aux.aux_key.size(), 8); break;
    case ASMG_EXPORT_FINE_COLOUR: put(h->fine_colour.data(), (int64_t)h->fine_colour.size(), 4); break;
    case ASMG_EXPORT_SMOOTH: {
      int k = level - (h->aux.c + 1);
      if (k < 0 || k >= (int)h->level_smooth_keys.size()) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "bad level");
      std::vector<uint64_t> v;
      for (size_t i = 0; i < h->level_smooth_keys[k].size(); ++i) {
        v.push_back(h->level_smooth_keys[k][i]);
        v.push_back((uint64_t)h->level_smooth_colour[k][i]);
      }
      put(v.data(), (int64_t)v.size(), 8);
      break;
    }
    case ASMG_EXPORT_LEVEL_ROWS: {
      int k = level - (h->aux.c + 1);
      std::vector<uint64_t> a, b2;
      std::vector<double> v;
      if (level == h->aux.c) {
        // coarsest level: full matrix from its triangles is not stored; export the inverse's source is not kept
        ASMG_FAIL(ASMG_ERR_INVALID_ARG, "the coarsest level keeps only its inverse");
      }
      if (k < 0 || k >= (int)h->level_rows.size()) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "bad level");
      const Triplets& t = h->level_rows[k];
      for (size_t q = 0; q < t.v.size(); ++q) {
        a.push_back(h->aux.aux_key[t.r[q]]);
        b2.push_back(h->aux.aux_key[t.c[q]]);
        v.push_back(t.v[q]);
      }
      trip(a, b2, v);
      break;
    }
    case ASMG_EXPORT_P: {
      std::vector<uint64_t> a, b2;
      std::vector<double> v;
      const Triplets& t = h->aux.P;
      for (size_t q = 0; q < t.v.size(); ++q) {
        a.push_back((uint64_t)h->vertex_of_free[t.r[q]]);
        b2.push_back(h->aux.aux_key[t.c[q]]);
        v.push_back(t.v[q]);
      }
      trip(a, b2, v);
      break;
    }
    case ASMG_EXPORT_FINE_A: {
      std::vector<uint64_t> a, b2;
      std::vector<double> v;
      const HostCSR& A = h->A_host;
      for (int64_t i = 0; i < A.nr; ++i)
        for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
          a.push_back((uint64_t)h->vertex_of_free[i]);
          b2.push_back((uint64_t)h->vertex_of_free[A.col[p]]);
          v.push_back(A.val[p]);
        }
      trip(a, b2, v);
      break;
    }
    default: ASMG_FAIL(ASMG_ERR_INVALID_ARG, "unknown export %d", what);
  }
  return ASMG_OK;
  API_END
}

}  // extern "C"
