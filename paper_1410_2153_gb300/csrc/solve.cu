// The solve phase on the device: PCG (Sec. 5.2) preconditioned by the
// multiplicative auxiliary-space preconditioner (Algorithm 1) whose
// auxiliary correction is the V-cycle of Algorithm 2 on the nested grids.
//
// Layout.  Fine vectors live in a permuted, padded order: free dofs grouped
// by colour, each colour block padded to a multiple of 32 rows, so a colour
// sweep is one contiguous range of SELL-32 slices.  Auxiliary vectors are
// indexed by the free nodes of the finest auxiliary level (lattice Morton
// order); every coarser level's nodes are a subset, so one rhs vector F and
// one correction vector U serve all levels and the V-cycle updates them in
// place:
//   down, level l:  save F on N~_l (first pre-sweep), nu_pre forward sweeps
//                   on N~_l, F -= A_l U on the rows E_l touched by N~_l,
//                   F[parent] += 1/2 F[new child] (I_l^T).  U is 0 on the
//                   whole down path: the level's correction lives in its
//                   saved array us (SM row order) and never enters U there;
//   coarsest:       U = A_c^{-1} F on its nodes (explicit FP64 inverse);
//   up, level l:    U[new] = (U[p0] + U[p1]) / 2 (I_l), U += saved values,
//                   nu_post backward sweeps with the saved F.
// New nodes are midpoints of coarse edges (Sec. 3.3), hence the 1/2 weights.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <type_traits>
#include <vector>

#include "handle.h"
#include "kernels.h"

namespace asmg {

namespace {

using namespace kern;

// ------------------------------------------------------------- fine grid
// one colour of a Gauss-Seidel sweep: u_i += (rhs_i - (A u)_i) / a_ii
template <class T, class R>
__global__ void k_gs_fine(int64_t r0, int64_t nrows, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                          const T* __restrict__ val, const T* __restrict__ dinv, const R* __restrict__ rhs, T* u) {
  const int64_t i = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = i < r0 + nrows;
  Row<T> row;
  T di = 0;
  if (act) {
    row_load(row, i, off, col, val);
    di = dinv[i];
  }
  pdl_wait();
  if (act) {
    const T s = (T)rhs[i] - row_dot(row, col, val, u);
    u[i] += s * di;
  }
  pdl_trigger();
}

// rho = r - A u
template <class T>
__global__ void k_resid_fine(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                             const T* __restrict__ val, const double* __restrict__ r, const T* __restrict__ u,
                             T* __restrict__ rho) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = i < n;
  Row<T> row;
  if (act) row_load(row, i, off, col, val);
  pdl_wait();
  if (act) rho[i] = (T)r[i] - row_dot(row, col, val, u);
  pdl_trigger();
}

// F = P^T rho on the auxiliary nodes, and U = 0 (start of the V-cycle)
template <class T>
__global__ void k_restrict_fine(int64_t nJ, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                const T* __restrict__ val, const T* __restrict__ rho, T* __restrict__ F,
                                T* __restrict__ U) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = k < nJ;
  Row<T> row;
  if (act) row_load(row, k, off, col, val);
  pdl_wait();
  if (act) {
    F[k] = row_dot(row, col, val, rho);
    U[k] = 0;
  }
  pdl_trigger();
}

// u += P U
template <class T>
__global__ void k_prolong_fine(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                               const T* __restrict__ val, const T* __restrict__ U, T* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = i < n;
  Row<T> row;
  if (act) row_load(row, i, off, col, val);
  pdl_wait();
  if (act) u[i] += row_dot(row, col, val, U);
  pdl_trigger();
}

// Jacobi smoother (S = D^{-1}): first step from zero, u = D^{-1} r
template <class T>
__global__ void k_jac_first(int64_t n, const T* __restrict__ dinv, const double* __restrict__ r, T* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = i < n;
  const T di = act ? dinv[i] : (T)0;
  pdl_wait();
  if (act) u[i] = di * (T)r[i];
  pdl_trigger();
}

// a further Jacobi step, u += D^{-1} rho with rho = r - A u taken before
template <class T>
__global__ void k_jac_add(int64_t n, const T* __restrict__ dinv, const T* __restrict__ rho, T* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = i < n;
  const T di = act ? dinv[i] : (T)0;
  pdl_wait();
  if (act) u[i] += di * rho[i];
  pdl_trigger();
}

// additive form: the auxiliary correction acts on r itself (rho = r)
template <class T>
__global__ void k_cast_fine(int64_t n, const double* __restrict__ r, T* __restrict__ rho) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  pdl_wait();
  if (i < n) rho[i] = (T)r[i];
  pdl_trigger();
}

// ------------------------------------------------------ auxiliary levels
// one colour of an up (post-smoothing) sweep on the smoothing rows of a
// level: U[i] += (fs_k - (A_l U)_i) / a_ii with the F saved on the way down
template <class T, class V>
__global__ void k_gs_aux(int64_t k0, int64_t nk, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                         const V* __restrict__ val, const T* __restrict__ dinv, const int32_t* __restrict__ rows,
                         const T* __restrict__ fs, T* U) {
  const int64_t k = k0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int32_t i = -1;
  Row<T> row;
  T di = 0;
  if (k < k0 + nk) {
    i = rows[k];
    if (i >= 0) {
      row_load(row, k, off, col, val);
      di = dinv[k];
    }
  }
  pdl_wait();
  if (i >= 0) {
    const T s = fs[k] - row_dot(row, col, val, U);
    U[i] += s * di;
  }
  pdl_trigger();
}

// one colour of a down (pre-smoothing) sweep, on the level's own correction
// us in SM row order.  The V-cycle reaches level l with U = 0, and the down
// path changes U only on N~_l, so the sweeps run on us alone with the rows'
// columns in N~_l (SMd).  In the first sweep us is 0 on this class and the
// later ones: only columns of earlier classes (below k0) are read, and the
// class's rows are set rather than updated.  The first sweep takes F and
// saves it in fs.
template <class T, class V>
__global__ void k_gs_aux_down(int64_t k0, int64_t nk, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                              const V* __restrict__ val, const T* __restrict__ dinv, const int32_t* __restrict__ rows,
                              const T* __restrict__ F, int first, T* __restrict__ fs, T* us) {
  const int64_t k = k0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int32_t i = -1;
  Row<T> row;
  T di = 0;
  if (k < k0 + nk) {
    i = rows[k];
    if (i >= 0) {
      row_load(row, k, off, col, val);
      di = dinv[k];
    }
  }
  pdl_wait();
  if (i >= 0) {
    T f, acc = 0;
    if (first) {
      f = F[i];
      fs[k] = f;
#pragma unroll
      for (int q = 0; q < MAXW; ++q)
        if (q < row.w && row.c[q] < k0) acc += row.v[q] * us[row.c[q]];
      for (int q = MAXW; q < row.w; ++q) {
        const int64_t e = row.b + ((int64_t)q << 5) + row.lane;
        const int32_t c = __ldg(col + e);
        if (c < k0) acc += (T)ldg_val(val + e) * us[c];
      }
      us[k] = (f - acc) * di;
    } else {
      f = fs[k];
      acc = row_dot(row, col, val, us);
      us[k] += (f - acc) * di;
    }
  }
  pdl_trigger();
}

// F_i -= sum_{j in N~_l} a_ij U_j on the rows E_l
template <class T, class V>
__global__ void k_resid_aux(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                            const V* __restrict__ val, const int32_t* __restrict__ rows, const T* __restrict__ U,
                            T* __restrict__ F) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int32_t i = -1;
  Row<T> row;
  if (k < n) {
    i = rows[k];
    if (i >= 0) row_load(row, k, off, col, val);
  }
  pdl_wait();
  if (i >= 0) F[i] -= row_dot(row, col, val, U);
  pdl_trigger();
}

// I_l^T: F[parent] += 1/2 sum F[new children]
template <class T>
__global__ void k_restrict_aux(int64_t npar, const int32_t* __restrict__ pid, const int32_t* __restrict__ pptr,
                               const int32_t* __restrict__ child, T* __restrict__ F) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int32_t par = -1, p0 = 0, p1 = 0;
  if (t < npar) {
    par = pid[t];
    p0 = pptr[t];
    p1 = pptr[t + 1];
  }
  pdl_wait();
  if (par >= 0) {
    T acc = 0;
    for (int32_t p = p0; p < p1; ++p) acc += F[child[p]];
    F[par] += (T)0.5 * acc;
  }
  pdl_trigger();
}

// I_l: U[new] = (U[p0] + U[p1]) / 2, Dirichlet parents contribute 0
template <class T>
__global__ void k_prolong_aux(int64_t nnew, const int32_t* __restrict__ id, const int32_t* __restrict__ p0,
                              const int32_t* __restrict__ p1, T* U) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int32_t a = -1, b = -1, me = -1;
  if (t < nnew) {
    a = p0[t];
    b = p1[t];
    me = id[t];
  }
  pdl_wait();
  if (me >= 0) {
    T v = 0;
    if (a >= 0) v += U[a];
    if (b >= 0) v += U[b];
    U[me] = (T)0.5 * v;
  }
  pdl_trigger();
}

template <class T>
__global__ void k_addsaved_aux(int64_t nsm, const int32_t* __restrict__ rows, const T* __restrict__ us, T* U) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int32_t i = t < nsm ? rows[t] : -1;
  pdl_wait();
  if (i >= 0) U[i] += us[t];
  pdl_trigger();
}

// coarsest level: U[cid] = A_c^{-1} F[cid] in FP64, one warp per row
template <class T>
__global__ void k_coarse(int64_t nc, const int32_t* __restrict__ cid, const double* __restrict__ inv,
                         const T* __restrict__ F, T* __restrict__ U) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  pdl_wait();
  if (row < nc) {
    double s = 0;
    for (int64_t j = lane; j < nc; j += 32) s += inv[row * nc + j] * (double)F[cid[j]];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) U[cid[row]] = (T)s;
  }
  pdl_trigger();
}

// ------------------------------------------- tiled sweeps (one launch each)
// One thread block per tile (see TileSweeps): the tile's rows -- its own rows
// of N~_l plus the halo its sweeps read -- are copied into shared memory with
// one bulk copy (cp.async.bulk, completion on an mbarrier), and the rows'
// rhs, diagonal inverse and current value live there too; the colour phases
// of all nu sweeps are separated by __syncthreads.  Each row is updated with
// the same arithmetic, over the same stored entries in the same order, as
// k_gs_aux_down / k_gs_aux do; the entries a tile leaves out are exactly
// those whose value cannot reach the tile's own rows' results, so those
// results equal the class-by-class launches bit for bit.  Halo results are
// discarded.
constexpr int TILE_TPB = 256;
// bound on the wait for the bulk copy (SM clock cycles, about 1 s): when it
// expires the block records the timeout, waits once more (bounded) for its
// copy to land, and skips its work
constexpr long long TILE_WAIT_CYCLES = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for phase 0 of the mbarrier
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, 0))
    if (clock64() - t0 > TILE_WAIT_CYCLES) return false;
  return true;
}

// Stage the tile's block of `bytes` bytes (16-byte aligned, multiple of 16)
// into shared memory: thread 0 arms the barrier and issues the copy.  The
// mbarrier lives in static shared memory.
__device__ __forceinline__ void tile_stage(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  if (threadIdx.x == 0) {
    const uint32_t b = smem_addr(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
  }
}

// Every thread waits for the copy (bounded); false in every thread when any
// thread's wait expired, after the timeout is recorded and the copy given a
// second bounded wait.  inject != 0 (failure injection, asmg_params::
// inject_timeout) takes the expired path without polling; the copy is still
// waited for before the block exits.
__device__ __forceinline__ bool tile_staged(uint64_t* bar, int* timeout, int inject) {
  const uint32_t b = smem_addr(bar);
  __syncthreads();  // the barrier was initialised by thread 0 before this point
  const bool ok = __syncthreads_and(!inject && mbar_wait_bounded(b));
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(timeout, 1);
    mbar_wait_bounded(b);
    __syncthreads();
  }
  return ok;
}

// the row's entries in stored order, four loaded ahead of their use (the sum
// is formed in the same order as a plain loop)
template <class T, class V>
__device__ __forceinline__ T tile_row_dot(int r, const int32_t* soff, const uint16_t* col, const V* val, const T* Ul) {
  const int sl = r >> 5, lane = r & 31;
  const int b = soff[sl], w = (soff[sl + 1] - b) >> 5;
  T acc = 0;
  int e = 0;
  for (; e + 4 <= w; e += 4) {
    const int q = b + (e << 5) + lane;
    const int c0 = col[q], c1 = col[q + 32], c2 = col[q + 64], c3 = col[q + 96];
    const T v0 = (T)val_of(val[q]), v1 = (T)val_of(val[q + 32]), v2 = (T)val_of(val[q + 64]),
            v3 = (T)val_of(val[q + 96]);
    const T x0 = Ul[c0], x1 = Ul[c1], x2 = Ul[c2], x3 = Ul[c3];
    acc += v0 * x0;
    acc += v1 * x1;
    acc += v2 * x2;
    acc += v3 * x3;
  }
  for (; e < w; ++e) {
    const int q = b + (e << 5) + lane;
    acc += (T)val_of(val[q]) * Ul[col[q]];
  }
  return acc;
}

// the staged block of a tile (TileLayout) and, after it, U (local rows and
// outside values) and F
template <class T, class V>
struct TileSmem {
  const int32_t* soff;
  const uint16_t* col;
  const V* val;
  const T* dinv;
  const int32_t* lsm;
  const int32_t* laux;
  const int32_t* ext;
  T *Ul, *Fl;
};

template <class T, class V>
__device__ __forceinline__ TileSmem<T, V> tile_smem(unsigned char* raw, int64_t maxblob, int maxloc, int maxext,
                                                    int nl, int nx) {
  TileSmem<T, V> t;
  t.soff = reinterpret_cast<const int32_t*>(raw);
  const TileLayout lay = tile_layout(nl, t.soff[nl >> 5], nx, (int64_t)sizeof(T), (int64_t)sizeof(V));
  t.col = reinterpret_cast<const uint16_t*>(raw + lay.col);
  t.val = reinterpret_cast<const V*>(raw + lay.val);
  t.dinv = reinterpret_cast<const T*>(raw + lay.dinv);
  t.lsm = reinterpret_cast<const int32_t*>(raw + lay.lsm);
  t.laux = reinterpret_cast<const int32_t*>(raw + lay.laux);
  t.ext = reinterpret_cast<const int32_t*>(raw + lay.ext);
  t.Ul = reinterpret_cast<T*>(raw + maxblob);
  t.Fl = t.Ul + maxloc + maxext;
  return t;
}

// pre-sweeps: us (the level's own correction, SM order) starts at 0; the
// first sweep saves F on the tile's own rows in fs.  The block is copied in
// while the previous kernel finishes.
template <class T, class V>
__global__ void __launch_bounds__(TILE_TPB) k_tile_down(const int64_t* __restrict__ loc_off,
                                                        const int64_t* __restrict__ blob_off,
                                                        const unsigned char* __restrict__ blob,
                                                        const int32_t* __restrict__ phase, int ncol, int64_t maxblob,
                                                        int maxloc, const T* __restrict__ F, T* __restrict__ fs,
                                                        T* __restrict__ us, int nu, int* timeout, int inject) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t base = loc_off[blockIdx.x];
  const int nl = (int)(loc_off[blockIdx.x + 1] - base);
  const int64_t b0 = blob_off[blockIdx.x];
  const uint32_t bytes = (uint32_t)(blob_off[blockIdx.x + 1] - b0);
  const int32_t* ph = phase + (int64_t)blockIdx.x * (ncol + 1);
  tile_stage(smraw, blob + b0, bytes, &bar);
  pdl_wait();
  if (tile_staged(&bar, timeout, inject)) {
    TileSmem<T, V> t = tile_smem<T, V>(smraw, maxblob, maxloc, 0, nl, 0);
    for (int k = threadIdx.x; k < nl; k += blockDim.x) {
      const int32_t g = t.lsm[k];
      T f = 0;
      if (g != -1) {
        f = F[t.laux[k]];
        if (g >= 0) fs[g] = f;
      }
      t.Fl[k] = f;
      t.Ul[k] = 0;
    }
    __syncthreads();
    for (int sw = 0; sw < nu; ++sw)
      for (int c = 0; c < ncol; ++c) {
        for (int k = ph[c] + threadIdx.x; k < ph[c + 1]; k += blockDim.x) {
          const T acc = tile_row_dot<T, V>(k, t.soff, t.col, t.val, t.Ul);
          t.Ul[k] += (t.Fl[k] - acc) * t.dinv[k];
        }
        __syncthreads();
      }
    for (int k = threadIdx.x; k < nl; k += blockDim.x) {
      const int32_t g = t.lsm[k];
      if (g >= 0) us[g] = t.Ul[k];
    }
  }
  pdl_trigger();
}

// start of the up path of a tiled level: the prolongation of the coarse
// correction (I_l: new nodes take the mean of their parents) plus the level's
// saved correction, and the saved rhs, written for every SM row to each place
// the row holds in the post-sweep tiles (own and halo copies; TileSweeps::
// pos).  U itself is not written, so the tiles can copy their start values in
// while other tiles write their results to U.
template <class T>
__global__ void k_up_init(int64_t nsm, const int32_t* __restrict__ rows, const int32_t* __restrict__ par0,
                          const int32_t* __restrict__ par1, const int64_t* __restrict__ pos_ptr,
                          const int32_t* __restrict__ pos, const T* __restrict__ U, const T* __restrict__ us,
                          const T* __restrict__ fs, T* __restrict__ ust, T* __restrict__ fsl) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int32_t i = -1, a = -3, b = -3;
  int64_t p0 = 0, p1 = 0;
  if (k < nsm) {
    i = rows[k];
    a = par0[k];
    b = par1[k];
    p0 = pos_ptr[k];
    p1 = pos_ptr[k + 1];
  }
  pdl_wait();
  if (i >= 0) {
    T v;
    if (a == -3) {
      v = U[i];
    } else {
      T p = 0;
      if (a >= 0) p += U[a];
      if (b >= 0) p += U[b];
      v = (T)0.5 * p;
    }
    v = v + us[k];
    const T f = fs[k];
    for (int64_t q = p0; q < p1; ++q) {
      const int32_t o = pos[q];
      ust[o] = v;
      fsl[o] = f;
    }
  }
  pdl_trigger();
}

// post-sweeps (backward colour order) from the start values and saved rhs
// that k_up_init wrote in tile order: both arrive by bulk copy after the
// wait on the previous kernel, the tile's block before it; the columns
// outside N~_l (the tile's outside values) are read from U once; the tile's
// own rows are written to U
template <class T, class V>
__global__ void __launch_bounds__(TILE_TPB) k_tile_up(const int64_t* __restrict__ loc_off,
                                                      const int64_t* __restrict__ blob_off,
                                                      const unsigned char* __restrict__ blob,
                                                      const int64_t* __restrict__ ext_off,
                                                      const int32_t* __restrict__ phase, int ncol, int64_t maxblob,
                                                      int maxloc, int maxext, const T* __restrict__ ust,
                                                      const T* __restrict__ fsl, T* U, int nu, int* timeout,
                                                      int inject) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar, bar2;
  const int64_t base = loc_off[blockIdx.x];
  const int nl = (int)(loc_off[blockIdx.x + 1] - base);
  const int64_t b0 = blob_off[blockIdx.x];
  const uint32_t bytes = (uint32_t)(blob_off[blockIdx.x + 1] - b0);
  const int nx = (int)(ext_off[blockIdx.x + 1] - ext_off[blockIdx.x]);
  const int32_t* ph = phase + (int64_t)blockIdx.x * (ncol + 1);
  T* Ul = reinterpret_cast<T*>(smraw + maxblob);
  T* Fl = Ul + maxloc + maxext;
  if (threadIdx.x == 0) {
    // initialised before tile_stage's fence.mbarrier_init, which covers it
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar2)) : "memory");
  }
  tile_stage(smraw, blob + b0, bytes, &bar);
  pdl_wait();
  if (threadIdx.x == 0) {
    const uint32_t b2 = smem_addr(&bar2), vb = (uint32_t)((int64_t)nl * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b2), "r"(2 * vb) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(Ul)),
                 "l"(ust + base), "r"(vb), "r"(b2)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(Fl)),
                 "l"(fsl + base), "r"(vb), "r"(b2)
                 : "memory");
  }
  const bool ok1 = tile_staged(&bar, timeout, inject);
  // the outside values, once the block (which holds their IDs) is in place
  TileSmem<T, V> t = tile_smem<T, V>(smraw, maxblob, maxloc, maxext, nl, nx);
  if (ok1)
    for (int e = threadIdx.x; e < nx; e += blockDim.x) t.Ul[nl + e] = U[t.ext[e]];
  const bool ok2 = tile_staged(&bar2, timeout, inject || !ok1);
  if (ok1 && ok2) {
    for (int sw = 0; sw < nu; ++sw)
      for (int c = ncol - 1; c >= 0; --c) {
        for (int k = ph[c] + threadIdx.x; k < ph[c + 1]; k += blockDim.x) {
          const T acc = tile_row_dot<T, V>(k, t.soff, t.col, t.val, t.Ul);
          t.Ul[k] += (t.Fl[k] - acc) * t.dinv[k];
        }
        __syncthreads();
      }
    for (int k = threadIdx.x; k < nl; k += blockDim.x)
      if (t.lsm[k] >= 0) U[t.laux[k]] = t.Ul[k];
  }
  pdl_trigger();
}

// ------------------------------------------- near-boundary solve (Alg. 3)
// After the coarse-grid correction of a level with mixed boundaries:
// r_J = f_J - (A_l U)_J on the near-boundary set J = J_{l,j}, then the exact
// solve A_JJ d = r_J by block cyclic reduction (NbDev), then U_J += d.

// r_J in the factor's order (the saved rhs of a whole-level smoothing set)
template <class T>
__global__ void k_nb_resid(int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                           const T* __restrict__ val, const int32_t* __restrict__ sm, const T* __restrict__ fs,
                           const T* U, double* __restrict__ rhs) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = q < m;
  Row<T> row;
  int32_t k = 0;
  if (act) {
    row_load(row, q, off, col, val);
    k = sm[q];
  }
  pdl_wait();
  if (act) rhs[q] = (double)(fs[k] - row_dot(row, col, val, U));
  pdl_trigger();
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// x := F^{-T} F^{-1} x for the lower Cholesky factor F (s x s, row-major) of
// a block, one warp; x in global memory (lane 0 writes, __syncwarp orders)
__device__ void nb_chol_solve(const double* __restrict__ F, int s, double* x) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < s; ++i) {
    double t = 0;
    for (int k = lane; k < i; k += 32) t += F[(int64_t)i * s + k] * x[k];
    t = warp_sum(t);
    if (lane == 0) x[i] = (x[i] - t) / F[(int64_t)i * s + i];
    __syncwarp();
  }
  for (int i = s - 1; i >= 0; --i) {
    double t = 0;
    for (int k = i + 1 + lane; k < s; k += 32) t += F[(int64_t)k * s + i] * x[k];
    t = warp_sum(t);
    if (lane == 0) x[i] = (x[i] - t) / F[(int64_t)i * s + i];
    __syncwarp();
  }
}

// y -= M z for M (r x c, row-major), one warp, lanes over the rows
__device__ void nb_gemv_sub(const double* __restrict__ M, int r, int c, const double* z, double* y) {
  for (int i = threadIdx.x & 31; i < r; i += 32) {
    double t = y[i];
    for (int j = 0; j < c; ++j) t -= M[(int64_t)i * c + j] * z[j];
    y[i] = t;
  }
  __syncwarp();
}

__device__ void nb_copy(const double* src, double* dst, int n) {
  for (int i = threadIdx.x & 31; i < n; i += 32) dst[i] = src[i];
  __syncwarp();
}

constexpr int NB_TPB = 1024;

// One thread block: the rounds of the reduction (odd blocks solved, even
// blocks' right-hand sides updated), the last block, then the rounds
// backwards (odd blocks from their even neighbours), then U_J += d.  The
// blocks of a step are independent: one warp each.
template <class T>
__global__ void __launch_bounds__(NB_TPB) k_nb_solve(int R, const int32_t* __restrict__ nblk,
                                                     const int32_t* __restrict__ boff, const int64_t* __restrict__ btab,
                                                     const int64_t* __restrict__ voff, const double* __restrict__ mats,
                                                     int last_size, int64_t last_off, int64_t m,
                                                     const int32_t* __restrict__ aux, double* rhs, double* sol, T* U) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  pdl_wait();
  for (int r = 0; r < R; ++r) {
    const int n = nblk[r];
    const int64_t* bt = btab + (int64_t)boff[r] * 5;
    double* V = rhs + voff[r];
    double* Y = sol + voff[r];
    double* Vn = rhs + voff[r + 1];
    const int64_t* btn = r + 1 < R ? btab + (int64_t)boff[r + 1] * 5 : nullptr;
    for (int k = 1 + 2 * warp; k < n; k += 2 * nw) {
      const int sk = (int)bt[5 * k];
      const int64_t o = bt[5 * k + 1];
      nb_copy(V + o, Y + o, sk);
      nb_chol_solve(mats + bt[5 * k + 2], sk, Y + o);
    }
    __syncthreads();
    for (int e = 2 * warp; e < n; e += 2 * nw) {
      const int se = (int)bt[5 * e];
      const int64_t o = bt[5 * e + 1], on = btn ? btn[5 * (e / 2) + 1] : 0;
      nb_copy(V + o, Vn + on, se);
      if (e > 0) nb_gemv_sub(mats + bt[5 * e + 3], se, (int)bt[5 * (e - 1)], Y + bt[5 * (e - 1) + 1], Vn + on);
      if (e + 1 < n) nb_gemv_sub(mats + bt[5 * e + 4], se, (int)bt[5 * (e + 1)], Y + bt[5 * (e + 1) + 1], Vn + on);
    }
    __syncthreads();
  }
  if (warp == 0) {
    nb_copy(rhs + voff[R], sol + voff[R], last_size);
    nb_chol_solve(mats + last_off, last_size, sol + voff[R]);
  }
  __syncthreads();
  for (int r = R - 1; r >= 0; --r) {
    const int n = nblk[r];
    const int64_t* bt = btab + (int64_t)boff[r] * 5;
    const double* V = rhs + voff[r];
    double* S = sol + voff[r];
    const double* Sn = sol + voff[r + 1];
    const int64_t* btn = r + 1 < R ? btab + (int64_t)boff[r + 1] * 5 : nullptr;
    for (int e = 2 * warp; e < n; e += 2 * nw) {
      const int64_t on = btn ? btn[5 * (e / 2) + 1] : 0;
      nb_copy(Sn + on, S + bt[5 * e + 1], (int)bt[5 * e]);
    }
    __syncthreads();
    for (int k = 1 + 2 * warp; k < n; k += 2 * nw) {
      const int sk = (int)bt[5 * k];
      const int64_t o = bt[5 * k + 1];
      nb_copy(V + o, S + o, sk);
      nb_gemv_sub(mats + bt[5 * k + 3], sk, (int)bt[5 * (k - 1)], S + bt[5 * (k - 1) + 1], S + o);
      if (k + 1 < n) nb_gemv_sub(mats + bt[5 * k + 4], sk, (int)bt[5 * (k + 1)], S + bt[5 * (k + 1) + 1], S + o);
      nb_chol_solve(mats + bt[5 * k + 2], sk, S + o);
    }
    __syncthreads();
  }
  for (int64_t q = threadIdx.x; q < m; q += blockDim.x) U[aux[q]] += (T)sol[q];
  pdl_trigger();
}

// ---------------------------------------------------- small levels, fused
// A run of small levels in one thread block.  Per level the rhs F and the
// correction U of the rows E_l, and the row pointers of its smoothing and
// residual rows, live in shared memory; colour phases are separated by
// __syncthreads instead of kernel boundaries.  The steps are those of
// k_gs_aux / k_resid_aux / k_restrict_aux (down) and k_prolong_aux /
// k_addsaved_aux / k_gs_aux (up).
constexpr int SMALL_TPB = 1024;
constexpr int SMALL_B = 8;  // row entries loaded in one batch

template <class T>
constexpr size_t small_smem() {
  return 2 * SMALL_LMAX * sizeof(T) + 2 * (SMALL_LMAX + 1) * sizeof(int32_t);
}

// acc - sum_p val[p] * x[col[p]] over p0 <= p < p1, the first SMALL_B
// entries loaded together (ascending p, as a plain loop would add them)
template <class T, class V>
__device__ __forceinline__ T small_row(T acc, int p0, int p1, const V* __restrict__ val,
                                       const uint16_t* __restrict__ col, const T* x) {
  T v[SMALL_B];
  uint16_t c[SMALL_B];
#pragma unroll
  for (int q = 0; q < SMALL_B; ++q)
    if (p0 + q < p1) {
      v[q] = (T)val_of(val[p0 + q]);
      c[q] = col[p0 + q];
    }
#pragma unroll
  for (int q = 0; q < SMALL_B; ++q)
    if (p0 + q < p1) acc -= v[q] * x[c[q]];
  for (int p = p0 + SMALL_B; p < p1; ++p) acc -= (T)val_of(val[p]) * x[col[p]];
  return acc;
}

template <class T, class V>
__global__ void __launch_bounds__(SMALL_TPB, 1)
    k_small_down(const SmallDesc<T>* __restrict__ D, int nlev, T* F, int nu) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ul = reinterpret_cast<T*>(smraw);
  T* Fl = Ul + SMALL_LMAX;
  int32_t* Psm = reinterpret_cast<int32_t*>(Fl + SMALL_LMAX);
  int32_t* Prs = Psm + SMALL_LMAX + 1;
  if (nlev > 0) small_prefetch<T, V>(D, true);
  pdl_wait();
  for (int d = 0; d < nlev; ++d) {
    const SmallDesc<T>& L = D[d];
    const int mS = L.mS, mE = L.mE;
    if (d + 1 < nlev) small_prefetch<T, V>(D + d + 1, true);
    for (int k = threadIdx.x; k <= mE; k += blockDim.x) {
      if (k < mE) {
        const T f = F[L.gid[k]];
        Fl[k] = f;
        Ul[k] = 0;
        if (k < mS) L.fs[k] = f;
      }
      if (k <= mS) Psm[k] = L.sm_ptr[k];
      Prs[k] = L.rs_ptr[k];
    }
    __syncthreads();
    for (int sw = 0; sw < nu; ++sw)
      for (int c = 0; c < L.ncol; ++c) {
        for (int k = L.cs[c] + threadIdx.x; k < L.cs[c + 1]; k += blockDim.x) {
          const T acc = small_row(Fl[k], Psm[k], Psm[k + 1], sm_vals(L, (const V*)nullptr), L.sm_col, Ul);
          Ul[k] += acc * L.dinv[k];
        }
        __syncthreads();
      }
    for (int k = threadIdx.x; k < mE; k += blockDim.x) Fl[k] = small_row(Fl[k], Prs[k], Prs[k + 1], rs_vals(L, (const V*)nullptr), L.rs_col, Ul);
    __syncthreads();
    for (int t = threadIdx.x; t < L.npar; t += blockDim.x) {
      T acc = 0;
      for (int p = L.rp_ptr[t]; p < L.rp_ptr[t + 1]; ++p) acc += Fl[L.rp_child[p]];
      Fl[L.rp_id[t]] += (T)0.5 * acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < mE; k += blockDim.x) {
      F[L.gid[k]] = Fl[k];
      if (k < mS) L.us[k] = Ul[k];
    }
    __syncthreads();
  }
  pdl_trigger();
}

template <class T, class V>
__global__ void __launch_bounds__(SMALL_TPB, 1)
    k_small_up(const SmallDesc<T>* __restrict__ D, int nlev, T* U, int nu) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ul = reinterpret_cast<T*>(smraw);
  T* Fl = Ul + SMALL_LMAX;
  int32_t* Psm = reinterpret_cast<int32_t*>(Fl + SMALL_LMAX);
  if (nlev > 0) small_prefetch<T, V>(D + nlev - 1, false);
  pdl_wait();
  for (int d = nlev - 1; d >= 0; --d) {
    const SmallDesc<T>& L = D[d];
    const int mS = L.mS, mE = L.mE;
    if (d > 0) small_prefetch<T, V>(D + d - 1, false);
    for (int k = threadIdx.x; k < mE; k += blockDim.x) {
      Ul[k] = U[L.gid[k]];
      if (k < mS) Fl[k] = L.fs[k];
      if (k <= mS) Psm[k] = L.sm_ptr[k];
    }
    if (mS == mE && threadIdx.x == 0) Psm[mS] = L.sm_ptr[mS];
    __syncthreads();
    for (int t = threadIdx.x; t < L.nnew; t += blockDim.x) {
      const int32_t a = L.nn_p0[t], b = L.nn_p1[t];
      T v = 0;
      if (a >= 0) v += Ul[a];
      if (b >= 0) v += Ul[b];
      Ul[L.nn_id[t]] = (T)0.5 * v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < mS; k += blockDim.x) Ul[k] += L.us[k];
    __syncthreads();
    for (int sw = 0; sw < nu; ++sw)
      for (int c = L.ncol - 1; c >= 0; --c) {
        for (int k = L.cs[c] + threadIdx.x; k < L.cs[c + 1]; k += blockDim.x) {
          const T acc = small_row(Fl[k], Psm[k], Psm[k + 1], sm_vals(L, (const V*)nullptr), L.sm_col, Ul);
          Ul[k] += acc * L.dinv[k];
        }
        __syncthreads();
      }
    for (int k = threadIdx.x; k < mS; k += blockDim.x) U[L.gid[k]] = Ul[k];
    __syncthreads();
  }
  pdl_trigger();
}

// ------------------------------------------------------------------ PCG
__device__ __forceinline__ void set_cond(PcgScalars* sc, int cond, cudaGraphConditionalHandle hnd, int use_hnd) {
  sc->cond = cond;
  if (use_hnd) cudaGraphSetConditional(hnd, cond ? 1u : 0u);
}

// r = b - A x;  ||b||, ||r||; PCG scalars initialised
__global__ void k_pcg_init(int64_t n, SellView<double> A, const double* __restrict__ b, const double* __restrict__ x,
                           double* __restrict__ r, double* partial, unsigned int* ticket, PcgScalars* sc, double rtol,
                           int maxit, double* hist, cudaGraphConditionalHandle hnd, int use_hnd) {
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  Row<double> row;
  if (i0 < n) row_load(row, i0, A.off, A.col, A.val);
  pdl_wait();
  double v[2] = {0, 0};
  for (int64_t i = i0; i < n; i += st) {
    if (i != i0) row_load(row, i, A.off, A.col, A.val);
    double ri = b[i] - row_dot(row, A.col, A.val, x);
    r[i] = ri;
    v[0] += b[i] * b[i];
    v[1] += ri * ri;
  }
  if (grid_reduce<2>(v, partial, ticket) && threadIdx.x == 0) {
    sc->bnorm = sqrt(v[0]);
    sc->tol = rtol * sc->bnorm;
    sc->rr = v[1];
    sc->k = 0;
    sc->maxit = maxit;
    sc->status = 1;
    sc->rz = 0;
    sc->alpha = 0;
    sc->beta = 0;
    sc->timeout = 0;
    hist[0] = sqrt(v[1]);
    const bool conv = sqrt(v[1]) <= sc->tol;
    if (conv) sc->status = 0;
    set_cond(sc, (!conv && maxit > 0) ? 1 : 0, hnd, use_hnd);
  }
}

// <z, r>, <z, q_prev>  ->  beta (flexible: -alpha <z_{k+1}, q_k> / <z_k, r_k>), rz
template <class T>
__global__ void k_dots(int64_t n, const T* __restrict__ z, const double* __restrict__ r, const double* __restrict__ q,
                       double* partial, unsigned int* ticket, PcgScalars* sc) {
  pdl_wait();
  double v[2] = {0, 0};
#pragma unroll 4
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double zi = (double)z[i];
    v[0] += zi * r[i];
    v[1] += zi * q[i];
  }
  if (grid_reduce<2>(v, partial, ticket) && threadIdx.x == 0) {
    if (sc->k == 0) {
      sc->beta = 0;
    } else {
      sc->beta = -sc->alpha * v[1] / sc->rz;
    }
    sc->rz = v[0];
    if (!(v[0] > 0)) sc->status = ASMG_ERR_BREAKDOWN;
  }
}

// p = z + beta p
template <class T>
__global__ void k_pupd(int64_t n, const T* __restrict__ z, double* __restrict__ p, const PcgScalars* __restrict__ sc) {
  pdl_wait();
  const double beta = sc->beta;
#pragma unroll 4
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (double)z[i] + beta * p[i];
  pdl_trigger();
}

// q = A p, <p, q>  ->  alpha.  Each row's entries are loaded into registers
// at once (row_load), the thread's first row before the wait on the previous
// kernel (graded 2049^2: 3.1 -> 4.3 TB/s against a plain loop over the row).
__global__ void k_spmv_dot(int64_t n, SellView<double> A, const double* __restrict__ p, double* __restrict__ q,
                           double* partial, unsigned int* ticket, PcgScalars* sc) {
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  Row<double> row;
  if (i0 < n) row_load(row, i0, A.off, A.col, A.val);
  pdl_wait();
  double v[1] = {0};
  for (int64_t i = i0; i < n; i += st) {
    if (i != i0) row_load(row, i, A.off, A.col, A.val);
    const double qi = row_dot(row, A.col, A.val, p);
    q[i] = qi;
    v[0] += p[i] * qi;
  }
  if (grid_reduce<1>(v, partial, ticket) && threadIdx.x == 0) {
    sc->pq = v[0];
    if (!(v[0] > 0) || sc->status == ASMG_ERR_BREAKDOWN) {
      sc->status = ASMG_ERR_BREAKDOWN;
      sc->alpha = 0;
    } else {
      sc->alpha = sc->rz / v[0];
    }
  }
}

// x += alpha p, r -= alpha q, ||r||  ->  history, stopping test
__global__ void k_axpy_norm(int64_t n, const double* __restrict__ p, const double* __restrict__ q,
                            double* __restrict__ x, double* __restrict__ r, double* partial, unsigned int* ticket,
                            PcgScalars* sc, double* hist, cudaGraphConditionalHandle hnd, int use_hnd) {
  pdl_wait();
  const double a = sc->alpha;
  double v[1] = {0};
#pragma unroll 4
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    double ri = r[i] - a * q[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  if (grid_reduce<1>(v, partial, ticket) && threadIdx.x == 0) {
    if (sc->status == ASMG_ERR_BREAKDOWN) {
      set_cond(sc, 0, hnd, use_hnd);
      return;
    }
    if (sc->timeout) {
      sc->status = ASMG_ERR_TIMEOUT;
      set_cond(sc, 0, hnd, use_hnd);
      return;
    }
    sc->k += 1;
    sc->rr = v[0];
    const double nr = sqrt(v[0]);
    hist[sc->k] = nr;
    bool conv = nr <= sc->tol;
    if (conv) sc->status = 0;
    bool more = !conv && sc->k < sc->maxit && isfinite(nr);
    if (!isfinite(nr)) sc->status = ASMG_ERR_BREAKDOWN;
    set_cond(sc, more ? 1 : 0, hnd, use_hnd);
  }
}

// ASMG iteration: x += z
template <class T>
__global__ void k_xpz(int64_t n, const T* __restrict__ z, double* __restrict__ x) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)z[i];
  pdl_trigger();
}

// ASMG iteration: r = b - A x, ||r||  ->  history, stopping test
__global__ void k_iter_resid(int64_t n, SellView<double> A, const double* __restrict__ b, const double* __restrict__ x,
                             double* __restrict__ r, double* partial, unsigned int* ticket, PcgScalars* sc, double* hist,
                             cudaGraphConditionalHandle hnd, int use_hnd) {
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  Row<double> row;
  if (i0 < n) row_load(row, i0, A.off, A.col, A.val);
  pdl_wait();
  double v[1] = {0};
  for (int64_t i = i0; i < n; i += st) {
    if (i != i0) row_load(row, i, A.off, A.col, A.val);
    const double ri = b[i] - row_dot(row, A.col, A.val, x);
    r[i] = ri;
    v[0] += ri * ri;
  }
  if (grid_reduce<1>(v, partial, ticket) && threadIdx.x == 0) {
    if (sc->timeout) {
      sc->status = ASMG_ERR_TIMEOUT;
      set_cond(sc, 0, hnd, use_hnd);
      return;
    }
    sc->k += 1;
    sc->rr = v[0];
    const double nr = sqrt(v[0]);
    hist[sc->k] = nr;
    const bool conv = nr <= sc->tol;
    if (conv) sc->status = 0;
    if (!isfinite(nr)) sc->status = ASMG_ERR_BREAKDOWN;
    set_cond(sc, (!conv && sc->k < sc->maxit && isfinite(nr)) ? 1 : 0, hnd, use_hnd);
  }
}

__global__ void k_gather(int64_t n, const int32_t* __restrict__ vrow, const double* __restrict__ src,
                         double* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t v = vrow[i];
  dst[i] = v >= 0 ? src[v] : 0.0;
}

template <class S>
__global__ void k_scatter(int64_t nv, const int32_t* __restrict__ rowv, const S* __restrict__ src,
                          double* __restrict__ dst) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int32_t r = rowv[v];
  dst[v] = r >= 0 ? (double)src[r] : 0.0;
}

// --------------------------------------------------------- profiling
// With a profiler installed, every launch of the solve is bracketed by CUDA
// events on its stream and tagged with its kernel class and algorithmic bytes.
struct Profiler {
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> ev;
  struct Rec {
    int cls;
    int64_t bytes;
    int e0;
    int level;  // index into Prec::lev of an auxiliary-level launch (down: level, up: -2 - level), else -1
  };
  std::vector<Rec> recs;
  int mark() {
    cudaEvent_t e;
    ASMG_CUDA(cudaEventCreate(&e));
    ASMG_CUDA(cudaEventRecord(e, s));
    ev.push_back(e);
    return (int)ev.size() - 1;
  }
  ~Profiler() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};
thread_local Profiler* g_prof = nullptr;
thread_local int g_prof_level = -1;

#define LAUNCH(cls, bytes, ...)                                                  \
  do {                                                                          \
    int e0_ = g_prof ? g_prof->mark() : -1;                                     \
    __VA_ARGS__;                                                                \
    if (g_prof) {                                                               \
      g_prof->mark();                                                           \
      g_prof->recs.push_back(Profiler::Rec{(int)(cls), (int64_t)(bytes), e0_, g_prof_level}); \
    }                                                                           \
  } while (0)

// --------------------------------------------------------- enqueueing
template <class T>
SellView<T> fine_smoother(asmg_s& h);
template <>
SellView<double> fine_smoother<double>(asmg_s& h) { return view(h.A64); }
template <>
SellView<float> fine_smoother<float>(asmg_s& h) { return view(h.p32.Af); }
template <class T>
const T* fine_dinv(asmg_s& h);
template <>
const double* fine_dinv<double>(asmg_s& h) { return h.dinv64.p; }
template <>
const float* fine_dinv<float>(asmg_s& h) { return h.p32.dinv_f.p; }

template <class T>
Prec<T>& prec(asmg_s& h);
template <>
Prec<double>& prec<double>(asmg_s& h) { return h.p64; }
template <>
Prec<float>& prec<float>(asmg_s& h) { return h.p32; }

template <class T>
SlotPrec<T>& slotprec(Slot& S);
template <>
SlotPrec<double>& slotprec<double>(Slot& S) { return S.s64; }
template <>
SlotPrec<float>& slotprec<float>(Slot& S) { return S.s32; }

template <class T, class V>
int64_t small_bytes(const Prec<T>& P, int first, int count, int nu, bool down) {
  const int64_t sz = sizeof(T), sv = sizeof(V);
  int64_t by = 0;
  for (int k = 0; k < count; ++k) {
    const SmallLevelDev<T>& S = P.lev[first + k].small;
    by += nu * (S.nnz_sm * (2 + sv) + (int64_t)S.mS * (4 + sz));
    if (down)
      by += (int64_t)S.mE * (4 + 2 * sz) + (int64_t)S.mS * 2 * sz + S.nnz_rs * (2 + sv) + (int64_t)S.mE * 4 +
            (int64_t)S.npar * 10 + S.nchild * 2;
    else
      by += (int64_t)S.mE * (4 + sz) + (int64_t)S.mS * 3 * sz + (int64_t)S.nnew * 10;
  }
  return by;
}

// the slot's timeout flag (PcgScalars::timeout, device memory)
int* timeout_flag(Slot& S) {
  return reinterpret_cast<int*>(reinterpret_cast<char*>(S.scal.p) + offsetof(PcgScalars, timeout));
}

// V: how the auxiliary-level matrices are read (T, or bf16v with level_bf16)
template <class T, class V>
int enqueue_vcycle(asmg_s& h, Slot& S, cudaStream_t s) {
  Prec<T>& P = prec<T>(h);
  SlotPrec<T>& SP = slotprec<T>(S);
  int launches = 0;
  const int64_t sz = sizeof(T), sv = sizeof(V);
  const int npre = h.prm.nu_pre, npost = h.prm.nu_post;
  const int nlev = (int)P.lev.size();
  const int ndeep = P.n_deep, nbot = P.n_bottom;  // fused runs at the top and at the bottom
  const size_t smem = small_smem<T>();
  if (ndeep) {
    LAUNCH(ASMG_PROF_AUX_SMALL, (small_bytes<T, V>(P, nlev - ndeep, ndeep, npre, true)),
           launch_smem(h.prm.use_pdl, k_small_down<T, V>, 1, SMALL_TPB, smem, s, SP.deep_desc.p, ndeep, SP.F.p, npre));
    ++launches;
  }
  for (int li = nlev - 1 - ndeep; li >= nbot; --li) {
    AuxLevelDev<T>& L = P.lev[li];
    auto SMd = view(L.SMd);
    g_prof_level = li;
    if (L.tiled_down) {
      // all pre-sweeps of the level in one launch (compulsory bytes: the
      // tiles' blocks once, F gathered and saved, us written)
      const TileSweeps<T>& Tl = L.tdown;
      const int64_t by = Tl.nnz_real * (sv + 2) + (Tl.interior + Tl.halo) * (8 + 2 * sz) + Tl.interior * (4 + sz);
      LAUNCH(ASMG_PROF_AUX_GS, by,
             launch_smem(h.prm.use_pdl, k_tile_down<T, V>, Tl.ntiles, Tl.tpb, Tl.smem(), s, Tl.loc_off.p,
                         Tl.blob_off.p, (const unsigned char*)Tl.blob.p, Tl.phase.p, L.ncolours, Tl.maxblob,
                         Tl.maxloc, (const T*)SP.F.p, SP.fs[li].p, SP.us[li].p, npre, timeout_flag(S),
                         h.prm.inject_timeout));
      ++launches;
    }
    // pre-sweeps on us (SM order); the first also saves F on N~_l for the
    // post-sweeps (nu_pre >= 1)
    for (int sweep = 0; sweep < (L.tiled_down ? 0 : npre); ++sweep) {
      for (int c = 0; c < L.ncolours; ++c) {
        int64_t k0 = L.cstart[c], nk = L.cstart[c + 1] - L.cstart[c];
        if (!nk) continue;
        const int64_t by = L.cnnz_d[c] * (sv + 4) + L.crows[c] * (4 + (sweep == 0 ? 4 + 4 * sz : 4 * sz));
        LAUNCH(ASMG_PROF_AUX_GS, by,
               launch(h.prm.use_pdl, k_gs_aux_down<T, V>, nblk(nk, rows_tpb(nk)), rows_tpb(nk), s, k0, nk, SMd.off,
                      SMd.col, sell_vals(L.SMd, (const V*)nullptr), L.sm_dinv.p, L.sm_rows.p, (const T*)SP.F.p, sweep == 0 ? 1 : 0, SP.fs[li].p,
                      SP.us[li].p));
        ++launches;
      }
    }
    auto RS = view(L.RS);
    LAUNCH(ASMG_PROF_AUX_RESID, L.RS.nnz_real * (sv + 4) + L.nrs_real * (4 + 2 * sz) + L.nsm_real * sz,
           launch(h.prm.use_pdl, k_resid_aux<T, V>, nblk(L.nrs, rows_tpb(L.nrs)), rows_tpb(L.nrs), s, L.nrs, RS.off, RS.col, sell_vals(L.RS, (const V*)nullptr), L.rs_rows.p,
                  (const T*)SP.us[li].p, SP.F.p));
    LAUNCH(ASMG_PROF_AUX_TRANSFER, L.nchild * (4 + sz) + L.npar * (8 + 2 * sz),
           launch(h.prm.use_pdl, k_restrict_aux<T>, nblk(L.npar, rows_tpb(L.npar)), rows_tpb(L.npar), s, L.npar, L.rp_id.p,
                  L.rp_ptr.p, L.rp_child.p, SP.F.p));
    launches += 2;
  }
  g_prof_level = -1;
  if (nbot) {
    LAUNCH(ASMG_PROF_AUX_SMALL, (small_bytes<T, V>(P, 0, nbot, npre, true)),
           launch_smem(h.prm.use_pdl, k_small_down<T, V>, 1, SMALL_TPB, smem, s, SP.bot_desc.p, nbot, SP.F.p, npre));
    ++launches;
  }
  if (h.nc > 0) {
    LAUNCH(ASMG_PROF_COARSE, h.nc * h.nc * 8 + h.nc * (4 + 2 * sz),
           launch(h.prm.use_pdl, k_coarse<T>, nblk(h.nc * 32), TPB, s, h.nc, h.d_cid.p, h.d_cinv.p, SP.F.p, SP.U.p));
    ++launches;
  }
  if (nbot) {
    LAUNCH(ASMG_PROF_AUX_SMALL, (small_bytes<T, V>(P, 0, nbot, npost, false)),
           launch_smem(h.prm.use_pdl, k_small_up<T, V>, 1, SMALL_TPB, smem, s, SP.bot_desc.p, nbot, SP.U.p, npost));
    ++launches;
  }
  for (int li = nbot; li <= nlev - 1 - ndeep; ++li) {
    AuxLevelDev<T>& L = P.lev[li];
    auto SM = view(L.SM);
    g_prof_level = -2 - li;
    if (L.tiled_up) {
      const TileSweeps<T>& Tl = L.tup;
      LAUNCH(ASMG_PROF_AUX_TRANSFER,
             L.nsm_real * (28 + 3 * sz) + L.nnew * 2 * sz + (L.nsm_real - L.nnew) * sz +
                 (Tl.interior + Tl.halo) * (4 + 2 * sz),
             launch(h.prm.use_pdl, k_up_init<T>, nblk(L.nsm, rows_tpb(L.nsm)), rows_tpb(L.nsm), s, L.nsm, L.sm_rows.p,
                    L.sm_par0.p, L.sm_par1.p, Tl.pos_ptr.p, Tl.pos.p, (const T*)SP.U.p, (const T*)SP.us[li].p,
                    (const T*)SP.fs[li].p, SP.ust[li].p, SP.fsl[li].p));
      const int64_t by = Tl.nnz_real * (sv + 2) + (Tl.interior + Tl.halo) * (8 + 3 * sz) + Tl.interior * (4 + sz);
      LAUNCH(ASMG_PROF_AUX_GS, by,
             launch_smem(h.prm.use_pdl, k_tile_up<T, V>, Tl.ntiles, Tl.tpb, Tl.smem(), s, Tl.loc_off.p, Tl.blob_off.p,
                         (const unsigned char*)Tl.blob.p, Tl.ext_off.p, Tl.phase.p, L.ncolours, Tl.maxblob,
                         Tl.maxloc, Tl.maxext, (const T*)SP.ust[li].p, (const T*)SP.fsl[li].p, SP.U.p, npost,
                         timeout_flag(S), h.prm.inject_timeout));
      launches += 2;
      continue;
    }
    if (L.nnew) {
      LAUNCH(ASMG_PROF_AUX_TRANSFER, L.nnew * (12 + 3 * sz),
             launch(h.prm.use_pdl, k_prolong_aux<T>, nblk(L.nnew, rows_tpb(L.nnew)), rows_tpb(L.nnew), s, L.nnew, L.nn_id.p, L.nn_p0.p, L.nn_p1.p,
                    SP.U.p));
      ++launches;
    }
    LAUNCH(ASMG_PROF_AUX_TRANSFER, L.nsm_real * (4 + 3 * sz),
           launch(h.prm.use_pdl, k_addsaved_aux<T>, nblk(L.nsm, rows_tpb(L.nsm)), rows_tpb(L.nsm), s, L.nsm, L.sm_rows.p, SP.us[li].p, SP.U.p));
    ++launches;
    if (L.nb.m > 0) {
      // Algorithm 3: exact solve on the near-boundary set after the coarse correction
      const NbDev& N = L.nb;
      LAUNCH(ASMG_PROF_AUX_NB, L.NB.nnz_real * (sz + 4) + N.m * (16 + 2 * sz),
             launch(h.prm.use_pdl, k_nb_resid<T>, nblk(N.m), TPB, s, N.m, L.NB.off.p, L.NB.col.p, L.NB.val.p, N.sm.p,
                    (const T*)SP.fs[li].p, (const T*)SP.U.p, SP.nbr[li].p));
      LAUNCH(ASMG_PROF_AUX_NB, (int64_t)N.mats.n * 8 + N.m * (8 + 2 * sz),
             launch(h.prm.use_pdl, k_nb_solve<T>, 1, NB_TPB, s, N.R, N.nblk.p, N.boff.p, N.btab.p, N.voff.p,
                    (const double*)N.mats.p, N.last_size, N.last_off, N.m, N.aux.p, SP.nbr[li].p, SP.nbs[li].p,
                    SP.U.p));
      launches += 2;
    }
    for (int sweep = 0; sweep < npost; ++sweep)
      for (int c = L.ncolours - 1; c >= 0; --c) {
        int64_t k0 = L.cstart[c], nk = L.cstart[c + 1] - L.cstart[c];
        if (!nk) continue;
        LAUNCH(ASMG_PROF_AUX_GS, L.cnnz[c] * (sv + 4) + L.crows[c] * (4 + 5 * sz),
               launch(h.prm.use_pdl, k_gs_aux<T, V>, nblk(nk, rows_tpb(nk)), rows_tpb(nk), s, k0, nk, SM.off, SM.col, sell_vals(L.SM, (const V*)nullptr), L.sm_dinv.p,
                      L.sm_rows.p, (const T*)SP.fs[li].p, SP.U.p));
        ++launches;
      }
  }
  g_prof_level = -1;
  if (ndeep) {
    LAUNCH(ASMG_PROF_AUX_SMALL, (small_bytes<T, V>(P, nlev - ndeep, ndeep, npost, false)),
           launch_smem(h.prm.use_pdl, k_small_up<T, V>, 1, SMALL_TPB, smem, s, SP.deep_desc.p, ndeep, SP.U.p, npost));
    ++launches;
  }
  return launches;
}

// the V-cycle with the level matrices read in BF16 (mixed form with
// level_bf16) or in the arithmetic type
template <class T>
int enqueue_vcycle_vals(asmg_s& h, Slot& S, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value)
    if (h.prm.level_bf16) return enqueue_vcycle<float, bf16v>(h, S, s);
  return enqueue_vcycle<T, T>(h, S, s);
}

template <class T>
int enqueue_precond(asmg_s& h, Slot& S, const double* r, cudaStream_t s) {
  Prec<T>& P = prec<T>(h);
  SlotPrec<T>& SP = slotprec<T>(S);
  const SellView<T> A = fine_smoother<T>(h);
  const T* dinv = fine_dinv<T>(h);
  const int64_t sz = sizeof(T), n = h.n, nJ = h.nJ;
  const bool jacobi = h.prm.smoother == 1, additive = h.prm.additive == 1;
  int launches = 0;
  ASMG_CUDA(cudaMemsetAsync(SP.uf.p, 0, sizeof(T) * h.npad, s));
  const int ncol = (int)h.fine_cstart.size() - 1;
  bool zero = true;  // uf is still 0
  // u <- u + S (r - A u) (forward) or u + S^t (r - A u) (backward), fine_sweeps times
  auto smooth = [&](bool forward) {
    for (int m = 0; m < h.prm.fine_sweeps; ++m) {
      if (!jacobi) {
        for (int q = 0; q < ncol; ++q) {
          const int c = forward ? q : ncol - 1 - q;
          int64_t r0 = h.fine_cstart[c], nr = h.fine_cstart[c + 1] - r0;
          if (!nr) continue;
          LAUNCH(ASMG_PROF_FINE_GS, h.fine_cnnz[c] * (sz + 4) + h.fine_crows[c] * (8 + 4 * sz),
                 launch(h.prm.use_pdl, k_gs_fine<T, double>, nblk(nr, rows_tpb(nr)), rows_tpb(nr), s, r0, nr, A.off,
                        A.col, A.val, dinv, r, SP.uf.p));
          ++launches;
        }
      } else if (zero) {
        LAUNCH(ASMG_PROF_FINE_GS, n * (8 + 2 * sz),
               launch(h.prm.use_pdl, k_jac_first<T>, nblk(h.npad), TPB, s, h.npad, dinv, r, SP.uf.p));
        ++launches;
      } else {
        LAUNCH(ASMG_PROF_FINE_GS, h.A64.nnz_real * (sz + 4) + n * (8 + 2 * sz),
               launch(h.prm.use_pdl, k_resid_fine<T>, nblk(h.npad), TPB, s, h.npad, A.off, A.col, A.val, r, SP.uf.p,
                      SP.rho.p));
        LAUNCH(ASMG_PROF_FINE_GS, n * 4 * sz,
               launch(h.prm.use_pdl, k_jac_add<T>, nblk(h.npad), TPB, s, h.npad, dinv, SP.rho.p, SP.uf.p));
        launches += 2;
      }
      zero = false;
    }
  };
  // (1) u1 = S r
  smooth(true);
  // (2) multiplicative: u2 = u1 + P Btilde P^T (r - A u1);  additive: u1 + P Btilde P^T r
  if (h.nJ > 0) {
    if (additive) {
      LAUNCH(ASMG_PROF_FINE_RESID, n * (8 + sz),
             launch(h.prm.use_pdl, k_cast_fine<T>, nblk(h.npad), TPB, s, h.npad, r, SP.rho.p));
    } else {
      LAUNCH(ASMG_PROF_FINE_RESID, h.A64.nnz_real * (sz + 4) + n * (8 + 2 * sz),
             launch(h.prm.use_pdl, k_resid_fine<T>, nblk(h.npad), TPB, s, h.npad, A.off, A.col, A.val, r, SP.uf.p,
                    SP.rho.p));
    }
    auto PT = view(P.PT);
    LAUNCH(ASMG_PROF_RESTRICT, P.PT.nnz_real * (sz + 4) + n * sz + 2 * nJ * sz,
           launch(h.prm.use_pdl, k_restrict_fine<T>, nblk(h.nJpad), TPB, s, h.nJpad, PT.off, PT.col, PT.val, SP.rho.p, SP.F.p, SP.U.p));
    launches += 2;
    launches += enqueue_vcycle_vals<T>(h, S, s);
    auto PP = view(P.P);
    LAUNCH(ASMG_PROF_PROLONG, P.P.nnz_real * (sz + 4) + nJ * sz + 2 * n * sz,
           launch(h.prm.use_pdl, k_prolong_fine<T>, nblk(h.npad), TPB, s, h.npad, PP.off, PP.col, PP.val, SP.U.p, SP.uf.p));
    ++launches;
  }
  // (3) multiplicative only: u3 = u2 + S^T (r - A u2)
  if (!additive) smooth(false);
  ASMG_CUDA(cudaGetLastError());
  return launches;
}

template <class T>
int enqueue_body(asmg_s& h, Slot& S, cudaStream_t s, cudaGraphConditionalHandle hnd, int use_hnd) {
  int launches = enqueue_precond<T>(h, S, S.r.p, s);
  const T* z = slotprec<T>(S).uf.p;
  const int G = RED_BLOCKS, GV = VEC_BLOCKS;
  const int64_t n = h.n, sz = sizeof(T);
  LAUNCH(ASMG_PROF_CG_VECTOR, n * (sz + 16),
         launch(h.prm.use_pdl, k_dots<T>, GV, TPB, s, h.npad, z, S.r.p, S.q.p, S.partial.p, S.ticket.p, S.scal.p));
  LAUNCH(ASMG_PROF_CG_VECTOR, n * (sz + 16), launch(h.prm.use_pdl, k_pupd<T>, GV, TPB, s, h.npad, z, S.p.p, S.scal.p));
  LAUNCH(ASMG_PROF_CG_SPMV, h.A64.nnz_real * 12 + n * 16,
         launch(h.prm.use_pdl, k_spmv_dot, G, TPB, s, h.npad, view(h.A64), S.p.p, S.q.p, S.partial.p, S.ticket.p, S.scal.p));
  LAUNCH(ASMG_PROF_CG_VECTOR, n * 48,
         launch(h.prm.use_pdl, k_axpy_norm, GV, TPB, s, h.npad, S.p.p, S.q.p, S.x.p, S.r.p, S.partial.p, S.ticket.p, S.scal.p,
                                       S.hist.p, hnd, use_hnd));
  ASMG_CUDA(cudaGetLastError());
  return launches + 4;
}

// the ASMG iteration: z = B r, x += z, r = b - A x, stopping test
template <class T>
int enqueue_iteration(asmg_s& h, Slot& S, cudaStream_t s, cudaGraphConditionalHandle hnd, int use_hnd) {
  int launches = enqueue_precond<T>(h, S, S.r.p, s);
  const T* z = slotprec<T>(S).uf.p;
  const int G = RED_BLOCKS;
  const int64_t n = h.n, sz = sizeof(T);
  LAUNCH(ASMG_PROF_CG_VECTOR, n * (sz + 16), launch(h.prm.use_pdl, k_xpz<T>, G, TPB, s, h.npad, z, S.x.p));
  LAUNCH(ASMG_PROF_CG_SPMV, h.A64.nnz_real * 12 + n * 24,
         launch(h.prm.use_pdl, k_iter_resid, G, TPB, s, h.npad, view(h.A64), S.b.p, S.x.p, S.r.p, S.partial.p,
                S.ticket.p, S.scal.p, S.hist.p, hnd, use_hnd));
  ASMG_CUDA(cudaGetLastError());
  return launches + 2;
}

int enqueue_body_any(asmg_s& h, Slot& S, cudaStream_t s, cudaGraphConditionalHandle hnd, int use_hnd) {
  if (h.prm.iteration == 1)
    return h.prm.precision == ASMG_MIXED ? enqueue_iteration<float>(h, S, s, hnd, use_hnd)
                                         : enqueue_iteration<double>(h, S, s, hnd, use_hnd);
  return h.prm.precision == ASMG_MIXED ? enqueue_body<float>(h, S, s, hnd, use_hnd)
                                       : enqueue_body<double>(h, S, s, hnd, use_hnd);
}

void enqueue_init(asmg_s& h, Slot& S, double rtol, cudaStream_t s, cudaGraphConditionalHandle hnd, int use_hnd) {
  LAUNCH(ASMG_PROF_CG_VECTOR, h.A64.nnz_real * 12 + h.n * 32,
         launch(h.prm.use_pdl, k_pcg_init, RED_BLOCKS, TPB, s, h.npad, view(h.A64), S.b.p, S.x.p, S.r.p, S.partial.p, S.ticket.p,
                                               S.scal.p, rtol, h.prm.max_iter, S.hist.p, hnd, use_hnd));
  ASMG_CUDA(cudaGetLastError());
}

}  // namespace

void gather_rows(asmg_s& h, const double* vsrc, double* dst, cudaStream_t s) {
  launch(false, k_gather, nblk(h.npad), TPB, s, h.npad, h.d_vertex_of_row.p, vsrc, dst);
  ASMG_CUDA(cudaGetLastError());
}

void scatter_rows(asmg_s& h, const void* src, bool src_float, double* vdst, cudaStream_t s) {
  if (src_float)
    launch(false, k_scatter<float>, nblk(h.mesh.nv), TPB, s, h.mesh.nv, h.d_row_of_vertex.p, (const float*)src, vdst);
  else
    launch(false, k_scatter<double>, nblk(h.mesh.nv), TPB, s, h.mesh.nv, h.d_row_of_vertex.p, (const double*)src, vdst);
  ASMG_CUDA(cudaGetLastError());
}

void precond_apply(asmg_s& h, const double* r_perm, cudaStream_t s) {
  Slot& S = *h.slots[0];
  if (h.prm.precision == ASMG_MIXED)
    enqueue_precond<float>(h, S, r_perm, s);
  else
    enqueue_precond<double>(h, S, r_perm, s);
}

__global__ void k_spmv64(int64_t n, SellView<double> A, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = sell_dot<double, double>(i, A.off, A.col, A.val, x);
}

void spmv64(asmg_s& h, const double* x, double* y, cudaStream_t s) {
  launch(false, k_spmv64, nblk(h.npad), TPB, s, h.npad, view(h.A64), x, y);
  ASMG_CUDA(cudaGetLastError());
}

// Capture the graph of one solve into `g` (independent of other nodes):
//   init (r = b - A x, norms, condition) -> WHILE(cond) { body }.
// Returns the WHILE node.
cudaGraphNode_t capture_solve(asmg_s& h, Slot& S, double rtol, cudaGraph_t g, const cudaGraphNode_t* deps,
                              size_t ndeps) {
  cudaGraphConditionalHandle hnd;
  ASMG_CUDA(cudaGraphConditionalHandleCreate(&hnd, g, 0, 0));
  cudaStream_t cs;
  ASMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  ASMG_CUDA(cudaStreamBeginCaptureToGraph(cs, g, deps, nullptr, ndeps, cudaStreamCaptureModeThreadLocal));
  enqueue_init(h, S, rtol, cs, hnd, 1);
  // the WHILE node depends on the captured init kernel (the leaf of this capture)
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* leaf = nullptr;
  size_t nleaf = 0;
  ASMG_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &leaf, nullptr, &nleaf));
  std::vector<cudaGraphNode_t> leaves(leaf, leaf + nleaf);
  cudaGraph_t gg;
  ASMG_CUDA(cudaStreamEndCapture(cs, &gg));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  ASMG_CUDA(cudaGraphAddNode(&cnode, g, leaves.data(), nullptr, leaves.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  ASMG_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  h.gpu_launches_per_iter = enqueue_body_any(h, S, cs, hnd, 1);
  cudaGraph_t bb;
  ASMG_CUDA(cudaStreamEndCapture(cs, &bb));
  ASMG_CUDA(cudaStreamDestroy(cs));
  return cnode;
}

static void build_graph(asmg_s& h, Slot& S, double rtol) {
  if (S.gexec) {
    cudaGraphExecDestroy(S.gexec);
    S.gexec = nullptr;
  }
  if (S.graph) {
    cudaGraphDestroy(S.graph);
    S.graph = nullptr;
  }
  cudaGraph_t g;
  ASMG_CUDA(cudaGraphCreate(&g, 0));
  capture_solve(h, S, rtol, g, nullptr, 0);
  ASMG_CUDA(cudaGraphInstantiate(&S.gexec, g, 0));
  S.graph = g;
}

int run_solve(asmg_s& h, Slot& S, double rtol, cudaStream_t s) {
  if (h.prm.use_graph) {
    // the graph bakes rtol into the init kernel's arguments: rebuild when it changes
    if (!S.gexec || S.graph_rtol != rtol) {
      build_graph(h, S, rtol);
      S.graph_rtol = rtol;
    }
    ASMG_CUDA(cudaGraphLaunch(S.gexec, s));
  } else {
    enqueue_init(h, S, rtol, s, 0, 0);
    for (int it = 0; it < h.prm.max_iter; ++it) {
      PcgScalars sc;
      ASMG_CUDA(cudaMemcpyAsync(&sc, S.scal.p, sizeof sc, cudaMemcpyDeviceToHost, s));
      ASMG_CUDA(cudaStreamSynchronize(s));
      if (!sc.cond) break;
      h.gpu_launches_per_iter = enqueue_body_any(h, S, s, 0, 0);
    }
  }
  return 0;
}

// One solve without the graph, every launch timed: per class launches,
// milliseconds and algorithmic bytes; returns the iteration count.
int profile_solve(asmg_s& h, double rtol, cudaStream_t s, double* out, double* out_levels, int nlev_out) {
  Slot& S = *h.slots[0];
  Profiler prof;
  prof.s = s;
  g_prof = &prof;
  int its = 0;
  try {
    enqueue_init(h, S, rtol, s, 0, 0);
    for (int it = 0; it < h.prm.max_iter; ++it) {
      PcgScalars sc;
      ASMG_CUDA(cudaMemcpyAsync(&sc, S.scal.p, sizeof sc, cudaMemcpyDeviceToHost, s));
      ASMG_CUDA(cudaStreamSynchronize(s));
      if (!sc.cond) break;
      enqueue_body_any(h, S, s, 0, 0);
      ++its;
    }
    ASMG_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    g_prof = nullptr;
    throw;
  }
  g_prof = nullptr;
  for (int k = 0; k < 3 * ASMG_PROF_NCLASS; ++k) out[k] = 0;
  if (out_levels)
    for (int k = 0; k < nlev_out * 2 * 3 * 3; ++k) out_levels[k] = 0;
  for (auto& r : prof.recs) {
    float ms = 0;
    ASMG_CUDA(cudaEventElapsedTime(&ms, prof.ev[r.e0], prof.ev[r.e0 + 1]));
    out[3 * r.cls] += 1;
    out[3 * r.cls + 1] += ms;
    out[3 * r.cls + 2] += (double)r.bytes;
    if (out_levels && r.level != -1) {
      // [level][down, up][sweeps, residual, transfer][launches, ms, bytes]
      const int li = r.level >= 0 ? r.level : -2 - r.level, dir = r.level >= 0 ? 0 : 1;
      const int kind = r.cls == ASMG_PROF_AUX_GS ? 0 : r.cls == ASMG_PROF_AUX_RESID ? 1 : 2;
      if (li < nlev_out) {
        double* o = out_levels + ((li * 2 + dir) * 3 + kind) * 3;
        o[0] += 1;
        o[1] += ms;
        o[2] += (double)r.bytes;
      }
    }
  }
  return its;
}

// The fused runs: the longest run of small levels from the finest level down
// and from the coarsest V-cycle level up (a level is small when its rows E_l
// fit SMALL_LMAX); their descriptors live in device memory.
template <class T>
void setup_small(Prec<T>& P) {
  const int nlev = (int)P.lev.size();
  int nd = 0;
  while (nd < nlev && P.lev[nlev - 1 - nd].small.ok) ++nd;
  int nb = 0;
  if (nd < nlev)
    while (nb < nlev - nd && P.lev[nb].small.ok) ++nb;
  P.n_deep = nd;
  P.n_bottom = nb;
  const int smem = (int)small_smem<T>();
  // the attribute belongs to the kernel, not to this handle: every handle sets
  // the same bound, for tiles the largest a tile may use
  auto attrs = [&](auto vtag) {
    using V = decltype(vtag);
    ASMG_CUDA(cudaFuncSetAttribute(k_small_down<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ASMG_CUDA(cudaFuncSetAttribute(k_small_up<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ASMG_CUDA(
        cudaFuncSetAttribute(k_tile_down<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM_LIMIT));
    ASMG_CUDA(
        cudaFuncSetAttribute(k_tile_up<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM_LIMIT));
  };
  attrs(T{});
  if constexpr (std::is_same<T, float>::value) attrs(bf16v{});
}

// Work state of one solve in precision T: vectors, per-level saved values,
// descriptors of the fused small-level runs (they point at this slot's
// saved values).
template <class T>
void alloc_slot_prec(asmg_s& h, Prec<T>& P, SlotPrec<T>& SP, cudaStream_t s) {
  SP.uf.alloc(h.npad);
  SP.rho.alloc(h.npad);
  SP.F.alloc(std::max<int64_t>(h.nJpad, 1));
  SP.U.alloc(std::max<int64_t>(h.nJpad, 1));
  SP.uf.zero(s);
  SP.rho.zero(s);
  SP.F.zero(s);
  SP.U.zero(s);
  const int nlev = (int)P.lev.size();
  SP.fs.clear();
  SP.us.clear();
  SP.fs.resize(nlev);
  SP.us.resize(nlev);
  SP.nbr.clear();
  SP.nbs.clear();
  SP.nbr.resize(nlev);
  SP.nbs.resize(nlev);
  SP.ust.clear();
  SP.fsl.clear();
  SP.ust.resize(nlev);
  SP.fsl.resize(nlev);
  for (int li = 0; li < nlev; ++li) {
    SP.fs[li].alloc(std::max<int64_t>(P.lev[li].nsm, 1));
    SP.us[li].alloc(std::max<int64_t>(P.lev[li].nsm, 1));
    SP.fs[li].zero(s);
    SP.us[li].zero(s);
    if (P.lev[li].tiled_up) {
      // post-sweep start values and saved rhs in tile order (padding rows stay 0)
      SP.ust[li].alloc(std::max<int64_t>(P.lev[li].tup.nloc, 1));
      SP.fsl[li].alloc(std::max<int64_t>(P.lev[li].tup.nloc, 1));
      SP.ust[li].zero(s);
      SP.fsl[li].zero(s);
    }
    const NbDev& N = P.lev[li].nb;
    if (N.m > 0) {
      // the pools: every round's vector and the last block's (voff[R + 1] doubles)
      int64_t pool = 0;
      {
        std::vector<int64_t> vo = N.voff.download(s);
        pool = vo.back();
      }
      SP.nbr[li].alloc(pool);
      SP.nbs[li].alloc(pool);
      SP.nbr[li].zero(s);
      SP.nbs[li].zero(s);
    }
  }
  auto desc = [&](int li) {
    AuxLevelDev<T>& L = P.lev[li];
    SmallDesc<T> d;
    SmallLevelDev<T>& M = L.small;
    d.mS = M.mS;
    d.mE = M.mE;
    d.ncol = M.ncol;
    d.nnew = M.nnew;
    d.npar = M.npar;
    d.nnz_sm = (int)M.nnz_sm;
    d.nnz_rs = (int)M.nnz_rs;
    d.nchild = (int)M.nchild;
    for (int c = 0; c <= SMALL_MAXC; ++c) d.cs[c] = c <= M.ncol ? M.cs[c] : M.mS;
    d.gid = M.gid.p;
    d.sm_ptr = M.sm_ptr.p;
    d.sm_col = M.sm_col.p;
    d.sm_val = M.sm_val.p;
    d.sm_v16 = M.sm_v16.p;
    d.dinv = M.dinv.p;
    d.rs_ptr = M.rs_ptr.p;
    d.rs_col = M.rs_col.p;
    d.rs_val = M.rs_val.p;
    d.rs_v16 = M.rs_v16.p;
    d.nn_id = M.nn_id.p;
    d.nn_p0 = M.nn_p0.p;
    d.nn_p1 = M.nn_p1.p;
    d.rp_id = M.rp_id.p;
    d.rp_ptr = M.rp_ptr.p;
    d.rp_child = M.rp_child.p;
    d.fs = SP.fs[li].p;
    d.us = SP.us[li].p;
    return d;
  };
  std::vector<SmallDesc<T>> deep, bot;
  for (int k = 0; k < P.n_deep; ++k) deep.push_back(desc(nlev - 1 - k));  // finest first (down order)
  for (int k = P.n_bottom - 1; k >= 0; --k) bot.push_back(desc(k));
  SP.deep_desc.upload(deep, s);
  SP.bot_desc.upload(bot, s);
}

// Schedule of the auxiliary levels (the autotuner, tile_rows = 0): each
// direction of a level that has tiles runs either its temporally blocked
// sweeps or its launches per colour class and sweep, with the same results.
// The choice is made on the device: one preconditioner application is
// captured as a CUDA graph and timed (median of 3 runs of 5 launches) with
// every level tiled both ways, then for each level in turn the post-sweeps
// and then the pre-sweeps are switched to class launches, each switch kept
// when it is faster by more than 0.5% (and 2 us).  Tiles of a direction left
// untiled are freed.
template <class T>
void autotune_levels(asmg_s& h, cudaStream_t s) {
  Prec<T>& P = prec<T>(h);
  Slot& S = *h.slots[0];
  const int nlev = (int)P.lev.size();
  std::vector<int> cand;
  for (int li = P.n_bottom; li <= nlev - 1 - P.n_deep; ++li)
    if (P.lev[li].tiled) cand.push_back(li);
  if (cand.empty()) return;
  cudaStream_t cs;
  ASMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  ASMG_CUDA(cudaEventCreate(&e0));
  ASMG_CUDA(cudaEventCreate(&e1));
  auto time_once = [&]() -> float {
    cudaGraph_t g;
    cudaGraphExec_t ge;
    ASMG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    enqueue_precond<T>(h, S, S.r.p, cs);
    ASMG_CUDA(cudaStreamEndCapture(cs, &g));
    ASMG_CUDA(cudaGraphInstantiate(&ge, g, 0));
    float best[3];
    for (int rep = 0; rep < 3; ++rep) {
      ASMG_CUDA(cudaGraphLaunch(ge, cs));
      ASMG_CUDA(cudaEventRecord(e0, cs));
      for (int k = 0; k < 5; ++k) ASMG_CUDA(cudaGraphLaunch(ge, cs));
      ASMG_CUDA(cudaEventRecord(e1, cs));
      ASMG_CUDA(cudaEventSynchronize(e1));
      ASMG_CUDA(cudaEventElapsedTime(&best[rep], e0, e1));
    }
    ASMG_CUDA(cudaGraphExecDestroy(ge));
    ASMG_CUDA(cudaGraphDestroy(g));
    std::sort(best, best + 3);
    return best[1] / 5;
  };
  try {
    float cur = time_once();
    for (int li : cand)
      for (bool* flag : {&P.lev[li].tiled_up, &P.lev[li].tiled_down}) {
        *flag = false;
        const float t = time_once();
        if (t < cur * 0.995f && cur - t > 0.002f) {
          cur = t;
        } else {
          *flag = true;
        }
      }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(cs);
    throw;
  }
  ASMG_CUDA(cudaEventDestroy(e0));
  ASMG_CUDA(cudaEventDestroy(e1));
  ASMG_CUDA(cudaStreamDestroy(cs));
  for (int li : cand) {
    AuxLevelDev<T>& L = P.lev[li];
    if (!L.tiled_down) L.tdown = TileSweeps<T>();
    if (!L.tiled_up) {
      L.tup = TileSweeps<T>();
      slotprec<T>(S).ust[li] = DBuf<T>();
      slotprec<T>(S).fsl[li] = DBuf<T>();
    }
    L.tiled = L.tiled_down || L.tiled_up;
  }
}

Slot& add_slot(asmg_s& h, cudaStream_t s) {
  h.slots.emplace_back(new Slot());
  Slot& S = *h.slots.back();
  S.b.alloc(h.npad);
  S.x.alloc(h.npad);
  S.r.alloc(h.npad);
  S.p.alloc(h.npad);
  S.q.alloc(h.npad);
  S.b.zero(s);
  S.x.zero(s);
  S.r.zero(s);
  S.p.zero(s);
  S.q.zero(s);
  S.vb.alloc(h.mesh.nv);
  S.vu.alloc(h.mesh.nv);
  S.partial.alloc(std::max(4 * RED_BLOCKS, 2 * VEC_BLOCKS));
  S.ticket.alloc(1);
  S.ticket.zero(s);
  S.scal.alloc(1);
  S.scal.zero(s);
  S.hist.alloc(h.prm.max_iter + 1);
  if (h.prm.precision == ASMG_MIXED)
    alloc_slot_prec(h, h.p32, S.s32, s);
  else
    alloc_slot_prec(h, h.p64, S.s64, s);
  ASMG_CUDA(cudaStreamSynchronize(s));
  return S;
}

// Levels inside the fused small-level runs never use their tiles: drop them.
template <class T>
void drop_unused_tiles(Prec<T>& P) {
  const int nlev = (int)P.lev.size();
  for (int li = 0; li < nlev; ++li)
    if (li < P.n_bottom || li > nlev - 1 - P.n_deep) {
      P.lev[li].tiled = P.lev[li].tiled_down = P.lev[li].tiled_up = false;
      P.lev[li].tdown = TileSweeps<T>();
      P.lev[li].tup = TileSweeps<T>();
    }
}

void setup_solve(asmg_s& h, cudaStream_t s) {
  if (h.prm.precision == ASMG_MIXED) {
    setup_small(h.p32);
    drop_unused_tiles(h.p32);
  } else {
    setup_small(h.p64);
    drop_unused_tiles(h.p64);
  }
  h.slots.clear();
  add_slot(h, s);
  if (h.prm.tile_rows == 0 && !h.prm.inject_timeout) {
    if (h.prm.precision == ASMG_MIXED)
      autotune_levels<float>(h, s);
    else
      autotune_levels<double>(h, s);
  }
}

}  // namespace asmg
