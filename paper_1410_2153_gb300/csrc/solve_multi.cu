// Several right-hand sides of one handle in one solve: the PCG of Sec. 5.2
// with the preconditioner of Algorithm 1 and the V-cycle of Algorithm 2, run
// on KRHS columns at once (the SpMM form).  Every vector is stored with its
// columns interleaved (element (i, j) at i * KRHS + j), so each matrix entry
// loaded by a kernel -- fine operator, transfer P and P^T, level operators --
// is used for all columns, and each gathered vector element is one 16-byte
// (FP32) or 32-byte (FP64) load.
//
// Per column the arithmetic is that of the single-column kernels of
// solve.cu, in the same order (the same row sums, the same reduction grid),
// and the scalars of the recurrences are kept per column.  A column stops on
// its own test (converged, iteration cap, breakdown): it then keeps alpha = 0,
// so its x and r no longer change, and the loop runs while any column is
// active.  The fused small-level kernels hold KRHS columns in shared memory,
// so a run of small levels is shorter here (SMALL_LMAX / KRHS rows per level
// in FP32); such a level's arithmetic then follows the per-level kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <type_traits>
#include <vector>

#include "handle.h"
#include "kernels.h"

namespace asmg {

namespace {

using namespace kern;
constexpr int K = KRHS;

// KRHS consecutive values (one row of an interleaved vector); 16-byte aligned
template <class T>
struct VK {
  T v[K];
};

template <class T>
__device__ __forceinline__ VK<T> ldk(const T* p) {
  VK<T> r;
  if constexpr (K == 4 && sizeof(T) == 4) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    r.v[0] = f.x;
    r.v[1] = f.y;
    r.v[2] = f.z;
    r.v[3] = f.w;
  } else if constexpr (K == 4 && sizeof(T) == 8) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    r.v[0] = a.x;
    r.v[1] = a.y;
    r.v[2] = b.x;
    r.v[3] = b.y;
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) r.v[j] = p[j];
  }
  return r;
}

template <class T>
__device__ __forceinline__ void stk(T* p, const VK<T>& r) {
  if constexpr (K == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else if constexpr (K == 4 && sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(r.v[2], r.v[3]);
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) p[j] = r.v[j];
  }
}

// acc[j] += sum_e a_e x[c_e][j] over a SELL row held in registers (the order of row_dot)
template <class T, class X, class V>
__device__ __forceinline__ void row_dot_k(const Row<T>& R, const int32_t* __restrict__ col, const V* __restrict__ val,
                                          const X* x, T (&acc)[K]) {
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = 0;
#pragma unroll
  for (int q = 0; q < MAXW; ++q)
    if (q < R.w) {
      const VK<X> xv = ldk<X>(x + (int64_t)R.c[q] * K);
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] += R.v[q] * (T)xv.v[j];
    }
  for (int q = MAXW; q < R.w; ++q) {
    const int64_t e = R.b + ((int64_t)q << 5) + R.lane;
    const T a = (T)ldg_val(val + e);
    const VK<X> xv = ldk<X>(x + (int64_t)__ldg(col + e) * K);
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] += a * (T)xv.v[j];
  }
}

// ------------------------------------------------------------- fine grid
template <class T>
__global__ void k_gs_fine_k(int64_t r0, int64_t nrows, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                            const T* __restrict__ val, const T* __restrict__ dinv, const double* __restrict__ rhs,
                            T* u) {
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
    T acc[K];
    row_dot_k<T, T>(row, col, val, u, acc);
    const VK<double> r = ldk<double>(rhs + i * K);
    VK<T> ui = ldk<T>(u + i * K);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const T s = (T)r.v[j] - acc[j];
      ui.v[j] += s * di;
    }
    stk<T>(u + i * K, ui);
  }
  pdl_trigger();
}

template <class T>
__global__ void k_resid_fine_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                               const T* __restrict__ val, const double* __restrict__ r, const T* __restrict__ u,
                               T* __restrict__ rho) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = i < n;
  Row<T> row;
  if (act) row_load(row, i, off, col, val);
  pdl_wait();
  if (act) {
    T acc[K];
    row_dot_k<T, T>(row, col, val, u, acc);
    const VK<double> rv = ldk<double>(r + i * K);
    VK<T> o;
#pragma unroll
    for (int j = 0; j < K; ++j) o.v[j] = (T)rv.v[j] - acc[j];
    stk<T>(rho + i * K, o);
  }
  pdl_trigger();
}

template <class T>
__global__ void k_restrict_fine_k(int64_t nJ, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                  const T* __restrict__ val, const T* __restrict__ rho, T* __restrict__ F,
                                  T* __restrict__ U) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = k < nJ;
  Row<T> row;
  if (act) row_load(row, k, off, col, val);
  pdl_wait();
  if (act) {
    T acc[K];
    row_dot_k<T, T>(row, col, val, rho, acc);
    VK<T> o, z;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      o.v[j] = acc[j];
      z.v[j] = 0;
    }
    stk<T>(F + k * K, o);
    stk<T>(U + k * K, z);
  }
  pdl_trigger();
}

template <class T>
__global__ void k_prolong_fine_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                 const T* __restrict__ val, const T* __restrict__ U, T* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = i < n;
  Row<T> row;
  if (act) row_load(row, i, off, col, val);
  pdl_wait();
  if (act) {
    T acc[K];
    row_dot_k<T, T>(row, col, val, U, acc);
    VK<T> ui = ldk<T>(u + i * K);
#pragma unroll
    for (int j = 0; j < K; ++j) ui.v[j] += acc[j];
    stk<T>(u + i * K, ui);
  }
  pdl_trigger();
}

// ------------------------------------------------------ auxiliary levels
template <class T, class V>
__global__ void k_gs_aux_k(int64_t k0, int64_t nk, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
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
    T acc[K];
    row_dot_k<T, T>(row, col, val, U, acc);
    const VK<T> f = ldk<T>(fs + k * K);
    VK<T> ui = ldk<T>(U + (int64_t)i * K);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const T s = f.v[j] - acc[j];
      ui.v[j] += s * di;
    }
    stk<T>(U + (int64_t)i * K, ui);
  }
  pdl_trigger();
}

template <class T, class V>
__global__ void k_gs_aux_down_k(int64_t k0, int64_t nk, const int64_t* __restrict__ off,
                                const int32_t* __restrict__ col, const V* __restrict__ val,
                                const T* __restrict__ dinv, const int32_t* __restrict__ rows, const T* __restrict__ F,
                                int first, T* __restrict__ fs, T* us) {
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
    T acc[K];
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = 0;
    if (first) {
      const VK<T> f = ldk<T>(F + (int64_t)i * K);
      stk<T>(fs + k * K, f);
#pragma unroll
      for (int q = 0; q < MAXW; ++q)
        if (q < row.w && row.c[q] < k0) {
          const VK<T> xv = ldk<T>(us + (int64_t)row.c[q] * K);
#pragma unroll
          for (int j = 0; j < K; ++j) acc[j] += row.v[q] * xv.v[j];
        }
      for (int q = MAXW; q < row.w; ++q) {
        const int64_t e = row.b + ((int64_t)q << 5) + row.lane;
        const int32_t c = __ldg(col + e);
        if (c < k0) {
          const T a = (T)ldg_val(val + e);
          const VK<T> xv = ldk<T>(us + (int64_t)c * K);
#pragma unroll
          for (int j = 0; j < K; ++j) acc[j] += a * xv.v[j];
        }
      }
      VK<T> o;
#pragma unroll
      for (int j = 0; j < K; ++j) o.v[j] = (f.v[j] - acc[j]) * di;
      stk<T>(us + k * K, o);
    } else {
      const VK<T> f = ldk<T>(fs + k * K);
      row_dot_k<T, T>(row, col, val, us, acc);
      VK<T> o = ldk<T>(us + k * K);
#pragma unroll
      for (int j = 0; j < K; ++j) o.v[j] += (f.v[j] - acc[j]) * di;
      stk<T>(us + k * K, o);
    }
  }
  pdl_trigger();
}

template <class T, class V>
__global__ void k_resid_aux_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
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
  if (i >= 0) {
    T acc[K];
    row_dot_k<T, T>(row, col, val, U, acc);
    VK<T> f = ldk<T>(F + (int64_t)i * K);
#pragma unroll
    for (int j = 0; j < K; ++j) f.v[j] -= acc[j];
    stk<T>(F + (int64_t)i * K, f);
  }
  pdl_trigger();
}

template <class T>
__global__ void k_restrict_aux_k(int64_t npar, const int32_t* __restrict__ pid, const int32_t* __restrict__ pptr,
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
    T acc[K];
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = 0;
    for (int32_t p = p0; p < p1; ++p) {
      const VK<T> c = ldk<T>(F + (int64_t)child[p] * K);
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] += c.v[j];
    }
    VK<T> f = ldk<T>(F + (int64_t)par * K);
#pragma unroll
    for (int j = 0; j < K; ++j) f.v[j] += (T)0.5 * acc[j];
    stk<T>(F + (int64_t)par * K, f);
  }
  pdl_trigger();
}

template <class T>
__global__ void k_prolong_aux_k(int64_t nnew, const int32_t* __restrict__ id, const int32_t* __restrict__ p0,
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
    T v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = 0;
    if (a >= 0) {
      const VK<T> x = ldk<T>(U + (int64_t)a * K);
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] += x.v[j];
    }
    if (b >= 0) {
      const VK<T> x = ldk<T>(U + (int64_t)b * K);
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] += x.v[j];
    }
    VK<T> o;
#pragma unroll
    for (int j = 0; j < K; ++j) o.v[j] = (T)0.5 * v[j];
    stk<T>(U + (int64_t)me * K, o);
  }
  pdl_trigger();
}

template <class T>
__global__ void k_addsaved_aux_k(int64_t nsm, const int32_t* __restrict__ rows, const T* __restrict__ us, T* U) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int32_t i = t < nsm ? rows[t] : -1;
  pdl_wait();
  if (i >= 0) {
    const VK<T> s = ldk<T>(us + t * K);
    VK<T> u = ldk<T>(U + (int64_t)i * K);
#pragma unroll
    for (int j = 0; j < K; ++j) u.v[j] += s.v[j];
    stk<T>(U + (int64_t)i * K, u);
  }
  pdl_trigger();
}

// coarsest level, FP64, one warp per row (the lanes' order of k_coarse per column)
template <class T>
__global__ void k_coarse_k(int64_t nc, const int32_t* __restrict__ cid, const double* __restrict__ inv,
                           const T* __restrict__ F, T* __restrict__ U) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  pdl_wait();
  if (row < nc) {
    double s[K];
#pragma unroll
    for (int j = 0; j < K; ++j) s[j] = 0;
    for (int64_t c = lane; c < nc; c += 32) {
      const double a = inv[row * nc + c];
      const VK<T> f = ldk<T>(F + (int64_t)cid[c] * K);
#pragma unroll
      for (int j = 0; j < K; ++j) s[j] += a * (double)f.v[j];
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
      for (int o = 16; o; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
    if (lane == 0) {
      VK<T> o;
#pragma unroll
      for (int j = 0; j < K; ++j) o.v[j] = (T)s[j];
      stk<T>(U + (int64_t)cid[row] * K, o);
    }
  }
  pdl_trigger();
}

// ---------------------------------------------------- small levels, fused
// As k_small_down / k_small_up of solve.cu with KRHS columns per row in
// shared memory; the levels of a run have at most small_lmax_k<T>() rows.
constexpr int SMALL_TPB_K = 1024;
constexpr int SMALL_B_K = 8;

template <class T>
__host__ __device__ constexpr int small_lmax_k() {
  return sizeof(T) == 4 ? 4096 : 2048;
}

template <class T>
constexpr size_t small_smem_k() {
  return 2 * (size_t)small_lmax_k<T>() * K * sizeof(T) + 2 * (size_t)(small_lmax_k<T>() + 1) * sizeof(int32_t);
}

// acc[j] - sum_p val[p] x[col[p]][j] over p0 <= p < p1 (the order of small_row)
template <class T, class V>
__device__ __forceinline__ void small_row_k(T (&acc)[K], int p0, int p1, const V* __restrict__ val,
                                            const uint16_t* __restrict__ col, const T* x) {
  T v[SMALL_B_K];
  uint16_t c[SMALL_B_K];
#pragma unroll
  for (int q = 0; q < SMALL_B_K; ++q)
    if (p0 + q < p1) {
      v[q] = (T)val_of(val[p0 + q]);
      c[q] = col[p0 + q];
    }
#pragma unroll
  for (int q = 0; q < SMALL_B_K; ++q)
    if (p0 + q < p1) {
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] -= v[q] * x[(int)c[q] * K + j];
    }
  for (int p = p0 + SMALL_B_K; p < p1; ++p) {
    const T a = (T)val_of(val[p]);
    const int cc = col[p];
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] -= a * x[cc * K + j];
  }
}

template <class T, class V>
__global__ void __launch_bounds__(SMALL_TPB_K, 1)
    k_small_down_k(const SmallDesc<T>* __restrict__ D, int nlev, T* F, int nu) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LM = small_lmax_k<T>();
  T* Ul = reinterpret_cast<T*>(smraw);
  T* Fl = Ul + LM * K;
  int32_t* Psm = reinterpret_cast<int32_t*>(Fl + LM * K);
  int32_t* Prs = Psm + LM + 1;
  if (nlev > 0) small_prefetch<T, V>(D, true);
  pdl_wait();
  for (int d = 0; d < nlev; ++d) {
    const SmallDesc<T>& L = D[d];
    const int mS = L.mS, mE = L.mE;
    if (d + 1 < nlev) small_prefetch<T, V>(D + d + 1, true);
    for (int k = threadIdx.x; k <= mE; k += blockDim.x) {
      if (k < mE) {
        const VK<T> f = ldk<T>(F + (int64_t)L.gid[k] * K);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          Fl[k * K + j] = f.v[j];
          Ul[k * K + j] = 0;
        }
        if (k < mS) stk<T>(L.fs + (int64_t)k * K, f);
      }
      if (k <= mS) Psm[k] = L.sm_ptr[k];
      Prs[k] = L.rs_ptr[k];
    }
    __syncthreads();
    for (int sw = 0; sw < nu; ++sw)
      for (int c = 0; c < L.ncol; ++c) {
        for (int k = L.cs[c] + threadIdx.x; k < L.cs[c + 1]; k += blockDim.x) {
          T acc[K];
#pragma unroll
          for (int j = 0; j < K; ++j) acc[j] = Fl[k * K + j];
          small_row_k(acc, Psm[k], Psm[k + 1], sm_vals(L, (const V*)nullptr), L.sm_col, Ul);
          const T di = L.dinv[k];
#pragma unroll
          for (int j = 0; j < K; ++j) Ul[k * K + j] += acc[j] * di;
        }
        __syncthreads();
      }
    for (int k = threadIdx.x; k < mE; k += blockDim.x) {
      T acc[K];
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] = Fl[k * K + j];
      small_row_k(acc, Prs[k], Prs[k + 1], rs_vals(L, (const V*)nullptr), L.rs_col, Ul);
#pragma unroll
      for (int j = 0; j < K; ++j) Fl[k * K + j] = acc[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < L.npar; t += blockDim.x) {
      T acc[K];
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] = 0;
      for (int p = L.rp_ptr[t]; p < L.rp_ptr[t + 1]; ++p)
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j] += Fl[(int)L.rp_child[p] * K + j];
      const int pr = L.rp_id[t];
#pragma unroll
      for (int j = 0; j < K; ++j) Fl[pr * K + j] += (T)0.5 * acc[j];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < mE; k += blockDim.x) {
      VK<T> f, u;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        f.v[j] = Fl[k * K + j];
        u.v[j] = Ul[k * K + j];
      }
      stk<T>(F + (int64_t)L.gid[k] * K, f);
      if (k < mS) stk<T>(L.us + (int64_t)k * K, u);
    }
    __syncthreads();
  }
  pdl_trigger();
}

template <class T, class V>
__global__ void __launch_bounds__(SMALL_TPB_K, 1)
    k_small_up_k(const SmallDesc<T>* __restrict__ D, int nlev, T* U, int nu) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LM = small_lmax_k<T>();
  T* Ul = reinterpret_cast<T*>(smraw);
  T* Fl = Ul + LM * K;
  int32_t* Psm = reinterpret_cast<int32_t*>(Fl + LM * K);
  if (nlev > 0) small_prefetch<T, V>(D + nlev - 1, false);
  pdl_wait();
  for (int d = nlev - 1; d >= 0; --d) {
    const SmallDesc<T>& L = D[d];
    const int mS = L.mS, mE = L.mE;
    if (d > 0) small_prefetch<T, V>(D + d - 1, false);
    for (int k = threadIdx.x; k < mE; k += blockDim.x) {
      const VK<T> u = ldk<T>(U + (int64_t)L.gid[k] * K);
#pragma unroll
      for (int j = 0; j < K; ++j) Ul[k * K + j] = u.v[j];
      if (k < mS) {
        const VK<T> f = ldk<T>(L.fs + (int64_t)k * K);
#pragma unroll
        for (int j = 0; j < K; ++j) Fl[k * K + j] = f.v[j];
      }
      if (k <= mS) Psm[k] = L.sm_ptr[k];
    }
    if (mS == mE && threadIdx.x == 0) Psm[mS] = L.sm_ptr[mS];
    __syncthreads();
    for (int t = threadIdx.x; t < L.nnew; t += blockDim.x) {
      const int32_t a = L.nn_p0[t], b = L.nn_p1[t];
      const int me = L.nn_id[t];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        T v = 0;
        if (a >= 0) v += Ul[a * K + j];
        if (b >= 0) v += Ul[b * K + j];
        Ul[me * K + j] = (T)0.5 * v;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < mS; k += blockDim.x) {
      const VK<T> s = ldk<T>(L.us + (int64_t)k * K);
#pragma unroll
      for (int j = 0; j < K; ++j) Ul[k * K + j] += s.v[j];
    }
    __syncthreads();
    for (int sw = 0; sw < nu; ++sw)
      for (int c = L.ncol - 1; c >= 0; --c) {
        for (int k = L.cs[c] + threadIdx.x; k < L.cs[c + 1]; k += blockDim.x) {
          T acc[K];
#pragma unroll
          for (int j = 0; j < K; ++j) acc[j] = Fl[k * K + j];
          small_row_k(acc, Psm[k], Psm[k + 1], sm_vals(L, (const V*)nullptr), L.sm_col, Ul);
          const T di = L.dinv[k];
#pragma unroll
          for (int j = 0; j < K; ++j) Ul[k * K + j] += acc[j] * di;
        }
        __syncthreads();
      }
    for (int k = threadIdx.x; k < mS; k += blockDim.x) {
      VK<T> u;
#pragma unroll
      for (int j = 0; j < K; ++j) u.v[j] = Ul[k * K + j];
      stk<T>(U + (int64_t)L.gid[k] * K, u);
    }
    __syncthreads();
  }
  pdl_trigger();
}

// ------------------------------------------------------------------ PCG
__device__ __forceinline__ void set_cond_k(MultiScalars* sc, int cond, cudaGraphConditionalHandle hnd, int use_hnd) {
  sc->cond = cond;
  if (use_hnd) cudaGraphSetConditional(hnd, cond ? 1u : 0u);
}

// r = b - A x; ||b||, ||r|| per column; scalars initialised, columns activated
__global__ void k_pcg_init_k(int64_t n, SellView<double> A, const double* __restrict__ b, const double* __restrict__ x,
                             double* __restrict__ r, double* partial, unsigned int* ticket, MultiScalars* sc,
                             double rtol, int maxit, double* hist, cudaGraphConditionalHandle hnd, int use_hnd) {
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  Row<double> row;
  if (i0 < n) row_load(row, i0, A.off, A.col, A.val);
  pdl_wait();
  double v[2 * K];
#pragma unroll
  for (int j = 0; j < 2 * K; ++j) v[j] = 0;
  for (int64_t i = i0; i < n; i += st) {
    if (i != i0) row_load(row, i, A.off, A.col, A.val);
    double ax[K];
    row_dot_k<double, double>(row, A.col, A.val, x, ax);
    const VK<double> bi = ldk<double>(b + i * K);
    VK<double> ri;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      ri.v[j] = bi.v[j] - ax[j];
      v[j] += bi.v[j] * bi.v[j];
      v[K + j] += ri.v[j] * ri.v[j];
    }
    stk<double>(r + i * K, ri);
  }
  if (grid_reduce<2 * K>(v, partial, ticket) && threadIdx.x == 0) {
    int any = 0;
    for (int j = 0; j < K; ++j) {
      sc->bnorm[j] = sqrt(v[j]);
      sc->tol[j] = rtol * sc->bnorm[j];
      sc->rr[j] = v[K + j];
      sc->k[j] = 0;
      sc->rz[j] = 0;
      sc->alpha[j] = 0;
      sc->beta[j] = 0;
      hist[(int64_t)j * (maxit + 1)] = sqrt(v[K + j]);
      const bool conv = sqrt(v[K + j]) <= sc->tol[j];
      sc->status[j] = conv ? 0 : 1;
      sc->active[j] = (!conv && maxit > 0) ? 1 : 0;
      any |= sc->active[j];
    }
    sc->maxit = maxit;
    sc->timeout = 0;
    set_cond_k(sc, any, hnd, use_hnd);
  }
}

// <z, r>, <z, q_prev>  ->  beta, rz per active column
template <class T>
__global__ void k_dots_k(int64_t n, const T* __restrict__ z, const double* __restrict__ r, const double* __restrict__ q,
                         double* partial, unsigned int* ticket, MultiScalars* sc) {
  pdl_wait();
  double v[2 * K];
#pragma unroll
  for (int j = 0; j < 2 * K; ++j) v[j] = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const VK<T> zi = ldk<T>(z + i * K);
    const VK<double> ri = ldk<double>(r + i * K), qi = ldk<double>(q + i * K);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const double zz = (double)zi.v[j];
      v[j] += zz * ri.v[j];
      v[K + j] += zz * qi.v[j];
    }
  }
  if (grid_reduce<2 * K>(v, partial, ticket) && threadIdx.x == 0) {
    for (int j = 0; j < K; ++j) {
      if (!sc->active[j]) {
        sc->beta[j] = 0;
        continue;
      }
      sc->beta[j] = sc->k[j] == 0 ? 0.0 : -sc->alpha[j] * v[K + j] / sc->rz[j];
      sc->rz[j] = v[j];
      if (!(v[j] > 0)) {
        sc->status[j] = ASMG_ERR_BREAKDOWN;
        sc->active[j] = 0;
        sc->beta[j] = 0;
      }
    }
  }
}

// p = z + beta p
template <class T>
__global__ void k_pupd_k(int64_t n, const T* __restrict__ z, double* __restrict__ p,
                         const MultiScalars* __restrict__ sc) {
  pdl_wait();
  double beta[K];
#pragma unroll
  for (int j = 0; j < K; ++j) beta[j] = sc->beta[j];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const VK<T> zi = ldk<T>(z + i * K);
    VK<double> pi = ldk<double>(p + i * K);
#pragma unroll
    for (int j = 0; j < K; ++j) pi.v[j] = (double)zi.v[j] + beta[j] * pi.v[j];
    stk<double>(p + i * K, pi);
  }
  pdl_trigger();
}

// q = A p, <p, q>  ->  alpha per active column
__global__ void k_spmv_dot_k(int64_t n, SellView<double> A, const double* __restrict__ p, double* __restrict__ q,
                             double* partial, unsigned int* ticket, MultiScalars* sc) {
  // the row's entries in registers at once, the first row before the wait
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  Row<double> row;
  if (i0 < n) row_load(row, i0, A.off, A.col, A.val);
  pdl_wait();
  double v[K];
#pragma unroll
  for (int j = 0; j < K; ++j) v[j] = 0;
  for (int64_t i = i0; i < n; i += st) {
    if (i != i0) row_load(row, i, A.off, A.col, A.val);
    double qi[K];
    row_dot_k<double, double>(row, A.col, A.val, p, qi);
    const VK<double> pi = ldk<double>(p + i * K);
    VK<double> qo;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      qo.v[j] = qi[j];
      v[j] += pi.v[j] * qi[j];
    }
    stk<double>(q + i * K, qo);
  }
  if (grid_reduce<K>(v, partial, ticket) && threadIdx.x == 0) {
    for (int j = 0; j < K; ++j) {
      if (!sc->active[j]) {
        sc->alpha[j] = 0;
        continue;
      }
      sc->pq[j] = v[j];
      if (!(v[j] > 0)) {
        sc->status[j] = ASMG_ERR_BREAKDOWN;
        sc->active[j] = 0;
        sc->alpha[j] = 0;
      } else {
        sc->alpha[j] = sc->rz[j] / v[j];
      }
    }
  }
}

// x += alpha p, r -= alpha q, ||r|| -> history and stopping test per column
__global__ void k_axpy_norm_k(int64_t n, const double* __restrict__ p, const double* __restrict__ q,
                              double* __restrict__ x, double* __restrict__ r, double* partial, unsigned int* ticket,
                              MultiScalars* sc, double* hist, cudaGraphConditionalHandle hnd, int use_hnd) {
  pdl_wait();
  double a[K];
#pragma unroll
  for (int j = 0; j < K; ++j) a[j] = sc->alpha[j];
  double v[K];
#pragma unroll
  for (int j = 0; j < K; ++j) v[j] = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const VK<double> pi = ldk<double>(p + i * K), qi = ldk<double>(q + i * K);
    VK<double> xi = ldk<double>(x + i * K), ri = ldk<double>(r + i * K);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      xi.v[j] += a[j] * pi.v[j];
      ri.v[j] = ri.v[j] - a[j] * qi.v[j];
      v[j] += ri.v[j] * ri.v[j];
    }
    stk<double>(x + i * K, xi);
    stk<double>(r + i * K, ri);
  }
  if (grid_reduce<K>(v, partial, ticket) && threadIdx.x == 0) {
    int any = 0;
    for (int j = 0; j < K; ++j) {
      if (!sc->active[j]) continue;
      if (sc->timeout) {
        sc->status[j] = ASMG_ERR_TIMEOUT;
        sc->active[j] = 0;
        continue;
      }
      sc->k[j] += 1;
      sc->rr[j] = v[j];
      const double nr = sqrt(v[j]);
      hist[(int64_t)j * (sc->maxit + 1) + sc->k[j]] = nr;
      if (nr <= sc->tol[j]) {
        sc->status[j] = 0;
        sc->active[j] = 0;
      } else if (!isfinite(nr)) {
        sc->status[j] = ASMG_ERR_BREAKDOWN;
        sc->active[j] = 0;
      } else if (sc->k[j] >= sc->maxit) {
        sc->active[j] = 0;
      }
      any |= sc->active[j];
    }
    set_cond_k(sc, any, hnd, use_hnd);
  }
}

// vertex-major columns [KRHS][nv] <-> permuted interleaved rows [npad][KRHS]
__global__ void k_gather_k(int64_t n, int64_t nv, const int32_t* __restrict__ vrow, const double* __restrict__ src,
                           double* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t v = vrow[i];
  VK<double> o;
#pragma unroll
  for (int j = 0; j < K; ++j) o.v[j] = v >= 0 ? src[(int64_t)j * nv + v] : 0.0;
  stk<double>(dst + i * K, o);
}

__global__ void k_scatter_k(int64_t nv, const int32_t* __restrict__ rowv, const double* __restrict__ src,
                            double* __restrict__ dst) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int32_t r = rowv[v];
  if (r >= 0) {
    const VK<double> x = ldk<double>(src + (int64_t)r * K);
#pragma unroll
    for (int j = 0; j < K; ++j) dst[(int64_t)j * nv + v] = x.v[j];
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) dst[(int64_t)j * nv + v] = 0.0;
  }
}

// --------------------------------------------------------- enqueueing
template <class T>
Prec<T>& prec_of(asmg_s& h);
template <>
Prec<double>& prec_of<double>(asmg_s& h) { return h.p64; }
template <>
Prec<float>& prec_of<float>(asmg_s& h) { return h.p32; }

template <class T>
MultiPrec<T>& mprec_of(MultiSlot& S);
template <>
MultiPrec<double>& mprec_of<double>(MultiSlot& S) { return S.m64; }
template <>
MultiPrec<float>& mprec_of<float>(MultiSlot& S) { return S.m32; }

template <class T>
SellView<T> fine_matrix(asmg_s& h);
template <>
SellView<double> fine_matrix<double>(asmg_s& h) { return view(h.A64); }
template <>
SellView<float> fine_matrix<float>(asmg_s& h) { return view(h.p32.Af); }

template <class T>
const T* fine_dinv_of(asmg_s& h);
template <>
const double* fine_dinv_of<double>(asmg_s& h) { return h.dinv64.p; }
template <>
const float* fine_dinv_of<float>(asmg_s& h) { return h.p32.dinv_f.p; }

// V: how the auxiliary-level matrices are read (T, or bf16v with level_bf16)
template <class T, class V>
void enqueue_vcycle_k(asmg_s& h, MultiSlot& S, cudaStream_t s) {
  Prec<T>& P = prec_of<T>(h);
  MultiPrec<T>& M = mprec_of<T>(S);
  const bool pdl = h.prm.use_pdl;
  const int npre = h.prm.nu_pre, npost = h.prm.nu_post;
  const int nlev = (int)P.lev.size();
  const int ndeep = M.n_deep, nbot = M.n_bottom;
  const size_t smem = small_smem_k<T>();
  if (ndeep) launch_smem(pdl, k_small_down_k<T, V>, 1, SMALL_TPB_K, smem, s, M.deep_desc.p, ndeep, M.F.p, npre);
  for (int li = nlev - 1 - ndeep; li >= nbot; --li) {
    AuxLevelDev<T>& L = P.lev[li];
    auto SMd = view(L.SMd);
    for (int sweep = 0; sweep < npre; ++sweep)
      for (int c = 0; c < L.ncolours; ++c) {
        const int64_t k0 = L.cstart[c], nk = L.cstart[c + 1] - L.cstart[c];
        if (!nk) continue;
        launch(pdl, k_gs_aux_down_k<T, V>, nblk(nk, rows_tpb(nk)), rows_tpb(nk), s, k0, nk, SMd.off, SMd.col, sell_vals(L.SMd, (const V*)nullptr),
               L.sm_dinv.p, L.sm_rows.p, (const T*)M.F.p, sweep == 0 ? 1 : 0, M.fs[li].p, M.us[li].p);
      }
    auto RS = view(L.RS);
    launch(pdl, k_resid_aux_k<T, V>, nblk(L.nrs, rows_tpb(L.nrs)), rows_tpb(L.nrs), s, L.nrs, RS.off, RS.col, sell_vals(L.RS, (const V*)nullptr),
           L.rs_rows.p, (const T*)M.us[li].p, M.F.p);
    launch(pdl, k_restrict_aux_k<T>, nblk(L.npar, rows_tpb(L.npar)), rows_tpb(L.npar), s, L.npar, L.rp_id.p,
           L.rp_ptr.p, L.rp_child.p, M.F.p);
  }
  if (nbot) launch_smem(pdl, k_small_down_k<T, V>, 1, SMALL_TPB_K, smem, s, M.bot_desc.p, nbot, M.F.p, npre);
  if (h.nc > 0)
    launch(pdl, k_coarse_k<T>, nblk(h.nc * 32), TPB, s, h.nc, h.d_cid.p, h.d_cinv.p, (const T*)M.F.p, M.U.p);
  if (nbot) launch_smem(pdl, k_small_up_k<T, V>, 1, SMALL_TPB_K, smem, s, M.bot_desc.p, nbot, M.U.p, npost);
  for (int li = nbot; li <= nlev - 1 - ndeep; ++li) {
    AuxLevelDev<T>& L = P.lev[li];
    auto SM = view(L.SM);
    if (L.nnew)
      launch(pdl, k_prolong_aux_k<T>, nblk(L.nnew, rows_tpb(L.nnew)), rows_tpb(L.nnew), s, L.nnew, L.nn_id.p,
             L.nn_p0.p, L.nn_p1.p, M.U.p);
    launch(pdl, k_addsaved_aux_k<T>, nblk(L.nsm, rows_tpb(L.nsm)), rows_tpb(L.nsm), s, L.nsm, L.sm_rows.p,
           (const T*)M.us[li].p, M.U.p);
    for (int sweep = 0; sweep < npost; ++sweep)
      for (int c = L.ncolours - 1; c >= 0; --c) {
        const int64_t k0 = L.cstart[c], nk = L.cstart[c + 1] - L.cstart[c];
        if (!nk) continue;
        launch(pdl, k_gs_aux_k<T, V>, nblk(nk, rows_tpb(nk)), rows_tpb(nk), s, k0, nk, SM.off, SM.col, sell_vals(L.SM, (const V*)nullptr),
               L.sm_dinv.p, L.sm_rows.p, (const T*)M.fs[li].p, M.U.p);
      }
  }
  if (ndeep) launch_smem(pdl, k_small_up_k<T, V>, 1, SMALL_TPB_K, smem, s, M.deep_desc.p, ndeep, M.U.p, npost);
}

// z = B_co r for KRHS columns (Algorithm 1, multiplicative, Gauss-Seidel)
template <class T>
void enqueue_vcycle_vals_k(asmg_s& h, MultiSlot& S, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value)
    if (h.prm.level_bf16) return enqueue_vcycle_k<float, bf16v>(h, S, s);
  enqueue_vcycle_k<T, T>(h, S, s);
}

template <class T>
void enqueue_precond_k(asmg_s& h, MultiSlot& S, const double* r, cudaStream_t s) {
  Prec<T>& P = prec_of<T>(h);
  MultiPrec<T>& M = mprec_of<T>(S);
  const SellView<T> A = fine_matrix<T>(h);
  const T* dinv = fine_dinv_of<T>(h);
  const bool pdl = h.prm.use_pdl;
  ASMG_CUDA(cudaMemsetAsync(M.uf.p, 0, sizeof(T) * h.npad * K, s));
  const int ncol = (int)h.fine_cstart.size() - 1;
  auto smooth = [&](bool forward) {
    for (int m = 0; m < h.prm.fine_sweeps; ++m)
      for (int q = 0; q < ncol; ++q) {
        const int c = forward ? q : ncol - 1 - q;
        const int64_t r0 = h.fine_cstart[c], nr = h.fine_cstart[c + 1] - r0;
        if (!nr) continue;
        launch(pdl, k_gs_fine_k<T>, nblk(nr, rows_tpb(nr)), rows_tpb(nr), s, r0, nr, A.off, A.col, A.val, dinv, r,
               M.uf.p);
      }
  };
  smooth(true);
  if (h.nJ > 0) {
    launch(pdl, k_resid_fine_k<T>, nblk(h.npad), TPB, s, h.npad, A.off, A.col, A.val, r, (const T*)M.uf.p, M.rho.p);
    auto PT = view(P.PT);
    launch(pdl, k_restrict_fine_k<T>, nblk(h.nJpad), TPB, s, h.nJpad, PT.off, PT.col, PT.val, (const T*)M.rho.p,
           M.F.p, M.U.p);
    enqueue_vcycle_vals_k<T>(h, S, s);
    auto PP = view(P.P);
    launch(pdl, k_prolong_fine_k<T>, nblk(h.npad), TPB, s, h.npad, PP.off, PP.col, PP.val, (const T*)M.U.p, M.uf.p);
  }
  smooth(false);
  ASMG_CUDA(cudaGetLastError());
}

template <class T>
void enqueue_body_k(asmg_s& h, MultiSlot& S, cudaStream_t s, cudaGraphConditionalHandle hnd, int use_hnd) {
  enqueue_precond_k<T>(h, S, S.r.p, s);
  const T* z = mprec_of<T>(S).uf.p;
  const bool pdl = h.prm.use_pdl;
  launch(pdl, k_dots_k<T>, RED_BLOCKS, TPB, s, h.npad, z, (const double*)S.r.p, (const double*)S.q.p, S.partial.p,
         S.ticket.p, S.scal.p);
  launch(pdl, k_pupd_k<T>, RED_BLOCKS, TPB, s, h.npad, z, S.p.p, (const MultiScalars*)S.scal.p);
  launch(pdl, k_spmv_dot_k, RED_BLOCKS, TPB, s, h.npad, view(h.A64), (const double*)S.p.p, S.q.p, S.partial.p,
         S.ticket.p, S.scal.p);
  launch(pdl, k_axpy_norm_k, RED_BLOCKS, TPB, s, h.npad, (const double*)S.p.p, (const double*)S.q.p, S.x.p, S.r.p,
         S.partial.p, S.ticket.p, S.scal.p, S.hist.p, hnd, use_hnd);
  ASMG_CUDA(cudaGetLastError());
}

void enqueue_body_any_k(asmg_s& h, MultiSlot& S, cudaStream_t s, cudaGraphConditionalHandle hnd, int use_hnd) {
  if (h.prm.precision == ASMG_MIXED)
    enqueue_body_k<float>(h, S, s, hnd, use_hnd);
  else
    enqueue_body_k<double>(h, S, s, hnd, use_hnd);
}

void enqueue_init_k(asmg_s& h, MultiSlot& S, double rtol, cudaStream_t s, cudaGraphConditionalHandle hnd,
                    int use_hnd) {
  launch(h.prm.use_pdl, k_pcg_init_k, RED_BLOCKS, TPB, s, h.npad, view(h.A64), (const double*)S.b.p,
         (const double*)S.x.p, S.r.p, S.partial.p, S.ticket.p, S.scal.p, rtol, h.prm.max_iter, S.hist.p, hnd, use_hnd);
  ASMG_CUDA(cudaGetLastError());
}

// Work state for KRHS columns in precision T, and the fused small-level runs
// whose levels fit small_lmax_k<T>() rows.
template <class T>
void alloc_multi_prec(asmg_s& h, MultiPrec<T>& M, cudaStream_t s) {
  Prec<T>& P = prec_of<T>(h);
  M.uf.alloc(h.npad * K);
  M.rho.alloc(h.npad * K);
  M.F.alloc(std::max<int64_t>(h.nJpad, 1) * K);
  M.U.alloc(std::max<int64_t>(h.nJpad, 1) * K);
  M.uf.zero(s);
  M.rho.zero(s);
  M.F.zero(s);
  M.U.zero(s);
  const int nlev = (int)P.lev.size();
  M.fs.clear();
  M.us.clear();
  M.fs.resize(nlev);
  M.us.resize(nlev);
  for (int li = 0; li < nlev; ++li) {
    M.fs[li].alloc(std::max<int64_t>(P.lev[li].nsm, 1) * K);
    M.us[li].alloc(std::max<int64_t>(P.lev[li].nsm, 1) * K);
    M.fs[li].zero(s);
    M.us[li].zero(s);
  }
  auto fits = [&](int li) {
    const SmallLevelDev<T>& q = P.lev[li].small;
    return q.ok && q.mE <= small_lmax_k<T>();
  };
  int nd = 0;
  while (nd < nlev && fits(nlev - 1 - nd)) ++nd;
  int nb = 0;
  if (nd < nlev)
    while (nb < nlev - nd && fits(nb)) ++nb;
  M.n_deep = nd;
  M.n_bottom = nb;
  auto desc = [&](int li) {
    AuxLevelDev<T>& L = P.lev[li];
    SmallLevelDev<T>& S = L.small;
    SmallDesc<T> d;
    d.mS = S.mS;
    d.mE = S.mE;
    d.ncol = S.ncol;
    d.nnew = S.nnew;
    d.npar = S.npar;
    d.nnz_sm = (int)S.nnz_sm;
    d.nnz_rs = (int)S.nnz_rs;
    d.nchild = (int)S.nchild;
    for (int c = 0; c <= SMALL_MAXC; ++c) d.cs[c] = c <= S.ncol ? S.cs[c] : S.mS;
    d.gid = S.gid.p;
    d.sm_ptr = S.sm_ptr.p;
    d.sm_col = S.sm_col.p;
    d.sm_val = S.sm_val.p;
    d.sm_v16 = S.sm_v16.p;
    d.dinv = S.dinv.p;
    d.rs_ptr = S.rs_ptr.p;
    d.rs_col = S.rs_col.p;
    d.rs_val = S.rs_val.p;
    d.rs_v16 = S.rs_v16.p;
    d.nn_id = S.nn_id.p;
    d.nn_p0 = S.nn_p0.p;
    d.nn_p1 = S.nn_p1.p;
    d.rp_id = S.rp_id.p;
    d.rp_ptr = S.rp_ptr.p;
    d.rp_child = S.rp_child.p;
    d.fs = M.fs[li].p;
    d.us = M.us[li].p;
    return d;
  };
  std::vector<SmallDesc<T>> deep, bot;
  for (int k = 0; k < nd; ++k) deep.push_back(desc(nlev - 1 - k));
  for (int k = nb - 1; k >= 0; --k) bot.push_back(desc(k));
  M.deep_desc.upload(deep, s);
  M.bot_desc.upload(bot, s);
  const int smem = (int)small_smem_k<T>();
  ASMG_CUDA(cudaFuncSetAttribute(k_small_down_k<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  ASMG_CUDA(cudaFuncSetAttribute(k_small_up_k<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  if constexpr (std::is_same<T, float>::value) {
    ASMG_CUDA(cudaFuncSetAttribute(k_small_down_k<T, bf16v>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ASMG_CUDA(cudaFuncSetAttribute(k_small_up_k<T, bf16v>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  }
}

void build_graph_k(asmg_s& h, MultiSlot& S, double rtol) {
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
  capture_solve_multi(h, S, rtol, g, nullptr, 0);
  ASMG_CUDA(cudaGraphInstantiate(&S.gexec, g, 0));
  S.graph = g;
}

}  // namespace

bool multi_supported(const asmg_s& h) {
  return !h.mesh.mixed && h.prm.smoother == 0 && h.prm.additive == 0 && h.prm.iteration == 0;
}

MultiSlot& add_multi_slot(asmg_s& h, cudaStream_t s) {
  h.mslots.emplace_back(new MultiSlot());
  MultiSlot& S = *h.mslots.back();
  for (DBuf<double>* v : {&S.b, &S.x, &S.r, &S.p, &S.q}) {
    v->alloc(h.npad * K);
    v->zero(s);
  }
  S.vb.alloc(h.mesh.nv * K);
  S.vu.alloc(h.mesh.nv * K);
  S.partial.alloc(2 * K * RED_BLOCKS);
  S.ticket.alloc(1);
  S.ticket.zero(s);
  S.scal.alloc(1);
  S.scal.zero(s);
  S.hist.alloc((int64_t)K * (h.prm.max_iter + 1));
  if (h.prm.precision == ASMG_MIXED)
    alloc_multi_prec(h, S.m32, s);
  else
    alloc_multi_prec(h, S.m64, s);
  ASMG_CUDA(cudaStreamSynchronize(s));
  return S;
}

void gather_multi(asmg_s& h, const double* vsrc, double* dst, cudaStream_t s) {
  launch(false, k_gather_k, nblk(h.npad), TPB, s, h.npad, h.mesh.nv, h.d_vertex_of_row.p, vsrc, dst);
  ASMG_CUDA(cudaGetLastError());
}

void scatter_multi(asmg_s& h, const double* src, double* vdst, cudaStream_t s) {
  launch(false, k_scatter_k, nblk(h.mesh.nv), TPB, s, h.mesh.nv, h.d_row_of_vertex.p, src, vdst);
  ASMG_CUDA(cudaGetLastError());
}

// The graph of one multiple solve into `g`: init -> WHILE(any column active) { body }.
cudaGraphNode_t capture_solve_multi(asmg_s& h, MultiSlot& S, double rtol, cudaGraph_t g, const cudaGraphNode_t* deps,
                                    size_t ndeps) {
  cudaGraphConditionalHandle hnd;
  ASMG_CUDA(cudaGraphConditionalHandleCreate(&hnd, g, 0, 0));
  cudaStream_t cs;
  ASMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  ASMG_CUDA(cudaStreamBeginCaptureToGraph(cs, g, deps, nullptr, ndeps, cudaStreamCaptureModeThreadLocal));
  enqueue_init_k(h, S, rtol, cs, hnd, 1);
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
  enqueue_body_any_k(h, S, cs, hnd, 1);
  cudaGraph_t bb;
  ASMG_CUDA(cudaStreamEndCapture(cs, &bb));
  ASMG_CUDA(cudaStreamDestroy(cs));
  return cnode;
}

void run_solve_multi(asmg_s& h, MultiSlot& S, double rtol, cudaStream_t s) {
  if (h.prm.use_graph) {
    if (!S.gexec || S.graph_rtol != rtol) {
      build_graph_k(h, S, rtol);
      S.graph_rtol = rtol;
    }
    ASMG_CUDA(cudaGraphLaunch(S.gexec, s));
  } else {
    enqueue_init_k(h, S, rtol, s, 0, 0);
    for (int it = 0; it < h.prm.max_iter; ++it) {
      MultiScalars sc;
      ASMG_CUDA(cudaMemcpyAsync(&sc, S.scal.p, sizeof sc, cudaMemcpyDeviceToHost, s));
      ASMG_CUDA(cudaStreamSynchronize(s));
      if (!sc.cond) break;
      enqueue_body_any_k(h, S, s, 0, 0);
    }
  }
}

}  // namespace asmg
