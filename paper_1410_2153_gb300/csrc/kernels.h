// Device and launch helpers shared by the solve kernels (solve.cu) and the
// multiple right-hand-side solve kernels (solve_multi.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace asmg {
namespace kern {

constexpr int TPB = 256;
constexpr int RED_BLOCKS = 152 * 4;  // persistent reduction grid: 4 CTAs per SM
constexpr int VEC_BLOCKS = 152 * 8;  // grid of the vector-only PCG kernels: 8 CTAs (full occupancy) per SM

inline int nblk(int64_t n, int t = TPB) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 1 << 24)); }

// Block size of a row-parallel launch: 256 threads when that fills every SM
// twice, else 64 so that small colour classes still spread over all SMs.
constexpr int NSM = 152;
inline int rows_tpb(int64_t rows) { return rows >= (int64_t)NSM * 2 * 256 ? 256 : 64; }

// Kernel launch with dynamic shared memory, optionally with programmatic dependent launch.
template <typename... KArgs, typename... Args>
void launch_smem(bool pdl, void (*kern)(KArgs...), int64_t grid, int block, size_t smem, cudaStream_t s,
                 Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  ASMG_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}

// Kernel launch, optionally with programmatic dependent launch (the kernel may
// start while its predecessor on the stream finishes; see pdl_wait below).
template <typename... KArgs, typename... Args>
void launch(bool pdl, void (*kern)(KArgs...), int64_t grid, int block, cudaStream_t s, Args... args) {
  if (!pdl) {
    kern<<<(unsigned)grid, (unsigned)block, 0, s>>>(static_cast<KArgs>(args)...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ASMG_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}

template <class T, class X>
__device__ __forceinline__ T sell_dot(int64_t row, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                      const T* __restrict__ val, const X* x) {
  const int64_t sl = row >> 5, lane = row & 31;
  const int64_t b = __ldg(off + sl), w = (__ldg(off + sl + 1) - b) >> 5;
  T s = 0;
  for (int64_t k = 0; k < w; ++k) {
    const int64_t e = b + (k << 5) + lane;
    s += __ldg(val + e) * (T)x[__ldg(col + e)];
  }
  return s;
}

// Programmatic dependent launch: every solve kernel first loads what was
// written at setup (matrix rows, index lists), then waits for the preceding
// kernel (griddepcontrol.wait), and lets the next kernel launch once its own
// work is done (griddepcontrol.launch_dependents).  Launched without the
// attribute, both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// A SELL-32 row held in registers (up to MAXW entries; longer rows read the rest later).
constexpr int MAXW = 10;
template <class T>
struct Row {
  int64_t b = 0, lane = 0;
  int w = 0;
  int32_t c[MAXW];
  T v[MAXW];
};

// Matrix values as stored (FP64, FP32 or BF16), widened to the arithmetic
// type exactly; the ldg forms read through the read-only path, the ldcs forms
// stream (evict first).
__device__ __forceinline__ double ldg_val(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_val(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_val(const bf16v* p) {
  return __uint_as_float((uint32_t)__ldg(&p->bits) << 16);
}
__device__ __forceinline__ double ldcs_val(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ldcs_val(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ldcs_val(const bf16v* p) {
  return __uint_as_float((uint32_t)__ldcs(&p->bits) << 16);
}
__device__ __forceinline__ double val_of(double v) { return v; }
__device__ __forceinline__ float val_of(float v) { return v; }
__device__ __forceinline__ float val_of(bf16v v) { return __uint_as_float((uint32_t)v.bits << 16); }

template <class T, class V>
__device__ __forceinline__ void row_load(Row<T>& R, int64_t row, const int64_t* __restrict__ off,
                                         const int32_t* __restrict__ col, const V* __restrict__ val) {
  const int64_t sl = row >> 5;
  R.lane = row & 31;
  R.b = __ldg(off + sl);
  R.w = (int)((__ldg(off + sl + 1) - R.b) >> 5);
#pragma unroll
  for (int k = 0; k < MAXW; ++k)
    if (k < R.w) {
      const int64_t e = R.b + ((int64_t)k << 5) + R.lane;
      R.c[k] = __ldcs(col + e);
      R.v[k] = (T)ldcs_val(val + e);
    }
}

template <class T, class V, class X>
__device__ __forceinline__ T row_dot(const Row<T>& R, const int32_t* __restrict__ col, const V* __restrict__ val,
                                     const X* x) {
  T s = 0;
#pragma unroll
  for (int k = 0; k < MAXW; ++k)
    if (k < R.w) s += R.v[k] * (T)x[R.c[k]];
  for (int k = MAXW; k < R.w; ++k) {
    const int64_t e = R.b + ((int64_t)k << 5) + R.lane;
    s += (T)ldg_val(val + e) * (T)x[__ldg(col + e)];
  }
  return s;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;  // valid in thread 0
}

// Deterministic grid reduction of NV values: partials per block, the last
// block to finish sums them in block order.  Returns true in that block.
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double* partial, unsigned int* ticket) {
  __shared__ double sh[32];
  __shared__ bool last;
  for (int j = 0; j < NV; ++j) {
    double t = block_sum(v[j], sh);
    if (threadIdx.x == 0) partial[j * gridDim.x + blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int j = 0; j < NV; ++j) {
    // the partials of this thread (blocks t, t + blockDim, ...) summed in
    // ascending order, eight loads in flight
    const double* pj = partial + (int64_t)j * gridDim.x;
    double s = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 8 * blockDim.x) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const unsigned bb = b + u * blockDim.x;
        x[u] = bb < gridDim.x ? __ldcg(pj + bb) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) s += x[u];
    }
    v[j] = block_sum(s, sh);
  }
  if (threadIdx.x == 0) *ticket = 0;
  return true;
}

// Ask L1 for the [p, p + bytes) lines (a hint: no data moves into registers,
// nothing is waited for); the block's threads share the lines.
__device__ __forceinline__ void l1_prefetch(const void* p, int64_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (int64_t o = (int64_t)threadIdx.x * 128; o < bytes; o += (int64_t)blockDim.x * 128)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(c + o));
}

// the level's stored values: FP32/FP64, or their BF16 copy
template <class T>
__device__ __forceinline__ const T* sm_vals(const SmallDesc<T>& L, const T*) { return L.sm_val; }
template <class T>
__device__ __forceinline__ const bf16v* sm_vals(const SmallDesc<T>& L, const bf16v*) { return L.sm_v16; }
template <class T>
__device__ __forceinline__ const T* rs_vals(const SmallDesc<T>& L, const T*) { return L.rs_val; }
template <class T>
__device__ __forceinline__ const bf16v* rs_vals(const SmallDesc<T>& L, const bf16v*) { return L.rs_v16; }

// The setup data one level of a fused run reads (never written by a solve, so
// it may be requested before the wait on the previous kernel): the level's
// own descriptor, row pointers, entries as the kernel reads them (V) and
// diagonal, and the tables of the restriction (down) or of the new nodes'
// parents (up).  Its phases then read
// these from L1 rather than waiting on L2 at every colour phase.
template <class T, class V>
__device__ __forceinline__ void small_prefetch(const SmallDesc<T>* Dd, bool down) {
  const SmallDesc<T>& L = *Dd;
  l1_prefetch(L.gid, (int64_t)L.mE * 4);
  l1_prefetch(L.sm_ptr, (int64_t)(L.mS + 1) * 4);
  l1_prefetch(L.sm_col, (int64_t)L.nnz_sm * 2);
  l1_prefetch(sm_vals(L, (const V*)nullptr), (int64_t)L.nnz_sm * sizeof(V));
  l1_prefetch(L.dinv, (int64_t)L.mS * sizeof(T));
  if (down) {
    l1_prefetch(L.rs_ptr, (int64_t)(L.mE + 1) * 4);
    l1_prefetch(L.rs_col, (int64_t)L.nnz_rs * 2);
    l1_prefetch(rs_vals(L, (const V*)nullptr), (int64_t)L.nnz_rs * sizeof(V));
    l1_prefetch(L.rp_id, (int64_t)L.npar * 2);
    l1_prefetch(L.rp_ptr, (int64_t)(L.npar + 1) * 4);
    l1_prefetch(L.rp_child, (int64_t)L.nchild * 2);
  } else {
    l1_prefetch(L.nn_id, (int64_t)L.nnew * 2);
    l1_prefetch(L.nn_p0, (int64_t)L.nnew * 4);
    l1_prefetch(L.nn_p1, (int64_t)L.nnew * 4);
  }
}

}  // namespace kern
}  // namespace asmg
