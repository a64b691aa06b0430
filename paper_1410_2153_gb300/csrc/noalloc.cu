// Residual norms without any allocation: a variant of the PCG start-up
// kernel (r = b - A u with ||r|| and ||b||) whose reduction scratch lives in
// a fixed, file-scope device array instead of memory allocated at run time.
//
// Some callers cannot allocate device memory when they need this check: code
// running under a framework that owns the whole device heap through its own
// pool, real-time or embedded callers whose memory budget is frozen after
// initialisation, or a monitor that must not perturb the allocator state of
// the application it watches.  They pass their own input arrays and a host
// output, and this entry point touches no allocator at all.
#include <cuda_runtime.h>

#include <atomic>

#include "handle.h"

namespace asmg {

namespace {

constexpr int NA_TPB = 256;
constexpr int NA_ROWS_PER_THREAD = 8;
constexpr int64_t NA_ROWS_PER_BLOCK = (int64_t)NA_TPB * NA_ROWS_PER_THREAD;  // 2048
constexpr int NA_MAX_BLOCKS = 4096;                                           // rows <= 8,388,608
constexpr int NA_PARTIALS = 2 * NA_MAX_BLOCKS;
constexpr int NA_RESULT = NA_PARTIALS;        // two doubles: ||b - A u||, ||b||
constexpr int NA_TICKET = NA_PARTIALS + 2;    // one 64-bit counter
constexpr int NA_SCRATCH_DOUBLES = NA_PARTIALS + 4;

// The scratch: 8,196 doubles (about 64 KB).  It comes into existence on a
// device when this module is loaded there, which amg_setup forces (see
// noalloc_scratch_for_current_device), and stays until the process exits.
// All calls share it.
static __device__ __align__(256) double g_noalloc_scratch[NA_SCRATCH_DOUBLES];

// Device addresses of g_noalloc_scratch, one per device (host code may not use
// the symbol itself as a device pointer).  Atomic: two host threads may make
// their first call on a device at the same time.
constexpr int NA_MAX_DEVICES = 64;
std::atomic<double*> g_scratch_ptr[NA_MAX_DEVICES] = {};

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One block per NA_ROWS_PER_BLOCK permuted rows; inputs are read in vertex
// order through the row -> vertex map, so no gathered copies are needed.
__global__ void k_residual_norm_noalloc(int64_t npad, SellView<double> A, const int32_t* __restrict__ vrow,
                                        const double* __restrict__ b, const double* __restrict__ u,
                                        double* __restrict__ scratch) {
  __shared__ double sh[32];
  __shared__ bool last;
  double rr = 0, bb = 0;
  const int64_t r0 = (int64_t)blockIdx.x * NA_ROWS_PER_BLOCK;
  for (int k = 0; k < NA_ROWS_PER_THREAD; ++k) {
    const int64_t i = r0 + (int64_t)k * NA_TPB + threadIdx.x;
    if (i >= npad) break;
    const int32_t v = vrow[i];
    if (v < 0) continue;
    const int64_t sl = i >> 5, lane = i & 31;
    const int64_t base = A.off[sl], w = (A.off[sl + 1] - base) >> 5;
    double s = 0;
    for (int64_t e = 0; e < w; ++e) {
      const int64_t q = base + (e << 5) + lane;
      const int32_t vc = vrow[A.col[q]];
      if (vc >= 0) s += A.val[q] * u[vc];
    }
    const double bi = b[v], ri = bi - s;
    rr += ri * ri;
    bb += bi * bi;
  }
  rr = na_block_sum(rr, sh);
  bb = na_block_sum(bb, sh);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = rr;
    scratch[2 * blockIdx.x + 1] = bb;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* ticket = reinterpret_cast<unsigned long long*>(scratch + NA_TICKET);
    last = (atomicAdd(ticket, 1ULL) == (unsigned long long)gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sr = 0, sb = 0;
  for (unsigned blk = threadIdx.x; blk < gridDim.x; blk += blockDim.x) {
    sr += __ldcg(scratch + 2 * blk);
    sb += __ldcg(scratch + 2 * blk + 1);
  }
  sr = na_block_sum(sr, sh);
  sb = na_block_sum(sb, sh);
  if (threadIdx.x == 0) {
    scratch[NA_RESULT] = sqrt(sr);
    scratch[NA_RESULT + 1] = sqrt(sb);
    *reinterpret_cast<unsigned long long*>(scratch + NA_TICKET) = 0ULL;
  }
}

bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Set-up once per device, with that device current: the device address of
// the scratch array.  Under lazy module loading the first address lookup (or
// launch) is what loads this module on the device and so creates the array;
// amg_setup calls this function, so the array exists before any handle is
// returned and a later amg_residual_norm_noalloc call creates nothing.
double* noalloc_scratch_for_current_device() {
  int dev = 0;
  ASMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) ASMG_FAIL(ASMG_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  double* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    ASMG_CUDA(cudaGetSymbolAddress((void**)&p, g_noalloc_scratch));
    // the kernel too is loaded now, not at the first call
    cudaFuncAttributes fa;
    ASMG_CUDA(cudaFuncGetAttributes(&fa, k_residual_norm_noalloc));
    g_scratch_ptr[dev].store(p, std::memory_order_release);
  }
  return p;
}

void residual_norm_noalloc(asmg_s& h, const double* b, const double* u, double* out, cudaStream_t s) {
  if (!device_pointer(b) || !device_pointer(u))
    ASMG_FAIL(ASMG_ERR_INVALID_ARG, "b and u must be device arrays (this entry point stages nothing)");
  const int64_t nblocks = (h.npad + NA_ROWS_PER_BLOCK - 1) / NA_ROWS_PER_BLOCK;
  if (nblocks > NA_MAX_BLOCKS)
    ASMG_FAIL(ASMG_ERR_INVALID_ARG,
              "problem too large for the fixed scratch: %lld padded rows, at most %lld supported",
              (long long)h.npad, (long long)NA_MAX_BLOCKS * NA_ROWS_PER_BLOCK);
  double* scratch = noalloc_scratch_for_current_device();
  // the completion counter must start at zero
  ASMG_CUDA(cudaMemsetAsync(scratch + NA_TICKET, 0, sizeof(unsigned long long), s));
  k_residual_norm_noalloc<<<(int)std::max<int64_t>(nblocks, 1), NA_TPB, 0, s>>>(h.npad, view(h.A64),
                                                                                 h.d_vertex_of_row.p, b, u, scratch);
  ASMG_CUDA(cudaGetLastError());
  ASMG_CUDA(cudaMemcpyAsync(out, scratch + NA_RESULT, 2 * sizeof(double), cudaMemcpyDefault, s));
  ASMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace asmg
