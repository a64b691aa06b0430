// The solver handle: everything amg_setup keeps on the device.
#pragma once

#include "internal.h"

namespace asmg {

template <class T>
struct SellView {
  const int64_t* off = nullptr;
  const int32_t* col = nullptr;
  const T* val = nullptr;
};

template <class T>
SellView<T> view(const Sell<T>& S) {
  return SellView<T>{S.off.p, S.col.p, S.val.p};
}

// a Sell's stored values, in the arithmetic type or in BF16 (level_bf16)
template <class T>
const T* sell_vals(const Sell<T>& S, const T*) {
  return S.val.p;
}
template <class T>
const bf16v* sell_vals(const Sell<T>& S, const bf16v*) {
  return S.v16.p;
}

// Scalars of the PCG recurrences, device resident.
struct PcgScalars {
  double rz;      // <r_k, z_k>
  double alpha, beta, pq, rr, bnorm, tol;
  int k, maxit, status, cond;
  int timeout;    // set by a kernel whose bounded wait expired (the solve then stops)
};

// Preconditioner data in the precision T of the smoother and V-cycle.
template <class T>
struct Prec {
  Sell<T> Af;                  // fine smoother matrix (mixed mode only; FP64 mode uses A64)
  DBuf<T> dinv_f;
  Sell<T> P, PT;               // Scott-Zhang transfer and its transpose
  std::vector<AuxLevelDev<T>> lev;  // levels c+1..J (index 0 = c+1)
  int n_deep = 0, n_bottom = 0;  // fused small-level runs (top of the hierarchy, bottom)
};

// Per-solve work state in precision T.
template <class T>
struct SlotPrec {
  DBuf<T> uf, rho, F, U;            // fine work vector, fine residual, aux rhs / correction
  std::vector<DBuf<T>> fs, us;      // per level: saved rhs / pre-smoothed values on N~_l
  std::vector<DBuf<double>> nbr, nbs;  // per level: near-boundary rhs / solution pools (mixed boundaries)
  std::vector<DBuf<T>> ust, fsl;    // per level with tiled post-sweeps: start values and saved rhs in tile order
  DBuf<SmallDesc<T>> deep_desc, bot_desc;
};

// Everything one solve writes: several slots let independent right-hand
// sides of one handle run concurrently (batched solves).
struct Slot {
  DBuf<double> b, x, r, p, q;        // permuted, padded
  DBuf<double> vb, vu;               // vertex-ordered staging for user arrays
  DBuf<double> partial, hist;
  DBuf<unsigned int> ticket;
  DBuf<PcgScalars> scal;
  SlotPrec<double> s64;
  SlotPrec<float> s32;
  cudaGraph_t graph = nullptr;       // single-solve graph
  cudaGraphExec_t gexec = nullptr;
  double graph_rtol = -1;
  ~Slot() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
  }
};

// Several right-hand sides of one handle in one solve (the SpMM form): every
// vector holds KRHS columns interleaved, element (i, j) at i * KRHS + j, so
// each matrix entry read serves all columns.  Columns converge on their own:
// a column that has stopped keeps alpha = 0 and takes no further steps.
constexpr int KRHS = 4;

struct MultiScalars {
  double rz[KRHS], alpha[KRHS], beta[KRHS], pq[KRHS], rr[KRHS], bnorm[KRHS], tol[KRHS];
  int k[KRHS], status[KRHS], active[KRHS];
  int maxit, cond, timeout;
};

template <class T>
struct MultiPrec {
  DBuf<T> uf, rho, F, U;                  // [rows][KRHS]
  std::vector<DBuf<T>> fs, us;            // per level [nsm][KRHS]
  DBuf<SmallDesc<T>> deep_desc, bot_desc;
  int n_deep = 0, n_bottom = 0;           // fused small-level runs for KRHS columns
};

struct MultiSlot {
  DBuf<double> b, x, r, p, q;             // [npad][KRHS]
  DBuf<double> vb, vu;                    // [KRHS][nv] vertex order (staging)
  DBuf<double> partial, hist;             // hist [KRHS][max_iter + 1]
  DBuf<unsigned int> ticket;
  DBuf<MultiScalars> scal;
  MultiPrec<double> m64;
  MultiPrec<float> m32;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double graph_rtol = -1;
  ~MultiSlot() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
  }
};

}  // namespace asmg

struct asmg_s {
  asmg_params prm{};
  asmg::MeshHost mesh;
  asmg::DBuf<double> dX, dCoeff;
  asmg::DBuf<int32_t> dE;
  asmg::DBuf<int64_t> d_v2e_ptr;  // elements around each vertex (CSR, ascending element), for the mass product
  asmg::DBuf<int32_t> d_v2e;
  asmg::TreeResult tree;
  asmg::AuxHost aux;

  // fine grid
  int64_t n = 0, npad = 0;
  std::vector<int32_t> free_of_vertex, vertex_of_free, fine_colour, row_of_free;
  std::vector<int64_t> fine_cstart;      // colour blocks in permuted rows (multiples of 32)
  std::vector<int64_t> fine_cnnz, fine_crows;  // real non-zeros / rows per colour block
  asmg::HostCSR A_host;                  // fine A, free-dof numbering (for export)
  asmg::Sell<double> A64;
  asmg::DBuf<double> dinv64;
  asmg::DBuf<int32_t> d_vertex_of_row, d_row_of_vertex, d_free_of_vertex;

  // auxiliary space
  int64_t nJ = 0, nJpad = 0, nc = 0;
  asmg::DBuf<int32_t> d_cid;
  asmg::DBuf<double> d_cinv;             // explicit inverse of the coarsest operator
  std::vector<std::vector<uint64_t>> level_smooth_keys;  // per level: node keys (export)
  std::vector<std::vector<int32_t>> level_smooth_colour;
  std::vector<asmg::Triplets> level_rows;                // per level: assembled rows (export)
  asmg::Prec<double> p64;
  asmg::Prec<float> p32;

  // per-solve state (slot 0 serves amg_solve)
  std::vector<std::unique_ptr<asmg::Slot>> slots;
  // multiple-right-hand-side solves (slot 0 serves amg_solve_multi)
  std::vector<std::unique_ptr<asmg::MultiSlot>> mslots;
  int64_t bytes_iter = 0;
  asmg::Stats stats;
  int gpu_launches_per_iter = 0;

  asmg::Slot& slot0() { return *slots.at(0); }
};

namespace asmg {
// solve.cu
void setup_solve(asmg_s& h, cudaStream_t s);
int profile_solve(asmg_s& h, double rtol, cudaStream_t s, double* out, double* out_levels = nullptr,
                  int nlev_out = 0);
// noalloc.cu
double* noalloc_scratch_for_current_device();
void residual_norm_noalloc(asmg_s& h, const double* b, const double* u, double* out, cudaStream_t s);
int run_solve(asmg_s& h, Slot& S, double rtol, cudaStream_t s);
Slot& add_slot(asmg_s& h, cudaStream_t s);
cudaGraphNode_t capture_solve(asmg_s& h, Slot& S, double rtol, cudaGraph_t g, const cudaGraphNode_t* deps,
                              size_t ndeps);
void precond_apply(asmg_s& h, const double* r_perm, cudaStream_t s);  // result in h.p*.uf
void spmv64(asmg_s& h, const double* x_perm, double* y_perm, cudaStream_t s);
void gather_rows(asmg_s& h, const double* vsrc, double* dst, cudaStream_t s);
void scatter_rows(asmg_s& h, const void* src, bool src_float, double* vdst, cudaStream_t s);
// solve_multi.cu
bool multi_supported(const asmg_s& h);
MultiSlot& add_multi_slot(asmg_s& h, cudaStream_t s);
void gather_multi(asmg_s& h, const double* vsrc, double* dst, cudaStream_t s);
void scatter_multi(asmg_s& h, const double* src, double* vdst, cudaStream_t s);
void run_solve_multi(asmg_s& h, MultiSlot& S, double rtol, cudaStream_t s);
cudaGraphNode_t capture_solve_multi(asmg_s& h, MultiSlot& S, double rtol, cudaGraph_t g, const cudaGraphNode_t* deps,
                                    size_t ndeps);
// assemble.cu
HostCSR assemble_mesh(int dim, int64_t ne, const double* dX, const int32_t* dE, const int32_t* dFree,
                      const double* dCoef, int64_t nfree, cudaStream_t s);
void mass_apply_gpu(int dim, int64_t nv, const int64_t* v2e_ptr, const int32_t* v2e, const double* dX,
                    const int32_t* dE, const double* df, double* db, cudaStream_t s);
void element_grad_gpu(int dim, int64_t ne, const double* dX, const int32_t* dE, const double* du, const double* dl,
                      const double* dscale, double* dg, cudaStream_t s);
}  // namespace asmg
