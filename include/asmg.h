/*
 * asmg.h -- C ABI of the GB300 (sm_103a) auxiliary-space multigrid solver.
 *
 * The library solves the P1 finite-element system A u = b of the problem
 * "find u with a(u, v) = <f, v> for all v" (Sec. 2, eq. bilinearform) by
 * conjugate gradients preconditioned with the multiplicative auxiliary-space
 * preconditioner of Algorithm 1: a Gauss-Seidel smoother on the given grid
 * plus a geometric V-cycle (Algorithm 2) on the nested auxiliary grids built
 * from the cluster tree of element barycenters (Sec. 3).
 *
 * Conventions for every entry point:
 *   - Return value: ASMG_OK (0) on success, > 0 for a warning, < 0 for an
 *     error.  On error, amg_last_error() returns a message for the calling
 *     thread; no output is partially written unless stated.
 *   - Arrays may be host or device (CUDA) pointers unless stated; the
 *     library detects which with cudaPointerGetAttributes and stages host
 *     arrays through device memory.  Arrays are caller-owned and need only
 *     stay valid for the duration of the call.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     enqueue their device work on it and synchronise it before returning.
 *   - Indices are 0-based.  Vertex arrays are indexed by vertex number.
 *   - The handle owns all device memory it allocates; amg_destroy frees it.
 *     A handle may be used from one host thread at a time.
 *   - Every reduction on the device (dot products, norms, the mass product)
 *     runs in a fixed order: with the same inputs and parameters every
 *     result is the same bit for bit from run to run, so no separate
 *     "deterministic" mode exists.
 */
#ifndef ASMG_H
#define ASMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct asmg_s* asmg_handle;

enum asmg_status {
  ASMG_OK = 0,
  ASMG_NOT_CONVERGED = 1,     /* max_iter reached; u holds the last iterate */
  ASMG_ERR_INVALID_ARG = -1,  /* null pointer, bad size or bad parameter */
  ASMG_ERR_BAD_MESH = -2,     /* index out of range, non-positive measure, bad flag or coefficient */
  ASMG_ERR_UNSUPPORTED = -3,  /* dim not supported, or a colouring beyond 128 colours */
  ASMG_ERR_BREAKDOWN = -4,    /* <p, A p> <= 0 or NaN, or <r, z> <= 0 in PCG */
  ASMG_ERR_CUDA = -5,         /* a CUDA runtime call failed */
  ASMG_ERR_OOM = -6,          /* device allocation failed */
  ASMG_ERR_TIMEOUT = -7       /* a bounded device wait expired: a tiled sweep's shared-memory copy did
                                 not complete within about a second; the solve stops, u holds the last
                                 iterate, and the context stays usable */
};

enum asmg_precision { ASMG_FP64 = 0, ASMG_MIXED = 1 };

typedef struct {
  int32_t n_min;           /* cluster size below which a box is not split; 3 (Sec. 3.1) */
  int32_t nu_pre;          /* pre-smoothing sweeps per auxiliary level; 2 (Sec. 5.1) */
  int32_t nu_post;         /* post-smoothing sweeps per auxiliary level; 2 */
  int32_t coarse_max_dofs; /* the V-cycle stops at the finest level with at most this many dofs,
                              solved exactly (B_0 = A_0^{-1}, Algorithm 2); 512 */
  int32_t precision;       /* ASMG_FP64: everything in FP64.  ASMG_MIXED: smoother, transfers and
                              V-cycle in FP32 inside the FP64 CG (coarse solve, dots and residual
                              recurrence stay FP64) */
  int32_t max_iter;        /* PCG iteration cap; 500 */
  int32_t smoothing;       /* 0: smooth the new/changed nodes N~_l of each level (Sec. 4.2, eq.
                              decomposition); 1: smooth every node of every level */
  int32_t use_graph;       /* 1: run the PCG loop as one CUDA graph with a device-side WHILE node */
  int32_t use_pdl;         /* 1: launch solve kernels with programmatic dependent launch */
  int32_t smoother;        /* fine smoother S (Sec. 4.1): 0 Gauss-Seidel (D - L)^{-1}, multicolour;
                              1 Jacobi D^{-1}; 0 */
  int32_t additive;        /* 0: multiplicative B of Algorithm 1; 1: additive B = S + Pi Btilde Pi^t
                              (eq. fasp), for use with PCG; 0 */
  int32_t fine_sweeps;     /* smoothing steps per application of S and of S^t, 1..8; 1 */
  int32_t iteration;       /* 0: PCG (Sec. 5.2); 1: the ASMG iteration u <- u + B (b - A u) (Sec. 5.1
                              rates), meaningful with the multiplicative B; 0 */
  int32_t tile_rows;       /* schedule of the auxiliary-level sweeps (results are the same bit for
                              bit): 0 = default, > 0 = own rows per tile (32..65536) of the temporally
                              blocked sweeps (every sweep of a level in one launch, one thread block
                              per tile), -1 = one launch per colour class and sweep; 0 */
  int32_t inject_timeout;  /* failure injection (testing): 1 = every tiled sweep takes the path of an
                              expired bounded wait (it still waits for its shared-memory copy, skips
                              its work and records the timeout), so solves and amg_precond_apply
                              return ASMG_ERR_TIMEOUT; 0 */
  int32_t nb_layers;       /* mixed boundaries: layers j of the near-boundary sets J_{l,j} of Algorithm 3
                              (Sec. 3.5), whose exact solve follows each coarse-grid correction;
                              -1 = no near-boundary correction, 0..16; 2 */
  int32_t colouring;       /* colour classes of the Gauss-Seidel sweeps: 0 = Jones-Plassmann with
                              splitmix64 priorities on every grid; 2 = on an auxiliary level whose
                              couplings the lattice parity (X + Y [+ Z]) / h_l mod 2 separates (uniform
                              levels), that parity (two classes), else Jones-Plassmann; 2 */
  int32_t level_bf16;      /* ASMG_MIXED only: 1 = the V-cycle reads the auxiliary-level matrices A_l
                              (sweeps and residuals) in BF16, each value the FP32 value rounded to
                              nearest even (arithmetic, diagonal inverses and vectors stay FP32);
                              0 = FP32.  A precision choice, not the paper's: the preconditioner
                              changes, the solve still stops at rtol on the FP64 residual; 0 */
} asmg_params;

/* Fill *p with the defaults listed above.  Returns ASMG_ERR_INVALID_ARG if p is NULL. */
int asmg_default_params(asmg_params* p);

/*
 * Build the solver for one mesh (Sec. 2-4).
 *   dim        2 (triangles; quadtree, triangular auxiliary grids) or 3
 *              (tetrahedra; octree, Kuhn and coned tetrahedral auxiliary
 *              grids on the 2^(J+1) lattice of the root cube, Sec. 3 in 3D).
 *              Other values return ASMG_ERR_UNSUPPORTED.
 *   nv, vertices   float64 [nv * dim], row-major coordinates.
 *   ne, elements   int32 [ne * (dim + 1)], vertex indices of each simplex,
 *                  positively oriented (counter-clockwise triangles;
 *                  tetrahedra with (p1-p0).((p2-p0)x(p3-p0)) > 0).
 *   boundary   uint8 [nv]: 0 free vertex, 1 Dirichlet vertex (u = 0), 2
 *              Neumann vertex (a boundary vertex that is an unknown: the
 *              natural condition).  With any Neumann vertex the auxiliary
 *              grids are the mixed grids of the remark in Sec. 3.4 (the
 *              simplices that meet the domain and not the Dirichlet boundary
 *              Gamma_D, Gamma_D being the boundary facets whose vertices are
 *              all Dirichlet), every level is smoothed as a whole, and the
 *              V-cycle adds the near-boundary correction of Algorithm 3 (an
 *              exact solve on J_{l,j}, see nb_layers).
 *   coeff      float64 [ne] per-element coefficient a_e > 0, or NULL for a = 1.
 *   params     NULL for the defaults.
 *   out        receives the handle (NULL on error).
 * The domain may be any polygon (polyhedron) inside the square (cube)
 * spanned by the vertices' bounding box (the root box of Sec. 3.1).  When the
 * element measures do not add up to that box (within 1e-12 relative), the
 * auxiliary grids are the Dirichlet grids of Sec. 3.4: the auxiliary
 * triangles (tetrahedra) the elements cover, with zero values on the
 * boundary of their union.  Inputs are
 * validated before any other work (ASMG_ERR_BAD_MESH).  The call copies what
 * it keeps: the caller may free every input afterwards.
 */
int amg_setup(int dim, int64_t nv, const double* vertices, int64_t ne, const int32_t* elements,
              const uint8_t* boundary, const double* coeff, const asmg_params* params, void* stream,
              asmg_handle* out);

/*
 * PCG solve of A u = b (Sec. 5.2) with the preconditioner of Algorithm 1.
 *   b            float64 [nv] assembled load vector; entries at Dirichlet
 *                vertices are ignored (see amg_mass_apply).
 *   u            float64 [nv]: in = initial guess, out = solution (0 at
 *                Dirichlet vertices).
 *   rtol         stop when ||r_k||_2 <= rtol * ||b||_2 (free entries).
 *   iterations   host int: PCG steps taken.
 *   res_history  host float64 [max_iter + 1] or NULL: ||r_k||_2, k = 0..iterations.
 * Returns ASMG_OK, ASMG_NOT_CONVERGED (u = last iterate, history filled) or
 * ASMG_ERR_BREAKDOWN.  Host or device b/u are accepted; a host call times the
 * copies inside the solve.
 */
int amg_solve(asmg_handle h, const double* b, double* u, double rtol, int* iterations, double* res_history,
              void* stream);

/*
 * k (1..4) right-hand sides of one handle solved together (not in the paper):
 * the PCG of amg_solve on k columns at once.  Vectors are kept with their
 * columns interleaved, so every matrix entry the solve reads (fine operator,
 * transfer, level operators) serves all k columns (the SpMM form).  Each
 * column has its own scalars and its own stopping test; a column that has
 * stopped takes no further steps.  Per column the arithmetic is that of
 * amg_solve, except on small auxiliary levels whose fused kernels hold fewer
 * rows here.
 *   b            float64 [k * nv]: right-hand side c at b + c * nv.
 *   u            float64 [k * nv]: initial guesses in, solutions out.
 *   iterations   host int [k]; status host int [k] or NULL (ASMG_OK,
 *                ASMG_NOT_CONVERGED, ASMG_ERR_BREAKDOWN per column).
 *   res_history  host float64 [k * (max_iter + 1)] or NULL: column c's
 *                residual norms at res_history + c * (max_iter + 1).
 * Returns the worst column status.  ASMG_ERR_UNSUPPORTED for handles with
 * Neumann vertices or with the Jacobi, additive or iteration variants.
 */
int amg_solve_multi(asmg_handle h, int k, const double* b, double* u, double rtol, int* iterations, int* status,
                    double* res_history, void* stream);

/*
 * b = M f_h: the consistent P1 mass matrix applied to nodal values f [nv]
 * (float64), result b [nv] with 0 at Dirichlet vertices.  This is the load
 * vector <f, phi_i> of eq. bilinearform for the interpolant f_h.  Each entry
 * is gathered over the elements around its vertex in ascending element order
 * (no atomics), so the result is the same bit for bit on every run.  The
 * first call builds that vertex-to-element list (device memory owned by the
 * handle).
 */
int amg_mass_apply(asmg_handle h, const double* f_nodal, double* b, void* stream);

/*
 * z = B_co r: one application of the preconditioner of Algorithm 1 (smooth,
 * auxiliary correction through the Scott-Zhang transfer of Sec. 4.1, smooth
 * back), r and z float64 [nv] (Dirichlet entries ignored / set to 0).
 */
int amg_precond_apply(asmg_handle h, const double* r, double* z, void* stream);

/*
 * y = A x with the fine stiffness matrix a_ij = int a grad phi_i . grad phi_j
 * (Sec. 2); x, y float64 [nv], Dirichlet entries ignored / set to 0.
 */
int amg_spmv(asmg_handle h, const double* x, double* y, void* stream);

/*
 * Sensitivity of L(u(a)) to the element coefficients: with u the solution and
 * lambda the adjoint solution (A lambda = dL/du), both float64 [nv],
 *   dL_dcoeff[e] = -lambda_e^T K_e^(1) u_e,
 * K_e^(1) the element stiffness for a_e = 1 (not in the paper).
 */
int amg_element_grad(asmg_handle h, const double* u, const double* lambda, double* dL_dcoeff, void* stream);

/*
 * The same sensitivity with respect to log-coefficients: for a = exp(g) (see
 * amg_set_log_coefficients), dL_dg[e] = a_e dL/da_e = -a_e lambda_e^T K_e^(1) u_e,
 * with a_e the handle's current coefficient (1 when none was given).  The
 * chain-rule factor is applied in the same kernel (not in the paper).
 */
int amg_element_grad_log(asmg_handle h, const double* u, const double* lambda, double* dL_dg, void* stream);

/*
 * Set the element coefficients to a_e = exp(g_e), g float64 [ne] finite, and
 * rebuild as amg_update_coefficients does (the log-parametrisation of a
 * coefficient field; not in the paper).
 */
int amg_set_log_coefficients(asmg_handle h, const double* g, void* stream);

/*
 * Replace the element coefficients (float64 [ne], > 0) and rebuild every
 * operator that depends on them (fine A, auxiliary operators, coarse
 * inverse).  The tree, the auxiliary grids, the transfer and the colourings
 * depend on geometry only and are kept.
 */
int amg_update_coefficients(asmg_handle h, const double* coeff, void* stream);

/*
 * The cluster tree alone (Sec. 3.1) for a 2D (triangles) or 3D (tetrahedra)
 * mesh: Morton keys of the quantised element barycenters (D = 31 bits per
 * coordinate in 2D, 21 in 3D) and the elements sorted by key (stable).
 *   keys  uint64 [ne] (element order), perm int32 [ne]; host or device.
 * Index range and orientation are checked (ASMG_ERR_BAD_MESH).
 */
int amg_cluster_tree(int dim, int64_t nv, const double* vertices, int64_t ne, const int32_t* elements, uint64_t* keys,
                     int32_t* perm, void* stream);

/* Integer facts about a handle (see enum asmg_info_what); *value receives it. */
enum asmg_info_what {
  ASMG_INFO_NFREE = 0,        /* free fine dofs n */
  ASMG_INFO_J = 1,            /* finest auxiliary level (tree depth) */
  ASMG_INFO_COARSE = 2,       /* coarsest level used by the V-cycle */
  ASMG_INFO_NAUX = 3,         /* free nodes of auxiliary level `level` */
  ASMG_INFO_NSMOOTH = 4,      /* smoothed nodes of level `level` (-1: fine grid) */
  ASMG_INFO_NCOLOURS = 5,     /* colours of level `level` (-1: fine grid) */
  ASMG_INFO_NTREE_LEVELS = 6, /* depths of the cluster tree */
  ASMG_INFO_NSEG = 7,         /* cluster-tree nodes at depth `level` */
  ASMG_INFO_NSPLIT = 8,       /* split boxes of the closed tree at depth `level` */
  ASMG_INFO_NNZ_A = 9,        /* stored non-zeros of the fine matrix */
  ASMG_INFO_NNZ_P = 10,       /* non-zeros of the transfer P */
  ASMG_INFO_NROWS_E = 11,     /* residual rows of level `level` */
  ASMG_INFO_BYTES_ITER = 12,  /* algorithmic bytes of one PCG iteration (current precision) */
  ASMG_INFO_NNZ_LEVEL = 13,   /* stored non-zeros of level `level` (smoothing + residual rows) */
  ASMG_INFO_NTILES = 14,      /* tiles of the temporally blocked pre-sweeps of level `level` (0: one
                                 launch per colour class and sweep) */
  ASMG_INFO_HALO_ROWS = 15,   /* halo rows of those tiles (pre-sweeps), summed over the tiles */
  ASMG_INFO_NTILES_UP = 16    /* tiles of the temporally blocked post-sweeps of level `level` (0: per class) */
};
int amg_info(asmg_handle h, int what, int level, int64_t* value);

/*
 * Copy internal setup data to a host buffer for testing (see enum
 * asmg_export_what).  With host_buf = NULL only *count (elements of the
 * stated type) is returned.
 */
enum asmg_export_what {
  ASMG_EXPORT_KEYS = 0,        /* uint64 [ne] element Morton keys */
  ASMG_EXPORT_PERM = 1,        /* int32 [ne] elements sorted by key (stable) */
  ASMG_EXPORT_SEG = 2,         /* int64 [nseg(level) * 4]: prefix, begin, end, split */
  ASMG_EXPORT_SPLIT = 3,       /* uint64 [nsplit(level)] Morton prefixes of split boxes, ascending */
  ASMG_EXPORT_AUX_KEYS = 4,    /* uint64 [naux(J)] lattice Morton keys of the finest-level free nodes
                                  (2D: 2^31 lattice; 3D: 2^(J+1) lattice, 21 bits per coordinate) */
  ASMG_EXPORT_FINE_COLOUR = 5, /* int32 [nfree] colour of each free dof (free dofs in vertex order) */
  ASMG_EXPORT_SMOOTH = 6,      /* uint64 [nsmooth(level) * 2]: node key, colour */
  ASMG_EXPORT_LEVEL_ROWS = 7,  /* (row key, col key, value) triplets of level `level`, as
                                  uint64, uint64, float64 (count = triplets; buffer 24 bytes each) */
  ASMG_EXPORT_P = 8,           /* (fine vertex, aux key, value) triplets of P, 24 bytes each */
  ASMG_EXPORT_FINE_A = 9       /* (row vertex, col vertex, value) triplets of A, 24 bytes each */
};
int amg_export(asmg_handle h, int what, int level, void* host_buf, int64_t* count);

/*
 * Profile one solve (tracing; not part of the paper): the solve of amg_solve
 * from u = 0 is run without the CUDA graph and every kernel launch is timed
 * with CUDA events on `stream`.  out: host float64 [3 * ASMG_PROF_NCLASS],
 * per kernel class (enum asmg_prof_class) the number of launches, their total
 * time in milliseconds and their algorithmic bytes (compulsory traffic of the
 * real rows and non-zeros each launch touches).  b: float64 [nv] as in
 * amg_solve.  The solution is discarded.
 */
enum asmg_prof_class {
  ASMG_PROF_FINE_GS = 0,      /* fine-grid Gauss-Seidel colour sweeps (Algorithm 1, steps 1 and 3) */
  ASMG_PROF_FINE_RESID = 1,   /* fine residual r - A u1 */
  ASMG_PROF_RESTRICT = 2,     /* P^T: fine residual to the finest auxiliary level */
  ASMG_PROF_PROLONG = 3,      /* P: auxiliary correction to the fine grid */
  ASMG_PROF_AUX_GS = 4,       /* auxiliary-level Gauss-Seidel sweeps (Algorithm 2) */
  ASMG_PROF_AUX_RESID = 5,    /* auxiliary-level residuals */
  ASMG_PROF_AUX_TRANSFER = 6, /* auxiliary restriction / prolongation / bookkeeping */
  ASMG_PROF_COARSE = 7,       /* coarsest-level solve */
  ASMG_PROF_CG_SPMV = 8,      /* PCG q = A p with <p, q> (FP64) */
  ASMG_PROF_CG_VECTOR = 9,    /* PCG vector updates and reductions */
  ASMG_PROF_AUX_SMALL = 10,   /* runs of small auxiliary levels fused into one thread block */
  ASMG_PROF_AUX_NB = 11,      /* near-boundary residual and exact solve (Algorithm 3, mixed boundaries) */
  ASMG_PROF_NCLASS = 12
};
int amg_profile(asmg_handle h, const double* b, double rtol, double* out, int* iterations, void* stream);

/*
 * amg_profile plus a split by auxiliary level (tracing; not part of the
 * paper).  out as for amg_profile; out_levels: host float64
 * [nlev * 2 * 3 * 3], for each level index k = l - (coarsest + 1) below nlev,
 * each direction (0 down, 1 up), each part (0 sweeps, 1 residual, 2 transfer
 * and bookkeeping): launches, milliseconds, algorithmic bytes.  Levels that
 * run inside the fused small-level kernels are counted under
 * ASMG_PROF_AUX_SMALL only.
 */
int amg_profile_levels(asmg_handle h, const double* b, double rtol, double* out, double* out_levels, int nlev,
                       int* iterations, void* stream);

/*
 * Batched solves (not in the paper): many independent problems, each with
 * several right-hand sides, solved by one CUDA graph launch.
 *   amg_batch_create  nprob handles (distinct meshes, any precisions), nrhs
 *                     right-hand sides per handle, the relative tolerance.
 *                     With nrhs > 1 (and handles amg_solve_multi accepts)
 *                     the right-hand sides of a problem are solved in groups
 *                     of 4 columns as by amg_solve_multi, so each matrix read
 *                     serves 4 right-hand sides; the batch captures one graph
 *                     in which every (problem, group) solve -- gather, PCG
 *                     start, WHILE loop, scatter -- is an independent branch,
 *                     so the device runs the solves of all problems
 *                     concurrently.  Otherwise every (problem, rhs) solve is
 *                     a branch of its own.  Handles must outlive the batch
 *                     and may not be destroyed before it.
 *   amg_batch_solve   bs[p * nrhs + j]: float64 [nv_p] right-hand side j of
 *                     problem p; us[...]: initial guess in, solution out (host
 *                     or device arrays).  iterations, status: host int
 *                     [nprob * nrhs], the PCG steps and the per-solve status
 *                     (ASMG_OK, ASMG_NOT_CONVERGED, ASMG_ERR_BREAKDOWN).
 *                     Returns the worst status.
 */
typedef struct asmg_batch_s* asmg_batch;
int amg_batch_create(int nprob, const asmg_handle* handles, int nrhs, double rtol, void* stream, asmg_batch* out);
int amg_batch_solve(asmg_batch batch, const double* const* bs, double* const* us, int* iterations, int* status,
                    void* stream);
void amg_batch_destroy(asmg_batch batch);

/*
 * ||b - A u||_2 and ||b||_2 over the free dofs, allocating nothing.  The
 * paper has no counterpart: this is a service entry point for callers that
 * cannot allocate device memory when they need the check -- code whose
 * device heap is owned by another framework's pool, real-time or embedded
 * callers whose memory budget is frozen after initialisation, or monitors
 * that must not disturb the allocator of the application they observe.
 *   b, u   DEVICE float64 [nv] arrays in vertex order.  Host arrays are
 *          rejected (ASMG_ERR_INVALID_ARG): staging them would need memory.
 *          Entries at Dirichlet vertices are ignored.
 *   out    float64 [2], host or device: ||b - A u||_2 and ||b||_2.
 * Scratch: one fixed 64 KB array inside the library (a static device array).
 * It is created on a device when amg_setup first runs there: amg_setup loads
 * the library module that holds it and looks up its device address, so under
 * lazy module loading too the memory appears at setup, never during a call
 * of this function.  It then stays until the process exits.  All calls on a
 * device share it and it keeps the last call's contents; calls that overlap
 * on the GPU (e.g. from two streams) race on it.  A call made while a device
 * other than the handle's is current would look the address up itself; make
 * every call with the handle's device current.  Meshes with more than
 * 8,388,608 padded fine rows are rejected with ASMG_ERR_INVALID_ARG.  No
 * cudaMalloc, cudaFree or other allocating routine is called.
 */
int amg_residual_norm_noalloc(asmg_handle h, const double* b, const double* u, double* out, void* stream);

/* Free the handle and all device memory it owns.  NULL is ignored. */
void amg_destroy(asmg_handle h);

/* Message of the last error on the calling thread ("" if none). */
const char* amg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ASMG_H */
