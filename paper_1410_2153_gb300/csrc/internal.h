// Internal declarations shared by the translation units of libasmg.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/asmg.h"
#include "nbsolve.h"

namespace asmg {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);

struct Error {
  int code;
  std::string msg;
};

#define ASMG_CUDA(call)                                                                          \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      throw ::asmg::Error{e_ == cudaErrorMemoryAllocation ? ASMG_ERR_OOM : ASMG_ERR_CUDA,        \
                          std::string(#call) + ": " + cudaGetErrorString(e_)};                   \
  } while (0)

#define ASMG_FAIL(code, ...)                                                                     \
  do {                                                                                           \
    char b_[512];                                                                                \
    snprintf(b_, sizeof b_, __VA_ARGS__);                                                        \
    throw ::asmg::Error{code, b_};                                                               \
  } while (0)

// ------------------------------------------------------- device buffers
template <class T>
struct DBuf {
  T* p = nullptr;
  int64_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(int64_t count) {
    release();
    n = count;
    if (count > 0) ASMG_CUDA(cudaMalloc((void**)&p, sizeof(T) * (size_t)count));
  }
  void zero(cudaStream_t s) {
    if (n) ASMG_CUDA(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n, s));
  }
  void upload(const std::vector<T>& h, cudaStream_t s) {
    alloc((int64_t)h.size());
    if (n) ASMG_CUDA(cudaMemcpyAsync(p, h.data(), sizeof(T) * (size_t)n, cudaMemcpyHostToDevice, s));
  }
  std::vector<T> download(cudaStream_t s) const {
    std::vector<T> h((size_t)n);
    if (n) ASMG_CUDA(cudaMemcpyAsync(h.data(), p, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, s));
    ASMG_CUDA(cudaStreamSynchronize(s));
    return h;
  }
  size_t bytes() const { return sizeof(T) * (size_t)n; }
};

// ---------------------------------------------------- host sparse rows
struct Triplets {  // row, col, value (host)
  std::vector<int32_t> r, c;
  std::vector<double> v;
};

struct HostCSR {
  int64_t nr = 0, nc = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

// SELL-32: rows in slices of 32; element k of row (32 s + t) at
// off[s] + 32 k + t.  Padding entries have col = pad_col, val = 0.
constexpr int SELL_C = 32;

// An auxiliary-level matrix value stored in BF16 (asmg_params::level_bf16):
// the upper 16 bits of its FP32 value rounded to nearest even, which widen
// back to FP32 exactly.
struct bf16v {
  uint16_t bits;
};

// FP32 -> BF16 bits, round to nearest even (finite values): adding 0x7FFF plus
// the lowest kept bit carries into the kept half exactly when the dropped half
// is above one half ulp, or equal to it with an odd kept half.
inline __host__ __device__ uint16_t bf16_bits(float f) {
  uint32_t u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(f);
#else
  std::memcpy(&u, &f, 4);
#endif
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

template <class T>
struct Sell {
  int64_t nrows = 0;   // multiple of 32
  int64_t nslices = 0;
  int64_t nnz = 0;     // stored (padded) entries
  int64_t nnz_real = 0;
  DBuf<int64_t> off;   // [nslices + 1]
  DBuf<int32_t> col;   // [nnz]
  DBuf<T> val;         // [nnz]
  DBuf<bf16v> v16;     // [nnz] the values in BF16 (auxiliary levels with level_bf16), else empty
};

// Build SELL-32 from host rows given as CSR in the SELL row order
// (row k of `rows` is SELL row k; rows.nr need not be a multiple of 32).
template <class T>
void sell_build(Sell<T>& S, const HostCSR& rows, int32_t pad_col, cudaStream_t s);

// Fill S.v16 with the BF16 form (bf16_bits) of S.val, on the device.
void sell_bf16(Sell<float>& S, cudaStream_t s);

// --------------------------------------------------------------- tree
struct TreeResult {
  double amin[3] = {0, 0, 0};
  double L = 0;
  int D = 31;
  std::vector<std::vector<int64_t>> seg;       // per depth: prefix, begin, end, split (4 per node)
  std::vector<std::vector<uint64_t>> split;    // per depth: sorted prefixes of split nodes
  DBuf<uint64_t> keys;                         // element keys (element order)
  DBuf<int32_t> perm;                          // elements sorted by key
};

// --------------------------------------------------------- aux hierarchy
// One auxiliary level above the coarsest (host description, aux node IDs
// index the free nodes of the finest level in lattice Morton order).
struct AuxLevelHost {
  int level = 0;
  std::vector<int32_t> smooth;            // N~_l, ascending aux ID
  std::vector<int32_t> new_id, new_p0, new_p1;  // new nodes and their parents (-1 = Dirichlet)
  // assembly input: triangles (aux IDs, -1 = Dirichlet) with lattice corners
  std::vector<int32_t> tri_id;            // [ntri * 3]
  std::vector<uint64_t> tri_key;          // [ntri * 3] lattice Morton keys
  std::vector<double> tri_coef;           // [ntri]
  // mixed boundaries: the near-boundary set J_{l,j} of Algorithm 3 (aux IDs,
  // ascending); empty otherwise
  std::vector<int32_t> nb_id;
  // mixed boundaries: A_l restricted to J_{l,j} (CSR over the positions in
  // nb_id) and its block cyclic reduction factor
  std::vector<int64_t> nb_ptr;
  std::vector<int32_t> nb_col;
  std::vector<double> nb_val;
  nb::Factor nb_fac;
};

// What the device Scott-Zhang kernel needs of the closed tree and the finest
// auxiliary grid: the boxes of every depth (ascending prefix within a depth,
// depths one after another) with, per box, the node index of its first child
// (children are consecutive) or -(leaf + 1); per leaf its finest simplices
// as lattice keys and the aux ID of every vertex (-1: no hat function there,
// i.e. a Dirichlet node, or a simplex outside Omega^D_J).
struct SZTable {
  int dim = 2;
  int D = 31;                     // lattice bits of a coordinate
  double amin[3] = {0, 0, 0}, L = 1;
  std::vector<uint64_t> node_key;
  std::vector<int64_t> node_pay;
  std::vector<int64_t> leaf_first;  // simplices of leaf q: [leaf_first[q], leaf_first[q + 1])
  std::vector<uint64_t> simp_key;   // dim + 1 keys per simplex
  std::vector<int32_t> simp_col;    // dim + 1 aux IDs per simplex
};

struct AuxHost {
  int J = 0, c = 0;
  int LB = 0;                                  // 3D: lattice bits of the node keys (J + 1)
  std::vector<std::vector<uint64_t>> split;   // closed tree: split prefixes per depth (sorted)
  std::vector<uint64_t> aux_key;               // free finest-level nodes, ascending key
  std::vector<int64_t> nlevel;                 // free nodes per level 0..J
  std::vector<AuxLevelHost> levels;            // levels c+1..J
  std::vector<int32_t> coarse_id;              // free nodes of level c (aux IDs)
  std::vector<int32_t> coarse_tri_id;          // triangles of level c
  std::vector<uint64_t> coarse_tri_key;
  std::vector<double> coarse_tri_coef;
  Triplets P;                                  // (free fine dof, aux ID, value)
  SZTable sz;                                  // input of the device transfer build
  // mixed boundaries: aux ID q is a free node of the levels phi[q] <= l <
  // psi[q] (free on one interval of levels); empty otherwise
  std::vector<int32_t> phi, psi;
};

struct MeshHost {
  int dim = 2;
  int64_t nv = 0, ne = 0;
  std::vector<double> X;
  std::vector<int32_t> E;
  std::vector<uint8_t> bflag;
  std::vector<double> coeff;  // empty: a = 1
  bool boxdomain = true;      // the elements fill the root box (else Dirichlet auxiliary grids, 2D)
  bool mixed = false;         // some vertex is Neumann (flag 2): mixed auxiliary grids (2D)
  int nb_layers = 2;          // mixed: layers j of the near-boundary sets (< 0: none)
};

// closure of the cluster tree, auxiliary grids and the Scott-Zhang transfer
void build_aux_host(const MeshHost& mesh, const TreeResult& tree, const asmg_params& prm, AuxHost& out);

// the same in 3D (octree, Kuhn / coned tetrahedral grids); tri_* arrays of
// the levels then hold 4 keys / ids per tetrahedron
void build_aux_host3(const MeshHost& mesh, const TreeResult& tree, const asmg_params& prm, AuxHost& out);

// Scott-Zhang transfer (transfer.cu, Sec. 4.1) from the table the host setup
// leaves in AuxHost::sz: P (rows: free fine dofs in free order, columns: aux
// IDs) as host triplets.  2D rows are computed on the device, 3D rows on host
// threads (the same row code).
void build_transfer(const MeshHost& mesh, const double* dX, const int32_t* dE,
                        const std::vector<int32_t>& vertex_of_free, const SZTable& tab, Triplets& P, cudaStream_t s);

// physical coordinate of a lattice key (2D: 2^D lattice; 3D: 2^LB lattice)
void lattice_point(const TreeResult& t, uint64_t key, double* p);
void lattice_point3(const TreeResult& t, int LB, uint64_t key, double* p);
uint64_t lattice_key2(uint64_t x, uint64_t y);
void lattice_xy2(uint64_t key, uint64_t& x, uint64_t& y);

// ----------------------------------------------------------------- GPU setup
void build_tree_gpu(int dim, int64_t nv, const double* dX, int64_t ne, const int32_t* dE, int n_min,
                    cudaStream_t s, TreeResult& out);

// Assemble sum of element matrices into CSR on the device and download.
//   simplices (triangles, dim 2; tetrahedra, dim 3) given by vertex
//   coordinates (dP [(dim+1)*n*dim]) and row/col ids (dID [(dim+1)*n], < 0
//   dropped), coefficient per simplex; entries are kept only where
//   keep(row) || keep(col) (keep == nullptr keeps all).
HostCSR assemble_simplices(int dim, int64_t n, const double* dP, const int32_t* dID, const double* dCoef,
                           const uint8_t* dKeep, int64_t nrows, cudaStream_t s);

// Jones-Plassmann colouring of the rows in `set` (CSR adjacency over all rows,
// priorities splitmix64(key)); returns colour per row (-1 outside the set).
std::vector<int32_t> jp_colour_gpu(const HostCSR& A, const std::vector<uint8_t>& inset,
                                   const std::vector<uint64_t>& prio_key, cudaStream_t s);

// A level small enough to run inside one thread block with its rhs and
// correction in shared memory (see k_small_down / k_small_up).  Local node
// k < mS is the k-th smoothing node (colour order); mS <= k < mE are the other
// nodes of the rows E_l.  Column indices are local (16 bit).
constexpr int SMALL_LMAX = 8192;
constexpr int SMALL_MAXC = 24;
template <class T>
struct SmallDesc {
  int mS, mE, ncol, nnew, npar;
  int nnz_sm, nnz_rs, nchild;  // entries of the smoothing / residual rows, children of the restriction
  int cs[SMALL_MAXC + 1];
  const int32_t* gid;
  const int32_t* sm_ptr;
  const uint16_t* sm_col;
  const T* sm_val;
  const bf16v* sm_v16;  // the same values in BF16 (level_bf16), else null
  const T* dinv;
  const int32_t* rs_ptr;
  const uint16_t* rs_col;
  const T* rs_val;
  const bf16v* rs_v16;
  const uint16_t* nn_id;
  const int32_t* nn_p0;
  const int32_t* nn_p1;
  const uint16_t* rp_id;
  const int32_t* rp_ptr;
  const uint16_t* rp_child;
  T* fs;
  T* us;
};

template <class T>
struct SmallLevelDev {
  bool ok = false;  // level fits the small-level kernels
  int mS = 0, mE = 0, ncol = 0, nnew = 0, npar = 0;
  int64_t nnz_sm = 0, nnz_rs = 0, nchild = 0;
  std::vector<int> cs;
  DBuf<int32_t> gid, sm_ptr, rs_ptr, nn_p0, nn_p1, rp_ptr;
  DBuf<uint16_t> sm_col, rs_col, nn_id, rp_id, rp_child;
  DBuf<T> sm_val, dinv, rs_val;
  DBuf<bf16v> sm_v16, rs_v16;  // level_bf16: sm_val / rs_val in BF16
};

// Temporal blocking of the sweeps of one auxiliary level (Algorithm 2's
// nu pre- or post-smoothing steps over all colour classes in one launch):
// the smoothing rows N~_l are cut into tiles of consecutive aux IDs (lattice
// Morton order, so a tile is a compact patch); each tile carries the halo
// rows whose values its sweeps read, found by a closure over (row, sweep)
// dependencies, so one thread block can run every sweep of its tile in
// shared memory and write back only the tile's own rows.  The results equal
// the class-by-class launches bit for bit (see build_tiles).
//
// A tile's rows are stored as one block of bytes (16-byte aligned, a multiple
// of 16 bytes long; layout in TileLayout) that the kernel copies into shared
// memory with one bulk copy: SELL-32 slice offsets (int32, relative to the
// tile), the column of every entry (uint16: a local row, or nl + e for the
// tile's e-th outside value), the values (T), then per local row its
// diagonal inverse (T), SM row (int32: own row k, halo row -2 - k, padding
// -1) and aux ID (int32), then the outside values' aux IDs.  Outside values
// are the columns outside N~_l of the post-sweeps' rows: the sweeps do not
// change them, so the tile reads them from U once.
// dynamic shared memory a tile launch may use (bytes)
constexpr size_t TILE_SMEM_LIMIT = 200 * 1024;

struct TileLayout {
  int64_t col, val, dinv, lsm, laux, ext, end;  // byte offsets of the parts, and the total
};

// nl local rows (a multiple of 32), ne stored entries, nx outside values, s bytes per value
// (diagonal inverses), sv bytes per stored matrix value
inline __host__ __device__ TileLayout tile_layout(int64_t nl, int64_t ne, int64_t nx, int64_t s, int64_t sv) {
  auto pad16 = [](int64_t b) { return (b + 15) & ~(int64_t)15; };
  TileLayout t;
  t.col = pad16(4 * (nl / 32 + 1));
  t.val = t.col + pad16(2 * ne);
  t.dinv = t.val + pad16(sv * ne);
  t.lsm = t.dinv + pad16(s * nl);
  t.laux = t.lsm + pad16(4 * nl);
  t.ext = t.laux + pad16(4 * nl);
  t.end = t.ext + pad16(4 * nx);
  return t;
}

template <class T>
struct TileSweeps {
  int64_t ntiles = 0, nloc = 0;  // tiles, local rows (each colour group padded to 32)
  int maxloc = 0, maxext = 0;    // largest local row count and outside-value count of a tile
  int tpb = 256;                 // threads per block
  int64_t maxblob = 0;           // largest tile block (bytes)
  int64_t interior = 0, halo = 0;  // real rows: the tiles' own, and halo copies
  int64_t nnz = 0, nnz_real = 0;   // stored / real entries over all tiles
  DBuf<int64_t> loc_off;         // [ntiles + 1] first local row of each tile (multiples of 32)
  DBuf<int64_t> blob_off;        // [ntiles + 1] byte offset of each tile's block
  DBuf<int64_t> ext_off;         // [ntiles + 1] first outside value of each tile
  DBuf<int32_t> phase;           // [ntiles * (ncol + 1)] colour-class starts within each tile
  DBuf<unsigned char> blob;      // the tiles' blocks
  // post-sweeps: every place (local row of some tile) where each SM row sits,
  // own or halo (CSR by SM row), so that k_up_init can write the start values
  // and saved rhs straight into tile order for the tiles to copy in
  DBuf<int64_t> pos_ptr;         // [nsm + 1]
  DBuf<int32_t> pos;             // positions in [0, nloc)
  // shared memory of a launch: the largest block, then U (rows and outside
  // values) and F of the largest tile
  size_t smem() const { return (size_t)maxblob + (size_t)(maxloc + maxext) * sizeof(T) + (size_t)maxloc * sizeof(T); }
};

// The exact near-boundary solve of Algorithm 3 on the device: the block
// cyclic reduction of nb::Factor flattened into arrays.  Ordered positions q
// (0..m-1) follow the factor's breadth-first order.  Round r has nblk[r]
// blocks; block k of round r is described by 5 int64 at btab[(boff[r] + k) * 5]:
// size, offset within the round's vector, and the offsets in `mats` of its
// Cholesky factor F (odd blocks), Lo and Up (-1 when absent); all matrices
// dense row-major FP64.  The round-r vectors live at voff[r] in the rhs and
// solution pools (voff[R] = pool size).  `last` is the factor of the one
// block left after the rounds.
struct NbDev {
  int64_t m = 0;
  int R = 0;
  int last_size = 0;
  int64_t last_off = 0;
  std::vector<int32_t> nblk_h;     // host copy of the per-round block counts
  DBuf<int32_t> nblk, boff;        // [R]
  DBuf<int64_t> btab, voff;        // [sum nblk * 5], [R + 1]
  DBuf<double> mats;
  DBuf<int32_t> aux;               // [m] aux ID of ordered position q
  DBuf<int32_t> sm;                // [m] SM row of ordered position q (the saved rhs fs is in SM order)
};

// ------------------------------------------------------------ solve data
template <class T>
struct AuxLevelDev {
  int level = 0;
  int ncolours = 0;
  std::vector<int64_t> cstart;   // colour class starts in SM rows (multiples of 32)
  std::vector<int64_t> cnnz, crows;  // real non-zeros / rows per colour class
  int64_t nsm = 0, nsm_real = 0; // padded / real smoothing rows
  DBuf<int32_t> sm_rows;         // aux ID per SM row (-1 padding)
  Sell<T> SM;                    // A_l rows of N~_l (all columns; the up sweeps)
  Sell<T> SMd;                   // the same rows, columns in N~_l only, as SM row indices (the down sweeps)
  std::vector<int64_t> cnnz_d;   // real non-zeros of SMd per colour class
  DBuf<T> sm_dinv;
  int64_t nrs = 0, nrs_real = 0;
  DBuf<int32_t> rs_rows;         // aux ID per residual row
  Sell<T> RS;                    // A_l rows of E_l, columns in N~_l only, as SM row indices
  int64_t nnew = 0;
  DBuf<int32_t> nn_id, nn_p0, nn_p1;  // prolongation of new nodes
  int64_t npar = 0, nchild = 0;
  DBuf<int32_t> rp_id;           // parents receiving restricted residuals
  DBuf<int32_t> rp_ptr, rp_child;
  SmallLevelDev<T> small;        // shared-memory form, when the level is small
  // temporal blocking (tiled = 1): pre-sweeps in one launch (k_tile_down), and
  // after k_up_init, post-sweeps in one launch (k_tile_up)
  bool tiled = false;                // tiles built for both directions
  bool tiled_down = false, tiled_up = false;  // the directions that run on them (the autotuner's choice)
  int tile_rows = 0;                 // own rows per tile
  TileSweeps<T> tdown, tup;
  DBuf<int32_t> sm_par0, sm_par1;    // per SM row: parents of a new node (-1 Dirichlet), -3 not new
  // mixed boundaries: the near-boundary correction of Algorithm 3 (nb.m > 0):
  // rows of A_l on J_{l,j} in ordered positions (all columns, aux IDs) and the
  // flattened factor
  NbDev nb;
  Sell<T> NB;
};

struct Stats {
  double t_tree = 0, t_aux = 0, t_fine = 0, t_levels = 0, t_total = 0;
  // parts of t_levels: level assembly, colouring, row selection + SELL packing
  // (+ shared-memory forms), export copies, coarsest inverse, transfer, solve state
  double t_lv_assemble = 0, t_lv_colour = 0, t_lv_pack = 0, t_lv_export = 0, t_coarse = 0, t_transfer = 0,
         t_slots = 0;
  double t_sz = 0;  // device Scott-Zhang build (after t_aux)
};

}  // namespace asmg

// ------------------------------------------------------------------ handle
struct asmg_s;
