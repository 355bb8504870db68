// Launchers of the sm_103a kernels (defined in fs_assembly.cu and
// fs_linalg.cu) and the plain views they take.  Host code only sees these
// declarations; every pointer in a view is a device pointer.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "fs_internal.h"

namespace fs {

// Counts kernel launches issued from the host (ignored while a stream is
// being captured into a graph; graph replays add their node count).
void count_launches(int64_t n);

// Programmatic dependent launch.  The solver's kernels run as chains of
// short dependent passes (a V-cycle's levels, the Gram-Schmidt passes), so
// the gap between one kernel's last block and the next kernel's first is a
// large part of a step.  A kernel launched by launch_k with the overlap mode
// on may be scheduled while its predecessor in the stream drains; its first
// statement is pdl_wait() (griddepcontrol.wait), which returns once every
// prerequisite grid has completed and its memory operations are visible, so
// no global access of the kernel can overlap the predecessor.  Without the
// attribute griddepcontrol.wait returns at once and the launch is an
// ordinary serialised one.  The mode is per calling thread, taken from the
// problem's schedule by the API entry points.
bool launch_overlap();

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

template <typename... KArgs, typename... Args>
inline void launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = launch_overlap() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Element-level reference integrals in constant memory (per dimension).
void upload_ref_tensors(const RefTensors& R2, const RefTensors& R3);

template <typename T>
struct DCsr {
  int32_t nrow = 0;
  // threads that share a row in the transfer kernels (1, 4 or 32, from the
  // mean row length: one thread per row for the 1-3 entries of a
  // prolongation row, a warp for the ~50 of a restriction row onto a grid
  // coarsened by 4)
  int32_t lanes = 4;
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const T* v = nullptr;
};

// Sliced ELLPACK with slices of 32 rows (one thread per row): the entries of
// row 32 s + t sit at off[s] + 32 u + t for the slot u < (off[s+1] - off[s]) / 32,
// so a warp's loads of one slot are contiguous.  Slots past a row's length
// hold coefficient 0 and the row itself as column.
template <typename T>
struct DSell {
  int64_t nrow = 0;
  const int64_t* off = nullptr;
  const int32_t* ci = nullptr;
  const T* v = nullptr;
  // > 0: every slice has this many slots (off[s] = 32 s width), so a
  // thread finds its slice without loading off
  int64_t width = 0;
};

// A vector addressed through the device-side Arnoldi step index: base +
// (*j) stride (base itself when j is null).  The kernels of one Arnoldi step
// take their Krylov vectors this way, so that one captured step can be
// replayed by a conditional loop node while j advances on the device.
template <typename T>
struct JVec {
  T* base = nullptr;
  const int* j = nullptr;
  int64_t stride = 0;
  JVec() = default;
  JVec(T* b) : base(b) {}
  JVec(T* b, const int* jj, int64_t st) : base(b), j(jj), stride(st) {}
  JVec<T> shifted(int64_t o) const { return JVec<T>(base + o, j, stride); }
  __device__ __forceinline__ T* get() const { return j ? base + (int64_t)(*j) * stride : base; }
};

// Mesh tables and block patterns of one problem on the device.
struct DMesh {
  int dim = 0, nloc = 0, nb = 0;
  int64_t nv = 0, n2 = 0, ncell = 0;
  const int32_t* c2d = nullptr;        // ncell x nloc
  const double* p2xyz = nullptr;       // n2 x dim
  const uint8_t* dirichlet = nullptr;  // n2
  const int32_t* dlist = nullptr;      // Dirichlet node ids
  int64_t ndir = 0;
  const int32_t *rpA = nullptr, *ciA = nullptr;    // P2-P2
  const int32_t *rpB = nullptr, *ciB = nullptr;    // P1-P2
  const int32_t *rpBT = nullptr, *ciBT = nullptr;  // P2-P1
  const int32_t *rpK = nullptr, *ciK = nullptr;    // P1-P1
  const uint8_t *posA = nullptr, *posB = nullptr, *posBT = nullptr, *posK = nullptr;
  const double* nu_cell = nullptr;     // per-cell viscosity (batches) or null
  const int32_t* color_cells = nullptr;  // cells grouped by colour (Mesh)
};

// Physical description of the manufactured problem.
struct DPhys {
  int kind = 0;
  double nu = 1.0;
  const double* nu_node = nullptr;  // per-P2-node viscosity (batches) or null
  double wconst[3] = {0, 0, 0};
};

// ---- assembly (fs_assembly.cu) -------------------------------------------
// Colour-ordered element kernels (color_ptr: the host copy of
// Mesh::color_ptr, one launch per colour): the cells of a colour share no
// node, so they add into the block values with plain read-modify-writes, no
// atomics, and every value is summed in the same order on every run.
// Step-invariant blocks (always colour-ordered), accumulated into zeroed
// arrays:
// base = mass_coef M + nu K (P2-P2), Mv = M, B (P1-P2, dim values per entry),
// BT (P2-P1, dim values), Kp (P1 stiffness), mpl (lumped P1 mass).
void launch_assemble_base(const DMesh& m, const std::vector<int64_t>& color_ptr,
                          double mass_coef, double nu, double* base, double* Mv, double* B,
                          double* BT, double* Kp, double* mpl, cudaStream_t s);
// valA += N(w) with w taken from the component-blocked vector w (ldw =
// component stride) or the constant field wc when w == nullptr; rows of
// Dirichlet nodes are skipped.  deterministic: colour by colour as the
// step-invariant blocks, a thread per (cell, row); otherwise one launch over
// all cells, a thread per cell, FP64 atomics (faster; the last bits of a
// value depend on the order its contributions arrive in).
void launch_assemble_conv(const DMesh& m, const std::vector<int64_t>& color_ptr,
                          const double* w, int64_t ldw, const double* wc, double* valA,
                          bool deterministic, cudaStream_t s);
// Np += the pressure-space convection int psi_q (w . grad psi_s) (P1-P1
// pattern, slot tables posK; w component-blocked with stride ldw, or the
// constant field wc when w == nullptr); rows of the vertices with fixed set
// stay untouched.  FP64 atomics.
void launch_assemble_conv_p1(const DMesh& m, const double* w, int64_t ldw, const double* wc,
                             const uint8_t* fixed, double* Np, cudaStream_t s);
// Dirichlet rows of the scalar block become identity rows.
template <typename T>
void launch_bc_rows(const DMesh& m, T* valA, cudaStream_t s);
// F[c][j] = mass_coef * u_c[j] + f_c(x_j, t) for every P2 node.
void launch_eval_load(const DMesh& m, const DPhys& ph, double t,
                      double mass_coef, const double* u, double* F,
                      cudaStream_t s);
// b = M F (velocity rows), Dirichlet rows = u_exact(t), b_p = 0 except the
// pinned rows (p_exact at their vertex).
void launch_rhs(const DMesh& m, const DPhys& ph, double t, const double* Mv,
                const double* F, const int32_t* pinned, int npinned, double* b,
                cudaStream_t s);
// Exact state I_h u, I_h p at time t (zero_interior: 0 off Dirichlet nodes).
void launch_exact_state(const DMesh& m, const DPhys& ph, double t,
                        int zero_interior, double* x, cudaStream_t s);
// Monolithic CSR values from the block values (export for parity checks).
// Monolithic CSR values in paper order (rows and columns of fs_dof_map):
// mrp holds that CSR's row pointers and nat the paper id of each internal
// P2 node; an entry's place in its row is the rank of its paper column.
void launch_expand_monolithic(const DMesh& m, const int32_t* nat, const double* valA,
                              const double* B, const double* BT, const double* diagp,
                              const int64_t* mrp, double* out, cudaStream_t s);
// n_dof vectors between the internal and the paper order of the P2 nodes:
// to_nat = 1: out[c n2 + nat[q]] = in[c n2 + q]; to_nat = 0: the inverse;
// pressure entries are copied.
void launch_dofs_perm(const DMesh& m, const int32_t* nat, const double* in, double* out,
                      int to_nat, cudaStream_t s);

// ---- Taylor-Hood P3/P2 on triangles (fs_assembly.cu) ----------------------
// m: a DMesh holding the P3 tables (c2d = the P3 map, 10 per cell; n2 = P3
// nodes; nv = P2 pressure nodes; p2xyz = P3 node coordinates; patterns and
// slot tables of P3Tables), c2p the P2 map (6 per cell), R the reference
// integrals in device memory.  Blocks as launch_assemble_base /
// launch_assemble_conv (FP64 atomics).
void launch_p3_base(const DMesh& m, const int32_t* c2p, const RefP3* R, double mass_coef,
                    double nu, double* base, double* Mv, double* B, double* BT, double* Kp,
                    cudaStream_t s);
void launch_p3_conv(const DMesh& m, const RefP3* R, const double* w, int64_t ldw,
                    const double* wc, double* valA, cudaStream_t s);
void launch_p3_exact_state(const DMesh& m, const DPhys& ph, double t, int zero_interior,
                           const double* pxyz, double* x, cudaStream_t s);

// ---- linear algebra (fs_linalg.cu) ---------------------------------------
// Saddle-point operator in block form.
struct SegState;

// Rows of a batch whose segment (instance) has converged in the current
// restart cycle: the union kernels skip them.  slice_seg[s] is the segment
// of rows 32 s .. 32 s + 31 of a level (-1 where a slice holds rows of two
// instances: never skipped); st is the Krylov segment state (null: nothing
// is skipped, as for single problems and for timing runs).
struct SegSkip {
  const int32_t* slice_seg = nullptr;
  const SegState* st = nullptr;
};

template <typename T>
struct DOp {
  int dim = 0;
  int64_t n2 = 0, nv = 0;
  // SELL-32 blocks.  B and BT hold dim values per slot, component-major
  // within a slot: the value of component c of row 32 s + t at slot u is at
  // (off[s] + 32 u) dim + 32 c + t.
  DSell<T> A, B, BT;
  const T* diagp = nullptr;
  int group = 0;  // slots issued together per thread (0: the default)
  // batches: segments of the velocity rows (union node order) and of the
  // pressure rows, for the Arnoldi steps' products
  SegSkip skip_u, skip_p;
};

// y = K x (resid == 0) or y = b - K x (resid == 1); vectors of type V.
// seg: skip the rows of converged segments (the Arnoldi step's product;
// residuals and timing runs take every row).
template <typename T, typename V>
void launch_spmv_full(const DOp<T>& op, JVec<const V> x, const V* b, JVec<V> y,
                      int resid, const int* skip, cudaStream_t s, bool seg = false);

// Scalar CSR values (row pointers rp) into a SELL-32 layout with slice
// offsets off: out64 (and out32 when not null) receive the n-row matrix.
void launch_csr_to_sell(int64_t n, const int32_t* rp, const double* in, const int64_t* off,
                        double* out64, float* out32, cudaStream_t s);

// Multigrid level on the device.
template <typename T>
struct DLevel {
  DSell<T> A;           // level operator
  DCsr<T> P, R;         // P: prolongation from level+1, R = P^T
  SegSkip skip;         // rows of this level by segment
  const T* dinv = nullptr;
  double inv_theta = 0, a1 = 0, b1 = 0, a2 = 0, b2 = 0;  // Chebyshev(3)
  double lmax = 0;  // estimate of the largest eigenvalue of D^-1 A (host set-up)
};
template <typename T>
struct DHier {
  int nlev = 0;
  int ncp = 1;  // components per row in the level vectors (1, 2 or 4)
  DLevel<T> lev[16];
  // coarsest level: block-diagonal dense inverses (one block per instance)
  const T* cinv = nullptr;           // concatenated row-major blocks
  const int32_t* row_blk = nullptr;  // coarsest row -> block
  const int64_t* blk_row = nullptr;  // block -> first row
  const int64_t* blk_n = nullptr;    // block -> size
  const int64_t* blk_dense = nullptr;  // block -> offset in cinv
  int64_t ncoarse = 0;
  int64_t dense_nb0 = 0;  // ncoarse when the coarsest level is one block, else 0
  // per level (all rows x ncp, row-interleaved components): right-hand
  // side b, and ping-pong pairs of the gather vector G (x + d, the point the
  // next residual is taken at) and the Chebyshev direction D
  T* b[16] = {};
  T* G0[16] = {};
  T* G1[16] = {};
  T* D0[16] = {};
  T* D1[16] = {};
  // level-0 block order vs the caller's vector order (batches): perm[r] is
  // the caller's row of block row r, iperm its inverse; null when equal
  const int32_t* perm = nullptr;
  const int32_t* iperm = nullptr;
  // slots issued together per thread in the smoothing passes (4 or 6)
  int group = 4;
  // Chebyshev degree of the pre- and post-smoothing below the finest level
  // and on the finest level (3 or 2 each)
  int coarse_deg = 2;
  int fine_deg = 3;
  // first level run by the fused cluster kernel (-1: none), its cluster size
  int tail = -1;
  int tail_cluster = 8;
  // a copy of this struct in device memory (read by the coarse kernels)
  const DHier<T>* dev = nullptr;
};

// The hierarchy with segment skipping off (timing and profiling runs, whose
// segment states are those of the last solve).
template <typename T>
inline DHier<T> without_skip(const DHier<T>& H) {
  DHier<T> C = H;
  for (int l = 0; l < 16; ++l) C.lev[l].skip.st = nullptr;
  return C;
}

// Gauss-Jordan inversion with partial pivoting of a dense n x n FP64
// matrix, held row-major as the augmented n x 2n array W = [A | I]; after
// the n pivot steps the right half holds A^-1 (the left half is not kept
// up to date).  piv, pval: device scratch for the pivot row and value; bad:
// device flag set when a pivot column is zero.  Set-up only.
void launch_gj_step(double* W, int64_t n, int64_t c, int64_t* piv, double* pval, int* bad,
                    cudaStream_t s);
// out (n x n, row-major) = the right half of W, converted to T.
template <typename T>
void launch_gj_extract(const double* W, int64_t n, T* out, cudaStream_t s);

// Cluster size (16 or 8 blocks) of the fused kernel for this arithmetic and
// row width.
template <typename T>
int mg_tail_cluster(int ncp);

// One fused Chebyshev step (mode STEP) on level 0 of H with its own work
// vectors, for kernel timing.
template <typename T>
void launch_cheb_step(const DHier<T>& H, int nc, cudaStream_t s);

// scratch[0] = sum_i (a_i - b_i)^2, scratch[1] = sum_i a_i^2 over i < n, in
// a fixed summation order; scratch holds diff_norms_scratch() doubles.
int diff_norms_scratch();
void launch_diff_norms(const double* a, const double* b, int64_t n, double* scratch,
                       cudaStream_t s);

// Reads `bytes` (a multiple of 16) of buf so that the L2 holds clean lines
// of it and nothing of the data timed next (kernel timing with a cold L2).
void launch_l2_flush(const void* buf, int64_t bytes, int* sink, cudaStream_t s);

// Polynomial extrapolation in time of the state x (x^n) through it and its
// nprev <= kExtrapMax previous values prev[j] = x^(n-1-j) to the next time
// level: x <- sum_j (-1)^j C(nprev+1, j+1) x^(n-j) over j = 0..nprev (x
// itself for nprev = 0); the old x goes to dst, which may be prev[nprev-1]
// (each entry is read before it is written).  n entries each.
void launch_extrapolate(double* x, const double* const* prev, int nprev, double* dst, int64_t n,
                        cudaStream_t s);

// Conversion out = (B)(in * scale) (scale = *scale or 1/*scale when inv).
template <typename A, typename B>
void launch_convert(const A* in, B* out, int64_t n, const double* scale,
                    int inv, cudaStream_t s);

// The convection part of the pressure convection-diffusion operator, for
// the Schur-complement approximation: the P1-P1 matrix Np (CSR rows of the
// pressure vertices) and the inverse lumped pressure mass.  v == nullptr:
// not used.
template <typename T>
struct PcdView {
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const T* v = nullptr;
  const T* invm = nullptr;
};

// z = P^-1 r, the block preconditioner.  mpl_inv_nu: nu over the lumped
// pressure mass per vertex, negative on the pinned vertices (their rows pass
// r_p through).  With pcd.v set, the Schur part is
// M_p^-1 (M_p / dt + nu K_p + N_p) K_p^-1 (pressure convection-diffusion)
// instead of nu M_p^-1 + dt^-1 K_p^-1 (Cahouet-Chabard).
template <typename T>
void launch_precond(const DOp<T>& op, const DHier<T>& HA, const DHier<T>& HK,
                    const T* mpl_inv_nu, double inv_dt, JVec<const T> r, JVec<T> z,
                    T* work_p, T* work_u,
                    const int* skip, cudaStream_t s, const PcdView<T>& pcd = PcdView<T>());

// ---- the block preconditioner as one persistent kernel (fs_linalg.cu) ----
// The passes of launch_precond (pressure load, the pressure V-cycle, the
// Cahouet-Chabard combination, the B^T coupling, the velocity V-cycle) become
// phases of a work-list of items (phase, instance, row range).  One
// cooperative launch (every block resident) walks it: block b takes items
// b, b + grid, ... in list order; an item of phase p of instance i starts
// once every item of phase p - 1 of instance i has finished (a counter per
// (phase, instance), incremented after each item with release semantics,
// polled with acquire loads by the block's first thread).  Instances are
// independent (every operator of a batch is block-diagonal), so no phase
// waits for the whole batch.  Items of instances that converged in the
// running cycle are skipped.  The list is ordered by phase, so every item's
// predecessors come before it and, all blocks being resident, every wait
// ends; each wait still gives up after one second (the segment is then
// marked with bad = 2 and the solve reports FS_ERR_TIMEOUT).  The last
// block to leave zeroes the counters for the next launch.
struct FlowItem {
  int32_t phase, seg, row0, row1;
};
struct FlowHost {
  std::vector<unsigned char> phases;  // nphase phase records (fs_linalg.cu)
  std::vector<FlowItem> items;
  std::vector<int32_t> need;          // items per (phase, instance): nphase x nseg
  int nphase = 0;
};
struct FlowDev {
  const void* phases = nullptr;
  const FlowItem* items = nullptr;
  int64_t nitems = 0;
  unsigned* cnt = nullptr;             // nphase x nseg, zero between launches
  const int32_t* need = nullptr;
  unsigned* ticket = nullptr;          // exit ticket, zero between launches
  int nphase = 0, nseg = 0, nblocks = 0;
};
// Resident blocks of the persistent kernel for this arithmetic and velocity
// row width (ncp 2 or 4): blocks per SM x SMs of the current device.
template <typename T>
int flow_blocks(int ncp);
// The work-list of one application.  offA / offK: per level of HA / HK the
// first row of each instance (nseg + 1 entries, block order); prow: the
// first caller pressure row of each instance (nseg + 1).  Items are
// sized so that a phase over all instances has at least `nblocks` of them
// when it has enough rows.
template <typename T>
void build_flow(const DHier<T>& HA, const DHier<T>& HK,
                const std::vector<std::vector<int64_t>>& offA,
                const std::vector<std::vector<int64_t>>& offK, const std::vector<int64_t>& prow,
                int nblocks, FlowHost& out);
// One application through the persistent kernel (same arguments as
// launch_precond, plus the plan; st: skip instances with done set, or null;
// flag: segment states that receive bad = 2 on a timed-out wait, or null).
template <typename T>
void launch_precond_flow(const FlowDev& f, const DOp<T>& op, const DHier<T>& HA,
                         const T* mpl_inv_nu, double inv_dt, JVec<const T> r, JVec<T> z,
                         T* work_p,
                         const SegState* st, SegState* flag, const int* skip, cudaStream_t s);

// ---- incremental pressure correction (fs_ipcs.cu) -----------------------
// Right-hand sides of the three stages (x = [u^n | p^n], b = the assembled
// load with the Dirichlet and pinned values of t^{n+1}); see fs_ipcs.cu.
void launch_ipcs_rhs1(const DMesh& m, const double* valA, const double* base, const double* BT,
                      const double* b, const double* x, double* r, cudaStream_t s);
void launch_ipcs_rhs2(const DMesh& m, const double* B, const double* ustar, double inv_dt,
                      const uint8_t* fixed, const double* b, const double* x, double* r,
                      cudaStream_t s);
void launch_ipcs_rhs3(const DMesh& m, const double* Mv, const double* BT, const double* b,
                      const double* ustar, const double* dp, double dt, double* r,
                      cudaStream_t s);
// y = A x for which = 0 (scalar P2 block `vals` on every component,
// identity at Dirichlet nodes) or 1 (P1 Laplacian `vals`, identity at the
// fixed vertices); part (may be null) receives per-block partials of x . y;
// returns the number of blocks.
int launch_ipcs_apply(const DMesh& m, int which, const double* vals, const uint8_t* fixed,
                      const double* x, double* y, double* part, cudaStream_t s);
void launch_ipcs_dinv(const DMesh& m, int which, const double* vals, const uint8_t* fixed,
                      double* dinv, cudaStream_t s);
void launch_ipcs_fix(const DMesh& m, int which, const uint8_t* fixed, const double* rhs,
                     double* x, cudaStream_t s);
void launch_ipcs_add(int64_t n, const double* x, double* y, cudaStream_t s);
// doubles of block-partial scratch the CG kernels need on this mesh
int ipcs_part_size(const DMesh& m);
// Jacobi-preconditioned CG steps; sc (4 doubles on the device): rz, alpha,
// beta, rr.
void launch_cg_init(int64_t n, const double* rhs, const double* y, const double* dinv, double* r,
                    double* z, double* p, double* part, double* sc, cudaStream_t s);
void launch_cg_alpha(const double* part, int nb, double* sc, cudaStream_t s);
void launch_cg_update(int64_t n, double* sc, const double* p, const double* q,
                      const double* dinv, double* x, double* r, double* z, double* part,
                      cudaStream_t s);
void launch_cg_dir(int64_t n, const double* sc, const double* z, double* p, cudaStream_t s);
// Flexible CG (preconditioner applied by the caller between the two):
// t = r, x += alpha p, r -= alpha q (rr into sc[3]); then with z = M(r),
// zeroed on the fixed rows, the dots r.z, t.z give beta (Polak-Ribiere) and
// the new rz; first = 1 starts the iteration (p = z, rz = r.z).
void launch_cg_update_flex(int64_t n, double* sc, const double* p, const double* q, double* x,
                           double* r, double* t, double* part, cudaStream_t s);
void launch_cg_dots_flex(int64_t n, const uint8_t* fixed, const double* r, const double* t,
                         double* z, double* p, int first, double* part, double* sc,
                         cudaStream_t s);

// z = one V-cycle of the single-component hierarchy H on r (n level-0 rows
// in the caller's order): the pressure Laplacian part of the block
// preconditioner, reused to precondition the IPCS pressure increment.
template <typename T>
void launch_vcycle_scalar(const DHier<T>& H, const T* r, T* z, int64_t n, cudaStream_t s);

// ---- segmented Krylov (fs_krylov.cu) -------------------------------------
constexpr int kTileLen = 2048;  // vector entries per reduction tile

// A contiguous range [start, start + len) of one segment's entries.
struct Tile {
  int64_t start;
  int32_t len;
  int32_t seg;
};
struct TileList {
  const Tile* tiles = nullptr;
  int ntiles = 0;
};

// Per-segment state of the restart cycle.  The first 64 bytes are the
// status block the host reads back after every part of a solve.
struct SegState {
  double beta;      // ||r0|| of the cycle
  double resid;     // Arnoldi residual estimate
  double bnorm;     // ||b|| (FP64 right-hand side of the segment)
  double rnorm;     // FP64 residual norm (refinement)
  double tol_abs;   // Arnoldi target of the cycle
  int done;         // converged / retired / broken: kernels skip the segment
  int k;            // Arnoldi steps taken in this cycle
  int bad;          // NaN/Inf seen
  int retired;      // set by the host: the segment no longer iterates
  int first_tile, ntiles;
  double rtol;      // set by the host: target of the next cycle, relative to
                    // beta or to bnorm (device data, so captured graphs stay
                    // valid when it changes)
  double hn;        // ||w|| before normalisation
  unsigned counter[8];
  double H[(kMaxRestart + 1) * kMaxRestart];
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1];
  double h2[kMaxRestart + 1];
};
#ifdef __CUDACC__
__device__ __forceinline__ bool seg_skipped(const SegSkip& k, int64_t row) {
  if (!k.st) return false;
  const int32_t g = k.slice_seg[row >> 5];
  return g >= 0 && k.st[g].done;
}
#endif

struct KCtl {
  int m;         // restart length
  int nseg;      // number of segments
  int ndone;     // segments done in this cycle
  int all_done;  // every segment done: the spanning kernels skip
  int j;         // Arnoldi step of the cycle (reset by the cycle init,
                 // advanced by the Givens step: its own kernel, or the
                 // second CGS2 pass for problems of one segment)
};

template <typename V>
void launch_seg_norm(const V* x, const TileList& tl, SegState* st, double* partial,
                     int field, cudaStream_t s);
// cond: the handle of a conditional loop node replaying the Arnoldi step
// (0 when the steps are launched one by one); the cycle init sets it to
// "not every segment done", the Givens kernel to "not done and j < m".
void launch_seg_cycle_init(SegState* st, KCtl* ctl, int relative_to_beta,
                           cudaGraphConditionalHandle cond, cudaStream_t s);
template <typename V>
void launch_seg_scale(JVec<V> x, const TileList& tl, const SegState* st, int field,
                      cudaStream_t s);
// CGS2 on w = V[j + 1] with j = ctl->j, ending with V[j + 1] normalised.
// with_givens (problems of one segment): the Givens step of column j and the
// advance of the step index (setting cond when not 0) are done by the
// second pass, in place of launch_seg_givens.
template <typename V>
void launch_seg_cgs2(V* Vb, int64_t n, const TileList& tl, SegState* st, KCtl* ctl,
                     double* partial, bool with_givens, cudaGraphConditionalHandle cond,
                     cudaStream_t s);
void launch_seg_givens(SegState* st, KCtl* ctl, int nseg, cudaGraphConditionalHandle cond,
                       cudaStream_t s);
// One pass of the CGS2 step alone (0: dot, 1: update + re-dot, 2: final
// update and normalisation; no Givens step), for kernel timing.
template <typename V>
void launch_seg_cgs2_pass(V* Vb, int64_t n, const TileList& tl, SegState* st, KCtl* ctl,
                          double* partial, int pass, cudaStream_t s);
template <typename V, typename X>
void launch_seg_update_x(const SegState* st, const KCtl* ctl, const V* Z, int64_t n,
                         const TileList& tl, X* x, cudaStream_t s);
template <typename A, typename B>
void launch_seg_normalise(const A* in, B* out, const TileList& tl, const SegState* st,
                          cudaStream_t s);
template <typename V, typename X>
void launch_seg_axpy(X* x, const V* d, const TileList& tl, const SegState* st,
                     cudaStream_t s);

}  // namespace fs
