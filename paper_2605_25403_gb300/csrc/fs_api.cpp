// C ABI of libfs (include/fs.h): problem lifecycle (single meshes and batches
// of independent instances), the per-step assembly driver, and the flexible
// GMRES(m) solve as a resumable state machine (FP64, or FP32 inner cycles
// with FP64 iterative refinement), replaying restart cycles as CUDA graphs.
//
// Paper Sec. 3.1 (ComputationModel workflow: assembly -> linear solver ->
// update) and Sec. 2.2.1 (Oseen step).  Host code only: every floating-point
// operation on the step's data runs in the kernels of fs_assembly.cu,
// fs_linalg.cu and fs_krylov.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <functional>
#include <initializer_list>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "fs_device.h"
#include "fs_internal.h"

struct fs_mesh {
  fs::Mesh m;
};

namespace fs {

namespace {
thread_local std::string g_err;
thread_local bool g_capturing = false;
// launch mode of the calling thread's current API call: -1 outside a call
// on a problem (overlap on), else 1 / 0 from the problem's schedule
thread_local int g_overlap = -1;
std::atomic<int64_t> g_launches{0};

RefTensors g_ref2, g_ref3;
std::once_flag g_ref_once;
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }

void count_launches(int64_t n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

bool launch_overlap() { return g_overlap != 0; }

}  // namespace fs

using namespace fs;

namespace {

#define FS_CUDA(call)                                                            \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? FS_ERR_OOM : FS_ERR_CUDA;         \
    }                                                                            \
  } while (0)

#define FS_TRY(expr)              \
  do {                            \
    int rc_ = (expr);             \
    if (rc_ != FS_OK) return rc_; \
  } while (0)

// Host mirror of the 64-byte status block at the head of SegState.
struct SegHost {
  double beta, resid, bnorm, rnorm, tol_abs;
  int done, k, bad, retired, first_tile, ntiles;
};
static_assert(sizeof(SegHost) == 64, "status block layout");
static_assert(offsetof(SegState, retired) == offsetof(SegHost, retired), "status layout");
static_assert(offsetof(SegState, ntiles) == offsetof(SegHost, ntiles), "status layout");

template <typename V>
struct Krylov {
  int m = 0;
  int64_t n = 0;
  V* Vb = nullptr;      // (m+1) x n basis
  V* Z = nullptr;       // m x n preconditioned directions
  V* work_p = nullptr;  // nv
  V* work_u = nullptr;  // dim x n2
  V* rhs = nullptr;     // inner right-hand side (precision mode)
  V* sol = nullptr;     // inner solution (precision mode)
  double* partial = nullptr;  // (m+1) x ntiles
  SegState* st = nullptr;
  KCtl* ctl = nullptr;
  cudaGraphExec_t g_check = nullptr, g_iter = nullptr;
  size_t n_check = 0, n_iter = 0;  // top-level nodes per graph
  size_t n_body = 0;               // kernels of one Arnoldi step (loop body)
  const void* g_x = nullptr;       // buffers the graphs were captured with
  const void* g_b = nullptr;
};

template <typename T>
struct Precision {
  DOp<T> op;
  DHier<T> HA, HK;
  T* mplinv_nu = nullptr;
  Krylov<T> kr;
  // the persistent form of the preconditioner: first row of each instance
  // per level of HA and HK, first caller pressure row of each instance, and
  // the work-lists (one per set of smoothing degrees, built on first use)
  std::vector<std::vector<int64_t>> offA, offK;
  std::vector<int64_t> prow;
  FlowDev flow[8];
  int flow_ratio[8] = {};  // the Chebyshev interval ratio each work-list holds
  int cheb_ratio = 8;      // the hierarchies' current Chebyshev interval ratio
  // pressure convection-diffusion form of the Schur part: inverse lumped
  // pressure mass, the pressure convection matrix in this precision
  T* invm = nullptr;
  T* Np = nullptr;
};

// The work-list built for the hierarchies' current smoothing degrees.
template <typename T>
int flow_index(const DHier<T>& HA, const DHier<T>& HK) {
  return (HA.coarse_deg == 3) | (HA.fine_deg == 3) << 1 | (HK.fine_deg == 3) << 2;
}

// Resumable solve / step state.
enum Phase { PH_IDLE, PH_CHECK, PH_ITER, PH_RES64, PH_INNER, PH_DONE };

struct SolveCtx {
  fs_solve_opts o{};
  double* x = nullptr;
  int phase = PH_IDLE;
  int steps_left = 0;
  fs_solve_stats* per_step = nullptr;  // caller array (blocking fs_step)
  int step_index = 0;
  int rc = FS_OK;
  // per segment
  std::vector<int> status, iters, cycles, refines;
  std::vector<double> relres, prev;
  std::vector<int> retired;
};

}  // namespace

struct fs_problem {
  fs_mesh* mesh = nullptr;
  fs_problem_desc desc{};
  std::vector<fs_problem_desc> inst_desc;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;  // captures the body of the Arnoldi loop node
  int dim = 0, nseg = 1;
  int64_t n2 = 0, nv = 0, ndof = 0;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  DMesh dm;
  DPhys ph;
  // FP64 data
  double *baseA = nullptr, *Mv = nullptr, *valA = nullptr, *B = nullptr, *BT = nullptr;
  double *Kp = nullptr, *mpl = nullptr, *diagp = nullptr;
  double *x = nullptr, *b = nullptr, *F = nullptr, *r64 = nullptr;
  // the states before the latest step, x^(n-1-j) in hist_buf[(hist_head - j)
  // mod kExtrapMax] for j < hist, for the initial guess of the next step's
  // solve; hist = how many are valid (0 after problem creation, a state set
  // by the caller at another time, or a direct solve)
  double* hist_buf[kExtrapMax] = {};
  int hist = 0, hist_head = 0;
  int32_t* pinned = nullptr;
  int npinned = 0;
  // vertices whose rows of the preconditioner's pressure Poisson are fixed,
  // and the pressure convection matrix (P1-P1 pattern, FP64; allocated when
  // a schedule asks for the convection-diffusion Schur part)
  uint8_t* pfix = nullptr;
  double* Np64 = nullptr;
  std::vector<int32_t> pinned_host;  // the same vertices, on the host
  // Taylor-Hood P3/P2 problems (fs_problem_create_p3): the P2 pressure map,
  // pressure node coordinates, reference integrals; stepped by IPCS only
  bool p3 = false;
  int32_t* c2p = nullptr;
  double* pxyz = nullptr;
  RefP3* p3ref = nullptr;
  int64_t p3nnzA = 0;
  // Picard iteration (allocated on first use): the state at the start of the
  // step, the convecting field of the current iterate, norm scratch
  double *xn = nullptr, *wpic = nullptr, *nrm = nullptr;
  // IPCS stepping (allocated on first use): tentative velocity, pressure
  // increment, right-hand side and CG vectors (velocity-sized), inverse
  // diagonals of the three operators, partials, CG scalars, fixed vertices
  double *ip_us = nullptr, *ip_dp = nullptr, *ip_rhs = nullptr, *ip_r = nullptr;
  double *ip_z = nullptr, *ip_p = nullptr, *ip_q = nullptr;
  double *ip_dA = nullptr, *ip_dM = nullptr, *ip_dK = nullptr, *ip_part = nullptr;
  double *ip_sc = nullptr, *ip_nrm = nullptr;
  uint8_t* ip_fixed = nullptr;
  // pressure stage preconditioned by a V-cycle of the pressure Laplacian
  // hierarchy (P2/P1 problems): old residual, FP32 copies for an FP32 hierarchy
  bool ip_mg = false;
  double* ip_t = nullptr;
  float *ip_rf = nullptr, *ip_zf = nullptr;
  int64_t* mrp = nullptr;  // paper-order monolithic row pointers (export)
  const int32_t* nat = nullptr;          // internal P2 node -> paper id
  // batches: instance of every 32-row slice of the velocity rows (union
  // node order) and of the pressure rows, -1 for slices of two instances
  const int32_t* slice_seg_u = nullptr;
  const int32_t* slice_seg_p = nullptr;
  double *natbuf = nullptr, *natbuf2 = nullptr;  // boundary conversions (lazy)
  // SELL-32 copies of the blocks for the iteration path (slice offsets and
  // columns shared by both precisions)
  const int64_t *offA = nullptr, *offB = nullptr, *offBT = nullptr;
  const int32_t *sciA = nullptr, *sciB = nullptr, *sciBT = nullptr;
  double *sA64 = nullptr, *sB64 = nullptr, *sBT64 = nullptr;
  // FP32 data (precision mode)
  float *sA32 = nullptr, *sB32 = nullptr, *sBT32 = nullptr, *diagp32 = nullptr;
  Precision<double> p64;
  Precision<float> p32;
  bool has32 = false;
  // work-list of the n_dof vectors and per-segment status mirrors
  Tile* tiles = nullptr;
  int ntiles = 0;
  SegHost* host_status = nullptr;  // pinned, nseg entries
  int* host_retired = nullptr;     // pinned, nseg entries
  double* host_rtol = nullptr;     // pinned, nseg entries
  cudaEvent_t ev = nullptr;
  SolveCtx ctx;
  std::vector<fs_solve_stats> last_stats;  // per instance, last solve
  double t = 0;
  bool assembled = false;
  fs_schedule sched{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};

  TileList tl() const { return TileList{tiles, ntiles}; }

  // Device memory is stream-ordered (cudaMallocAsync on the problem's
  // stream): creating or destroying a problem does not synchronise the
  // device while other problems run.
  template <typename T>
  int alloc(T** p, int64_t count) {
    size_t bytes_ = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, bytes_, stream);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMalloc of ") + std::to_string(bytes_) + " bytes: " +
                cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? FS_ERR_OOM : FS_ERR_CUDA;
    }
    allocs.push_back(q);
    bytes += (int64_t)bytes_;
    *p = (T*)q;
    return FS_OK;
  }
  template <typename T>
  int upload(T** p, const std::vector<T>& h) {
    FS_TRY(alloc(p, (int64_t)h.size()));
    if (!h.empty())
      FS_CUDA(cudaMemcpyAsync(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, stream));
    return FS_OK;
  }
  ~fs_problem() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto* k : {&p64.kr.g_check, &p64.kr.g_iter, &p32.kr.g_check, &p32.kr.g_iter})
      if (*k) cudaGraphExecDestroy(*k);
    for (void* q : allocs) cudaFreeAsync(q, stream);
    if (stream) cudaStreamSynchronize(stream);
    if (host_status) cudaFreeHost(host_status);
    if (host_retired) cudaFreeHost(host_retired);
    if (host_rtol) cudaFreeHost(host_rtol);
    if (ev) cudaEventDestroy(ev);
    if (own_stream && stream) cudaStreamDestroy(stream);
    if (side) cudaStreamDestroy(side);
  }
};

namespace {

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return FS_ERR_CUDA;
  }
  return FS_OK;
}

// Scratch vectors of the paper-order conversions at the boundary.
int nat_buffers(fs_problem* P) {
  if (!P->natbuf) FS_TRY(P->alloc(&P->natbuf, P->ndof));
  if (!P->natbuf2) FS_TRY(P->alloc(&P->natbuf2, P->ndof));
  return FS_OK;
}

template <typename T>
int upload_csr(fs_problem* P, const HostCsr& H, DCsr<T>& d) {
  int32_t *rp, *ci;
  T* v;
  FS_TRY(P->upload(&rp, H.rowptr));
  FS_TRY(P->upload(&ci, H.col));
  std::vector<T> hv(H.val.begin(), H.val.end());
  FS_TRY(P->upload(&v, hv));
  d.nrow = (int32_t)H.nrow;
  const double mean = H.nrow > 0 ? (double)H.col.size() / (double)H.nrow : 0.0;
  d.lanes = mean <= 3.5 ? 1 : mean <= 16.0 ? 4 : 32;
  d.rp = rp;
  d.ci = ci;
  d.v = v;
  return FS_OK;
}

// SELL-32 layout of a CSR pattern: slice offsets (slices of 32 rows, width
// = the longest row of the slice) and slot-major columns.  Padding slots
// point at the row itself in a square matrix (a read the row makes anyway)
// and at column 0 in a rectangular one, so that every column is in range.
// uniform_slack > 0: when padding every slice to the widest costs at most
// that fraction more slots, all slices get that width; *width receives it
// (0 when the slices keep their own widths).
void sell_layout(const HostCsr& H, std::vector<int64_t>& off, std::vector<int32_t>& ci,
                 double uniform_slack = 0.0, int64_t* width = nullptr) {
  const bool square = H.nrow == H.ncol;
  const int64_t n = H.nrow, ns = (n + 31) / 32;
  std::vector<int64_t> ws(ns, 0);
  int64_t wmax = 0, sum = 0;
  for (int64_t sl = 0; sl < ns; ++sl) {
    int64_t w = 0;
    for (int64_t r = 32 * sl; r < std::min(n, 32 * sl + 32); ++r)
      w = std::max<int64_t>(w, H.rowptr[r + 1] - H.rowptr[r]);
    ws[sl] = w;
    wmax = std::max(wmax, w);
    sum += w;
  }
  const bool uniform = uniform_slack > 0 && ns > 0 && wmax * ns <= (1.0 + uniform_slack) * sum;
  if (width) *width = uniform ? wmax : 0;
  off.assign(ns + 1, 0);
  for (int64_t sl = 0; sl < ns; ++sl) off[sl + 1] = off[sl] + 32 * (uniform ? wmax : ws[sl]);
  ci.assign(off[ns], 0);
  for (int64_t r = 0; r < n; ++r) {
    const int64_t sl = r >> 5, t = r & 31, w = (off[sl + 1] - off[sl]) / 32;
    const int64_t len = H.rowptr[r + 1] - H.rowptr[r];
    for (int64_t u = 0; u < w; ++u)
      ci[off[sl] + 32 * u + t] = u < len ? H.col[H.rowptr[r] + u] : (square ? (int32_t)r : 0);
  }
}

// Values of a CSR matrix with dimv values per entry (vals, entry-major) in
// the SELL-32 layout off: component c of slot u of row 32 s + t at
// (off[s] + 32 u) dimv + 32 c + t; padding slots hold 0.
template <typename T>
std::vector<T> sell_values(const HostCsr& H, const std::vector<int64_t>& off, const double* vals,
                           int dimv) {
  std::vector<T> v(off.back() * dimv, T(0));
  for (int64_t r = 0; r < H.nrow; ++r) {
    const int64_t sl = r >> 5, t = r & 31;
    for (int64_t u = 0; u < H.rowptr[r + 1] - H.rowptr[r]; ++u)
      for (int c = 0; c < dimv; ++c)
        v[(off[sl] + 32 * u) * dimv + 32 * c + t] = (T)vals[(H.rowptr[r] + u) * dimv + c];
  }
  return v;
}

template <typename T>
int upload_sell(fs_problem* P, const HostCsr& H, DSell<T>& d, double uniform_slack = 0.0) {
  std::vector<int64_t> off;
  std::vector<int32_t> ci;
  int64_t width = 0;
  sell_layout(H, off, ci, uniform_slack, &width);
  std::vector<T> v = sell_values<T>(H, off, H.val.data(), 1);
  int64_t* doff;
  int32_t* dci;
  T* dv;
  FS_TRY(P->upload(&doff, off));
  FS_TRY(P->upload(&dci, ci));
  FS_TRY(P->upload(&dv, v));
  d.nrow = H.nrow;
  d.off = doff;
  d.ci = dci;
  d.v = dv;
  d.width = width;
  return FS_OK;
}

// Chebyshev(3) coefficients on [lmax/8, 1.1 lmax] of D^-1 A.
template <typename T>
void cheb_coeffs(double lmax, DLevel<T>& L, double ratio = 8.0) {
  double hi = 1.1 * lmax, lo = hi / ratio;
  L.lmax = lmax;
  double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  double sigma = theta / delta;
  double rho0 = 1.0 / sigma;
  double rho1 = 1.0 / (2.0 * sigma - rho0);
  double rho2 = 1.0 / (2.0 * sigma - rho1);
  L.inv_theta = 1.0 / theta;
  L.a1 = rho1 * rho0;
  L.b1 = 2.0 * rho1 / delta;
  L.a2 = rho2 * rho1;
  L.b2 = 2.0 * rho2 / delta;
}

// Inverse of a coarsest operator too large for the host (set-up only):
// Gauss-Jordan with partial pivoting on the device in FP64, in temporary
// device memory; the result, in the solver's precision, goes to *out.  It
// is accepted only if A times it is the identity to within the solver
// precision's rounding on four sampled columns.
template <typename T>
int invert_on_device(fs_problem* P, const HostCsr& A, T** out) {
  const int64_t n = A.nrow;
  if (n < 1 || n > 65535) {
    set_error("coarsest operator of unsupported size for the device inverse");
    return FS_ERR_UNSUPPORTED;
  }
  cudaStream_t s = P->stream;
  std::vector<double> W((size_t)(n * 2 * n), 0.0);
  for (int64_t r = 0; r < n; ++r) {
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) W[r * 2 * n + A.col[k]] += A.val[k];
    W[r * 2 * n + n + r] = 1.0;
  }
  double *dW = nullptr, *pval = nullptr;
  int64_t* piv = nullptr;
  int* bad = nullptr;
  auto release = [&]() {
    for (void* q : {(void*)dW, (void*)pval, (void*)piv, (void*)bad})
      if (q) cudaFreeAsync(q, s);
    cudaStreamSynchronize(s);
  };
  cudaError_t e = cudaMallocAsync((void**)&dW, sizeof(double) * W.size(), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&pval, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&piv, sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&bad, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dW, W.data(), sizeof(double) * W.size(),
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    release();
    set_error(std::string("device inverse: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FS_ERR_OOM : FS_ERR_CUDA;
  }
  for (int64_t c = 0; c < n; ++c) launch_gj_step(dW, n, c, piv, pval, bad, s);
  int rc = P->alloc(out, n * n);
  if (rc == FS_OK) launch_gj_extract<T>(dW, n, *out, s);
  int hbad = 0;
  std::vector<T> inv;
  if (rc == FS_OK) {
    inv.resize((size_t)(n * n));
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(inv.data(), *out, sizeof(T) * inv.size(), cudaMemcpyDeviceToHost, s);
  }
  release();
  if (rc != FS_OK) return rc;
  FS_TRY(check_launch("device inverse"));
  double err = hbad ? INFINITY : 0.0;
  for (int64_t k : {(int64_t)0, n / 3, (2 * n) / 3, n - 1}) {
    for (int64_t r = 0; r < n && std::isfinite(err); ++r) {
      double y = 0;
      for (int32_t q = A.rowptr[r]; q < A.rowptr[r + 1]; ++q)
        y += A.val[q] * (double)inv[(size_t)(A.col[q] * n + k)];
      err = std::max(err, std::fabs(y - (r == k ? 1.0 : 0.0)));
    }
  }
  const double tol = std::is_same<T, float>::value ? 1e-2 : 1e-8;
  if (!(err <= tol)) {
    set_error("device inverse of the coarsest operator failed its check (singular or "
              "too badly conditioned)");
    return FS_ERR_NUMERIC;
  }
  return FS_OK;
}

template <typename T>
int upload_hierarchy(fs_problem* P, const UnionHierarchy& U, int nc, DHier<T>& D) {
  const HostHierarchy& H = U.H;
  D.nlev = (int)H.levels.size();
  D.ncp = nc == 3 ? 4 : nc;
  if (D.nlev > 16) {
    set_error("multigrid hierarchy deeper than 16 levels");
    return FS_ERR_UNSUPPORTED;
  }
  for (int l = 0; l < D.nlev; ++l) {
    const HostLevel& hl = H.levels[l];
    DLevel<T>& dl = D.lev[l];
    // level operators: one slice width where padding costs at most 15%
    // more slots (the structured P1 levels); the class-ordered P2 level
    // keeps its per-slice widths
    FS_TRY(upload_sell<T>(P, hl.A, dl.A, 0.15));
    if (l + 1 < D.nlev) {
      FS_TRY(upload_csr<T>(P, hl.P, dl.P));
      FS_TRY(upload_csr<T>(P, hl.R, dl.R));
    }
    std::vector<T> di(hl.dinv.begin(), hl.dinv.end());
    T* dinv;
    FS_TRY(P->upload(&dinv, di));
    dl.dinv = dinv;
    cheb_coeffs<T>(hl.lmax, dl);
    const int64_t rows = hl.A.nrow;
    // batches: the segment (instance) of every 32-row slice of the level,
    // -1 where a slice spans two instances
    if (l < (int)U.inst_off.size() && U.inst_off[l].size() > 2) {
      const std::vector<int64_t>& off = U.inst_off[l];
      const int64_t nsl = (rows + 31) / 32;
      std::vector<int32_t> ss(nsl);
      for (int64_t q = 0; q < nsl; ++q) {
        const int64_t r0 = 32 * q, r1 = std::min(rows, r0 + 32) - 1;
        const auto seg = [&](int64_t r) {
          return (int32_t)(std::upper_bound(off.begin(), off.end(), r) - off.begin() - 1);
        };
        const int32_t g0 = seg(r0);
        ss[q] = g0 == seg(r1) ? g0 : -1;
      }
      int32_t* dss;
      FS_TRY(P->upload(&dss, ss));
      dl.skip.slice_seg = dss;
    }
    // padded components stay zero
    for (T** v : {&D.b[l], &D.G0[l], &D.G1[l], &D.D0[l], &D.D1[l]}) {
      FS_TRY(P->alloc(v, (int64_t)D.ncp * rows));
      FS_CUDA(cudaMemsetAsync(*v, 0, sizeof(T) * D.ncp * rows, P->stream));
    }
  }
  T* cinv;
  if (!U.dense.empty()) {
    std::vector<T> ci(U.dense.begin(), U.dense.end());
    FS_TRY(P->upload(&cinv, ci));
  } else {
    FS_TRY(invert_on_device<T>(P, U.H.levels.back().A, &cinv));
  }
  D.cinv = cinv;
  int32_t* rb;
  int64_t *br, *bn, *bd;
  FS_TRY(P->upload(&rb, U.row_blk));
  FS_TRY(P->upload(&br, U.blk_row));
  FS_TRY(P->upload(&bn, U.blk_n));
  FS_TRY(P->upload(&bd, U.blk_dense));
  D.row_blk = rb;
  D.blk_row = br;
  D.blk_n = bn;
  D.blk_dense = bd;
  D.ncoarse = H.ncoarse;
  D.dense_nb0 = U.blk_n.size() == 1 ? H.ncoarse : 0;
  if (!U.perm.empty()) {
    std::vector<int32_t> inv(U.perm.size());
    for (size_t r = 0; r < U.perm.size(); ++r) inv[U.perm[r]] = (int32_t)r;
    int32_t *pm, *ip;
    FS_TRY(P->upload(&pm, U.perm));
    FS_TRY(P->upload(&ip, inv));
    D.perm = pm;
    D.iperm = ip;
  }
  DHier<T>* dev;
  FS_TRY(P->alloc(&dev, 1));
  D.dev = dev;
  return FS_OK;
}

// Slot-group depths of the SpMV (this precision's operator; the FP64
// residual operator of the refinement keeps its default) and of the
// smoothing passes; the device copies of the hierarchies are refreshed by
// apply_tail.
template <typename T>
void apply_groups(fs_problem* P, Precision<T>& pr, const fs_schedule& sc) {
  (void)P;
  pr.op.group = sc.spmv_group;
  pr.HA.group = pr.HK.group = sc.smooth_group ? sc.smooth_group : 4;
  pr.HA.coarse_deg = pr.HK.coarse_deg = sc.coarse_degree ? sc.coarse_degree : 2;
  pr.HA.fine_deg = pr.HK.fine_deg = sc.fine_degree ? sc.fine_degree : 2;
  const int ratio = sc.cheb_ratio ? sc.cheb_ratio : 8;
  if (ratio != pr.cheb_ratio) {
    for (DHier<T>* H : {&pr.HA, &pr.HK})
      for (int l = 0; l < H->nlev; ++l) cheb_coeffs<T>(H->lev[l].lmax, H->lev[l], ratio);
    pr.cheb_ratio = ratio;
  }
}

// The fused cluster kernel takes the levels with at most tail_rows rows
// (from the first such level that still has a level below it; 0 = none);
// the device copy of the hierarchy is refreshed.
template <typename T>
int apply_tail(fs_problem* P, DHier<T>& D, int64_t tail_rows) {
  D.tail = -1;
  // (the fused cluster tail smooths with degree 2 or 3)
  if (tail_rows > 0 && D.coarse_deg != 1 && D.fine_deg != 1)
    for (int l = 0; l + 1 < D.nlev; ++l)
      if (D.lev[l].A.nrow <= tail_rows) {
        D.tail = l;
        break;
      }
  if (D.tail >= 0) D.tail_cluster = mg_tail_cluster<T>(D.ncp);
  FS_CUDA(cudaMemcpyAsync((void*)D.dev, &D, sizeof(DHier<T>), cudaMemcpyHostToDevice,
                          P->stream));
  FS_CUDA(cudaStreamSynchronize(P->stream));
  return FS_OK;
}

// The work-list of the persistent preconditioner for the hierarchies' current
// coarse smoothing degree (built and uploaded on first use).
template <typename T>
int apply_flow(fs_problem* P, Precision<T>& pr) {
  const int idx = flow_index(pr.HA, pr.HK);
  FlowDev& f = pr.flow[idx];
  // a work-list holds the smoothing coefficients it was built with: one
  // built for another interval is replaced (its buffers stay with the
  // problem until it is destroyed)
  if (f.items && pr.flow_ratio[idx] == pr.cheb_ratio) return FS_OK;
  pr.flow_ratio[idx] = pr.cheb_ratio;
  const int nb = flow_blocks<T>(pr.HA.ncp);
  if (nb <= 0) {
    set_error("persistent preconditioner: its kernel cannot be resident on this device");
    return FS_ERR_UNSUPPORTED;
  }
  FlowHost h;
  build_flow<T>(pr.HA, pr.HK, pr.offA, pr.offK, pr.prow, nb, h);
  unsigned char* ph;
  FlowItem* it;
  int32_t* need;
  unsigned *cnt, *ticket;
  FS_TRY(P->upload(&ph, h.phases));
  FS_TRY(P->upload(&it, h.items));
  FS_TRY(P->upload(&need, h.need));
  FS_TRY(P->alloc(&cnt, (int64_t)h.need.size()));
  FS_TRY(P->alloc(&ticket, 1));
  FS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * h.need.size(), P->stream));
  FS_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), P->stream));
  FS_CUDA(cudaStreamSynchronize(P->stream));  // host sources go out of scope
  f.phases = ph;
  f.items = it;
  f.nitems = (int64_t)h.items.size();
  f.cnt = cnt;
  f.need = need;
  f.ticket = ticket;
  f.nphase = h.nphase;
  f.nseg = P->nseg;
  f.nblocks = nb;
  return FS_OK;
}

// One application of the block preconditioner on r into z: the per-pass
// launches, or the persistent kernel when the schedule asks for it (st: the
// segment states whose done instances are skipped, or null).
template <typename T>
void issue_precond(fs_problem* P, Precision<T>& pr, const DHier<T>& HA, const DHier<T>& HK,
                   JVec<const T> r, JVec<T> z, const SegState* st, const int* skip,
                   cudaStream_t q) {
  if (P->sched.persistent_precond)
    launch_precond_flow<T>(pr.flow[flow_index(HA, HK)], pr.op, HA, pr.mplinv_nu,
                           1.0 / P->desc.dt, r, z, pr.kr.work_p, st,
                           pr.kr.st, skip, q);
  else {
    PcdView<T> pcd;
    if (P->sched.schur) pcd = PcdView<T>{P->dm.rpK, P->dm.ciK, pr.Np, pr.invm};
    launch_precond<T>(pr.op, HA, HK, pr.mplinv_nu, 1.0 / P->desc.dt, r,
                      z, pr.kr.work_p, pr.kr.work_u, skip, q, pcd);
  }
}

// Work-list over the n_dof entries: for every instance its vertex and edge
// ranges in each component block and its pressure range, cut into tiles of
// at most kTileLen entries; tiles of one instance are consecutive.
void build_tiles(const fs_problem* P, int sms, std::vector<Tile>& tiles,
                 std::vector<int>& first, std::vector<int>& count) {
  const Mesh& me = P->mesh->m;
  const int d = P->dim;
  struct Range {
    int64_t start, len;
    int seg;
  };
  std::vector<Range> ranges;
  for (int s = 0; s < P->nseg; ++s) {
    const Instance& I = me.inst[s];
    for (int c = 0; c < d; ++c) {
      ranges.push_back({c * me.n2 + I.voff, I.nv, s});
      ranges.push_back({c * me.n2 + me.nv + I.eoff, I.ne, s});
    }
    ranges.push_back({(int64_t)d * me.n2 + I.voff, I.nv, s});
  }
  // tile length: one block per tile in the Krylov passes.  With fewer than
  // four tiles of kTileLen per SM the SMs holding one tile more than others
  // set the time, so the count is brought to at most a multiple of the SM
  // count (every SM then holds the same number): the smallest multiple of
  // 32 whose count fits that bound.  With more tiles the imbalance is small
  // and longer tiles cost less overhead.
  auto ntiles_for = [&](int64_t L) {
    int64_t k = 0;
    for (const Range& r : ranges) k += (r.len + L - 1) / L;
    return k;
  };
  int64_t total = 0;
  for (const Range& r : ranges) total += r.len;
  const int64_t S = std::max(1, sms);
  const int64_t waves = std::max<int64_t>(1, (total + S * kTileLen - 1) / (S * kTileLen));
  int64_t L = kTileLen;
  const bool balance = ntiles_for(kTileLen) < 4 * S;
  for (int64_t w = waves; balance && L == kTileLen && w < waves + 4; ++w) {
    const int64_t bound = S * w;
    for (int64_t c = 32; c <= kTileLen; c += 32)
      if (ntiles_for(c) <= bound) {
        L = c;
        break;
      }
    if (ntiles_for(L) <= bound) break;
  }
  // ranges are in segment order, so the tiles of a segment are consecutive
  tiles.clear();
  first.assign(P->nseg, 0);
  count.assign(P->nseg, 0);
  int seg = -1;
  for (const Range& r : ranges) {
    for (; seg < r.seg; ++seg) first[seg + 1] = (int)tiles.size();
    for (int64_t o = 0; o < r.len; o += L) {
      Tile t;
      t.start = r.start + o;
      t.len = (int32_t)std::min<int64_t>(L, r.len - o);
      t.seg = r.seg;
      tiles.push_back(t);
      count[r.seg] += 1;
    }
  }
  for (; seg + 1 < P->nseg; ++seg) first[seg + 1] = (int)tiles.size();
}

template <typename V>
int alloc_krylov(fs_problem* P, Krylov<V>& K, int m, const std::vector<int>& first,
                 const std::vector<int>& count) {
  K.m = m;
  K.n = P->ndof;
  FS_TRY(P->alloc(&K.Vb, (int64_t)(m + 1) * K.n));
  FS_TRY(P->alloc(&K.Z, (int64_t)m * K.n));
  FS_TRY(P->alloc(&K.work_p, P->nv));
  FS_TRY(P->alloc(&K.work_u, (int64_t)P->dim * P->n2));
  FS_TRY(P->alloc(&K.rhs, K.n));
  FS_TRY(P->alloc(&K.sol, K.n));
  FS_TRY(P->alloc(&K.partial, (int64_t)(kMaxRestart + 1) * P->ntiles));
  FS_TRY(P->alloc(&K.st, P->nseg));
  FS_TRY(P->alloc(&K.ctl, 1));
  FS_CUDA(cudaMemsetAsync(K.st, 0, sizeof(SegState) * P->nseg, P->stream));
  std::vector<SegHost> init(P->nseg);
  std::memset(init.data(), 0, sizeof(SegHost) * init.size());
  for (int s = 0; s < P->nseg; ++s) {
    init[s].first_tile = first[s];
    init[s].ntiles = count[s];
  }
  FS_CUDA(cudaMemcpy2DAsync(K.st, sizeof(SegState), init.data(), sizeof(SegHost),
                            sizeof(SegHost), P->nseg, cudaMemcpyHostToDevice, P->stream));
  KCtl c{m, P->nseg, 0, 0, 0};
  FS_CUDA(cudaMemcpyAsync(K.ctl, &c, sizeof(KCtl), cudaMemcpyHostToDevice, P->stream));
  FS_CUDA(cudaStreamSynchronize(P->stream));  // host sources go out of scope
  return FS_OK;
}

// Pressure vertices whose Poisson rows are fixed in the preconditioner: the
// pinned vertex when the whole boundary is Dirichlet, else the vertices on
// the sides with a natural (do-nothing) velocity condition.  Local ids.
std::vector<int32_t> poisson_fixed(const fs_mesh_desc& d, bool pin) {
  std::vector<int32_t> out;
  const int dim = d.dim;
  const int all = dim == 2 ? 0x0F : 0x3F;
  int natural = all & ~d.dirichlet_sides;
  if (natural == 0) {
    if (pin) out.push_back(0);
    return out;
  }
  const int* n = d.n;
  int64_t sx = n[0] + 1, sy = n[1] + 1;
  int64_t nv = sx * sy * (dim == 3 ? (n[2] + 1) : 1);
  for (int64_t v = 0; v < nv; ++v) {
    int64_t ijk[3] = {v % sx, (v / sx) % sy, dim == 3 ? v / (sx * sy) : 0};
    int bits = 0;
    for (int a = 0; a < dim; ++a) {
      if (ijk[a] == 0) bits |= 1 << (2 * a);
      if (ijk[a] == n[a]) bits |= 1 << (2 * a + 1);
    }
    if ((bits & natural) && !(bits & d.dirichlet_sides)) out.push_back((int32_t)v);
  }
  return out;
}

// The iteration-path operator of one precision from its SELL-32 values.
template <typename T>
void set_op(fs_problem* P, DOp<T>& op, const T* A, const T* B, const T* BT, const T* diagp) {
  op.dim = P->dim;
  op.n2 = P->n2;
  op.nv = P->nv;
  op.A = {P->n2, P->offA, P->sciA, A};
  op.B = {P->nv, P->offB, P->sciB, B};
  op.BT = {P->n2, P->offBT, P->sciBT, BT};
  op.diagp = diagp;
}

template <typename T>
int setup_precision(fs_problem* P, Precision<T>& pr, const UnionHierarchy& HA,
                    const UnionHierarchy& HK, const std::vector<double>& mplinv_nu, int m,
                    const std::vector<int>& first, const std::vector<int>& count) {
  FS_TRY(upload_hierarchy<T>(P, HA, P->dim, pr.HA));
  FS_TRY(upload_hierarchy<T>(P, HK, 1, pr.HK));
  pr.offA = HA.inst_off;
  pr.offK = HK.inst_off;
  pr.prow = HK.inst_off[0];  // vertices are numbered instance by instance
  FS_TRY(apply_tail<T>(P, pr.HA, P->sched.tail_rows_velocity));
  FS_TRY(apply_tail<T>(P, pr.HK, P->sched.tail_rows_pressure));
  apply_groups<T>(P, pr, P->sched);
  std::vector<T> mi(mplinv_nu.begin(), mplinv_nu.end());
  FS_TRY(P->upload(&pr.mplinv_nu, mi));
  FS_TRY(alloc_krylov<T>(P, pr.kr, m, first, count));
  // batches: the union kernels skip the rows of instances that have
  // converged in the running cycle
  if (P->nseg > 1) {
    for (DHier<T>* H : {&pr.HA, &pr.HK})
      for (int l = 0; l < H->nlev; ++l)
        if (H->lev[l].skip.slice_seg) H->lev[l].skip.st = pr.kr.st;
    pr.op.skip_u = {P->slice_seg_u, pr.kr.st};
    pr.op.skip_p = {P->slice_seg_p, pr.kr.st};
  }
  return FS_OK;
}

// ---------------------------------------------------------------------------
// Device parts of a solve (enqueued on the problem's stream)
// ---------------------------------------------------------------------------
template <typename T>
void issue_check(fs_problem* P, Precision<T>& pr, const T* x, const T* b) {
  Krylov<T>& K = pr.kr;
  cudaStream_t s = P->stream;
  launch_spmv_full<T, T>(pr.op, x, b, K.Vb, 1, nullptr, s);
  launch_seg_norm<T>(K.Vb, P->tl(), K.st, K.partial, 0, s);
}

// One restart cycle: init (tolerances relative to ||b|| or to beta), v0,
// up to m Arnoldi steps, update of x.  Launched directly, the m steps are
// issued one by one (steps after convergence exit at once).  Captured in a
// graph, one step is captured as the body of a conditional WHILE node whose
// condition the device sets (the cycle init, then every step's Givens
// kernel), so the graph runs exactly the steps the cycle needs.
template <typename T>
int issue_iter(fs_problem* P, Precision<T>& pr, T* x, int relative_to_beta) {
  Krylov<T>& K = pr.kr;
  cudaStream_t s = P->stream;
  const int64_t n = K.n;
  const TileList tl = P->tl();
  const bool loop = g_capturing;
  // Steps launched directly run to m and exit at once after convergence,
  // through the cycle's all-done flag.  The loop node runs its body only
  // while that flag is clear (the condition is checked before every pass),
  // so captured steps skip the check and the load it costs each kernel.
  const int* skip = loop ? nullptr : &K.ctl->all_done;
  cudaGraphConditionalHandle cond = 0;
  if (loop) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg;
    FS_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
    FS_CUDA(cudaGraphConditionalHandleCreate(&cond, cg, 0, 0));
  }
  launch_seg_cycle_init(K.st, K.ctl, relative_to_beta, cond, s);
  launch_seg_scale<T>(K.Vb, tl, K.st, 0, s);
  const int* jp = &K.ctl->j;
  auto step = [&](cudaStream_t q) {
    const JVec<const T> vj(K.Vb, jp, n);
    const JVec<T> zj(K.Z, jp, n);
    const JVec<const T> zjc(K.Z, jp, n);
    const JVec<T> w(K.Vb + n, jp, n);
    issue_precond<T>(P, pr, pr.HA, pr.HK, vj, zj, P->nseg > 1 ? K.st : nullptr, skip, q);
    launch_spmv_full<T, T>(pr.op, zjc, nullptr, w, 0, skip, q, /*seg=*/true);
    // one segment: the Givens step rides in the second CGS2 pass
    const bool fuse = P->nseg == 1;
    launch_seg_cgs2<T>(K.Vb, n, tl, K.st, K.ctl, K.partial, fuse, cond, q);
    if (!fuse) launch_seg_givens(K.st, K.ctl, P->nseg, cond, q);
  };
  if (loop) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    FS_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cn;
    FS_CUDA(cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    FS_CUDA(cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1,
                                                cudaStreamSetCaptureDependencies));
    FS_CUDA(cudaStreamBeginCaptureToGraph(P->side, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    step(P->side);
    cudaGraph_t got;
    FS_CUDA(cudaStreamEndCapture(P->side, &got));
    FS_CUDA(cudaGraphGetNodes(body, nullptr, &K.n_body));
  } else {
    for (int j = 0; j < K.m; ++j) step(s);
  }
  launch_seg_update_x<T, T>(K.st, K.ctl, K.Z, n, tl, x, s);
  return FS_OK;
}

// Runs `issue` directly or as a cached CUDA graph (keyed by x and b).
template <typename T>
int run_graph(fs_problem* P, Krylov<T>& K, bool check, const void* x, const void* b,
              bool use_graph, const std::function<int()>& issue) {
  if (!use_graph) {
    FS_TRY(issue());
    return check_launch("gmres cycle");
  }
  if (K.g_x != x || K.g_b != b) {
    if (K.g_check) cudaGraphExecDestroy(K.g_check);
    if (K.g_iter) cudaGraphExecDestroy(K.g_iter);
    K.g_check = K.g_iter = nullptr;
    K.g_x = x;
    K.g_b = b;
  }
  cudaGraphExec_t* g = check ? &K.g_check : &K.g_iter;
  size_t* nodes = check ? &K.n_check : &K.n_iter;
  if (!*g) {
    cudaGraph_t graph;
    FS_CUDA(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    int rc = issue();
    g_capturing = false;
    cudaError_t ec = cudaStreamEndCapture(P->stream, &graph);
    if (rc != FS_OK) {
      if (ec == cudaSuccess) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) {
      set_error(std::string("graph capture: ") + cudaGetErrorString(ec));
      return FS_ERR_CUDA;
    }
    // kernel nodes at the top level (a loop node counts as one)
    cudaGraphGetNodes(graph, nullptr, nodes);
    cudaError_t e = cudaGraphInstantiate(g, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      return FS_ERR_CUDA;
    }
  }
  FS_CUDA(cudaGraphLaunch(*g, P->stream));
  count_launches((int64_t)*nodes);
  return FS_OK;
}

// Status read-back (64 bytes per segment) and the completion event.
template <typename T>
int enqueue_status(fs_problem* P, Krylov<T>& K) {
  FS_CUDA(cudaMemcpy2DAsync(P->host_status, sizeof(SegHost), K.st, sizeof(SegState),
                            sizeof(SegHost), P->nseg, cudaMemcpyDeviceToHost, P->stream));
  FS_CUDA(cudaEventRecord(P->ev, P->stream));
  return FS_OK;
}

template <typename T>
int push_retired(fs_problem* P, Krylov<T>& K) {
  for (int s = 0; s < P->nseg; ++s) P->host_retired[s] = P->ctx.retired[s];
  FS_CUDA(cudaMemcpy2DAsync(&K.st[0].retired, sizeof(SegState), P->host_retired, sizeof(int),
                            sizeof(int), P->nseg, cudaMemcpyHostToDevice, P->stream));
  return FS_OK;
}

// Per-segment cycle targets (read by the cycle-init kernel).
template <typename T>
int push_rtol(fs_problem* P, Krylov<T>& K, const std::vector<double>& rtol) {
  for (int s = 0; s < P->nseg; ++s) P->host_rtol[s] = rtol[s];
  FS_CUDA(cudaMemcpy2DAsync(&K.st[0].rtol, sizeof(SegState), P->host_rtol, sizeof(double),
                            sizeof(double), P->nseg, cudaMemcpyHostToDevice, P->stream));
  return FS_OK;
}

// The Oseen system of the step to t_next: convecting field w (the state
// when null; a Picard iterate otherwise) and the previous time level u_old in
// the load (the state when null).
// Problems whose convecting field is a given constant (the polynomial
// exactness problems), not the state.
bool const_w(const fs_problem* P) {
  return P->desc.problem == FS_PROBLEM_POLY_OSEEN || P->desc.problem == FS_PROBLEM_POLY_OSEEN_T ||
         P->desc.problem == FS_PROBLEM_POLY3;
}

// The pressure convection matrix of the convection-diffusion Schur part,
// for the convecting field w (or the constant wc), in FP64 and, for the
// FP32 inner solves, converted to FP32.
void assemble_np(fs_problem* P, const double* w, const double* wc) {
  cudaStream_t s = P->stream;
  const int64_t nnz = P->mesh->m.Kp.nnz();
  cudaMemsetAsync(P->Np64, 0, sizeof(double) * nnz, s);
  launch_assemble_conv_p1(P->dm, w, P->n2, wc, P->pfix, P->Np64, s);
  if (P->has32) launch_convert<double, float>(P->Np64, P->p32.Np, nnz, nullptr, 0, s);
}

int assemble_impl(fs_problem* P, double t_next, const double* w = nullptr,
                  const double* u_old = nullptr) {
  cudaStream_t s = P->stream;
  const Mesh& me = P->mesh->m;
  const int64_t nnzA = me.A.nnz();
  if (!w) w = P->x;
  if (!u_old) u_old = P->x;
  const bool constw = const_w(P);
  if (P->p3) {
    const int64_t nnz3 = P->p3nnzA;
    FS_CUDA(cudaMemcpyAsync(P->valA, P->baseA, sizeof(double) * nnz3, cudaMemcpyDeviceToDevice,
                            s));
    launch_p3_conv(P->dm, P->p3ref, constw ? nullptr : w, P->n2,
                   constw ? P->desc.wconst : nullptr, P->valA, s);
    launch_bc_rows<double>(P->dm, P->valA, s);
    launch_eval_load(P->dm, P->ph, t_next, 1.0 / P->desc.dt, u_old, P->F, s);
    launch_rhs(P->dm, P->ph, t_next, P->Mv, P->F, P->pinned, P->npinned, P->b, s);
    FS_TRY(check_launch("P3/P2 assembly"));
    P->assembled = true;
    return FS_OK;
  }
  FS_CUDA(cudaMemcpyAsync(P->valA, P->baseA, sizeof(double) * nnzA, cudaMemcpyDeviceToDevice, s));
  launch_assemble_conv(P->dm, me.color_ptr, constw ? nullptr : w, P->n2,
                       constw ? P->desc.wconst : nullptr, P->valA, P->desc.deterministic != 0, s);
  launch_bc_rows<double>(P->dm, P->valA, s);
  launch_eval_load(P->dm, P->ph, t_next, 1.0 / P->desc.dt, u_old, P->F, s);
  launch_rhs(P->dm, P->ph, t_next, P->Mv, P->F, P->pinned, P->npinned, P->b, s);
  launch_csr_to_sell(P->n2, P->dm.rpA, P->valA, P->offA, P->sA64, P->has32 ? P->sA32 : nullptr,
                     s);
  if (P->sched.schur) assemble_np(P, constw ? nullptr : w, constw ? P->desc.wconst : nullptr);
  FS_TRY(check_launch("assembly"));
  P->assembled = true;
  return FS_OK;
}

// ---------------------------------------------------------------------------
// The solve state machine.  start_solve enqueues the first device part;
// advance() runs once that part's event has completed: it reads the
// per-segment status and enqueues the next part (or finishes).
// ---------------------------------------------------------------------------
int start_solve(fs_problem* P, double* x) {
  SolveCtx& c = P->ctx;
  const int S = P->nseg;
  c.x = x;
  c.status.assign(S, FS_OK);
  c.iters.assign(S, 0);
  c.cycles.assign(S, 0);
  c.refines.assign(S, 0);
  c.relres.assign(S, 0.0);
  c.prev.assign(S, INFINITY);
  c.retired.assign(S, 0);
  cudaStream_t s = P->stream;
  if (P->desc.precision == FS_PREC_FP64) {
    Krylov<double>& K = P->p64.kr;
    FS_TRY(push_retired(P, K));
    launch_seg_norm<double>(P->b, P->tl(), K.st, K.partial, 1, s);
    FS_TRY(run_graph<double>(P, K, true, x, P->b, c.o.use_graph != 0, [&]() {
      issue_check<double>(P, P->p64, x, P->b);
      return FS_OK;
    }));
    FS_TRY(enqueue_status(P, K));
    c.phase = PH_CHECK;
  } else {
    Krylov<float>& K = P->p32.kr;
    FS_TRY(push_retired(P, K));
    launch_seg_norm<double>(P->b, P->tl(), K.st, K.partial, 1, s);
    launch_spmv_full<double, double>(P->p64.op, x, P->b, P->r64, 1, nullptr, s);
    launch_seg_norm<double>(P->r64, P->tl(), K.st, K.partial, 2, s);
    FS_TRY(enqueue_status(P, K));
    c.phase = PH_RES64;
  }
  return check_launch("solve start");
}

void finish_solve(fs_problem* P) {
  SolveCtx& c = P->ctx;
  P->last_stats.assign(P->nseg, fs_solve_stats{});
  for (int s = 0; s < P->nseg; ++s) {
    fs_solve_stats& st = P->last_stats[s];
    st.iters = c.iters[s];
    st.refinements = c.refines[s];
    st.cycles = c.cycles[s];
    st.status = c.status[s];
    st.rel_res = c.relres[s];
  }
  c.rc = FS_OK;
  for (int s = 0; s < P->nseg; ++s)
    if (c.status[s] != FS_OK && c.rc == FS_OK) c.rc = c.status[s];
  if (c.rc != FS_OK) set_error("the solve did not reach rtol in every instance");
  c.phase = PH_DONE;
}

fs_solve_stats aggregate_stats(const fs_problem* P) {
  fs_solve_stats a{};
  for (const auto& st : P->last_stats) {
    a.iters = std::max(a.iters, st.iters);
    a.refinements = std::max(a.refinements, st.refinements);
    a.cycles = std::max(a.cycles, st.cycles);
    a.rel_res = std::max(a.rel_res, st.rel_res);
    if (a.status == FS_OK) a.status = st.status;
  }
  return a;
}

// Per segment, after its true residual r (beta, or rnorm in the refinement)
// is known: converged, stagnated at the rounding floor (accepted within
// 100 rtol), out of budget, or continue.  Returns true when every segment
// is retired.
bool retire_segments(fs_problem* P, bool refinement) {
  SolveCtx& c = P->ctx;
  const double rtol = c.o.rtol;
  bool all = true;
  for (int s = 0; s < P->nseg; ++s) {
    if (c.retired[s]) continue;
    const SegHost& h = P->host_status[s];
    const double bn = h.bnorm > 0 ? h.bnorm : 1.0;
    const double r = refinement ? h.rnorm : h.beta;
    c.relres[s] = r / bn;
    if (!std::isfinite(r)) {
      c.status[s] = FS_ERR_NUMERIC;
      c.retired[s] = 1;
    } else if (r <= rtol * bn) {
      c.retired[s] = 1;
    } else if (r > (refinement ? 0.5 : 0.9) * c.prev[s]) {
      c.retired[s] = 1;
      if (r > 100.0 * rtol * bn) c.status[s] = FS_ERR_NOT_CONVERGED;
    } else if (c.iters[s] >= c.o.max_iter || (refinement && c.refines[s] >= c.o.max_refine)) {
      c.retired[s] = 1;
      c.status[s] = FS_ERR_NOT_CONVERGED;
    }
    c.prev[s] = r;
    if (!c.retired[s]) all = false;
  }
  return all;
}

// Kernels run by a graph's Arnoldi loop node: the body ran until every
// segment was done, i.e. as many times as the most steps a segment took.
template <typename T>
void count_body_launches(fs_problem* P, const Krylov<T>& K, bool graph) {
  if (!graph) return;
  int kmax = 0;
  for (int q = 0; q < P->nseg; ++q)
    if (!P->ctx.retired[q]) kmax = std::max(kmax, P->host_status[q].k);
  count_launches((int64_t)K.n_body * kmax);
}

int advance(fs_problem* P) {
  SolveCtx& c = P->ctx;
  cudaStream_t s = P->stream;
  const bool graph = c.o.use_graph != 0;
  switch (c.phase) {
    case PH_CHECK: {  // FP64: true residual known
      if (retire_segments(P, false)) {
        finish_solve(P);
        return FS_OK;
      }
      Krylov<double>& K = P->p64.kr;
      FS_TRY(push_retired(P, K));
      FS_TRY(push_rtol(P, K, std::vector<double>(P->nseg, c.o.rtol)));
      FS_TRY(run_graph<double>(P, K, false, c.x, P->b, graph,
                               [&]() { return issue_iter<double>(P, P->p64, c.x, 0); }));
      FS_TRY(enqueue_status(P, K));
      c.phase = PH_ITER;
      return FS_OK;
    }
    case PH_ITER: {
      count_body_launches(P, P->p64.kr, graph);
      for (int q = 0; q < P->nseg; ++q) {
        if (c.retired[q]) continue;
        c.iters[q] += P->host_status[q].k;
        c.cycles[q] += 1;
        if (P->host_status[q].bad) {
          c.status[q] = P->host_status[q].bad == 2 ? FS_ERR_TIMEOUT : FS_ERR_NUMERIC;
          c.retired[q] = 1;
        } else if (P->host_status[q].k == 0) {
          c.status[q] = FS_ERR_NOT_CONVERGED;
          c.retired[q] = 1;
        }
      }
      Krylov<double>& K = P->p64.kr;
      FS_TRY(push_retired(P, K));
      FS_TRY(run_graph<double>(P, K, true, c.x, P->b, graph, [&]() {
        issue_check<double>(P, P->p64, c.x, P->b);
        return FS_OK;
      }));
      FS_TRY(enqueue_status(P, K));
      c.phase = PH_CHECK;
      return FS_OK;
    }
    case PH_RES64: {  // refinement: FP64 residual known
      if (retire_segments(P, true)) {
        finish_solve(P);
        return FS_OK;
      }
      Precision<float>& pr = P->p32;
      Krylov<float>& K = pr.kr;
      FS_TRY(push_retired(P, K));
      // One inner cycle per refinement, whose Arnoldi estimate stops at a
      // target relative to its own initial residual: inner_rtol, or the
      // reduction still missing to reach rtol (with a 0.3 margin) when that
      // is less, so the last refinement does not run a full cycle.  The
      // FP32 operator limits what one refinement gains (about 1e-5 here),
      // so deeper targets only cost iterations.
      {
        std::vector<double> tgt(P->nseg, c.o.inner_rtol);
        for (int q = 0; q < P->nseg; ++q) {
          const SegHost& h = P->host_status[q];
          const double bn = h.bnorm > 0 ? h.bnorm : 1.0;
          if (!c.retired[q] && h.rnorm > 0)
            tgt[q] = std::min(0.5, std::max(c.o.inner_rtol, 0.3 * c.o.rtol * bn / h.rnorm));
        }
        FS_TRY(push_rtol(P, K, tgt));
      }
      launch_seg_normalise<double, float>(P->r64, K.rhs, P->tl(), K.st, s);
      FS_CUDA(cudaMemsetAsync(K.sol, 0, sizeof(float) * P->ndof, s));
      FS_TRY(run_graph<float>(P, K, false, K.sol, K.rhs, graph, [&]() {
        issue_check<float>(P, pr, K.sol, K.rhs);
        return issue_iter<float>(P, pr, K.sol, 1);
      }));
      launch_seg_axpy<float, double>(c.x, K.sol, P->tl(), K.st, s);
      launch_spmv_full<double, double>(P->p64.op, c.x, P->b, P->r64, 1, nullptr, s);
      launch_seg_norm<double>(P->r64, P->tl(), K.st, K.partial, 2, s);
      FS_TRY(enqueue_status(P, K));
      for (int q = 0; q < P->nseg; ++q)
        if (!c.retired[q]) c.refines[q] += 1;
      c.phase = PH_INNER;
      return check_launch("refinement");
    }
    case PH_INNER: {  // inner cycle finished and FP64 residual recomputed
      count_body_launches(P, P->p32.kr, graph);
      for (int q = 0; q < P->nseg; ++q) {
        if (c.retired[q]) continue;
        c.iters[q] += P->host_status[q].k;
        c.cycles[q] += 1;
        if (P->host_status[q].bad) {
          c.status[q] = P->host_status[q].bad == 2 ? FS_ERR_TIMEOUT : FS_ERR_NUMERIC;
          c.retired[q] = 1;
        }
      }
      c.phase = PH_RES64;
      return advance(P);
    }
    default:
      return FS_OK;
  }
}

// Blocking drive of the state machine until the solve is done.
int run_solve(fs_problem* P, double* x) {
  FS_TRY(start_solve(P, x));
  while (P->ctx.phase != PH_DONE) {
    FS_CUDA(cudaEventSynchronize(P->ev));
    FS_TRY(advance(P));
  }
  return P->ctx.rc;
}

// Captured CUDA graphs depend on the schedule: drop them.
template <typename T>
void drop_graphs(Krylov<T>& K) {
  if (K.g_check) cudaGraphExecDestroy(K.g_check);
  if (K.g_iter) cudaGraphExecDestroy(K.g_iter);
  K.g_check = K.g_iter = nullptr;
  K.g_x = K.g_b = nullptr;
}

template <typename T>
int install_schedule(fs_problem* P, Precision<T>& pr, const fs_schedule& sc) {
  apply_groups<T>(P, pr, sc);
  FS_TRY(apply_tail<T>(P, pr.HA, sc.tail_rows_velocity));
  FS_TRY(apply_tail<T>(P, pr.HK, sc.tail_rows_pressure));
  if (sc.persistent_precond) FS_TRY(apply_flow<T>(P, pr));
  drop_graphs(pr.kr);
  return FS_OK;
}

int install_schedule(fs_problem* P, const fs_schedule& sc) {
  if (sc.schur && !P->Np64) {
    const int64_t nnz = P->mesh->m.Kp.nnz();
    FS_TRY(P->alloc(&P->Np64, nnz));
    P->p64.Np = P->Np64;
    if (P->has32) FS_TRY(P->alloc(&P->p32.Np, nnz));
  }
  const bool fresh_np = sc.schur && !P->sched.schur;
  if (P->desc.precision == FS_PREC_FP64)
    FS_TRY(install_schedule<double>(P, P->p64, sc));
  else
    FS_TRY(install_schedule<float>(P, P->p32, sc));
  P->sched = sc;
  // a system assembled before gets its pressure convection from the state
  if (fresh_np && P->assembled) {
    assemble_np(P, const_w(P) ? nullptr : P->x, const_w(P) ? P->desc.wconst : nullptr);
    FS_TRY(check_launch("pressure convection"));
  }
  return FS_OK;
}

// One application of the block preconditioner (mean over a CUDA graph of
// `reps` applications on the Krylov scratch vectors, after one warm launch).
template <typename T>
int time_precond(fs_problem* P, Precision<T>& pr, int reps, int persistent, double* ms) {
  Krylov<T>& K = pr.kr;
  cudaStream_t s = P->stream;
  FS_CUDA(cudaMemsetAsync(K.Vb, 0, sizeof(T) * K.n, s));
  cudaGraph_t g;
  FS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  g_capturing = true;
  const DHier<T> HA = without_skip(pr.HA), HK = without_skip(pr.HK);
  const int saved = P->sched.persistent_precond;
  P->sched.persistent_precond = persistent;
  for (int i = 0; i < reps; ++i) issue_precond<T>(P, pr, HA, HK, K.Vb, K.Z, nullptr, nullptr, s);
  P->sched.persistent_precond = saved;
  g_capturing = false;
  FS_CUDA(cudaStreamEndCapture(s, &g));
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  cudaGraphExec_t ge;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return FS_ERR_CUDA;
  }
  cudaEvent_t e0, e1;
  FS_CUDA(cudaEventCreate(&e0));
  FS_CUDA(cudaEventCreate(&e1));
  FS_CUDA(cudaGraphLaunch(ge, s));
  FS_CUDA(cudaEventRecord(e0, s));
  for (int i = 0; i < 3; ++i) FS_CUDA(cudaGraphLaunch(ge, s));
  FS_CUDA(cudaEventRecord(e1, s));
  FS_CUDA(cudaEventSynchronize(e1));
  float t = 0;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  count_launches((int64_t)nodes * 4);
  FS_TRY(check_launch("preconditioner timing"));
  *ms = t / (3.0 * reps);
  return FS_OK;
}

int time_precond(fs_problem* P, int reps, int persistent, double* ms) {
  if (P->desc.precision == FS_PREC_FP64)
    return time_precond<double>(P, P->p64, reps, persistent, ms);
  return time_precond<float>(P, P->p32, reps, persistent, ms);
}

// One saddle-point SpMV in the solver arithmetic (mean of `reps` launches
// on the Krylov scratch vectors, after 3 warm-up launches).
template <typename T>
int time_spmv(fs_problem* P, Precision<T>& pr, int reps, double* ms) {
  cudaStream_t s = P->stream;
  auto launch = [&]() {
    launch_spmv_full<T, T>(pr.op, pr.kr.Vb, nullptr, pr.kr.Vb + P->ndof, 0, nullptr, s);
  };
  cudaEvent_t e0, e1;
  FS_CUDA(cudaEventCreate(&e0));
  FS_CUDA(cudaEventCreate(&e1));
  for (int i = 0; i < 3; ++i) launch();
  FS_CUDA(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) launch();
  FS_CUDA(cudaEventRecord(e1, s));
  FS_CUDA(cudaEventSynchronize(e1));
  float t = 0;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FS_TRY(check_launch("SpMV timing"));
  *ms = t / reps;
  return FS_OK;
}

int time_spmv(fs_problem* P, int reps, double* ms) {
  if (P->desc.precision == FS_PREC_FP64) return time_spmv<double>(P, P->p64, reps, ms);
  return time_spmv<float>(P, P->p32, reps, ms);
}

int solve_opts(const fs_solve_opts* opts, fs_solve_opts& o) {
  fs_default_solve_opts(&o);
  if (opts) o = *opts;
  if (o.restart != 30) {
    set_error("the library runs GMRES(30) restart cycles (restart must be 30)");
    return FS_ERR_UNSUPPORTED;
  }
  return FS_OK;
}

// Sets the calling thread's launch mode from the problem's schedule for the
// duration of one API call.
struct OverlapScope {
  int old;
  explicit OverlapScope(const fs_problem* P) : old(g_overlap) {
    g_overlap = (P && P->sched.serial_launches) ? 0 : 1;
  }
  ~OverlapScope() { g_overlap = old; }
};

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* fs_last_error(void) { return fs::g_err.c_str(); }

void fs_default_solve_opts(fs_solve_opts* o) {
  if (!o) return;
  o->restart = 30;
  o->max_iter = 2000;
  o->rtol = 1e-14;
  o->inner_rtol = 1e-5;
  o->max_refine = 30;
  o->use_graph = 1;
}

int fs_mesh_create(const fs_mesh_desc* desc, fs_mesh** out) {
  return fs_mesh_create_batch(desc, 1, out);
}

int fs_mesh_create_batch(const fs_mesh_desc* descs, int count, fs_mesh** out) {
  if (!descs || !out || count < 1) {
    set_error("fs_mesh_create: null argument or count < 1");
    return FS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  auto* h = new (std::nothrow) fs_mesh;
  if (!h) return FS_ERR_OOM;
  int rc = count == 1 ? build_mesh(descs[0], h->m) : build_batch_mesh(descs, count, h->m);
  if (rc != FS_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return FS_OK;
}

int fs_mesh_destroy(fs_mesh* mesh) {
  delete mesh;
  return FS_OK;
}

int fs_mesh_instances(const fs_mesh* mesh, int64_t* offsets) {
  if (!mesh) {
    set_error("fs_mesh_instances: null mesh");
    return -FS_ERR_INVALID_ARG;
  }
  const Mesh& m = mesh->m;
  if (offsets)
    for (size_t i = 0; i < m.inst.size(); ++i) {
      offsets[6 * i + 0] = m.inst[i].voff;
      offsets[6 * i + 1] = m.inst[i].nv;
      offsets[6 * i + 2] = m.nv + m.inst[i].eoff;
      offsets[6 * i + 3] = m.inst[i].ne;
      offsets[6 * i + 4] = m.inst[i].coff;
      offsets[6 * i + 5] = m.inst[i].ncell;
    }
  return (int)m.inst.size();
}

int fs_dof_map(const fs_mesh* mesh, fs_dofmap_info* info, double* coords, int32_t* cell2dof,
               int64_t* rowptr, int32_t* col, uint8_t* dirichlet) {
  if (!mesh || !info) {
    set_error("fs_dof_map: null argument");
    return FS_ERR_INVALID_ARG;
  }
  const Mesh& m = mesh->m;
  info->dim = m.dim;
  info->nloc = m.nloc;
  info->n_vert = m.nv;
  info->n_edge = m.ne;
  info->n_p2 = m.n2;
  info->n_cell = m.ncell;
  info->n_dof = m.dim * m.n2 + m.nv;
  info->nnz_a = m.A.nnz();
  info->nnz_b = m.B.nnz();
  info->nnz = m.dim * (m.A.nnz() + m.BT.nnz() + m.B.nnz()) + m.nv;
  if (coords) std::memcpy(coords, m.coords.data(), sizeof(double) * m.coords.size());
  if (cell2dof || dirichlet || rowptr || col) {
    // the device works in an internal node order; this is the paper's
    std::vector<int32_t> c2d, ci;
    std::vector<uint8_t> dir;
    std::vector<int64_t> rp;
    natural_dof_map(m, cell2dof ? &c2d : nullptr, dirichlet ? &dir : nullptr,
                    rowptr ? &rp : nullptr, col ? &ci : nullptr);
    if (cell2dof) std::memcpy(cell2dof, c2d.data(), sizeof(int32_t) * c2d.size());
    if (dirichlet) std::memcpy(dirichlet, dir.data(), dir.size());
    if (rowptr) std::memcpy(rowptr, rp.data(), sizeof(int64_t) * rp.size());
    if (col) std::memcpy(col, ci.data(), sizeof(int32_t) * ci.size());
  }
  return FS_OK;
}

int fs_problem_create(fs_mesh* mesh, const fs_problem_desc* desc, void* stream,
                      fs_problem** out) {
  if (!mesh || !desc) {
    set_error("fs_problem_create: null argument");
    return FS_ERR_INVALID_ARG;
  }
  // one description for every instance of the mesh
  std::vector<fs_problem_desc> d(mesh->m.inst.size(), *desc);
  return fs_problem_create_batch(mesh, d.data(), (int)d.size(), stream, out);
}

int fs_problem_create_p3(fs_mesh* mesh, const fs_problem_desc* desc, void* stream,
                         fs_problem** out) {
  if (!mesh || !desc || !out) {
    set_error("fs_problem_create_p3: null argument");
    return FS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const Mesh& me = mesh->m;
  const fs_problem_desc& d = *desc;
  if (me.dim != 2 || me.inst.size() != 1) {
    set_error("fs_problem_create_p3: P3/P2 problems need a single 2D mesh");
    return FS_ERR_UNSUPPORTED;
  }
  if (!(d.dt > 0) || !std::isfinite(d.dt) || !(d.nu > 0) || d.problem < 0 || d.problem > 6 ||
      d.problem == FS_PROBLEM_CUBE) {
    set_error("fs_problem_create_p3: need a finite dt > 0, nu > 0 and a 2D problem kind");
    return FS_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    set_error("fs_problem_create_p3: no CUDA device");
    return FS_ERR_CUDA;
  }
  P3Tables T;
  FS_TRY(build_p3_tables(me, T));
  std::unique_ptr<fs_problem> P(new fs_problem);
  P->mesh = mesh;
  P->desc = d;
  P->inst_desc.assign(1, d);
  P->nseg = 1;
  P->dim = 2;
  P->p3 = true;
  P->n2 = T.n3;
  P->nv = T.np;
  P->ndof = 2 * T.n3 + T.np;
  P->t = d.t0;
  if (stream) {
    P->stream = (cudaStream_t)stream;
  } else {
    FS_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    P->own_stream = true;
  }
  FS_CUDA(cudaEventCreateWithFlags(&P->ev, cudaEventDisableTiming));
  cudaStream_t s = P->stream;
  DMesh& dm = P->dm;
  dm.dim = 2;
  dm.nloc = 10;
  dm.nb = 6;
  dm.nv = T.np;
  dm.n2 = T.n3;
  dm.ncell = T.ncell;
  dm.ndir = (int64_t)T.dlist.size();
  {
    int32_t *c2u, *dl, *c2p;
    double *xyz, *pxyz;
    uint8_t* dir;
    FS_TRY(P->upload(&c2u, T.c2u));
    FS_TRY(P->upload(&xyz, T.xyz));
    FS_TRY(P->upload(&dir, T.dir));
    FS_TRY(P->upload(&dl, T.dlist));
    FS_TRY(P->upload(&c2p, T.c2p));
    FS_TRY(P->upload(&pxyz, T.pxyz));
    dm.c2d = c2u; dm.p2xyz = xyz; dm.dirichlet = dir; dm.dlist = dl;
    P->c2p = c2p;
    P->pxyz = pxyz;
    int32_t *a, *b, *c, *e, *f, *g, *h, *k;
    FS_TRY(P->upload(&a, T.A.rowptr)); FS_TRY(P->upload(&b, T.A.col));
    FS_TRY(P->upload(&c, T.B.rowptr)); FS_TRY(P->upload(&e, T.B.col));
    FS_TRY(P->upload(&f, T.BT.rowptr)); FS_TRY(P->upload(&g, T.BT.col));
    FS_TRY(P->upload(&h, T.Kp.rowptr)); FS_TRY(P->upload(&k, T.Kp.col));
    dm.rpA = a; dm.ciA = b; dm.rpB = c; dm.ciB = e; dm.rpBT = f; dm.ciBT = g;
    dm.rpK = h; dm.ciK = k;
    uint8_t *pa, *pb, *pbt, *pk;
    FS_TRY(P->upload(&pa, T.posA)); FS_TRY(P->upload(&pb, T.posB));
    FS_TRY(P->upload(&pbt, T.posBT)); FS_TRY(P->upload(&pk, T.posK));
    dm.posA = pa; dm.posB = pb; dm.posBT = pbt; dm.posK = pk;
    static RefP3 ref;
    static bool have_ref = false;
    static std::mutex ref_mu;
    {
      std::lock_guard<std::mutex> lk(ref_mu);
      if (!have_ref) {
        p3_ref_tensors(ref);
        have_ref = true;
      }
    }
    std::vector<RefP3> rv(1, ref);
    FS_TRY(P->upload(&P->p3ref, rv));
  }
  P->ph.kind = d.problem;
  P->ph.nu = d.nu;
  for (int a = 0; a < 3; ++a) P->ph.wconst[a] = d.wconst[a];
  const int64_t nnzA = T.A.nnz(), nnzB = T.B.nnz(), nnzBT = T.BT.nnz(), nnzK = T.Kp.nnz();
  P->p3nnzA = nnzA;
  FS_TRY(P->alloc(&P->baseA, nnzA));
  FS_TRY(P->alloc(&P->Mv, nnzA));
  FS_TRY(P->alloc(&P->valA, nnzA));
  FS_TRY(P->alloc(&P->B, nnzB * 2));
  FS_TRY(P->alloc(&P->BT, nnzBT * 2));
  FS_TRY(P->alloc(&P->Kp, nnzK));
  for (auto pr : {std::make_pair(P->baseA, nnzA), std::make_pair(P->Mv, nnzA),
                  std::make_pair(P->B, nnzB * 2), std::make_pair(P->BT, nnzBT * 2),
                  std::make_pair(P->Kp, nnzK)})
    FS_CUDA(cudaMemsetAsync(pr.first, 0, sizeof(double) * pr.second, s));
  launch_p3_base(dm, P->c2p, P->p3ref, 1.0 / d.dt, d.nu, P->baseA, P->Mv, P->B, P->BT, P->Kp,
                 s);
  FS_TRY(check_launch("P3/P2 step-invariant blocks"));
  if (d.pin_pressure) {
    std::vector<int32_t> pin(1, 0);
    FS_TRY(P->upload(&P->pinned, pin));
    P->npinned = 1;
    P->pinned_host = pin;
  }
  FS_TRY(P->alloc(&P->x, P->ndof));
  FS_TRY(P->alloc(&P->b, P->ndof));
  FS_TRY(P->alloc(&P->F, 2 * T.n3));
  launch_p3_exact_state(dm, P->ph, d.t0, d.init == 1, P->pxyz, P->x, s);
  FS_TRY(check_launch("P3/P2 initial state"));
  FS_CUDA(cudaStreamSynchronize(s));
  *out = P.release();
  return FS_OK;
}

int fs_problem_sizes(const fs_problem* P, int64_t* sizes) {
  if (!P || !sizes) {
    set_error("fs_problem_sizes: null argument");
    return FS_ERR_INVALID_ARG;
  }
  sizes[0] = P->n2;
  sizes[1] = P->nv;
  sizes[2] = P->ndof;
  return FS_OK;
}

int fs_problem_create_batch(fs_mesh* mesh, const fs_problem_desc* descs, int count,
                            void* stream, fs_problem** out) {
  if (!mesh || !descs || !out) {
    set_error("fs_problem_create: null argument");
    return FS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const Mesh& me = mesh->m;
  if (count != (int)me.inst.size()) {
    set_error("fs_problem_create_batch: one description per mesh instance is required");
    return FS_ERR_INVALID_ARG;
  }
  const fs_problem_desc& d0 = descs[0];
  for (int i = 0; i < count; ++i) {
    const fs_problem_desc& d = descs[i];
    if (!(d.dt > 0) || !(d.nu > 0) || d.problem < 0 || d.problem > 6 ||
        (d.precision != FS_PREC_FP64 && d.precision != FS_PREC_FP32_REFINE)) {
      set_error("fs_problem_create: need dt > 0, nu > 0, a known problem and precision");
      return FS_ERR_INVALID_ARG;
    }
    if (d.problem != d0.problem || d.dt != d0.dt || d.t0 != d0.t0 ||
        d.precision != d0.precision || d.init != d0.init ||
        std::memcmp(d.wconst, d0.wconst, sizeof(d.wconst)) != 0 ||
        d.deterministic != d0.deterministic) {
      set_error("fs_problem_create_batch: instances may differ only in nu and pin_pressure");
      return FS_ERR_INVALID_ARG;
    }
  }
  if ((d0.problem == FS_PROBLEM_CUBE) != (me.dim == 3) && d0.problem != FS_PROBLEM_POLY_OSEEN &&
      d0.problem != FS_PROBLEM_POLY_OSEEN_T) {
    set_error("fs_problem_create: problem kind does not match the mesh dimension");
    return FS_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    set_error("fs_problem_create: no CUDA device");
    return FS_ERR_CUDA;
  }
  std::unique_ptr<fs_problem> P(new fs_problem);
  P->mesh = mesh;
  P->desc = d0;
  P->inst_desc.assign(descs, descs + count);
  P->nseg = count;
  P->dim = me.dim;
  P->n2 = me.n2;
  P->nv = me.nv;
  P->ndof = me.dim * me.n2 + me.nv;
  P->t = d0.t0;
  if (stream) {
    P->stream = (cudaStream_t)stream;
  } else {
    FS_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    P->own_stream = true;
  }
  FS_CUDA(cudaEventCreateWithFlags(&P->ev, cudaEventDisableTiming));
  FS_CUDA(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
  FS_CUDA(cudaMallocHost(&P->host_status, sizeof(SegHost) * count));
  FS_CUDA(cudaMallocHost(&P->host_retired, sizeof(int) * count));
  FS_CUDA(cudaMallocHost(&P->host_rtol, sizeof(double) * count));
  std::call_once(g_ref_once, []() {
    ref_tensors(2, g_ref2);
    ref_tensors(3, g_ref3);
  });
  upload_ref_tensors(g_ref2, g_ref3);
  FS_TRY(check_launch("upload reference tensors"));

  // mesh tables
  DMesh& dm = P->dm;
  dm.dim = me.dim;
  dm.nloc = me.nloc;
  dm.nb = me.nb;
  dm.nv = me.nv;
  dm.n2 = me.n2;
  dm.ncell = me.ncell;
  dm.ndir = (int64_t)me.dlist.size();
  {
    int32_t* c2d; double* xyz; uint8_t* dir; int32_t* dl;
    FS_TRY(P->upload(&c2d, me.c2d));
    FS_TRY(P->upload(&xyz, me.p2xyz));
    FS_TRY(P->upload(&dir, me.dirichlet));
    FS_TRY(P->upload(&dl, me.dlist));
    dm.c2d = c2d; dm.p2xyz = xyz; dm.dirichlet = dir; dm.dlist = dl;
    int32_t *a, *b, *c, *d, *e, *f, *g, *h;
    FS_TRY(P->upload(&a, me.A.rowptr)); FS_TRY(P->upload(&b, me.A.col));
    FS_TRY(P->upload(&c, me.B.rowptr)); FS_TRY(P->upload(&d, me.B.col));
    FS_TRY(P->upload(&e, me.BT.rowptr)); FS_TRY(P->upload(&f, me.BT.col));
    FS_TRY(P->upload(&g, me.Kp.rowptr)); FS_TRY(P->upload(&h, me.Kp.col));
    dm.rpA = a; dm.ciA = b; dm.rpB = c; dm.ciB = d; dm.rpBT = e; dm.ciBT = f;
    dm.rpK = g; dm.ciK = h;
    uint8_t *pa, *pb, *pbt, *pk;
    FS_TRY(P->upload(&pa, me.posA)); FS_TRY(P->upload(&pb, me.posB));
    FS_TRY(P->upload(&pbt, me.posBT)); FS_TRY(P->upload(&pk, me.posKp));
    dm.posA = pa; dm.posB = pb; dm.posBT = pbt; dm.posK = pk;
    int32_t* cc;
    FS_TRY(P->upload(&cc, me.color_cells));
    dm.color_cells = cc;
  }
  P->ph.kind = d0.problem;
  P->ph.nu = d0.nu;
  for (int a = 0; a < 3; ++a) P->ph.wconst[a] = d0.wconst[a];
  bool varnu = false;
  for (int i = 1; i < count; ++i) varnu = varnu || descs[i].nu != d0.nu;
  std::vector<double> nu_vert(me.nv, d0.nu);
  if (varnu) {
    std::vector<double> nu_cell(me.ncell), nu_node(me.n2);
    for (int i = 0; i < count; ++i) {
      const Instance& I = me.inst[i];
      for (int64_t c = 0; c < I.ncell; ++c) nu_cell[I.coff + c] = descs[i].nu;
      for (int64_t j = 0; j < I.n2(); ++j) nu_node[union_node(me, i, j)] = descs[i].nu;
      for (int64_t v = 0; v < I.nv; ++v) nu_vert[I.voff + v] = descs[i].nu;
    }
    double *nc, *nn;
    FS_TRY(P->upload(&nc, nu_cell));
    FS_TRY(P->upload(&nn, nu_node));
    dm.nu_cell = nc;
    P->ph.nu_node = nn;
  }

  // step-invariant blocks
  const int64_t nnzA = me.A.nnz(), nnzB = me.B.nnz(), nnzBT = me.BT.nnz(), nnzK = me.Kp.nnz();
  const int dim = me.dim;
  FS_TRY(P->alloc(&P->baseA, nnzA));
  FS_TRY(P->alloc(&P->Mv, nnzA));
  FS_TRY(P->alloc(&P->valA, nnzA));
  FS_TRY(P->alloc(&P->B, nnzB * dim));
  FS_TRY(P->alloc(&P->BT, nnzBT * dim));
  FS_TRY(P->alloc(&P->Kp, nnzK));
  FS_TRY(P->alloc(&P->mpl, P->nv));
  FS_TRY(P->alloc(&P->diagp, P->nv));
  cudaStream_t s = P->stream;
  FS_CUDA(cudaMemsetAsync(P->baseA, 0, sizeof(double) * nnzA, s));
  FS_CUDA(cudaMemsetAsync(P->Mv, 0, sizeof(double) * nnzA, s));
  FS_CUDA(cudaMemsetAsync(P->B, 0, sizeof(double) * nnzB * dim, s));
  FS_CUDA(cudaMemsetAsync(P->BT, 0, sizeof(double) * nnzBT * dim, s));
  FS_CUDA(cudaMemsetAsync(P->Kp, 0, sizeof(double) * nnzK, s));
  FS_CUDA(cudaMemsetAsync(P->mpl, 0, sizeof(double) * P->nv, s));
  launch_assemble_base(dm, me.color_ptr, 1.0 / d0.dt, d0.nu, P->baseA, P->Mv, P->B, P->BT, P->Kp,
                       P->mpl, s);
  FS_TRY(check_launch("assemble_base"));
  HostCsr A0 = me.A, Kp = me.Kp;
  A0.val.resize(nnzA);
  Kp.val.resize(nnzK);
  std::vector<double> Bh(nnzB * dim), BTh(nnzBT * dim), mplh(P->nv);
  FS_CUDA(cudaMemcpyAsync(A0.val.data(), P->baseA, sizeof(double) * nnzA, cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaMemcpyAsync(Kp.val.data(), P->Kp, sizeof(double) * nnzK, cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaMemcpyAsync(Bh.data(), P->B, sizeof(double) * Bh.size(), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaMemcpyAsync(BTh.data(), P->BT, sizeof(double) * BTh.size(), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaMemcpyAsync(mplh.data(), P->mpl, sizeof(double) * P->nv, cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  // boundary rows: Dirichlet velocity rows -> identity in A0, zero in BT;
  // pinned pressure rows -> zero B row, unit diagonal
  for (int32_t i : me.dlist) {
    for (int32_t k = A0.rowptr[i]; k < A0.rowptr[i + 1]; ++k) A0.val[k] = (A0.col[k] == i) ? 1.0 : 0.0;
    for (int32_t k = me.BT.rowptr[i]; k < me.BT.rowptr[i + 1]; ++k)
      for (int c = 0; c < dim; ++c) BTh[(int64_t)k * dim + c] = 0.0;
  }
  std::vector<double> dp(P->nv, 0.0);
  std::vector<int32_t> pin, kfix;
  for (int i = 0; i < count; ++i) {
    const Instance& I = me.inst[i];
    if (descs[i].pin_pressure) pin.push_back((int32_t)I.voff);
    for (int32_t q : poisson_fixed(I.desc, descs[i].pin_pressure != 0))
      kfix.push_back((int32_t)(I.voff + q));
  }
  for (int32_t q : pin) {
    for (int32_t k = me.B.rowptr[q]; k < me.B.rowptr[q + 1]; ++k)
      for (int c = 0; c < dim; ++c) Bh[(int64_t)k * dim + c] = 0.0;
    dp[q] = 1.0;
  }
  if (!pin.empty()) {
    FS_TRY(P->upload(&P->pinned, pin));
    P->npinned = (int)pin.size();
    P->pinned_host = pin;
  }
  FS_CUDA(cudaMemcpyAsync(P->B, Bh.data(), sizeof(double) * Bh.size(), cudaMemcpyHostToDevice, s));
  FS_CUDA(cudaMemcpyAsync(P->BT, BTh.data(), sizeof(double) * BTh.size(), cudaMemcpyHostToDevice,
                          s));
  FS_CUDA(cudaMemcpyAsync(P->diagp, dp.data(), sizeof(double) * P->nv, cudaMemcpyHostToDevice, s));
  // pressure Poisson of the preconditioner with its fixed rows
  std::vector<double> invm(P->nv);
  {
    std::vector<uint8_t> fixed(P->nv, 0);
    for (int32_t q : kfix) fixed[q] = 1;
    for (int64_t q = 0; q < P->nv; ++q)
      for (int32_t k = Kp.rowptr[q]; k < Kp.rowptr[q + 1]; ++k)
        if (fixed[q] || fixed[Kp.col[k]]) Kp.val[k] = (Kp.col[k] == q) ? 1.0 : 0.0;
    FS_TRY(P->upload(&P->pfix, fixed));
    for (int64_t q = 0; q < P->nv; ++q) invm[q] = 1.0 / mplh[q];
  }
  // nu over the lumped pressure mass; a pinned vertex is marked by -1 (its
  // row of the preconditioner passes r_p through)
  std::vector<double> mplinv_nu(P->nv);
  for (int64_t q = 0; q < P->nv; ++q) mplinv_nu[q] = nu_vert[q] / mplh[q];
  for (int32_t q : P->pinned_host) mplinv_nu[q] = -1.0;
  UnionHierarchy HA, HK;
  // coarsest size.  Large problems stop coarsening at 3500 rows in 3D and
  // 2000 in 2D: the dense inverse (on the device, ~0.1 s of set-up) then
  // replaces the one or two latency-bound coarsest levels of each V-cycle
  // with one dense matvec.  In 2D a grid of 2000 to 3500 rows coarsened by
  // 4 once more is cheaper than that matvec (a 3,225 x 3,225 inverse is
  // 41.6 MB in FP32).  Small problems would pay the device inversion in
  // their set-up latency (the serving loop creates many), so they keep 800
  // rows; batches keep small per-instance blocks.
  const int64_t cmax = count > 1 ? 400 : me.n2 >= 100000 ? (me.dim == 3 ? 3500 : 2000) : 800;
  build_union_hierarchy(me, {}, A0, true, me.dlist, cmax, HA);
  build_union_hierarchy(me, {}, Kp, false, kfix, cmax, HK);

  // vectors, work-list
  FS_TRY(P->alloc(&P->x, P->ndof));
  for (double*& h : P->hist_buf) FS_TRY(P->alloc(&h, P->ndof));
  FS_TRY(P->alloc(&P->b, P->ndof));
  FS_TRY(P->alloc(&P->F, (int64_t)dim * P->n2));
  FS_TRY(P->alloc(&P->r64, P->ndof));
  std::vector<Tile> tiles;
  std::vector<int> first, tcount;
  int dev = 0, sms = 0;
  FS_CUDA(cudaGetDevice(&dev));
  FS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  build_tiles(P.get(), sms, tiles, first, tcount);
  FS_TRY(P->upload(&P->tiles, tiles));
  P->ntiles = (int)tiles.size();
  // SELL-32 blocks of the iteration path: layouts once, B and BT values
  // once (step-invariant), A values scattered after every assembly
  {
    std::vector<int64_t> oA, oB, oBT;
    std::vector<int32_t> cA, cB, cBT;
    sell_layout(me.A, oA, cA);
    sell_layout(me.B, oB, cB);
    sell_layout(me.BT, oBT, cBT);
    int64_t *a, *b, *c;
    int32_t *ca, *cb, *cc;
    FS_TRY(P->upload(&a, oA)); FS_TRY(P->upload(&ca, cA));
    FS_TRY(P->upload(&b, oB)); FS_TRY(P->upload(&cb, cB));
    FS_TRY(P->upload(&c, oBT)); FS_TRY(P->upload(&cc, cBT));
    P->offA = a; P->sciA = ca; P->offB = b; P->sciB = cb; P->offBT = c; P->sciBT = cc;
    FS_TRY(P->alloc(&P->sA64, oA.back()));
    FS_CUDA(cudaMemsetAsync(P->sA64, 0, sizeof(double) * oA.back(), s));
    FS_TRY(P->upload(&P->sB64, sell_values<double>(me.B, oB, Bh.data(), dim)));
    FS_TRY(P->upload(&P->sBT64, sell_values<double>(me.BT, oBT, BTh.data(), dim)));
    set_op<double>(P.get(), P->p64.op, P->sA64, P->sB64, P->sBT64, P->diagp);
    if (d0.precision == FS_PREC_FP32_REFINE) {
      P->has32 = true;
      FS_TRY(P->alloc(&P->sA32, oA.back()));
      FS_CUDA(cudaMemsetAsync(P->sA32, 0, sizeof(float) * oA.back(), s));
      FS_TRY(P->upload(&P->sB32, sell_values<float>(me.B, oB, Bh.data(), dim)));
      FS_TRY(P->upload(&P->sBT32, sell_values<float>(me.BT, oBT, BTh.data(), dim)));
      std::vector<float> d32(dp.begin(), dp.end());
      FS_TRY(P->upload(&P->diagp32, d32));
      set_op<float>(P.get(), P->p32.op, P->sA32, P->sB32, P->sBT32, P->diagp32);
    }
    int32_t* nat;
    FS_TRY(P->upload(&nat, me.node_nat));
    P->nat = nat;
  }
  if (count > 1) {
    std::vector<int32_t> own_u(me.n2), own_p(me.nv);
    for (int i = 0; i < count; ++i) {
      const Instance& I = me.inst[i];
      for (int64_t q = 0; q < I.nv; ++q) own_u[I.voff + q] = own_p[I.voff + q] = i;
      for (int64_t e = 0; e < I.ne; ++e) own_u[me.nv + I.eoff + e] = i;
    }
    const auto slices = [](const std::vector<int32_t>& own) {
      const int64_t n = (int64_t)own.size(), ns = (n + 31) / 32;
      std::vector<int32_t> ss(ns);
      for (int64_t q = 0; q < ns; ++q) {
        const int64_t r0 = 32 * q, r1 = std::min(n, r0 + 32);
        ss[q] = own[r0];
        for (int64_t r = r0 + 1; r < r1; ++r)
          if (own[r] != own[r0]) ss[q] = -1;
      }
      return ss;
    };
    int32_t *su, *sp;
    FS_TRY(P->upload(&su, slices(own_u)));
    FS_TRY(P->upload(&sp, slices(own_p)));
    P->slice_seg_u = su;
    P->slice_seg_p = sp;
  }
  const int m = 30;
  if (d0.precision == FS_PREC_FP64) {
    FS_TRY(setup_precision<double>(P.get(), P->p64, HA, HK, mplinv_nu, m, first, tcount));
    FS_TRY(P->upload(&P->p64.invm, invm));
  } else {
    FS_TRY(setup_precision<float>(P.get(), P->p32, HA, HK, mplinv_nu, m, first, tcount));
    std::vector<float> im(invm.begin(), invm.end());
    FS_TRY(P->upload(&P->p32.invm, im));
  }
  launch_exact_state(dm, P->ph, d0.t0, d0.init == 1, P->x, s);
  FS_TRY(check_launch("initial state"));
  FS_CUDA(cudaStreamSynchronize(s));
  *out = P.release();
  return FS_OK;
}

int fs_problem_destroy(fs_problem* prob) {
  delete prob;
  return FS_OK;
}

int64_t fs_problem_device_bytes(const fs_problem* prob) { return prob ? prob->bytes : 0; }

int fs_assemble_step(fs_problem* P, double t_next, double* val_out, double* b_out) {
  if (!P) {
    set_error("fs_assemble_step: null problem");
    return FS_ERR_INVALID_ARG;
  }
  if (P->p3 && (val_out || b_out)) {
    set_error("fs_assemble_step: no monolithic export for P3/P2 problems");
    return FS_ERR_UNSUPPORTED;
  }
  FS_TRY(assemble_impl(P, t_next));
  if (val_out) {
    if (!P->mrp) {
      // paper-order row pointers from the internal row lengths
      const Mesh& me = P->mesh->m;
      const int64_t n2 = me.n2, dim = me.dim;
      std::vector<int64_t> rp(P->ndof + 1, 0);
      for (int64_t q = 0; q < n2; ++q)
        for (int64_t c = 0; c < dim; ++c)
          rp[c * n2 + me.node_nat[q] + 1] =
              (me.A.rowptr[q + 1] - me.A.rowptr[q]) + (me.BT.rowptr[q + 1] - me.BT.rowptr[q]);
      for (int64_t q = 0; q < me.nv; ++q)
        rp[dim * n2 + q + 1] = dim * (me.B.rowptr[q + 1] - me.B.rowptr[q]) + 1;
      for (int64_t r = 0; r < P->ndof; ++r) rp[r + 1] += rp[r];
      FS_TRY(P->upload(&P->mrp, rp));
    }
    launch_expand_monolithic(P->dm, P->nat, P->valA, P->B, P->BT, P->diagp, P->mrp, val_out,
                             P->stream);
    FS_TRY(check_launch("expand_monolithic"));
  }
  if (b_out) {
    launch_dofs_perm(P->dm, P->nat, P->b, b_out, 1, P->stream);
    FS_TRY(check_launch("fs_assemble_step export"));
  }
  return FS_OK;
}

int fs_solve(fs_problem* P, const fs_solve_opts* opts, double* x, fs_solve_stats* stats) {
  OverlapScope overlap(P);
  if (P && P->p3) {
    set_error("fs_solve: P3/P2 problems are stepped by fs_step_ipcs");
    return FS_ERR_UNSUPPORTED;
  }
  if (!P) {
    set_error("fs_solve: null problem");
    return FS_ERR_INVALID_ARG;
  }
  if (!P->assembled) {
    set_error("fs_solve: call fs_assemble_step first");
    return FS_ERR_INVALID_ARG;
  }
  if (P->ctx.phase != PH_IDLE && P->ctx.phase != PH_DONE) {
    set_error("fs_solve: an asynchronous step is in progress");
    return FS_ERR_BUSY;
  }
  FS_TRY(solve_opts(opts, P->ctx.o));
  P->hist = 0;  // the state no longer follows the stepped history
  if (x) {  // the caller's vector is in paper order
    FS_TRY(nat_buffers(P));
    launch_dofs_perm(P->dm, P->nat, x, P->natbuf, 0, P->stream);
    FS_TRY(check_launch("fs_solve"));
  }
  int rc = run_solve(P, x ? P->natbuf : P->x);
  if (P->ctx.phase == PH_DONE && stats) *stats = aggregate_stats(P);
  P->ctx.phase = PH_IDLE;
  if (x) {
    launch_dofs_perm(P->dm, P->nat, P->natbuf, x, 1, P->stream);
    FS_TRY(check_launch("fs_solve"));
    FS_CUDA(cudaStreamSynchronize(P->stream));
  }
  return rc;
}

// Solve of the step whose system was just assembled (from the state x^n):
// the Krylov solve starts from the polynomial extrapolation in time through
// x^n and the hist previous states (order hist <= kExtrapMax; x^n itself on
// the first step of a history), whose residual is O(dt^(hist+1)) instead of
// the O(dt) of x^n.  The converged state does not depend on the starting
// point beyond the solver tolerance.  x^n goes to the ring slot after the
// newest one (the oldest, read first by the same thread).
static int start_step_solve(fs_problem* P) {
  const double* prev[kExtrapMax] = {};
  for (int j = 0; j < P->hist; ++j)
    prev[j] = P->hist_buf[(P->hist_head - j + kExtrapMax) % kExtrapMax];
  const int next = (P->hist_head + 1) % kExtrapMax;
  launch_extrapolate(P->x, prev, P->hist, P->hist_buf[next], P->ndof, P->stream);
  FS_TRY(check_launch("extrapolate"));
  P->hist_head = next;
  P->hist = P->hist < kExtrapMax ? P->hist + 1 : kExtrapMax;
  return start_solve(P, P->x);
}

int fs_step_begin(fs_problem* P, int nsteps, const fs_solve_opts* opts) {
  OverlapScope overlap(P);
  if (P && P->p3) {
    set_error("fs_step: P3/P2 problems are stepped by fs_step_ipcs");
    return FS_ERR_UNSUPPORTED;
  }
  if (!P || nsteps < 1) {
    set_error("fs_step_begin: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  if (P->ctx.phase != PH_IDLE && P->ctx.phase != PH_DONE) {
    set_error("fs_step_begin: a step is already in progress");
    return FS_ERR_BUSY;
  }
  if (!std::isfinite(P->desc.dt)) {
    set_error("fs_step_begin: a steady problem (dt = inf) is solved by fs_solve_steady");
    return FS_ERR_INVALID_ARG;
  }
  FS_TRY(solve_opts(opts, P->ctx.o));
  P->ctx.steps_left = nsteps;
  P->ctx.step_index = 0;
  P->ctx.per_step = nullptr;
  FS_TRY(assemble_impl(P, P->t + P->desc.dt));
  return start_step_solve(P);
}

int fs_step_poll(fs_problem* P, int wait, int* done) {
  OverlapScope overlap(P);
  if (!P || !done) {
    set_error("fs_step_poll: null argument");
    return FS_ERR_INVALID_ARG;
  }
  *done = 0;
  SolveCtx& c = P->ctx;
  if (c.phase == PH_IDLE) {
    *done = 1;
    return FS_OK;
  }
  while (true) {
    if (c.phase == PH_DONE) {
      fs_solve_stats st = aggregate_stats(P);
      if (c.per_step) c.per_step[c.step_index] = st;
      c.step_index += 1;
      P->t += P->desc.dt;  // the state holds the best iterate even on failure
      c.steps_left -= 1;
      if (c.rc != FS_OK || c.steps_left == 0) {
        int rc = c.rc;
        c.phase = PH_IDLE;
        c.per_step = nullptr;
        *done = 1;
        return rc;
      }
      FS_TRY(assemble_impl(P, P->t + P->desc.dt));
      FS_TRY(start_step_solve(P));
    }
    cudaError_t q = wait ? cudaEventSynchronize(P->ev) : cudaEventQuery(P->ev);
    if (q == cudaErrorNotReady) return FS_OK;
    if (q != cudaSuccess) {
      set_error(std::string("fs_step_poll: ") + cudaGetErrorString(q));
      return FS_ERR_CUDA;
    }
    FS_TRY(advance(P));
  }
}

int fs_step(fs_problem* P, int nsteps, const fs_solve_opts* opts, fs_solve_stats* per_step) {
  OverlapScope overlap(P);
  if (!P || nsteps < 0) {
    set_error("fs_step: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  if (nsteps == 0) return FS_OK;
  FS_TRY(fs_step_begin(P, nsteps, opts));
  P->ctx.per_step = per_step;
  int done = 0;
  int rc = FS_OK;
  while (!done) {
    rc = fs_step_poll(P, 1, &done);
    if (rc != FS_OK && !done) {
      // an error before the steps finished (a failed CUDA call, e.g. after a
      // device fault): give up on the remaining steps instead of polling on
      P->ctx.phase = PH_IDLE;
      P->ctx.per_step = nullptr;
      break;
    }
  }
  return rc;
}

// ---------------------------------------------------------------------------
// Picard iteration (paper Sec. 2.2.1: the nonlinear convection term
// linearised around the latest iterate, ((u^{k} . grad) u^{k+1}, v), one
// Oseen solve per iterate; Sec. 3.3: model.run(maxstep, tol) iterates until
// the update falls below tol).  The first iterate of a time step convects
// with u^n (so one iteration is exactly fs_step's Oseen step); every
// iterate keeps u^n in the backward-Euler load.
// ---------------------------------------------------------------------------
static int picard_buffers(fs_problem* P) {
  if (P->xn) return FS_OK;
  FS_TRY(P->alloc(&P->xn, P->ndof));
  FS_TRY(P->alloc(&P->wpic, P->ndof));
  FS_TRY(P->alloc(&P->nrm, diff_norms_scratch()));
  return FS_OK;
}

// Drives the solve state machine started by start_solve/start_step_solve to
// its end (blocking); returns the solve's status.
static int drive_solve(fs_problem* P) {
  while (P->ctx.phase != PH_DONE) {
    FS_CUDA(cudaEventSynchronize(P->ev));
    FS_TRY(advance(P));
  }
  return P->ctx.rc;
}

// The Picard iterates of one nonlinear system at t1.  extrapolate: start the
// first solve from the state history (a time step); steady problems start
// every solve from the latest iterate.
static int picard_iterate(fs_problem* P, double t1, bool extrapolate, double tol, int maxit,
                          fs_picard_stats* st) {
  cudaStream_t s = P->stream;
  const int64_t nvel = (int64_t)P->dim * P->n2;
  *st = fs_picard_stats{};
  FS_CUDA(cudaMemcpyAsync(P->xn, P->x, sizeof(double) * P->ndof, cudaMemcpyDeviceToDevice, s));
  int rc = FS_OK;
  for (int k = 0; k < maxit; ++k) {
    FS_CUDA(cudaMemcpyAsync(P->wpic, P->x, sizeof(double) * P->ndof, cudaMemcpyDeviceToDevice,
                            s));
    FS_TRY(assemble_impl(P, t1, P->wpic, P->xn));
    if (k == 0 && extrapolate)
      FS_TRY(start_step_solve(P));
    else
      FS_TRY(start_solve(P, P->x));
    rc = drive_solve(P);
    const fs_solve_stats ls = aggregate_stats(P);
    P->ctx.phase = PH_IDLE;
    st->picard_iters = k + 1;
    st->krylov_iters += ls.iters;
    st->rel_res = ls.rel_res;
    launch_diff_norms(P->x, P->wpic, nvel, P->nrm, s);
    FS_TRY(check_launch("picard update norm"));
    double h[2] = {0, 0};
    FS_CUDA(cudaMemcpyAsync(h, P->nrm, sizeof(h), cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
    const double du = std::sqrt(h[0]), un = std::sqrt(h[1]);
    st->update = du / std::max(1.0, un);
    if (rc != FS_OK) break;
    if (!std::isfinite(st->update)) {
      rc = FS_ERR_NUMERIC;
      break;
    }
    if (du <= tol * std::max(1.0, un)) break;
    if (k + 1 == maxit) rc = FS_ERR_NOT_CONVERGED;
  }
  st->status = rc;
  if (rc != FS_OK) set_error("Picard iteration: the nonlinear update did not reach tol");
  return rc;
}

static int picard_args(fs_problem* P, const fs_solve_opts* opts, double tol, int maxit,
                       const char* who) {
  if (P && P->p3) {
    set_error("Picard iteration: P3/P2 problems are stepped by fs_step_ipcs");
    return FS_ERR_UNSUPPORTED;
  }
  if (!P || !(tol > 0) || maxit < 1) {
    set_error(std::string(who) + ": bad argument");
    return FS_ERR_INVALID_ARG;
  }
  if (P->nseg != 1) {
    set_error(std::string(who) + ": batched problems are stepped by fs_step");
    return FS_ERR_UNSUPPORTED;
  }
  if (P->ctx.phase != PH_IDLE && P->ctx.phase != PH_DONE) {
    set_error(std::string(who) + ": a step is in progress");
    return FS_ERR_BUSY;
  }
  FS_TRY(solve_opts(opts, P->ctx.o));
  return picard_buffers(P);
}

int fs_step_picard(fs_problem* P, int nsteps, const fs_solve_opts* opts, double nl_tol,
                   int max_picard, fs_picard_stats* per_step) {
  OverlapScope overlap(P);
  FS_TRY(picard_args(P, opts, nl_tol, max_picard, "fs_step_picard"));
  if (nsteps < 0 || !std::isfinite(P->desc.dt)) {
    set_error("fs_step_picard: need nsteps >= 0 and a finite dt");
    return FS_ERR_INVALID_ARG;
  }
  for (int n = 0; n < nsteps; ++n) {
    fs_picard_stats st;
    const int rc = picard_iterate(P, P->t + P->desc.dt, true, nl_tol, max_picard, &st);
    P->t += P->desc.dt;
    if (per_step) per_step[n] = st;
    if (rc != FS_OK) return rc;
  }
  return FS_OK;
}

int fs_solve_steady(fs_problem* P, const fs_solve_opts* opts, double nl_tol, int max_picard,
                    fs_picard_stats* stats) {
  OverlapScope overlap(P);
  FS_TRY(picard_args(P, opts, nl_tol, max_picard, "fs_solve_steady"));
  if (!std::isinf(P->desc.dt)) {
    set_error("fs_solve_steady: create the problem with dt = inf (no mass term)");
    return FS_ERR_INVALID_ARG;
  }
  P->hist = 0;
  fs_picard_stats st;
  const int rc = picard_iterate(P, P->t, false, nl_tol, max_picard, &st);
  if (stats) *stats = st;
  return rc;
}

// ---------------------------------------------------------------------------
// Incremental pressure-correction stepping (paper Sec. 2.2.1, IPCS): three
// symmetric positive definite systems per step, each solved by CG in FP64
// (kernels in fs_ipcs.cu): Jacobi-preconditioned for the velocity stages,
// multigrid-preconditioned for the P2/P1 pressure stage.
// ---------------------------------------------------------------------------
static int ipcs_setup(fs_problem* P) {
  if (P->ip_us) return FS_OK;
  const int64_t nvel = (int64_t)P->dim * P->n2, nv = P->nv;
  for (double** v : {&P->ip_us, &P->ip_rhs, &P->ip_r, &P->ip_z, &P->ip_p, &P->ip_q, &P->ip_dA,
                     &P->ip_dM})
    FS_TRY(P->alloc(v, nvel));
  FS_TRY(P->alloc(&P->ip_dp, nv));
  FS_TRY(P->alloc(&P->ip_dK, nv));
  FS_TRY(P->alloc(&P->ip_part, ipcs_part_size(P->dm)));
  FS_TRY(P->alloc(&P->ip_sc, 4));
  FS_TRY(P->alloc(&P->ip_nrm, diff_norms_scratch()));
  std::vector<uint8_t> fixed(nv, 0);
  for (int32_t q : P->pinned_host) fixed[q] = 1;
  FS_TRY(P->upload(&P->ip_fixed, fixed));
  // The pressure hierarchy's Laplacian fixes the same rows as the stage-2
  // operator (the pin, on a closed domain), so one V-cycle of it is a
  // spectrally equivalent preconditioner there.
  const bool fp64 = P->desc.precision == FS_PREC_FP64;
  P->ip_mg = !P->p3 && (fp64 ? P->p64.HK.nlev : P->p32.HK.nlev) > 0;
  if (P->ip_mg) {
    FS_TRY(P->alloc(&P->ip_t, nv));
    if (!fp64) {
      FS_TRY(P->alloc(&P->ip_rf, nv));
      FS_TRY(P->alloc(&P->ip_zf, nv));
    }
  }
  cudaStream_t s = P->stream;
  launch_ipcs_dinv(P->dm, 0, P->baseA, nullptr, P->ip_dA, s);
  launch_ipcs_dinv(P->dm, 0, P->Mv, nullptr, P->ip_dM, s);
  launch_ipcs_dinv(P->dm, 1, P->Kp, P->ip_fixed, P->ip_dK, s);
  return check_launch("ipcs set-up");
}

// z = one V-cycle of the pressure hierarchy on r (FP64 I/O; an FP32
// hierarchy works on converted copies).
static void ipcs_vcycle(fs_problem* P, const double* r, double* z) {
  cudaStream_t s = P->stream;
  const int64_t n = P->nv;
  if (P->desc.precision == FS_PREC_FP64) {
    launch_vcycle_scalar<double>(P->p64.HK, r, z, n, s);
  } else {
    launch_convert<double, float>(r, P->ip_rf, n, nullptr, 0, s);
    launch_vcycle_scalar<float>(P->p32.HK, P->ip_rf, P->ip_zf, n, s);
    launch_convert<float, double>(P->ip_zf, z, n, nullptr, 0, s);
  }
}

// Solves A x = rhs (which 0: scalar P2 block `vals` on every component; 1:
// the pressure Laplacian) by CG from the guess in x (whose fixed unknowns are
// set first), to a recursive relative residual of rtol, checked every 8
// iterations; reports the true relative residual.  The velocity stages and
// P3/P2 pressure take Jacobi preconditioning; the P2/P1 pressure stage takes
// one V-cycle per iteration in flexible CG (Polak-Ribiere beta), which keeps
// the iteration count flat in the mesh size.
static int ipcs_cg(fs_problem* P, int which, const double* vals, const double* dinv,
                   const double* rhs, double* x, double rtol, int max_iter, int* iters,
                   double* relres) {
  cudaStream_t s = P->stream;
  const DMesh& m = P->dm;
  const int64_t n = which == 1 ? P->nv : (int64_t)P->dim * P->n2;
  const uint8_t* fixed = which == 1 ? P->ip_fixed : nullptr;
  const bool mg = which == 1 && P->ip_mg;
  launch_ipcs_fix(m, which, fixed, rhs, x, s);
  launch_diff_norms(rhs, rhs, n, P->ip_nrm, s);
  launch_ipcs_apply(m, which, vals, fixed, x, P->ip_q, nullptr, s);
  launch_cg_init(n, rhs, P->ip_q, dinv, P->ip_r, P->ip_z, P->ip_p, P->ip_part, P->ip_sc, s);
  if (mg) {
    ipcs_vcycle(P, P->ip_r, P->ip_z);
    launch_cg_dots_flex(n, fixed, P->ip_r, P->ip_t, P->ip_z, P->ip_p, 1, P->ip_part, P->ip_sc, s);
  }
  FS_TRY(check_launch("ipcs cg init"));
  double h[4] = {0, 0, 0, 0};
  FS_CUDA(cudaMemcpyAsync(h, P->ip_nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaMemcpyAsync(h + 2, P->ip_sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  const double bn = std::sqrt(h[1]);
  const double tol2 = (rtol * bn) * (rtol * bn);
  double rr = h[2 + 3];
  int it = 0;
  while (rr > tol2 && it < max_iter && std::isfinite(rr)) {
    for (int c = 0; c < 8 && it < max_iter; ++c, ++it) {
      const int nb = launch_ipcs_apply(m, which, vals, fixed, P->ip_p, P->ip_q, P->ip_part, s);
      launch_cg_alpha(P->ip_part, nb, P->ip_sc, s);
      if (mg) {
        launch_cg_update_flex(n, P->ip_sc, P->ip_p, P->ip_q, x, P->ip_r, P->ip_t, P->ip_part, s);
        ipcs_vcycle(P, P->ip_r, P->ip_z);
        launch_cg_dots_flex(n, fixed, P->ip_r, P->ip_t, P->ip_z, P->ip_p, 0, P->ip_part,
                            P->ip_sc, s);
      } else {
        launch_cg_update(n, P->ip_sc, P->ip_p, P->ip_q, dinv, x, P->ip_r, P->ip_z, P->ip_part,
                         s);
      }
      launch_cg_dir(n, P->ip_sc, P->ip_z, P->ip_p, s);
    }
    FS_TRY(check_launch("ipcs cg"));
    FS_CUDA(cudaMemcpyAsync(&rr, P->ip_sc + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
  }
  // true residual
  launch_ipcs_apply(m, which, vals, fixed, x, P->ip_q, nullptr, s);
  launch_diff_norms(rhs, P->ip_q, n, P->ip_nrm, s);
  FS_TRY(check_launch("ipcs cg residual"));
  FS_CUDA(cudaMemcpyAsync(h, P->ip_nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  *iters = it;
  *relres = bn > 0 ? std::sqrt(h[0]) / bn : std::sqrt(h[0]);
  if (!std::isfinite(*relres)) return FS_ERR_NUMERIC;
  return *relres <= 100.0 * rtol ? FS_OK : FS_ERR_NOT_CONVERGED;
}

static int ipcs_step_impl(fs_problem* P, double rtol, int max_iter, fs_ipcs_stats* st) {
  cudaStream_t s = P->stream;
  const int64_t nvel = (int64_t)P->dim * P->n2;
  const double t1 = P->t + P->desc.dt, dt = P->desc.dt;
  *st = fs_ipcs_stats{};
  // convection matrix N(u^n) and the load M (u^n/dt + I_h f^{n+1}) with the
  // boundary values of t^{n+1}
  FS_TRY(assemble_impl(P, t1));
  // stage 1: tentative velocity, from u^n
  launch_ipcs_rhs1(P->dm, P->valA, P->baseA, P->BT, P->b, P->x, P->ip_rhs, s);
  FS_CUDA(cudaMemcpyAsync(P->ip_us, P->x, sizeof(double) * nvel, cudaMemcpyDeviceToDevice, s));
  int rc = ipcs_cg(P, 0, P->baseA, P->ip_dA, P->ip_rhs, P->ip_us, rtol, max_iter, &st->iters[0],
                   &st->rel_res[0]);
  // stage 2: pressure increment, from 0
  if (rc == FS_OK) {
    launch_ipcs_rhs2(P->dm, P->B, P->ip_us, 1.0 / dt, P->ip_fixed, P->b, P->x, P->ip_rhs, s);
    FS_CUDA(cudaMemsetAsync(P->ip_dp, 0, sizeof(double) * P->nv, s));
    rc = ipcs_cg(P, 1, P->Kp, P->ip_dK, P->ip_rhs, P->ip_dp, rtol, max_iter, &st->iters[1],
                 &st->rel_res[1]);
  }
  // stage 3: corrected velocity, from u*; then p^{n+1} = p^n + dp
  if (rc == FS_OK) {
    launch_ipcs_rhs3(P->dm, P->Mv, P->BT, P->b, P->ip_us, P->ip_dp, dt, P->ip_rhs, s);
    FS_CUDA(cudaMemcpyAsync(P->x, P->ip_us, sizeof(double) * nvel, cudaMemcpyDeviceToDevice, s));
    rc = ipcs_cg(P, 0, P->Mv, P->ip_dM, P->ip_rhs, P->x, rtol, max_iter, &st->iters[2],
                 &st->rel_res[2]);
    launch_ipcs_add(P->nv, P->ip_dp, P->x + nvel, s);
    FS_TRY(check_launch("ipcs pressure update"));
  }
  P->t = t1;
  P->hist = 0;  // the coupled solve's state history does not cover these states
  st->status = rc;
  return rc;
}

int fs_step_ipcs(fs_problem* P, int nsteps, double rtol, int max_iter, fs_ipcs_stats* per_step) {
  OverlapScope overlap(P);
  if (!P || nsteps < 0 || !(rtol > 0) || max_iter < 1) {
    set_error("fs_step_ipcs: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  if (P->nseg != 1) {
    set_error("fs_step_ipcs: batched problems are stepped by fs_step");
    return FS_ERR_UNSUPPORTED;
  }
  const fs_mesh_desc& md = P->mesh->m.inst[0].desc;
  const int all = md.dim == 2 ? 0x0F : 0x3F;
  if ((md.dirichlet_sides & all) != all || !P->desc.pin_pressure ||
      !std::isfinite(P->desc.dt)) {
    set_error("fs_step_ipcs: needs Dirichlet velocity on the whole boundary, the pressure "
              "pin and a finite dt");
    return FS_ERR_UNSUPPORTED;
  }
  if (P->ctx.phase != PH_IDLE && P->ctx.phase != PH_DONE) {
    set_error("fs_step_ipcs: a step is in progress");
    return FS_ERR_BUSY;
  }
  FS_TRY(ipcs_setup(P));
  for (int k = 0; k < nsteps; ++k) {
    fs_ipcs_stats st;
    const int rc = ipcs_step_impl(P, rtol, max_iter, &st);
    if (per_step) per_step[k] = st;
    if (rc != FS_OK) {
      set_error("fs_step_ipcs: a stage's CG did not reach rtol");
      return rc;
    }
  }
  return FS_OK;
}

int fs_instance_stats(const fs_problem* P, fs_solve_stats* per_instance) {
  if (!P || !per_instance) {
    set_error("fs_instance_stats: null argument");
    return FS_ERR_INVALID_ARG;
  }
  for (size_t i = 0; i < P->last_stats.size(); ++i) per_instance[i] = P->last_stats[i];
  return FS_OK;
}

int fs_apply_operator(fs_problem* P, const double* x, double* y) {
  OverlapScope overlap(P);
  if (P && P->p3) {
    set_error("fs_apply_operator: P3/P2 problems are stepped by fs_step_ipcs");
    return FS_ERR_UNSUPPORTED;
  }
  if (!P || !x || !y) {
    set_error("fs_apply_operator: null argument");
    return FS_ERR_INVALID_ARG;
  }
  if (!P->assembled) {
    set_error("fs_apply_operator: call fs_assemble_step first");
    return FS_ERR_INVALID_ARG;
  }
  FS_TRY(nat_buffers(P));
  launch_dofs_perm(P->dm, P->nat, x, P->natbuf, 0, P->stream);
  launch_spmv_full<double, double>(P->p64.op, P->natbuf, nullptr, P->natbuf2, 0, nullptr,
                                   P->stream);
  launch_dofs_perm(P->dm, P->nat, P->natbuf2, y, 1, P->stream);
  return check_launch("fs_apply_operator");
}

int fs_get_state(fs_problem* P, double* x_out, int host, double* t_out) {
  if (!P) {
    set_error("fs_get_state: null problem");
    return FS_ERR_INVALID_ARG;
  }
  if (x_out && P->p3) {  // the P3/P2 state is stored in its boundary order
    FS_CUDA(cudaMemcpyAsync(x_out, P->x, sizeof(double) * P->ndof,
                            host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, P->stream));
  } else if (x_out) {
    FS_TRY(nat_buffers(P));
    launch_dofs_perm(P->dm, P->nat, P->x, P->natbuf, 1, P->stream);
    FS_TRY(check_launch("fs_get_state"));
    FS_CUDA(cudaMemcpyAsync(x_out, P->natbuf, sizeof(double) * P->ndof,
                            host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, P->stream));
  }
  FS_CUDA(cudaStreamSynchronize(P->stream));
  if (t_out) *t_out = P->t;
  return FS_OK;
}

int fs_set_state(fs_problem* P, const double* x_in, int host, double t) {
  if (!P) {
    set_error("fs_set_state: null problem");
    return FS_ERR_INVALID_ARG;
  }
  if (x_in && P->p3) {
    FS_CUDA(cudaMemcpyAsync(P->x, x_in, sizeof(double) * P->ndof,
                            host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, P->stream));
  } else if (x_in) {
    FS_TRY(nat_buffers(P));
    FS_CUDA(cudaMemcpyAsync(P->natbuf, x_in, sizeof(double) * P->ndof,
                            host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, P->stream));
    launch_dofs_perm(P->dm, P->nat, P->natbuf, P->x, 0, P->stream);
    FS_TRY(check_launch("fs_set_state"));
  }
  FS_CUDA(cudaStreamSynchronize(P->stream));
  // a state at the current time continues the history (e.g. a round trip
  // through host memory); any other time starts a new one
  if (t != P->t) P->hist = 0;
  P->t = t;
  return FS_OK;
}

int64_t fs_launch_count(void) { return g_launches.load(); }

int fs_profile_kernel(fs_problem* P, int kernel, int reps, double* avg_ms, double* alg_bytes) {
  OverlapScope overlap(P);
  if (P && P->p3) {
    set_error("fs_profile_kernel: P3/P2 problems are stepped by fs_step_ipcs");
    return FS_ERR_UNSUPPORTED;
  }
  if (!P || reps < 1 || !avg_ms || !alg_bytes) {
    set_error("fs_profile_kernel: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  const bool cold = (kernel & FS_PROFILE_COLD_L2) != 0;
  kernel &= ~FS_PROFILE_COLD_L2;
  if (cold && kernel == FS_KERNEL_PRECOND) {
    set_error("fs_profile_kernel: the preconditioner is timed as a graph, warm only");
    return FS_ERR_INVALID_ARG;
  }
  if (!P->assembled) FS_TRY(assemble_impl(P, P->t + P->desc.dt));
  const Mesh& me = P->mesh->m;
  const int d = P->dim;
  const bool f32 = P->has32;
  const double s = f32 ? 4.0 : 8.0;
  const int64_t nnzA = me.A.nnz(), nnzB = me.B.nnz(), nnzBT = me.BT.nnz();
  double bytes = 0;
  std::function<void()> launch;
  switch (kernel) {
    case FS_KERNEL_SPMV:  // saddle-point SpMV in the solver's arithmetic
    case FS_KERNEL_SPMV_FP64: {
      const bool use32 = f32 && kernel == FS_KERNEL_SPMV;
      const double sz = use32 ? 4.0 : 8.0;
      bytes = nnzA * (4 + sz) + nnzBT * (4 + d * sz) + nnzB * (4 + d * sz) +
              4.0 * (2 * (P->n2 + 1) + (P->nv + 1)) + P->nv * sz + 2.0 * P->ndof * sz;
      if (use32) {
        auto& pr = P->p32;
        launch = [P, &pr]() {
          launch_spmv_full<float, float>(pr.op, pr.kr.Vb, nullptr, pr.kr.Vb + P->ndof, 0, nullptr,
                                         P->stream);
        };
      } else {
        launch = [P]() {
          launch_spmv_full<double, double>(P->p64.op, P->x, nullptr, P->r64, 0, nullptr,
                                           P->stream);
        };
      }
      break;
    }
    case FS_KERNEL_CHEB: {  // one fused Chebyshev step on the finest velocity level
      const int64_t n = P->n2;
      bytes = nnzA * (4 + s) + 4.0 * (n + 1) + n * s + 5.0 * d * n * s;
      if (f32) {
        const DHier<float> H = without_skip(P->p32.HA);
        launch = [P, H, d]() { launch_cheb_step<float>(H, d, P->stream); };
      } else {
        const DHier<double> H = without_skip(P->p64.HA);
        launch = [P, H, d]() { launch_cheb_step<double>(H, d, P->stream); };
      }
      break;
    }
    case FS_KERNEL_ASSEMBLE_CONV: {  // per-step convection assembly (FP64)
      bytes = me.ncell * (double)me.nloc * (4 + me.nloc) + me.nv * d * 8.0 +
              (double)d * P->n2 * 8.0 + 4.0 * (P->n2 + 1) + P->n2 + 16.0 * nnzA;
      launch = [P]() {
        launch_assemble_conv(P->dm, P->mesh->m.color_ptr, P->x, P->n2, nullptr, P->valA,
                             P->desc.deterministic != 0, P->stream);
      };
      break;
    }
    case FS_KERNEL_PRECOND: {
      FS_TRY(time_precond(P, reps, P->sched.persistent_precond, avg_ms));
      *alg_bytes = 0;
      return FS_OK;
    }
    case FS_KERNEL_CGS:  // one CGS2 step of the Arnoldi process at j = m/2
    case FS_KERNEL_CGS_DOT:
    case FS_KERNEL_CGS_UPD:
    case FS_KERNEL_CGS_FIN: {
      // Krylov scratch only (basis, cycle state): the next solve rebuilds it.
      // Step index j and active segments are set on the device first.
      auto prime = [P](auto& K, int* jout) -> int {
        const int j = K.m / 2;
        *jout = j;
        std::vector<int> zero(P->nseg, 0);
        FS_CUDA(cudaMemcpyAsync(&K.ctl->j, &j, sizeof(int), cudaMemcpyHostToDevice, P->stream));
        FS_CUDA(cudaMemcpy2DAsync(&K.st[0].done, sizeof(SegState), zero.data(), sizeof(int),
                                  sizeof(int), P->nseg, cudaMemcpyHostToDevice, P->stream));
        FS_CUDA(cudaStreamSynchronize(P->stream));
        return FS_OK;
      };
      int j = 0;
      const int pass = kernel == FS_KERNEL_CGS ? -1 : kernel - FS_KERNEL_CGS_DOT;
      if (f32) {
        auto& K = P->p32.kr;
        FS_TRY(prime(K, &j));
        launch = [P, &K, pass]() {
          if (pass < 0)
            launch_seg_cgs2<float>(K.Vb, K.n, P->tl(), K.st, K.ctl, K.partial, false, 0,
                                   P->stream);
          else
            launch_seg_cgs2_pass<float>(K.Vb, K.n, P->tl(), K.st, K.ctl, K.partial, pass,
                                        P->stream);
        };
      } else {
        auto& K = P->p64.kr;
        FS_TRY(prime(K, &j));
        launch = [P, &K, pass]() {
          if (pass < 0)
            launch_seg_cgs2<double>(K.Vb, K.n, P->tl(), K.st, K.ctl, K.partial, false, 0,
                                    P->stream);
          else
            launch_seg_cgs2_pass<double>(K.Vb, K.n, P->tl(), K.st, K.ctl, K.partial, pass,
                                         P->stream);
        };
      }
      // basis vectors each pass must touch, each counted once: dot reads
      // V[0..j] and w; update reads V[0..j] and w and writes w (its re-dot
      // reads V[0..j] again, which is not counted); final the same
      const double sweeps = pass < 0 ? 3.0 * j + 8.0 : pass == 0 ? j + 2.0 : j + 3.0;
      bytes = sweeps * (double)P->ndof * s;
      break;
    }
    default:
      set_error("fs_profile_kernel: unknown kernel id");
      return FS_ERR_INVALID_ARG;
  }
  float ms = 0;
  if (!cold) {
    cudaEvent_t e0, e1;
    FS_CUDA(cudaEventCreate(&e0));
    FS_CUDA(cudaEventCreate(&e1));
    for (int i = 0; i < 3; ++i) launch();
    FS_CUDA(cudaEventRecord(e0, P->stream));
    for (int i = 0; i < reps; ++i) launch();
    FS_CUDA(cudaEventRecord(e1, P->stream));
    FS_CUDA(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  } else {
    // every launch after the L2 was filled with other data (a read of twice
    // its size), each timed by its own pair of events
    int dev = 0, l2 = 0;
    FS_CUDA(cudaGetDevice(&dev));
    FS_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const int64_t fb = ((std::max<int64_t>(2 * (int64_t)l2, 256ll << 20) + 15) / 16) * 16;
    void* flush = nullptr;
    FS_CUDA(cudaMallocAsync(&flush, (size_t)fb, P->stream));
    FS_CUDA(cudaMemsetAsync(flush, 0, (size_t)fb, P->stream));
    std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
    int rc = FS_OK;
    for (auto& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) rc = FS_ERR_CUDA;
    if (rc == FS_OK) {
      for (int i = 0; i < 3; ++i) launch();
      for (int i = 0; i < reps; ++i) {
        launch_l2_flush(flush, fb, nullptr, P->stream);
        cudaEventRecord(ev[2 * i], P->stream);
        launch();
        cudaEventRecord(ev[2 * i + 1], P->stream);
      }
      if (cudaEventSynchronize(ev.back()) != cudaSuccess) rc = FS_ERR_CUDA;
      for (int i = 0; i < reps && rc == FS_OK; ++i) {
        float t = 0;
        cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
        ms += t;
      }
    }
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    cudaFreeAsync(flush, P->stream);
    if (rc != FS_OK) {
      set_error("fs_profile_kernel: event failure in the L2-cold timing");
      return rc;
    }
  }
  FS_TRY(check_launch("fs_profile_kernel"));
  *avg_ms = ms / reps;
  *alg_bytes = bytes;
  if (kernel == FS_KERNEL_ASSEMBLE_CONV) FS_TRY(assemble_impl(P, P->t + P->desc.dt));
  return FS_OK;
}

int fs_get_schedule(const fs_problem* P, fs_schedule* out) {
  if (!P || !out) {
    set_error("fs_get_schedule: null argument");
    return FS_ERR_INVALID_ARG;
  }
  *out = P->sched;
  return FS_OK;
}

int fs_set_schedule(fs_problem* P, const fs_schedule* sc) {
  if (P && P->p3) {
    set_error("fs_set_schedule: P3/P2 problems are stepped by fs_step_ipcs");
    return FS_ERR_UNSUPPORTED;
  }
  const auto in = [](int v, std::initializer_list<int> ok) {
    return std::find(ok.begin(), ok.end(), v) != ok.end();
  };
  if (!P || !sc || sc->tail_rows_velocity < 0 || sc->tail_rows_pressure < 0 ||
      !in(sc->spmv_group, {0, 4, 6, 8}) || !in(sc->smooth_group, {0, 4, 6}) ||
      !in(sc->coarse_degree, {0, 1, 2, 3}) || !in(sc->serial_launches, {0, 1}) ||
      !in(sc->persistent_precond, {0, 1}) || !in(sc->fine_degree, {0, 1, 2, 3}) ||
      (sc->cheb_ratio != 0 && (sc->cheb_ratio < 2 || sc->cheb_ratio > 64)) ||
      !in(sc->schur, {0, 1})) {
    set_error("fs_set_schedule: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  if (sc->persistent_precond && (sc->schur || sc->coarse_degree == 1 || sc->fine_degree == 1)) {
    set_error("fs_set_schedule: the persistent preconditioner takes the Cahouet-Chabard "
              "Schur part and smoothing degrees 2 and 3 only");
    return FS_ERR_UNSUPPORTED;
  }
  if (P->ctx.phase != PH_IDLE && P->ctx.phase != PH_DONE) {
    set_error("fs_set_schedule: a step is in progress");
    return FS_ERR_BUSY;
  }
  return install_schedule(P, *sc);
}

int fs_autotune(fs_problem* P, int reps, fs_tune_report* report) {
  OverlapScope overlap(P);
  if (P && P->p3) {
    set_error("fs_autotune: P3/P2 problems are stepped by fs_step_ipcs");
    return FS_ERR_UNSUPPORTED;
  }
  if (!P || reps < 1) {
    set_error("fs_autotune: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  if (P->ctx.phase != PH_IDLE && P->ctx.phase != PH_DONE) {
    set_error("fs_autotune: a step is in progress");
    return FS_ERR_BUSY;
  }
  if (!P->assembled) FS_TRY(assemble_impl(P, P->t + P->desc.dt));
  const int64_t cand[4] = {0, 4096, 16384, 65536};
  const int sgroups[2] = {4, 6}, pgroups[3] = {4, 6, 8};
  fs_tune_report r{};
  r.best = P->sched;
  FS_TRY(time_precond(P, reps, P->sched.persistent_precond, &r.default_ms));
  FS_TRY(time_spmv(P, reps, &r.spmv_default_ms));
  r.best_ms = r.default_ms;
  r.spmv_best_ms = r.spmv_default_ms;
  r.candidates = 1;
  // puts a schedule in place without dropping graphs (timing only) and
  // returns the choices it makes, so equal choices are timed once
  auto apply = [&](const fs_schedule& sc) {
    std::array<int, 4> k;
    if (P->desc.precision == FS_PREC_FP64) {
      auto& pr = P->p64;
      apply_groups<double>(P, pr, sc);
      apply_tail<double>(P, pr.HA, sc.tail_rows_velocity);
      apply_tail<double>(P, pr.HK, sc.tail_rows_pressure);
      k = {pr.HA.tail, pr.HK.tail, pr.HA.group, pr.op.group};
    } else {
      auto& pr = P->p32;
      apply_groups<float>(P, pr, sc);
      apply_tail<float>(P, pr.HA, sc.tail_rows_velocity);
      apply_tail<float>(P, pr.HK, sc.tail_rows_pressure);
      k = {pr.HA.tail, pr.HK.tail, pr.HA.group, pr.op.group};
    }
    return k;
  };
  // the preconditioner: fused-tail thresholds x smoothing group depths
  std::vector<std::array<int, 4>> seen{apply(P->sched)};
  const fs_schedule base = P->sched;
  for (int g : sgroups)
    for (int64_t v : cand)
      for (int64_t p : cand) {
        fs_schedule sc = base;
        sc.tail_rows_velocity = v;
        sc.tail_rows_pressure = p;
        sc.smooth_group = g;
        std::array<int, 4> k = apply(sc);
        if (std::find(seen.begin(), seen.end(), k) != seen.end()) continue;
        seen.push_back(k);
        double ms = 0;
        FS_TRY(time_precond(P, reps, 0, &ms));
        r.candidates += 1;
        if (ms < r.best_ms) {
          r.best_ms = ms;
          r.best = sc;
        }
      }
  // the persistent preconditioner against the best per-pass schedule (its
  // own time with that schedule's smoothing degree)
  {
    fs_schedule sc = r.best;
    sc.persistent_precond = 0;
    apply(sc);
    double ms0 = 0, ms1 = 0;
    FS_TRY(time_precond(P, reps, 0, &ms0));
    int rc = FS_ERR_UNSUPPORTED;
    if (!base.schur && base.coarse_degree != 1 && base.fine_degree != 1)
      rc = P->desc.precision == FS_PREC_FP64 ? apply_flow<double>(P, P->p64)
                                             : apply_flow<float>(P, P->p32);
    if (rc == FS_OK) rc = time_precond(P, reps, 1, &ms1);
    if (rc != FS_OK && rc != FS_ERR_UNSUPPORTED) return rc;
    r.candidates += 1;
    r.persistent_ms = rc == FS_OK ? ms1 : 0.0;
    sc.persistent_precond = rc == FS_OK && ms1 < ms0 ? 1 : 0;
    r.best = sc;
    r.best_ms = sc.persistent_precond ? ms1 : std::min(r.best_ms, ms0);
  }
  // the SpMV: group depths, with the preconditioner's choice in place
  for (int g : pgroups) {
    fs_schedule sc = r.best;
    sc.spmv_group = g;
    apply(sc);
    double ms = 0;
    FS_TRY(time_spmv(P, reps, &ms));
    r.candidates += 1;
    if (ms < r.spmv_best_ms) {
      r.spmv_best_ms = ms;
      r.best.spmv_group = g;
    }
  }
  FS_TRY(install_schedule(P, r.best));
  if (report) *report = r;
  return FS_OK;
}

int fs_autotune_smoother(fs_problem* P, int nsteps, const int32_t* cand, int ncand,
                         double* ms_out, double* iters_out, fs_schedule* best_out) {
  if (P && P->p3) {
    set_error("fs_autotune_smoother: P3/P2 problems are stepped by fs_step_ipcs");
    return FS_ERR_UNSUPPORTED;
  }
  if (!P || nsteps < 1 || !cand || ncand < 1 || ncand > 64) {
    set_error("fs_autotune_smoother: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  if (P->ctx.phase != PH_IDLE && P->ctx.phase != PH_DONE) {
    set_error("fs_autotune_smoother: a step is in progress");
    return FS_ERR_BUSY;
  }
  const fs_schedule base = P->sched;
  std::vector<fs_schedule> scs(ncand, base);
  for (int q = 0; q < ncand; ++q) {
    const int32_t* c = cand + 3 * q;
    if (c[0]) scs[q].cheb_ratio = c[0];
    if (c[1]) scs[q].coarse_degree = c[1];
    if (c[2]) scs[q].fine_degree = c[2];
    const fs_schedule& sc = scs[q];
    if ((sc.cheb_ratio != 0 && (sc.cheb_ratio < 2 || sc.cheb_ratio > 64)) ||
        sc.coarse_degree < 0 || sc.coarse_degree > 3 || sc.fine_degree < 0 ||
        sc.fine_degree > 3) {
      set_error("fs_autotune_smoother: a candidate field is out of range");
      return FS_ERR_INVALID_ARG;
    }
    if (sc.persistent_precond && (sc.coarse_degree == 1 || sc.fine_degree == 1)) {
      set_error("fs_autotune_smoother: degree 1 with the persistent preconditioner");
      return FS_ERR_UNSUPPORTED;
    }
  }
  cudaStream_t s = P->stream;
  const double t0 = P->t;
  // the state at the call, in a scratch copy freed before returning
  double* x0 = nullptr;
  FS_CUDA(cudaMallocAsync((void**)&x0, sizeof(double) * P->ndof, s));
  auto restore = [&]() {
    cudaMemcpyAsync(P->x, x0, sizeof(double) * P->ndof, cudaMemcpyDeviceToDevice, s);
    P->t = t0;
    P->hist = 0;
    P->assembled = false;
    return cudaStreamSynchronize(s);
  };
  cudaMemcpyAsync(x0, P->x, sizeof(double) * P->ndof, cudaMemcpyDeviceToDevice, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<fs_solve_stats> st(nsteps);
  int rc = FS_OK, best = -1;
  double best_ms = 0;
  for (int q = 0; q < ncand && rc == FS_OK; ++q) {
    rc = install_schedule(P, scs[q]);
    // one untimed step captures the solver's graphs for this schedule
    if (rc == FS_OK && restore() != cudaSuccess) rc = FS_ERR_CUDA;
    if (rc == FS_OK) rc = fs_step(P, 1, nullptr, st.data());
    if (rc == FS_OK && restore() != cudaSuccess) rc = FS_ERR_CUDA;
    if (rc != FS_OK) break;
    cudaEventRecord(e0, s);
    rc = fs_step(P, nsteps, nullptr, st.data());
    cudaEventRecord(e1, s);
    if (rc != FS_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      if (rc == FS_OK) rc = FS_ERR_CUDA;
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    double it = 0;
    for (const fs_solve_stats& x : st) it += x.iters;
    if (ms_out) ms_out[q] = ms / nsteps;
    if (iters_out) iters_out[q] = it / nsteps;
    if (best < 0 || ms < best_ms) {
      best = q;
      best_ms = ms;
    }
  }
  const fs_schedule fin = rc == FS_OK ? scs[best] : base;
  const std::string err = rc == FS_OK ? std::string() : fs_last_error();
  int rc2 = install_schedule(P, fin);
  if (restore() != cudaSuccess && rc2 == FS_OK) rc2 = FS_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(x0, s);
  cudaStreamSynchronize(s);
  if (rc != FS_OK) {
    set_error("fs_autotune_smoother: " + err);
    return rc;
  }
  if (rc2 != FS_OK) return rc2;
  if (best_out) *best_out = P->sched;
  return FS_OK;
}

}  // extern "C"
