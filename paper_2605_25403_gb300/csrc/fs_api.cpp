// C ABI of libfs (include/fs.h): problem lifecycle, the per-step assembly
// driver, flexible GMRES(m) with FP64 or FP32-plus-FP64-refinement
// arithmetic, and CUDA-graph replay of restart cycles.
//
// Paper Sec. 3.1 (ComputationModel workflow: assembly -> linear solver ->
// update) and Sec. 2.2.1 (Oseen step).  Host code only: every floating-point
// operation on the step's data runs in the kernels of fs_assembly.cu and
// fs_linalg.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <string>
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
std::atomic<int64_t> g_launches{0};

RefTensors g_ref2, g_ref3;
bool g_ref_ready = false;
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }

void count_launches(int64_t n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

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

#define FS_TRY(expr)            \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ != FS_OK) return rc_; \
  } while (0)

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
  double* partial = nullptr;
  GmresState* st = nullptr;
  cudaGraphExec_t g_check = nullptr, g_iter = nullptr;
  size_t n_check = 0, n_iter = 0;  // kernel nodes per graph
  const void* g_x = nullptr;  // buffers the graphs were captured with
  const void* g_b = nullptr;
};

template <typename T>
struct Precision {
  DOp<T> op;
  DHier<T> HA, HK;
  T* mplinv_nu = nullptr;
  Krylov<T> kr;
  int lanes = 4;
};

}  // namespace

struct fs_problem {
  fs_mesh* mesh = nullptr;
  fs_problem_desc desc{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int dim = 0;
  int64_t n2 = 0, nv = 0, ndof = 0;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  DMesh dm;
  DPhys ph;
  // FP64 data
  double *baseA = nullptr, *Mv = nullptr, *valA = nullptr, *B = nullptr, *BT = nullptr;
  double *Kp = nullptr, *mpl = nullptr, *diagp = nullptr;
  double *x = nullptr, *b = nullptr, *F = nullptr, *r64 = nullptr;
  double* scal = nullptr;  // device scalars: [0] ||b||, [1] ||r||, ...
  unsigned* counters = nullptr;
  double* partial64 = nullptr;
  int32_t* pinned = nullptr;
  int npinned = 0;
  int64_t* mrp = nullptr;  // monolithic row pointers (export)
  // FP32 data (precision mode)
  float *valA32 = nullptr, *B32 = nullptr, *BT32 = nullptr, *diagp32 = nullptr;
  Precision<double> p64;
  Precision<float> p32;
  bool has64 = false, has32 = false;
  double t = 0;
  bool assembled = false;

  template <typename T>
  int alloc(T** p, int64_t count) {
    size_t bytes_ = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes_);
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
    if (!h.empty()) FS_CUDA(cudaMemcpy(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return FS_OK;
  }
  ~fs_problem() {
    for (auto* k : {&p64.kr.g_check, &p64.kr.g_iter, &p32.kr.g_check, &p32.kr.g_iter})
      if (*k) cudaGraphExecDestroy(*k);
    for (void* q : allocs) cudaFree(q);
    if (own_stream && stream) cudaStreamDestroy(stream);
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

template <typename T>
int upload_csr(fs_problem* P, const HostCsr& H, DCsr<T>& d, const int32_t** rp_keep = nullptr) {
  int32_t *rp, *ci;
  T* v;
  FS_TRY(P->upload(&rp, H.rowptr));
  FS_TRY(P->upload(&ci, H.col));
  std::vector<T> hv(H.val.begin(), H.val.end());
  FS_TRY(P->upload(&v, hv));
  d.nrow = (int32_t)H.nrow;
  d.rp = rp;
  d.ci = ci;
  d.v = v;
  if (rp_keep) *rp_keep = rp;
  return FS_OK;
}

// Chebyshev(3) coefficients on [lmax/8, 1.1 lmax] of D^-1 A.
template <typename T>
void cheb_coeffs(double lmax, DLevel<T>& L) {
  double hi = 1.1 * lmax, lo = hi / 8.0;
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

template <typename T>
int upload_hierarchy(fs_problem* P, const HostHierarchy& H, int nc, DHier<T>& D) {
  D.nlev = (int)H.levels.size();
  if (D.nlev > 16) {
    set_error("multigrid hierarchy deeper than 16 levels");
    return FS_ERR_UNSUPPORTED;
  }
  for (int l = 0; l < D.nlev; ++l) {
    const HostLevel& hl = H.levels[l];
    DLevel<T>& dl = D.lev[l];
    FS_TRY(upload_csr<T>(P, hl.A, dl.A));
    if (l + 1 < D.nlev) {
      FS_TRY(upload_csr<T>(P, hl.P, dl.P));
      FS_TRY(upload_csr<T>(P, hl.R, dl.R));
    }
    std::vector<T> di(hl.dinv.begin(), hl.dinv.end());
    T* dinv;
    FS_TRY(P->upload(&dinv, di));
    dl.dinv = dinv;
    cheb_coeffs<T>(hl.lmax, dl);
    double avg = hl.A.nrow ? (double)hl.A.nnz() / (double)hl.A.nrow : 0;
    dl.lanes = avg >= 20.0 ? 8 : 4;
    int64_t len = (int64_t)nc * hl.A.nrow;
    FS_TRY(P->alloc(&D.xw[l], len));
    FS_TRY(P->alloc(&D.xw2[l], len));
    FS_TRY(P->alloc(&D.dw[l], len));
    FS_TRY(P->alloc(&D.dw2[l], len));
    FS_TRY(P->alloc(&D.bw[l], len));
  }
  std::vector<T> ci(H.coarse_inv.begin(), H.coarse_inv.end());
  T* cinv;
  FS_TRY(P->upload(&cinv, ci));
  D.cinv = cinv;
  D.ncoarse = H.ncoarse;
  return FS_OK;
}

template <typename V>
int alloc_krylov(fs_problem* P, Krylov<V>& K, int m) {
  K.m = m;
  K.n = P->ndof;
  FS_TRY(P->alloc(&K.Vb, (int64_t)(m + 1) * K.n));
  FS_TRY(P->alloc(&K.Z, (int64_t)m * K.n));
  FS_TRY(P->alloc(&K.work_p, P->nv));
  FS_TRY(P->alloc(&K.work_u, (int64_t)P->dim * P->n2));
  FS_TRY(P->alloc(&K.rhs, K.n));
  FS_TRY(P->alloc(&K.sol, K.n));
  // partial sums: (restart + 1) vectors x at most 4 x 152 blocks (CGS2
  // passes) or one block per 4096 entries (norms)
  int64_t nblk = std::max<int64_t>((K.n + 4095) / 4096 + 1, 4 * 152);
  FS_TRY(P->alloc(&K.partial, (int64_t)(kMaxRestart + 1) * nblk));
  FS_TRY(P->alloc(&K.st, 1));
  FS_CUDA(cudaMemset(K.st, 0, sizeof(GmresState)));
  return FS_OK;
}

// Pressure vertices whose Poisson rows are fixed in the preconditioner: the
// pinned vertex when the whole boundary is Dirichlet, else the vertices on
// the sides with a natural (do-nothing) velocity condition.
std::vector<int32_t> poisson_fixed(const Mesh& m, bool pin) {
  std::vector<int32_t> out;
  const int dim = m.dim;
  const int all = dim == 2 ? 0x0F : 0x3F;
  int natural = all & ~m.desc.dirichlet_sides;
  if (natural == 0) {
    if (pin) out.push_back(0);
    return out;
  }
  const int* n = m.desc.n;
  int64_t sx = n[0] + 1, sy = n[1] + 1;
  for (int64_t v = 0; v < m.nv; ++v) {
    int64_t ijk[3] = {v % sx, (v / sx) % sy, dim == 3 ? v / (sx * sy) : 0};
    int bits = 0;
    for (int a = 0; a < dim; ++a) {
      if (ijk[a] == 0) bits |= 1 << (2 * a);
      if (ijk[a] == n[a]) bits |= 1 << (2 * a + 1);
    }
    // vertices on a natural side that are not on a Dirichlet side
    if ((bits & natural) && !(bits & m.desc.dirichlet_sides)) out.push_back((int32_t)v);
  }
  return out;
}

template <typename T>
int setup_precision(fs_problem* P, Precision<T>& pr, const HostHierarchy& HA,
                    const HostHierarchy& HK, const std::vector<double>& mpl_h,
                    const T* valA, const T* B, const T* BT, const T* diagp, int m) {
  const Mesh& me = P->mesh->m;
  pr.op.dim = P->dim;
  pr.op.n2 = P->n2;
  pr.op.nv = P->nv;
  pr.op.A = {(int32_t)P->n2, P->dm.rpA, P->dm.ciA, valA};
  pr.op.B = {(int32_t)P->nv, P->dm.rpB, P->dm.ciB, B};
  pr.op.BT = {(int32_t)P->n2, P->dm.rpBT, P->dm.ciBT, BT};
  pr.op.diagp = diagp;
  double avg = (double)(me.A.nnz() + me.BT.nnz()) / (double)P->n2;
  pr.lanes = avg >= 24.0 ? 8 : 4;
  FS_TRY(upload_hierarchy<T>(P, HA, P->dim, pr.HA));
  FS_TRY(upload_hierarchy<T>(P, HK, 1, pr.HK));
  std::vector<T> mi(P->nv);
  for (int64_t q = 0; q < P->nv; ++q) mi[q] = (T)(P->desc.nu / mpl_h[q]);
  FS_TRY(P->upload(&pr.mplinv_nu, mi));
  FS_TRY(alloc_krylov<T>(P, pr.kr, m));
  return FS_OK;
}

// ---------------------------------------------------------------------------
// Flexible GMRES(m), right preconditioned, restart cycles split in a "check"
// part (true residual, norm, cycle init) and an "iteration" part (m Arnoldi
// steps with CGS2, Givens rotations on the device, update of x).
// ---------------------------------------------------------------------------
template <typename T>
void issue_check(fs_problem* P, Precision<T>& pr, const T* x, const T* b) {
  Krylov<T>& K = pr.kr;
  cudaStream_t s = P->stream;
  launch_spmv_full<T, T>(pr.op, x, b, K.Vb, 1, nullptr, pr.lanes, s);
  launch_norm2<T>(K.Vb, K.n, K.partial, &K.st->counter[0], &K.st->beta, 0, nullptr, s);
  launch_cycle_init(K.st, s);
}

template <typename T>
void issue_iter(fs_problem* P, Precision<T>& pr, T* x) {
  Krylov<T>& K = pr.kr;
  cudaStream_t s = P->stream;
  const int* skip = &K.st->done;
  const int64_t n = K.n;
  launch_scale<T>(K.Vb, n, nullptr, &K.st->beta, 0, skip, s);
  for (int j = 0; j < K.m; ++j) {
    T* vj = K.Vb + (int64_t)j * n;
    T* zj = K.Z + (int64_t)j * n;
    T* w = K.Vb + (int64_t)(j + 1) * n;
    launch_precond<T>(pr.op, pr.HA, pr.HK, pr.mplinv_nu, 1.0 / P->desc.dt, P->pinned,
                      P->npinned, vj, zj, K.work_p, K.work_u, skip, s);
    launch_spmv_full<T, T>(pr.op, zj, nullptr, w, 0, skip, pr.lanes, s);
    launch_cgs2<T>(K.Vb, n, j, K.st, K.partial, skip, s);
    launch_scale<T>(w, n, nullptr, &K.st->hn, 0, skip, s);
    launch_givens(K.st, j, s);
  }
  launch_update_x<T, T>(K.st, K.Z, n, x, 1.0, s);
}

template <typename T>
int run_part(fs_problem* P, Precision<T>& pr, bool check, const T* x, const T* b,
             bool use_graph) {
  Krylov<T>& K = pr.kr;
  cudaGraphExec_t* g = check ? &K.g_check : &K.g_iter;
  if (use_graph && (K.g_x != (const void*)x || K.g_b != (const void*)b)) {
    if (K.g_check) cudaGraphExecDestroy(K.g_check);
    if (K.g_iter) cudaGraphExecDestroy(K.g_iter);
    K.g_check = K.g_iter = nullptr;
    K.g_x = x;
    K.g_b = b;
  }
  if (!use_graph) {
    if (check) issue_check<T>(P, pr, x, b);
    else issue_iter<T>(P, pr, const_cast<T*>(x));
    return check_launch("gmres cycle");
  }
  size_t* nodes = check ? &K.n_check : &K.n_iter;
  if (!*g) {
    cudaGraph_t graph;
    FS_CUDA(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    if (check) issue_check<T>(P, pr, x, b);
    else issue_iter<T>(P, pr, const_cast<T*>(x));
    g_capturing = false;
    FS_CUDA(cudaStreamEndCapture(P->stream, &graph));
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

struct CycleInfo {
  double beta, resid;
  int done, k, bad;
};

template <typename T>
int read_state(fs_problem* P, Precision<T>& pr, CycleInfo& ci) {
  GmresState* st = pr.kr.st;
  FS_CUDA(cudaMemcpyAsync(&ci.beta, &st->beta, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  FS_CUDA(cudaMemcpyAsync(&ci.resid, &st->resid, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  FS_CUDA(cudaMemcpyAsync(&ci.done, &st->done, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  FS_CUDA(cudaMemcpyAsync(&ci.k, &st->k, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  FS_CUDA(cudaMemcpyAsync(&ci.bad, &st->bad, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  FS_CUDA(cudaStreamSynchronize(P->stream));
  return FS_OK;
}

// Solves K x = b to ||b - K x|| <= tol_abs (true residual, in the arithmetic
// of T).  iters is incremented; returns FS_OK / NOT_CONVERGED / NUMERIC.
// single_cycle: run one restart cycle whose Arnoldi estimate stops at
// tol_abs and return (the inner solve of the refinement, whose own true
// residual cannot be trusted below the FP32 rounding floor).
template <typename T>
int gmres(fs_problem* P, Precision<T>& pr, T* x, const T* b, double tol_abs, int max_iter,
          bool use_graph, int& iters, int& cycles, double& final_res,
          bool single_cycle = false) {
  Krylov<T>& K = pr.kr;
  double tol = tol_abs;
  FS_CUDA(cudaMemcpyAsync(&K.st->tol_abs, &tol, sizeof(double), cudaMemcpyHostToDevice, P->stream));
  int m = K.m;
  FS_CUDA(cudaMemcpyAsync(&K.st->m, &m, sizeof(int), cudaMemcpyHostToDevice, P->stream));
  int start_iters = iters;
  double prev = INFINITY;
  while (true) {
    FS_TRY(run_part<T>(P, pr, true, x, b, use_graph));
    CycleInfo ci;
    FS_TRY(read_state<T>(P, pr, ci));
    final_res = ci.beta;
    if (ci.bad) {
      set_error("non-finite residual in GMRES");
      return FS_ERR_NUMERIC;
    }
    if (ci.beta <= tol_abs) return FS_OK;
    if (iters - start_iters >= max_iter) {
      set_error("GMRES reached max_iter with residual " + std::to_string(ci.beta));
      return FS_ERR_NOT_CONVERGED;
    }
    // a whole restart cycle that did not reduce the true residual by 10%
    // means the rounding floor of the arithmetic has been reached: accept it
    // within 100 tol_abs, else report non-convergence
    if (!single_cycle && ci.beta > 0.9 * prev) {
      if (ci.beta <= 100.0 * tol_abs) return FS_OK;
      set_error("GMRES stagnated at true residual " + std::to_string(ci.beta));
      return FS_ERR_NOT_CONVERGED;
    }
    prev = ci.beta;
    FS_TRY(run_part<T>(P, pr, false, x, b, use_graph));
    FS_TRY(read_state<T>(P, pr, ci));
    iters += ci.k;
    cycles += 1;
    if (ci.bad) {
      set_error("non-finite value in the Arnoldi process");
      return FS_ERR_NUMERIC;
    }
    if (single_cycle) return FS_OK;
    if (ci.k == 0) {
      set_error("GMRES stagnated (no Arnoldi step possible)");
      return FS_ERR_NOT_CONVERGED;
    }
  }
}

int solve_impl(fs_problem* P, const fs_solve_opts& o, double* x, fs_solve_stats& st) {
  st = fs_solve_stats{};
  double bn = 0;
  launch_norm2<double>(P->b, P->ndof, P->partial64, &P->counters[0], &P->scal[0], 0, nullptr,
                       P->stream);
  FS_CUDA(cudaMemcpyAsync(&bn, &P->scal[0], sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  FS_CUDA(cudaStreamSynchronize(P->stream));
  if (bn == 0) bn = 1;
  const double tol_abs = o.rtol * bn;
  int rc = FS_OK;
  if (P->desc.precision == FS_PREC_FP64) {
    double res = 0;
    rc = gmres<double>(P, P->p64, x, P->b, tol_abs, o.max_iter, o.use_graph != 0, st.iters,
                       st.cycles, res);
    st.rel_res = res / bn;
  } else {
    // FP64 iterative refinement around an FP32 inner FGMRES
    rc = FS_ERR_NOT_CONVERGED;
    Precision<float>& pr = P->p32;
    double prev_rn = INFINITY;
    for (int it = 0; it <= o.max_refine; ++it) {
      launch_spmv_full<double, double>(P->p64.op, x, P->b, P->r64, 1, nullptr, P->p64.lanes,
                                       P->stream);
      launch_norm2<double>(P->r64, P->ndof, P->partial64, &P->counters[1], &P->scal[1], 0,
                           nullptr, P->stream);
      double rn = 0;
      FS_CUDA(cudaMemcpyAsync(&rn, &P->scal[1], sizeof(double), cudaMemcpyDeviceToHost,
                              P->stream));
      FS_CUDA(cudaStreamSynchronize(P->stream));
      st.rel_res = rn / bn;
      if (!std::isfinite(rn)) {
        set_error("non-finite FP64 residual");
        rc = FS_ERR_NUMERIC;
        break;
      }
      if (rn <= tol_abs) {
        rc = FS_OK;
        break;
      }
      // refinement no longer contracting: the FP64 rounding floor
      if (rn > 0.5 * prev_rn && rn <= 100.0 * tol_abs) {
        rc = FS_OK;
        break;
      }
      prev_rn = rn;
      if (it == o.max_refine || st.iters >= o.max_iter) {
        set_error("refinement did not reach rtol: " + std::to_string(rn / bn));
        break;
      }
      st.refinements += 1;
      launch_convert<double, float>(P->r64, pr.kr.rhs, P->ndof, &P->scal[1], 1, P->stream);
      FS_CUDA(cudaMemsetAsync(pr.kr.sol, 0, sizeof(float) * P->ndof, P->stream));
      double ires = 0;
      int irc = gmres<float>(P, pr, pr.kr.sol, pr.kr.rhs, o.inner_rtol, o.max_iter - st.iters,
                             o.use_graph != 0, st.iters, st.cycles, ires, true);
      if (irc == FS_ERR_NUMERIC) {
        rc = irc;
        break;
      }
      launch_axpy_mixed<float, double>(x, pr.kr.sol, P->ndof, &P->scal[1], P->stream);
      FS_TRY(check_launch("refinement update"));
    }
  }
  st.status = rc;
  return rc;
}

int assemble_impl(fs_problem* P, double t_next) {
  cudaStream_t s = P->stream;
  const Mesh& me = P->mesh->m;
  const int64_t nnzA = me.A.nnz();
  FS_CUDA(cudaMemcpyAsync(P->valA, P->baseA, sizeof(double) * nnzA, cudaMemcpyDeviceToDevice, s));
  const bool constw = P->desc.problem == FS_PROBLEM_POLY_OSEEN;
  launch_assemble_conv(P->dm, constw ? nullptr : P->x, P->n2, constw ? P->desc.wconst : nullptr,
                       P->valA, s);
  launch_bc_rows<double>(P->dm, P->valA, s);
  launch_eval_load(P->dm, P->ph, t_next, 1.0 / P->desc.dt, P->x, P->F, s);
  launch_rhs(P->dm, P->ph, t_next, P->Mv, P->F, P->desc.pin_pressure, P->b, s);
  if (P->has32) launch_convert<double, float>(P->valA, P->valA32, nnzA, nullptr, 0, s);
  FS_TRY(check_launch("assembly"));
  P->assembled = true;
  return FS_OK;
}

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
  if (!desc || !out) {
    set_error("fs_mesh_create: null argument");
    return FS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  auto* h = new (std::nothrow) fs_mesh;
  if (!h) return FS_ERR_OOM;
  int rc = build_mesh(*desc, h->m);
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
  if (cell2dof) std::memcpy(cell2dof, m.c2d.data(), sizeof(int32_t) * m.c2d.size());
  if (dirichlet) std::memcpy(dirichlet, m.dirichlet.data(), m.dirichlet.size());
  if (rowptr || col) {
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    monolithic_pattern(m, rp, ci);
    if (rowptr) std::memcpy(rowptr, rp.data(), sizeof(int64_t) * rp.size());
    if (col) std::memcpy(col, ci.data(), sizeof(int32_t) * ci.size());
  }
  return FS_OK;
}

int fs_problem_create(fs_mesh* mesh, const fs_problem_desc* desc, void* stream,
                      fs_problem** out) {
  if (!mesh || !desc || !out) {
    set_error("fs_problem_create: null argument");
    return FS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!(desc->dt > 0) || !(desc->nu > 0) || desc->problem < 0 || desc->problem > 4 ||
      (desc->precision != FS_PREC_FP64 && desc->precision != FS_PREC_FP32_REFINE)) {
    set_error("fs_problem_create: need dt > 0, nu > 0, a known problem and precision");
    return FS_ERR_INVALID_ARG;
  }
  const Mesh& me = mesh->m;
  if ((desc->problem == FS_PROBLEM_CUBE) != (me.dim == 3) &&
      desc->problem != FS_PROBLEM_POLY_OSEEN) {
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
  P->desc = *desc;
  P->dim = me.dim;
  P->n2 = me.n2;
  P->nv = me.nv;
  P->ndof = me.dim * me.n2 + me.nv;
  P->t = desc->t0;
  if (stream) {
    P->stream = (cudaStream_t)stream;
  } else {
    FS_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    P->own_stream = true;
  }
  if (!g_ref_ready) {
    ref_tensors(2, g_ref2);
    ref_tensors(3, g_ref3);
    g_ref_ready = true;
  }
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
  }
  P->ph.kind = desc->problem;
  P->ph.nu = desc->nu;
  for (int a = 0; a < 3; ++a) P->ph.wconst[a] = desc->wconst[a];

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
  launch_assemble_base(dm, 1.0 / desc->dt, desc->nu, P->baseA, P->Mv, P->B, P->BT, P->Kp,
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
  // pinned pressure row -> zero B row, unit diagonal
  for (int32_t i : me.dlist) {
    for (int32_t k = A0.rowptr[i]; k < A0.rowptr[i + 1]; ++k) A0.val[k] = (A0.col[k] == i) ? 1.0 : 0.0;
    for (int32_t k = me.BT.rowptr[i]; k < me.BT.rowptr[i + 1]; ++k)
      for (int c = 0; c < dim; ++c) BTh[(int64_t)k * dim + c] = 0.0;
  }
  std::vector<double> dp(P->nv, 0.0);
  if (desc->pin_pressure) {
    for (int32_t k = me.B.rowptr[0]; k < me.B.rowptr[1]; ++k)
      for (int c = 0; c < dim; ++c) Bh[(int64_t)k * dim + c] = 0.0;
    dp[0] = 1.0;
    std::vector<int32_t> pin = {0};
    FS_TRY(P->upload(&P->pinned, pin));
    P->npinned = 1;
  }
  FS_CUDA(cudaMemcpy(P->B, Bh.data(), sizeof(double) * Bh.size(), cudaMemcpyHostToDevice));
  FS_CUDA(cudaMemcpy(P->BT, BTh.data(), sizeof(double) * BTh.size(), cudaMemcpyHostToDevice));
  FS_CUDA(cudaMemcpy(P->diagp, dp.data(), sizeof(double) * P->nv, cudaMemcpyHostToDevice));
  // pressure Poisson of the preconditioner with its fixed rows
  std::vector<int32_t> kfix = poisson_fixed(me, desc->pin_pressure != 0);
  {
    std::vector<uint8_t> fixed(P->nv, 0);
    for (int32_t q : kfix) fixed[q] = 1;
    for (int64_t q = 0; q < P->nv; ++q)
      for (int32_t k = Kp.rowptr[q]; k < Kp.rowptr[q + 1]; ++k)
        if (fixed[q] || fixed[Kp.col[k]]) Kp.val[k] = (Kp.col[k] == q) ? 1.0 : 0.0;
  }
  HostHierarchy HA, HK;
  build_hierarchy(me, A0, true, me.dlist, 800, HA);
  build_hierarchy(me, Kp, false, kfix, 800, HK);

  // vectors
  FS_TRY(P->alloc(&P->x, P->ndof));
  FS_TRY(P->alloc(&P->b, P->ndof));
  FS_TRY(P->alloc(&P->F, (int64_t)dim * P->n2));
  FS_TRY(P->alloc(&P->r64, P->ndof));
  FS_TRY(P->alloc(&P->scal, 16));
  FS_TRY(P->alloc(&P->counters, 16));
  FS_CUDA(cudaMemset(P->counters, 0, sizeof(unsigned) * 16));
  FS_TRY(P->alloc(&P->partial64, (P->ndof + 4095) / 4096 + 1));
  const int m = 30;
  // FP64 operator is always present (assembly, residual of the refinement)
  {
    P->has64 = true;
    auto& pr = P->p64;
    if (desc->precision == FS_PREC_FP64) {
      FS_TRY(setup_precision<double>(P.get(), pr, HA, HK, mplh, P->valA, P->B, P->BT,
                                     P->diagp, m));
    } else {
      pr.op.dim = dim;
      pr.op.n2 = P->n2;
      pr.op.nv = P->nv;
      pr.op.A = {(int32_t)P->n2, dm.rpA, dm.ciA, P->valA};
      pr.op.B = {(int32_t)P->nv, dm.rpB, dm.ciB, P->B};
      pr.op.BT = {(int32_t)P->n2, dm.rpBT, dm.ciBT, P->BT};
      pr.op.diagp = P->diagp;
      double avg = (double)(me.A.nnz() + me.BT.nnz()) / (double)P->n2;
      pr.lanes = avg >= 24.0 ? 8 : 4;
    }
  }
  if (desc->precision == FS_PREC_FP32_REFINE) {
    P->has32 = true;
    FS_TRY(P->alloc(&P->valA32, nnzA));
    std::vector<float> b32(Bh.begin(), Bh.end()), bt32(BTh.begin(), BTh.end()),
        d32(dp.begin(), dp.end());
    FS_TRY(P->upload(&P->B32, b32));
    FS_TRY(P->upload(&P->BT32, bt32));
    FS_TRY(P->upload(&P->diagp32, d32));
    FS_TRY(setup_precision<float>(P.get(), P->p32, HA, HK, mplh, P->valA32, P->B32, P->BT32,
                                  P->diagp32, m));
  }
  launch_exact_state(dm, P->ph, desc->t0, desc->init == 1, P->x, s);
  FS_TRY(check_launch("initial state"));
  FS_CUDA(cudaStreamSynchronize(s));
  *out = P.release();
  return FS_OK;
}

int fs_problem_destroy(fs_problem* prob) {
  if (prob) {
    cudaStreamSynchronize(prob->stream);
    delete prob;
  }
  return FS_OK;
}

int64_t fs_problem_device_bytes(const fs_problem* prob) { return prob ? prob->bytes : 0; }

int fs_assemble_step(fs_problem* P, double t_next, double* val_out, double* b_out) {
  if (!P) {
    set_error("fs_assemble_step: null problem");
    return FS_ERR_INVALID_ARG;
  }
  FS_TRY(assemble_impl(P, t_next));
  if (val_out) {
    if (!P->mrp) {
      std::vector<int64_t> rp;
      std::vector<int32_t> ci;
      monolithic_pattern(P->mesh->m, rp, ci);
      FS_TRY(P->upload(&P->mrp, rp));
    }
    launch_expand_monolithic(P->dm, P->valA, P->B, P->BT, P->diagp, P->mrp, val_out, P->stream);
    FS_TRY(check_launch("expand_monolithic"));
  }
  if (b_out)
    FS_CUDA(cudaMemcpyAsync(b_out, P->b, sizeof(double) * P->ndof, cudaMemcpyDeviceToDevice,
                            P->stream));
  return FS_OK;
}

int fs_solve(fs_problem* P, const fs_solve_opts* opts, double* x, fs_solve_stats* stats) {
  if (!P) {
    set_error("fs_solve: null problem");
    return FS_ERR_INVALID_ARG;
  }
  if (!P->assembled) {
    set_error("fs_solve: call fs_assemble_step first");
    return FS_ERR_INVALID_ARG;
  }
  fs_solve_opts o;
  fs_default_solve_opts(&o);
  if (opts) o = *opts;
  if (o.restart != 30) {
    set_error("fs_solve: this build runs GMRES(30) restart cycles");
    return FS_ERR_UNSUPPORTED;
  }
  fs_solve_stats st;
  int rc = solve_impl(P, o, x ? x : P->x, st);
  if (stats) *stats = st;
  return rc;
}

int fs_step(fs_problem* P, int nsteps, const fs_solve_opts* opts, fs_solve_stats* per_step) {
  if (!P || nsteps < 0) {
    set_error("fs_step: bad argument");
    return FS_ERR_INVALID_ARG;
  }
  fs_solve_opts o;
  fs_default_solve_opts(&o);
  if (opts) o = *opts;
  for (int k = 0; k < nsteps; ++k) {
    double t1 = P->t + P->desc.dt;
    FS_TRY(assemble_impl(P, t1));
    fs_solve_stats st;
    int rc = solve_impl(P, o, P->x, st);
    if (per_step) per_step[k] = st;
    P->t = t1;  // the state holds the best iterate even when rc != FS_OK
    if (rc != FS_OK) return rc;
  }
  return FS_OK;
}

int fs_apply_operator(fs_problem* P, const double* x, double* y) {
  if (!P || !x || !y) {
    set_error("fs_apply_operator: null argument");
    return FS_ERR_INVALID_ARG;
  }
  launch_spmv_full<double, double>(P->p64.op, x, nullptr, y, 0, nullptr, P->p64.lanes, P->stream);
  return check_launch("fs_apply_operator");
}

int fs_get_state(fs_problem* P, double* x_out, int host, double* t_out) {
  if (!P) {
    set_error("fs_get_state: null problem");
    return FS_ERR_INVALID_ARG;
  }
  if (x_out)
    FS_CUDA(cudaMemcpyAsync(x_out, P->x, sizeof(double) * P->ndof,
                            host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, P->stream));
  FS_CUDA(cudaStreamSynchronize(P->stream));
  if (t_out) *t_out = P->t;
  return FS_OK;
}

int fs_set_state(fs_problem* P, const double* x_in, int host, double t) {
  if (!P) {
    set_error("fs_set_state: null problem");
    return FS_ERR_INVALID_ARG;
  }
  if (x_in)
    FS_CUDA(cudaMemcpyAsync(P->x, x_in, sizeof(double) * P->ndof,
                            host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, P->stream));
  FS_CUDA(cudaStreamSynchronize(P->stream));
  P->t = t;
  return FS_OK;
}

int64_t fs_launch_count(void) { return g_launches.load(); }

int fs_profile_kernel(fs_problem* P, int kernel, int reps, double* avg_ms, double* alg_bytes) {
  if (!P || reps < 1 || !avg_ms || !alg_bytes) {
    set_error("fs_profile_kernel: bad argument");
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
    case FS_KERNEL_SPMV:      // saddle-point SpMV in the solver's arithmetic
    case FS_KERNEL_SPMV_FP64: {
      const bool use32 = f32 && kernel == FS_KERNEL_SPMV;
      const double sz = use32 ? 4.0 : 8.0;
      bytes = nnzA * (4 + sz) + nnzBT * (4 + d * sz) + nnzB * (4 + d * sz) +
              4.0 * (2 * (P->n2 + 1) + (P->nv + 1)) + P->nv * sz + 2.0 * P->ndof * sz;
      if (use32) {
        auto& pr = P->p32;
        launch = [P, &pr]() {
          launch_spmv_full<float, float>(pr.op, pr.kr.Vb, nullptr, pr.kr.Vb + P->ndof, 0, nullptr,
                                         pr.lanes, P->stream);
        };
      } else {
        launch = [P]() {
          launch_spmv_full<double, double>(P->p64.op, P->x, nullptr, P->r64, 0, nullptr,
                                           P->p64.lanes, P->stream);
        };
      }
      break;
    }
    case FS_KERNEL_CHEB: {  // one fused Chebyshev step on the finest velocity level
      const int64_t n = P->n2;
      bytes = nnzA * (4 + s) + 4.0 * (n + 1) + n * s + (1 + 4.0) * d * n * s;
      if (f32) {
        auto& H = P->p32.HA;
        launch = [P, &H, d]() { launch_cheb_step<float>(H, d, P->stream); };
      } else {
        auto& H = P->p64.HA;
        launch = [P, &H, d]() { launch_cheb_step<double>(H, d, P->stream); };
      }
      break;
    }
    case FS_KERNEL_ASSEMBLE_CONV: {  // per-step convection assembly (FP64)
      bytes = me.ncell * (double)me.nloc * (4 + me.nloc) + me.nv * d * 8.0 +
              (double)d * P->n2 * 8.0 + 4.0 * (P->n2 + 1) + P->n2 + 16.0 * nnzA;
      launch = [P]() {
        launch_assemble_conv(P->dm, P->x, P->n2, nullptr, P->valA, P->stream);
      };
      break;
    }
    default:
      set_error("fs_profile_kernel: unknown kernel id");
      return FS_ERR_INVALID_ARG;
  }
  cudaEvent_t e0, e1;
  FS_CUDA(cudaEventCreate(&e0));
  FS_CUDA(cudaEventCreate(&e1));
  for (int i = 0; i < 3; ++i) launch();
  FS_CUDA(cudaEventRecord(e0, P->stream));
  for (int i = 0; i < reps; ++i) launch();
  FS_CUDA(cudaEventRecord(e1, P->stream));
  FS_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FS_TRY(check_launch("fs_profile_kernel"));
  *avg_ms = ms / reps;
  *alg_bytes = bytes;
  if (kernel == FS_KERNEL_ASSEMBLE_CONV) FS_TRY(assemble_impl(P, P->t + P->desc.dt));
  return FS_OK;
}

}  // extern "C"
