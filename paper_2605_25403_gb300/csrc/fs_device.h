// Launchers of the sm_103a kernels (defined in fs_assembly.cu and
// fs_linalg.cu) and the plain views they take.  Host code only sees these
// declarations; every pointer in a view is a device pointer.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fs_internal.h"

namespace fs {

// Counts kernel launches issued from the host (ignored while a stream is
// being captured into a graph; graph replays add their node count).
void count_launches(int64_t n);

// Element-level reference integrals in constant memory (per dimension).
void upload_ref_tensors(const RefTensors& R2, const RefTensors& R3);

template <typename T>
struct DCsr {
  int32_t nrow = 0;
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const T* v = nullptr;
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
};

// Physical description of the manufactured problem.
struct DPhys {
  int kind = 0;
  double nu = 1.0;
  double wconst[3] = {0, 0, 0};
};

// ---- assembly (fs_assembly.cu) -------------------------------------------
// Step-invariant blocks, accumulated with atomics into zeroed arrays:
// base = mass_coef M + nu K (P2-P2), Mv = M, B (P1-P2, dim values per entry),
// BT (P2-P1, dim values), Kp (P1 stiffness), mpl (lumped P1 mass).
void launch_assemble_base(const DMesh& m, double mass_coef, double nu,
                          double* base, double* Mv, double* B, double* BT,
                          double* Kp, double* mpl, cudaStream_t s);
// valA += N(w) with w taken from the component-blocked vector w (ldw =
// component stride) or the constant field wc when w == nullptr; rows of
// Dirichlet nodes are skipped.
void launch_assemble_conv(const DMesh& m, const double* w, int64_t ldw,
                          const double* wc, double* valA, cudaStream_t s);
// Dirichlet rows of the scalar block become identity rows.
template <typename T>
void launch_bc_rows(const DMesh& m, T* valA, cudaStream_t s);
// F[c][j] = mass_coef * u_c[j] + f_c(x_j, t) for every P2 node.
void launch_eval_load(const DMesh& m, const DPhys& ph, double t,
                      double mass_coef, const double* u, double* F,
                      cudaStream_t s);
// b = M F (velocity rows), Dirichlet rows = u_exact(t), b_p = 0 except the
// pinned row (p_exact(x_0, t)).
void launch_rhs(const DMesh& m, const DPhys& ph, double t, const double* Mv,
                const double* F, int pin, double* b, cudaStream_t s);
// Exact state I_h u, I_h p at time t (zero_interior: 0 off Dirichlet nodes).
void launch_exact_state(const DMesh& m, const DPhys& ph, double t,
                        int zero_interior, double* x, cudaStream_t s);
// Monolithic CSR values from the block values (export for parity checks).
void launch_expand_monolithic(const DMesh& m, const double* valA,
                              const double* B, const double* BT,
                              const double* diagp, const int64_t* mrp,
                              double* out, cudaStream_t s);

// ---- linear algebra (fs_linalg.cu) ---------------------------------------
// Saddle-point operator in block form.
template <typename T>
struct DOp {
  int dim = 0;
  int64_t n2 = 0, nv = 0;
  DCsr<T> A, B, BT;     // B, BT values hold dim entries per nonzero
  const T* diagp = nullptr;
};

// y = K x (resid == 0) or y = b - K x (resid == 1); vectors of type V.
template <typename T, typename V>
void launch_spmv_full(const DOp<T>& op, const V* x, const V* b, V* y,
                      int resid, const int* skip, int lanes, cudaStream_t s);

// Multigrid level on the device.
template <typename T>
struct DLevel {
  DCsr<T> A, P, R;      // P: prolongation from level+1, R = P^T
  const T* dinv = nullptr;
  double inv_theta = 0, a1 = 0, b1 = 0, a2 = 0, b2 = 0;  // Chebyshev(3)
  int lanes = 4;
};
template <typename T>
struct DHier {
  int nlev = 0;
  DLevel<T> lev[16];
  const T* cinv = nullptr;  // dense inverse of the coarsest operator
  int64_t ncoarse = 0;
  // work vectors per level, nc components each (component stride = nrow):
  // xw/xw2 ping-pong iterates (xw also holds the level's result), dw/dw2
  // ping-pong Chebyshev directions, bw the level's right-hand side
  T* xw[16] = {};
  T* xw2[16] = {};
  T* dw[16] = {};
  T* dw2[16] = {};
  T* bw[16] = {};
};
// x = V-cycle(b) for nc right-hand sides (stride ld between components);
// x must not alias b.
template <typename T>
void mg_vcycle(const DHier<T>& H, int nc, const T* b, int64_t ld, T* x,
               const int* skip, cudaStream_t s);

// One fused Chebyshev step (mode STEP) on level 0 of H with its own work
// vectors, for kernel timing.
template <typename T>
void launch_cheb_step(const DHier<T>& H, int nc, cudaStream_t s);

// Krylov helpers (fs_linalg.cu).  Results land in device doubles.
struct GmresState;
template <typename V>
void launch_norm2(const V* x, int64_t n, double* partial, unsigned* counter,
                  double* out, int op, const int* skip, cudaStream_t s);
template <typename V>
void launch_scale(V* x, int64_t n, const double* num, const double* den,
                  int inv_sqrt_den, const int* skip, cudaStream_t s);
template <typename V>
void launch_cgs2(V* Vb, int64_t n, int j, GmresState* st, double* partial,
                 const int* skip, cudaStream_t s);
void launch_givens(GmresState* st, int j, cudaStream_t s);
void launch_cycle_init(GmresState* st, cudaStream_t s);
template <typename V, typename X>
void launch_update_x(GmresState* st, const V* Z, int64_t n, X* x,
                     double xscale_from_beta, cudaStream_t s);
template <typename A, typename B>
void launch_convert(const A* in, B* out, int64_t n, const double* scale,
                    int inv, cudaStream_t s);
template <typename V, typename X>
void launch_axpy_mixed(X* x, const V* d, int64_t n, const double* alpha,
                       cudaStream_t s);
template <typename T>
void launch_precond(const DOp<T>& op, const DHier<T>& HA, const DHier<T>& HK,
                    const T* mpl_inv_nu, double inv_dt, const int32_t* pinned,
                    int npinned, const T* r, T* z, T* work_p, T* work_u,
                    const int* skip, cudaStream_t s);

// Device-resident restart-cycle state of flexible GMRES(m).
struct GmresState {
  double H[(kMaxRestart + 1) * kMaxRestart];
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1];
  double y[kMaxRestart];
  double h2[kMaxRestart + 1];
  double beta;      // ||r0|| of the cycle
  double tol_abs;   // Arnoldi residual target
  double resid;     // current residual estimate |g_{k}|
  double hn;        // ||w|| before normalisation
  int m;            // restart length
  int done;         // 1: converged (or breakdown) -> kernels skip
  int k;            // iterations taken in this cycle
  int bad;          // NaN/Inf seen
  unsigned counter[4];
};

}  // namespace fs
