// Incremental pressure-correction stepping (paper Sec. 2.2.1, IPCS) on
// sm_103a: the right-hand sides of its three stages, the operators of their
// three symmetric positive definite systems, and the kernels of the
// Jacobi-preconditioned conjugate gradient method that solves them.
//
// Everything is FP64 and in the problem's internal node order; velocity
// vectors are component-blocked [u_x | u_y | (u_z)] (d n2 entries), pressure
// vectors hold one entry per vertex.  A system's fixed unknowns (Dirichlet
// velocity nodes, the pinned pressure vertex) are identity rows of its
// operator: the CG iterates start with their values in place, so the
// residual and every search direction vanish there, and on the free
// unknowns the operator acts as the symmetric block the elimination of the
// fixed ones leaves.
#include <cuda_runtime.h>

#include "fs_device.h"

namespace fs {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCgThreads = 256;

inline unsigned row_blocks(int64_t rows) {
  const int64_t g = (rows + kCgThreads - 1) / kCgThreads;
  return (unsigned)(g < 1 ? 1 : g);
}

// Block sums of two values (valid in thread 0).
__device__ __forceinline__ void block_sum2(double& s0, double& s1) {
  __shared__ double sh[2][kCgThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(kFull, s0, off);
    s1 += __shfl_xor_sync(kFull, s1, off);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0][w] = s0;
    sh[1][w] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s0 = s1 = 0;
    for (int i = 0; i < kCgThreads / 32; ++i) {
      s0 += sh[0][i];
      s1 += sh[1][i];
    }
  }
}

__device__ __forceinline__ void write_part(double* part, double s0, double s1) {
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

// ---- right-hand sides ------------------------------------------------------
// Stage 1 (tentative velocity): r = M (u^n/dt + I_h f^{n+1}) - N(w) u^n +
// B^T p^n on free rows, where b holds the first term and N(w) = valA - base
// off the Dirichlet rows; r = b (the Dirichlet value) on Dirichlet rows.
template <int DIM>
__global__ void __launch_bounds__(kCgThreads) k_ipcs_rhs1(DMesh m, const double* __restrict__ valA,
                                                          const double* __restrict__ base,
                                                          const double* __restrict__ BT,
                                                          const double* __restrict__ b,
                                                          const double* __restrict__ x,
                                                          double* __restrict__ r) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n2 = m.n2;
  if (i >= n2) return;
  if (m.dirichlet[i]) {
#pragma unroll
    for (int c = 0; c < DIM; ++c) r[c * n2 + i] = b[c * n2 + i];
    return;
  }
  double s[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) s[c] = b[c * n2 + i];
  for (int32_t k = m.rpA[i]; k < m.rpA[i + 1]; ++k) {
    const double a = valA[k] - base[k];
    const int32_t j = m.ciA[k];
#pragma unroll
    for (int c = 0; c < DIM; ++c) s[c] -= a * x[c * n2 + j];
  }
  const double* __restrict__ p = x + DIM * n2;
  for (int32_t k = m.rpBT[i]; k < m.rpBT[i + 1]; ++k) {
    const double pq = p[m.ciBT[k]];
#pragma unroll
    for (int c = 0; c < DIM; ++c) s[c] += BT[(int64_t)k * DIM + c] * pq;
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) r[c * n2 + i] = s[c];
}

// Stage 2 (pressure increment): r_q = -(1/dt) (div u*, psi_q) = -(1/dt)
// (B u*)_q; a fixed vertex takes p_exact(x_q, t^{n+1}) - p^n_q (b holds the
// exact value in its pressure row, x the state).
template <int DIM>
__global__ void __launch_bounds__(kCgThreads) k_ipcs_rhs2(DMesh m, const double* __restrict__ B,
                                                          const double* __restrict__ ustar,
                                                          double inv_dt,
                                                          const uint8_t* __restrict__ fixed,
                                                          const double* __restrict__ b,
                                                          const double* __restrict__ x,
                                                          double* __restrict__ r) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n2 = m.n2;
  if (q >= m.nv) return;
  if (fixed[q]) {
    r[q] = b[DIM * n2 + q] - x[DIM * n2 + q];
    return;
  }
  double s = 0;
  for (int32_t k = m.rpB[q]; k < m.rpB[q + 1]; ++k) {
    const int32_t j = m.ciB[k];
#pragma unroll
    for (int c = 0; c < DIM; ++c) s += B[(int64_t)k * DIM + c] * ustar[c * n2 + j];
  }
  r[q] = -inv_dt * s;
}

// Stage 3 (velocity correction): r = M u* + dt B^T dp on free rows (the
// weak gradient of dp against test functions vanishing on the boundary),
// the Dirichlet value on Dirichlet rows.
template <int DIM>
__global__ void __launch_bounds__(kCgThreads) k_ipcs_rhs3(DMesh m, const double* __restrict__ Mv,
                                                          const double* __restrict__ BT,
                                                          const double* __restrict__ b,
                                                          const double* __restrict__ ustar,
                                                          const double* __restrict__ dp,
                                                          double dt, double* __restrict__ r) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n2 = m.n2;
  if (i >= n2) return;
  if (m.dirichlet[i]) {
#pragma unroll
    for (int c = 0; c < DIM; ++c) r[c * n2 + i] = b[c * n2 + i];
    return;
  }
  double s[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) s[c] = 0;
  for (int32_t k = m.rpA[i]; k < m.rpA[i + 1]; ++k) {
    const double a = Mv[k];
    const int32_t j = m.ciA[k];
#pragma unroll
    for (int c = 0; c < DIM; ++c) s[c] += a * ustar[c * n2 + j];
  }
  for (int32_t k = m.rpBT[i]; k < m.rpBT[i + 1]; ++k) {
    const double d = dp[m.ciBT[k]];
#pragma unroll
    for (int c = 0; c < DIM; ++c) s[c] += dt * BT[(int64_t)k * DIM + c] * d;
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) r[c * n2 + i] = s[c];
}

// ---- operators (y = A x, with per-block partials of x . y and 0) -----------
// The scalar P2 block with values vals (M/dt + nu K for stage 1, M for
// stage 3) on every component; identity rows at Dirichlet nodes.
template <int DIM>
__global__ void __launch_bounds__(kCgThreads) k_ipcs_apply_vel(DMesh m,
                                                               const double* __restrict__ vals,
                                                               const double* __restrict__ x,
                                                               double* __restrict__ y,
                                                               double* part) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n2 = m.n2;
  double xy = 0;
  if (i < n2) {
    double s[DIM];
    if (m.dirichlet[i]) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) s[c] = x[c * n2 + i];
    } else {
#pragma unroll
      for (int c = 0; c < DIM; ++c) s[c] = 0;
      for (int32_t k = m.rpA[i]; k < m.rpA[i + 1]; ++k) {
        const double a = vals[k];
        const int32_t j = m.ciA[k];
#pragma unroll
        for (int c = 0; c < DIM; ++c) s[c] += a * x[c * n2 + j];
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      y[c * n2 + i] = s[c];
      xy += x[c * n2 + i] * s[c];
    }
  }
  if (part) write_part(part, xy, 0.0);
}

// The P1 pressure Laplacian; identity rows at the fixed vertices.
__global__ void __launch_bounds__(kCgThreads) k_ipcs_apply_p(DMesh m, const double* __restrict__ Kp,
                                                             const uint8_t* __restrict__ fixed,
                                                             const double* __restrict__ x,
                                                             double* __restrict__ y,
                                                             double* part) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double xy = 0;
  if (q < m.nv) {
    double s = 0;
    if (fixed[q]) {
      s = x[q];
    } else {
      for (int32_t k = m.rpK[q]; k < m.rpK[q + 1]; ++k) s += Kp[k] * x[m.ciK[k]];
    }
    y[q] = s;
    xy = x[q] * s;
  }
  if (part) write_part(part, xy, 0.0);
}

// Inverse diagonals of the three operators (1 on fixed rows), laid out like
// the vectors they scale.
template <int DIM>
__global__ void k_ipcs_dinv_vel(DMesh m, const double* __restrict__ vals,
                                double* __restrict__ dinv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m.n2) return;
  double d = 1.0;
  if (!m.dirichlet[i])
    for (int32_t k = m.rpA[i]; k < m.rpA[i + 1]; ++k)
      if (m.ciA[k] == i) d = 1.0 / vals[k];
#pragma unroll
  for (int c = 0; c < DIM; ++c) dinv[c * m.n2 + i] = d;
}

__global__ void k_ipcs_dinv_p(DMesh m, const double* __restrict__ Kp,
                              const uint8_t* __restrict__ fixed, double* __restrict__ dinv) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= m.nv) return;
  double d = 1.0;
  if (!fixed[q])
    for (int32_t k = m.rpK[q]; k < m.rpK[q + 1]; ++k)
      if (m.ciK[k] == q) d = 1.0 / Kp[k];
  dinv[q] = d;
}

// Start vector of a system: its fixed unknowns take their values (held by
// the right-hand side there), the others keep the guess in x.
template <int DIM>
__global__ void k_ipcs_fix_vel(DMesh m, const double* __restrict__ rhs, double* __restrict__ x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m.n2 || !m.dirichlet[i]) return;
#pragma unroll
  for (int c = 0; c < DIM; ++c) x[c * m.n2 + i] = rhs[c * m.n2 + i];
}
__global__ void k_ipcs_fix_p(int64_t nv, const uint8_t* __restrict__ fixed,
                             const double* __restrict__ rhs, double* __restrict__ x) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < nv && fixed[q]) x[q] = rhs[q];
}
// y += x (n entries)
__global__ void k_ipcs_add(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// ---- conjugate gradient vector kernels ---------------------------------
// sc: the CG scalars on the device: 0 rz = r.z, 1 alpha, 2 beta, 3 rr = r.r
constexpr int kFlatBlocks = 304;

// r = rhs - y, z = dinv r, p = z; partials (r.z, r.r)
__global__ void __launch_bounds__(kCgThreads) k_cg_init(int64_t n, const double* __restrict__ rhs,
                                                        const double* __restrict__ y,
                                                        const double* __restrict__ dinv,
                                                        double* __restrict__ r,
                                                        double* __restrict__ z,
                                                        double* __restrict__ p, double* part) {
  double rz = 0, rr = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = rhs[i] - y[i], zi = dinv[i] * ri;
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
  }
  write_part(part, rz, rr);
}

// x += alpha p, r -= alpha q, z = dinv r; partials (r.z, r.r)
__global__ void __launch_bounds__(kCgThreads) k_cg_update(int64_t n, const double* __restrict__ sc,
                                                          const double* __restrict__ p,
                                                          const double* __restrict__ q,
                                                          const double* __restrict__ dinv,
                                                          double* __restrict__ x,
                                                          double* __restrict__ r,
                                                          double* __restrict__ z, double* part) {
  const double alpha = sc[1];
  double rz = 0, rr = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i], zi = dinv[i] * ri;
    r[i] = ri;
    z[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
  }
  write_part(part, rz, rr);
}

// Flexible CG (variable preconditioner): t = r, x += alpha p, r -= alpha q;
// partials (0, r.r)
__global__ void __launch_bounds__(kCgThreads) k_cg_update_flex(
    int64_t n, const double* __restrict__ sc, const double* __restrict__ p,
    const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
    double* __restrict__ t, double* part) {
  const double alpha = sc[1];
  double rr = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ro = r[i], ri = ro - alpha * q[i];
    t[i] = ro;
    r[i] = ri;
    rr += ri * ri;
  }
  write_part(part, 0.0, rr);
}

// z = 0 on fixed rows (so that the search directions keep the fixed values),
// then partials (r.z, t.z); with first, also p = z (the start of the
// iteration)
__global__ void __launch_bounds__(kCgThreads) k_cg_dots_flex(int64_t n,
                                                             const uint8_t* __restrict__ fixed,
                                                             const double* __restrict__ r,
                                                             const double* __restrict__ t,
                                                             double* __restrict__ z,
                                                             double* __restrict__ p, int first,
                                                             double* part) {
  double rz = 0, tz = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double zi = z[i];
    if (fixed && fixed[i]) {
      zi = 0.0;
      z[i] = 0.0;
    }
    rz += r[i] * zi;
    tz += (first ? 0.0 : t[i] * zi);
    if (first) p[i] = zi;
  }
  write_part(part, rz, tz);
}

// p = z + beta p
__global__ void __launch_bounds__(kCgThreads) k_cg_dir(int64_t n, const double* __restrict__ sc,
                                                       const double* __restrict__ z,
                                                       double* __restrict__ p) {
  const double beta = sc[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// Sums nb block partials in a fixed order, then (one thread):
//   mode 0 (after init):   rz = s0, rr = s1
//   mode 1 (after apply):  alpha = rz / s0 (s0 = p . A p)
//   mode 2 (after update): beta = s0 / rz, rz = s0, rr = s1
//   mode 3 (after a flexible update): rr = s1
//   mode 4 (after the flexible dots): beta = (s0 - s1) / rz, rz = s0
//     (Polak-Ribiere: z_new . (r_new - r_old) / (z_old . r_old))
//   mode 5 (first flexible dots): rz = s0
__global__ void __launch_bounds__(kCgThreads) k_cg_scalars(const double* part, int nb, int mode,
                                                           double* sc) {
  double s0 = 0, s1 = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s0 += part[2 * i];
    s1 += part[2 * i + 1];
  }
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    if (mode == 0) {
      sc[0] = s0;
      sc[3] = s1;
    } else if (mode == 1) {
      sc[1] = s0 != 0.0 ? sc[0] / s0 : 0.0;
    } else if (mode == 2) {
      sc[2] = sc[0] != 0.0 ? s0 / sc[0] : 0.0;
      sc[0] = s0;
      sc[3] = s1;
    } else if (mode == 3) {
      sc[3] = s1;
    } else if (mode == 4) {
      sc[2] = sc[0] != 0.0 ? (s0 - s1) / sc[0] : 0.0;
      sc[0] = s0;
    } else {
      sc[0] = s0;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
int ipcs_part_size(const DMesh& m) {
  const int64_t rows = m.n2 > m.nv ? m.n2 : m.nv;
  const int64_t nb = row_blocks(rows);
  return (int)(2 * (nb > kFlatBlocks ? nb : kFlatBlocks));
}

void launch_ipcs_rhs1(const DMesh& m, const double* valA, const double* base, const double* BT,
                      const double* b, const double* x, double* r, cudaStream_t s) {
  if (m.dim == 2)
    k_ipcs_rhs1<2><<<row_blocks(m.n2), kCgThreads, 0, s>>>(m, valA, base, BT, b, x, r);
  else
    k_ipcs_rhs1<3><<<row_blocks(m.n2), kCgThreads, 0, s>>>(m, valA, base, BT, b, x, r);
  count_launches(1);
}

void launch_ipcs_rhs2(const DMesh& m, const double* B, const double* ustar, double inv_dt,
                      const uint8_t* fixed, const double* b, const double* x, double* r,
                      cudaStream_t s) {
  if (m.dim == 2)
    k_ipcs_rhs2<2><<<row_blocks(m.nv), kCgThreads, 0, s>>>(m, B, ustar, inv_dt, fixed, b, x, r);
  else
    k_ipcs_rhs2<3><<<row_blocks(m.nv), kCgThreads, 0, s>>>(m, B, ustar, inv_dt, fixed, b, x, r);
  count_launches(1);
}

void launch_ipcs_rhs3(const DMesh& m, const double* Mv, const double* BT, const double* b,
                      const double* ustar, const double* dp, double dt, double* r,
                      cudaStream_t s) {
  if (m.dim == 2)
    k_ipcs_rhs3<2><<<row_blocks(m.n2), kCgThreads, 0, s>>>(m, Mv, BT, b, ustar, dp, dt, r);
  else
    k_ipcs_rhs3<3><<<row_blocks(m.n2), kCgThreads, 0, s>>>(m, Mv, BT, b, ustar, dp, dt, r);
  count_launches(1);
}

int launch_ipcs_apply(const DMesh& m, int which, const double* vals, const uint8_t* fixed,
                      const double* x, double* y, double* part, cudaStream_t s) {
  if (which == 1) {
    const unsigned g = row_blocks(m.nv);
    k_ipcs_apply_p<<<g, kCgThreads, 0, s>>>(m, vals, fixed, x, y, part);
    count_launches(1);
    return (int)g;
  }
  const unsigned g = row_blocks(m.n2);
  if (m.dim == 2)
    k_ipcs_apply_vel<2><<<g, kCgThreads, 0, s>>>(m, vals, x, y, part);
  else
    k_ipcs_apply_vel<3><<<g, kCgThreads, 0, s>>>(m, vals, x, y, part);
  count_launches(1);
  return (int)g;
}

void launch_ipcs_dinv(const DMesh& m, int which, const double* vals, const uint8_t* fixed,
                      double* dinv, cudaStream_t s) {
  if (which == 1) {
    k_ipcs_dinv_p<<<row_blocks(m.nv), kCgThreads, 0, s>>>(m, vals, fixed, dinv);
  } else if (m.dim == 2) {
    k_ipcs_dinv_vel<2><<<row_blocks(m.n2), kCgThreads, 0, s>>>(m, vals, dinv);
  } else {
    k_ipcs_dinv_vel<3><<<row_blocks(m.n2), kCgThreads, 0, s>>>(m, vals, dinv);
  }
  count_launches(1);
}

void launch_ipcs_fix(const DMesh& m, int which, const uint8_t* fixed, const double* rhs,
                     double* x, cudaStream_t s) {
  if (which == 1)
    k_ipcs_fix_p<<<row_blocks(m.nv), kCgThreads, 0, s>>>(m.nv, fixed, rhs, x);
  else if (m.dim == 2)
    k_ipcs_fix_vel<2><<<row_blocks(m.n2), kCgThreads, 0, s>>>(m, rhs, x);
  else
    k_ipcs_fix_vel<3><<<row_blocks(m.n2), kCgThreads, 0, s>>>(m, rhs, x);
  count_launches(1);
}

void launch_ipcs_add(int64_t n, const double* x, double* y, cudaStream_t s) {
  k_ipcs_add<<<kFlatBlocks, kCgThreads, 0, s>>>(n, x, y);
  count_launches(1);
}

void launch_cg_init(int64_t n, const double* rhs, const double* y, const double* dinv, double* r,
                    double* z, double* p, double* part, double* sc, cudaStream_t s) {
  k_cg_init<<<kFlatBlocks, kCgThreads, 0, s>>>(n, rhs, y, dinv, r, z, p, part);
  k_cg_scalars<<<1, kCgThreads, 0, s>>>(part, kFlatBlocks, 0, sc);
  count_launches(2);
}

void launch_cg_alpha(const double* part, int nb, double* sc, cudaStream_t s) {
  k_cg_scalars<<<1, kCgThreads, 0, s>>>(part, nb, 1, sc);
  count_launches(1);
}

void launch_cg_update(int64_t n, double* sc, const double* p, const double* q,
                      const double* dinv, double* x, double* r, double* z, double* part,
                      cudaStream_t s) {
  k_cg_update<<<kFlatBlocks, kCgThreads, 0, s>>>(n, sc, p, q, dinv, x, r, z, part);
  k_cg_scalars<<<1, kCgThreads, 0, s>>>(part, kFlatBlocks, 2, sc);
  count_launches(2);
}

void launch_cg_update_flex(int64_t n, double* sc, const double* p, const double* q, double* x,
                           double* r, double* t, double* part, cudaStream_t s) {
  k_cg_update_flex<<<kFlatBlocks, kCgThreads, 0, s>>>(n, sc, p, q, x, r, t, part);
  k_cg_scalars<<<1, kCgThreads, 0, s>>>(part, kFlatBlocks, 3, sc);
  count_launches(2);
}

void launch_cg_dots_flex(int64_t n, const uint8_t* fixed, const double* r, const double* t,
                         double* z, double* p, int first, double* part, double* sc,
                         cudaStream_t s) {
  k_cg_dots_flex<<<kFlatBlocks, kCgThreads, 0, s>>>(n, fixed, r, t, z, p, first, part);
  k_cg_scalars<<<1, kCgThreads, 0, s>>>(part, kFlatBlocks, first ? 5 : 4, sc);
  count_launches(2);
}

void launch_cg_dir(int64_t n, const double* sc, const double* z, double* p, cudaStream_t s) {
  k_cg_dir<<<kFlatBlocks, kCgThreads, 0, s>>>(n, sc, z, p);
  count_launches(1);
}

}  // namespace fs
