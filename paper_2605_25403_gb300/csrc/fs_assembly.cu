// Per-element assembly of the Oseen system on sm_103a, the right-hand side
// and the boundary rows.
//
// Paper Sec. 2.2.1 (Oseen equation): the bilinear form
//   (u/dt, v) + ((w.grad) u, v) + nu (grad u, grad v) - (p, div v) + (div u, q)
// on P2/P1 Taylor-Hood elements, and the load (f^{n+1}, v) + (u^n/dt, v).
// Sec. 3.1 names these BForm / LForm; here they are element kernels that
// scatter into the fixed block-CSR pattern through per-element slot tables
// (row offset + uint8 position), so no sort and no COO step runs per step.
//
// Element integrals: with grad(lambda_r) the (constant) barycentric
// gradients and D = |det J|, each block is D times a contraction of a
// reference-simplex integral with geometric coefficients:
//   M_ij = D mass_ij,   K_ij = D sum_rs (grad l_r . grad l_s) stiff_ijrs,
//   N_ij = D sum_k sum_(j,r) (w_k . grad l_r) conv_ik(j,r),
//   B^c_qj = D sum_r (d l_r/d x_c) div_qjr.
// The reference integrals come from a degree-5 Grundmann-Moeller rule
// (exact for these polynomial integrands) evaluated once on the host.
#include <cuda_runtime.h>

#include <cstdio>

#include "fs_device.h"

namespace fs {

struct CRef {
  double mass[kMaxLoc][kMaxLoc];
  double stiff[kMaxLoc][kMaxLoc][4][4];
  double conv[kMaxLoc][kMaxLoc][16];
  double div[4][kMaxLoc][4];
  double pmass[4][kMaxLoc];
};
__constant__ CRef c_ref[2];

void upload_ref_tensors(const RefTensors& R2, const RefTensors& R3) {
  CRef h[2];
  const RefTensors* src[2] = {&R2, &R3};
  for (int d = 0; d < 2; ++d) {
    memcpy(h[d].mass, src[d]->mass, sizeof(h[d].mass));
    memcpy(h[d].stiff, src[d]->stiff, sizeof(h[d].stiff));
    memcpy(h[d].conv, src[d]->conv, sizeof(h[d].conv));
    memcpy(h[d].div, src[d]->div, sizeof(h[d].div));
    memcpy(h[d].pmass, src[d]->pmass, sizeof(h[d].pmass));
  }
  cudaMemcpyToSymbol(c_ref, h, sizeof(h));
}

namespace {

// Nonzero (j, r) pairs of d phi_j / d lambda_r in the local node order
// (vertices, then edges (1,2),(2,0),(0,1) / (0,1),(0,2),(0,3),(1,2),(1,3),
// (2,3)); the host reference tensors use the same order.
template <int DIM> struct Pairs;
template <> struct Pairs<2> {
  static constexpr int n = 9;
  __device__ static constexpr int j(int p) {
    constexpr int t[9] = {0, 1, 2, 3, 3, 4, 4, 5, 5};
    return t[p];
  }
  __device__ static constexpr int r(int p) {
    constexpr int t[9] = {0, 1, 2, 1, 2, 2, 0, 0, 1};
    return t[p];
  }
};
template <> struct Pairs<3> {
  static constexpr int n = 16;
  __device__ static constexpr int j(int p) {
    constexpr int t[16] = {0, 1, 2, 3, 4, 4, 5, 5, 6, 6, 7, 7, 8, 8, 9, 9};
    return t[p];
  }
  __device__ static constexpr int r(int p) {
    constexpr int t[16] = {0, 1, 2, 3, 0, 1, 0, 2, 0, 3, 1, 2, 1, 3, 2, 3};
    return t[p];
  }
};

template <int DIM> struct Loc { static constexpr int nb = DIM + 1, nl = DIM == 2 ? 6 : 10; };

// Barycentric gradients of one affine simplex: with edge vectors e_r =
// x_{r+1} - x_0, the gradients of lambda_1..d form the dual basis of
// (e_1..e_d); grad lambda_0 = -(sum of the others).  Returns |det J|.
template <int DIM>
__device__ __forceinline__ double bary_grads(const double (&xv)[DIM + 1][DIM],
                                             double (&gl)[DIM + 1][DIM]) {
  double e[DIM][DIM];
#pragma unroll
  for (int r = 0; r < DIM; ++r)
#pragma unroll
    for (int a = 0; a < DIM; ++a) e[r][a] = xv[r + 1][a] - xv[0][a];
  double det;
  if constexpr (DIM == 2) {
    det = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    double id = 1.0 / det;
    // dual basis: g1 . e1 = 1, g1 . e2 = 0, ...
    gl[1][0] = e[1][1] * id;  gl[1][1] = -e[1][0] * id;
    gl[2][0] = -e[0][1] * id; gl[2][1] = e[0][0] * id;
  } else {
    double c12[3] = {e[1][1] * e[2][2] - e[1][2] * e[2][1],
                     e[1][2] * e[2][0] - e[1][0] * e[2][2],
                     e[1][0] * e[2][1] - e[1][1] * e[2][0]};
    double c20[3] = {e[2][1] * e[0][2] - e[2][2] * e[0][1],
                     e[2][2] * e[0][0] - e[2][0] * e[0][2],
                     e[2][0] * e[0][1] - e[2][1] * e[0][0]};
    double c01[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1],
                     e[0][2] * e[1][0] - e[0][0] * e[1][2],
                     e[0][0] * e[1][1] - e[0][1] * e[1][0]};
    det = e[0][0] * c12[0] + e[0][1] * c12[1] + e[0][2] * c12[2];
    double id = 1.0 / det;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      gl[1][a] = c12[a] * id;
      gl[2][a] = c20[a] * id;
      gl[3][a] = c01[a] * id;
    }
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double s = 0;
#pragma unroll
    for (int r = 1; r <= DIM; ++r) s += gl[r][a];
    gl[0][a] = -s;
  }
  return fabs(det);
}

template <int DIM>
__device__ __forceinline__ void load_cell(const DMesh& m, int64_t e,
                                          int32_t (&g)[Loc<DIM>::nl],
                                          double (&xv)[DIM + 1][DIM]) {
  constexpr int NL = Loc<DIM>::nl;
#pragma unroll
  for (int a = 0; a < NL; ++a) g[a] = __ldg(m.c2d + e * NL + a);
#pragma unroll
  for (int v = 0; v <= DIM; ++v)
#pragma unroll
    for (int a = 0; a < DIM; ++a) xv[v][a] = __ldg(m.p2xyz + (int64_t)g[v] * DIM + a);
}

template <int DIM>
__global__ void __launch_bounds__(128) k_assemble_base(
    DMesh m, int64_t c0, int64_t c1, double mass_coef, double nu, double* __restrict__ base,
    double* __restrict__ Mv, double* __restrict__ B, double* __restrict__ BT,
    double* __restrict__ Kp, double* __restrict__ mpl) {
  constexpr int NB = DIM + 1, NL = Loc<DIM>::nl;
  const CRef& R = c_ref[DIM - 2];
  for (int64_t idx = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < c1;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = m.color_cells[idx];
    int32_t g[NL];
    double xv[NB][DIM], gl[NB][DIM];
    load_cell<DIM>(m, e, g, xv);
    double D = bary_grads<DIM>(xv, gl);
    const double nu_e = m.nu_cell ? m.nu_cell[e] : nu;
    double G[NB][NB];
#pragma unroll
    for (int r = 0; r < NB; ++r)
#pragma unroll
      for (int s = 0; s < NB; ++s) {
        double t = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) t += gl[r][a] * gl[s][a];
        G[r][s] = t;
      }
    for (int i = 0; i < NL; ++i) {
      int32_t rowbase = __ldg(m.rpA + g[i]);
      const uint8_t* pos = m.posA + (e * NL + i) * NL;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        double mm = D * R.mass[i][j];
        double kk = 0;
#pragma unroll
        for (int r = 0; r < NB; ++r)
#pragma unroll
          for (int s = 0; s < NB; ++s) kk += G[r][s] * R.stiff[i][j][r][s];
        kk *= D;
        int32_t slot = rowbase + pos[j];
        base[slot] += mass_coef * mm + nu_e * kk;
        Mv[slot] += mm;
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q)
      for (int j = 0; j < NL; ++j) {
        double bv[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          double s = 0;
#pragma unroll
          for (int r = 0; r < NB; ++r) s += gl[r][c] * R.div[q][j][r];
          bv[c] = D * s;
        }
        int64_t sB = __ldg(m.rpB + g[q]) + m.posB[(e * NB + q) * NL + j];
        int64_t sBT = __ldg(m.rpBT + g[j]) + m.posBT[(e * NL + j) * NB + q];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          B[sB * DIM + c] += bv[c];
          BT[sBT * DIM + c] += bv[c];
        }
      }
    const double vol = D / (DIM == 2 ? 2.0 : 6.0);
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      int32_t rb = __ldg(m.rpK + g[q]);
#pragma unroll
      for (int s = 0; s < NB; ++s) Kp[rb + m.posK[(e * NB + q) * NB + s]] += vol * G[q][s];
      mpl[g[q]] += vol / NB;
    }
  }
}

// Convection element matrices N_K(w) (the per-step part of the Oseen
// operator), added into valA colour by colour: a launch takes the cells
// color_cells[c0 .. c1) of one colour (they share no node, so the plain
// read-modify-writes of different cells never meet, and every value is
// summed in the colour order on every run).  One thread per (cell, row i):
// a block takes kConvCells cells; one thread per cell computes D = |det J|
// and the barycentric gradients, every thread the coefficients
// cw[k][r] = D (w_k . grad lambda_r) of its node k = i, and then its row
//   N_ij = sum_k sum_(j,r) cw[k][r] conv_ik(j,r)
// from the reference tensor staged in shared memory.  Rows of Dirichlet
// nodes are skipped.  A thread does one row's nloc x pairs FMAs (160 in 3D)
// instead of a cell's ten rows: ten times the threads and a fifth of the
// registers, which keeps the FP64 pipe busy even when a colour holds a
// sixteenth of the cells.
template <int DIM>
struct ConvCfg {
  static constexpr int NL = Loc<DIM>::nl, NB = DIM + 1, NP = Pairs<DIM>::n;
  static constexpr int CPB = 128 / NL;  // cells per block (21 / 12)
  // shared-memory row strides (doubles) padded so that the rows the threads
  // of a warp read at one (k, q) fall in different banks: 3D 160 -> 161
  // (a multiple of 32 banks put the ten rows of a cell in one bank)
  static constexpr int RS = NL * NP + (DIM == 3 ? 1 : 0);
  static constexpr int CS = NL * NB + (DIM == 3 ? 1 : 0);
};

template <int DIM>
__global__ void __launch_bounds__(128) k_conv_elem(DMesh m, int64_t c0, int64_t c1,
                                                   const double* __restrict__ w, int64_t ldw,
                                                   double wc0, double wc1, double wc2,
                                                   double* __restrict__ valA) {
  using C = ConvCfg<DIM>;
  constexpr int NL = C::NL, NB = C::NB, NP = C::NP, CPB = C::CPB;
  constexpr int RS = C::RS, CS = C::CS;
  __shared__ double s_conv[NL * RS];  // row i of the tensor at i RS + k NP + q
  __shared__ double s_gl[CPB][NB][DIM];
  __shared__ double s_D[CPB];
  __shared__ double s_cw[CPB * CS];   // cell c's cw[k][r] at c CS + k NB + r
  __shared__ int32_t s_g[CPB][NL];
  const CRef& R = c_ref[DIM - 2];
  for (int t = threadIdx.x; t < NL * NL * NP; t += blockDim.x) {
    const int i = t / (NL * NP), k = (t / NP) % NL, q = t % NP;
    s_conv[i * RS + k * NP + q] = R.conv[i][k][q];
  }
  const int cl = threadIdx.x / NL, i = threadIdx.x % NL;
  const int64_t idx = c0 + blockIdx.x * (int64_t)CPB + cl;
  const bool active = cl < CPB && idx < c1;
  const int64_t e = active ? __ldg(m.color_cells + idx) : 0;
  int32_t gi = 0;
  if (active) {
    gi = __ldg(m.c2d + e * NL + i);
    s_g[cl][i] = gi;
  }
  __syncthreads();
  if (active && i == 0) {
    double xv[NB][DIM], gl[NB][DIM];
#pragma unroll
    for (int v = 0; v < NB; ++v)
#pragma unroll
      for (int a = 0; a < DIM; ++a) xv[v][a] = __ldg(m.p2xyz + (int64_t)s_g[cl][v] * DIM + a);
    s_D[cl] = bary_grads<DIM>(xv, gl);
#pragma unroll
    for (int r = 0; r < NB; ++r)
#pragma unroll
      for (int a = 0; a < DIM; ++a) s_gl[cl][r][a] = gl[r][a];
  }
  __syncthreads();
  if (active) {
    double wk[DIM];
    if (w) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) wk[c] = __ldg(w + c * ldw + gi);
    } else {
      wk[0] = wc0;
      wk[1] = wc1;
      if constexpr (DIM == 3) wk[2] = wc2;
    }
    const double D = s_D[cl];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      double t = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) t += wk[c] * s_gl[cl][r][c];
      s_cw[cl * CS + i * NB + r] = D * t;
    }
  }
  __syncthreads();
  if (!active || __ldg(m.dirichlet + gi)) return;
  double acc[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) acc[j] = 0.0;
#pragma unroll
  for (int k = 0; k < NL; ++k)
#pragma unroll
    for (int q = 0; q < NP; ++q)
      acc[Pairs<DIM>::j(q)] +=
          s_cw[cl * CS + k * NB + Pairs<DIM>::r(q)] * s_conv[i * RS + k * NP + q];
  double* __restrict__ row = valA + __ldg(m.rpA + gi);
  const uint8_t* pos = m.posA + (e * NL + i) * NL;
#pragma unroll
  for (int j = 0; j < NL; ++j) row[__ldg(pos + j)] += acc[j];
}

// Convection on the pressure space, Np[q][s] = int psi_q (w . grad psi_s)
// over P1 basis functions psi (the vertices of the cell) with the P2 field w
// (the convection part of the pressure convection-diffusion operator of the
// Schur-complement approximation): a thread per cell, FP64 atomics into the
// P1-P1 pattern; rows of fixed vertices stay zero.
template <int DIM>
__global__ void __launch_bounds__(128) k_conv_p1(DMesh m, const double* __restrict__ w,
                                                 int64_t ldw, double wc0, double wc1,
                                                 double wc2, const uint8_t* __restrict__ fixed,
                                                 double* __restrict__ Np) {
  constexpr int NB = DIM + 1, NL = Loc<DIM>::nl;
  const CRef& R = c_ref[DIM - 2];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.ncell;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t g[NL];
    double xv[NB][DIM], gl[NB][DIM];
    load_cell<DIM>(m, e, g, xv);
    const double D = bary_grads<DIM>(xv, gl);
    // wg[s][q] = sum_k (w_k . grad lambda_s) int lambda_q phi_k
    double wg[NB][NB];
#pragma unroll
    for (int s = 0; s < NB; ++s)
#pragma unroll
      for (int q = 0; q < NB; ++q) wg[s][q] = 0.0;
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      double wk[DIM];
      if (w) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) wk[c] = __ldg(w + c * ldw + g[k]);
      } else {
        wk[0] = wc0;
        wk[1] = wc1;
        if constexpr (DIM == 3) wk[2] = wc2;
      }
#pragma unroll
      for (int s = 0; s < NB; ++s) {
        double t = 0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) t += wk[c] * gl[s][c];
#pragma unroll
        for (int q = 0; q < NB; ++q) wg[s][q] += t * R.pmass[q][k];
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (fixed && __ldg(fixed + g[q])) continue;
      const int32_t rb = __ldg(m.rpK + g[q]);
#pragma unroll
      for (int s = 0; s < NB; ++s)
        atomicAdd(Np + rb + m.posK[(e * NB + q) * NB + s], D * wg[s][q]);
    }
  }
}

// The same element matrices, a thread per cell over all cells at once,
// added with FP64 atomics: the fastest form (one launch, no colour
// serialisation), but the order in which a value's contributions arrive,
// and so its last bits, changes from run to run.
template <int DIM>
__global__ void __launch_bounds__(128) k_conv_atomic(DMesh m,
                                                       const double* __restrict__ w,
                                                       int64_t ldw, double wc0,
                                                       double wc1, double wc2,
                                                       double* __restrict__ valA) {
  constexpr int NB = DIM + 1, NL = Loc<DIM>::nl;
  const CRef& R = c_ref[DIM - 2];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.ncell;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t g[NL];
    double xv[NB][DIM], gl[NB][DIM];
    load_cell<DIM>(m, e, g, xv);
    double D = bary_grads<DIM>(xv, gl);
    // cw[k][r] = D (w_k . grad lambda_r)
    double cw[NL][NB];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      double wk[DIM];
      if (w) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) wk[c] = __ldg(w + c * ldw + g[k]);
      } else {
        wk[0] = wc0;
        wk[1] = wc1;
        if constexpr (DIM == 3) wk[2] = wc2;
      }
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        double t = 0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) t += wk[c] * gl[r][c];
        cw[k][r] = D * t;
      }
    }
    for (int i = 0; i < NL; ++i) {
      if (__ldg(m.dirichlet + g[i])) continue;
      double acc[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) acc[j] = 0.0;
#pragma unroll
      for (int k = 0; k < NL; ++k)
#pragma unroll
        for (int p = 0; p < Pairs<DIM>::n; ++p)
          acc[Pairs<DIM>::j(p)] += cw[k][Pairs<DIM>::r(p)] * R.conv[i][k][p];
      int32_t rowbase = __ldg(m.rpA + g[i]);
      const uint8_t* pos = m.posA + (e * NL + i) * NL;
#pragma unroll
      for (int j = 0; j < NL; ++j) atomicAdd(valA + rowbase + pos[j], acc[j]);
    }
  }
}


template <typename T>
__global__ void k_bc_rows(DMesh m, T* __restrict__ valA) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m.ndir;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t i = m.dlist[t];
    for (int32_t k = m.rpA[i]; k < m.rpA[i + 1]; ++k) valA[k] = (m.ciA[k] == i) ? T(1) : T(0);
  }
}

// ---------------------------------------------------------------------------
// Manufactured solutions (the problem library): velocity, pressure and the
// load f = u_t - nu Lap u + (w . grad) u + grad p, w = u except for the
// polynomial Oseen problem (w = wconst).
// ---------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

struct Fields {
  double u[3], p, f[3];
};

// g(s) = sin^2(pi s) and derivatives 0..3
__device__ __forceinline__ void g_ders(double s, double (&g)[4]) {
  double sn = sin(kPi * s), s2 = sin(2.0 * kPi * s), c2 = cos(2.0 * kPi * s);
  g[0] = sn * sn;
  g[1] = kPi * s2;
  g[2] = 2.0 * kPi * kPi * c2;
  g[3] = -4.0 * kPi * kPi * kPi * s2;
}

template <int DIM>
__device__ Fields eval_fields(const DPhys& ph, double nu, const double* x, double t,
                              bool want_f) {
  Fields F{};
  double X = x[0], Y = x[1];
  switch (ph.kind) {
    case FS_PROBLEM_UNSTEADY_BENCH: {
      double S = sin(t), C = cos(t);
      double sx = sin(kPi * X), cx = cos(kPi * X), sy = sin(kPi * Y), cy = cos(kPi * Y);
      double u1 = 2 * kPi * S * sx * sx * sy * cy;
      double u2 = -2 * kPi * S * sx * cx * sy * sy;
      F.u[0] = u1;
      F.u[1] = u2;
      F.p = 20 * S * (X * X * Y - 1.0 / 6.0);
      if (want_f) {
        double pi2 = kPi * kPi, pi3 = pi2 * kPi;
        double u1t = 2 * kPi * C * sx * sx * sy * cy, u2t = -2 * kPi * C * sx * cx * sy * sy;
        double u1x = 4 * pi2 * S * sx * cx * sy * cy;
        double u1y = 2 * pi2 * S * sx * sx * (cy * cy - sy * sy);
        double u2x = -2 * pi2 * S * (cx * cx - sx * sx) * sy * sy;
        double u2y = -4 * pi2 * S * sx * cx * sy * cy;
        double lap1 = 4 * pi3 * S * (cx * cx - sx * sx) * sy * cy - 8 * pi3 * S * sx * sx * sy * cy;
        double lap2 = 8 * pi3 * S * sx * cx * sy * sy - 4 * pi3 * S * sx * cx * (cy * cy - sy * sy);
        F.f[0] = u1t - nu * lap1 + u1 * u1x + u2 * u1y + 40 * S * X * Y;
        F.f[1] = u2t - nu * lap2 + u1 * u2x + u2 * u2y + 20 * S * X * X;
      }
      break;
    }
    case FS_PROBLEM_STEADY_POLY: {
      // u = 10 a(x) b(y), v = -10 b(x) a(y), a(s) = s^2 (s-1)^2,
      // b(s) = s (s-1)(2s-1)
      auto a0 = [](double s) { return s * s * (s - 1) * (s - 1); };
      auto a1 = [](double s) { return 4 * s * s * s - 6 * s * s + 2 * s; };
      auto a2 = [](double s) { return 12 * s * s - 12 * s + 2; };
      auto b0 = [](double s) { return s * (s - 1) * (2 * s - 1); };
      auto b1 = [](double s) { return 6 * s * s - 6 * s + 1; };
      auto b2 = [](double s) { return 12 * s - 6; };
      double u1 = 10 * a0(X) * b0(Y), u2 = -10 * b0(X) * a0(Y);
      F.u[0] = u1;
      F.u[1] = u2;
      F.p = 10 * (2 * X - 1) * (2 * Y - 1);
      if (want_f) {
        double u1x = 10 * a1(X) * b0(Y), u1y = 10 * a0(X) * b1(Y);
        double u2x = -10 * b1(X) * a0(Y), u2y = -10 * b0(X) * a1(Y);
        double lap1 = 10 * (a2(X) * b0(Y) + a0(X) * b2(Y));
        double lap2 = -10 * (b2(X) * a0(Y) + b0(X) * a2(Y));
        F.f[0] = -nu * lap1 + u1 * u1x + u2 * u1y + 20 * (2 * Y - 1);
        F.f[1] = -nu * lap2 + u1 * u2x + u2 * u2y + 20 * (2 * X - 1);
      }
      break;
    }
    case FS_PROBLEM_CHANNEL: {
      const double H = 0.41, L = 2.2, U = 1.5;
      F.u[0] = 4 * U * Y * (H - Y) / (H * H);
      F.u[1] = 0;
      F.p = 8 * nu * U * (L - X) / (H * H);
      F.f[0] = F.f[1] = 0;  // Poiseuille solves the steady equations with f = 0
      break;
    }
    case FS_PROBLEM_CUBE: {
      if constexpr (DIM == 3) {
        double S = sin(t), C = cos(t);
        double gx[4], gy[4], gz[4];
        g_ders(X, gx);
        g_ders(Y, gy);
        g_ders(x[2], gz);
        // D(a,b,c) Phi = g^(a)(x) g^(b)(y) g^(c)(z)
        auto Dp = [&](int a, int b, int c) { return gx[a] * gy[b] * gz[c]; };
        // u_i = S (d_{i+1} Phi - d_{i+2} Phi), indices mod 3
        int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        double du[3][3], lap[3], uu[3];
        for (int i = 0; i < 3; ++i) {
          const int* ep = e[(i + 1) % 3];
          const int* em = e[(i + 2) % 3];
          uu[i] = Dp(ep[0], ep[1], ep[2]) - Dp(em[0], em[1], em[2]);
          lap[i] = 0;
          for (int j = 0; j < 3; ++j) {
            int a[3] = {ep[0] + e[j][0], ep[1] + e[j][1], ep[2] + e[j][2]};
            int b[3] = {em[0] + e[j][0], em[1] + e[j][1], em[2] + e[j][2]};
            du[i][j] = S * (Dp(a[0], a[1], a[2]) - Dp(b[0], b[1], b[2]));
            lap[i] += Dp(a[0] + e[j][0], a[1] + e[j][1], a[2] + e[j][2]) -
                      Dp(b[0] + e[j][0], b[1] + e[j][1], b[2] + e[j][2]);
          }
          F.u[i] = S * uu[i];
        }
        double Z = x[2];
        F.p = S * (X * X * Y * Z - 1.0 / 12.0);
        if (want_f) {
          double gp[3] = {2 * X * Y * Z, X * X * Z, X * X * Y};
          for (int i = 0; i < 3; ++i) {
            double conv = F.u[0] * du[i][0] + F.u[1] * du[i][1] + F.u[2] * du[i][2];
            F.f[i] = C * uu[i] - nu * S * lap[i] + conv + S * gp[i];
          }
        }
      }
      break;
    }
    case FS_PROBLEM_POLY_OSEEN:
    case FS_PROBLEM_POLY_OSEEN_T: {
      // spatial fields u0 = (x^2, -2xy[, xy]), p0 = x + y [+ z] - 1 and the
      // steady Oseen load g0 = -nu Lap u0 + (w.grad) u0 + grad p0; the
      // time-affine kind is (1 + t)(u0, p0) with load u0 + (1 + t) g0
      double w1 = ph.wconst[0], w2 = ph.wconst[1];
      double s = ph.kind == FS_PROBLEM_POLY_OSEEN_T ? 1.0 + t : 1.0;
      double ut = ph.kind == FS_PROBLEM_POLY_OSEEN_T ? 1.0 : 0.0;
      F.u[0] = s * (X * X);
      F.u[1] = s * (-2 * X * Y);
      F.p = s * (X + Y - 1);
      F.f[0] = ut * (X * X) + s * (-2 * nu + 2 * X * w1 + 1);
      F.f[1] = ut * (-2 * X * Y) + s * (-2 * Y * w1 - 2 * X * w2 + 1);
      if constexpr (DIM == 3) {
        F.u[2] = s * (X * Y);
        F.p = s * (X + Y + x[2] - 1);
        F.f[2] = ut * (X * Y) + s * (Y * w1 + X * w2 + 1);
      }
      break;
    }
    case FS_PROBLEM_POLY3: {
      // u = (x^3, -3 x^2 y), p = x^2 - y^2; f = -nu Lap u + (w.grad) u + grad p
      const double w1 = ph.wconst[0], w2 = ph.wconst[1];
      F.u[0] = X * X * X;
      F.u[1] = -3 * X * X * Y;
      F.p = X * X - Y * Y;
      F.f[0] = -6 * nu * X + 3 * X * X * w1 + 2 * X;
      F.f[1] = 6 * nu * Y - 6 * X * Y * w1 - 3 * X * X * w2 - 2 * Y;
      break;
    }
    default:
      break;
  }
  return F;
}

template <int DIM>
__global__ void k_eval_load(DMesh m, DPhys ph, double t, double mass_coef,
                            const double* __restrict__ u, double* __restrict__ F) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m.n2;
       j += (int64_t)gridDim.x * blockDim.x) {
    double x[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = m.p2xyz[j * DIM + a];
    const double nu = ph.nu_node ? ph.nu_node[j] : ph.nu;
    Fields f = eval_fields<DIM>(ph, nu, x, t, true);
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      F[c * m.n2 + j] = (u ? mass_coef * u[c * m.n2 + j] : 0.0) + f.f[c];
  }
}

// b_c[i] = sum_k Mv[k] F_c[col k]; L lanes per row.
template <int DIM, int L>
__global__ void k_rhs_vel(DMesh m, DPhys ph, double t, const double* __restrict__ Mv,
                          const double* __restrict__ F, double* __restrict__ b) {
  int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t i = gt / L;
  int lane = (int)(gt % L);
  bool live = i < m.n2;
  double acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = 0;
  bool dir = live && m.dirichlet[i];
  if (live && !dir) {
    for (int32_t k = m.rpA[i] + lane; k < m.rpA[i + 1]; k += L) {
      double a = Mv[k];
      int32_t col = m.ciA[k];
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[c] += a * F[c * m.n2 + col];
    }
  }
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1)
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
  if (live && lane == 0) {
    if (dir) {
      double x[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) x[a] = m.p2xyz[i * DIM + a];
      const double nu = ph.nu_node ? ph.nu_node[i] : ph.nu;
      Fields f = eval_fields<DIM>(ph, nu, x, t, false);
#pragma unroll
      for (int c = 0; c < DIM; ++c) b[c * m.n2 + i] = f.u[c];
    } else {
#pragma unroll
      for (int c = 0; c < DIM; ++c) b[c * m.n2 + i] = acc[c];
    }
  }
}

// b_p = 0, then the pinned rows hold p_exact at their vertex
template <int DIM>
__global__ void k_rhs_p(DMesh m, DPhys ph, double t, const int32_t* __restrict__ pinned,
                        int npinned, double* __restrict__ b) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.nv;
       q += (int64_t)gridDim.x * blockDim.x)
    b[DIM * m.n2 + q] = 0.0;
}
template <int DIM>
__global__ void k_rhs_pin(DMesh m, DPhys ph, double t, const int32_t* __restrict__ pinned,
                          int npinned, double* __restrict__ b) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npinned) return;
  const int64_t q = pinned[k];
  double x[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) x[a] = m.p2xyz[q * DIM + a];
  const double nu = ph.nu_node ? ph.nu_node[q] : ph.nu;
  b[DIM * m.n2 + q] = eval_fields<DIM>(ph, nu, x, t, false).p;
}

template <int DIM>
__global__ void k_exact_state(DMesh m, DPhys ph, double t, int zero_interior,
                              double* __restrict__ x) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m.n2;
       j += (int64_t)gridDim.x * blockDim.x) {
    double xx[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xx[a] = m.p2xyz[j * DIM + a];
    const double nu = ph.nu_node ? ph.nu_node[j] : ph.nu;
    Fields f = eval_fields<DIM>(ph, nu, xx, t, false);
    bool keep = !zero_interior || m.dirichlet[j];
#pragma unroll
    for (int c = 0; c < DIM; ++c) x[c * m.n2 + j] = keep ? f.u[c] : 0.0;
    if (j < m.nv) x[DIM * m.n2 + j] = f.p;
  }
}

// Monolithic values in paper order, one internal row per thread.  The
// paper-order row of internal velocity row (c, q) is c n2 + nat[q]; its
// columns are the row's P2 neighbours in paper order (the rank of nat[j]
// among the row's entries gives the place), then its pressure neighbours
// (vertex ids are the same in both orders).  A pressure row keeps its place
// and holds, per component, its P2 neighbours ranked the same way, then the
// diagonal.
__global__ void k_expand_monolithic(DMesh m, const int32_t* __restrict__ nat,
                                    const double* __restrict__ valA,
                                    const double* __restrict__ B,
                                    const double* __restrict__ BT,
                                    const double* __restrict__ diagp,
                                    const int64_t* __restrict__ mrp,
                                    double* __restrict__ out) {
  const int dim = m.dim;
  const int64_t nrow = dim * m.n2 + m.nv;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrow;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (r < dim * m.n2) {
      const int c = (int)(r / m.n2);
      const int64_t i = r % m.n2;
      int64_t o = mrp[c * m.n2 + nat[i]];
      const int32_t k0 = m.rpA[i], k1 = m.rpA[i + 1];
      for (int32_t k = k0; k < k1; ++k) {
        const int32_t key = nat[m.ciA[k]];
        int rank = 0;
        for (int32_t k2 = k0; k2 < k1; ++k2) rank += nat[m.ciA[k2]] < key;
        out[o + rank] = valA[k];
      }
      o += k1 - k0;
      for (int32_t k = m.rpBT[i]; k < m.rpBT[i + 1]; ++k) out[o++] = -BT[(int64_t)k * dim + c];
    } else {
      const int64_t q = r - dim * m.n2;
      int64_t o = mrp[r];
      const int32_t k0 = m.rpB[q], k1 = m.rpB[q + 1];
      for (int c = 0; c < dim; ++c) {
        for (int32_t k = k0; k < k1; ++k) {
          const int32_t key = nat[m.ciB[k]];
          int rank = 0;
          for (int32_t k2 = k0; k2 < k1; ++k2) rank += nat[m.ciB[k2]] < key;
          out[o + rank] = B[(int64_t)k * dim + c];
        }
        o += k1 - k0;
      }
      out[o] = diagp[q];
    }
  }
}

__global__ void k_dofs_perm(int dim, int64_t n2, int64_t nv, const int32_t* __restrict__ nat,
                            const double* __restrict__ in, double* __restrict__ out,
                            int to_nat) {
  const int64_t n = dim * n2 + nv;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (r < dim * n2) {
      const int64_t c = r / n2, q = r % n2;
      const int64_t rn = c * n2 + nat[q];
      if (to_nat)
        out[rn] = in[r];
      else
        out[r] = in[rn];
    } else {
      out[r] = in[r];
    }
  }
}

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)g;
}

}  // namespace

void launch_assemble_base(const DMesh& m, const std::vector<int64_t>& color_ptr,
                          double mass_coef, double nu, double* base, double* Mv, double* B,
                          double* BT, double* Kp, double* mpl, cudaStream_t s) {
  for (size_t c = 0; c + 1 < color_ptr.size(); ++c) {
    const int64_t c0 = color_ptr[c], c1 = color_ptr[c + 1];
    const unsigned g = grid_for(c1 - c0, 128);
    if (m.dim == 2)
      k_assemble_base<2><<<g, 128, 0, s>>>(m, c0, c1, mass_coef, nu, base, Mv, B, BT, Kp, mpl);
    else
      k_assemble_base<3><<<g, 128, 0, s>>>(m, c0, c1, mass_coef, nu, base, Mv, B, BT, Kp, mpl);
    count_launches(1);
  }
}

void launch_assemble_conv(const DMesh& m, const std::vector<int64_t>& color_ptr,
                          const double* w, int64_t ldw, const double* wc, double* valA,
                          bool deterministic, cudaStream_t s) {
  const double w0 = wc ? wc[0] : 0, w1 = wc ? wc[1] : 0, w2 = wc ? wc[2] : 0;
  if (!deterministic) {
    const unsigned g = grid_for(m.ncell, 128);
    if (m.dim == 2)
      k_conv_atomic<2><<<g, 128, 0, s>>>(m, w, ldw, w0, w1, w2, valA);
    else
      k_conv_atomic<3><<<g, 128, 0, s>>>(m, w, ldw, w0, w1, w2, valA);
    count_launches(1);
    return;
  }
  for (size_t c = 0; c + 1 < color_ptr.size(); ++c) {
    const int64_t c0 = color_ptr[c], c1 = color_ptr[c + 1];
    if (m.dim == 2) {
      constexpr int CPB = ConvCfg<2>::CPB;
      const unsigned g = (unsigned)((c1 - c0 + CPB - 1) / CPB);
      k_conv_elem<2><<<g, 128, 0, s>>>(m, c0, c1, w, ldw, w0, w1, w2, valA);
    } else {
      constexpr int CPB = ConvCfg<3>::CPB;
      const unsigned g = (unsigned)((c1 - c0 + CPB - 1) / CPB);
      k_conv_elem<3><<<g, 128, 0, s>>>(m, c0, c1, w, ldw, w0, w1, w2, valA);
    }
    count_launches(1);
  }
}

void launch_assemble_conv_p1(const DMesh& m, const double* w, int64_t ldw, const double* wc,
                             const uint8_t* fixed, double* Np, cudaStream_t s) {
  const unsigned g = grid_for(m.ncell, 128);
  const double w0 = wc ? wc[0] : 0, w1 = wc ? wc[1] : 0, w2 = wc ? wc[2] : 0;
  if (m.dim == 2)
    k_conv_p1<2><<<g, 128, 0, s>>>(m, w, ldw, w0, w1, w2, fixed, Np);
  else
    k_conv_p1<3><<<g, 128, 0, s>>>(m, w, ldw, w0, w1, w2, fixed, Np);
  count_launches(1);
}

template <typename T>
void launch_bc_rows(const DMesh& m, T* valA, cudaStream_t s) {
  if (m.ndir == 0) return;
  k_bc_rows<T><<<grid_for(m.ndir, 256), 256, 0, s>>>(m, valA);
  count_launches(1);
}
template void launch_bc_rows<double>(const DMesh&, double*, cudaStream_t);
template void launch_bc_rows<float>(const DMesh&, float*, cudaStream_t);

void launch_eval_load(const DMesh& m, const DPhys& ph, double t,
                      double mass_coef, const double* u, double* F,
                      cudaStream_t s) {
  unsigned g = grid_for(m.n2, 256);
  if (m.dim == 2)
    k_eval_load<2><<<g, 256, 0, s>>>(m, ph, t, mass_coef, u, F);
  else
    k_eval_load<3><<<g, 256, 0, s>>>(m, ph, t, mass_coef, u, F);
    count_launches(1);
}

void launch_rhs(const DMesh& m, const DPhys& ph, double t, const double* Mv,
                const double* F, const int32_t* pinned, int npinned, double* b,
                cudaStream_t s) {
  constexpr int L = 4;
  unsigned g = (unsigned)((m.n2 * L + 255) / 256);
  unsigned gp = (unsigned)((npinned + 127) / 128);
  if (m.dim == 2) {
    k_rhs_vel<2, L><<<g, 256, 0, s>>>(m, ph, t, Mv, F, b);
    k_rhs_p<2><<<grid_for(m.nv, 256), 256, 0, s>>>(m, ph, t, pinned, npinned, b);
    if (npinned > 0) k_rhs_pin<2><<<gp, 128, 0, s>>>(m, ph, t, pinned, npinned, b);
  } else {
    k_rhs_vel<3, L><<<g, 256, 0, s>>>(m, ph, t, Mv, F, b);
    k_rhs_p<3><<<grid_for(m.nv, 256), 256, 0, s>>>(m, ph, t, pinned, npinned, b);
    if (npinned > 0) k_rhs_pin<3><<<gp, 128, 0, s>>>(m, ph, t, pinned, npinned, b);
  }
  count_launches(npinned > 0 ? 3 : 2);
}

void launch_exact_state(const DMesh& m, const DPhys& ph, double t,
                        int zero_interior, double* x, cudaStream_t s) {
  unsigned g = grid_for(m.n2, 256);
  if (m.dim == 2)
    k_exact_state<2><<<g, 256, 0, s>>>(m, ph, t, zero_interior, x);
  else
    k_exact_state<3><<<g, 256, 0, s>>>(m, ph, t, zero_interior, x);
    count_launches(1);
}

void launch_expand_monolithic(const DMesh& m, const int32_t* nat, const double* valA,
                              const double* B, const double* BT, const double* diagp,
                              const int64_t* mrp, double* out, cudaStream_t s) {
  int64_t nrow = m.dim * m.n2 + m.nv;
  k_expand_monolithic<<<grid_for(nrow, 256), 256, 0, s>>>(m, nat, valA, B, BT, diagp, mrp, out);
  count_launches(1);
}

void launch_dofs_perm(const DMesh& m, const int32_t* nat, const double* in, double* out,
                      int to_nat, cudaStream_t s) {
  int64_t n = m.dim * m.n2 + m.nv;
  k_dofs_perm<<<grid_for(n, 256), 256, 0, s>>>(m.dim, m.n2, m.nv, nat, in, out, to_nat);
  count_launches(1);
}

// ---------------------------------------------------------------------------
// Taylor-Hood P3/P2 on triangles (paper Sec. 4.1, the P3-P2 experiment):
// the same blocks with the P3 velocity map c2u (m.c2d, 10 nodes per cell)
// and the P2 pressure map c2p (6 per cell); reference integrals R (a RefP3
// in device memory; see fs_internal.h) times |det J|.  A thread per cell,
// FP64 atomics into the slot-indexed values.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ double p3_grads(const DMesh& m, int64_t e, int32_t (&g)[10],
                                           double (&gl)[3][2]) {
#pragma unroll
  for (int a = 0; a < 10; ++a) g[a] = __ldg(m.c2d + e * 10 + a);
  double xv[3][2];
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int a = 0; a < 2; ++a) xv[v][a] = __ldg(m.p2xyz + (int64_t)g[v] * 2 + a);
  return bary_grads<2>(xv, gl);
}

__global__ void __launch_bounds__(128) k_p3_base(DMesh m, const int32_t* __restrict__ c2p,
                                                 const RefP3* __restrict__ R, double mass_coef,
                                                 double nu, double* __restrict__ base,
                                                 double* __restrict__ Mv,
                                                 double* __restrict__ B,
                                                 double* __restrict__ BT,
                                                 double* __restrict__ Kp) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.ncell;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t g[10], gp[6];
    double gl[3][2];
    const double D = p3_grads(m, e, g, gl);
#pragma unroll
    for (int q = 0; q < 6; ++q) gp[q] = __ldg(c2p + e * 6 + q);
    double G[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int t = 0; t < 3; ++t) G[r][t] = gl[r][0] * gl[t][0] + gl[r][1] * gl[t][1];
    for (int i = 0; i < 10; ++i) {
      const int32_t rb = __ldg(m.rpA + g[i]);
      const uint8_t* pos = m.posA + (e * 10 + i) * 10;
      for (int j = 0; j < 10; ++j) {
        double kk = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int t = 0; t < 3; ++t) kk += G[r][t] * R->stiff[i][j][r][t];
        const double mm = D * R->mass[i][j];
        atomicAdd(base + rb + pos[j], mass_coef * mm + nu * D * kk);
        atomicAdd(Mv + rb + pos[j], mm);
      }
    }
    for (int q = 0; q < 6; ++q)
      for (int j = 0; j < 10; ++j) {
        double bv[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          double s = 0;
#pragma unroll
          for (int r = 0; r < 3; ++r) s += gl[r][c] * R->div[q][j][r];
          bv[c] = D * s;
        }
        const int64_t sB = __ldg(m.rpB + gp[q]) + m.posB[(e * 6 + q) * 10 + j];
        const int64_t sBT = __ldg(m.rpBT + g[j]) + m.posBT[(e * 10 + j) * 6 + q];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          atomicAdd(B + sB * 2 + c, bv[c]);
          atomicAdd(BT + sBT * 2 + c, bv[c]);
        }
      }
    for (int q = 0; q < 6; ++q) {
      const int32_t rb = __ldg(m.rpK + gp[q]);
      for (int s2 = 0; s2 < 6; ++s2) {
        double kk = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int t = 0; t < 3; ++t) kk += G[r][t] * R->pstiff[q][s2][r][t];
        atomicAdd(Kp + rb + m.posK[(e * 6 + q) * 6 + s2], D * kk);
      }
    }
  }
}

// valA += N(w) of every cell (rows of Dirichlet nodes skipped):
//   N_ij = D sum_k sum_r (w_k . grad lambda_r) conv[i][k][j][r]
__global__ void __launch_bounds__(128) k_p3_conv(DMesh m, const RefP3* __restrict__ R,
                                                 const double* __restrict__ w, int64_t ldw,
                                                 double wc0, double wc1,
                                                 double* __restrict__ valA) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.ncell;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t g[10];
    double gl[3][2];
    const double D = p3_grads(m, e, g, gl);
    double cw[10][3];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const double w0 = w ? __ldg(w + g[k]) : wc0, w1 = w ? __ldg(w + ldw + g[k]) : wc1;
#pragma unroll
      for (int r = 0; r < 3; ++r) cw[k][r] = D * (w0 * gl[r][0] + w1 * gl[r][1]);
    }
    for (int i = 0; i < 10; ++i) {
      if (__ldg(m.dirichlet + g[i])) continue;
      double acc[10];
#pragma unroll
      for (int j = 0; j < 10; ++j) acc[j] = 0;
      for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int j = 0; j < 10; ++j)
#pragma unroll
          for (int r = 0; r < 3; ++r) acc[j] += cw[k][r] * R->conv[i][k][j][r];
      const int32_t rb = __ldg(m.rpA + g[i]);
      const uint8_t* pos = m.posA + (e * 10 + i) * 10;
#pragma unroll
      for (int j = 0; j < 10; ++j) atomicAdd(valA + rb + pos[j], acc[j]);
    }
  }
}

// Interpolant of the exact state at t: u at the P3 nodes, p at the P2
// nodes (coordinates pxyz); zero_interior: u = 0 off the Dirichlet nodes.
__global__ void k_p3_exact_state(DMesh m, DPhys ph, double t, int zero_interior,
                                 const double* __restrict__ pxyz, double* __restrict__ x) {
  const int64_t n = m.n2 + m.nv;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < m.n2) {
      const double xy[2] = {m.p2xyz[k * 2], m.p2xyz[k * 2 + 1]};
      Fields f = eval_fields<2>(ph, ph.nu, xy, t, false);
      const bool keep = !zero_interior || m.dirichlet[k];
      x[k] = keep ? f.u[0] : 0.0;
      x[m.n2 + k] = keep ? f.u[1] : 0.0;
    } else {
      const int64_t q = k - m.n2;
      const double xy[2] = {pxyz[q * 2], pxyz[q * 2 + 1]};
      x[2 * m.n2 + q] = eval_fields<2>(ph, ph.nu, xy, t, false).p;
    }
  }
}

}  // namespace

void launch_p3_base(const DMesh& m, const int32_t* c2p, const RefP3* R, double mass_coef,
                    double nu, double* base, double* Mv, double* B, double* BT, double* Kp,
                    cudaStream_t s) {
  k_p3_base<<<grid_for(m.ncell, 128), 128, 0, s>>>(m, c2p, R, mass_coef, nu, base, Mv, B, BT,
                                                   Kp);
  count_launches(1);
}

void launch_p3_conv(const DMesh& m, const RefP3* R, const double* w, int64_t ldw,
                    const double* wc, double* valA, cudaStream_t s) {
  k_p3_conv<<<grid_for(m.ncell, 128), 128, 0, s>>>(m, R, w, ldw, wc ? wc[0] : 0.0,
                                                   wc ? wc[1] : 0.0, valA);
  count_launches(1);
}

void launch_p3_exact_state(const DMesh& m, const DPhys& ph, double t, int zero_interior,
                           const double* pxyz, double* x, cudaStream_t s) {
  k_p3_exact_state<<<grid_for(m.n2 + m.nv, 256), 256, 0, s>>>(m, ph, t, zero_interior, pxyz,
                                                              x);
  count_launches(1);
}

}  // namespace fs
