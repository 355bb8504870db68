// Sparse linear algebra of the Krylov solve on sm_103a: the saddle-point
// SpMV in block form, the multigrid V-cycle and block preconditioner, and the
// reductions of flexible GMRES(m) (paper Sec. 3.2: GMRES).
//
// Row kernels use "L lanes per row": a group of L consecutive lanes walks one
// CSR row with stride L (coalesced within the group) and reduces with
// xor-shuffles inside the group.  The scalar P2 block A is stored once and
// applied to all velocity components in the same pass (one read of the
// matrix for d right-hand sides).  Reductions are two-level: per-block
// partials, then the last block to finish (atomic ticket, no waiting) sums
// them in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fs_device.h"

namespace fs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

inline unsigned blocks_for(int64_t threads, int block = 256) {
  int64_t g = (threads + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int L, typename V>
__device__ __forceinline__ V group_sum(V v) {
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// ---------------------------------------------------------------------------
// y = K x  or  y = b - K x with K = [A (per component), -BT; B, diag(D)]
// ---------------------------------------------------------------------------
template <typename T, typename V, int DIM, int L>
__global__ void __launch_bounds__(256) k_spmv_full(DOp<T> op, const V* __restrict__ x,
                                                   const V* __restrict__ b,
                                                   V* __restrict__ y, int resid,
                                                   const int* skip) {
  if (skip && *skip) return;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt / L;
  const int lane = (int)(gt % L);
  const int64_t n2 = op.n2, ntot = op.n2 + op.nv;
  const V* __restrict__ xp = x + DIM * n2;
  V acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = V(0);
  if (row < n2) {
    const int32_t b0 = op.A.rp[row], b1 = op.A.rp[row + 1];
    for (int32_t k = b0 + lane; k < b1; k += L) {
      const V a = (V)op.A.v[k];
      const int32_t c0 = op.A.ci[k];
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[c] += a * x[c * n2 + c0];
    }
    const int32_t t0 = op.BT.rp[row], t1 = op.BT.rp[row + 1];
    for (int32_t k = t0 + lane; k < t1; k += L) {
      const V p = xp[op.BT.ci[k]];
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[c] -= (V)op.BT.v[(int64_t)k * DIM + c] * p;
    }
  } else if (row < ntot) {
    const int64_t q = row - n2;
    const int32_t b0 = op.B.rp[q], b1 = op.B.rp[q + 1];
    for (int32_t k = b0 + lane; k < b1; k += L) {
      const int32_t c0 = op.B.ci[k];
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[0] += (V)op.B.v[(int64_t)k * DIM + c] * x[c * n2 + c0];
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = group_sum<L>(acc[c]);
  if (lane != 0 || row >= ntot) return;
  if (row < n2) {
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t r = c * n2 + row;
      y[r] = resid ? b[r] - acc[c] : acc[c];
    }
  } else {
    const int64_t q = row - n2;
    const V v = acc[0] + (V)op.diagp[q] * xp[q];
    const int64_t r = DIM * n2 + q;
    y[r] = resid ? b[r] - v : v;
  }
}

// ---------------------------------------------------------------------------
// Multigrid kernels (NC right-hand sides, component stride = level rows)
// Chebyshev smoothing (Saad, Iterative Methods, Alg. 12.1) with Jacobi
// scaling, one fused SpMV kernel per step:
//   mode 0 FIRST: x_in = 0, d_in = D^-1 b / theta (implicit)
//   mode 1 STEP : y = x_in + d_in; r = b - A y; x_out = y;
//                 d_out = alpha d_in + beta D^-1 r
//   mode 2 RESID: y = x_in + d_in; x_out = y; d_out = r = b - A y
//   mode 3 START: y = x_in; d_out = D^-1 (b - A y) / theta
//   mode 4 LAST : y = x_in + d_in; d = alpha d_in + beta D^-1 r;
//                 x_out = y + d
// ---------------------------------------------------------------------------
template <typename T, int NC, int L, int MODE>
__global__ void __launch_bounds__(256) k_cheb(DCsr<T> A, const T* __restrict__ dinv,
                                              const T* __restrict__ b,
                                              const T* __restrict__ x_in,
                                              const T* __restrict__ d_in, T inv_theta,
                                              T alpha, T beta, T* __restrict__ x_out,
                                              T* __restrict__ d_out, const int* skip) {
  if (skip && *skip) return;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt / L;
  const int lane = (int)(gt % L);
  const int64_t n = A.nrow;
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  if (row < n) {
    const int32_t b0 = A.rp[row], b1 = A.rp[row + 1];
    for (int32_t k = b0 + lane; k < b1; k += L) {
      const T a = A.v[k];
      const int32_t j = A.ci[k];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int64_t o = c * n + j;
        T yj;
        if (MODE == 0) yj = dinv[j] * b[o] * inv_theta;
        else if (MODE == 3) yj = x_in[o];
        else yj = x_in[o] + d_in[o];
        acc[c] += a * yj;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = group_sum<L>(acc[c]);
  if (lane != 0 || row >= n) return;
  const T di = dinv[row];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int64_t o = c * n + row;
    const T r = b[o] - acc[c];
    if (MODE == 0) {
      const T d0 = di * b[o] * inv_theta;
      x_out[o] = d0;
      d_out[o] = alpha * d0 + beta * di * r;
    } else if (MODE == 1) {
      const T dd = d_in[o];
      x_out[o] = x_in[o] + dd;
      d_out[o] = alpha * dd + beta * di * r;
    } else if (MODE == 2) {
      x_out[o] = x_in[o] + d_in[o];
      d_out[o] = r;
    } else if (MODE == 3) {
      d_out[o] = di * r * inv_theta;
    } else {
      const T dd = d_in[o];
      const T dn = alpha * dd + beta * di * r;
      x_out[o] = x_in[o] + dd + dn;
    }
  }
}

// y (+)= M x for NC components: add == 0 stores, add == 1 accumulates.
template <typename T, int NC, int L>
__global__ void __launch_bounds__(256) k_csr_nc(DCsr<T> M, int64_t ldx, const T* __restrict__ x,
                                                int64_t ldy, T* __restrict__ y, int add,
                                                const int* skip) {
  if (skip && *skip) return;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt / L;
  const int lane = (int)(gt % L);
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  if (row < M.nrow) {
    for (int32_t k = M.rp[row] + lane; k < M.rp[row + 1]; k += L) {
      const T a = M.v[k];
      const int32_t j = M.ci[k];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += a * x[c * ldx + j];
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = group_sum<L>(acc[c]);
  if (lane != 0 || row >= M.nrow) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int64_t o = c * ldy + row;
    y[o] = add ? y[o] + acc[c] : acc[c];
  }
}

// Coarsest solve x = blockdiag(Cinv) b; one warp per row, the row's block
// found through row_blk.
template <typename T, int NC>
__global__ void k_dense(const T* __restrict__ C, const int32_t* __restrict__ row_blk,
                        const int64_t* __restrict__ blk_row, const int64_t* __restrict__ blk_n,
                        const int64_t* __restrict__ blk_dense, int64_t n,
                        const T* __restrict__ b, T* __restrict__ x, const int* skip) {
  if (skip && *skip) return;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  if (row < n) {
    const int blk = row_blk[row];
    const int64_t r0 = blk_row[blk], nb = blk_n[blk];
    const T* Cr = C + blk_dense[blk] + (row - r0) * nb;
    for (int64_t j = lane; j < nb; j += 32) {
      const T a = Cr[j];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += a * b[c * n + r0 + j];
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = group_sum<32>(acc[c]);
  if (lane == 0 && row < n)
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c * n + row] = acc[c];
}

template <typename T, int NC>
void vcycle_level(const DHier<T>& H, int l, const T* b, T* out, const int* skip,
                  cudaStream_t s) {
  if (l == H.nlev - 1) {
    const int64_t n = H.ncoarse;
    k_dense<T, NC><<<blocks_for(n * 32), 256, 0, s>>>(H.cinv, H.row_blk, H.blk_row, H.blk_n,
                                                      H.blk_dense, n, b, out, skip);
    count_launches(1);
    return;
  }
  const DLevel<T>& L = H.lev[l];
  const int64_t n = L.A.nrow;
  const unsigned g4 = blocks_for(n * 4), g8 = blocks_for(n * 8);
  T *X0 = H.xw[l], *X1 = H.xw2[l], *D0 = H.dw[l], *D1 = H.dw2[l];
  // the coarse right-hand side lives in bw[l+1] and its solution in xw[l+1]
  const T it = (T)L.inv_theta, a1 = (T)L.a1, b1 = (T)L.b1, a2 = (T)L.a2, b2 = (T)L.b2;
#define FS_CHEB(MODE, XI, DI, AL, BE, XO, DO)                                          \
  do {                                                                                \
    if (L.lanes == 8)                                                                 \
      k_cheb<T, NC, 8, MODE><<<g8, 256, 0, s>>>(L.A, L.dinv, b, XI, DI, it, AL, BE, XO, \
                                                DO, skip);                            \
    else                                                                              \
      k_cheb<T, NC, 4, MODE><<<g4, 256, 0, s>>>(L.A, L.dinv, b, XI, DI, it, AL, BE, XO, \
                                                DO, skip);                            \
    count_launches(1);                                                                \
  } while (0)
  // pre-smoothing: x1 = d0, d1; x2, d2; x3 = x2 + d2, r3
  FS_CHEB(0, nullptr, nullptr, a1, b1, X0, D0);
  FS_CHEB(1, X0, D0, a2, b2, X1, D1);
  FS_CHEB(2, X1, D1, T(0), T(0), X0, D0);
  // restrict r3 to the coarse right-hand side
  const DLevel<T>& C = H.lev[l + 1];
  const int64_t nc_rows = C.A.nrow;
  {
    DCsr<T> R = L.R;
    k_csr_nc<T, NC, 4><<<blocks_for(R.nrow * 4), 256, 0, s>>>(R, n, D0, nc_rows, H.bw[l + 1], 0,
                                                               skip);
    count_launches(1);
  }
  vcycle_level<T, NC>(H, l + 1, H.bw[l + 1], H.xw[l + 1], skip, s);
  // prolongate and correct
  {
    DCsr<T> P = L.P;
    k_csr_nc<T, NC, 4><<<blocks_for(P.nrow * 4), 256, 0, s>>>(P, nc_rows, H.xw[l + 1], n, X0, 1,
                                                               skip);
    count_launches(1);
  }
  // post-smoothing from x0 = X0
  FS_CHEB(3, X0, nullptr, T(0), T(0), nullptr, D0);
  FS_CHEB(1, X0, D0, a1, b1, X1, D1);
  FS_CHEB(4, X1, D1, a2, b2, out, nullptr);
#undef FS_CHEB
}

// out[c][r] = in[c][perm[r]] (gather) or out[c][perm[r]] = in[c][r] (scatter)
template <typename T>
__global__ void k_permute(const int32_t* __restrict__ perm, int64_t n, int nc,
                          const T* __restrict__ in, T* __restrict__ out, int scatter,
                          const int* skip) {
  if (skip && *skip) return;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[r];
    for (int c = 0; c < nc; ++c) {
      if (scatter) out[c * n + p] = in[c * n + r];
      else out[c * n + r] = in[c * n + p];
    }
  }
}

// ---------------------------------------------------------------------------
// Block preconditioner pieces
// ---------------------------------------------------------------------------
// z_p = nu Mp^-1 r_p + dt^-1 y_K ; pinned rows: z_p = r_p
template <typename T>
__global__ void k_prec_p(int64_t nv, const T* __restrict__ rp, const T* __restrict__ yk,
                         const T* __restrict__ mpl_inv_nu, T inv_dt,
                         const int32_t* __restrict__ pinned, int npinned,
                         T* __restrict__ zp, const int* skip) {
  if (skip && *skip) return;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x)
    zp[q] = mpl_inv_nu[q] * rp[q] + inv_dt * yk[q];
}
template <typename T>
__global__ void k_pin_rows(const int32_t* __restrict__ pinned, int npinned,
                           const T* __restrict__ rp, T* __restrict__ zp, const int* skip) {
  if (skip && *skip) return;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < npinned) zp[pinned[t]] = rp[pinned[t]];
}

// t_c = r_c + BT_c z_p over the velocity rows
template <typename T, int DIM, int L>
__global__ void __launch_bounds__(256) k_bt_add(DCsr<T> BT, int64_t n2, const T* __restrict__ r,
                                                const T* __restrict__ zp, T* __restrict__ t,
                                                const int* skip) {
  if (skip && *skip) return;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt / L;
  const int lane = (int)(gt % L);
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
  if (row < n2) {
    for (int32_t k = BT.rp[row] + lane; k < BT.rp[row + 1]; k += L) {
      const T p = zp[BT.ci[k]];
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[c] += BT.v[(int64_t)k * DIM + c] * p;
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = group_sum<L>(acc[c]);
  if (lane == 0 && row < n2)
#pragma unroll
    for (int c = 0; c < DIM; ++c) t[c * n2 + row] = r[c * n2 + row] + acc[c];
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, int64_t n,
                          const double* scale, int inv) {
  double s = scale ? *scale : 1.0;
  if (scale && inv) s = 1.0 / s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (B)((double)in[i] * s);
}

inline unsigned grid_stride_blocks(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T, typename V>
void launch_spmv_full(const DOp<T>& op, const V* x, const V* b, V* y, int resid,
                      const int* skip, int lanes, cudaStream_t s) {
  const int64_t rows = op.n2 + op.nv;
  if (op.dim == 2) {
    if (lanes == 8)
      k_spmv_full<T, V, 2, 8><<<blocks_for(rows * 8), 256, 0, s>>>(op, x, b, y, resid, skip);
    else
      k_spmv_full<T, V, 2, 4><<<blocks_for(rows * 4), 256, 0, s>>>(op, x, b, y, resid, skip);
      count_launches(1);
  } else {
    if (lanes == 4)
      k_spmv_full<T, V, 3, 4><<<blocks_for(rows * 4), 256, 0, s>>>(op, x, b, y, resid, skip);
    else
      k_spmv_full<T, V, 3, 8><<<blocks_for(rows * 8), 256, 0, s>>>(op, x, b, y, resid, skip);
      count_launches(1);
  }
}
template void launch_spmv_full<double, double>(const DOp<double>&, const double*, const double*,
                                               double*, int, const int*, int, cudaStream_t);
template void launch_spmv_full<float, float>(const DOp<float>&, const float*, const float*,
                                             float*, int, const int*, int, cudaStream_t);

template <typename T>
void launch_cheb_step(const DHier<T>& H, int nc, cudaStream_t s) {
  const DLevel<T>& L = H.lev[0];
  const int64_t n = L.A.nrow;
  const T it = (T)L.inv_theta, a1 = (T)L.a1, b1 = (T)L.b1;
#define FS_STEP(NCV)                                                                   \
  if (L.lanes == 8)                                                                    \
    k_cheb<T, NCV, 8, 1><<<blocks_for(n * 8), 256, 0, s>>>(L.A, L.dinv, H.bw[0], H.xw[0], \
                                                           H.dw[0], it, a1, b1, H.xw2[0],  \
                                                           H.dw2[0], nullptr);          \
  else                                                                                 \
    k_cheb<T, NCV, 4, 1><<<blocks_for(n * 4), 256, 0, s>>>(L.A, L.dinv, H.bw[0], H.xw[0], \
                                                           H.dw[0], it, a1, b1, H.xw2[0],  \
                                                           H.dw2[0], nullptr);
  if (nc == 2) {
    FS_STEP(2)
  } else if (nc == 3) {
    FS_STEP(3)
  } else {
    FS_STEP(1)
  }
#undef FS_STEP
  count_launches(1);
}
template void launch_cheb_step<double>(const DHier<double>&, int, cudaStream_t);
template void launch_cheb_step<float>(const DHier<float>&, int, cudaStream_t);

template <typename T>
void mg_vcycle(const DHier<T>& H, int nc, const T* b, int64_t ld, T* x, const int* skip,
               cudaStream_t s) {
  (void)ld;  // level-0 vectors are stored with stride = level rows
  const T* bb = b;
  T* xx = x;
  const int64_t n0 = H.lev[0].A.nrow;
  const unsigned gp = (unsigned)std::min<int64_t>((n0 + 255) / 256, 152 * 16);
  if (H.perm) {  // into block order
    k_permute<T><<<gp, 256, 0, s>>>(H.perm, n0, nc, b, H.pin, 0, skip);
    count_launches(1);
    bb = H.pin;
    xx = H.pout;
  }
  if (nc == 1) vcycle_level<T, 1>(H, 0, bb, xx, skip, s);
  else if (nc == 2) vcycle_level<T, 2>(H, 0, bb, xx, skip, s);
  else vcycle_level<T, 3>(H, 0, bb, xx, skip, s);
  if (H.perm) {  // back to the caller's order
    k_permute<T><<<gp, 256, 0, s>>>(H.perm, n0, nc, H.pout, x, 1, skip);
    count_launches(1);
  }
}
template void mg_vcycle<double>(const DHier<double>&, int, const double*, int64_t, double*,
                                const int*, cudaStream_t);
template void mg_vcycle<float>(const DHier<float>&, int, const float*, int64_t, float*,
                               const int*, cudaStream_t);

template <typename T>
void launch_precond(const DOp<T>& op, const DHier<T>& HA, const DHier<T>& HK,
                    const T* mpl_inv_nu, double inv_dt, const int32_t* pinned,
                    int npinned, const T* r, T* z, T* work_p, T* work_u,
                    const int* skip, cudaStream_t s) {
  const int64_t n2 = op.n2, nv = op.nv;
  const int dim = op.dim;
  const T* rp = r + dim * n2;
  T* zp = z + dim * n2;
  // pressure: Cahouet-Chabard  z_p = nu Mp^-1 r_p + dt^-1 Kp^-1 r_p
  mg_vcycle<T>(HK, 1, rp, nv, work_p, skip, s);
  k_prec_p<T><<<grid_stride_blocks(nv), 256, 0, s>>>(nv, rp, work_p, mpl_inv_nu, (T)inv_dt,
                                                     pinned, npinned, zp, skip);
  count_launches(1);
  if (npinned > 0)
    k_pin_rows<T><<<blocks_for(npinned), 256, 0, s>>>(pinned, npinned, rp, zp, skip);
    count_launches(1);
  // velocity: z_u = A^-1 (r_u + BT z_p) by one V-cycle on all components
  if (dim == 2)
    k_bt_add<T, 2, 4><<<blocks_for(n2 * 4), 256, 0, s>>>(op.BT, n2, r, zp, work_u, skip);
  else
    k_bt_add<T, 3, 4><<<blocks_for(n2 * 4), 256, 0, s>>>(op.BT, n2, r, zp, work_u, skip);
    count_launches(1);
  mg_vcycle<T>(HA, dim, work_u, n2, z, skip, s);
}
template void launch_precond<double>(const DOp<double>&, const DHier<double>&,
                                     const DHier<double>&, const double*, double,
                                     const int32_t*, int, const double*, double*, double*,
                                     double*, const int*, cudaStream_t);
template void launch_precond<float>(const DOp<float>&, const DHier<float>&,
                                    const DHier<float>&, const float*, double,
                                    const int32_t*, int, const float*, float*, float*,
                                    float*, const int*, cudaStream_t);

template <typename A, typename B>
void launch_convert(const A* in, B* out, int64_t n, const double* scale, int inv,
                    cudaStream_t s) {
  k_convert<A, B><<<grid_stride_blocks(n), 256, 0, s>>>(in, out, n, scale, inv);
  count_launches(1);
}
template void launch_convert<double, float>(const double*, float*, int64_t, const double*, int,
                                            cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, const double*, int,
                                            cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, const double*,
                                             int, cudaStream_t);

}  // namespace fs
