// Sparse linear algebra of the Krylov solve on sm_103a: the saddle-point
// SpMV in block form, the multigrid V-cycle and block preconditioner, and the
// reductions of flexible GMRES(m) (paper Sec. 3.2: GMRES).
//
// Matrices on the iteration path are sliced ELLPACK with 32-row slices, one
// thread per row: a warp reads one slot of 32 consecutive rows at a time, so
// matrix loads are contiguous, and with the P2 nodes numbered by parity
// class (see the mesh builder) the x entries the warp gathers at a slot are
// contiguous too.  The scalar P2 block A is stored once and applied to all
// velocity components in the same pass (one read of the matrix for d
// right-hand sides).  Transfer operators of the multigrid stay CSR with a
// few lanes per row reducing by xor-shuffles.  Reductions are two-level:
// per-block partials, then the last block to finish (atomic ticket, no
// waiting) sums them in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include <cooperative_groups.h>

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

// Row loops take kU slots at a time (loads issued before the FMAs); padding
// slots have coefficient 0 and a valid column.  The FP32 saddle-point SpMV
// takes kUSpmv: its rows read more per slot (d gathers, or d values), and
// deeper groups measured faster there (cube 48^3: 0.115 -> 0.090 ms), while
// the smoothing pass and the FP64 SpMV are fastest at 4.
constexpr int kU = 4;
constexpr int kUSpmv = 6;

// ---------------------------------------------------------------------------
// y = K x  or  y = b - K x with K = [A (per component), -BT; B, diag(D)]
// Threads [0, wp) take the pressure rows (wp = nv rounded up to a warp), the
// following ones the velocity rows, so no warp mixes the two.  The pressure
// rows come first: each holds d components of every P2 neighbour (62 slots
// x 3 values in 3D), the longest work per thread, and the blocks scheduled
// first start first instead of forming a tail.
// ---------------------------------------------------------------------------
template <typename T, typename V, int DIM, int kUS>
__global__ void __launch_bounds__(256) k_spmv_full(DOp<T> op, JVec<const V> xv,
                                                   const V* __restrict__ b, JVec<V> yv,
                                                   int resid, SegSkip sku, SegSkip skp,
                                                   const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const V* __restrict__ x = xv.get();
  V* __restrict__ y = yv.get();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n2 = op.n2, nv = op.nv, wp = (nv + 31) & ~(int64_t)31;
  const V* __restrict__ xp = x + DIM * n2;
  if (t >= wp) {
    const int64_t row = t - wp;
    if (row >= n2 || seg_skipped(sku, row)) return;
    V acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = V(0);
    {
      const int64_t o1 = op.A.off[(row >> 5) + 1];
      for (int64_t o = op.A.off[row >> 5] + (row & 31); o < o1; o += kUS * 32) {
        V a[kUS];
        int32_t j[kUS];
#pragma unroll
        for (int u = 0; u < kUS; ++u) {
          const int64_t oo = o + u * 32;
          const bool ok = oo < o1;
          a[u] = ok ? (V)op.A.v[oo] : V(0);
          j[u] = ok ? op.A.ci[oo] : (int32_t)row;
        }
        V xv[kUS][DIM];
#pragma unroll
        for (int u = 0; u < kUS; ++u)
#pragma unroll
          for (int c = 0; c < DIM; ++c) xv[u][c] = x[c * n2 + j[u]];
#pragma unroll
        for (int u = 0; u < kUS; ++u)
#pragma unroll
          for (int c = 0; c < DIM; ++c) acc[c] += a[u] * xv[u][c];
      }
    }
    {
      // d values per slot, component-major: component c of slot u at
      // (slice offset + 32 u) d + 32 c + t
      const int64_t t32 = row & 31, o1 = op.BT.off[(row >> 5) + 1];
      for (int64_t o = op.BT.off[row >> 5] + t32; o < o1; o += kU * 32) {
        V p[kU], bv[kU][DIM];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int64_t oo = o + u * 32;
          const bool ok = oo < o1;
          const int64_t base = (oo - t32) * DIM + t32;
          p[u] = ok ? xp[op.BT.ci[oo]] : V(0);
#pragma unroll
          for (int c = 0; c < DIM; ++c) bv[u][c] = ok ? (V)op.BT.v[base + 32 * c] : V(0);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
#pragma unroll
          for (int c = 0; c < DIM; ++c) acc[c] -= bv[u][c] * p[u];
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t r = c * n2 + row;
      y[r] = resid ? b[r] - acc[c] : acc[c];
    }
  } else {
    const int64_t q = t;
    if (q >= nv || seg_skipped(skp, q)) return;
    V acc = V(0);
    const int64_t t32 = q & 31, o1 = op.B.off[(q >> 5) + 1];
    for (int64_t o = op.B.off[q >> 5] + t32; o < o1; o += kUS * 32) {
      V bv[kUS][DIM], xv[kUS][DIM];
#pragma unroll
      for (int u = 0; u < kUS; ++u) {
        const int64_t oo = o + u * 32;
        const bool ok = oo < o1;
        const int64_t base = (oo - t32) * DIM + t32;
        const int32_t j = ok ? op.B.ci[oo] : 0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          bv[u][c] = ok ? (V)op.B.v[base + 32 * c] : V(0);
          xv[u][c] = x[c * n2 + j];
        }
      }
#pragma unroll
      for (int u = 0; u < kUS; ++u)
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc += bv[u][c] * xv[u][c];
    }
    const V v = acc + (V)op.diagp[q] * xp[q];
    const int64_t r = DIM * n2 + q;
    y[r] = resid ? b[r] - v : v;
  }
}

// CSR -> SELL-32 value scatter, one thread per row.
__global__ void k_csr_to_sell(int64_t n, const int32_t* __restrict__ rp,
                              const double* __restrict__ in, const int64_t* __restrict__ off,
                              double* __restrict__ out64, float* __restrict__ out32) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t base = off[r >> 5] + (r & 31);
  const int32_t k0 = rp[r], len = rp[r + 1] - k0;
  for (int32_t u = 0; u < len; ++u) {
    const double v = in[k0 + u];
    out64[base + 32 * u] = v;
    if (out32) out32[base + 32 * u] = (float)v;
  }
}

// ---------------------------------------------------------------------------
// Multigrid V-cycle.  Level vectors are row-major with the components of a
// row contiguous (nc padded to NCP in {1, 2, 4}), so a neighbour is one
// NCP-wide load.  A level's Chebyshev state is kept as the gather vector G
// (the point the next residual is taken at, x + d, read at every neighbour)
// and the direction D (read at the own row only).
//
// Chebyshev smoothing (Saad, Iterative Methods, Alg. 12.1) with Jacobi
// scaling, one fused SpMV pass per step; the first step's direction
// d0 = D^-1 b / theta is written by whichever pass produces the level's
// right-hand side (restriction, or the preconditioner's load kernels).
// Modes, with r = b - A Gin:
//   STEP : dn = alpha D + beta Dinv r;  Gout = Gin + dn, Dout = dn
//   RESID: Gout = r                      (Gin = x3 stays for the correction)
//   START: d0 = Dinv r / theta;         Gout = Gin + d0, Dout = d0  (Gin = x0)
//   LAST : Gin + alpha D + beta Dinv r, the level's result, to Gout, or on
//          level 0 (out != null) its first nc components to the caller's
//          blocked vector at row perm[r].
//
// The levels below a per-problem row threshold (the schedule; see
// fs_autotune) can run as one kernel on one thread-block cluster
// (k_mg_tail): the passes that are separate kernels on the large levels
// become phases separated by cluster barriers, which removes a kernel launch
// per pass where the levels are too small to fill the GPU.  Both forms share
// the per-row code below, so they compute the same values.
// ---------------------------------------------------------------------------
enum { MG_STEP = 0, MG_RESID = 1, MG_START = 2, MG_LAST = 3 };

template <typename T, int N>
__device__ __forceinline__ void vload(const T* __restrict__ p, T (&v)[N]) {
  if constexpr (std::is_same<T, float>::value && N == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (std::is_same<T, float>::value && N == 2) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else if constexpr (std::is_same<T, double>::value && N >= 2) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const double2 q = *reinterpret_cast<const double2*>(p + i);
      v[i] = q.x; v[i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}

template <typename T, int N>
__device__ __forceinline__ void vstore(T* __restrict__ p, const T (&v)[N]) {
  if constexpr (std::is_same<T, float>::value && N == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (std::is_same<T, float>::value && N == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (std::is_same<T, double>::value && N >= 2) {
#pragma unroll
    for (int i = 0; i < N; i += 2) *reinterpret_cast<double2*>(p + i) = make_double2(v[i], v[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v[i];
  }
}

// One row of a Chebyshev pass (thread per row on the SELL-32 operator).
template <typename T, int NC, int NCP, int MODE, int G = kU>
__device__ __forceinline__ void mg_row(const DSell<T>& A, const T* __restrict__ dinv,
                                       const T* __restrict__ b, const T* __restrict__ Gin,
                                       const T* __restrict__ Din, T* __restrict__ Gout,
                                       T* __restrict__ Dout, T alpha, T beta, T inv_theta,
                                       T* __restrict__ out, int64_t out_ld,
                                       const int32_t* __restrict__ perm, int nc, int64_t row) {
  const int64_t sl = row >> 5;
  const int64_t o0 = (A.width ? sl * 32 * A.width : A.off[sl]) + (row & 31);
  const int64_t o1 = A.width ? (sl + 1) * 32 * A.width : A.off[sl + 1];
  T acc[NCP];
#pragma unroll
  for (int c = 0; c < NCP; ++c) acc[c] = T(0);
  // the slot count is the same for the whole slice: no divergence
  for (int64_t o = o0; o < o1; o += G * 32) {
    T a[G];
    int32_t j[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int64_t oo = o + u * 32;
      const bool ok = oo < o1;
      a[u] = ok ? A.v[oo] : T(0);
      j[u] = ok ? A.ci[oo] : (int32_t)row;
    }
    T g[G][NCP];
#pragma unroll
    for (int u = 0; u < G; ++u) vload<T, NCP>(Gin + (int64_t)j[u] * NCP, g[u]);
#pragma unroll
    for (int u = 0; u < G; ++u)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += a[u] * g[u][c];
  }
  T gx[NCP], d[NCP], bb[NCP];
  vload<T, NCP>(Gin + row * NCP, gx);
  if (MODE == MG_STEP || MODE == MG_LAST) vload<T, NCP>(Din + row * NCP, d);
  vload<T, NCP>(b + row * NCP, bb);
  const T di = dinv[row];
  T go[NCP], dout[NCP];
#pragma unroll
  for (int c = 0; c < NCP; ++c) {
    go[c] = T(0);
    dout[c] = T(0);
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T r = bb[c] - acc[c];
    if (MODE == MG_STEP) {
      dout[c] = alpha * d[c] + beta * di * r;
      go[c] = gx[c] + dout[c];
    } else if (MODE == MG_RESID) {
      go[c] = r;
    } else if (MODE == MG_START) {
      dout[c] = di * r * inv_theta;
      go[c] = gx[c] + dout[c];
    } else {
      go[c] = gx[c] + (alpha * d[c] + beta * di * r);
    }
  }
  if (MODE == MG_LAST && out) {
    const int64_t dst = perm ? perm[row] : row;
    for (int c = 0; c < nc; ++c) out[c * out_ld + dst] = go[c];
    return;
  }
  vstore<T, NCP>(Gout + row * NCP, go);
  if (MODE == MG_STEP || MODE == MG_START) vstore<T, NCP>(Dout + row * NCP, dout);
}

// Restriction row (L lanes; every lane of the group calls it, `active`
// false past the last row): bc = R r, and the coarse level's first step from
// x = 0: Gc = Dc = d0 = Dinv_c bc / theta (bc only when dinvc is null: the
// coarse level is solved densely).
template <typename T, int NCP, int L>
__device__ __forceinline__ void restrict_row(const DCsr<T>& R, const T* __restrict__ Rf,
                                             T* __restrict__ bc, T* __restrict__ Gc,
                                             T* __restrict__ Dc, const T* __restrict__ dinvc,
                                             T inv_theta_c, int64_t row, int lane, bool active) {
  T acc[NCP];
#pragma unroll
  for (int c = 0; c < NCP; ++c) acc[c] = T(0);
  if (active) {
    for (int32_t k = R.rp[row] + lane; k < R.rp[row + 1]; k += L) {
      const T a = R.v[k];
      T rj[NCP];
      vload<T, NCP>(Rf + (int64_t)R.ci[k] * NCP, rj);
#pragma unroll
      for (int c = 0; c < NCP; ++c) acc[c] += a * rj[c];
    }
  }
#pragma unroll
  for (int c = 0; c < NCP; ++c) acc[c] = group_sum<L>(acc[c]);
  if (lane != 0 || !active) return;
  vstore<T, NCP>(bc + row * NCP, acc);
  if (!dinvc) return;
  T d0[NCP];
  const T s = dinvc[row] * inv_theta_c;
#pragma unroll
  for (int c = 0; c < NCP; ++c) d0[c] = s * acc[c];
  vstore<T, NCP>(Gc + row * NCP, d0);
  vstore<T, NCP>(Dc + row * NCP, d0);
}

// Correction row x0 = x3 + P xc, in place in the fine gather vector Gf
// (each row reads and writes only its own entry there).
template <typename T, int NCP, int L>
__device__ __forceinline__ void prolong_row(const DCsr<T>& P, const T* __restrict__ Xc,
                                            T* __restrict__ Gf, int64_t row, int lane,
                                            bool active) {
  T acc[NCP];
#pragma unroll
  for (int c = 0; c < NCP; ++c) acc[c] = T(0);
  if (active) {
    for (int32_t k = P.rp[row] + lane; k < P.rp[row + 1]; k += L) {
      const T a = P.v[k];
      T xj[NCP];
      vload<T, NCP>(Xc + (int64_t)P.ci[k] * NCP, xj);
#pragma unroll
      for (int c = 0; c < NCP; ++c) acc[c] += a * xj[c];
    }
  }
#pragma unroll
  for (int c = 0; c < NCP; ++c) acc[c] = group_sum<L>(acc[c]);
  if (lane != 0 || !active) return;
  T x[NCP];
  vload<T, NCP>(Gf + row * NCP, x);
#pragma unroll
  for (int c = 0; c < NCP; ++c) x[c] += acc[c];
  vstore<T, NCP>(Gf + row * NCP, x);
}

// The coarsest level's dense blocks as a kernel reads them: one block of
// nb0 rows at offset 0 (a single problem, no lookups), or per row its block
// from the tables.
template <typename T>
struct DenseView {
  const T* cinv;
  const int32_t* row_blk;
  const int64_t *blk_row, *blk_n, *blk_dense;
  int64_t nb0;
};
template <typename T>
__host__ __device__ __forceinline__ DenseView<T> dense_view(const DHier<T>& H) {
  return DenseView<T>{H.cinv, H.row_blk, H.blk_row, H.blk_n, H.blk_dense, H.dense_nb0};
}

// Coarsest-level row x = blockdiag(Cinv) b (a warp per row); the result goes
// to X, or (level 0 being the coarsest) to the caller's blocked out.  The row
// of Cinv is read in 16-byte loads (a scalar head up to the first 16-byte
// boundary and a scalar tail), eight per lane in flight: a 3,500-row block
// has only ~23 rows per SM, so the loads of one warp must cover the memory
// latency.  b is re-read by every row from L1/L2.
template <typename T, int NCP, int U = 8>
__device__ __forceinline__ void dense_row(const DenseView<T>& D, const T* __restrict__ b,
                                          T* __restrict__ X, T* __restrict__ out,
                                          int64_t out_ld, const int32_t* __restrict__ perm,
                                          int nc, int64_t row, int lane, bool active) {
  T acc[NCP];
#pragma unroll
  for (int c = 0; c < NCP; ++c) acc[c] = T(0);
  if (active) {
    int64_t r0 = 0, nb = D.nb0, off = 0;
    if (nb == 0) {
      const int blk = D.row_blk[row];
      r0 = D.blk_row[blk];
      nb = D.blk_n[blk];
      off = D.blk_dense[blk];
    }
    const T* Cr = D.cinv + off + (row - r0) * nb;
    const T* bb = b + r0 * NCP;
    auto add = [&](T a, int64_t j) {
      T bj[NCP];
      vload<T, NCP>(bb + j * NCP, bj);
#pragma unroll
      for (int c = 0; c < NCP; ++c) acc[c] += a * bj[c];
    };
    using V = typename std::conditional<std::is_same<T, float>::value, float4, double2>::type;
    constexpr int E = 16 / sizeof(T);
    int64_t h = (int64_t)(((16 - ((uintptr_t)Cr & 15)) & 15) / sizeof(T));
    if (h > nb) h = nb;
    if (lane < h) add(Cr[lane], lane);
    const int64_t nvec = (nb - h) / E;
    const V* Cv = reinterpret_cast<const V*>(Cr + h);
    for (int64_t v0 = lane; v0 < nvec; v0 += 32 * U) {
      V q[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (v0 + 32 * u < nvec) q[u] = Cv[v0 + 32 * u];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (v0 + 32 * u >= nvec) break;
        const int64_t j = h + (v0 + 32 * u) * E;
        if constexpr (E == 4) {
          add(q[u].x, j);
          add(q[u].y, j + 1);
          add(q[u].z, j + 2);
          add(q[u].w, j + 3);
        } else {
          add(q[u].x, j);
          add(q[u].y, j + 1);
        }
      }
    }
    const int64_t t0 = h + nvec * E;  // fewer than E entries remain
    if (t0 + lane < nb) add(Cr[t0 + lane], t0 + lane);
  }
#pragma unroll
  for (int c = 0; c < NCP; ++c) acc[c] = group_sum<32>(acc[c]);
  if (lane != 0 || !active) return;
  if (out) {
    const int64_t dst = perm ? perm[row] : row;
    for (int c = 0; c < nc; ++c) out[c * out_ld + dst] = acc[c];
  } else {
    vstore<T, NCP>(X + row * NCP, acc);
  }
}

template <typename T, int NC, int NCP, int MODE, int G>
__global__ void __launch_bounds__(256) k_mg(DSell<T> A, const T* __restrict__ dinv,
                                            const T* __restrict__ b,
                                            const T* __restrict__ Gin,
                                            const T* __restrict__ Din,
                                            T* __restrict__ Gout, T* __restrict__ Dout,
                                            T alpha, T beta, T inv_theta, JVec<T> outv,
                                            int64_t out_ld, const int32_t* __restrict__ perm,
                                            int nc, SegSkip sk, const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= A.nrow || seg_skipped(sk, row)) return;
  mg_row<T, NC, NCP, MODE, G>(A, dinv, b, Gin, Din, Gout, Dout, alpha, beta, inv_theta,
                                  MODE == MG_LAST ? outv.get() : nullptr, out_ld, perm, nc, row);
}

template <typename T, int NCP, int L>
__global__ void __launch_bounds__(256) k_mg_restrict(DCsr<T> R, const T* __restrict__ Rf,
                                                     T* __restrict__ bc, T* __restrict__ Gc,
                                                     T* __restrict__ Dc,
                                                     const T* __restrict__ dinvc,
                                                     T inv_theta_c, SegSkip sk,
                                                     const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt / L;
  // skipped rows stay in the lane groups' shuffles (inactive)
  restrict_row<T, NCP, L>(R, Rf, bc, Gc, Dc, dinvc, inv_theta_c, row, (int)(gt % L),
                          row < R.nrow && !seg_skipped(sk, row));
}

template <typename T, int NCP, int L>
__global__ void __launch_bounds__(256) k_mg_prolong(DCsr<T> P, const T* __restrict__ Xc,
                                                    T* __restrict__ Gf, SegSkip sk,
                                                    const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gt / L;
  prolong_row<T, NCP, L>(P, Xc, Gf, row, (int)(gt % L), row < P.nrow && !seg_skipped(sk, row));
}

// The coarsest level's solve; every pointer and size comes by value, so no
// load precedes the rows' streams.
template <typename T, int NCP>
__global__ void k_mg_dense(DenseView<T> D, int64_t ncoarse, const T* __restrict__ b,
                           T* __restrict__ X, const int32_t* __restrict__ perm, JVec<T> outv,
                           int64_t out_ld, int nc, SegSkip sk, const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  dense_row<T, NCP>(D, b, X, outv.get(), out_ld, perm, nc, row, threadIdx.x & 31,
                    row < ncoarse && !seg_skipped(sk, row));
}

// The V-cycle from level l0 (its right-hand side and first step in place)
// down to the coarsest level and back, on one thread-block cluster: each
// pass of the kernel form is a phase here, every thread takes rows strided
// by the cluster's thread count (a warp still takes 32 consecutive rows of
// the SELL operator), and a cluster barrier (release/acquire) separates the
// phases.  Every thread reaches every barrier.  The level's result ends in
// G1[l0], or in `out` when l0 = 0.  Vectors written in one phase and read in
// the next go through plain loads: the barrier (barrier.cluster arrive with
// release, wait with acquire semantics) orders them at cluster scope.
// The transfer passes of the fused tail: every thread of the cluster takes
// rows LN at a time (LN consecutive lanes of one warp per row).
template <typename T, int NCP, int LN>
__device__ __forceinline__ void tail_restrict(const DCsr<T>& R, const T* Rf, T* bc, T* Gc, T* Dc,
                                              const T* dinvc, T inv_theta_c, int64_t tid,
                                              int64_t nth) {
  const int64_t nr = R.nrow, groups = nth / LN, sweeps = (nr + groups - 1) / groups;
  for (int64_t q = 0; q < sweeps; ++q) {
    const int64_t r = q * groups + tid / LN;
    restrict_row<T, NCP, LN>(R, Rf, bc, Gc, Dc, dinvc, inv_theta_c, r, (int)(tid % LN), r < nr);
  }
}

template <typename T, int NCP, int LN>
__device__ __forceinline__ void tail_prolong(const DCsr<T>& P, const T* Xc, T* Gf, int64_t tid,
                                             int64_t nth) {
  const int64_t nr = P.nrow, groups = nth / LN, sweeps = (nr + groups - 1) / groups;
  for (int64_t q = 0; q < sweeps; ++q) {
    const int64_t r = q * groups + tid / LN;
    prolong_row<T, NCP, LN>(P, Xc, Gf, r, (int)(tid % LN), r < nr);
  }
}

template <typename T, int NCP, int NT>
__global__ void __launch_bounds__(NT, 1) k_mg_tail(const DHier<T>* __restrict__ Hp, int l0,
                                                   JVec<T> outv, int64_t out_ld, int nc,
                                                   const int* skip) {
  if (skip && *skip) return;  // the same value for every thread of the cluster
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  constexpr int NC = NCP == 4 ? 3 : NCP;
  const DHier<T>& H = *Hp;
  const int64_t tid = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * NT;
  const int last = H.nlev - 1;
  const int lane32 = threadIdx.x & 31;
  for (int l = l0; l < last; ++l) {
    const DLevel<T>& L = H.lev[l];
    const int64_t n = L.A.nrow;
    T *G0 = H.G0[l], *G1 = H.G1[l], *D0 = H.D0[l], *D1 = H.D1[l];
    const T* b = H.b[l];
    const T a1 = (T)L.a1, b1 = (T)L.b1, a2 = (T)L.a2, b2 = (T)L.b2, it = (T)L.inv_theta;
    // degree 2 below the finest level: the phases of vcycle_level's light path
    const bool light = (l > 0 ? H.coarse_deg : H.fine_deg) == 2;
    for (int64_t r = tid; r < n; r += nth)
      mg_row<T, NC, NCP, MG_STEP>(L.A, L.dinv, b, G0, D0, G1, D1, a1, b1, it, nullptr, 0,
                                        nullptr, nc, r);
    cl.sync();
    if (light) {
      for (int64_t r = tid; r < n; r += nth)
        mg_row<T, NC, NCP, MG_RESID>(L.A, L.dinv, b, G1, D1, D0, nullptr, T(0), T(0), it,
                                     nullptr, 0, nullptr, nc, r);
    } else {
      for (int64_t r = tid; r < n; r += nth)
        mg_row<T, NC, NCP, MG_STEP>(L.A, L.dinv, b, G1, D1, G0, D0, a2, b2, it, nullptr, 0,
                                    nullptr, nc, r);
      cl.sync();
      for (int64_t r = tid; r < n; r += nth)
        mg_row<T, NC, NCP, MG_RESID>(L.A, L.dinv, b, G0, D0, G1, nullptr, T(0), T(0), it,
                                     nullptr, 0, nullptr, nc, r);
    }
    cl.sync();
    const DLevel<T>& C = H.lev[l + 1];
    const bool dense_next = l + 1 == last;
    const T* resid = light ? D0 : G1;
    const T* dinvc = dense_next ? nullptr : C.dinv;
    if (L.R.lanes == 32)
      tail_restrict<T, NCP, 32>(L.R, resid, H.b[l + 1], H.G0[l + 1], H.D0[l + 1], dinvc,
                                (T)C.inv_theta, tid, nth);
    else if (L.R.lanes == 1)
      tail_restrict<T, NCP, 1>(L.R, resid, H.b[l + 1], H.G0[l + 1], H.D0[l + 1], dinvc,
                               (T)C.inv_theta, tid, nth);
    else
      tail_restrict<T, NCP, 4>(L.R, resid, H.b[l + 1], H.G0[l + 1], H.D0[l + 1], dinvc,
                               (T)C.inv_theta, tid, nth);
    cl.sync();
  }
  {
    const int64_t nr = H.ncoarse, groups = nth / 32, sweeps = (nr + groups - 1) / groups;
    for (int64_t q = 0; q < sweeps; ++q) {
      const int64_t r = q * groups + tid / 32;
      dense_row<T, NCP>(dense_view(H), H.b[last], H.G1[last], nullptr, 0, nullptr, nc, r, lane32,
                              r < nr);
    }
    cl.sync();
  }
  T* out = outv.get();
  for (int l = last - 1; l >= l0; --l) {
    const DLevel<T>& L = H.lev[l];
    const int64_t n = L.A.nrow;
    T *G0 = H.G0[l], *G1 = H.G1[l], *D0 = H.D0[l], *D1 = H.D1[l];
    const T* b = H.b[l];
    const T a1 = (T)L.a1, b1 = (T)L.b1, a2 = (T)L.a2, b2 = (T)L.b2, it = (T)L.inv_theta;
    const bool light = (l > 0 ? H.coarse_deg : H.fine_deg) == 2;
    {
      T* corrected = light ? G1 : G0;
      if (L.P.lanes == 32)
        tail_prolong<T, NCP, 32>(L.P, H.G1[l + 1], corrected, tid, nth);
      else if (L.P.lanes == 1)
        tail_prolong<T, NCP, 1>(L.P, H.G1[l + 1], corrected, tid, nth);
      else
        tail_prolong<T, NCP, 4>(L.P, H.G1[l + 1], corrected, tid, nth);
    }
    cl.sync();
    if (light) {
      for (int64_t r = tid; r < n; r += nth)
        mg_row<T, NC, NCP, MG_START>(L.A, L.dinv, b, G1, nullptr, G0, D0, T(0), T(0), it,
                                     nullptr, 0, nullptr, nc, r);
      cl.sync();
      const bool top = l == 0 && out;
      for (int64_t r = tid; r < n; r += nth)
        mg_row<T, NC, NCP, MG_LAST>(L.A, L.dinv, b, G0, D0, G1, nullptr, a1, b1, it,
                                    top ? out : nullptr, out_ld, top ? H.perm : nullptr, nc, r);
      if (l > l0) cl.sync();
      continue;
    }
    for (int64_t r = tid; r < n; r += nth)
      mg_row<T, NC, NCP, MG_START>(L.A, L.dinv, b, G0, nullptr, G1, D1, T(0), T(0), it,
                                         nullptr, 0, nullptr, nc, r);
    cl.sync();
    for (int64_t r = tid; r < n; r += nth)
      mg_row<T, NC, NCP, MG_STEP>(L.A, L.dinv, b, G1, D1, G0, D0, a1, b1, it, nullptr, 0,
                                        nullptr, nc, r);
    cl.sync();
    const bool top = l == 0 && out;
    for (int64_t r = tid; r < n; r += nth)
      mg_row<T, NC, NCP, MG_LAST>(L.A, L.dinv, b, G0, D0, G1, nullptr, a2, b2, it,
                                        top ? out : nullptr, out_ld, top ? H.perm : nullptr, nc,
                                        r);
    if (l > l0) cl.sync();
  }
}

// Transfer passes with R.lanes / P.lanes threads per row.
// sk: the segments of R's rows (the coarse level) / of P's rows (the fine one).
template <typename T, int NCP>
void launch_restrict(const DCsr<T>& R, const T* Rf, T* bc, T* Gc, T* Dc, const T* dinvc,
                     T inv_theta_c, const SegSkip& sk, const int* skip, cudaStream_t s) {
  const int64_t rows = R.nrow;
  if (R.lanes == 32)
    launch_k(k_mg_restrict<T, NCP, 32>, blocks_for(rows * 32), 256, 0, s, R, Rf, bc, Gc, Dc,
             dinvc, inv_theta_c, sk, skip);
  else if (R.lanes == 1)
    launch_k(k_mg_restrict<T, NCP, 1>, blocks_for(rows), 256, 0, s, R, Rf, bc, Gc, Dc, dinvc,
             inv_theta_c, sk, skip);
  else
    launch_k(k_mg_restrict<T, NCP, 4>, blocks_for(rows * 4), 256, 0, s, R, Rf, bc, Gc, Dc,
             dinvc, inv_theta_c, sk, skip);
  count_launches(1);
}

template <typename T, int NCP>
void launch_prolong(const DCsr<T>& P, const T* Xc, T* Gf, const SegSkip& sk, const int* skip,
                    cudaStream_t s) {
  const int64_t rows = P.nrow;
  if (P.lanes == 32)
    launch_k(k_mg_prolong<T, NCP, 32>, blocks_for(rows * 32), 256, 0, s, P, Xc, Gf, sk, skip);
  else if (P.lanes == 1)
    launch_k(k_mg_prolong<T, NCP, 1>, blocks_for(rows), 256, 0, s, P, Xc, Gf, sk, skip);
  else
    launch_k(k_mg_prolong<T, NCP, 4>, blocks_for(rows * 4), 256, 0, s, P, Xc, Gf, sk, skip);
  count_launches(1);
}

template <typename T, int NCP>
void launch_mg(int mode, const DLevel<T>& L, const T* b, const T* Gin, const T* Din, T* Gout,
               T* Dout, T alpha, T beta, JVec<T> out, int64_t out_ld, const int32_t* perm, int nc,
               const int* skip, int group, cudaStream_t s) {
  const int64_t n = L.A.nrow;
  const T it = (T)L.inv_theta;
  constexpr int NC = NCP == 4 ? 3 : NCP;  // real components (3D pads 3 to 4)
#define FS_MG(M, G)                                                                        \
  launch_k(k_mg<T, NC, NCP, M, G>, blocks_for(n), 256, 0, s, L.A, L.dinv, b, Gin, Din, Gout,    \
           Dout, alpha, beta, it, out, out_ld, perm, nc, L.skip, skip)
  if (group == 6) {
    if (mode == MG_STEP) FS_MG(MG_STEP, 6);
    else if (mode == MG_RESID) FS_MG(MG_RESID, 6);
    else if (mode == MG_START) FS_MG(MG_START, 6);
    else FS_MG(MG_LAST, 6);
  } else {
    if (mode == MG_STEP) FS_MG(MG_STEP, 4);
    else if (mode == MG_RESID) FS_MG(MG_RESID, 4);
    else if (mode == MG_START) FS_MG(MG_START, 4);
    else FS_MG(MG_LAST, 4);
  }
#undef FS_MG
  count_launches(1);
}

// Threads per block of the cluster kernel: FP64 rows need twice the
// registers of FP32 ones.
template <typename T>
constexpr int tail_threads() {
  return std::is_same<T, float>::value ? 1024 : 512;
}

template <typename T, int NCP>
void launch_tail(const DHier<T>& H, int l0, JVec<T> out, int64_t out_ld, int nc, const int* skip,
                 cudaStream_t s) {
  constexpr int NT = tail_threads<T>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(H.tail_cluster);
  cfg.blockDim = dim3(NT);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = H.tail_cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_mg_tail<T, NCP, NT>, H.dev, l0, out, out_ld, nc, skip);
  count_launches(1);
}

// V-cycle below a level whose right-hand side b_l and first step (G0, D0)
// are in place; the level's result ends in G1[l], or in `out` for level 0.
template <typename T, int NCP>
void vcycle_level(const DHier<T>& H, int l, JVec<T> out, int64_t out_ld, int nc,
                  const int* skip, cudaStream_t s, bool first_done = false) {
  const bool top = l == 0;
  if (H.tail >= 0 && l == H.tail) {
    launch_tail<T, NCP>(H, l, top ? out : JVec<T>(), out_ld, nc, skip, s);
    return;
  }
  if (l == H.nlev - 1) {
    launch_k(k_mg_dense<T, NCP>, blocks_for(H.ncoarse * 32), 256, 0, s,
        dense_view(H), H.ncoarse, H.b[l], H.G1[l], top ? H.perm : nullptr,
        top ? out : JVec<T>(), out_ld, nc, H.lev[l].skip, skip);
    count_launches(1);
    return;
  }
  const DLevel<T>& L = H.lev[l];
  const DLevel<T>& C = H.lev[l + 1];
  const T a1 = (T)L.a1, b1 = (T)L.b1, a2 = (T)L.a2, b2 = (T)L.b2;
  T *G0 = H.G0[l], *G1 = H.G1[l], *D0 = H.D0[l], *D1 = H.D1[l];
  const T* b = H.b[l];
  const bool coarsest_next = l + 1 == H.nlev - 1;
  if ((top ? H.fine_deg : H.coarse_deg) == 1) {
    // degree 1: the first step of the load or restriction (x1 in G0, D0) is
    // the whole pre-smoothing; the residual into the free G1, the correction
    // into G0, and one step from there (the first step's formula, alpha = 0)
    // gives the level's result in G1
    launch_mg<T, NCP>(MG_RESID, L, b, G0, D0, G1, nullptr, T(0), T(0), JVec<T>(), 0, nullptr,
                      nc, skip, H.group, s);
    launch_restrict<T, NCP>(L.R, G1, H.b[l + 1], H.G0[l + 1], H.D0[l + 1],
                            coarsest_next ? nullptr : C.dinv, (T)C.inv_theta, C.skip, skip, s);
    vcycle_level<T, NCP>(H, l + 1, JVec<T>(), 0, nc, skip, s);
    launch_prolong<T, NCP>(L.P, H.G1[l + 1], G0, L.skip, skip, s);
    launch_mg<T, NCP>(MG_LAST, L, b, G0, D0, G1, nullptr, T(0), (T)L.inv_theta,
                      top ? out : JVec<T>(), out_ld, top ? H.perm : nullptr, nc, skip, H.group, s);
    return;
  }
  if ((top ? H.fine_deg : H.coarse_deg) == 2) {
    // degree 2 on a coarse level: one step after the restriction's first
    // (x2 in G1), the residual into the free D0, the correction into G1,
    // then the first post step and the last with the first step's
    // coefficients (the result in G1, as the degree-3 cycle leaves it);
    // first_done: the caller's load already took the first of these steps
    if (!first_done)
      launch_mg<T, NCP>(MG_STEP, L, b, G0, D0, G1, D1, a1, b1, JVec<T>(), 0, nullptr, nc, skip,
                        H.group, s);
    launch_mg<T, NCP>(MG_RESID, L, b, G1, D1, D0, nullptr, T(0), T(0), JVec<T>(), 0, nullptr,
                      nc, skip, H.group, s);
    launch_restrict<T, NCP>(L.R, D0, H.b[l + 1], H.G0[l + 1], H.D0[l + 1],
                            coarsest_next ? nullptr : C.dinv, (T)C.inv_theta, C.skip, skip, s);
    vcycle_level<T, NCP>(H, l + 1, JVec<T>(), 0, nc, skip, s);
    launch_prolong<T, NCP>(L.P, H.G1[l + 1], G1, L.skip, skip, s);
    launch_mg<T, NCP>(MG_START, L, b, G1, nullptr, G0, D0, T(0), T(0), JVec<T>(), 0, nullptr,
                      nc, skip, H.group, s);
    launch_mg<T, NCP>(MG_LAST, L, b, G0, D0, G1, nullptr, a1, b1, top ? out : JVec<T>(),
                      out_ld, top ? H.perm : nullptr, nc, skip, H.group, s);
    return;
  }
  if (!first_done)
    launch_mg<T, NCP>(MG_STEP, L, b, G0, D0, G1, D1, a1, b1, JVec<T>(), 0, nullptr, nc, skip,
                      H.group, s);
  launch_mg<T, NCP>(MG_STEP, L, b, G1, D1, G0, D0, a2, b2, JVec<T>(), 0, nullptr, nc, skip,
                    H.group, s);
  // residual of x3 = G0 into G1; G0 keeps x3 for the correction
  launch_mg<T, NCP>(MG_RESID, L, b, G0, D0, G1, nullptr, T(0), T(0), JVec<T>(), 0, nullptr, nc,
                    skip, H.group, s);
  launch_restrict<T, NCP>(L.R, G1, H.b[l + 1], H.G0[l + 1], H.D0[l + 1],
                          coarsest_next ? nullptr : C.dinv, (T)C.inv_theta, C.skip, skip, s);
  vcycle_level<T, NCP>(H, l + 1, JVec<T>(), 0, nc, skip, s);
  launch_prolong<T, NCP>(L.P, H.G1[l + 1], G0, L.skip, skip, s);
  launch_mg<T, NCP>(MG_START, L, b, G0, nullptr, G1, D1, T(0), T(0), JVec<T>(), 0, nullptr, nc,
                    skip, H.group, s);
  launch_mg<T, NCP>(MG_STEP, L, b, G1, D1, G0, D0, a1, b1, JVec<T>(), 0, nullptr, nc, skip,
                    H.group, s);
  launch_mg<T, NCP>(MG_LAST, L, b, G0, D0, G1, nullptr, a2, b2, top ? out : JVec<T>(), out_ld,
                    top ? H.perm : nullptr, nc, skip,
                    H.group, s);
}

// Cluster size of the fused V-cycle tail: 16 blocks (one per SM) where the
// device schedules such clusters, else the portable 8.
template <typename T, int NCP>
int tail_cluster_size() {
  constexpr int NT = tail_threads<T>();
  auto k = k_mg_tail<T, NCP, NT>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(NT);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) == cudaSuccess && nclusters > 0)
      return 16;
  }
  cudaGetLastError();
  return 8;
}

// ---------------------------------------------------------------------------
// Block preconditioner pieces
// ---------------------------------------------------------------------------
// Load of a single-component level-0 right-hand side (caller row q goes to
// level-0 row iperm[q]): b0 = r and the first step from x = 0,
// G0 = D0 = D^-1 r / theta.
template <typename T>
__global__ void k_mg_load1(int64_t n, JVec<const T> rv,
                           const int32_t* __restrict__ iperm, const T* __restrict__ dinv0,
                           T inv_theta0, T* __restrict__ b0, T* __restrict__ G0,
                           T* __restrict__ D0, const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const T* __restrict__ r = rv.get();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dst = iperm ? iperm[q] : q;
    const T v = r[q];
    const T d0 = dinv0 ? dinv0[dst] * v * inv_theta0 : T(0);
    b0[dst] = v;
    G0[dst] = d0;
    D0[dst] = d0;
  }
}

// The load of a single-component level 0 whose rows are in the caller's
// order, fused with its first Chebyshev step: the load's first step from
// x = 0 (G0 = D0 = D^-1 r / theta, b = r) is formed on the fly at every
// neighbour instead of being stored and read back, so the pass reads r and
// D^-1 at the neighbours and writes b, G1 and D1 (the same values, in the
// same order of operations, as k_mg_load1 followed by the STEP pass).
template <typename T, int G>
__global__ void __launch_bounds__(256) k_mg_first1(DSell<T> A, const T* __restrict__ dinv,
                                                   JVec<const T> rv, T inv_theta, T alpha,
                                                   T beta, T* __restrict__ b,
                                                   T* __restrict__ Gout, T* __restrict__ Dout,
                                                   SegSkip sk, const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= A.nrow || seg_skipped(sk, row)) return;
  const T* __restrict__ r = rv.get();
  const int64_t sl = row >> 5;
  const int64_t o0 = (A.width ? sl * 32 * A.width : A.off[sl]) + (row & 31);
  const int64_t o1 = A.width ? (sl + 1) * 32 * A.width : A.off[sl + 1];
  T acc = T(0);
  for (int64_t o = o0; o < o1; o += G * 32) {
    T a[G];
    int32_t j[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int64_t oo = o + u * 32;
      const bool ok = oo < o1;
      a[u] = ok ? A.v[oo] : T(0);
      j[u] = ok ? A.ci[oo] : (int32_t)row;
    }
    T g[G];
#pragma unroll
    for (int u = 0; u < G; ++u) g[u] = dinv[j[u]] * r[j[u]] * inv_theta;
#pragma unroll
    for (int u = 0; u < G; ++u) acc += a[u] * g[u];
  }
  const T v = r[row], di = dinv[row];
  const T g0 = di * v * inv_theta;
  const T d = alpha * g0 + beta * di * (v - acc);
  b[row] = v;
  Gout[row] = g0 + d;
  Dout[row] = d;
}

// Pressure part of the preconditioner in the convection-diffusion form:
// z_p = nu Mp^-1 r_p + dt^-1 y_K + Mp^-1 (N_p y_K), y_K = K_p^-1 r_p the
// pressure V-cycle's output (r_p on pinned rows, marked by a negative mpl).
template <typename T>
__global__ void __launch_bounds__(256) k_prec_pcd(int64_t nv, JVec<const T> rpv,
                                                  const T* __restrict__ yk,
                                                  const T* __restrict__ mpl, T inv_dt,
                                                  PcdView<T> pcd, JVec<T> zpv,
                                                  const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nv) return;
  const T* __restrict__ rp = rpv.get();
  const T m = mpl[q], p = rp[q];
  T z = p;
  if (m >= T(0)) {
    T acc = T(0);
    for (int32_t k = pcd.rp[q]; k < pcd.rp[q + 1]; ++k) acc += pcd.v[k] * yk[pcd.ci[k]];
    z = m * p + inv_dt * yk[q] + pcd.invm[q] * acc;
  }
  zpv.get()[q] = z;
}

// The Cahouet-Chabard combination and the velocity right-hand side of the
// V-cycle in one pass.  Threads [0, nvp) (nv rounded up to a warp) write the
// pressure part of the result, z_p = nu Mp^-1 r_p + dt^-1 y_K (y_K the
// pressure V-cycle's output), or z_p = r_p on a pinned row, which the
// scaling vector marks with a negative entry.  The following threads take
// the velocity rows (caller order): t_c = r_c + BT_c z_p, with z_p at each
// BT column evaluated from the same formula instead of being read back, stored
// at the level-0 (block-order) row iperm[i] as b0, with the first step from
// x = 0, G0 = D0 = D^-1 t / theta.
template <typename T>
__device__ __forceinline__ T cc_combine(const T* __restrict__ mpl, const T* __restrict__ rp,
                                        const T* __restrict__ yk, T inv_dt, int64_t q) {
  const T m = mpl[q], p = rp[q];
  return m < T(0) ? p : m * p + inv_dt * yk[q];
}

template <typename T, int DIM, int NCP, bool ZREAD>
__global__ void __launch_bounds__(256) k_bt_add_mg(DSell<T> BT, int64_t n2, int64_t nv,
                                                   JVec<const T> rv, const T* __restrict__ yk,
                                                   const T* __restrict__ mpl, T inv_dt,
                                                   JVec<T> zv, const int32_t* __restrict__ iperm,
                                                   const T* __restrict__ dinv0, T inv_theta0,
                                                   T* __restrict__ b0, T* __restrict__ G0,
                                                   T* __restrict__ D0, SegSkip sk0,
                                                   const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const T* __restrict__ r = rv.get();
  const T* __restrict__ rp = r + DIM * n2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nvp = (nv + 31) & ~(int64_t)31;
  // ZREAD: z_p was written by the pressure kernel before (convection-
  // diffusion form), read it back
  const T* __restrict__ zp = zv.get() + DIM * n2;
  if (t < nvp) {
    if (!ZREAD && t < nv) zv.get()[DIM * n2 + t] = cc_combine(mpl, rp, yk, inv_dt, t);
    return;
  }
  const int64_t row = t - nvp;
  if (row >= n2) return;
  const int64_t dst = iperm ? iperm[row] : row;
  if (seg_skipped(sk0, dst)) return;
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
  const int64_t o1 = BT.off[(row >> 5) + 1];
  for (int64_t o = BT.off[row >> 5] + (row & 31); o < o1; o += 32) {
    const int64_t base = (o - (row & 31)) * DIM + (row & 31);
    const T p = ZREAD ? zp[BT.ci[o]] : cc_combine(mpl, rp, yk, inv_dt, BT.ci[o]);
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] += BT.v[base + 32 * c] * p;
  }
  T tv[NCP], d0[NCP];
  const T sc = dinv0 ? dinv0[dst] * inv_theta0 : T(0);
#pragma unroll
  for (int c = 0; c < NCP; ++c) {
    tv[c] = c < DIM ? r[c * n2 + row] + acc[c] : T(0);
    d0[c] = sc * tv[c];
  }
  vstore<T, NCP>(b0 + dst * NCP, tv);
  vstore<T, NCP>(G0 + dst * NCP, d0);
  vstore<T, NCP>(D0 + dst * NCP, d0);
}

// Gauss-Jordan step c on W = [A | I] (n x 2n, row-major).  The pivot is the
// largest |W[r][c]| over r >= c (one block); the pivot row is swapped into
// row c and scaled by 1 / pivot; every other row r then subtracts
// W[r][c] times row c over the columns j > c.  Column c itself is left as it
// is (later steps never read it), so no thread writes what another reads.
__global__ void __launch_bounds__(1024) k_gj_pivot(const double* __restrict__ W, int64_t n,
                                                   int64_t c, int64_t* piv, double* pval,
                                                   int* bad) {
  __shared__ double bv[1024];
  __shared__ int64_t br[1024];
  double best = -1.0;
  int64_t arg = c;
  for (int64_t r = c + threadIdx.x; r < n; r += blockDim.x) {
    const double v = fabs(W[r * 2 * n + c]);
    if (v > best) {
      best = v;
      arg = r;
    }
  }
  bv[threadIdx.x] = best;
  br[threadIdx.x] = arg;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st && bv[threadIdx.x + st] > bv[threadIdx.x]) {
      bv[threadIdx.x] = bv[threadIdx.x + st];
      br[threadIdx.x] = br[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *piv = br[0];
    *pval = W[br[0] * 2 * n + c];
    if (!(bv[0] > 0.0)) *bad = 1;
  }
}

__global__ void k_gj_swap_scale(double* __restrict__ W, int64_t n, int64_t c,
                                const int64_t* __restrict__ piv,
                                const double* __restrict__ pval) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= 2 * n) return;
  const int64_t p = *piv;
  const double inv = 1.0 / *pval;
  const double a = W[c * 2 * n + j], b = W[p * 2 * n + j];
  W[c * 2 * n + j] = b * inv;
  if (p != c) W[p * 2 * n + j] = a;
}

__global__ void k_gj_eliminate(double* __restrict__ W, int64_t n, int64_t c) {
  const int64_t r = blockIdx.y;
  const int64_t j = c + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r == c || j >= 2 * n) return;
  const double f = W[r * 2 * n + c];
  if (f != 0.0) W[r * 2 * n + j] -= f * W[c * 2 * n + j];
}

template <typename T>
__global__ void k_gj_extract(const double* __restrict__ W, int64_t n, T* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = (T)W[(q / n) * 2 * n + n + q % n];
}

// Initial guess of a step's solve by extrapolation in time.
// x^(n+1) guess = sum_j c[j] x^(n-j): c[0] for x itself, c[j + 1] for p[j].
struct Extrap {
  const double* p[kExtrapMax];
  double c[kExtrapMax + 1];
};
__global__ void k_extrapolate(double* x, Extrap e, int nprev, double* dst, int64_t n) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = x[i];
    double g = e.c[0] * a;
#pragma unroll
    for (int j = 0; j < kExtrapMax; ++j)
      if (j < nprev) g += e.c[j + 1] * e.p[j][i];
    dst[i] = a;
    x[i] = g;
  }
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, int64_t n,
                          const double* scale, int inv) {
  pdl_wait();
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
void launch_spmv_full(const DOp<T>& op, JVec<const V> x, const V* b, JVec<V> y, int resid,
                      const int* skip, cudaStream_t s, bool seg) {
  const int64_t threads = ((op.nv + 31) & ~(int64_t)31) + op.n2;
  const SegSkip su = seg ? op.skip_u : SegSkip{}, sp = seg ? op.skip_p : SegSkip{};
  // slots per group: the schedule's, else 6 in FP32 and 4 in FP64 (FP64
  // rows are partly bound by FP64 arithmetic and do best shallower)
  const int g = op.group ? op.group : (std::is_same<V, float>::value ? kUSpmv : kU);
#define FS_SPMV(D, G) \
  launch_k(k_spmv_full<T, V, D, G>, blocks_for(threads), 256, 0, s, op, x, b, y, resid, su, sp, \
           skip)
  if (op.dim == 2) {
    if (g == 8) FS_SPMV(2, 8);
    else if (g == 6) FS_SPMV(2, 6);
    else FS_SPMV(2, 4);
  } else {
    if (g == 8) FS_SPMV(3, 8);
    else if (g == 6) FS_SPMV(3, 6);
    else FS_SPMV(3, 4);
  }
#undef FS_SPMV
  count_launches(1);
}
template void launch_spmv_full<double, double>(const DOp<double>&, JVec<const double>,
                                               const double*, JVec<double>, int, const int*,
                                               cudaStream_t, bool);
template void launch_spmv_full<float, float>(const DOp<float>&, JVec<const float>, const float*,
                                             JVec<float>, int, const int*, cudaStream_t, bool);

void launch_csr_to_sell(int64_t n, const int32_t* rp, const double* in, const int64_t* off,
                        double* out64, float* out32, cudaStream_t s) {
  k_csr_to_sell<<<blocks_for(n), 256, 0, s>>>(n, rp, in, off, out64, out32);
  count_launches(1);
}

template <typename T>
void launch_cheb_step(const DHier<T>& H, int nc, cudaStream_t s) {
  (void)nc;
  const DLevel<T>& L = H.lev[0];
  if (H.ncp == 4)
    launch_mg<T, 4>(MG_STEP, L, H.b[0], H.G0[0], H.D0[0], H.G1[0], H.D1[0], (T)L.a1, (T)L.b1,
                    nullptr, 0, nullptr, 3, nullptr, H.group, s);
  else if (H.ncp == 2)
    launch_mg<T, 2>(MG_STEP, L, H.b[0], H.G0[0], H.D0[0], H.G1[0], H.D1[0], (T)L.a1, (T)L.b1,
                    nullptr, 0, nullptr, 2, nullptr, H.group, s);
  else
    launch_mg<T, 1>(MG_STEP, L, H.b[0], H.G0[0], H.D0[0], H.G1[0], H.D1[0], (T)L.a1, (T)L.b1,
                    nullptr, 0, nullptr, 1, nullptr, H.group, s);
}
template <typename T>
int mg_tail_cluster(int ncp) {
  return ncp == 4 ? tail_cluster_size<T, 4>()
                  : ncp == 2 ? tail_cluster_size<T, 2>() : tail_cluster_size<T, 1>();
}
template int mg_tail_cluster<double>(int);
template int mg_tail_cluster<float>(int);

template void launch_cheb_step<double>(const DHier<double>&, int, cudaStream_t);
template void launch_cheb_step<float>(const DHier<float>&, int, cudaStream_t);

template <typename T>
void launch_precond(const DOp<T>& op, const DHier<T>& HA, const DHier<T>& HK,
                    const T* mpl_inv_nu, double inv_dt, JVec<const T> r, JVec<T> z,
                    T* work_p, T* work_u,
                    const int* skip, cudaStream_t s, const PcdView<T>& pcd) {
  (void)work_u;
  const int64_t n2 = op.n2, nv = op.nv;
  const int dim = op.dim;
  const JVec<const T> rp = r.shifted(dim * n2);
  // pressure: Cahouet-Chabard  z_p = nu Mp^-1 r_p + dt^-1 Kp^-1 r_p; the
  // load and the first smoothing step in one pass when level 0 is smoothed
  // by the per-pass kernels and its rows are in the caller's order
  {
    const bool k1 = HK.nlev > 1;
    const DLevel<T>& L0 = HK.lev[0];
    if (k1 && HK.tail != 0 && !HK.perm && HK.fine_deg != 1) {
      if (HK.group == 6)
        launch_k(k_mg_first1<T, 6>, blocks_for(nv), 256, 0, s, L0.A, L0.dinv, rp,
                 (T)L0.inv_theta, (T)L0.a1, (T)L0.b1, HK.b[0], HK.G1[0], HK.D1[0], L0.skip, skip);
      else
        launch_k(k_mg_first1<T, 4>, blocks_for(nv), 256, 0, s, L0.A, L0.dinv, rp,
                 (T)L0.inv_theta, (T)L0.a1, (T)L0.b1, HK.b[0], HK.G1[0], HK.D1[0], L0.skip, skip);
      count_launches(1);
      vcycle_level<T, 1>(HK, 0, JVec<T>(work_p), nv, 1, skip, s, /*first_done=*/true);
    } else {
      launch_k(k_mg_load1<T>, grid_stride_blocks(nv), 256, 0, s, nv, rp, HK.iperm,
               k1 ? L0.dinv : nullptr, (T)L0.inv_theta, HK.b[0], HK.G0[0], HK.D0[0], skip);
      count_launches(1);
      vcycle_level<T, 1>(HK, 0, JVec<T>(work_p), nv, 1, skip, s);
    }
  }
  // z_p and the velocity right-hand side in one pass (pinned rows are
  // marked in mpl_inv_nu), then z_u = A^-1 (r_u + BT z_p) by one V-cycle
  // on all components
  const bool a1 = HA.nlev > 1;
  const T* d0 = a1 ? HA.lev[0].dinv : nullptr;
  const T it0 = (T)HA.lev[0].inv_theta;
  const unsigned nb = blocks_for(((nv + 31) & ~(int64_t)31) + n2);
  const bool pc = pcd.v != nullptr;
  if (pc) {
    launch_k(k_prec_pcd<T>, blocks_for(nv), 256, 0, s, nv, rp, (const T*)work_p, mpl_inv_nu,
             (T)inv_dt, pcd, z.shifted(dim * n2), skip);
    count_launches(1);
  }
  if (dim == 2) {
    launch_k(pc ? k_bt_add_mg<T, 2, 2, true> : k_bt_add_mg<T, 2, 2, false>, nb, 256, 0, s,
             op.BT, n2, nv, r, (const T*)work_p, mpl_inv_nu, (T)inv_dt, z, HA.iperm, d0, it0,
             HA.b[0], HA.G0[0], HA.D0[0], HA.lev[0].skip, skip);
    count_launches(1);
    vcycle_level<T, 2>(HA, 0, z, n2, 2, skip, s);
  } else {
    launch_k(pc ? k_bt_add_mg<T, 3, 4, true> : k_bt_add_mg<T, 3, 4, false>, nb, 256, 0, s,
             op.BT, n2, nv, r, (const T*)work_p, mpl_inv_nu, (T)inv_dt, z, HA.iperm, d0, it0,
             HA.b[0], HA.G0[0], HA.D0[0], HA.lev[0].skip, skip);
    count_launches(1);
    vcycle_level<T, 4>(HA, 0, z, n2, 3, skip, s);
  }
}
template void launch_precond<double>(const DOp<double>&, const DHier<double>&,
                                     const DHier<double>&, const double*, double,
                                     JVec<const double>, JVec<double>,
                                     double*, double*, const int*, cudaStream_t,
                                     const PcdView<double>&);
template void launch_precond<float>(const DOp<float>&, const DHier<float>&,
                                    const DHier<float>&, const float*, double,
                                    JVec<const float>, JVec<float>, float*,
                                    float*, const int*, cudaStream_t, const PcdView<float>&);

// ---------------------------------------------------------------------------
// The block preconditioner as one persistent kernel over a work-list
// ---------------------------------------------------------------------------
namespace {

constexpr int kFlowThreads = 512;
constexpr uint64_t kFlowWaitNs = 1000000000ull;  // one second per wait

enum { FL_LOAD_P = 0, FL_MG, FL_RESTRICT, FL_PROLONG, FL_DENSE, FL_PREC_P, FL_BT_ADD };

// One phase of the application: which pass, on which hierarchy (0 pressure,
// 1 velocity), and every pointer and coefficient it takes.
template <typename T>
struct FlowPhase {
  int32_t kind = 0, hier = 0, mode = 0, lanes = 1;
  int32_t top = 0;  // writes the caller's vector (the last pass of level 0)
  DSell<T> A;       // FL_MG: level operator
  DCsr<T> X;        // FL_RESTRICT: R; FL_PROLONG: P
  // FL_MG: the level's inverse diagonal; FL_RESTRICT: the coarse level's
  // (null when the coarse level is solved densely); FL_LOAD_P, FL_BT_ADD:
  // level 0's (null for a hierarchy of one level)
  const T* dinv = nullptr;
  const T* b = nullptr;    // FL_MG, FL_DENSE: the level's right-hand side
  const T* in = nullptr;   // FL_MG: G in; FL_RESTRICT: fine residual; FL_PROLONG: coarse x
  const T* din = nullptr;  // FL_MG: D in
  T* out0 = nullptr;  // FL_MG: G out; FL_RESTRICT: coarse b; FL_PROLONG: fine G (in place);
                      // FL_DENSE: x; FL_LOAD_P, FL_BT_ADD: level-0 b
  T* out1 = nullptr;  // FL_MG: D out; FL_RESTRICT, FL_LOAD_P, FL_BT_ADD: G0
  T* out2 = nullptr;  // FL_RESTRICT, FL_LOAD_P, FL_BT_ADD: D0
  T alpha = 0, beta = 0, inv_theta = 0;
  const int32_t* perm = nullptr;  // level-0 block row -> caller row (or null)
  DenseView<T> dense{};           // FL_DENSE
};

template <typename T>
struct FlowArgs {
  FlowDev f;
  DSell<T> BT;
  JVec<const T> r;
  JVec<T> z;
  T* work_p;
  const T* mpl;
  T inv_dt;
  int64_t n2, nv;
  int dim;
  const SegState* st;
  SegState* flag;
  const int* skip;
};

__device__ __forceinline__ unsigned flow_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t flow_clock_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Chebyshev pass over rows [r0, r1) of one hierarchy (NC real components
// padded to NCP), a thread per row; the phase's fields are read once.
template <typename T, int NC, int NCP, int MODE>
__device__ __forceinline__ void flow_mg_rows(const FlowPhase<T>& ph, int64_t r0, int64_t r1,
                                             T* out, int64_t out_ld, int nc) {
  const DSell<T> A = ph.A;
  const T* dinv = ph.dinv;
  const T *b = ph.b, *in = ph.in, *din = ph.din;
  T *o0 = ph.out0, *o1 = ph.out1;
  const T al = ph.alpha, be = ph.beta, it = ph.inv_theta;
  const bool top = MODE == MG_LAST && ph.top;
  T* dst = top ? out : nullptr;
  const int32_t* perm = top ? ph.perm : nullptr;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += kFlowThreads)
    mg_row<T, NC, NCP, MODE, kU>(A, dinv, b, in, din, o0, o1, al, be, it, dst, out_ld, perm, nc,
                                 r);
}
template <typename T, int NC, int NCP>
__device__ __forceinline__ void flow_mg(const FlowPhase<T>& ph, int64_t r0, int64_t r1, T* out,
                                        int64_t out_ld, int nc) {
  switch (ph.mode) {
    case MG_STEP: flow_mg_rows<T, NC, NCP, MG_STEP>(ph, r0, r1, out, out_ld, nc); break;
    case MG_RESID: flow_mg_rows<T, NC, NCP, MG_RESID>(ph, r0, r1, out, out_ld, nc); break;
    case MG_START: flow_mg_rows<T, NC, NCP, MG_START>(ph, r0, r1, out, out_ld, nc); break;
    default: flow_mg_rows<T, NC, NCP, MG_LAST>(ph, r0, r1, out, out_ld, nc);
  }
}

// Transfer passes: L lanes per row, every thread of the block runs the same
// number of sweeps (the lane groups' shuffles need all 32 lanes).
template <typename T, int NCP, int L>
__device__ __forceinline__ void flow_restrict(const FlowPhase<T>& ph, int64_t r0, int64_t r1) {
  constexpr int rows = kFlowThreads / L;
  for (int64_t base = r0; base < r1; base += rows) {
    const int64_t r = base + threadIdx.x / L;
    restrict_row<T, NCP, L>(ph.X, ph.in, ph.out0, ph.out1, ph.out2, ph.dinv, ph.inv_theta, r,
                            (int)(threadIdx.x % L), r < r1);
  }
}
template <typename T, int NCP, int L>
__device__ __forceinline__ void flow_prolong(const FlowPhase<T>& ph, int64_t r0, int64_t r1) {
  constexpr int rows = kFlowThreads / L;
  for (int64_t base = r0; base < r1; base += rows) {
    const int64_t r = base + threadIdx.x / L;
    prolong_row<T, NCP, L>(ph.X, ph.in, ph.out0, r, (int)(threadIdx.x % L), r < r1);
  }
}
template <typename T, int NCP>
__device__ __forceinline__ void flow_transfer(const FlowPhase<T>& ph, int64_t r0, int64_t r1) {
  if (ph.kind == FL_RESTRICT) {
    if (ph.lanes == 32) flow_restrict<T, NCP, 32>(ph, r0, r1);
    else if (ph.lanes == 1) flow_restrict<T, NCP, 1>(ph, r0, r1);
    else flow_restrict<T, NCP, 4>(ph, r0, r1);
  } else {
    if (ph.lanes == 32) flow_prolong<T, NCP, 32>(ph, r0, r1);
    else if (ph.lanes == 1) flow_prolong<T, NCP, 1>(ph, r0, r1);
    else flow_prolong<T, NCP, 4>(ph, r0, r1);
  }
}
template <typename T, int NCP>
__device__ __forceinline__ void flow_dense(const FlowPhase<T>& ph, int64_t r0, int64_t r1,
                                           T* out, int64_t out_ld, int nc) {
  constexpr int rows = kFlowThreads / 32;
  for (int64_t base = r0; base < r1; base += rows) {
    const int64_t r = base + threadIdx.x / 32;
    dense_row<T, NCP, 2>(ph.dense, ph.b, ph.out0, ph.top ? out : nullptr, out_ld,
                      ph.top ? ph.perm : nullptr, nc, r, threadIdx.x & 31, r < r1);
  }
}

template <typename T, int NCP>
__device__ __forceinline__ void flow_item(const FlowArgs<T>& a, const FlowPhase<T>& ph,
                                          int64_t r0, int64_t r1) {
  constexpr int NC = NCP == 4 ? 3 : NCP;
  const int64_t vel = (int64_t)a.dim * a.n2;
  switch (ph.kind) {
    case FL_MG:
      if (ph.hier == 0) flow_mg<T, 1, 1>(ph, r0, r1, a.work_p, a.nv, 1);
      else flow_mg<T, NC, NCP>(ph, r0, r1, a.z.get(), a.n2, a.dim);
      break;
    case FL_RESTRICT:
    case FL_PROLONG:
      if (ph.hier == 0) flow_transfer<T, 1>(ph, r0, r1);
      else flow_transfer<T, NCP>(ph, r0, r1);
      break;
    case FL_DENSE:
      if (ph.hier == 0) flow_dense<T, 1>(ph, r0, r1, a.work_p, a.nv, 1);
      else flow_dense<T, NCP>(ph, r0, r1, a.z.get(), a.n2, a.dim);
      break;
    case FL_LOAD_P: {
      // level-0 rows of the pressure hierarchy: b0 = r_p, G0 = D0 = D^-1 r_p / theta
      const T* __restrict__ rp = a.r.get() + vel;
      for (int64_t d = r0 + threadIdx.x; d < r1; d += kFlowThreads) {
        const int64_t q = ph.perm ? ph.perm[d] : d;
        const T v = rp[q];
        const T d0 = ph.dinv ? ph.dinv[d] * v * ph.inv_theta : T(0);
        ph.out0[d] = v;
        ph.out1[d] = d0;
        ph.out2[d] = d0;
      }
      break;
    }
    case FL_PREC_P: {
      // caller pressure rows: z_p = nu Mp^-1 r_p + dt^-1 y_K (r_p on the
      // pinned rows, marked in the scaling vector)
      const T* __restrict__ rp = a.r.get() + vel;
      T* __restrict__ zp = a.z.get() + vel;
      for (int64_t q = r0 + threadIdx.x; q < r1; q += kFlowThreads)
        zp[q] = cc_combine(a.mpl, rp, a.work_p, a.inv_dt, q);
      break;
    }
    default: {  // FL_BT_ADD over level-0 rows of the velocity hierarchy
      const T* __restrict__ r = a.r.get();
      const T* __restrict__ zp = a.z.get() + vel;
      constexpr int DIM = NC;
      for (int64_t d = r0 + threadIdx.x; d < r1; d += kFlowThreads) {
        const int64_t row = ph.perm ? ph.perm[d] : d;
        T acc[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] = T(0);
        const int64_t o1 = a.BT.off[(row >> 5) + 1];
        for (int64_t o = a.BT.off[row >> 5] + (row & 31); o < o1; o += 32) {
          const int64_t base = (o - (row & 31)) * DIM + (row & 31);
          const T p = zp[a.BT.ci[o]];
#pragma unroll
          for (int c = 0; c < DIM; ++c) acc[c] += a.BT.v[base + 32 * c] * p;
        }
        T t[NCP], d0[NCP];
        const T sc = ph.dinv ? ph.dinv[d] * ph.inv_theta : T(0);
#pragma unroll
        for (int c = 0; c < NCP; ++c) {
          t[c] = c < DIM ? r[c * a.n2 + row] + acc[c] : T(0);
          d0[c] = sc * t[c];
        }
        vstore<T, NCP>(ph.out0 + d * NCP, t);
        vstore<T, NCP>(ph.out1 + d * NCP, d0);
        vstore<T, NCP>(ph.out2 + d * NCP, d0);
      }
    }
  }
}

template <typename T, int NCP>
__global__ void __launch_bounds__(kFlowThreads, 2) k_prec_flow(FlowArgs<T> a) {
  pdl_wait();
  if (a.skip && *a.skip) return;  // the same for every block: no counter is touched
  __shared__ int s_go[2];
  __shared__ int s_last;
  const FlowPhase<T>* __restrict__ phs = static_cast<const FlowPhase<T>*>(a.f.phases);
  const int nseg = a.f.nseg;
  int ok_p = -1, ok_s = -1;  // (phase, instance) whose predecessor was seen complete
  int par = 0;
  for (int64_t k = blockIdx.x; k < a.f.nitems; k += gridDim.x, par ^= 1) {
    const FlowItem it = a.f.items[k];
    if (threadIdx.x == 0) {
      int go = 1;
      if (a.st && a.st[it.seg].done) {
        go = 0;
      } else if (it.phase > 0 && !(it.phase == ok_p && it.seg == ok_s)) {
        const int64_t q = (int64_t)(it.phase - 1) * nseg + it.seg;
        const unsigned need = (unsigned)a.f.need[q];
        if (flow_ld_acquire(a.f.cnt + q) < need) {
          const uint64_t t0 = flow_clock_ns();
          while (flow_ld_acquire(a.f.cnt + q) < need) {
            if (flow_clock_ns() - t0 > kFlowWaitNs) {
              // give up: the item runs on stale data and the solve reports it
              if (a.flag) a.flag[it.seg].bad = 2;
              break;
            }
          }
        }
        ok_p = it.phase;
        ok_s = it.seg;
      }
      s_go[par] = go;
    }
    __syncthreads();
    if (!s_go[par]) continue;
    flow_item<T, NCP>(a, phs[it.phase], it.row0, it.row1);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.f.cnt + (int64_t)it.phase * nseg + it.seg, 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(a.f.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    const int64_t nc = (int64_t)a.f.nphase * nseg;
    for (int64_t i = threadIdx.x; i < nc; i += kFlowThreads) a.f.cnt[i] = 0;
    if (threadIdx.x == 0) *a.f.ticket = 0;
  }
}


// Phases of one application, in the order launch_precond issues its passes.
template <typename T>
struct FlowGen {
  std::vector<FlowPhase<T>> ph;
  std::vector<std::vector<int64_t>> rows;  // per phase: first row of each instance
  std::vector<int> sweep;                  // rows one block covers in one sweep

  void add(const FlowPhase<T>& p, const std::vector<int64_t>& r, int sw) {
    ph.push_back(p);
    rows.push_back(r);
    sweep.push_back(sw);
  }
  FlowPhase<T> mg(const DHier<T>& H, int hier, int l, int mode, const T* Gin, const T* Din,
                  T* Gout, T* Dout, double alpha, double beta, bool top) {
    FlowPhase<T> p;
    const DLevel<T>& L = H.lev[l];
    p.kind = FL_MG;
    p.hier = hier;
    p.mode = mode;
    p.top = top;
    p.A = L.A;
    p.dinv = L.dinv;
    p.b = H.b[l];
    p.in = Gin;
    p.din = Din;
    p.out0 = Gout;
    p.out1 = Dout;
    p.alpha = (T)alpha;
    p.beta = (T)beta;
    p.inv_theta = (T)L.inv_theta;
    p.perm = top ? H.perm : nullptr;
    return p;
  }
  // mirrors vcycle_level (without the fused cluster tail)
  void vcycle(const DHier<T>& H, int hier, const std::vector<std::vector<int64_t>>& off, int l) {
    const bool top = l == 0;
    const int kT = kFlowThreads;
    if (l == H.nlev - 1) {
      FlowPhase<T> p;
      p.kind = FL_DENSE;
      p.hier = hier;
      p.top = top;
      p.b = H.b[l];
      p.out0 = H.G1[l];
      p.perm = top ? H.perm : nullptr;
      p.dense = dense_view(H);
      add(p, off[l], kT / 32);
      return;
    }
    const DLevel<T>& L = H.lev[l];
    const DLevel<T>& C = H.lev[l + 1];
    T *G0 = H.G0[l], *G1 = H.G1[l], *D0 = H.D0[l], *D1 = H.D1[l];
    const bool coarsest_next = l + 1 == H.nlev - 1;
    auto restrict_from = [&](const T* resid) {
      FlowPhase<T> p;
      p.kind = FL_RESTRICT;
      p.hier = hier;
      p.lanes = L.R.lanes;
      p.X = L.R;
      p.in = resid;
      p.out0 = H.b[l + 1];
      p.out1 = H.G0[l + 1];
      p.out2 = H.D0[l + 1];
      p.dinv = coarsest_next ? nullptr : C.dinv;
      p.inv_theta = (T)C.inv_theta;
      add(p, off[l + 1], kT / p.lanes);
    };
    auto prolong_into = [&](T* Gf) {
      FlowPhase<T> p;
      p.kind = FL_PROLONG;
      p.hier = hier;
      p.lanes = L.P.lanes;
      p.X = L.P;
      p.in = H.G1[l + 1];
      p.out0 = Gf;
      add(p, off[l], kT / p.lanes);
    };
    if ((top ? H.fine_deg : H.coarse_deg) == 2) {
      add(mg(H, hier, l, MG_STEP, G0, D0, G1, D1, L.a1, L.b1, false), off[l], kT);
      add(mg(H, hier, l, MG_RESID, G1, D1, D0, nullptr, 0, 0, false), off[l], kT);
      restrict_from(D0);
      vcycle(H, hier, off, l + 1);
      prolong_into(G1);
      add(mg(H, hier, l, MG_START, G1, nullptr, G0, D0, 0, 0, false), off[l], kT);
      add(mg(H, hier, l, MG_LAST, G0, D0, G1, nullptr, L.a1, L.b1, top), off[l], kT);
      return;
    }
    add(mg(H, hier, l, MG_STEP, G0, D0, G1, D1, L.a1, L.b1, false), off[l], kT);
    add(mg(H, hier, l, MG_STEP, G1, D1, G0, D0, L.a2, L.b2, false), off[l], kT);
    add(mg(H, hier, l, MG_RESID, G0, D0, G1, nullptr, 0, 0, false), off[l], kT);
    restrict_from(G1);
    vcycle(H, hier, off, l + 1);
    prolong_into(G0);
    add(mg(H, hier, l, MG_START, G0, nullptr, G1, D1, 0, 0, false), off[l], kT);
    add(mg(H, hier, l, MG_STEP, G1, D1, G0, D0, L.a1, L.b1, false), off[l], kT);
    add(mg(H, hier, l, MG_LAST, G0, D0, G1, nullptr, L.a2, L.b2, top), off[l], kT);
  }
};

}  // namespace

template <typename T>
int flow_blocks(int ncp) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto k = ncp == 4 ? k_prec_flow<T, 4> : k_prec_flow<T, 2>;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kFlowThreads, 0);
  cudaGetLastError();
  return std::max(0, per) * sms;
}
template int flow_blocks<double>(int);
template int flow_blocks<float>(int);

template <typename T>
void build_flow(const DHier<T>& HA, const DHier<T>& HK,
                const std::vector<std::vector<int64_t>>& offA,
                const std::vector<std::vector<int64_t>>& offK, const std::vector<int64_t>& prow,
                int nblocks, FlowHost& out) {
  FlowGen<T> g;
  const int kT = kFlowThreads;
  {
    FlowPhase<T> p;
    p.kind = FL_LOAD_P;
    p.hier = 0;
    p.perm = HK.perm;
    p.dinv = HK.nlev > 1 ? HK.lev[0].dinv : nullptr;
    p.inv_theta = (T)HK.lev[0].inv_theta;
    p.out0 = HK.b[0];
    p.out1 = HK.G0[0];
    p.out2 = HK.D0[0];
    g.add(p, offK[0], kT);
  }
  g.vcycle(HK, 0, offK, 0);
  {
    FlowPhase<T> p;
    p.kind = FL_PREC_P;
    g.add(p, prow, kT);
  }
  {
    FlowPhase<T> p;
    p.kind = FL_BT_ADD;
    p.hier = 1;
    p.perm = HA.perm;
    p.dinv = HA.nlev > 1 ? HA.lev[0].dinv : nullptr;
    p.inv_theta = (T)HA.lev[0].inv_theta;
    p.out0 = HA.b[0];
    p.out1 = HA.G0[0];
    p.out2 = HA.D0[0];
    g.add(p, offA[0], kT);
  }
  g.vcycle(HA, 1, offA, 0);
  const int nphase = (int)g.ph.size();
  const int nseg = (int)prow.size() - 1;
  out.nphase = nphase;
  out.phases.resize(sizeof(FlowPhase<T>) * nphase);
  std::memcpy(out.phases.data(), g.ph.data(), out.phases.size());
  out.items.clear();
  out.need.assign((size_t)nphase * nseg, 0);
  const int64_t nb = std::max(1, nblocks);
  for (int p = 0; p < nphase; ++p) {
    const std::vector<int64_t>& r = g.rows[p];
    const int64_t sw = g.sweep[p];
    const int64_t total = r.back() - r.front();
    // enough items to reach every block when the phase has the rows for it
    const int64_t chunk = sw * std::max<int64_t>(1, total / (nb * sw));
    for (int s = 0; s < nseg; ++s)
      for (int64_t a = r[s]; a < r[s + 1]; a += chunk) {
        out.items.push_back(
            FlowItem{p, s, (int32_t)a, (int32_t)std::min(a + chunk, r[s + 1])});
        out.need[(size_t)p * nseg + s] += 1;
      }
  }
}
template void build_flow<double>(const DHier<double>&, const DHier<double>&,
                                 const std::vector<std::vector<int64_t>>&,
                                 const std::vector<std::vector<int64_t>>&,
                                 const std::vector<int64_t>&, int, FlowHost&);
template void build_flow<float>(const DHier<float>&, const DHier<float>&,
                                const std::vector<std::vector<int64_t>>&,
                                const std::vector<std::vector<int64_t>>&,
                                const std::vector<int64_t>&, int, FlowHost&);

template <typename T>
void launch_precond_flow(const FlowDev& f, const DOp<T>& op, const DHier<T>& HA,
                         const T* mpl_inv_nu, double inv_dt, JVec<const T> r, JVec<T> z,
                         T* work_p,
                         const SegState* st, SegState* flag, const int* skip, cudaStream_t s) {
  FlowArgs<T> a;
  a.f = f;
  a.BT = op.BT;
  a.r = r;
  a.z = z;
  a.work_p = work_p;
  a.mpl = mpl_inv_nu;
  a.inv_dt = (T)inv_dt;
  a.n2 = op.n2;
  a.nv = op.nv;
  a.dim = op.dim;
  a.st = st;
  a.flag = flag;
  a.skip = skip;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(f.nblocks);
  cfg.blockDim = dim3(kFlowThreads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  auto k = HA.ncp == 4 ? k_prec_flow<T, 4> : k_prec_flow<T, 2>;
  cudaLaunchKernelEx(&cfg, k, a);
  count_launches(1);
}
template void launch_precond_flow<double>(const FlowDev&, const DOp<double>&,
                                          const DHier<double>&, const double*, double,
                                          JVec<const double>,
                                          JVec<double>, double*, const SegState*, SegState*,
                                          const int*, cudaStream_t);
template void launch_precond_flow<float>(const FlowDev&, const DOp<float>&, const DHier<float>&,
                                         const float*, double,
                                         JVec<const float>, JVec<float>, float*,
                                         const SegState*, SegState*, const int*, cudaStream_t);

template <typename T>
void launch_vcycle_scalar(const DHier<T>& H, const T* r, T* z, int64_t n, cudaStream_t s) {
  const bool k1 = H.nlev > 1;
  launch_k(k_mg_load1<T>, grid_stride_blocks(n), 256, 0, s,
      n, JVec<const T>(r), H.iperm, k1 ? H.lev[0].dinv : nullptr, (T)H.lev[0].inv_theta, H.b[0],
      H.G0[0], H.D0[0], nullptr);
  count_launches(1);
  vcycle_level<T, 1>(H, 0, JVec<T>(z), n, 1, nullptr, s);
}
template void launch_vcycle_scalar<double>(const DHier<double>&, const double*, double*, int64_t,
                                           cudaStream_t);
template void launch_vcycle_scalar<float>(const DHier<float>&, const float*, float*, int64_t,
                                          cudaStream_t);

void launch_gj_step(double* W, int64_t n, int64_t c, int64_t* piv, double* pval, int* bad,
                    cudaStream_t s) {
  k_gj_pivot<<<1, 1024, 0, s>>>(W, n, c, piv, pval, bad);
  k_gj_swap_scale<<<blocks_for(2 * n), 256, 0, s>>>(W, n, c, piv, pval);
  const int64_t cols = 2 * n - c - 1;  // >= n >= 1
  k_gj_eliminate<<<dim3(blocks_for(cols), (unsigned)n), 256, 0, s>>>(W, n, c);
  count_launches(3);
}

template <typename T>
void launch_gj_extract(const double* W, int64_t n, T* out, cudaStream_t s) {
  k_gj_extract<T><<<grid_stride_blocks(n * n), 256, 0, s>>>(W, n, out);
  count_launches(1);
}
template void launch_gj_extract<double>(const double*, int64_t, double*, cudaStream_t);
template void launch_gj_extract<float>(const double*, int64_t, float*, cudaStream_t);

// Streams a buffer through the L2 with plain loads: afterwards the L2 holds
// clean lines of it (evicted without write-back) and nothing of the data
// the next timed kernel reads.  The sum is stored only when it is an
// impossible value, so the loads are not removed and nothing is written.
static __global__ void k_l2_flush(const int4* __restrict__ buf, int64_t n, int* sink) {
  int acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int4 v = buf[i];
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x7fffffff && sink) *sink = acc;
}

// Sums of (a_i - b_i)^2 and a_i^2 over i < n, in a fixed order: per-block
// partial sums of a grid of kNormBlocks blocks, then one block adds the
// partials.  Deterministic for a given n.
constexpr int kNormBlocks = 304;
static __device__ __forceinline__ void block_sum2(double& s0, double& s1) {
  __shared__ double sh[2][8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0][w] = s0;
    sh[1][w] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s0 = s1 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      s0 += sh[0][i];
      s1 += sh[1][i];
    }
  }
}
static __global__ void __launch_bounds__(256) k_diff_norms_part(const double* __restrict__ a,
                                                                const double* __restrict__ b,
                                                                int64_t n, double* part) {
  double s0 = 0, s1 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[i], d = x - b[i];
    s0 += d * d;
    s1 += x * x;
  }
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}
static __global__ void __launch_bounds__(256) k_diff_norms_fin(const double* part, int nb,
                                                               double* out) {
  double s0 = 0, s1 = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s0 += part[2 * i];
    s1 += part[2 * i + 1];
  }
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    out[0] = s0;
    out[1] = s1;
  }
}

int diff_norms_scratch() { return 2 * kNormBlocks + 2; }

void launch_diff_norms(const double* a, const double* b, int64_t n, double* scratch,
                       cudaStream_t s) {
  k_diff_norms_part<<<kNormBlocks, 256, 0, s>>>(a, b, n, scratch + 2);
  k_diff_norms_fin<<<1, 256, 0, s>>>(scratch + 2, kNormBlocks, scratch);
  count_launches(2);
}

void launch_l2_flush(const void* buf, int64_t bytes, int* sink, cudaStream_t s) {
  const int64_t n = bytes / 16;
  k_l2_flush<<<grid_stride_blocks(n), 256, 0, s>>>(static_cast<const int4*>(buf), n, sink);
}

void launch_extrapolate(double* x, const double* const* prev, int nprev, double* dst, int64_t n,
                        cudaStream_t s) {
  // Lagrange extrapolation to the next level of equally spaced levels:
  // (-1)^j C(nprev+1, j+1) for x^(n-j), j = 0..nprev
  Extrap e{};
  double binom = 1.0;  // C(nprev+1, j+1), built up over j
  for (int j = 0; j <= nprev; ++j) {
    binom = binom * (nprev + 1 - j) / (j + 1);
    e.c[j] = (j % 2 ? -1.0 : 1.0) * binom;
    if (j < nprev) e.p[j] = prev[j];
  }
  launch_k(k_extrapolate, grid_stride_blocks(n), 256, 0, s, x, e, nprev, dst, n);
  count_launches(1);
}

template <typename A, typename B>
void launch_convert(const A* in, B* out, int64_t n, const double* scale, int inv,
                    cudaStream_t s) {
  launch_k(k_convert<A, B>, grid_stride_blocks(n), 256, 0, s, in, out, n, scale, inv);
  count_launches(1);
}
template void launch_convert<double, float>(const double*, float*, int64_t, const double*, int,
                                            cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, const double*, int,
                                            cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, const double*,
                                             int, cudaStream_t);

}  // namespace fs
