// Segmented reductions and updates of flexible GMRES(m) (paper Sec. 3.2,
// GMRES) on sm_103a.
//
// A problem holds one or more independent instances ("segments": the
// instances of a batch, or the single mesh of an ordinary problem).  Every
// segment runs its own Arnoldi process: its own Hessenberg matrix, Givens
// rotations, convergence flag and update, so a segment's iterates do not
// depend on the other segments.  Vectors are walked through a work-list of
// tiles, each a contiguous range of one segment (at most kTileLen entries);
// one thread block per tile.  Per-tile partial sums go to scratch; the last
// tile of a segment to finish (per-segment atomic ticket, never waited on)
// reduces them in FP64.  Kernels that span all segments (SpMV, multigrid)
// skip their work once every segment has converged (KCtl::all_done).
#include <cuda_runtime.h>

#include <cmath>

#include <type_traits>

#include "fs_device.h"

namespace fs {

namespace {

constexpr unsigned kFull = 0xffffffffu;
// threads per tile block: the orthogonalisation passes stream the basis
// with few blocks (one per tile), so each block brings many warps, and each
// thread issues several independent loads, to keep enough bytes in flight
constexpr int kKB = 512;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// Block sum (all threads participate); valid in every thread afterwards.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sm[kKB / 32];
  __shared__ double total;
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < kKB / 32; ++i) t += sm[i];
    total = t;
  }
  __syncthreads();
  return total;
}

// True in every thread of the last tile block of its segment to arrive.
__device__ __forceinline__ bool last_of_segment(unsigned* counter, int ntiles) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)(ntiles - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum of partial[v * ntiles_total + t] over the segment's tiles, for v <
// nvec; result in res[v] (shared), all threads of the block participate.
__device__ void reduce_segment(const double* partial, int64_t stride, int first, int count,
                               int nvec, double* res) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = w; v < nvec; v += nw) {
    double s = 0;
    for (int t = lane; t < count; t += 32)
      s += ((volatile const double*)partial)[(int64_t)v * stride + first + t];
    s = warp_sum(s);
    if (lane == 0) res[v] = s;
  }
  __syncthreads();
}

// field: 0 beta, 1 bnorm, 2 rnorm
template <typename V>
__global__ void __launch_bounds__(kKB) k_seg_norm(const V* __restrict__ x, const Tile* tiles,
                                                  int ntiles, SegState* st, double* partial,
                                                  int field) {
  const Tile t = tiles[blockIdx.x];
  SegState& S = st[t.seg];
  double acc = 0;
  for (int e = threadIdx.x; e < t.len; e += kKB) {
    const double v = (double)x[t.start + e];
    acc += v * v;
  }
  const double bs = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs;
  if (!last_of_segment(&S.counter[4 + field], S.ntiles)) return;
  __shared__ double res[1];
  reduce_segment(partial, ntiles, S.first_tile, S.ntiles, 1, res);
  if (threadIdx.x == 0) {
    const double n = sqrt(res[0]);
    if (field == 0) S.beta = n;
    else if (field == 1) S.bnorm = n;
    else S.rnorm = n;
    S.counter[4 + field] = 0;
  }
}

// Start of a restart cycle: tolerances, right-hand side of the least-squares
// problem, done flags (converged, retired by the host, or non-finite).
// tol_abs = rtol * (relative_to_beta ? beta : bnorm).
__global__ void k_seg_cycle_init(SegState* st, KCtl* ctl, int relative_to_beta,
                                 cudaGraphConditionalHandle cond) {
  __shared__ int ndone;
  if (threadIdx.x == 0) ndone = 0;
  __syncthreads();
  const int m = ctl->m;
  for (int s = threadIdx.x; s < ctl->nseg; s += blockDim.x) {
    SegState& S = st[s];
    const double beta = S.beta;
    S.tol_abs = S.rtol * (relative_to_beta ? beta : S.bnorm);
    S.k = 0;
    S.bad = isfinite(beta) ? 0 : 1;
    S.resid = beta;
    for (int i = 0; i <= m; ++i) S.g[i] = 0.0;
    S.g[0] = beta;
    S.done = (S.retired || S.bad || beta <= S.tol_abs || beta == 0.0) ? 1 : 0;
    if (S.done) atomicAdd(&ndone, 1);
    for (int c = 0; c < 4; ++c) S.counter[c] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->ndone = ndone;
    ctl->all_done = ndone == ctl->nseg ? 1 : 0;
    ctl->j = 0;
    if (cond) cudaGraphSetConditional(cond, ndone == ctl->nseg ? 0u : 1u);
  }
}

// x *= 1 / (field 0: beta, 1: hn) of the tile's segment (skipped once done)
template <typename V>
__global__ void __launch_bounds__(kKB) k_seg_scale(JVec<V> xv, const Tile* tiles,
                                                   const SegState* st, int field) {
  const Tile t = tiles[blockIdx.x];
  const SegState& S = st[t.seg];
  if (S.done) return;
  V* __restrict__ x = xv.get();
  const V f = (V)(1.0 / (field == 0 ? S.beta : S.hn));
  for (int e = threadIdx.x; e < t.len; e += kKB) x[t.start + e] *= f;
}

// Classical Gram-Schmidt with one reorthogonalisation (CGS2) of the new
// Arnoldi vector w = V[j+1] against V[0..j], j = ctl->j, in three passes:
//   dot : h = V^T w                                    -> H[0..j, j]
//   upd : w' = w - V h;  h2 = V^T w';  ||w'||^2         -> H[0..j, j] += h2,
//         H[j+1, j] = hn = sqrt(||w'||^2 - ||h2||^2)
//   fin : V[j+1] = (w' - V h2) / hn
// hn is the norm of w'' = w' - V h2 by Pythagoras (V^T w' = h2 and V
// orthonormal); h2 is a rounding-size correction, so the difference loses
// nothing.  A block takes one tile: its slice of w is staged in shared
// memory, the dots are taken by warps over (vector, chunk) units with the
// per-lane sums in the vector type and the cross-lane and cross-tile sums in
// FP64, and the updates by threads over elements with the coefficients in
// shared memory.

// Dots of the staged tile slice ws with the first nvec basis vectors (and
// ws . ws as entry nvec when `norm`), added into sums[] (shared).
template <typename V>
__device__ __forceinline__ void tile_dots(const V* __restrict__ Vb, int64_t n, const Tile& t,
                                          const V* ws, int nvec, bool norm, double* sums) {
  constexpr int NW = kKB / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nout = nvec + (norm ? 1 : 0);
  const int split = nout >= NW ? 1 : (NW + nout - 1) / nout;
  const int chunk = ((t.len + split - 1) / split + 31) & ~31;
  for (int u = warp; u < nout * split; u += NW) {
    const int v = u / split, c = u % split;
    const int e0 = c * chunk, e1 = min(t.len, e0 + chunk);
    V acc = V(0);
    if (e1 <= e0) {
      // an empty chunk (the last ones of a short tile)
    } else if (v < nvec) {
      // 16-byte loads of the basis vector: a scalar head up to its first
      // 16-byte boundary in [e0, e1), the aligned body, a scalar tail (the
      // stride n is arbitrary, so the boundary differs between vectors);
      // ws is read with scalar shared loads
      using VV = typename std::conditional<sizeof(V) == 4, float4, double2>::type;
      constexpr int E = 16 / sizeof(V);
      const V* __restrict__ p = Vb + (int64_t)v * n + t.start + e0;
      const int len = e1 - e0;
      int h = (int)(((16 - ((uintptr_t)p & 15)) & 15) / sizeof(V));
      if (h > len) h = len;
      if (lane < h) acc += p[lane] * ws[e0 + lane];
      const int nq = (len - h) / E;
      const VV* __restrict__ q = reinterpret_cast<const VV*>(p + h);
      const V* wq = ws + e0 + h;
#pragma unroll 4
      for (int k = lane; k < nq; k += 32) {
        const VV x = q[k];
        if constexpr (E == 4) {
          acc += x.x * wq[4 * k] + x.y * wq[4 * k + 1] + x.z * wq[4 * k + 2] +
                 x.w * wq[4 * k + 3];
        } else {
          acc += x.x * wq[2 * k] + x.y * wq[2 * k + 1];
        }
      }
      const int t0 = h + nq * E;  // fewer than E entries remain
      if (t0 + lane < len) acc += p[t0 + lane] * ws[e0 + t0 + lane];
    } else {
#pragma unroll 8
      for (int e = e0 + lane; e < e1; e += 32) acc += ws[e] * ws[e];
    }
    const double sv = warp_sum((double)acc);
    if (lane == 0) atomicAdd(&sums[v], sv);
  }
}

// The thread's elements of a tile: e = threadIdx.x + k kKB, k < kElems.
constexpr int kElems = kTileLen / kKB;
static_assert(kElems * kKB == kTileLen, "tile length must be a multiple of the block size");

// w_e <- w_e - sum_v coef[v] V[v]_e for all the thread's elements at once
// (w[k] for element k; entries past the tile are left alone): U basis
// vectors at a time for every element (4 in FP32, 2 in FP64 to keep the
// registers for two blocks per SM), so up to U kElems loads are in flight
// per thread.
template <typename V>
__device__ __forceinline__ void tile_update(const V* __restrict__ Vb, int64_t n, const Tile& t,
                                            const V* coef, int nvec, V (&w)[kElems]) {
  constexpr int U = sizeof(V) == 4 ? 4 : 2;
  V acc[kElems][U];
#pragma unroll
  for (int k = 0; k < kElems; ++k)
#pragma unroll
    for (int u = 0; u < U; ++u) acc[k][u] = V(0);
  int v = 0;
  for (; v + U <= nvec; v += U) {
#pragma unroll
    for (int k = 0; k < kElems; ++k) {
      const int e = threadIdx.x + k * kKB;
      if (e < t.len) {
        const V* __restrict__ p = Vb + (int64_t)v * n + t.start + e;
#pragma unroll
        for (int u = 0; u < U; ++u) acc[k][u] += coef[v + u] * p[(int64_t)u * n];
      }
    }
  }
  for (; v < nvec; ++v) {
#pragma unroll
    for (int k = 0; k < kElems; ++k) {
      const int e = threadIdx.x + k * kKB;
      if (e < t.len) acc[k][0] += coef[v] * Vb[(int64_t)v * n + t.start + e];
    }
  }
#pragma unroll
  for (int k = 0; k < kElems; ++k) {
    V sum = V(0);
#pragma unroll
    for (int u = 0; u < U; ++u) sum += acc[k][u];
    w[k] -= sum;
  }
}

// Givens rotations of column j of one active segment's Hessenberg matrix,
// its least-squares residual, and the end of its cycle (converged, broken
// or at the restart length): the segment is then marked done and counted.
__device__ void givens_segment(SegState& S, KCtl* ctl, int j, int m) {
  double* H = S.H;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], b = H[(i + 1) * m + j];
    H[i * m + j] = S.cs[i] * a + S.sn[i] * b;
    H[(i + 1) * m + j] = -S.sn[i] * a + S.cs[i] * b;
  }
  const double a = H[j * m + j], b = H[(j + 1) * m + j];
  const double den = hypot(a, b);
  const double c = den == 0.0 ? 1.0 : a / den, sn = den == 0.0 ? 0.0 : b / den;
  S.cs[j] = c;
  S.sn[j] = sn;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  S.g[j + 1] = -sn * S.g[j];
  S.g[j] = c * S.g[j];
  S.resid = fabs(S.g[j + 1]);
  S.k = j + 1;
  bool finish = false;
  if (!isfinite(S.resid) || !isfinite(den) || den == 0.0) {
    S.bad = isfinite(S.resid) && isfinite(den) ? S.bad : 1;
    S.k = j;  // drop the broken column
    finish = true;
  } else if (S.resid <= S.tol_abs || b == 0.0 || j + 1 >= m) {
    finish = true;
  }
  if (finish) {
    S.done = 1;
    if (atomicAdd(&ctl->ndone, 1) + 1 == ctl->nseg) ctl->all_done = 1;
  }
}

// The step index advances and the loop node's condition (if any) becomes
// "a segment is still active and j + 1 < m" (one thread).
__device__ void end_arnoldi_step(KCtl* ctl, int j, int m, cudaGraphConditionalHandle cond) {
  const int all = atomicAdd(&ctl->all_done, 0);
  ctl->j = j + 1;
  if (cond) cudaGraphSetConditional(cond, (!all && j + 1 < m) ? 1u : 0u);
}

template <typename V>
__global__ void __launch_bounds__(kKB) k_seg_dot(const V* __restrict__ Vb, int64_t n,
                                                 const Tile* tiles, int ntiles, SegState* st,
                                                 const KCtl* ctl, double* partial) {
  const Tile t = tiles[blockIdx.x];
  SegState& S = st[t.seg];
  if (S.done) return;
  const int j = ctl->j, m = ctl->m, nvec = j + 1;
  __shared__ V ws[kTileLen];
  __shared__ double sums[kMaxRestart + 2];
  const V* __restrict__ w = Vb + (int64_t)(j + 1) * n + t.start;
  for (int e = threadIdx.x; e < t.len; e += kKB) ws[e] = w[e];
  for (int v = threadIdx.x; v < nvec; v += kKB) sums[v] = 0.0;
  __syncthreads();
  tile_dots<V>(Vb, n, t, ws, nvec, false, sums);
  __syncthreads();
  for (int v = threadIdx.x; v < nvec; v += kKB) partial[(int64_t)v * ntiles + blockIdx.x] = sums[v];
  if (!last_of_segment(&S.counter[1], S.ntiles)) return;
  __shared__ double res[kMaxRestart + 2];
  reduce_segment(partial, ntiles, S.first_tile, S.ntiles, nvec, res);
  if (threadIdx.x == 0) {
    for (int i = 0; i < nvec; ++i) S.H[i * m + j] = res[i];
    S.counter[1] = 0;
  }
}

// GIV (problems of one segment): the last block also takes the step's
// Givens rotations and advances the step index (no separate Givens kernel);
// the final pass then reads j as ctl->j - 1.
template <typename V, bool GIV>
__global__ void __launch_bounds__(kKB) k_seg_upd(V* __restrict__ Vb, int64_t n,
                                                 const Tile* tiles, int ntiles, SegState* st,
                                                 KCtl* ctl, double* partial,
                                                 cudaGraphConditionalHandle cond) {
  const Tile t = tiles[blockIdx.x];
  SegState& S = st[t.seg];
  if (S.done) return;
  const int j = ctl->j, m = ctl->m, nvec = j + 1;
  __shared__ V ws[kTileLen];
  __shared__ V coef[kMaxRestart + 1];
  __shared__ double sums[kMaxRestart + 2];
  for (int v = threadIdx.x; v < nvec; v += kKB) coef[v] = (V)S.H[v * m + j];
  for (int v = threadIdx.x; v <= nvec; v += kKB) sums[v] = 0.0;
  __syncthreads();
  V* __restrict__ w = Vb + (int64_t)(j + 1) * n;
  V wv[kElems];
#pragma unroll
  for (int k = 0; k < kElems; ++k) {
    const int e = threadIdx.x + k * kKB;
    wv[k] = e < t.len ? w[t.start + e] : V(0);
  }
  tile_update<V>(Vb, n, t, coef, nvec, wv);
#pragma unroll
  for (int k = 0; k < kElems; ++k) {
    const int e = threadIdx.x + k * kKB;
    if (e < t.len) {
      ws[e] = wv[k];
      w[t.start + e] = wv[k];
    }
  }
  __syncthreads();
  tile_dots<V>(Vb, n, t, ws, nvec, true, sums);
  __syncthreads();
  for (int v = threadIdx.x; v <= nvec; v += kKB)
    partial[(int64_t)v * ntiles + blockIdx.x] = sums[v];
  if (!last_of_segment(&S.counter[2], S.ntiles)) return;
  __shared__ double res[kMaxRestart + 2];
  reduce_segment(partial, ntiles, S.first_tile, S.ntiles, nvec + 1, res);
  if (threadIdx.x == 0) {
    double hh = 0;
    for (int i = 0; i < nvec; ++i) {
      S.h2[i] = res[i];
      S.H[i * m + j] += res[i];
      hh += res[i] * res[i];
    }
    const double hn = sqrt(fmax(res[nvec] - hh, 0.0));
    S.hn = hn;
    S.H[(j + 1) * m + j] = hn;
    S.counter[2] = 0;
    if constexpr (GIV) {
      givens_segment(S, ctl, j, m);
      end_arnoldi_step(ctl, j, m, cond);
    }
  }
}

template <typename V>
__global__ void __launch_bounds__(kKB) k_seg_fin(V* __restrict__ Vb, int64_t n,
                                                 const Tile* tiles, SegState* st,
                                                 const KCtl* ctl, int jshift) {
  const Tile t = tiles[blockIdx.x];
  const SegState& S = st[t.seg];
  if (S.done) return;
  const int j = ctl->j - jshift, nvec = j + 1;
  __shared__ V coef[kMaxRestart + 1];
  for (int v = threadIdx.x; v < nvec; v += kKB) coef[v] = (V)S.h2[v];
  __syncthreads();
  const V f = (V)(1.0 / S.hn);
  V* __restrict__ w = Vb + (int64_t)(j + 1) * n;
  V wv[kElems];
#pragma unroll
  for (int k = 0; k < kElems; ++k) {
    const int e = threadIdx.x + k * kKB;
    wv[k] = e < t.len ? w[t.start + e] : V(0);
  }
  tile_update<V>(Vb, n, t, coef, nvec, wv);
#pragma unroll
  for (int k = 0; k < kElems; ++k) {
    const int e = threadIdx.x + k * kKB;
    if (e < t.len) w[t.start + e] = wv[k] * f;
  }
}

// Givens rotations of column j = ctl->j of every active segment (one block,
// segments strided over its threads); then the step index advances and the
// condition of the loop node (if any) becomes "a segment is still active and
// j < m".
__global__ void k_seg_givens(SegState* st, KCtl* ctl, cudaGraphConditionalHandle cond) {
  const int m = ctl->m;
  const int j = ctl->j;
  for (int s = threadIdx.x; s < ctl->nseg; s += blockDim.x) {
    SegState& S = st[s];
    if (!S.done) givens_segment(S, ctl, j, m);
  }
  __syncthreads();
  if (threadIdx.x == 0) end_arnoldi_step(ctl, j, m, cond);
}

// y = H(0:k,0:k)^-1 g(0:k) of the tile's segment, then x += xscale Z y
template <typename V, typename X>
__global__ void __launch_bounds__(kKB) k_seg_update_x(const SegState* st, const KCtl* ctl,
                                                      const V* __restrict__ Z, int64_t n,
                                                      const Tile* tiles, X* __restrict__ x) {
  __shared__ double y[kMaxRestart];
  const Tile t = tiles[blockIdx.x];
  const SegState& S = st[t.seg];
  const int k = S.k;
  if (k == 0) return;
  if (threadIdx.x == 0) {
    const int m = ctl->m;
    for (int i = k - 1; i >= 0; --i) {
      double s = S.g[i];
      for (int c = i + 1; c < k; ++c) s -= S.H[i * m + c] * y[c];
      y[i] = s / S.H[i * m + i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < t.len; e += kKB) {
    const int64_t i = t.start + e;
    // four directions at a time into separate sums (independent loads)
    double s[4] = {0, 0, 0, 0};
    int c = 0;
    for (; c + 4 <= k; c += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) s[u] += y[c + u] * (double)Z[(int64_t)(c + u) * n + i];
    }
    for (; c < k; ++c) s[0] += y[c] * (double)Z[(int64_t)c * n + i];
    x[i] = (X)((double)x[i] + ((s[0] + s[1]) + (s[2] + s[3])));
  }
}

// out = in / rnorm of the segment (0 for retired segments)
template <typename A, typename B>
__global__ void __launch_bounds__(kKB) k_seg_normalise(const A* __restrict__ in,
                                                       B* __restrict__ out, const Tile* tiles,
                                                       const SegState* st) {
  const Tile t = tiles[blockIdx.x];
  const SegState& S = st[t.seg];
  const double f = (S.retired || S.rnorm == 0.0) ? 0.0 : 1.0 / S.rnorm;
  for (int e = threadIdx.x; e < t.len; e += kKB)
    out[t.start + e] = (B)((double)in[t.start + e] * f);
}

// x += rnorm d for the segments that are still refined
template <typename V, typename X>
__global__ void __launch_bounds__(kKB) k_seg_axpy(X* __restrict__ x, const V* __restrict__ d,
                                                  const Tile* tiles, const SegState* st) {
  const Tile t = tiles[blockIdx.x];
  const SegState& S = st[t.seg];
  if (S.retired) return;
  const double a = S.rnorm;
  for (int e = threadIdx.x; e < t.len; e += kKB)
    x[t.start + e] = (X)((double)x[t.start + e] + a * (double)d[t.start + e]);
}

}  // namespace

// ---------------------------------------------------------------------------
template <typename V>
void launch_seg_norm(const V* x, const TileList& tl, SegState* st, double* partial, int field,
                     cudaStream_t s) {
  k_seg_norm<V><<<tl.ntiles, kKB, 0, s>>>(x, tl.tiles, tl.ntiles, st, partial, field);
  count_launches(1);
}
template void launch_seg_norm<double>(const double*, const TileList&, SegState*, double*, int,
                                      cudaStream_t);
template void launch_seg_norm<float>(const float*, const TileList&, SegState*, double*, int,
                                     cudaStream_t);

void launch_seg_cycle_init(SegState* st, KCtl* ctl, int relative_to_beta,
                           cudaGraphConditionalHandle cond, cudaStream_t s) {
  k_seg_cycle_init<<<1, 256, 0, s>>>(st, ctl, relative_to_beta, cond);
  count_launches(1);
}

template <typename V>
void launch_seg_scale(JVec<V> x, const TileList& tl, const SegState* st, int field,
                      cudaStream_t s) {
  k_seg_scale<V><<<tl.ntiles, kKB, 0, s>>>(x, tl.tiles, st, field);
  count_launches(1);
}
template void launch_seg_scale<double>(JVec<double>, const TileList&, const SegState*, int,
                                       cudaStream_t);
template void launch_seg_scale<float>(JVec<float>, const TileList&, const SegState*, int,
                                      cudaStream_t);

template <typename V>
void launch_seg_cgs2(V* Vb, int64_t n, const TileList& tl, SegState* st, KCtl* ctl,
                     double* partial, bool with_givens, cudaGraphConditionalHandle cond,
                     cudaStream_t s) {
  k_seg_dot<V><<<tl.ntiles, kKB, 0, s>>>(Vb, n, tl.tiles, tl.ntiles, st, ctl, partial);
  if (with_givens)
    k_seg_upd<V, true><<<tl.ntiles, kKB, 0, s>>>(Vb, n, tl.tiles, tl.ntiles, st, ctl, partial,
                                                 cond);
  else
    k_seg_upd<V, false><<<tl.ntiles, kKB, 0, s>>>(Vb, n, tl.tiles, tl.ntiles, st, ctl, partial,
                                                  0);
  k_seg_fin<V><<<tl.ntiles, kKB, 0, s>>>(Vb, n, tl.tiles, st, ctl, with_givens ? 1 : 0);
  count_launches(3);
}
template void launch_seg_cgs2<double>(double*, int64_t, const TileList&, SegState*, KCtl*,
                                      double*, bool, cudaGraphConditionalHandle, cudaStream_t);
template void launch_seg_cgs2<float>(float*, int64_t, const TileList&, SegState*, KCtl*, double*,
                                     bool, cudaGraphConditionalHandle, cudaStream_t);

template <typename V>
void launch_seg_cgs2_pass(V* Vb, int64_t n, const TileList& tl, SegState* st, KCtl* ctl,
                          double* partial, int pass, cudaStream_t s) {
  if (pass == 0)
    k_seg_dot<V><<<tl.ntiles, kKB, 0, s>>>(Vb, n, tl.tiles, tl.ntiles, st, ctl, partial);
  else if (pass == 1)
    k_seg_upd<V, false><<<tl.ntiles, kKB, 0, s>>>(Vb, n, tl.tiles, tl.ntiles, st, ctl, partial,
                                                  0);
  else
    k_seg_fin<V><<<tl.ntiles, kKB, 0, s>>>(Vb, n, tl.tiles, st, ctl, 0);
  count_launches(1);
}
template void launch_seg_cgs2_pass<double>(double*, int64_t, const TileList&, SegState*, KCtl*,
                                           double*, int, cudaStream_t);
template void launch_seg_cgs2_pass<float>(float*, int64_t, const TileList&, SegState*, KCtl*,
                                          double*, int, cudaStream_t);

void launch_seg_givens(SegState* st, KCtl* ctl, int nseg, cudaGraphConditionalHandle cond,
                       cudaStream_t s) {
  (void)nseg;
  k_seg_givens<<<1, 256, 0, s>>>(st, ctl, cond);
  count_launches(1);
}

template <typename V, typename X>
void launch_seg_update_x(const SegState* st, const KCtl* ctl, const V* Z, int64_t n,
                         const TileList& tl, X* x, cudaStream_t s) {
  k_seg_update_x<V, X><<<tl.ntiles, kKB, 0, s>>>(st, ctl, Z, n, tl.tiles, x);
  count_launches(1);
}
template void launch_seg_update_x<double, double>(const SegState*, const KCtl*, const double*,
                                                  int64_t, const TileList&, double*,
                                                  cudaStream_t);
template void launch_seg_update_x<float, float>(const SegState*, const KCtl*, const float*,
                                                int64_t, const TileList&, float*, cudaStream_t);

template <typename A, typename B>
void launch_seg_normalise(const A* in, B* out, const TileList& tl, const SegState* st,
                          cudaStream_t s) {
  k_seg_normalise<A, B><<<tl.ntiles, kKB, 0, s>>>(in, out, tl.tiles, st);
  count_launches(1);
}
template void launch_seg_normalise<double, float>(const double*, float*, const TileList&,
                                                  const SegState*, cudaStream_t);

template <typename V, typename X>
void launch_seg_axpy(X* x, const V* d, const TileList& tl, const SegState* st, cudaStream_t s) {
  k_seg_axpy<V, X><<<tl.ntiles, kKB, 0, s>>>(x, d, tl.tiles, st);
  count_launches(1);
}
template void launch_seg_axpy<float, double>(double*, const float*, const TileList&,
                                             const SegState*, cudaStream_t);

}  // namespace fs
