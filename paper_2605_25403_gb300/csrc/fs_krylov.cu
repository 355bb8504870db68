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

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
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
// A warp per vector; a lane reads its tiles four at a time (loads from L2,
// where the other blocks' partials are visible after the ticket) into four
// sums, added in a fixed order.
__device__ void reduce_segment(const double* partial, int64_t stride, int first, int count,
                               int nvec, double* res) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = w; v < nvec; v += nw) {
    const double* p = partial + (int64_t)v * stride + first;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int t = lane;
    for (; t + 96 < count; t += 128) {
      const double a0 = __ldcg(p + t), a1 = __ldcg(p + t + 32), a2 = __ldcg(p + t + 64),
                   a3 = __ldcg(p + t + 96);
      s0 += a0;
      s1 += a1;
      s2 += a2;
      s3 += a3;
    }
    for (; t < count; t += 32) s0 += __ldcg(p + t);
    double s = warp_sum((s0 + s1) + (s2 + s3));
    if (lane == 0) res[v] = s;
  }
  __syncthreads();
}

// field: 0 beta, 1 bnorm, 2 rnorm
template <typename V>
__global__ void __launch_bounds__(kKB) k_seg_norm(const V* __restrict__ x, const Tile* tiles,
                                                  int ntiles, SegState* st, double* partial,
                                                  int field) {
  pdl_wait();
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
  pdl_wait();
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
  pdl_wait();
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
// nothing.
//
// A block takes one tile (at most kTileLen = 2,048 entries); thread t of the
// block takes the entries t + 512 k, k < kLE = 4, so every warp has entries
// while the tile is longer than 1,536 (coalesced scalar loads whatever the
// alignment of a vector, whose stride n is arbitrary).  A lane reads the
// basis vectors in batches of kNB (8 in FP32, 4 in FP64): the kNB x kLE loads
// of a batch are issued together and held in registers, so a pass takes
// ceil((j + 1) / kNB) load rounds, and the update pass takes the dots of the
// updated w' with its last batch from the registers, re-reading only the
// earlier batches.  Dot products are summed per lane in the vector type,
// across the warp by shuffles in the vector type too (four products per
// lane, then a reduce-scatter over the batch's vectors: in FP32 a sum of 128
// terms with far less rounding than a sequential one; FP64 arithmetic runs
// at 1/58 of the FP32 rate on this GPU, and one FP64 warp reduction per
// vector per warp made the whole pass 2.3x slower), then in FP64 across
// warps in a fixed order and across tiles by the segment's last block.
constexpr int kLE = kTileLen / kKB;
static_assert(kLE * kKB == kTileLen, "tile length must be a multiple of the block size");
static_assert(kLE == 4, "a lane takes four entries of its warp's 128");
constexpr int kNW = kKB / 32;  // warps per block

template <typename V>
struct Batch {
  static constexpr int NB = sizeof(V) == 4 ? 8 : 4;  // basis vectors per load round
};

// The thread's entries of one vector of the tile (0 past the tile's end).
template <typename V>
__device__ __forceinline__ void lane_load(const V* __restrict__ p, int e0, int len,
                                          V (&x)[kLE]) {
#pragma unroll
  for (int k = 0; k < kLE; ++k) x[k] = e0 + kKB * k < len ? p[e0 + kKB * k] : V(0);
}

// Loads basis vectors v0 .. v0 + nb - 1 (nb <= NB) of the tile at once.
template <typename V, int NB>
__device__ __forceinline__ void batch_load(const V* __restrict__ base, int64_t n, int v0, int nb,
                                           int e0, int len, V (&x)[NB][kLE]) {
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (b < nb) lane_load(base + (int64_t)(v0 + b) * n, e0, len, x[b]);
}

// Reduce-scatter of NB per-lane values over a warp (NB a power of two):
// at the level with xor offset o, a lane keeps half of its slots (the upper
// half when bit o of its index is set) and adds the partner's copy of them,
// so after log2(NB) levels lane l holds slot l / (32 / NB) summed over the
// lanes that share it, and the remaining levels finish that sum.  NB - 1 +
// 5 - log2(NB) additions per lane instead of 5 NB for NB separate sums.
template <int NB, typename R>
__device__ __forceinline__ R warp_transpose_sum(R (&v)[NB]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int half = NB / 2, off = 16; half >= 1; half /= 2, off /= 2) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const R send = hi ? v[i] : v[i + half];
      const R keep = hi ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, off);
    }
  }
  R s = v[0];
#pragma unroll
  for (int off = 16 / NB; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  return s;
}

// wpart[warp][v0 + b] = warp sum of x[b] . y over the lane's entries, b < nb.
template <typename V, int NB>
__device__ __forceinline__ void batch_dots(const V (&x)[NB][kLE], const V (&y)[kLE], int v0,
                                           int nb, double (*wpart)[kMaxRestart + 2]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  V d[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    d[b] = V(0);
    if (b < nb) {
#pragma unroll
      for (int k = 0; k < kLE; ++k) d[b] += x[b][k] * y[k];
    }
  }
  const V s = warp_transpose_sum<NB, V>(d);
  constexpr int kShare = 32 / NB;  // lanes holding one slot's sum
  const int slot = lane / kShare;
  if (lane % kShare == 0 && slot < nb) wpart[warp][v0 + slot] = (double)s;
}

// acc -= sum_b coef[v0 + b] x[b] (per entry)
template <typename V, int NB>
__device__ __forceinline__ void batch_axpy(const V (&x)[NB][kLE], const V* coef, int v0, int nb,
                                           V (&acc)[kLE]) {
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (b < nb) {
      const V c = coef[v0 + b];
#pragma unroll
      for (int k = 0; k < kLE; ++k) acc[k] += c * x[b][k];
    }
}

// partial[v ntiles + tile] = sum over the block's warps (fixed order) of
// wpart[.][v], v < nout.
__device__ __forceinline__ void block_partials(double (*wpart)[kMaxRestart + 2], int nout,
                                               double* partial, int ntiles) {
  __syncthreads();
  for (int v = threadIdx.x; v < nout; v += kKB) {
    double sum = 0;
#pragma unroll
    for (int q = 0; q < kNW; ++q) sum += wpart[q][v];
    partial[(int64_t)v * ntiles + blockIdx.x] = sum;
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
__global__ void __launch_bounds__(kKB, 2) k_seg_dot(const V* __restrict__ Vb, int64_t n,
                                                    const Tile* tiles, int ntiles, SegState* st,
                                                    const KCtl* ctl, double* partial) {
  pdl_wait();
  constexpr int NB = Batch<V>::NB;
  const Tile t = tiles[blockIdx.x];
  SegState& S = st[t.seg];
  if (S.done) return;
  const int j = ctl->j, m = ctl->m, nvec = j + 1;
  __shared__ double wpart[kNW][kMaxRestart + 2];
  const int e0 = threadIdx.x;
  const V* __restrict__ base = Vb + t.start;
  V w[kLE];
  lane_load(base + (int64_t)(j + 1) * n, e0, t.len, w);
  V x[NB][kLE];
  for (int v0 = 0; v0 < nvec; v0 += NB) {
    const int nb = min(NB, nvec - v0);
    batch_load<V, NB>(base, n, v0, nb, e0, t.len, x);
    batch_dots<V, NB>(x, w, v0, nb, wpart);
  }
  block_partials(wpart, nvec, partial, ntiles);
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
__global__ void __launch_bounds__(kKB, 2) k_seg_upd(V* __restrict__ Vb, int64_t n,
                                                    const Tile* tiles, int ntiles, SegState* st,
                                                    KCtl* ctl, double* partial,
                                                    cudaGraphConditionalHandle cond) {
  pdl_wait();
  constexpr int NB = Batch<V>::NB;
  const Tile t = tiles[blockIdx.x];
  SegState& S = st[t.seg];
  if (S.done) return;
  const int j = ctl->j, m = ctl->m, nvec = j + 1;
  __shared__ V coef[kMaxRestart + 1];
  __shared__ double wpart[kNW][kMaxRestart + 2];
  for (int v = threadIdx.x; v < nvec; v += kKB) coef[v] = (V)S.H[v * m + j];
  __syncthreads();
  const int e0 = threadIdx.x, lane = threadIdx.x & 31;
  const V* __restrict__ base = Vb + t.start;
  V* __restrict__ wp = Vb + (int64_t)(j + 1) * n + t.start;
  V w[kLE], acc[kLE];
  lane_load(wp, e0, t.len, w);
#pragma unroll
  for (int k = 0; k < kLE; ++k) acc[k] = V(0);
  V x[NB][kLE];
  int last0 = 0;
  for (int v0 = 0; v0 < nvec; v0 += NB) {
    const int nb = min(NB, nvec - v0);
    batch_load<V, NB>(base, n, v0, nb, e0, t.len, x);
    batch_axpy<V, NB>(x, coef, v0, nb, acc);
    last0 = v0;
  }
  V nn = V(0);
#pragma unroll
  for (int k = 0; k < kLE; ++k) {
    w[k] -= acc[k];
    nn += w[k] * w[k];
    if (e0 + kKB * k < t.len) wp[e0 + kKB * k] = w[k];
  }
  // re-dot: the last batch is still in registers, the earlier ones are
  // read again
  batch_dots<V, NB>(x, w, last0, nvec - last0, wpart);
  for (int v0 = 0; v0 < last0; v0 += NB) {
    batch_load<V, NB>(base, n, v0, NB, e0, t.len, x);
    batch_dots<V, NB>(x, w, v0, NB, wpart);
  }
  nn = warp_sum(nn);
  if (lane == 0) wpart[threadIdx.x >> 5][nvec] = (double)nn;
  block_partials(wpart, nvec + 1, partial, ntiles);
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
__global__ void __launch_bounds__(kKB, 2) k_seg_fin(V* __restrict__ Vb, int64_t n,
                                                    const Tile* tiles, SegState* st,
                                                    const KCtl* ctl, int jshift) {
  pdl_wait();
  constexpr int NB = Batch<V>::NB;
  const Tile t = tiles[blockIdx.x];
  const SegState& S = st[t.seg];
  if (S.done) return;
  const int j = ctl->j - jshift, nvec = j + 1;
  __shared__ V coef[kMaxRestart + 1];
  for (int v = threadIdx.x; v < nvec; v += kKB) coef[v] = (V)S.h2[v];
  __syncthreads();
  const V f = (V)(1.0 / S.hn);
  const int e0 = threadIdx.x;
  const V* __restrict__ base = Vb + t.start;
  V* __restrict__ wp = Vb + (int64_t)(j + 1) * n + t.start;
  V w[kLE], acc[kLE];
  lane_load(wp, e0, t.len, w);
#pragma unroll
  for (int k = 0; k < kLE; ++k) acc[k] = V(0);
  V x[NB][kLE];
  for (int v0 = 0; v0 < nvec; v0 += NB) {
    const int nb = min(NB, nvec - v0);
    batch_load<V, NB>(base, n, v0, nb, e0, t.len, x);
    batch_axpy<V, NB>(x, coef, v0, nb, acc);
  }
#pragma unroll
  for (int k = 0; k < kLE; ++k)
    if (e0 + kKB * k < t.len) wp[e0 + kKB * k] = (w[k] - acc[k]) * f;
}

// Givens rotations of column j = ctl->j of every active segment (one block,
// segments strided over its threads); then the step index advances and the
// condition of the loop node (if any) becomes "a segment is still active and
// j < m".
__global__ void k_seg_givens(SegState* st, KCtl* ctl, cudaGraphConditionalHandle cond) {
  pdl_wait();
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
  pdl_wait();
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
  pdl_wait();
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
  pdl_wait();
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
  launch_k(k_seg_norm<V>, tl.ntiles, kKB, 0, s, x, tl.tiles, tl.ntiles, st, partial, field);
  count_launches(1);
}
template void launch_seg_norm<double>(const double*, const TileList&, SegState*, double*, int,
                                      cudaStream_t);
template void launch_seg_norm<float>(const float*, const TileList&, SegState*, double*, int,
                                     cudaStream_t);

void launch_seg_cycle_init(SegState* st, KCtl* ctl, int relative_to_beta,
                           cudaGraphConditionalHandle cond, cudaStream_t s) {
  launch_k(k_seg_cycle_init, 1, 256, 0, s, st, ctl, relative_to_beta, cond);
  count_launches(1);
}

template <typename V>
void launch_seg_scale(JVec<V> x, const TileList& tl, const SegState* st, int field,
                      cudaStream_t s) {
  launch_k(k_seg_scale<V>, tl.ntiles, kKB, 0, s, x, tl.tiles, st, field);
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
  launch_k(k_seg_dot<V>, tl.ntiles, kKB, 0, s, Vb, n, tl.tiles, tl.ntiles, st, ctl, partial);
  if (with_givens)
    launch_k(k_seg_upd<V, true>, tl.ntiles, kKB, 0, s, Vb, n, tl.tiles, tl.ntiles, st, ctl, partial,
                                                 cond);
  else
    launch_k(k_seg_upd<V, false>, tl.ntiles, kKB, 0, s, Vb, n, tl.tiles, tl.ntiles, st, ctl, partial,
                                                  0);
  launch_k(k_seg_fin<V>, tl.ntiles, kKB, 0, s, Vb, n, tl.tiles, st, ctl, with_givens ? 1 : 0);
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
    launch_k(k_seg_dot<V>, tl.ntiles, kKB, 0, s, Vb, n, tl.tiles, tl.ntiles, st, ctl, partial);
  else if (pass == 1)
    launch_k(k_seg_upd<V, false>, tl.ntiles, kKB, 0, s, Vb, n, tl.tiles, tl.ntiles, st, ctl, partial,
                                                  0);
  else
    launch_k(k_seg_fin<V>, tl.ntiles, kKB, 0, s, Vb, n, tl.tiles, st, ctl, 0);
  count_launches(1);
}
template void launch_seg_cgs2_pass<double>(double*, int64_t, const TileList&, SegState*, KCtl*,
                                           double*, int, cudaStream_t);
template void launch_seg_cgs2_pass<float>(float*, int64_t, const TileList&, SegState*, KCtl*,
                                          double*, int, cudaStream_t);

void launch_seg_givens(SegState* st, KCtl* ctl, int nseg, cudaGraphConditionalHandle cond,
                       cudaStream_t s) {
  (void)nseg;
  launch_k(k_seg_givens, 1, 256, 0, s, st, ctl, cond);
  count_launches(1);
}

template <typename V, typename X>
void launch_seg_update_x(const SegState* st, const KCtl* ctl, const V* Z, int64_t n,
                         const TileList& tl, X* x, cudaStream_t s) {
  launch_k(k_seg_update_x<V, X>, tl.ntiles, kKB, 0, s, st, ctl, Z, n, tl.tiles, x);
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
  launch_k(k_seg_normalise<A, B>, tl.ntiles, kKB, 0, s, in, out, tl.tiles, st);
  count_launches(1);
}
template void launch_seg_normalise<double, float>(const double*, float*, const TileList&,
                                                  const SegState*, cudaStream_t);

template <typename V, typename X>
void launch_seg_axpy(X* x, const V* d, const TileList& tl, const SegState* st, cudaStream_t s) {
  launch_k(k_seg_axpy<V, X>, tl.ntiles, kKB, 0, s, x, d, tl.tiles, st);
  count_launches(1);
}
template void launch_seg_axpy<float, double>(double*, const float*, const TileList&,
                                             const SegState*, cudaStream_t);

}  // namespace fs
