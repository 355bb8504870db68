// FP64 residual norms of a monolithic CSR system on the device: the check a
// caller runs on a solution against the system exported by fs_dof_map /
// fs_assemble_step (paper Sec. 3.1: the error/residual step after the linear
// solver).  One fused pass: every row group computes r_i = b_i - (A x)_i and
// accumulates r_i^2 and b_i^2; per-block partial sums go to scratch and the
// last block to finish (atomic ticket, no waiting) reduces them in FP64.
#include <cuda_runtime.h>

#include <string>

#include "fs_device.h"

namespace fs {

namespace {

constexpr int kResBlock = 256;
constexpr int kResLanes = 8;
constexpr int kRowsPerBlock = kResBlock / kResLanes;

// partial: 2 doubles per block; counter: one unsigned (zero on entry);
// out: 2 doubles (||b - A x||^2 summed, ||b||^2 summed) -> sqrt applied.
__global__ void __launch_bounds__(kResBlock) k_csr_resid(
    int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const double* __restrict__ va, const double* __restrict__ x,
    const double* __restrict__ b, double* partial, unsigned* counter, double* out) {
  __shared__ double sm_r[kResBlock / 32], sm_b[kResBlock / 32];
  __shared__ bool last;
  const int lane = threadIdx.x % kResLanes;
  double rr = 0.0, bb = 0.0;
  // the loop bound is uniform over the block so that every lane reaches the
  // shuffles; rows past n contribute nothing
  for (int64_t base = (int64_t)blockIdx.x * kRowsPerBlock; base < n;
       base += (int64_t)gridDim.x * kRowsPerBlock) {
    const int64_t row = base + threadIdx.x / kResLanes;
    double acc = 0.0;
    if (row < n)
      for (int64_t k = rp[row] + lane; k < rp[row + 1]; k += kResLanes) acc += va[k] * x[ci[k]];
#pragma unroll
    for (int off = kResLanes / 2; off > 0; off >>= 1)
      acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0 && row < n) {
      const double r = b[row] - acc;
      rr += r * r;
      bb += b[row] * b[row];
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, off);
    bb += __shfl_xor_sync(0xffffffffu, bb, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sm_r[w] = rr;
    sm_b[w] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0, tb = 0;
    for (int i = 0; i < kResBlock / 32; ++i) {
      tr += sm_r[i];
      tb += sm_b[i];
    }
    partial[2 * blockIdx.x] = tr;
    partial[2 * blockIdx.x + 1] = tb;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tr = 0, tb = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    tr += ((volatile double*)partial)[2 * i];
    tb += ((volatile double*)partial)[2 * i + 1];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, off);
    tb += __shfl_xor_sync(0xffffffffu, tb, off);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sm_r[w] = tr;
    sm_b[w] = tb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, c = 0;
    for (int i = 0; i < kResBlock / 32; ++i) {
      a += sm_r[i];
      c += sm_b[i];
    }
    out[0] = sqrt(a);
    out[1] = sqrt(c);
    *counter = 0;
  }
}

unsigned resid_grid(int64_t n) {
  int64_t g = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

}  // namespace fs

using namespace fs;

extern "C" int fs_csr_residual_norm(int64_t n, const int64_t* rowptr, const int32_t* col,
                                    const double* val, const double* x, const double* b,
                                    double* out2, void* stream) {
  if (n < 1 || !rowptr || !col || !val || !x || !b || !out2) {
    set_error("fs_csr_residual_norm: null pointer or n < 1");
    return FS_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = resid_grid(n);
  // scratch: 2 partial sums per block, the ticket counter and the 2 results
  const size_t bytes = sizeof(double) * (2 * (size_t)grid + 2) + 256;
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, bytes, s);
  if (e != cudaSuccess) {
    set_error(std::string("fs_csr_residual_norm: cudaMallocAsync: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FS_ERR_OOM : FS_ERR_CUDA;
  }
  double* partial = (double*)scratch;
  double* out = partial + 2 * (size_t)grid;
  unsigned* counter = (unsigned*)(out + 2);
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    k_csr_resid<<<grid, kResBlock, 0, s>>>(n, rowptr, col, val, x, b, partial, counter, out);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out2, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaError_t ef = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("fs_csr_residual_norm: ") + cudaGetErrorString(e));
    return FS_ERR_CUDA;
  }
  return FS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the same check.
//
// Some callers cannot allocate device memory when they want to check a
// solution: a serving process whose device memory is already committed to
// resident problems under a fixed budget, or a host application that does
// not let libraries grow their device footprint after start-up.  This entry point
// runs the same kernel with its scratch (per-block partial sums, the ticket
// counter and the two results) in a fixed array of the library's static
// device memory instead: kNoAllocBlocks blocks of 512 rows each, so systems
// of at most kNoAllocMaxRows rows.  Every GPU that loads the library holds
// the array (about 128 KB) until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace fs {
namespace {

constexpr int kNoAllocBlocks = 8192;
constexpr int64_t kNoAllocRowsPerBlock = 512;
constexpr int64_t kNoAllocMaxRows = kNoAllocBlocks * kNoAllocRowsPerBlock;  // 4,194,304

// [0, 2*kNoAllocBlocks): partial sums; then the 2 results; then the counter
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocBlocks + 4];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};  // device address of the array, per device

}  // namespace
}  // namespace fs

extern "C" int fs_csr_residual_norm_noalloc(int64_t n, const int64_t* rowptr,
                                            const int32_t* col, const double* val,
                                            const double* x, const double* b, double* out2,
                                            void* stream) {
  if (n < 1 || !rowptr || !col || !val || !x || !b || !out2) {
    set_error("fs_csr_residual_norm_noalloc: null pointer or n < 1");
    return FS_ERR_INVALID_ARG;
  }
  if (n > kNoAllocMaxRows) {
    set_error("fs_csr_residual_norm_noalloc: " + std::to_string(n) +
              " rows exceed the limit of its static scratch (" +
              std::to_string(kNoAllocMaxRows) + " rows); use fs_csr_residual_norm");
    return FS_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_error("fs_csr_residual_norm_noalloc: no usable current device");
    return FS_ERR_CUDA;
  }
  double* base = nullptr;
  {
    // first call on this device: resolve the array's device address with the
    // device current (the host-side name is only a stand-in)
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_error(std::string("fs_csr_residual_norm_noalloc: cudaGetSymbolAddress: ") +
                  cudaGetErrorString(e));
        return FS_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = (double*)p;
    }
    base = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((n + kNoAllocRowsPerBlock - 1) / kNoAllocRowsPerBlock);
  double* partial = base;
  double* out = base + 2 * kNoAllocBlocks;
  unsigned* counter = (unsigned*)(base + 2 * kNoAllocBlocks + 2);
  // the array keeps the previous call's contents: the ticket counter must
  // start at zero
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    k_csr_resid<<<grid, kResBlock, 0, s>>>(n, rowptr, col, val, x, b, partial, counter, out);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out2, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("fs_csr_residual_norm_noalloc: ") + cudaGetErrorString(e));
    return FS_ERR_CUDA;
  }
  return FS_OK;
}
