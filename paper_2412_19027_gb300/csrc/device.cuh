// Device-side helpers shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/clr.h"

namespace clr {

constexpr int kSMs = 152;          // GB300: 2 dies x 76 SMs
constexpr int kRedBlocks = 2 * kSMs;  // fixed grid of every reduction kernel (deterministic partials)
constexpr int kRedThreads = 256;

// Records the first CUDA error of the calling host thread.
void set_cuda_error(cudaError_t e, const char* where);
#define CLR_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      clr::set_cuda_error(e_, #call);                    \
      return CLR_E_CUDA;                                 \
    }                                                    \
  } while (0)
#define CLR_CHECK_LAUNCH()                               \
  do {                                                   \
    cudaError_t e_ = cudaGetLastError();                 \
    if (e_ != cudaSuccess) {                             \
      clr::set_cuda_error(e_, __FILE__);                 \
      return CLR_E_CUDA;                                 \
    }                                                    \
  } while (0)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reductions in a fixed order (warp shuffles, then warp 0 over the
// per-warp values), result valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : -INFINITY;
  if (wid == 0) v = warp_max(v);
  return v;
}
__device__ __forceinline__ double block_min(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_min(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : INFINITY;
  if (wid == 0) v = warp_min(v);
  return v;
}

inline int grid_for(int64_t n, int threads, int cap = 8 * kSMs) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Device memory owned by a solver, released together.
class DeviceArena {
 public:
  ~DeviceArena() { release(); }
  void* alloc(size_t bytes);
  template <typename T>
  T* alloc_n(int64_t n) {
    return static_cast<T*>(alloc(sizeof(T) * (size_t)(n > 0 ? n : 1)));
  }
  template <typename T>
  T* upload(const T* h, int64_t n) {
    T* d = alloc_n<T>(n);
    if (!d || n <= 0) return d;
    const cudaError_t e = async_ ? cudaMemcpyAsync(d, h, sizeof(T) * (size_t)n, cudaMemcpyHostToDevice, async_)
                                 : cudaMemcpy(d, h, sizeof(T) * (size_t)n, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? d : nullptr;
  }
  void release();
  size_t bytes() const { return total_; }
  // Stream-ordered mode: allocations and frees go through cudaMallocAsync /
  // cudaFreeAsync on `s` and uploads are ordered on it, so that a solver built
  // and torn down while other solvers run does not synchronise the device.
  // Only without a user allocator hook; set before the first allocation.
  void set_stream_ordered(cudaStream_t s) { async_ = s; }

 private:
  struct Block {
    void* p;
    size_t n;
  };
  Block* blocks_ = nullptr;
  size_t nblocks_ = 0, cap_ = 0, total_ = 0;
  cudaStream_t async_ = nullptr;
};

// Pinned host buffers reused across solvers (cudaMallocHost / cudaFreeHost
// synchronise the device; a serving loop creates and drops solvers while
// others run).  Blocks are kept for the life of the process.
void* pinned_get(size_t bytes);
void pinned_put(void* p, size_t bytes);

}  // namespace clr
