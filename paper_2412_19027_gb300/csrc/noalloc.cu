// Allocation-free dense LDL^T factor-and-solve for small quasi-definite systems.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code that runs while a CUDA graph is being captured (cudaMalloc is
// not allowed there), real-time control loops that must not allocate after
// start-up (for example a model-predictive controller that solves one small
// KKT system per control period), and plug-ins whose device memory is owned
// and budgeted by a host framework.  This entry point takes only caller-owned
// device buffers and keeps its working matrix in one fixed, file-scope device
// array, so it never calls cudaMalloc or cudaFree.
//
// It is the small-front factorization of the solver (one CTA, right-looking
// LDL^T with the dynamic-regularisation rule) applied to a whole dense matrix,
// followed by the forward, diagonal and backward solves.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/clr.h"
#include "device.cuh"

namespace clr {

constexpr int kNoAllocMaxN = CLR_NOALLOC_MAX_N;

// Working matrix (column-major N x N, lower triangle used) shared by every call
// on a device; held by each GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_work[kNoAllocMaxN * kNoAllocMaxN];

// The caller's buffers carry no __restrict__: rhs and x may be the same buffer
// (an in-place solve reads every rhs entry into x before anything else is written).
__global__ void k_noalloc_ldl(double* __restrict__ W, const double* K, const double* signs, int N, const double* rhs,
                              double* x, double* D, double eps, double delta, int* hits) {
  __shared__ double dsh;
  __shared__ int nhit;
  const int tid = threadIdx.x;
  if (tid == 0) nhit = 0;
  for (int q = tid; q < N * N; q += blockDim.x) W[q] = K[q];
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      double d = W[k + k * N];
      const double sg = signs[k] > 0 ? 1.0 : -1.0;
      if (sg * d <= eps) {
        d = sg * delta;
        ++nhit;
      }
      W[k + k * N] = d;
      dsh = d;
    }
    __syncthreads();
    const double inv = 1.0 / dsh;
    const int m = N - k - 1;
    for (int q = tid; q < m * m; q += blockDim.x) {
      const int i = k + 1 + q % m, j = k + 1 + q / m;
      if (i >= j) W[i + j * N] -= W[i + k * N] * W[j + k * N] * inv;
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < N; i += blockDim.x) W[i + k * N] *= inv;
    __syncthreads();
  }
  // L y = rhs, then y /= D, then L^T x = y (x holds y in place)
  for (int i = tid; i < N; i += blockDim.x) x[i] = rhs[i];
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    const double yk = x[k];
    for (int i = k + 1 + tid; i < N; i += blockDim.x) x[i] -= W[i + k * N] * yk;
    __syncthreads();
  }
  for (int i = tid; i < N; i += blockDim.x) {
    x[i] /= W[i + i * N];
    if (D) D[i] = W[i + i * N];
  }
  __syncthreads();
  for (int k = N - 1; k >= 0; --k) {
    if (tid < 32) {
      double s = 0.0;
      for (int i = k + 1 + tid; i < N; i += 32) s += W[i + k * N] * x[i];
      s = warp_sum(s);
      if (tid == 0) x[k] -= s;
    }
    __syncthreads();
  }
  if (tid == 0 && hits) *hits = nhit;
}

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};  // device address of g_noalloc_work, per device ordinal
}  // namespace

}  // namespace clr

extern "C" int clr_dense_ldl_solve_noalloc(const double* K, const double* signs, int32_t N, const double* rhs,
                                           double* x, double* D, double dyn_reg_eps, double dyn_reg_delta,
                                           int32_t* dyn_hits, void* stream) {
  using namespace clr;
  if (N < 0 || !K || !signs || !rhs || !x) return CLR_E_INVALID;
  if (N > kNoAllocMaxN) return CLR_E_UNSUPPORTED;
  if (N == 0) return CLR_OK;
  int dev = 0;
  CLR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return CLR_E_UNSUPPORTED;
  double* work = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // first call on this device: resolve the device address of the static array
      // (must happen outside stream capture; see include/clr.h)
      CLR_CUDA(cudaGetSymbolAddress((void**)&g_noalloc_ptr[dev], g_noalloc_work));
    }
    work = g_noalloc_ptr[dev];
  }
  k_noalloc_ldl<<<1, 256, 0, (cudaStream_t)stream>>>(work, K, signs, N, rhs, x, D, dyn_reg_eps, dyn_reg_delta,
                                                      dyn_hits);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}
