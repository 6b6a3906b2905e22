// Arithmetic peaks of the GPU this library runs on, measured by its own kernels
// (the denominators of the roofline fractions the benchmark reports):
//   * FP64 and FP32 FMA throughput of the CUDA cores (the pipes the FP64 cone
//     kernels and the FP32 / FP64 factorization use): 8 independent FMA chains
//     per thread, 8 CTAs of 256 threads per SM;
//   * tcgen05 tensor-core throughput, kind::tf32 and kind::f16 (BF16 operands,
//     FP32 accumulation): one CTA per SM, one thread issuing M = 128, N = 256
//     MMAs back to back into one tensor-memory accumulator from operand tiles
//     resident in shared memory (the issue pattern of a GEMM main loop without
//     its loads), completion on an mbarrier with a bounded wait.
// Each figure is the best of `reps` launches timed with CUDA events on the
// caller's stream.  Nothing here changes a clock or any other GPU setting.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"

namespace clr {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_probe_fma(const T* __restrict__ seed, T* __restrict__ out, int iters) {
  T a[8];
  const T b = seed[0], c = seed[1];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = seed[2] + (T)(u * 0.125) + (T)(threadIdx.x * 1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(a[u], b, c);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += a[u];
  if (s == (T)12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// K-major operand tile without swizzle: core matrices of 8 rows x 16 bytes,
// (row group g, 16-byte k group h) at g * kSBO + h * kLBO; 32 bytes of K per row.
constexpr uint32_t kLBO = 128, kSBO = 256;
__device__ __forceinline__ uint64_t sdesc(uint32_t a) {
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind 0: kind::f16 with BF16 operands (K = 16 per MMA); kind 1: kind::tf32 (K = 8).
// Launched with kTcPad bytes of dynamic shared memory (unused) so that one CTA
// runs per SM.
constexpr int kTcPad = 120 * 1024;
template <int KIND>
__global__ void __launch_bounds__(128) k_probe_tc(int mmas, int* err) {
  constexpr int M = 128, N = 256;
  __shared__ __align__(1024) uint8_t sA[M * 32];
  __shared__ __align__(1024) uint8_t sB[N * 32];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, wid = tid >> 5;
  // small operand values: 1/64 in the operand's format, so the sums stay finite
  for (int i = tid; i < M * 8; i += blockDim.x)
    reinterpret_cast<uint32_t*>(sA)[i] = KIND == 0 ? 0x3C803C80u : 0x3C800000u;
  for (int i = tid; i < N * 8; i += blockDim.x)
    reinterpret_cast<uint32_t*>(sB)[i] = KIND == 0 ? 0x3C803C80u : 0x3C800000u;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tslot)), "r"(N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  if (tid == 0) {
    // D F32 (bit 4); A, B format at bits 7-9 / 10-12 (BF16 = 1, TF32 = 2); K-major;
    // N >> 3 at bit 17, M >> 4 at bit 24
    constexpr uint32_t fmt = KIND == 0 ? 1u : 2u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) |
                           ((uint32_t)(M >> 4) << 24);
    const uint64_t ad = sdesc(saddr(sA)), bd = sdesc(saddr(sB));
    for (int k = 0; k < mmas; ++k) {
      const uint32_t acc = k > 0 ? 1u : 0u;
      if (KIND == 0)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&mbar)));
  }
  uint32_t done = 0;
  for (int it = 0; it < (1 << 26) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(saddr(&mbar)), "r"(0));
  }
  if (!done && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N));
}

template <typename F>
int best_ms(cudaStream_t st, int reps, F launch, float* best) {
  cudaEvent_t a, b;
  CLR_CUDA(cudaEventCreate(&a));
  CLR_CUDA(cudaEventCreate(&b));
  launch();  // warm-up
  *best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      set_cuda_error(e, "probe");
      return CLR_E_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    *best = std::min(*best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

}  // namespace
}  // namespace clr

extern "C" int clr_probe_peaks(int32_t reps, void* stream, clr_peaks* out) {
  using namespace clr;
  if (!out || reps < 1) return CLR_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int nsm = kSMs;
  int dev = 0;
  CLR_CUDA(cudaGetDevice(&dev));
  CLR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  *out = clr_peaks{};
  out->sms = nsm;
  // scratch: seeds + FMA outputs + error flag (a few MB, freed before returning)
  const int fma_blocks = 8 * nsm, fma_threads = 256;
  double* dseed = nullptr;
  float* fseed = nullptr;
  double* dout = nullptr;
  float* fout = nullptr;
  int* err = nullptr;
  CLR_CUDA(cudaMalloc(&dseed, 3 * sizeof(double)));
  CLR_CUDA(cudaMalloc(&fseed, 3 * sizeof(float)));
  CLR_CUDA(cudaMalloc(&dout, (size_t)fma_blocks * fma_threads * sizeof(double)));
  CLR_CUDA(cudaMalloc(&fout, (size_t)fma_blocks * fma_threads * sizeof(float)));
  CLR_CUDA(cudaMalloc(&err, sizeof(int)));
  const double hd[3] = {0.999999, 1e-7, 0.5};
  const float hf[3] = {0.9999f, 1e-4f, 0.5f};
  int rc = CLR_OK;
  do {
    if (cudaMemcpyAsync(dseed, hd, sizeof(hd), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(fseed, hf, sizeof(hf), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
      rc = CLR_E_CUDA;
      break;
    }
    float ms = 0.f;
    const int it64 = 4096, it32 = 65536;
    rc = best_ms(st, reps, [&] { k_probe_fma<double><<<fma_blocks, fma_threads, 0, st>>>(dseed, dout, it64); }, &ms);
    if (rc) break;
    out->fp64_fma_tflops = 2.0 * 8.0 * it64 * fma_blocks * fma_threads / (ms * 1e-3) / 1e12;
    out->fp64_ms = ms;
    rc = best_ms(st, reps, [&] { k_probe_fma<float><<<fma_blocks, fma_threads, 0, st>>>(fseed, fout, it32); }, &ms);
    if (rc) break;
    out->fp32_fma_tflops = 2.0 * 8.0 * it32 * fma_blocks * fma_threads / (ms * 1e-3) / 1e12;
    out->fp32_ms = ms;
    const int mmas = 8192;
    if (cudaFuncSetAttribute(k_probe_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcPad) != cudaSuccess ||
        cudaFuncSetAttribute(k_probe_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcPad) != cudaSuccess) {
      rc = CLR_E_CUDA;
      break;
    }
    rc = best_ms(st, reps, [&] { k_probe_tc<0><<<nsm, 128, kTcPad, st>>>(mmas, err); }, &ms);
    if (rc) break;
    out->bf16_tc_tflops = 2.0 * 128 * 256 * 16 * (double)mmas * nsm / (ms * 1e-3) / 1e12;
    out->bf16_ms = ms;
    rc = best_ms(st, reps, [&] { k_probe_tc<1><<<nsm, 128, kTcPad, st>>>(mmas, err); }, &ms);
    if (rc) break;
    out->tf32_tc_tflops = 2.0 * 128 * 256 * 8 * (double)mmas * nsm / (ms * 1e-3) / 1e12;
    out->tf32_ms = ms;
    int herr = 0;
    if (cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = CLR_E_CUDA;
      break;
    }
    out->tc_timeouts = herr;
  } while (0);
  cudaFree(dseed);
  cudaFree(fseed);
  cudaFree(dout);
  cudaFree(fout);
  cudaFree(err);
  return rc;
}
