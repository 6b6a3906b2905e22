// Large fronts: blocked LDL^T with the augmented inverse block E (see bigfront.cuh).
//
// Panel p covers pivots K = [k0, k0 + pw), k0 = 64 p.  Three launches per panel:
//   A  (one CTA per front): LDL^T of the pw x pw diagonal block (one barrier per
//      pivot, bfdiag.cuh), its pivots, and Linv = L_KK^{-1};
//   B  L_IK = F_IK L_KK^{-T} D_K^{-1} for the rows I below K, as the product
//      F_IK Linv^T scaled by D^{-1}; the same launch finalises the E rows of
//      this panel: E_KC <- Linv E_KC (C < K) and E_KK = Linv;
//   C  64 x 64 tiles: trailing update F_IJ -= L_IK D_K L_JK^T (I >= J below K)
//      and the augmented rows E_IC -= L_IK E_KC for C <= K.
// After the last panel E = L^{-1} [I; 0].  Forward solve: y = E_top w1,
// u = w2 + E_bottom w1; backward: x1 = E^T [D^{-1} y; x2].
#include <cuda_bf16.h>

#include <type_traits>

#include "bfdiag.cuh"
#include "bigfront.cuh"

namespace clr {

namespace {
constexpr int NB = kBfNB;
constexpr int LD = NB + 1;

__device__ __forceinline__ void locate(const WorkList& wl, int64_t bid, int64_t* b, int64_t* q) {
  int64_t lo = 0, hi = wl.nfront - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (wl.pref[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  *b = wl.front[lo];
  *q = bid - wl.pref[lo];
}

template <typename T>
__device__ __forceinline__ T reg_pivot(T d, int sgn, T eps, T delta, bool* hit) {
  if ((T)sgn * d <= eps) {
    *hit = true;
    return (T)sgn * delta;
  }
  *hit = false;
  return d;
}
}  // namespace

// ------------------------------------------------------------------ A: diagonal block

// Diagonal block of panel p (one CTA per front): LDL^T with dynamic
// regularisation and Linv = L_KK^{-1} (bfdiag.cuh).  Outputs: L (unit lower, d
// on the diagonal) into the front, pivots to Dp, Linv (64 x 64, column-major,
// zero padded) into the front's slot of the panel's parity.
template <typename T>
__global__ void __launch_bounds__(256) k_bf_diag(BigFrontDev bf, WorkList wl, int p, T* __restrict__ F,
                                                 T* __restrict__ Dp, T* __restrict__ Linv,
                                                 const int8_t* __restrict__ dsign, double eps_d, double delta_d,
                                                 int* hits, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ DiagScratch<T> sh;
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b], k0 = (int64_t)p * NB;
  const int pw = (int)min((int64_t)NB, c - k0);
  const int64_t kp = bf.k0pos[b] + k0;
  T* LB = Linv + (b * 2 + (p & 1)) * (int64_t)(NB * NB);
  const int nhit = bf_diag_block<T>(F + bf.goff[b] + k0 + k0 * f, f, pw, Dp + kp, LB, NB, true, dsign + kp,
                                    (T)eps_d, (T)delta_d, reinterpret_cast<T*>(smraw), sh);
  if (threadIdx.x == 0 && nhit) atomicAdd(hits, nhit);
}

// ------------------------------------------------------------------ B: panel rows + E finalisation
// CTAs q < trsm blocks: rows r0 .. r0+63 below the panel, L_IK = F_IK Linv^T D^{-1}
// (each thread 4 x 4 outputs).  The remaining p + 1 CTAs finalise the E rows of
// this panel: E_KC <- Linv E_KC for the column blocks C < K (all their updates
// from earlier panels are in), E_KK = Linv.
template <typename T>
__global__ void __launch_bounds__(256) k_bf_trsm(BigFrontDev bf, WorkList wl, int p, T* __restrict__ F,
                                                 T* __restrict__ E, const T* __restrict__ Dp,
                                                 const T* __restrict__ Linv, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ls = reinterpret_cast<T*>(smraw);  // NB x LD
  T* Xs = Ls + NB * LD;                 // NB x LD
  __shared__ T dl[NB];
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b];
  const int tid = threadIdx.x;
  const int64_t ntr = bf_trsm_blocks(f, c, p);
  const int64_t k0 = (int64_t)p * NB;
  const int pw = (int)min((int64_t)NB, c - k0);
  const T* LB = Linv + (b * 2 + (p & 1)) * (int64_t)(NB * NB);
  if (q < ntr) {
    T* G = F + bf.goff[b];
    const int64_t r0 = k0 + pw + (int64_t)kTrsmRows * q;
    const int nr = (int)min((int64_t)kTrsmRows, f - r0);
#pragma unroll 8
    for (int idx = tid; idx < NB * NB; idx += 256) {
      const int i = idx % NB, j = idx / NB;
      Ls[i * LD + j] = LB[i + j * NB];
      Xs[i * LD + j] = (i < nr && j < pw) ? G[(r0 + i) + (k0 + j) * f] : (T)0;
    }
    for (int j = tid; j < pw; j += blockDim.x) dl[j] = Dp[bf.k0pos[b] + k0 + j];
    __syncthreads();
    const int tr = tid % 16, tc = tid / 16;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
    for (int l = 0; l < pw; ++l) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Xs[(tr + 16 * a) * LD + l];
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) bv[bb] = Ls[(tc + 16 * bb) * LD + l];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
    }
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int j = tc + 16 * bb;
      if (j >= pw) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = tr + 16 * a;
        if (i < nr) G[(r0 + i) + (k0 + j) * f] = acc[a][bb] / dl[j];
      }
    }
    return;
  }
  const int64_t e = q - ntr;
  T* Eb = E + bf.eoff[b];
  if (e < p) {
    const int64_t cb = e * NB;
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      const int i = idx % NB, j = idx / NB;
      Ls[i * LD + j] = LB[i + j * NB];
      Xs[i * LD + j] = (i < pw) ? Eb[(k0 + i) + (cb + j) * f] : (T)0;
    }
    __syncthreads();
    for (int idx = tid; idx < pw * NB; idx += blockDim.x) {
      const int i = idx % pw, j = idx / pw;
      T acc = (T)0;
      for (int l = 0; l <= i; ++l) acc += Ls[i * LD + l] * Xs[l * LD + j];
      Eb[(k0 + i) + (cb + j) * f] = acc;
    }
  } else {
    for (int idx = tid; idx < pw * pw; idx += blockDim.x) {
      const int i = idx % pw, j = idx / pw;
      if (i >= j) Eb[(k0 + i) + (k0 + j) * f] = LB[i + j * NB];
    }
  }
}

// ------------------------------------------------------------------ C: trailing and E tiles
// 64 x 64 output tiles, 256 threads, 4 x 4 outputs per thread; operands staged
// K-major in shared memory (for each k the 64 rows / columns contiguous) and
// read as 4-element vectors.  The 4-element units of a K-row are XOR-swizzled
// by the row's k so that the column-wise staging of E_KC does not hit one bank.
//   trailing tile (I >= J below K): F_IJ -= L_IK (D_K L_JK^T)
//   E tile (rows I below K, column block C <= K): E_IC -= L_IK E_KC, with the
//   E rows of K already finalised by this panel's B launch (E_KK = Linv).
constexpr int LDK = NB + 4;  // 16-byte aligned rows of the K-major tiles

template <typename T>
__device__ __forceinline__ int swz(int k, int r) {  // element r of K-row k: 4-element units swizzled by k
  return k * LDK + (((r >> 2) ^ (k & 7)) << 2) + (r & 3);
}
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

template <typename T>
__global__ void __launch_bounds__(256) k_bf_update(BigFrontDev bf, WorkList wl, int p, T* __restrict__ F,
                                                   T* __restrict__ E, const T* __restrict__ Dp, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ak = reinterpret_cast<T*>(smraw);  // [k][row], swizzled chunks
  T* Bk = Ak + NB * LDK;                 // [k][col], swizzled chunks
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b], k0 = (int64_t)p * NB;
  const int pw = (int)min((int64_t)NB, c - k0);
  const int64_t t0 = k0 + pw;
  const int64_t nt = (f - t0 + NB - 1) / NB;
  const int64_t na = nt * (nt + 1) / 2;
  T* G = F + bf.goff[b];
  const T* Dk = Dp + bf.k0pos[b] + k0;
  const int tid = threadIdx.x;
  const bool etile = q >= na;
  int64_t i0, j0 = 0, colbase = 0;
  int ncols = NB;
  T* Eb = E + bf.eoff[b];
  if (!etile) {
    int64_t bi = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) / 2.0);
    while (bi * (bi + 1) / 2 > q) --bi;
    while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
    const int64_t bj = q - bi * (bi + 1) / 2;
    i0 = t0 + bi * NB;
    j0 = t0 + bj * NB;
#pragma unroll 8
    for (int idx = tid; idx < NB * NB; idx += 256) {
      const int r = idx % NB, k = idx / NB;
      const int64_t ia = i0 + r, ib = j0 + r;
      Ak[swz<T>(k, r)] = (k < pw && ia < f) ? G[ia + (k0 + k) * f] : (T)0;
      Bk[swz<T>(k, r)] = (k < pw && ib < f) ? G[ib + (k0 + k) * f] * Dk[k] : (T)0;
    }
  } else {
    const int64_t e = q - na;
    const int64_t bi = e / (p + 1), cb = e % (p + 1);
    i0 = t0 + bi * NB;
    colbase = cb * NB;
    if (cb == p) ncols = pw;
#pragma unroll 8
    for (int idx = tid; idx < NB * NB; idx += 256) {
      const int r = idx % NB, k = idx / NB;
      const int64_t ia = i0 + r;
      Ak[swz<T>(k, r)] = (k < pw && ia < f) ? G[ia + (k0 + k) * f] : (T)0;
      // E_KC: consecutive threads read consecutive rows k0 + kk of column colbase + cc
      const int kk = idx % NB, cc = idx / NB;
      Bk[swz<T>(kk, cc)] = (kk < pw && cc < ncols) ? Eb[(k0 + kk) + (colbase + cc) * f] : (T)0;
    }
  }
  __syncthreads();
  const int tr = tid % 16, tc = tid / 16;  // rows 4 tr .. 4 tr + 3, columns 4 tc .. 4 tc + 3
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  for (int k = 0; k < pw; ++k) {
    T av[4], bv[4];
    ld4<T>(Ak + swz<T>(k, 4 * tr), av);
    ld4<T>(Bk + swz<T>(k, 4 * tc), bv);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
  if (!etile) {
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int64_t j = j0 + 4 * tc + bb;
      if (j >= f) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + 4 * tr + a;
        if (i < f && i >= j) G[i + j * f] -= acc[a][bb];
      }
    }
  } else {
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int cc = 4 * tc + bb;
      if (cc >= ncols) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + 4 * tr + a;
        if (i < f) Eb[i + (colbase + cc) * f] -= acc[a][bb];
      }
    }
  }
}

// ------------------------------------------------------------------ C on the tensor cores
// The same updates as k_bf_update with 16-bit products: 128 x 64 output tiles,
// each FP32 operand split into two BF16 parts (hi = bf16(v), lo = bf16(v - hi))
// and the product formed as hi*hi + hi*lo + lo*hi (the lo*lo term, ~2^-16
// relative, is dropped), accumulated in FP32 in tensor memory by tcgen05.mma
// kind::f16 (M = 128, N = 64, K = 16, 12 instructions per panel).  Operands are
// staged K-major in shared memory as 8-row x 16-byte core matrices (no
// swizzle; core matrix (row group g, k group h) at g * 1024 + h * 128 bytes).
// One thread issues the MMAs; completion is signalled on an mbarrier whose
// wait is bounded (on time-out the tile is skipped and *err set).
namespace {
constexpr uint32_t kTcLBO = 128, kTcSBO = 1024;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((kTcLBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kTcSBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}
__device__ __forceinline__ uint32_t tc_off(int r, int k) {  // byte offset of element (r, k) of a 16-bit tile
  return (uint32_t)((r >> 3) * kTcSBO + (k >> 3) * kTcLBO + (r & 7) * 16 + (k & 7) * 2);
}
// v = hi + lo + O(2^-16 |v|), hi and lo BF16 (round to nearest)
__device__ __forceinline__ void split_bf16(float v, uint16_t* hi, uint16_t* lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  *hi = *reinterpret_cast<const uint16_t*>(&h);
  *lo = *reinterpret_cast<const uint16_t*>(&l);
}
constexpr int kTcA = 128 * kBfNB * 2, kTcB = 64 * kBfNB * 2;  // bytes of one BF16 operand tile
constexpr size_t kTcSmem = 2 * (size_t)kTcA + 2 * (size_t)kTcB + 1024;  // hi and lo of A and B, alignment slack
}  // namespace

__global__ void __launch_bounds__(128) k_bf_update_tc(BigFrontDev bf, WorkList wl, int p, float* __restrict__ F,
                                                      float* __restrict__ E, const float* __restrict__ Dp, int* err,
                                                      const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) uint8_t tcraw[];
  // operand tiles from a 1024-byte aligned base: A hi, A lo, B hi, B lo
  uint8_t* sA = tcraw + ((1024 - (smem_addr(tcraw) & 1023)) & 1023);
  uint8_t* sAl = sA + kTcA;
  uint8_t* sB = sAl + kTcA;
  uint8_t* sBl = sB + kTcB;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b], k0 = (int64_t)p * NB;
  const int pw = (int)min((int64_t)NB, c - k0);
  const int64_t t0 = k0 + pw, nr = f - t0;
  const int64_t n128 = (nr + 127) / 128, n64 = (nr + 63) / 64;
  float* G = F + bf.goff[b];
  float* Eb = E + bf.eoff[b];
  const float* Dk = Dp + bf.k0pos[b] + k0;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  bool etile = true;
  int64_t bi = 0, bj = 0;
  for (int64_t j = 0; j < n64; ++j) {
    const int64_t cnt = n128 - j / 2;
    if (q < cnt) {
      bi = j / 2 + q;
      bj = j;
      etile = false;
      break;
    }
    q -= cnt;
  }
  int64_t cb = 0;
  if (etile) {
    bi = q / (p + 1);
    cb = q % (p + 1);
  }
  const int64_t i0 = t0 + 128 * bi;
  const int64_t j0 = etile ? cb * NB : t0 + 64 * bj;  // first output column
  const int ncols = etile ? (cb == p ? pw : NB) : (int)min((int64_t)64, f - j0);
  // stage A = L rows i0 .. i0+127 of the panel, B = D L rows j0.. (trailing) or E_KC (E tile)
  for (int e = tid; e < 128 * NB; e += blockDim.x) {
    const int r = e % 128, k = e / 128;
    const int64_t i = i0 + r;
    const float v = (k < pw && i < f) ? G[i + (k0 + k) * f] : 0.f;
    split_bf16(v, reinterpret_cast<uint16_t*>(sA + tc_off(r, k)), reinterpret_cast<uint16_t*>(sAl + tc_off(r, k)));
  }
  if (!etile) {
    for (int e = tid; e < 64 * NB; e += blockDim.x) {
      const int r = e % 64, k = e / 64;
      const int64_t j = j0 + r;
      const float v = (k < pw && j < f) ? G[j + (k0 + k) * f] * Dk[k] : 0.f;
      split_bf16(v, reinterpret_cast<uint16_t*>(sB + tc_off(r, k)), reinterpret_cast<uint16_t*>(sBl + tc_off(r, k)));
    }
  } else {
    for (int e = tid; e < 64 * NB; e += blockDim.x) {
      const int k = e % 64, r = e / 64;  // consecutive k: consecutive rows of E
      const float v = (k < pw && r < ncols) ? Eb[(k0 + k) + (j0 + r) * f] : 0.f;
      split_bf16(v, reinterpret_cast<uint16_t*>(sB + tc_off(r, k)), reinterpret_cast<uint16_t*>(sBl + tc_off(r, k)));
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(64));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    // D F32 (bit 4), A and B BF16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at 17, M >> 4 at 24
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint8_t* As[3] = {sA, sA, sAl};
    const uint8_t* Bs[3] = {sB, sBl, sB};
    for (int ks = 0; ks < NB / 16; ++ks)
      for (int t = 0; t < 3; ++t) {  // hi*hi, hi*lo, lo*hi
        const uint64_t ad = tc_desc(smem_addr(As[t]) + ks * 2 * kTcLBO);
        const uint64_t bd = tc_desc(smem_addr(Bs[t]) + ks * 2 * kTcLBO);
        const uint32_t acc = (ks > 0 || t > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_addr(&mbar)));
  }
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(&mbar)), "r"(0));
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!done) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    const int64_t i = i0 + 32 * wid + lane;
    for (int cc = 0; cc < 64; cc += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * wid) << 16) + (uint32_t)cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (i < f) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int col = cc + jj;
          if (col >= ncols) continue;
          const int64_t j = j0 + col;
          if (!etile) {
            if (i >= j) G[i + j * f] -= __uint_as_float(v[jj]);
          } else {
            Eb[i + j * f] -= __uint_as_float(v[jj]);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
}

// ------------------------------------------------------------------ solves
// Forward: rows r0 .. r0+31 of z = E w1; 16 warps split the columns, 8 columns in
// flight per lane, partial sums reduced in a fixed order.  Rows < c store
// v = y / D (what the backward sweep needs), rows >= c update w2.
template <typename T>
__global__ void k_bf_fwd(BigFrontDev bf, WorkList wl, const T* __restrict__ E, const T* __restrict__ Dp,
                         T* __restrict__ w, T* __restrict__ ybuf, const int* skip) {
  if (skip && *skip) return;
  __shared__ T red[16][33];
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b];
  const int64_t r0 = 32 * q;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* Eb = E + bf.eoff[b];
  const T* w1 = w + bf.woff[b];
  const int64_t i = r0 + lane;
  const int64_t jmax = min(c, r0 + 32);
  T a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = (T)0;
  if (i < f) {
    int64_t j = wid;
    for (; j + 15 * 8 < jmax; j += 16 * 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] += Eb[i + (j + 16 * u) * f] * w1[j + 16 * u];
    }
    for (; j < jmax; j += 16) a[0] += Eb[i + j * f] * w1[j];
  }
  T acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  red[wid][lane] = acc;
  __syncthreads();
  if (wid == 0 && i < f) {
    T z = (T)0;
    for (int k = 0; k < 16; ++k) z += red[k][lane];
    if (i < c) ybuf[bf.yoff[b] + i] = z / Dp[bf.k0pos[b] + i];
    else w[bf.woff[b] + i] += z;
  }
}

// Backward: x_j = sum_{i >= j} E[i, j] v_i, v = [y / D; x2]; one warp per column.
template <typename T>
__global__ void k_bf_bwd(BigFrontDev bf, WorkList wl, const T* __restrict__ E, const T* __restrict__ ybuf,
                         T* __restrict__ xs, const int32_t* __restrict__ rows_kkt, const int* skip) {
  if (skip && *skip) return;
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t j = 8 * q + wid;
  if (j >= c) return;
  const T* Ec = E + bf.eoff[b] + j * f;
  const T* v = ybuf + bf.yoff[b];
  const int32_t* rk = rows_kkt + bf.rk[b];
  T a[4] = {(T)0, (T)0, (T)0, (T)0};
  const int64_t iend = min(f, c);
  int64_t i = j + lane;
  for (; i + 96 < iend; i += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] += Ec[i + 32 * u] * v[i + 32 * u];
  }
  for (; i < iend; i += 32) a[0] += Ec[i] * v[i];
  for (i = max(j, c) + lane; i < f; i += 32) a[1] += Ec[i] * xs[rk[i]];
  T acc = (a[0] + a[1]) + (a[2] + a[3]);
  acc = warp_sum(acc);
  if (lane == 0) xs[rk[j]] = acc;
}

// ------------------------------------------------------------------ host

template <typename T>
int BigFrontOps<T>::setup_attributes() {
  CLR_CUDA(cudaFuncSetAttribute(k_bf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDiagSmem * sizeof(T)));
  CLR_CUDA(cudaFuncSetAttribute(k_bf_trsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * NB * LD * sizeof(T)));
  CLR_CUDA(cudaFuncSetAttribute(k_bf_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * NB * LDK * sizeof(T)));
  if (std::is_same<T, float>::value)
    CLR_CUDA(cudaFuncSetAttribute(k_bf_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  return CLR_OK;
}

template <typename T>
int BigFrontOps<T>::factor_level(cudaStream_t st, const BigFrontDev& bf, const BigLevelPlan& plan, T* F, T* E, T* Dp,
                                 T* Linv, const int8_t* dsign, double eps, double delta, int* hits, const int* skip,
                                 bool tc16, int* err) {
  const size_t s2 = 2 * NB * LD * sizeof(T), su = 2 * NB * LDK * sizeof(T);
  for (size_t p = 0; p < plan.A.size(); ++p) {
    if (plan.A[p].nblocks > 0)
      k_bf_diag<T><<<(unsigned)plan.A[p].nblocks, 256, kDiagSmem * sizeof(T), st>>>(bf, plan.A[p], (int)p, F, Dp, Linv,
                                                                                  dsign, eps, delta, hits, skip);
    if (plan.B[p].nblocks > 0)
      k_bf_trsm<T><<<(unsigned)plan.B[p].nblocks, 256, s2, st>>>(bf, plan.B[p], (int)p, F, E, Dp, Linv, skip);
    if constexpr (std::is_same<T, float>::value) {
      if (tc16) {
        if (plan.Ctc[p].nblocks > 0)
          k_bf_update_tc<<<(unsigned)plan.Ctc[p].nblocks, 128, kTcSmem, st>>>(bf, plan.Ctc[p], (int)p, F, E, Dp, err,
                                                                          skip);
        continue;
      }
    }
    if (plan.C[p].nblocks > 0)
      k_bf_update<T><<<(unsigned)plan.C[p].nblocks, 256, su, st>>>(bf, plan.C[p], (int)p, F, E, Dp, skip);
  }
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

template <typename T>
int BigFrontOps<T>::fwd(cudaStream_t st, const BigFrontDev& bf, const WorkList& wl, const T* E, const T* Dp, T* w,
                        T* ybuf, const int* skip) {
  if (wl.nblocks == 0) return CLR_OK;
  k_bf_fwd<T><<<(unsigned)wl.nblocks, 512, 0, st>>>(bf, wl, E, Dp, w, ybuf, skip);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

template <typename T>
int BigFrontOps<T>::bwd(cudaStream_t st, const BigFrontDev& bf, const WorkList& wl, const T* E, const T* Dp,
                        const T* ybuf, T* xs, const int32_t* rows_kkt, const int* skip) {
  if (wl.nblocks == 0) return CLR_OK;
  k_bf_bwd<T><<<(unsigned)wl.nblocks, 256, 0, st>>>(bf, wl, E, ybuf, xs, rows_kkt, skip);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

template struct BigFrontOps<double>;
template struct BigFrontOps<float>;

}  // namespace clr
