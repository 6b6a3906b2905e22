// Dataflow factorization of the big fronts of one level: one persistent launch
// in which CTAs take 64 x 64 tile tasks from a counter in a topological order
// of the task graph and wait (bounded) for the version words of the tiles they
// read.  The arithmetic of each task is that of the per-panel kernels
// (bigfront.cu); only the scheduling differs: the diagonal block of panel p + 1
// starts as soon as its own tile has received panel p's update, while the rest
// of panel p's updates are still running.
//
// FP32 factor, tensor-core variant (TC): the producers of L and E_KC tiles also
// store them as packed FP32 operand tiles (bigfront.cuh, FlowTc); the U and EU
// tasks load their two operand tiles with one TMA tensor copy each
// (cp.async.bulk.tensor, completion on an mbarrier), split them in shared
// memory into high and low TF32 parts and issue 16 tcgen05.mma kind::tf32
// (M = 128, N = 64, K = 8) into a 128 x 64 FP32 accumulator in tensor memory:
// A = [L_hi; L_lo] (128 rows), B = the high then the low part of the other
// operand, so that lanes 0-63 hold L_hi B and lanes 64-127 L_lo B; their sum is
// the FP32 product to ~2^-21 relative (every partial product of two TF32 parts
// is exact in FP32).
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "bfdiag.cuh"
#include "bigfront.cuh"

namespace clr {
namespace {
constexpr int NB = kBfNB;
constexpr int LD = NB + 1;   // odd stride: column accesses free of bank conflicts
constexpr int LDK = NB + 4;  // 16-byte aligned rows of the K-major operand tiles
constexpr int NT = kFlowThreads;
constexpr uint32_t kSpin = 1u << 21;  // polls of one wait (about 2 s) before it gives up

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait until *p >= v.  False if the wait ran out (err := 2) or another
// CTA has given up (err != 0).
__device__ bool wait_ge(const int* p, int v, int* err) {
  for (uint32_t it = 0; it < kSpin; ++it) {
    if (ld_acquire(p) >= v) return true;
    if (it >= 16) {
      if (ld_acquire(err) != 0) return false;
      __nanosleep(64);
    }
  }
  atomicExch(err, 2);
  return false;
}

struct Geo {
  int64_t f, c, P, nbf;
};
__device__ __forceinline__ int64_t brow0(const Geo& g, int64_t b) { return b < g.P ? NB * b : g.c + NB * (b - g.P); }
__device__ __forceinline__ int bnrow(const Geo& g, int64_t b) {
  return (int)(b < g.P ? min((int64_t)NB, g.c - NB * b) : min((int64_t)NB, g.f - g.c - NB * (b - g.P)));
}
struct Words {
  int *tile, *etile, *diag, *trsm, *pe, *txc, *uxc;
  int64_t P;
  __device__ int* t(int64_t i, int64_t j) const { return tile + i * (i + 1) / 2 + j; }
  __device__ int* e(int64_t i, int64_t c) const { return etile + i * P + c; }
};
__device__ __forceinline__ Words words_of(int* base, const Geo& g) {
  Words w;
  w.P = g.P;
  w.tile = base;
  w.etile = base + g.nbf * (g.nbf + 1) / 2;
  w.diag = w.etile + g.nbf * g.P;
  w.trsm = w.diag + g.P;
  w.pe = w.trsm + g.nbf;
  w.txc = w.pe + g.P;
  w.uxc = w.txc + g.P;
  return w;
}

// element r of K-row k of a K-major operand tile: 4-element units XOR-swizzled by k
__device__ __forceinline__ int swz(int k, int r) { return k * LDK + (((r >> 2) ^ (k & 7)) << 2) + (r & 3); }
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

// ---------------------------------------------------------------- tensor-core helpers
// Packed FP32 operand tile (global memory, and the TMA staging copy): element
// (row, k) at word (k / 4) * 256 + row * 4 + k % 4.  The split operand the MMA
// reads: 128 rows (0-63 the high TF32 parts, 64-127 the low parts), element
// (row, k) at word (k / 4) * 512 + row * 4 + k % 4 -- K-major core matrices of 8
// rows x 16 bytes, adjacent in K 2048 bytes apart and in rows 128 bytes apart.
__device__ __forceinline__ int pk_word(int row, int k) { return ((k >> 2) << 8) + (row << 2) + (k & 3); }
// v = hi + lo + O(2^-22 |v|): hi = v with its 13 low mantissa bits cleared (a TF32
// value, so the tensor core reads it unchanged), lo = v - hi (exact) rounded to TF32.
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
  uint32_t l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(v - hi));
  lo = __uint_as_float(l);
}
// All threads: store the 64 x 64 tile val(row, k) as a packed operand tile at
// dst (each pass of the CTA writes 1 KB, contiguous).
template <typename V>
__device__ __forceinline__ void pk_write(float* dst, V val) {
#pragma unroll 4
  for (int it = 0; it < 16; ++it) {
    const int idx = threadIdx.x + NT * it;
    const int q = idx & 3, r = (idx >> 2) & 63, kg = idx >> 8;
    dst[(kg << 8) + (r << 2) + q] = val(r, 4 * kg + q);
  }
}
// All threads: split the staged packed tile src into its high and low parts in
// the MMA's layout at dst, each k-column scaled by sc[k] first (sc null: 1).
__device__ __forceinline__ void pk_split(const float* src, float* dst, const float* sc) {
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int ch = threadIdx.x + NT * it;  // 16-byte chunk (k group kg, row r)
    const int kg = ch >> 6, r = ch & 63;
    float4 v = reinterpret_cast<const float4*>(src)[ch];
    if (sc) {
      v.x *= sc[4 * kg];
      v.y *= sc[4 * kg + 1];
      v.z *= sc[4 * kg + 2];
      v.w *= sc[4 * kg + 3];
    }
    float4 h, l;
    split_tf32(v.x, h.x, l.x);
    split_tf32(v.y, h.y, l.y);
    split_tf32(v.z, h.z, l.z);
    split_tf32(v.w, h.w, l.w);
    reinterpret_cast<float4*>(dst)[kg * 128 + r] = h;
    reinterpret_cast<float4*>(dst)[kg * 128 + 64 + r] = l;
  }
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// Tile indices within a front's packed tiles: PL(p, i), i > p; PE(p, e), e <= p.
__device__ __forceinline__ int64_t pk_l(int64_t nbf, int p, int64_t i) {
  return (int64_t)p * (nbf - 1) - (int64_t)p * (p - 1) / 2 + (i - p - 1);
}
__device__ __forceinline__ int64_t pk_e(int64_t nL, int p, int64_t e) { return nL + (int64_t)p * (p + 1) / 2 + e; }
struct PkRef {  // the packed tiles of the front a task works on
  float* pk = nullptr;  // the level's tiles
  int64_t base = 0;     // first tile of the front
  int64_t nL = 0;
  __device__ float* tile(int64_t t) const { return pk + kPkWords * (base + t); }
};
__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory descriptor of a packed tile (K-major, no swizzle; LBO 2048, SBO 128 bytes)
__device__ __forceinline__ uint64_t pk_desc(uint32_t a) {
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)(2048 >> 4) << 16;
  d |= (uint64_t)(128 >> 4) << 32;
  d |= (uint64_t)1 << 46;  // tcgen05 descriptor version; base offset 0, no swizzle
  return d;
}
// bounded wait on an mbarrier phase (false: it ran out)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// one TMA tensor copy of packed tile `tile` (16 rows of 256 floats of the map) to dst
__device__ __forceinline__ void tma_tile(uint32_t dst, const CUtensorMap* map, int64_t tile, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"((int)(tile * 16)), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
constexpr int kTcOpBytes = 128 * NB * 4;   // one split operand (high and low parts, 32 KB)
constexpr int kTcPkBytes = NB * NB * 4;    // one packed FP32 tile (16 KB)
// split A, split B, staged A, staged B and the 1024-byte alignment slack
constexpr size_t kTcSmemFlow = 2 * (size_t)kTcOpBytes + 2 * (size_t)kTcPkBytes + 1024;
// M = 128, N = 64, D FP32 (bit 4), A and B TF32 (format 2 at bits 7 and 10), both K-major
constexpr uint32_t kTf32Idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) |
                                ((uint32_t)(128 >> 4) << 24);

// two consecutive rows r, r + 1 (r even) of K-row k of a K-major tile
template <typename T>
__device__ __forceinline__ void ld2(const T* p, T (&v)[2]);
template <>
__device__ __forceinline__ void ld2<float>(const float* p, float (&v)[2]) {
  const float2 a = *reinterpret_cast<const float2*>(p);
  v[0] = a.x;
  v[1] = a.y;
}
template <>
__device__ __forceinline__ void ld2<double>(const double* p, double (&v)[2]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  v[0] = a.x;
  v[1] = a.y;
}

// D(p): LDL^T of the pw x pw diagonal block with dynamic regularisation (see
// bfdiag.cuh); L and the pivots written back, Linv = L_KK^{-1} written into
// E_KK, which it equals (the zeros above its diagonal are the E pool's).
template <typename T, bool TC>
__device__ void task_diag(const BigFrontDev& bf, int64_t b, const Geo& g, int p, T* F, T* E, T* Dp,
                          const int8_t* dsign, T eps, T delta, int* hits, T* sm, DiagScratch<T>& sh, const PkRef& pkr) {
  const int64_t f = g.f, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);
  const int64_t kp = bf.k0pos[b] + k0;
  T* G = F + bf.goff[b] + k0 + k0 * f;
  T* Li = E + bf.eoff[b] + k0 + k0 * f;
  const int nhit = bf_diag_block<T>(G, f, pw, Dp + kp, Li, f, false, dsign + kp, eps, delta, sm, sh);
  if (threadIdx.x == 0 && nhit) atomicAdd(hits, nhit);
}

// DX(p), 1 <= p < P: the three links of the critical chain in one task, kept in
// shared memory between them -- the panel row T(p-1, p) (its L rows stored and
// published through the trsm word of block p as soon as they are written), the
// update of the diagonal tile (p, p) by panel p-1, and D(p).  Same arithmetic,
// in the same order, as the three separate tasks.
template <typename T, bool TC>
__device__ int task_dx(const BigFrontDev& bf, int64_t b, const Geo& g, int p, T* F, T* E, T* Dp, const int8_t* dsign,
                       T eps, T delta, T* sm, DiagScratch<T>& sh, T* dl, int* trsm_word, const PkRef& pkr) {
  T* Bk = sm;                // K-major Linv of panel p - 1 (row j, k = l); work space of the factorization afterwards
  T* Xk = sm + NB * LDK;     // K-major F_{p,p-1} (row i, k = l), then L_{p,p-1}
  T* A = sm + 2 * NB * LDK;  // the diagonal tile (p, p), lower triangle, row stride LD
  const int64_t f = g.f, kq = (int64_t)(p - 1) * NB, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);  // panel p - 1 is a full 64-column panel (p - 1 < P - 1)
  T* G = F + bf.goff[b];
  T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
  {  // all loads in one batch, then into shared memory
    T ra[16], rb[16], rc[16];
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      ra[it] = __ldcg(Eb + (kq + i) + (kq + l) * f);
      rb[it] = (i < pw) ? __ldcg(G + (k0 + i) + (kq + l) * f) : (T)0;
      rc[it] = (i < pw && l < pw && i >= l) ? __ldcg(G + (k0 + i) + (k0 + l) * f) : (T)0;
    }
    if (tid < NB) dl[tid] = __ldcg(Dp + bf.k0pos[b] + kq + tid);
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      Bk[swz(l, i)] = ra[it];
      Xk[swz(l, i)] = rb[it];
      A[i * LD + l] = rc[it];
    }
  }
  __syncthreads();
  // L_{p,p-1} = F_{p,p-1} Linv^T D^{-1} (divided by the pivots, as the separate panel-row
  // task T divides).  Linv is unit lower triangular, so column
  // block tc needs only l <= 4 tc + 3 (the terms skipped are exact zeros).  A warp
  // instruction holds an FP64 sub-partition pipe as long whatever its active lanes,
  // so the work is split evenly over the warps with one trip count per warp: warp w
  // takes column blocks w and 15 - w, each lane the rows 2 lane, 2 lane + 1.
  const int wid = tid >> 5, lane = tid & 31;
  T acc[2][2][4];
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const int tc = ph == 0 ? wid : 15 - wid;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[ph][a][bb] = (T)0;
    for (int l = 0; l < 4 * tc + 4; ++l) {
      T av[2], bv[4];
      ld2<T>(Xk + swz(l, 2 * lane), av);
      ld4<T>(Bk + swz(l, 4 * tc), bv);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) acc[ph][a][bb] += av[a] * bv[bb];
    }
  }
  __syncthreads();  // every thread has read F_{p,p-1}
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const int tc = ph == 0 ? wid : 15 - wid;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int j = 4 * tc + bb;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int i = 2 * lane + a;
        Xk[swz(j, i)] = (i < pw) ? acc[ph][a][bb] / dl[j] : (T)0;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int idx = tid; idx < NB * NB; idx += NT) {
    const int i = idx % NB, j = idx / NB;
    if (i < pw) G[(k0 + i) + (kq + j) * f] = Xk[swz(j, i)];
  }
  if constexpr (TC) {  // PL(p-1, p) before the L rows are published
    pk_write(pkr.tile(pk_l(g.nbf, p - 1, p)), [&](int r, int k) -> float { return r < pw ? (float)Xk[swz(k, r)] : 0.f; });
    fence_proxy_async_global();
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    st_release(trsm_word, p);
  }
  // A_ij -= sum_l L_il (L_jl d_l), i >= j: only the 136 4 x 4 blocks on or below
  // the diagonal, one per thread (threads 136 .. 255 idle), each summed in the
  // same order as a full-tile product would
  if (tid < 136) {
    int lr = 0;
    while ((lr + 1) * (lr + 2) / 2 <= tid) ++lr;  // block row; tid = lr (lr + 1) / 2 + lc
    const int lc = tid - lr * (lr + 1) / 2;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
    for (int l = 0; l < NB; ++l) {
      T av[4], bv[4];
      ld4<T>(Xk + swz(l, 4 * lr), av);
      ld4<T>(Xk + swz(l, 4 * lc), bv);
      const T dlv = dl[l];
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) bv[bb] *= dlv;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
    }
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int j = 4 * lc + bb;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = 4 * lr + a;
        if (i < pw && i >= j) A[i * LD + j] -= acc[a][bb];
      }
    }
  }
  __syncthreads();
  const int64_t kp = bf.k0pos[b] + k0;
  const int nhit = bf_diag_factor<T>(A, Bk, G + k0 + k0 * f, f, pw, Dp + kp, Eb + k0 + k0 * f, f, false, dsign + kp,
                                     eps, delta, sh);
  return nhit;
}

// TX(p, q), FP64 split chain: rows 16 q .. 16 q + 15 of T(p-1, p), L = F Linv^T D^{-1}
// with the products of DX(p) (thread: row tid % 16, column block tid / 16; the
// zero half of Linv skipped) -- same sums, same division.
template <typename T>
__device__ void task_tx(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int q, T* F, const T* E, const T* Dp,
                        T* sm, T* dl) {
  T* Bk = sm;             // K-major Linv of panel p - 1 (row j, k = l)
  T* Xk = sm + NB * LDK;  // K-major F rows of the part (row rr, k = l)
  const int64_t f = g.f, kq = (int64_t)(p - 1) * NB, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);  // panel p - 1 is a full 64-column panel
  const int r0 = 16 * q, nr = max(0, min(16, pw - r0));
  if (nr == 0) return;  // uniform over the CTA
  T* G = F + bf.goff[b];
  const T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
  {  // all loads in one batch, then into shared memory
    T ra[16], rx[4];
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      ra[it] = __ldcg(Eb + (kq + i) + (kq + l) * f);
    }
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int idx = tid + NT * it;
      const int rr = idx % 16, l = idx / 16;
      rx[it] = (rr < nr) ? __ldcg(G + (k0 + r0 + rr) + (kq + l) * f) : (T)0;
    }
    if (tid < NB) dl[tid] = __ldcg(Dp + bf.k0pos[b] + kq + tid);
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      Bk[swz(idx / NB, idx % NB)] = ra[it];
    }
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int idx = tid + NT * it;
      Xk[swz(idx / 16, idx % 16)] = rx[it];
    }
  }
  __syncthreads();
  const int rr = tid % 16, cq = tid / 16;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int l = 0; l < 4 * cq + 4; ++l) {
    const T a = Xk[swz(l, rr)];
    T bv[4];
    ld4<T>(Bk + swz(l, 4 * cq), bv);
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[bb] += a * bv[bb];
  }
  if (rr < nr)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) G[(k0 + r0 + rr) + (kq + 4 * cq + bb) * f] = acc[bb] / dl[4 * cq + bb];
}

// UX(p, q), FP64 split chain: the lower entries of rows [cut_q, cut_{q+1}) of the
// diagonal tile (p, p) minus sum_l L_rl (L_cl d_l), panel p-1 (equal-area row slabs
// 0, 32, 45, 55, 64), an entry per thread at a time -- the sums of DX(p).
template <typename T>
__device__ void task_ux(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int q, T* F, const T* Dp, T* sm,
                        T* dl) {
  T* Xk = sm;  // K-major L rows of block p, panel p - 1 (row i, k = l)
  const int64_t f = g.f, kq = (int64_t)(p - 1) * NB, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);
  constexpr int kCut[5] = {0, 32, 45, 55, 64};
  const int r0 = min(kCut[q], pw), r1 = min(kCut[q + 1], pw);
  if (r0 >= r1) return;  // uniform over the CTA
  T* G = F + bf.goff[b];
  const int tid = threadIdx.x;
  {
    T rl[16];
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      rl[it] = (i < r1) ? __ldcg(G + (k0 + i) + (kq + l) * f) : (T)0;
    }
    if (tid < NB) dl[tid] = __ldcg(Dp + bf.k0pos[b] + kq + tid);
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      Xk[swz(idx / NB, idx % NB)] = rl[it];
    }
  }
  __syncthreads();
  const int base = r0 * (r0 + 1) / 2;
  const int ne = r1 * (r1 + 1) / 2 - base;  // entries (r, c), r0 <= r < r1, c <= r
  for (int e = tid; e < ne; e += NT) {
    int r = r0;
    while ((r + 1) * (r + 2) / 2 - base <= e) ++r;
    const int c = e - (r * (r + 1) / 2 - base);
    T acc = (T)0;
    for (int l = 0; l < NB; ++l) acc += Xk[swz(l, r)] * (Xk[swz(l, c)] * dl[l]);
    T* t = G + (k0 + r) + (k0 + c) * f;
    *t = __ldcg(t) - acc;
  }
}

// T(p, i): L_IK = F_IK Linv^T D_K^{-1} for the rows of block i (each thread 4 x 4).
template <typename T, bool TC>
__device__ void task_trsm(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int64_t bi, T* F, const T* E,
                          const T* Dp, T* sm, T* dl, const PkRef& pkr) {
  T* Bk = sm;             // K-major Linv (row j, k = l)
  T* Xk = sm + NB * LDK;  // K-major F_IK (row i, k = l), then L_IK (row i, k = j)
  const int64_t f = g.f, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);
  const int64_t r0 = brow0(g, bi);
  const int nr = bnrow(g, bi);
  T* G = F + bf.goff[b];
  const T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
  {  // all loads in one batch, then into shared memory
    T ra[16], rb[16];
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      ra[it] = (i < pw && l < pw) ? __ldcg(Eb + (k0 + i) + (k0 + l) * f) : (T)0;
      rb[it] = (i < nr && l < pw) ? __ldcg(G + (r0 + i) + (k0 + l) * f) : (T)0;
    }
    if (tid < pw) dl[tid] = __ldcg(Dp + bf.k0pos[b] + k0 + tid);
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      Bk[swz(l, i)] = ra[it];
      Xk[swz(l, i)] = rb[it];
    }
  }
  __syncthreads();
  // the product of the fused chain task: warp w, column blocks w and 15 - w, rows
  // 2 lane, 2 lane + 1; Linv lower triangular: only l <= 4 tc + 3
  const int wid = tid >> 5, lane = tid & 31;
  T acc[2][2][4];
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const int tc = ph == 0 ? wid : 15 - wid;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[ph][a][bb] = (T)0;
    const int lend = min(pw, 4 * tc + 4);
    for (int l = 0; l < lend; ++l) {
      T av[2], bv[4];
      ld2<T>(Xk + swz(l, 2 * lane), av);
      ld4<T>(Bk + swz(l, 4 * tc), bv);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) acc[ph][a][bb] += av[a] * bv[bb];
    }
  }
  __syncthreads();  // every thread has read F_IK
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const int tc = ph == 0 ? wid : 15 - wid;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int j = 4 * tc + bb;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int i = 2 * lane + a;
        if (j < pw) Xk[swz(j, i)] = acc[ph][a][bb] / dl[j];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int idx = tid; idx < NB * NB; idx += NT) {
    const int i = idx % NB, j = idx / NB;
    if (i < nr && j < pw) G[(r0 + i) + (k0 + j) * f] = Xk[swz(j, i)];
  }
  if constexpr (TC) {  // PL(p, i)
    pk_write(pkr.tile(pk_l(g.nbf, p, bi)),
             [&](int r, int k) -> float { return (r < nr && k < pw) ? (float)Xk[swz(k, r)] : 0.f; });
    fence_proxy_async_global();
  }
}

// Efin(p, e): E_KC <- Linv E_KC for the E rows of panel p and column block e < p.
template <typename T, bool TC>
__device__ void task_efin(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int64_t e, T* E, T* sm,
                          const PkRef& pkr) {
  T* Ls = sm;
  T* Xs = sm + NB * LD;
  const int64_t f = g.f, k0 = (int64_t)p * NB, cb = (int64_t)e * NB;
  const int pw = bnrow(g, p);
  T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
#pragma unroll
  for (int idx = tid; idx < NB * NB; idx += NT) {
    const int i = idx % NB, j = idx / NB;
    Ls[i * LD + j] = (i < pw && j < pw) ? __ldcg(Eb + (k0 + i) + (k0 + j) * f) : (T)0;
    Xs[i * LD + j] = (i < pw) ? __ldcg(Eb + (k0 + i) + (cb + j) * f) : (T)0;
  }
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
    for (int a = 0; a < 4; ++a) av[a] = Ls[(tr + 16 * a) * LD + l];
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) bv[bb] = Xs[l * LD + tc + 16 * bb];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = tr + 16 * a;
    if (i >= pw) continue;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) Eb[(k0 + i) + (cb + tc + 16 * bb) * f] = acc[a][bb];
  }
  if constexpr (TC) {  // PE(p, e): row n = E column cb + n, k = E row k0 + i
    float* dst = pkr.tile(pk_e(pkr.nL, p, e));
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) {
        const int i = tr + 16 * a, n = tc + 16 * bb;
        dst[pk_word(n, i)] = i < pw ? (float)acc[a][bb] : 0.f;
      }
    fence_proxy_async_global();
  }
}

// U(p, i, j): F_IJ -= L_IK (D_K L_JK^T) (lower part only on a diagonal tile);
// EU(p, i, e): E_IC -= L_IK E_KC.  4 x 4 outputs per thread from K-major tiles.
template <typename T>
__device__ void task_update(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int64_t bi, int64_t bj,
                            bool etile, T* F, T* E, const T* Dp, T* sm, T* dl) {
  T* Ak = sm;
  T* Bk = sm + NB * LDK;
  const int64_t f = g.f, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);
  const int64_t i0 = brow0(g, bi);
  const int ni = bnrow(g, bi);
  T* G = F + bf.goff[b];
  T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
  const int64_t c0 = etile ? bj * NB : brow0(g, bj);
  const int nc = bnrow(g, bj);
  const bool diag = !etile && bi == bj;
  T* base = etile ? Eb : G;
  const int tr = tid % 16, tc = tid / 16;  // rows 4 tr .. 4 tr + 3, columns 4 tc .. 4 tc + 3
  // every global load of the task in one batch: both operand tiles, the pivots
  // and this thread's 4 x 4 outputs of the target tile (its inputs are complete
  // once the task runs), so the task pays one round trip to L2
  T ra[16], rb[16], tv[4][4];
#pragma unroll
  for (int it = 0; it < 16; ++it) {
    const int idx = tid + NT * it;
    const int r = idx % NB, k = idx / NB;
    ra[it] = (k < pw && r < ni) ? __ldcg(G + (i0 + r) + (k0 + k) * f) : (T)0;
    if (!etile)
      rb[it] = (k < pw && r < nc) ? __ldcg(G + (c0 + r) + (k0 + k) * f) : (T)0;
    else  // E_KC: consecutive threads read consecutive rows k0 + kk of column c0 + cc
      rb[it] = (r < pw && k < nc) ? __ldcg(Eb + (k0 + r) + (c0 + k) * f) : (T)0;
  }
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    const int cc = 4 * tc + bb;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = 4 * tr + a;
      tv[a][bb] = (r < ni && cc < nc && (!diag || r >= cc)) ? __ldcg(base + (i0 + r) + (c0 + cc) * f) : (T)0;
    }
  }
  if (!etile && tid < NB) dl[tid] = tid < pw ? __ldcg(Dp + bf.k0pos[b] + k0 + tid) : (T)0;
  if (!etile) __syncthreads();
#pragma unroll
  for (int it = 0; it < 16; ++it) {
    const int idx = tid + NT * it;
    const int r = idx % NB, k = idx / NB;
    Ak[swz(k, r)] = ra[it];
    if (!etile)
      Bk[swz(k, r)] = rb[it] * dl[k];
    else
      Bk[swz(r, k)] = rb[it];
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  for (int k = 0; k < pw; ++k) {
    T av[4], bv[4];
    ld4<T>(Ak + swz(k, 4 * tr), av);
    ld4<T>(Bk + swz(k, 4 * tc), bv);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    const int cc = 4 * tc + bb;
    if (cc >= nc) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = 4 * tr + a;
      if (r < ni && (!diag || r >= cc)) base[(i0 + r) + (c0 + cc) * f] = tv[a][bb] - acc[a][bb];
    }
  }
}


// U(p, i, j) / EU(p, i, e) on the tensor cores (FP32 factor): thread 0 copies
// the packed operand tiles A = PL(p, i) and B = PL(p, j) (U) or PE(p, e) (EU)
// into shared memory with two TMA tensor copies while the other threads load
// the target tile and (U) the pivots D_K; all threads split A and B into high
// and low TF32 parts (B scaled by D_K for U), thread 0 issues the 16 MMAs.
// Lanes 0-63 of the accumulator hold L_hi B, lanes 64-127 L_lo B; warps 2, 3,
// 6, 7 pass the low halves through shared memory, warps 0, 1, 4, 5 form
// target - (high + low) and store it (rows 32 (w % 4) + lane, columns 32 (w / 4)
// ...).  Returns false, with *err = 2, if a wait ran out (the caller then stops;
// copies and MMAs in flight were waited for once more, with the same bound).
__device__ __noinline__ bool task_update_tc(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int64_t bi, int64_t bj,
                               bool etile, float* F, float* E, const float* Dp, const CUtensorMap* tmap,
                               const PkRef& pkr, unsigned char* smtc, float* dl, uint32_t bar_ld, uint32_t bar_mma,
                               uint32_t parity, uint32_t tmem, int* err, int* s_flag) {
  const int64_t f = g.f;
  const int64_t i0 = brow0(g, bi);
  const int ni = bnrow(g, bi);
  const int64_t c0 = etile ? bj * NB : brow0(g, bj);
  const int nc = bnrow(g, bj);
  const int pw = bnrow(g, p);
  const bool diag = !etile && bi == bj;
  float* base = etile ? E + bf.eoff[b] : F + bf.goff[b];
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  // split A and B (32 KB each; the other tasks' scratch lies in the same 64 KB),
  // then the staged tiles (16 KB each; written only by the TMA)
  float* opA = reinterpret_cast<float*>(smtc);
  float* opB = reinterpret_cast<float*>(smtc + kTcOpBytes);
  float* stA = reinterpret_cast<float*>(smtc + 2 * kTcOpBytes);
  float* stB = stA + NB * NB;
  if (tid == 0) {
    const int64_t ta = pkr.base + pk_l(g.nbf, p, bi);
    const int64_t tb = pkr.base + (etile ? pk_e(pkr.nL, p, bj) : pk_l(g.nbf, p, bj));
    fence_proxy_async_global();  // the tiles were released by generic stores (acquired above)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_ld), "r"(2 * kTcPkBytes)
                 : "memory");
    tma_tile(s_addr(stA), tmap, ta, bar_ld);
    tma_tile(s_addr(stB), tmap, tb, bar_ld);
  }
  if (!etile && tid < NB) dl[tid] = tid < pw ? __ldcg(Dp + bf.k0pos[b] + (int64_t)p * NB + tid) : 0.f;
  const int q = wid & 3, h = wid >> 2;
  const int r = 32 * q + lane;  // output row of the top warps (q < 2)
  float tv[32];
  if (q < 2) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const int cc = 32 * h + jj;
      tv[jj] = (r < ni && cc < nc && (!diag || r >= cc)) ? __ldcg(base + (i0 + r) + (c0 + cc) * f) : 0.f;
    }
  }
  if (!mbar_wait(bar_ld, parity)) atomicExch(s_flag, 1);
  __syncthreads();
  if (*s_flag) {
    if (tid == 0) {
      atomicExch(err, 2);
      mbar_wait(bar_ld, parity);  // once more for the copies in flight
    }
    return false;
  }
  pk_split(stA, opA, nullptr);
  pk_split(stB, opB, etile ? nullptr : dl);  // U: B = L_JK D_K
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the split operands are read by the MMAs
  __syncthreads();
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t sA = s_addr(opA), sB = s_addr(opB);
#pragma unroll
    for (int ks = 0; ks < NB / 8; ++ks) {
      const uint32_t ko = (uint32_t)ks * 4096u;  // K = 8: two core matrices along K
      mma_tf32(tmem, pk_desc(sA + ko), pk_desc(sB + ko), kTf32Idesc, ks > 0 ? 1u : 0u);
      mma_tf32(tmem, pk_desc(sA + ko), pk_desc(sB + 1024u + ko), kTf32Idesc, 1u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_mma)
                 : "memory");
  }
  if (!mbar_wait(bar_mma, parity)) atomicExch(s_flag, 1);
  __syncthreads();
  if (*s_flag) {
    if (tid == 0) {
      atomicExch(err, 2);
      mbar_wait(bar_mma, parity);
    }
    return false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t v[32];
  tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h), v);
  float* X = opA;  // the low halves (16 KB; the MMAs have read the operands)
  if (q >= 2) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) X[(32 * h + jj) * 64 + 32 * (q - 2) + lane] = __uint_as_float(v[jj]);
  }
  __syncthreads();
  if (q < 2) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const int cc = 32 * h + jj;
      if (r < ni && cc < nc && (!diag || r >= cc))
        base[(i0 + r) + (c0 + cc) * f] = tv[jj] - (__uint_as_float(v[jj]) + X[(32 * h + jj) * 64 + r]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  return true;
}

template <typename T, bool TC>
__global__ void __launch_bounds__(NT, 2)
    k_bf_flow(BigFrontDev bf, const FlowTask* __restrict__ task, int64_t t0, int64_t nt, int* __restrict__ state,
              int64_t head_off, const int64_t* __restrict__ soff, T* F, T* E, T* Dp, const int8_t* __restrict__ dsign,
              double eps_d, double delta_d, int* hits, int* err, const int* skip, const __grid_constant__ CUtensorMap tmap,
              float* pk) {
  static_assert(!TC || sizeof(T) == 4, "tensor-core products: FP32 factor only");
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  // TC: packed tiles need a 1024-byte aligned base (the other tasks use the same space)
  unsigned char* smtc = smraw + (TC ? ((1024u - (s_addr(smraw) & 1023u)) & 1023u) : 0u);
  T* sm = reinterpret_cast<T*>(smtc);
  __shared__ DiagScratch<T> dsh;
  __shared__ T dl[NB];
  __shared__ FlowTask s_task;
  __shared__ int s_go;
  __shared__ __align__(8) uint64_t s_bar[2];  // TC: TMA and MMA completion
  __shared__ uint32_t s_tmem;
  __shared__ int s_flag;
  int* head = state + head_off;
  const int tid = threadIdx.x;
  uint32_t tmem = 0, parity = 0;
  if constexpr (TC) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(&s_bar[0])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(&s_bar[1])), "r"(1));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      s_flag = 0;
    }
    if ((tid >> 5) == 0) {  // 64 columns: the 128 x 64 FP32 accumulator
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&s_tmem)), "r"(64));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = s_tmem;
    if (tid == 0) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
  }
  for (;;) {
    if (tid == 0) {
      // The next ticket is taken only once this CTA is free: a ticket reserved
      // while the current task still waits for its inputs would be held back
      // for the whole wait, although another CTA could run it at once.
      const int cur = atomicAdd(head, 1);
      int go = 0;
      if (cur < nt) {
        const FlowTask tk = task[t0 + cur];
        s_task = tk;
        const int64_t b = tk.bf;
        const Geo g{bf.f[b], bf.c[b], (bf.c[b] + NB - 1) / NB, flow_nbf(bf.f[b], bf.c[b])};
        const Words w = words_of(state + soff[b], g);
        const int p = tk.p;
        // the version words this task reads and the versions it needs
        const int* wp[3];
        int wv[3];
        int nw;
        switch (tk.kind) {
          case 0:
            wp[0] = w.t(p, p), wv[0] = p;
            nw = 1;
            break;
          case 5:
            wp[0] = w.diag + p - 1, wv[0] = 1;
            wp[1] = w.t(p, p - 1), wv[1] = p - 1;
            wp[2] = w.t(p, p), wv[2] = p - 1;
            nw = 3;
            break;
          case 1:
            wp[0] = w.diag + p, wv[0] = 1;
            wp[1] = w.t(tk.i, p), wv[1] = p;
            nw = 2;
            break;
          case 6:  // TX(p, q): Linv of panel p - 1, F_{p,p-1} updated by panels < p - 1
            wp[0] = w.diag + p - 1, wv[0] = 1;
            wp[1] = w.t(p, p - 1), wv[1] = p - 1;
            nw = 2;
            break;
          case 7:  // UX(p, q): every part of TX(p), the tile updated by panels < p - 1
            wp[0] = w.trsm + p, wv[0] = p;
            wp[1] = w.t(p, p), wv[1] = p - 1;
            nw = 2;
            break;
          case 2:
            wp[0] = w.diag + p, wv[0] = 1;
            wp[1] = w.e(p, tk.j), wv[1] = p - tk.j;
            nw = 2;
            break;
          case 3:
            wp[0] = w.trsm + tk.i, wv[0] = p + 1;
            wp[1] = w.trsm + tk.j, wv[1] = p + 1;
            wp[2] = w.t(tk.i, tk.j), wv[2] = p;
            nw = 3;
            break;
          default:
            wp[0] = w.trsm + tk.i, wv[0] = p + 1;
            if (tk.j < p)
              wp[1] = w.e(p, tk.j), wv[1] = p - tk.j + 1;
            else if (TC)  // the packed E_KK, stored after the diagonal task's release
              wp[1] = w.pe + p, wv[1] = 1;
            else
              wp[1] = w.diag + p, wv[1] = 1;
            wp[2] = w.e(tk.i, tk.j), wv[2] = p - tk.j;
            nw = 3;
            break;
        }
        // one round trip when the inputs are already there (the loads are issued
        // together; the fence below orders them before the task's reads), else
        // bounded waits word by word
        int got[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < nw) got[q] = ld_relaxed(wp[q]);
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < nw && got[q] < wv[q]) ok = ok && wait_ge(wp[q], wv[q], err);
        go = ok ? 1 : 0;
        if (ok) __threadfence();
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const FlowTask tk = s_task;
    const int64_t b = tk.bf;
    const Geo g{bf.f[b], bf.c[b], (bf.c[b] + NB - 1) / NB, flow_nbf(bf.f[b], bf.c[b])};
    PkRef pkr;
    if constexpr (TC) {
      pkr.pk = pk;
      pkr.base = bf.pkoff[b];
      pkr.nL = flow_pk_nl(g.f, g.c);
    }
    bool stop = false;
    switch (tk.kind) {
      case 0:
        task_diag<T, TC>(bf, b, g, tk.p, F, E, Dp, dsign, (T)eps_d, (T)delta_d, hits, sm, dsh, pkr);
        break;
      case 5:  // the fused chain task: FP32 tables only (FP64 ones split it)
        if constexpr (sizeof(T) == 4) {
          const Words w = words_of(state + soff[b], g);
          const int nhit =
              task_dx<T, TC>(bf, b, g, tk.p, F, E, Dp, dsign, (T)eps_d, (T)delta_d, sm, dsh, dl, w.trsm + tk.p, pkr);
          if (tid == 0 && nhit) atomicAdd(hits, nhit);
        }
        break;
      case 1:
        task_trsm<T, TC>(bf, b, g, tk.p, tk.i, F, E, Dp, sm, dl, pkr);
        break;
      case 2:
        task_efin<T, TC>(bf, b, g, tk.p, tk.j, E, sm, pkr);
        break;
      case 6:  // the split chain tasks: FP64 tables only
        if constexpr (sizeof(T) == 8) task_tx<T>(bf, b, g, tk.p, tk.i, F, E, Dp, sm, dl);
        break;
      case 7:
        if constexpr (sizeof(T) == 8) task_ux<T>(bf, b, g, tk.p, tk.i, F, Dp, sm, dl);
        break;
      default:
        if constexpr (TC) {
          stop = !task_update_tc(bf, b, g, tk.p, tk.i, tk.j, tk.kind != 3, F, E, Dp, &tmap, pkr, smtc, dl,
                                 s_addr(&s_bar[0]), s_addr(&s_bar[1]), parity, tmem, err, &s_flag);
          parity ^= 1u;
        } else {
          task_update<T>(bf, b, g, tk.p, tk.i, tk.j, tk.kind != 3, F, E, Dp, sm, dl);
        }
        break;
    }
    // (TC: only the TMA writes the staging tiles, and generic code only reads
    // them; the generic writes to the split operands and the other tasks'
    // scratch are ordered before the MMAs by the proxy fence in task_update_tc)
    __syncthreads();
    if (stop) break;
    if (tid == 0) {
      const Words w = words_of(state + soff[b], g);
      const int p = tk.p;
      __threadfence();
      switch (tk.kind) {
        case 0:
          st_release(w.diag + p, 1);
          break;
        case 5:
          st_release(w.t(p, p), p);
          st_release(w.diag + p, 1);
          break;
        case 1:
          st_release(w.trsm + tk.i, p + 1);
          break;
        case 2:
          st_release(w.e(p, tk.j), p - tk.j + 1);
          break;
        case 6:  // the last part of TX(p) publishes the L rows of block p
          if (atomicAdd(w.txc + p, 1) == 3) {
            __threadfence();
            st_release(w.trsm + p, p);
          }
          break;
        case 7:  // the last part of UX(p) publishes the updated diagonal tile
          if (atomicAdd(w.uxc + p, 1) == 3) {
            __threadfence();
            st_release(w.t(p, p), p);
          }
          break;
        case 3:
          st_release(w.t(tk.i, tk.j), p + 1);
          break;
        default:
          st_release(w.e(tk.i, tk.j), p - tk.j + 1);
          break;
      }
    }
    if constexpr (TC) {
      if (tk.kind == 0 || tk.kind == 5) {
        // PE(p, p) = E_KK (Linv, unit lower; rows = its columns) from the diagonal
        // task's copy in shared memory, after the release above so that the
        // chain of diagonal tasks does not wait for it; EU(p, i, p) waits for
        // the pe word instead
        const int p = tk.p, pw = bnrow(g, p);
        const T* V = tk.kind == 0 ? sm + 64 * kDiagLD : sm;
        pk_write(pkr.tile(pk_e(pkr.nL, p, p)), [&](int n, int k) -> float {
          return (k < pw && n < pw && k >= n) ? (k == n ? 1.f : (float)V[k * kDiagLD + n]) : 0.f;
        });
        fence_proxy_async_global();
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          st_release(words_of(state + soff[b], g).pe + p, 1);
        }
      }
    }
  }
  if constexpr (TC) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((tid >> 5) == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
  }
}

template <typename T>
size_t flow_smem() {  // the fused chain task's three blocks; the others need less
  constexpr int n = 2 * NB * LDK + NB * LD;
  static_assert(n >= kDiagSmem && NB * LDK >= NB * kDiagLD && LD == kDiagLD, "shared memory of the flow tasks");
  return n * sizeof(T);
}
// TC launch: the two packed operand tiles of a U / EU task (the other tasks
// fit in the same space) from a 1024-byte aligned base
size_t flow_smem_tc() {
  static_assert(2 * (size_t)NB * LDK * 4 + (size_t)NB * LD * 4 <= 2 * (size_t)kTcOpBytes,
                "the other tasks' scratch stays clear of the TMA staging tiles");
  static_assert(kTcSmemFlow <= 120 * 1024, "the one-CTA-per-SM launch covers the TC tiles");
  return kTcSmemFlow;
}
}  // namespace

// dynamic shared memory of a launch with one CTA per SM (more than half an SM's)
template <typename T>
size_t flow_smem_one() {
  return flow_smem<T>() > (size_t)120 * 1024 ? flow_smem<T>() : (size_t)120 * 1024;
}

int flow_tc_encode(FlowTc* tc) {
  if (!tc || !tc->pk || tc->tiles <= 0 || (reinterpret_cast<uintptr_t>(tc->pk) & 15) != 0) return CLR_E_INVALID;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  CLR_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess) return CLR_E_CUDA;
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  // rows of 256 floats (1 KB), 16 rows per packed tile; one box = one tile
  const cuuint64_t dims[2] = {256, (cuuint64_t)tc->tiles * 16};
  const cuuint64_t strides[1] = {256 * sizeof(float)};
  const cuuint32_t box[2] = {256, 16};
  const cuuint32_t estr[2] = {1, 1};
  CUtensorMap m;
  const CUresult r = reinterpret_cast<Encode>(fn)(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, tc->pk, dims, strides, box,
                                                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_cuda_error(cudaErrorInvalidValue, "cuTensorMapEncodeTiled");
    return CLR_E_CUDA;
  }
  static_assert(sizeof(CUtensorMap) == sizeof(tc->tmap), "tensor map size");
  std::memcpy(tc->tmap, &m, sizeof(m));
  return CLR_OK;
}

template <typename T>
int BigFrontOps<T>::flow_occupancy(bool tc) {
  // the whole unified L1 / shared memory as shared memory, so that two CTAs of
  // the TC launch (97 KB each) fit on an SM
  CLR_CUDA(cudaFuncSetAttribute(k_bf_flow<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)flow_smem_one<T>()));
  CLR_CUDA(cudaFuncSetAttribute(k_bf_flow<T, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
  int n = 0;
  if (tc && sizeof(T) == 4) {
    CLR_CUDA(cudaFuncSetAttribute(k_bf_flow<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)flow_smem_one<float>()));
    CLR_CUDA(cudaFuncSetAttribute(k_bf_flow<float, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared));
    // from the kernel's resources: the occupancy calculator reports one CTA per
    // SM for this launch although two are resident (measured with per-task
    // timestamps: SM ids and overlapping task intervals)
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, regs_sm = 0, resv = 0;
    CLR_CUDA(cudaFuncGetAttributes(&fa, k_bf_flow<float, true>));
    CLR_CUDA(cudaGetDevice(&dev));
    CLR_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    CLR_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    CLR_CUDA(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    const size_t per_cta = flow_smem_tc() + fa.sharedSizeBytes + (size_t)resv;
    const int by_smem = (int)((size_t)smem_sm / per_cta);
    const int by_regs = fa.numRegs > 0 ? regs_sm / (fa.numRegs * NT) : 1;
    n = std::min(2, std::min(by_smem, by_regs));
  } else {
    CLR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bf_flow<T, false>, NT, flow_smem<T>()));
  }
  return n > 0 ? n : 1;
}

template <typename T>
int BigFrontOps<T>::flow_level(cudaStream_t st, const BigFrontDev& bf, const FlowTask* task, int64_t t0, int64_t nt,
                               int* state, int64_t head_off, const int64_t* soff, int grid, bool one_per_sm, T* F,
                               T* E, T* Dp, const int8_t* dsign, double eps, double delta, int* hits, int* err,
                               const int* skip, const FlowTc* tc) {
  if (nt <= 0) return CLR_OK;
  const unsigned g = (unsigned)(nt < grid ? nt : grid);
  CUtensorMap m;
  if constexpr (sizeof(T) == 4) {
    if (tc) {
      std::memcpy(&m, tc->tmap, sizeof(m));
      const size_t smem = one_per_sm ? flow_smem_one<float>() : flow_smem_tc();
      k_bf_flow<float, true><<<g, NT, smem, st>>>(bf, task, t0, nt, state, head_off, soff, F, E, Dp, dsign, eps,
                                                  delta, hits, err, skip, m, tc->pk);
      CLR_CHECK_LAUNCH();
      return CLR_OK;
    }
  }
  std::memset(&m, 0, sizeof(m));
  const size_t smem = one_per_sm ? flow_smem_one<T>() : flow_smem<T>();
  k_bf_flow<T, false><<<g, NT, smem, st>>>(bf, task, t0, nt, state, head_off, soff, F, E, Dp, dsign, eps, delta, hits,
                                           err, skip, m, nullptr);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

#define CLR_FLOW_INST(T)                                                                                         \
  template int BigFrontOps<T>::flow_occupancy(bool);                                                               \
  template int BigFrontOps<T>::flow_level(cudaStream_t, const BigFrontDev&, const FlowTask*, int64_t, int64_t, int*, \
                                          int64_t, const int64_t*, int, bool, T*, T*, T*, const int8_t*, double,     \
                                          double, int*, int*, const int*, const FlowTc*);
CLR_FLOW_INST(double)
CLR_FLOW_INST(float)
#undef CLR_FLOW_INST

}  // namespace clr
