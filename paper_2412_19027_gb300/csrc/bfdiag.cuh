// Diagonal block of a big-front panel: LDL^T of a pw x pw (pw <= 64) symmetric
// block and the inverse of its unit lower factor, by one CTA of 256 threads.
//
// Blocked by 16 columns (four sub-panels), right-looking:
//   1. warp 0 factors the 16 x 16 diagonal sub-block in registers (lane r holds
//      row r; pivot k: d = a_kk, replaced by sign_k * delta when sign_k * d <= eps
//      -- dynamic regularisation of a pivot of the wrong sign or too small;
//      l_rk = a_rk / d; a_rc -= l_rk a_ck) and, with the same row operations on
//      the identity, the inverse of its unit lower factor;
//   2. the rows below, by substitution along each row: L_RQ D_Q L_QQ^T = A_RQ;
//   3. the trailing block: A_RR' -= L_RQ D_Q L_R'Q^T;
// then the off-diagonal blocks of L^{-1} by block rows:
//   Linv_QP = -Linv_QQ sum_{P <= M < Q} L_QM Linv_MP.
// About 20 barriers in all (one per pivot before), each phase a few dozen
// independent multiply-adds per thread.
#pragma once

#include <cstdint>

namespace clr {

constexpr int kDiagLD = 65;                     // row stride of the shared blocks
constexpr int kDiagSmem = 2 * 64 * kDiagLD;     // elements of shared memory bf_diag_block needs

// Small shared scratch of bf_diag_block.
template <typename T>
struct DiagScratch {
  T dv[64];
  int8_t sgn[64];
};

// Warp-level LDL^T of the w x w (w <= 16) diagonal sub-block at (c0, c0) of A and the
// inverse of its unit lower factor (into the same place of V): lane r keeps row r
// of both in registers; column k and row k of the inverse come by shuffles.
template <typename T>
__device__ __forceinline__ void diag_sub16(T* A, T* V, int c0, int w, DiagScratch<T>& sh, T eps, T delta,
                                           int& nhit) {
  constexpr int LDD = kDiagLD;
  constexpr unsigned FULL = 0xffffffffu;
  const int r = threadIdx.x & 31;
  T v[16], g[16];
#pragma unroll 16
  for (int c = 0; c < 16; ++c) {
    v[c] = (r < w && c <= r) ? A[(c0 + r) * LDD + c0 + c] : (T)0;
    g[c] = (c == r) ? (T)1 : (T)0;
  }
#pragma unroll 16
  for (int k = 0; k < 16; ++k) {
    if (k < w) {
      T d = __shfl_sync(FULL, v[k], k);
      const T sg = (T)sh.sgn[c0 + k];
      if (sg * d <= eps) {
        d = sg * delta;
        ++nhit;
      }
      const T inv = (T)1 / d;
      const T lik = (r > k && r < w) ? v[k] * inv : (T)0;
#pragma unroll 16
      for (int c = k + 1; c < 16; ++c) {
        const T ack = __shfl_sync(FULL, v[k], c);  // a_ck: row c of column k
        v[c] = (c <= r) ? v[c] - lik * ack : v[c];
      }
#pragma unroll 16
      for (int c = 0; c <= k; ++c) {
        const T gkc = __shfl_sync(FULL, g[c], k);  // row k of the inverse
        g[c] -= lik * gkc;
      }
      v[k] = (r == k) ? d : ((r > k) ? lik : v[k]);
      if (r == 0) sh.dv[c0 + k] = d;
    }
  }
#pragma unroll 16
  for (int c = 0; c < 16; ++c)
    if (r < w && c <= r) {
      A[(c0 + r) * LDD + c0 + c] = v[c];
      V[(c0 + r) * LDD + c0 + c] = g[c];
    }
}

// G: the block (column-major, leading dimension f, lower triangle read).
// Writes L (unit lower, pivots on the diagonal) back into G's lower triangle,
// the pivots to D[0 .. pw), and the lower triangle of L^{-1} (unit diagonal) to
// Li (leading dimension ldi); with zero_rest, also zeros in the rest of the
// 64 x 64 Li block.  smem: kDiagSmem elements.  Returns the number of
// regularised pivots (in thread 0).
// The factorization proper: A (64 x 65 in shared memory) holds the lower triangle
// of the block, zeros elsewhere; V (64 x 65) is work space.  Outputs as for
// bf_diag_block.
template <typename T>
__device__ int bf_diag_factor(T* A, T* V, T* G, int64_t f, int pw, T* D, T* Li, int64_t ldi, bool zero_rest,
                              const int8_t* dsign, T eps, T delta, DiagScratch<T>& sh) {
  constexpr int LDD = kDiagLD;
  const int tid = threadIdx.x, wid = tid >> 5, nth = blockDim.x;
  for (int idx = tid; idx < 64 * 64; idx += nth) V[(idx % 64) * LDD + idx / 64] = (T)0;
  if (tid < 64) sh.sgn[tid] = tid < pw ? dsign[tid] : (int8_t)1;
  __syncthreads();
  int nhit = 0;
  for (int c0 = 0; c0 < pw; c0 += 16) {
    const int w = min(16, pw - c0);
    if (wid == 0) diag_sub16<T>(A, V, c0, w, sh, eps, delta, nhit);
    __syncthreads();
    const int r0 = c0 + w, nr = pw - r0;
    if (nr > 0) {
      // rows below, by substitution along each row (one thread per row, as the
      // elimination computes them): l_rc = (a_rc - sum_{m<c} l_rm d_m l_cm) / d_c
      for (int rr = r0 + tid; rr < pw; rr += nth) {
        T* Arow = A + rr * LDD + c0;
#pragma unroll 16
        for (int c = 0; c < 16; ++c) {
          if (c < w) {
            const T* Lc = A + (c0 + c) * LDD + c0;
            T v = Arow[c];
            for (int m = 0; m < c; ++m) v -= Arow[m] * (sh.dv[c0 + m] * Lc[m]);
            Arow[c] = v / sh.dv[c0 + c];
          }
        }
      }
      __syncthreads();
      // trailing block: a_rs -= sum_m l_rm d_m l_sm, r >= s >= r0
      const int ntr = nr * (nr + 1) / 2;
      for (int e = tid; e < ntr; e += nth) {
        int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (i * (i + 1) / 2 > e) --i;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        const int j = e - i * (i + 1) / 2;
        const int rr = r0 + i, ss = r0 + j;
        T acc = (T)0;
#pragma unroll
        for (int m = 0; m < 16; ++m)
          if (m < w) acc += A[rr * LDD + c0 + m] * sh.dv[c0 + m] * A[ss * LDD + c0 + m];
        A[rr * LDD + ss] -= acc;
      }
      __syncthreads();
    }
  }
  // off-diagonal blocks of L^{-1}, block row by block row
  const int nq = (pw + 15) / 16;
  for (int q = 1; q < nq; ++q) {
    const int R0 = 16 * q;
    // X_QP = sum_{P <= M < Q} L_QM Linv_MP for all P < Q: element (a, b) of the
    // 16 x 16q strip, column b in block P = b / 16
    T x[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int idx = tid + nth * t;
      x[t] = (T)0;
      if (idx < 16 * R0) {
        const int a = idx % 16, b = idx / 16;
        T acc = (T)0;
#pragma unroll 4
        for (int m = (b / 16) * 16; m < R0; ++m) acc += A[(R0 + a) * LDD + m] * V[m * LDD + b];
        x[t] = acc;
      }
    }
    // stage X in the strip's place in V (still zero), then Linv_QP = -Linv_QQ X_QP
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int idx = tid + nth * t;
      if (idx < 16 * R0) V[(R0 + idx % 16) * LDD + idx / 16] = x[t];
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int idx = tid + nth * t;
      x[t] = (T)0;
      if (idx < 16 * R0) {
        const int a = idx % 16, b = idx / 16;
        T acc = (T)0;
#pragma unroll
        for (int m = 0; m < 16; ++m)
          if (m <= a) acc += V[(R0 + a) * LDD + R0 + m] * V[(R0 + m) * LDD + b];
        x[t] = -acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int idx = tid + nth * t;
      if (idx < 16 * R0) V[(R0 + idx % 16) * LDD + idx / 16] = x[t];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < pw * pw; idx += nth) {
    const int i = idx % pw, j = idx / pw;
    if (i >= j) {
      G[i + (int64_t)j * f] = A[i * LDD + j];
      Li[i + (int64_t)j * ldi] = (i == j) ? (T)1 : V[i * LDD + j];
    }
  }
  for (int i = tid; i < pw; i += nth) D[i] = sh.dv[i];
  if (zero_rest)
    for (int idx = tid; idx < 64 * 64; idx += nth) {
      const int i = idx % 64, j = idx / 64;
      if (i < j || i >= pw) Li[i + (int64_t)j * ldi] = (T)0;
    }
  return nhit;
}

template <typename T>
__device__ int bf_diag_block(T* G, int64_t f, int pw, T* D, T* Li, int64_t ldi, bool zero_rest, const int8_t* dsign,
                             T eps, T delta, T* smem, DiagScratch<T>& sh) {
  constexpr int LDD = kDiagLD;
  T* A = smem;             // the block as it is eliminated; L and the pivots at the end
  T* V = smem + 64 * LDD;  // L^{-1}
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
    const int i = idx % 64, j = idx / 64;
    A[i * LDD + j] = (i < pw && j < pw && i >= j) ? __ldcg(G + i + (int64_t)j * f) : (T)0;
  }
  return bf_diag_factor<T>(A, V, G, f, pw, D, Li, ldi, zero_rest, dsign, eps, delta, sh);
}

}  // namespace clr
