// Diagonal block of a big-front panel: LDL^T of a pw x pw (pw <= 64) symmetric
// block and the inverse of its unit lower factor, by one CTA of 256 threads.
//
// Blocked by 16 columns (four sub-panels), right-looking:
//   1. warp 0 factors the 16 x 16 diagonal sub-block in registers (lane r holds
//      row r; pivot k: d = a_kk, replaced by sign_k * delta when sign_k * d <= eps
//      -- dynamic regularisation of a pivot of the wrong sign or too small;
//      l_rk = a_rk / d; a_rc -= l_rk a_ck), all shuffles of column k issued
//      before the pivot's reciprocal;
//   2. the rows below, by substitution along each row (one thread per row):
//      L_RQ D_Q L_QQ^T = A_RQ, with the scaled columns d_m l_cm of the sub-block
//      and the pivots' reciprocals from step 1;
//   3. the trailing block, 2 x 2 outputs per thread: A_RR' -= L_RQ D_Q L_R'Q^T;
// then L^{-1}: the four 16 x 16 diagonal blocks by forward substitution (one
// warp per block, one lane per column), and the off-diagonal blocks by block rows,
//   Linv_QP = -Linv_QQ sum_{P <= M < Q} L_QM Linv_MP,
// 2 x 2 outputs per thread.
#pragma once

#include <cstdint>

namespace clr {

constexpr int kDiagLD = 65;                     // row stride of the shared blocks
constexpr int kDiagSmem = 2 * 64 * kDiagLD;     // elements of shared memory bf_diag_block needs

// Small shared scratch of bf_diag_block.
template <typename T>
struct DiagScratch {
  T dv[64];    // pivots
  T dinv[64];  // their reciprocals
  int8_t sgn[64];
};

__device__ __forceinline__ float diag_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double diag_rcp(double x) { return __drcp_rn(x); }

// Warp-level LDL^T of the w x w (w <= 16) diagonal sub-block at (c0, c0) of A:
// lane r keeps row r in registers; column k comes by shuffles.  Writes L (pivots
// on the diagonal) back into A, the pivots and their reciprocals to sh, and the
// scaled rows l_rc d_c (c < r) into the same place of W.  The pivot loop has no
// branches: rows and pivots past w are padded with the identity (pivot 1, no
// multipliers), so the whole loop is one block the compiler can schedule across
// pivots; the expected signs come in as one bit mask.
template <typename T>
__device__ __forceinline__ void diag_sub16(T* A, T* W, int c0, int w, DiagScratch<T>& sh, T eps, T delta,
                                           int& nhit) {
  constexpr int LDD = kDiagLD;
  constexpr unsigned FULL = 0xffffffffu;
  const int r = threadIdx.x & 31;
  const unsigned neg = __ballot_sync(FULL, r < 16 && sh.sgn[c0 + r] < 0);
  T v[16], dd[16], di[16];
#pragma unroll
  for (int c = 0; c < 16; ++c)
    v[c] = (r < w && c <= r) ? A[(c0 + r) * LDD + c0 + c] : ((c == r) ? (T)1 : (T)0);
  int hits = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    T col[16];
#pragma unroll
    for (int c = k; c < 16; ++c) col[c] = __shfl_sync(FULL, v[k], c);  // a_ck, held by lane c
    const T sg = ((neg >> k) & 1u) ? (T)-1 : (T)1;
    const bool bad = sg * col[k] <= eps;
    const T d = bad ? sg * delta : col[k];
    hits += bad ? 1 : 0;
    const T inv = diag_rcp(d);
    const T lik = (r > k) ? v[k] * inv : (T)0;
#pragma unroll
    for (int c = k + 1; c < 16; ++c) v[c] = (c <= r) ? v[c] - lik * col[c] : v[c];
    v[k] = (r == k) ? d : ((r > k) ? lik : v[k]);
    dd[k] = d;
    di[k] = inv;
  }
  nhit += hits;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    if (r < w && c <= r) {
      A[(c0 + r) * LDD + c0 + c] = v[c];
      if (c < r) W[(c0 + r) * LDD + c0 + c] = v[c] * dd[c];
    }
    if (r == 0 && c < w) {
      sh.dv[c0 + c] = dd[c];
      sh.dinv[c0 + c] = di[c];
    }
  }
}

// G: the block (column-major, leading dimension f, lower triangle read).
// Writes L (unit lower, pivots on the diagonal) back into G's lower triangle,
// the pivots to D[0 .. pw), and the lower triangle of L^{-1} (unit diagonal) to
// Li (leading dimension ldi); with zero_rest, also zeros in the rest of the
// 64 x 64 Li block.  smem: kDiagSmem elements.  Returns the number of
// regularised pivots (in thread 0).
// The factorization proper: A (64 x 65 in shared memory) holds the lower triangle
// of the block, zeros elsewhere; V (64 x 65) is work space (its contents on entry
// are never read).  Needs blockDim.x >= 192 (every caller runs 256 threads).
// Outputs as for bf_diag_block.
template <typename T>
__device__ int bf_diag_factor(T* A, T* V, T* G, int64_t f, int pw, T* D, T* Li, int64_t ldi, bool zero_rest,
                              const int8_t* dsign, T eps, T delta, DiagScratch<T>& sh) {
  constexpr int LDD = kDiagLD;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31, nth = blockDim.x;
  if (tid < 64) sh.sgn[tid] = tid < pw ? dsign[tid] : (int8_t)1;
  __syncthreads();
  int nhit = 0;
  for (int c0 = 0; c0 < pw; c0 += 16) {
    const int w = min(16, pw - c0);
    if (wid == 0) diag_sub16<T>(A, V, c0, w, sh, eps, delta, nhit);
    __syncthreads();
    const int r0 = c0 + w;
    if (r0 < pw) {  // then w == 16
      // rows below: l_rc = (a_rc - sum_{m<c} l_rm (d_m l_cm)) / d_c; V keeps l_rc d_c
      for (int rr = r0 + tid; rr < pw; rr += nth) {
        T* Arow = A + rr * LDD + c0;
        T* Vrow = V + rr * LDD + c0;
        T l[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          T v = Arow[c];
#pragma unroll
          for (int m = 0; m < c; ++m) v -= l[m] * V[(c0 + c) * LDD + c0 + m];
          l[c] = v * sh.dinv[c0 + c];
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          Arow[c] = l[c];
          Vrow[c] = l[c] * sh.dv[c0 + c];
        }
      }
      __syncthreads();
      // trailing block: a_rs -= sum_m l_rm (l_sm d_m), r >= s >= r0, by 2 x 2 blocks
      const int nr = pw - r0, nb2 = (nr + 1) >> 1, nblk = nb2 * (nb2 + 1) / 2;
      for (int e = tid; e < nblk; e += nth) {
        int bi = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (bi * (bi + 1) / 2 > e) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= e) ++bi;
        const int bj = e - bi * (bi + 1) / 2;
        const int ra = r0 + 2 * bi, sa = r0 + 2 * bj;  // ra >= sa, both < pw
        const int rb = min(ra + 1, pw - 1), sb = min(sa + 1, pw - 1);
        T a00 = (T)0, a01 = (T)0, a10 = (T)0, a11 = (T)0;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const T x0 = A[ra * LDD + c0 + m], x1 = A[rb * LDD + c0 + m];
          const T y0 = V[sa * LDD + c0 + m], y1 = V[sb * LDD + c0 + m];
          a00 += x0 * y0;
          a01 += x0 * y1;
          a10 += x1 * y0;
          a11 += x1 * y1;
        }
        A[ra * LDD + sa] -= a00;
        if (sa + 1 <= ra) A[ra * LDD + sa + 1] -= a01;
        if (ra + 1 < pw) {
          A[(ra + 1) * LDD + sa] -= a10;
          A[(ra + 1) * LDD + sa + 1] -= a11;
        }
      }
      __syncthreads();
    }
  }
  // diagonal blocks of L^{-1}: warp q, lane c solves L_QQ x = e_c; zeros above
  // the diagonal and outside the block's pw - 16 q rows
  const int nq = (pw + 15) / 16;
  if (wid < nq && lane < 16) {
    const int Q0 = 16 * wid, wq = min(16, pw - Q0), c = lane;
    T x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      T s = (r == c) ? (T)1 : (T)0;
#pragma unroll
      for (int m = 0; m < r; ++m) s -= A[(Q0 + r) * LDD + Q0 + m] * x[m];
      x[r] = (r >= c && r < wq && c < wq) ? s : (T)0;
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) V[(Q0 + r) * LDD + Q0 + c] = x[r];
  }
  __syncthreads();
  // off-diagonal blocks, block row by block row; thread t: rows a, a + 1 and
  // columns b, b + 1 of the 16 x 16q strip (b, b + 1 in one 16-column block P)
  for (int q = 1; q < nq; ++q) {
    const int R0 = 16 * q;
    const bool act = tid < 4 * R0;
    const int a = 2 * (tid & 7), b = 2 * (tid >> 3);
    T y00 = (T)0, y01 = (T)0, y10 = (T)0, y11 = (T)0;
    if (act) {
      // X_QP = sum_{P <= M < Q} L_QM Linv_MP, staged in the strip's place in V
      T x00 = (T)0, x01 = (T)0, x10 = (T)0, x11 = (T)0;
      for (int m = (b >> 4) << 4; m < R0; ++m) {
        const T p0 = A[(R0 + a) * LDD + m], p1 = A[(R0 + a + 1) * LDD + m];
        const T q0 = V[m * LDD + b], q1 = V[m * LDD + b + 1];
        x00 += p0 * q0;
        x01 += p0 * q1;
        x10 += p1 * q0;
        x11 += p1 * q1;
      }
      V[(R0 + a) * LDD + b] = x00;
      V[(R0 + a) * LDD + b + 1] = x01;
      V[(R0 + a + 1) * LDD + b] = x10;
      V[(R0 + a + 1) * LDD + b + 1] = x11;
    }
    __syncthreads();
    if (act) {
      // Linv_QP = -Linv_QQ X_QP (Linv_QQ is zero above its diagonal)
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const T l0 = V[(R0 + a) * LDD + R0 + m], l1 = V[(R0 + a + 1) * LDD + R0 + m];
        const T z0 = V[(R0 + m) * LDD + b], z1 = V[(R0 + m) * LDD + b + 1];
        y00 += l0 * z0;
        y01 += l0 * z1;
        y10 += l1 * z0;
        y11 += l1 * z1;
      }
    }
    __syncthreads();
    if (act) {
      V[(R0 + a) * LDD + b] = -y00;
      V[(R0 + a) * LDD + b + 1] = -y01;
      V[(R0 + a + 1) * LDD + b] = -y10;
      V[(R0 + a + 1) * LDD + b + 1] = -y11;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < 64 * 64; idx += nth) {
    const int i = idx & 63, j = idx >> 6;
    if (i < pw && j < pw && i >= j) {
      G[i + (int64_t)j * f] = A[i * LDD + j];
      Li[i + (int64_t)j * ldi] = (i == j) ? (T)1 : V[i * LDD + j];
    }
  }
  for (int i = tid; i < pw; i += nth) D[i] = sh.dv[i];
  if (zero_rest)
    for (int idx = tid; idx < 64 * 64; idx += nth) {
      const int i = idx & 63, j = idx >> 6;
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
