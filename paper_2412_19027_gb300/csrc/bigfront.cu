// Large fronts: blocked LDL^T with the augmented inverse block E (see bigfront.cuh).
//
// Panel p covers pivots K = [k0, k0 + pw), k0 = 64 p.  Three launches per panel:
//   A  (one CTA per front): LDL^T of the pw x pw diagonal block (32 x 32 blocks
//      factored and inverted by one warp in registers), its pivots, and
//      Linv = L_KK^{-1};
//   B  L_IK = F_IK L_KK^{-T} D_K^{-1} for the rows I below K, as the product
//      F_IK Linv^T scaled by D^{-1}; the same launch finalises the E rows of
//      this panel: E_KC <- Linv E_KC (C < K) and E_KK = Linv;
//   C  64 x 64 tiles: trailing update F_IJ -= L_IK D_K L_JK^T (I >= J below K)
//      and the augmented rows E_IC -= L_IK E_KC for C <= K.
// After the last panel E = L^{-1} [I; 0].  Forward solve: y = E_top w1,
// u = w2 + E_bottom w1; backward: x1 = E^T [D^{-1} y; x2].
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
constexpr unsigned FULLMASK = 0xffffffffu;

// LDL^T of a 32 x 32 symmetric block held by one warp in registers: lane i
// holds row i (r[j], j <= i; zero above).  Right-looking: pivot k is lane k's
// r[k]; every lane updates its row with the unscaled column k broadcast from
// the lanes below (S_ij -= L_ik S_jk), then scales its multiplier.  A pivot
// with the wrong sign or magnitude <= eps is replaced by sign * delta (dynamic
// regularisation).  Afterwards r[j] = L_ij (j < i) and r[i] = d_i.  Rows >= n
// are padding (zero rows).
template <typename T>
__device__ __forceinline__ void warp_ldl32(T (&r)[32], int n, const int8_t* sgn, T eps, T delta, int* nhit) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < n) {
      T d = __shfl_sync(FULLMASK, r[k], k);
      const T sg = (T)sgn[k];
      if (sg * d <= eps) {
        d = sg * delta;
        ++*nhit;
      }
      const T lik = (lane > k) ? r[k] / d : (T)0;
#pragma unroll
      for (int j = k + 1; j < 32; ++j) {
        const T sjk = __shfl_sync(FULLMASK, r[k], j);
        if (lane >= j) r[j] -= lik * sjk;
      }
      if (lane > k) r[k] = lik;
      else if (lane == k) r[k] = d;
    }
  }
}

// Column `lane` of the inverse of the unit lower triangle whose rows are held
// as above (forward substitution with the rows broadcast from their lanes).
template <typename T>
__device__ __forceinline__ void warp_inv_unit32(const T (&r)[32], T (&x)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    T acc = (i == lane) ? (T)1 : (T)0;
#pragma unroll
    for (int l = 0; l < i; ++l) acc -= __shfl_sync(FULLMASK, r[l], i) * x[l];
    x[i] = acc;
  }
}

// Diagonal block of panel p (pw <= 64 pivots) as 2 x 2 blocks of 32:
//   A11 = L11 D1 L11^T by warp 0 in registers, with L11^{-1};
//   W21 = A21 L11^{-T} (= L21 D1), L21 = W21 D1^{-1};  A22 -= L21 W21^T;
//   A22 = L22 D2 L22^T by warp 0, with L22^{-1};
//   (L^{-1})_21 = -L22^{-1} L21 L11^{-1}.
// Outputs: L (unit lower, d on the diagonal) into the front, pivots to Dp, and
// Linv = L^{-1} (64 x 64, column-major, zero padded).
template <typename T>
__global__ void __launch_bounds__(256) k_bf_diag(BigFrontDev bf, WorkList wl, int p, T* __restrict__ F,
                                                 T* __restrict__ Dp, T* __restrict__ Linv,
                                                 const int8_t* __restrict__ dsign, double eps_d, double delta_d,
                                                 int* hits, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);  // NB x LD: the block (lower part); rows 0..31 of cols 32..63 as scratch
  T* Lo = S + NB * LD;                 // NB x LD: L, d on the diagonal
  T* Li = Lo + NB * LD;                // NB x LD: L^{-1}
  __shared__ int8_t sgn[NB];
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b], k0 = (int64_t)p * NB;
  const int pw = (int)min((int64_t)NB, c - k0);
  const int cw0 = min(32, pw), cw1 = pw - cw0;
  T* G = F + bf.goff[b];
  const int64_t kp = bf.k0pos[b] + k0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const T eps = (T)eps_d, delta = (T)delta_d;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx % NB, j = idx / NB;
    S[i * LD + j] = (i < pw && j < pw && i >= j) ? G[(k0 + i) + (k0 + j) * f] : (T)0;
    Lo[i * LD + j] = (T)0;
    Li[i * LD + j] = (T)0;
  }
  if (tid < NB) sgn[tid] = tid < pw ? dsign[kp + tid] : (int8_t)1;
  __syncthreads();
  int nhit = 0;
  if (wid == 0) {
    T r[32], x[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = S[lane * LD + j];
    warp_ldl32(r, cw0, sgn, eps, delta, &nhit);
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j <= lane) Lo[lane * LD + j] = r[j];
    warp_inv_unit32(r, x);
#pragma unroll
    for (int i = 0; i < 32; ++i) Li[i * LD + lane] = x[i];
  }
  __syncthreads();
  if (cw1 > 0) {
    for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
      const int i = idx % 32, j = idx / 32;
      T acc = (T)0;
      for (int l = 0; l <= j; ++l) acc += S[(32 + i) * LD + l] * Li[j * LD + l];
      S[i * LD + 32 + j] = acc;                    // W21
      Lo[(32 + i) * LD + j] = acc / Lo[j * LD + j];  // L21
    }
    __syncthreads();
    for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
      const int i = idx % 32, j = idx / 32;
      if (i < j) continue;
      T acc = (T)0;
      for (int l = 0; l < 32; ++l) acc += Lo[(32 + i) * LD + l] * S[j * LD + 32 + l];
      S[(32 + i) * LD + 32 + j] -= acc;
    }
    __syncthreads();
    if (wid == 0) {
      T r[32], x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) r[j] = (j <= lane) ? S[(32 + lane) * LD + 32 + j] : (T)0;
      warp_ldl32(r, cw1, sgn + 32, eps, delta, &nhit);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j <= lane) Lo[(32 + lane) * LD + 32 + j] = r[j];
      warp_inv_unit32(r, x);
#pragma unroll
      for (int i = 0; i < 32; ++i) Li[(32 + i) * LD + 32 + lane] = x[i];
    }
    __syncthreads();
    for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {  // X = L21 L11^{-1} (scratch in S)
      const int i = idx % 32, j = idx / 32;
      T acc = (T)0;
      for (int l = j; l < 32; ++l) acc += Lo[(32 + i) * LD + l] * Li[l * LD + j];
      S[i * LD + 32 + j] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
      const int i = idx % 32, j = idx / 32;
      T acc = (T)0;
      for (int l = 0; l <= i; ++l) acc += Li[(32 + i) * LD + 32 + l] * S[l * LD + 32 + j];
      Li[(32 + i) * LD + j] = -acc;
    }
    __syncthreads();
  }
  if (tid == 0 && nhit) atomicAdd(hits, nhit);
  for (int idx = tid; idx < pw * pw; idx += blockDim.x) {
    const int i = idx % pw, j = idx / pw;
    if (i >= j) G[(k0 + i) + (k0 + j) * f] = Lo[i * LD + j];
  }
  for (int i = tid; i < pw; i += blockDim.x) Dp[kp + i] = Lo[i * LD + i];
  T* LB = Linv + (b * 2 + (p & 1)) * (int64_t)(NB * NB);
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx % NB, j = idx / NB;
    LB[i + j * NB] = (i < pw && j < pw) ? Li[i * LD + j] : (T)0;
  }
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
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
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
// 64 x 64 output tiles, 64 threads, 8 x 8 outputs per thread; operands staged
// K-major in shared memory (row/column index contiguous for each k) so that a
// thread reads its 8 rows and 8 columns with vector loads.
//   trailing tile (I >= J below K): F_IJ -= L_IK (D_K L_JK^T)
//   E tile (rows I below K, column block C <= K): E_IC -= L_IK E_KC, with the
//   E rows of K already finalised by this panel's B launch (E_KK = Linv).
constexpr int LDK = NB + 4;  // 16-byte aligned rows of the K-major tiles

template <typename T>
__device__ __forceinline__ void ld8(const T* p, T (&v)[8]);
template <>
__device__ __forceinline__ void ld8<float>(const float* p, float (&v)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <>
__device__ __forceinline__ void ld8<double>(const double* p, double (&v)[8]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double2 a = *reinterpret_cast<const double2*>(p + 2 * u);
    v[2 * u] = a.x;
    v[2 * u + 1] = a.y;
  }
}

template <typename T>
__global__ void __launch_bounds__(64) k_bf_update(BigFrontDev bf, WorkList wl, int p, T* __restrict__ F,
                                                  T* __restrict__ E, const T* __restrict__ Dp, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ak = reinterpret_cast<T*>(smraw);  // [l][row]
  T* Bk = Ak + NB * LDK;                 // [l][col]
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
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      const int r = idx % NB, l = idx / NB;
      const int64_t ia = i0 + r, ib = j0 + r;
      Ak[l * LDK + r] = (l < pw && ia < f) ? G[ia + (k0 + l) * f] : (T)0;
      Bk[l * LDK + r] = (l < pw && ib < f) ? G[ib + (k0 + l) * f] * Dk[l] : (T)0;
    }
  } else {
    const int64_t e = q - na;
    const int64_t bi = e / (p + 1), cb = e % (p + 1);
    i0 = t0 + bi * NB;
    colbase = cb * NB;
    if (cb == p) ncols = pw;
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      const int r = idx % NB, l = idx / NB;
      const int64_t ia = i0 + r;
      Ak[l * LDK + r] = (l < pw && ia < f) ? G[ia + (k0 + l) * f] : (T)0;
      // E_KC: row k0 + l, column colbase + r (consecutive l are consecutive in memory)
      const int l2 = idx % NB, cc = idx / NB;
      Bk[l2 * LDK + cc] = (l2 < pw && cc < ncols) ? Eb[(k0 + l2) + (colbase + cc) * f] : (T)0;
    }
  }
  __syncthreads();
  const int tr = tid % 8, tc = tid / 8;
  T acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) acc[a][bb] = (T)0;
  for (int l = 0; l < pw; ++l) {
    T av[8], bv[8];
    ld8<T>(Ak + l * LDK + 8 * tr, av);
    ld8<T>(Bk + l * LDK + 8 * tc, bv);
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int bb = 0; bb < 8; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
  if (!etile) {
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) {
      const int64_t j = j0 + 8 * tc + bb;
      if (j >= f) continue;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t i = i0 + 8 * tr + a;
        if (i < f && i >= j) G[i + j * f] -= acc[a][bb];
      }
    }
  } else {
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) {
      const int cc = 8 * tc + bb;
      if (cc >= ncols) continue;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t i = i0 + 8 * tr + a;
        if (i < f) Eb[i + (colbase + cc) * f] -= acc[a][bb];
      }
    }
  }
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
namespace {
size_t smem_diag() { return 0; }
}  // namespace

template <typename T>
int BigFrontOps<T>::setup_attributes() {
  CLR_CUDA(cudaFuncSetAttribute(k_bf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * NB * LD * sizeof(T)));
  CLR_CUDA(cudaFuncSetAttribute(k_bf_trsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * NB * LD * sizeof(T)));
  CLR_CUDA(cudaFuncSetAttribute(k_bf_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * NB * LDK * sizeof(T)));
  (void)smem_diag;
  return CLR_OK;
}

template <typename T>
int BigFrontOps<T>::factor_level(cudaStream_t st, const BigFrontDev& bf, const BigLevelPlan& plan, T* F, T* E, T* Dp,
                                 T* Linv, const int8_t* dsign, double eps, double delta, int* hits, const int* skip) {
  const size_t s2 = 2 * NB * LD * sizeof(T), s3 = 3 * NB * LD * sizeof(T), su = 2 * NB * LDK * sizeof(T);
  for (size_t p = 0; p < plan.A.size(); ++p) {
    if (plan.A[p].nblocks > 0)
      k_bf_diag<T><<<(unsigned)plan.A[p].nblocks, 256, s3, st>>>(bf, plan.A[p], (int)p, F, Dp, Linv, dsign, eps, delta,
                                                                  hits, skip);
    if (plan.B[p].nblocks > 0)
      k_bf_trsm<T><<<(unsigned)plan.B[p].nblocks, 256, s2, st>>>(bf, plan.B[p], (int)p, F, E, Dp, Linv, skip);
    if (plan.C[p].nblocks > 0)
      k_bf_update<T><<<(unsigned)plan.C[p].nblocks, 64, su, st>>>(bf, plan.C[p], (int)p, F, E, Dp, skip);
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
