// Large fronts: blocked LDL^T with the augmented inverse block E (see bigfront.cuh).
//
// Panel p covers pivots K = [k0, k0 + pw), k0 = 64 p.  Three launches per panel:
//   A  (one CTA per front): LDL^T of the pw x pw diagonal block (two 32-column
//      sub-panels, each factored by one warp), its pivots, and Linv = L_KK^{-1};
//   B  L_IK = F_IK L_KK^{-T} D_K^{-1} for the rows I below K, as the product
//      F_IK Linv^T scaled by D^{-1}; the same launch finalises the E rows of the
//      previous panel: E_K',C <- Linv' E_K',C and E_K'K' = Linv';
//   C  64 x 64 tiles: trailing update F_IJ -= L_IK D_K L_JK^T (I >= J below K)
//      and the augmented rows E_IC -= L_IK (Linv E_KC) for C < K, E_IK -= L_IK Linv.
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
// Inverse of a unit lower n x n block (n <= 32) held in S (rows/cols from r0):
// lane j of the calling warp computes column j in Li (same offsets), reading the
// already computed entries of its column from shared memory.
template <typename T>
__device__ __forceinline__ void warp_inv32(const T* S, T* Li, int r0, int n) {
  const int j = threadIdx.x & 31;
  if (j < n) {
    Li[(r0 + j) * LD + r0 + j] = (T)1;
    for (int i = j + 1; i < n; ++i) {
      T acc = (T)0;
      for (int l = j; l < i; ++l) acc += S[(r0 + i) * LD + r0 + l] * Li[(r0 + l) * LD + r0 + j];
      Li[(r0 + i) * LD + r0 + j] = -acc;
    }
  }
}

// Diagonal block of panel p: LDL^T by the whole CTA, right-looking, one barrier
// per pivot: 4 threads per row update that row's entries left of the diagonal;
// the pivot column is read unscaled from S (never written again) and its scaled
// values go to Lo.  Pivots to Dp; then Linv = [A^-1 0; -B^-1 C A^-1  B^-1] for
// L = [A 0; C B] (32-blocks).
template <typename T>
__global__ void k_bf_diag(BigFrontDev bf, WorkList wl, int p, T* __restrict__ F, T* __restrict__ Dp,
                          T* __restrict__ Linv, const int8_t* __restrict__ dsign, double eps_d, double delta_d,
                          int* hits, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);  // NB x LD, trailing part of the block as it is eliminated
  T* Lo = S + NB * LD;                 // NB x LD, unit lower L (diagonal holds d)
  T* Li = Lo + NB * LD;                // NB x LD, L^{-1}
  __shared__ T dd[NB];
  __shared__ int8_t sgn[NB];
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b], k0 = (int64_t)p * NB;
  const int pw = (int)min((int64_t)NB, c - k0);
  T* G = F + bf.goff[b];
  const int64_t kp = bf.k0pos[b] + k0;
  const int tid = threadIdx.x;  // blockDim.x == 256
  const T eps = (T)eps_d, delta = (T)delta_d;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx % NB, j = idx / NB;
    S[i * LD + j] = (i < pw && j < pw && i >= j) ? G[(k0 + i) + (k0 + j) * f] : (T)0;
    Lo[i * LD + j] = (T)0;
    Li[i * LD + j] = (T)0;
  }
  if (tid < NB) sgn[tid] = tid < pw ? dsign[kp + tid] : (int8_t)1;
  __syncthreads();
  const int row = tid >> 2, part = tid & 3;
  for (int kk = 0; kk < pw; ++kk) {
    T d = S[kk * LD + kk];
    const bool hit = (T)sgn[kk] * d <= eps;
    if (hit) d = (T)sgn[kk] * delta;
    const T inv = (T)1 / d;
    if (tid == 0) {
      if (hit) atomicAdd(hits, 1);
      dd[kk] = d;
      Lo[kk * LD + kk] = d;
    }
    if (row > kk && row < pw) {
      const T fik = S[row * LD + kk];
      const T li = fik * inv;
      for (int j = kk + 1 + part; j <= row; j += 4) S[row * LD + j] -= li * S[j * LD + kk];
      if (part == 0) Lo[row * LD + kk] = li;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < pw * pw; idx += blockDim.x) {
    const int i = idx % pw, j = idx / pw;
    if (i >= j) G[(k0 + i) + (k0 + j) * f] = Lo[i * LD + j];
  }
  for (int i = tid; i < pw; i += blockDim.x) Dp[kp + i] = dd[i];
  const int cw0 = min(32, pw), cw1 = pw - cw0;
  const int wid = tid >> 5;
  if (wid == 0) warp_inv32(Lo, Li, 0, cw0);
  if (wid == 1 && cw1 > 0) warp_inv32(Lo, Li, 32, cw1);
  __syncthreads();
  if (cw1 > 0) {
    // X = C A^-1 (into S, free now), then Li_21 = -B^-1 X
    for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
      const int i = idx % 32, j = idx / 32;
      T acc = (T)0;
      if (i < cw1)
        for (int l = j; l < 32; ++l) acc += Lo[(32 + i) * LD + l] * Li[l * LD + j];
      S[i * LD + j] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
      const int i = idx % 32, j = idx / 32;
      if (i >= cw1) continue;
      T acc = (T)0;
      for (int l = 0; l <= i; ++l) acc += Li[(32 + i) * LD + 32 + l] * S[l * LD + j];
      Li[(32 + i) * LD + j] = -acc;
    }
    __syncthreads();
  }
  T* LB = Linv + (b * 2 + (p & 1)) * (int64_t)(NB * NB);
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx % NB, j = idx / NB;
    LB[i + j * NB] = (i < pw && j < pw) ? Li[i * LD + j] : (T)0;
  }
}

// ------------------------------------------------------------------ B: panel rows + E finalisation
template <typename T>
__global__ void k_bf_trsm(BigFrontDev bf, WorkList wl, int p, T* __restrict__ F, T* __restrict__ E,
                          const T* __restrict__ Dp, const T* __restrict__ Linv, const int* skip) {
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
  if (q < ntr) {
    const int64_t k0 = (int64_t)p * NB;
    const int pw = (int)min((int64_t)NB, c - k0);
    T* G = F + bf.goff[b];
    const int64_t r0 = k0 + pw + kTrsmRows * q;
    const int nr = (int)min((int64_t)kTrsmRows, f - r0);
    const T* LB = Linv + (b * 2 + (p & 1)) * (int64_t)(NB * NB);
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      const int i = idx % NB, j = idx / NB;
      Ls[i * LD + j] = LB[i + j * NB];
    }
    for (int idx = tid; idx < kTrsmRows * NB; idx += blockDim.x) {
      const int i = idx % kTrsmRows, j = idx / kTrsmRows;
      Xs[i * LD + j] = (i < nr && j < pw) ? G[(r0 + i) + (k0 + j) * f] : (T)0;
    }
    for (int j = tid; j < pw; j += blockDim.x) dl[j] = Dp[bf.k0pos[b] + k0 + j];
    __syncthreads();
    for (int idx = tid; idx < kTrsmRows * pw; idx += blockDim.x) {
      const int i = idx % kTrsmRows, j = idx / kTrsmRows;
      if (i >= nr) continue;
      T acc = (T)0;
      for (int l = 0; l <= j; ++l) acc += Xs[i * LD + l] * Ls[j * LD + l];
      G[(r0 + i) + (k0 + j) * f] = acc / dl[j];
    }
    return;
  }
  // finalise the E rows of panel pp = p - 1
  const int pp = p - 1;
  const int64_t e = q - ntr;
  const int64_t k0p = (int64_t)pp * NB;
  const int pwp = (int)min((int64_t)NB, c - k0p);
  const T* LB = Linv + (b * 2 + (pp & 1)) * (int64_t)(NB * NB);
  T* Eb = E + bf.eoff[b];
  if (e < pp) {
    const int64_t cb = e * NB;
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      const int i = idx % NB, j = idx / NB;
      Ls[i * LD + j] = LB[i + j * NB];
      Xs[i * LD + j] = (i < pwp) ? Eb[(k0p + i) + (cb + j) * f] : (T)0;
    }
    __syncthreads();
    for (int idx = tid; idx < pwp * NB; idx += blockDim.x) {
      const int i = idx % pwp, j = idx / pwp;
      T acc = (T)0;
      for (int l = 0; l <= i; ++l) acc += Ls[i * LD + l] * Xs[l * LD + j];
      Eb[(k0p + i) + (cb + j) * f] = acc;
    }
  } else {
    for (int idx = tid; idx < pwp * pwp; idx += blockDim.x) {
      const int i = idx % pwp, j = idx / pwp;
      if (i >= j) Eb[(k0p + i) + (k0p + j) * f] = LB[i + j * NB];
    }
  }
}

// ------------------------------------------------------------------ C: trailing and E tiles
template <typename T>
__global__ void k_bf_update(BigFrontDev bf, WorkList wl, int p, T* __restrict__ F, T* __restrict__ E,
                            const T* __restrict__ Dp, const T* __restrict__ Linv, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* As = reinterpret_cast<T*>(smraw);  // rows x K
  T* Bt = As + NB * LD;                 // cols x K
  T* Ws = Bt + NB * LD;                 // Linv
  T* Es = Ws + NB * LD;                 // E_KC
  int64_t b, q;
  locate(wl, blockIdx.x, &b, &q);
  const int64_t f = bf.f[b], c = bf.c[b], k0 = (int64_t)p * NB;
  const int pw = (int)min((int64_t)NB, c - k0);
  const int64_t t0 = k0 + pw;
  const int64_t nt = (f - t0 + NB - 1) / NB;
  const int64_t na = nt * (nt + 1) / 2;
  T* G = F + bf.goff[b];
  const T* Dk = Dp + bf.k0pos[b] + k0;
  const int tid = threadIdx.x, tr = tid % 16, tc = tid / 16;
  bool etile = q >= na;
  int64_t i0, j0 = 0, colbase = 0;
  int ncols = NB;
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
      As[r * LD + l] = (l < pw && ia < f) ? G[ia + (k0 + l) * f] : (T)0;
      Bt[r * LD + l] = (l < pw && ib < f) ? G[ib + (k0 + l) * f] * Dk[l] : (T)0;
    }
    __syncthreads();
  } else {
    const int64_t e = q - na;
    const int64_t bi = e / (p + 1), cb = e % (p + 1);
    i0 = t0 + bi * NB;
    const T* LB = Linv + (b * 2 + (p & 1)) * (int64_t)(NB * NB);
    const T* Eb = E + bf.eoff[b];
    for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
      const int r = idx % NB, l = idx / NB;
      const int64_t ia = i0 + r;
      As[r * LD + l] = (l < pw && ia < f) ? G[ia + (k0 + l) * f] : (T)0;
    }
    if (cb < p) {
      colbase = cb * NB;
      for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int i = idx % NB, j = idx / NB;
        Ws[i * LD + j] = LB[i + j * NB];
        Es[i * LD + j] = (i < pw) ? Eb[(k0 + i) + (colbase + j) * f] : (T)0;
      }
      __syncthreads();
      // Bt[cc][l] = (Linv E_KC)[l][cc]
      for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int l = idx % NB, cc = idx / NB;
        T acc = (T)0;
        for (int l2 = 0; l2 <= l; ++l2) acc += Ws[l * LD + l2] * Es[l2 * LD + cc];
        Bt[cc * LD + l] = (l < pw) ? acc : (T)0;
      }
    } else {
      colbase = k0;
      ncols = pw;
      for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int l = idx % NB, cc = idx / NB;
        Bt[cc * LD + l] = (l < pw && cc < pw) ? LB[l + cc * NB] : (T)0;
      }
    }
    __syncthreads();
  }
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  for (int l = 0; l < pw; ++l) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[(tr + 16 * a) * LD + l];
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) bv[bb] = Bt[(tc + 16 * bb) * LD + l];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
  if (!etile) {
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int64_t j = j0 + tc + 16 * bb;
      if (j >= f) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + tr + 16 * a;
        if (i < f && i >= j) G[i + j * f] -= acc[a][bb];
      }
    }
  } else {
    T* Eb = E + bf.eoff[b];
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int cc = tc + 16 * bb;
      if (cc >= ncols) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + tr + 16 * a;
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
  CLR_CUDA(cudaFuncSetAttribute(k_bf_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * NB * LD * sizeof(T)));
  (void)smem_diag;
  return CLR_OK;
}

template <typename T>
int BigFrontOps<T>::factor_level(cudaStream_t st, const BigFrontDev& bf, const BigLevelPlan& plan, T* F, T* E, T* Dp,
                                 T* Linv, const int8_t* dsign, double eps, double delta, int* hits, const int* skip) {
  const size_t s2 = 2 * NB * LD * sizeof(T), s3 = 3 * NB * LD * sizeof(T), s4 = 4 * NB * LD * sizeof(T);
  for (size_t p = 0; p < plan.A.size(); ++p) {
    if (plan.A[p].nblocks > 0)
      k_bf_diag<T><<<(unsigned)plan.A[p].nblocks, 256, s3, st>>>(bf, plan.A[p], (int)p, F, Dp, Linv, dsign, eps, delta,
                                                                  hits, skip);
    if (plan.B[p].nblocks > 0)
      k_bf_trsm<T><<<(unsigned)plan.B[p].nblocks, 256, s2, st>>>(bf, plan.B[p], (int)p, F, E, Dp, Linv, skip);
    if (plan.C[p].nblocks > 0)
      k_bf_update<T><<<(unsigned)plan.C[p].nblocks, 256, s4, st>>>(bf, plan.C[p], (int)p, F, E, Dp, Linv, skip);
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
