// Numeric multifrontal LDL^T and triangular solves (see ldl.cuh).
//
// Factor, per level of the supernodal tree (leaves first):
//   1. extend-add: every target entry of the fronts of the level sums the
//      update-matrix entries of its children in a fixed order (pull map),
//   2. partial LDL^T of each front: small fronts one CTA each in shared
//      memory; large fronts by 32-column panels (panel kernel: diagonal block
//      + row blocks of L21; update kernel: lower tiles of the trailing matrix).
// Pivots whose sign differs from the quasi-definite sign, or that are too
// small, are replaced (dynamic regularisation, Sec. 3.6).
//
// Solve: forward sweep leaves -> root (gather children's update vectors,
// unit-lower triangular solve of the front's diagonal block, update of its
// below-diagonal rows), backward sweep root -> leaves (D^{-1}, then L^T with
// the ancestors' solution gathered by KKT index).
#include <algorithm>

#include "ldl.cuh"

namespace clr {

// ------------------------------------------------------------------ factor
template <typename T>
__global__ void k_scatter_kval(T* __restrict__ F, const double* __restrict__ kval, const int64_t* __restrict__ kdest,
                               int64_t nk, const int* skip) {
  if (skip && *skip) return;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nk; p += (int64_t)gridDim.x * blockDim.x)
    F[kdest[p]] = (T)kval[p];
}

template <typename T>
__global__ void k_add_reg(T* __restrict__ F, const int64_t* __restrict__ diag_pos, const int8_t* __restrict__ dsign,
                          int64_t N, const double* delta, const int* skip) {
  if (skip && *skip) return;
  const double d = *delta;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
    F[diag_pos[k]] += (T)(dsign[k] * d);
}

template <typename T>
__global__ void k_pull(T* __restrict__ X, const int64_t* __restrict__ tgt, const int64_t* __restrict__ ptr,
                       const int64_t* __restrict__ src, int64_t t0, int64_t t1, const int* skip) {
  if (skip && *skip) return;
  for (int64_t t = t0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < t1; t += (int64_t)gridDim.x * blockDim.x) {
    T acc = X[tgt[t]];
    for (int64_t q = ptr[t]; q < ptr[t + 1]; ++q) acc += X[src[q]];
    X[tgt[t]] = acc;
  }
}

template <typename T>
__device__ __forceinline__ T regularise(T d, int sgn, T eps, T delta, bool* hit) {
  if ((T)sgn * d <= eps) {
    *hit = true;
    return (T)sgn * delta;
  }
  *hit = false;
  return d;
}

// One CTA per front with f <= small_max: whole front in shared memory.
template <typename T>
__global__ void k_factor_small(T* __restrict__ F, T* __restrict__ Dp, const int64_t* __restrict__ fronts,
                               const int64_t* __restrict__ sn_ptr, const int64_t* __restrict__ row_ptr,
                               const int64_t* __restrict__ front_off, const int8_t* __restrict__ dsign, int small_max,
                               double eps_d, double delta_d, int* dyn_hits, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);
  __shared__ T dsh;
  const int64_t J = fronts[blockIdx.x];
  const int c = (int)(sn_ptr[J + 1] - sn_ptr[J]);
  const int f = (int)(row_ptr[J + 1] - row_ptr[J]);
  if (f > small_max) return;
  T* G = F + front_off[J];
  const int64_t k0 = sn_ptr[J];
  const T eps = (T)eps_d, delta = (T)delta_d;
  for (int q = threadIdx.x; q < f * f; q += blockDim.x) S[q] = G[q];
  __syncthreads();
  for (int k = 0; k < c; ++k) {
    if (threadIdx.x == 0) {
      bool hit;
      T d = regularise(S[k + k * f], (int)dsign[k0 + k], eps, delta, &hit);
      if (hit) atomicAdd(dyn_hits, 1);
      S[k + k * f] = d;
      Dp[k0 + k] = d;
      dsh = d;
    }
    __syncthreads();
    const T inv = (T)1 / dsh;
    const int m = f - k - 1;
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
      const int i = k + 1 + q % m, j = k + 1 + q / m;
      if (i >= j) S[i + j * f] -= S[i + k * f] * S[j + k * f] * inv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < f; i += blockDim.x) S[i + k * f] *= inv;
    __syncthreads();
  }
  for (int q = threadIdx.x; q < f * f; q += blockDim.x) G[q] = S[q];
}

// Large fronts, panel of pw <= 32 columns starting at k0.
// k_big_diag (one warp): LDL^T of the pw x pw diagonal block, in place, pivots to Dp.
template <typename T>
__global__ void k_big_diag(T* __restrict__ G, int64_t f, int64_t k0, int pw, T* __restrict__ Dp,
                           const int8_t* __restrict__ dsg, double eps_d, double delta_d, int* dyn_hits,
                           const int* skip) {
  if (skip && *skip) return;
  __shared__ T Ld[32][33];
  __shared__ T dd[32];
  const int tid = threadIdx.x;  // blockDim.x == 32
  for (int j = 0; j < 32; ++j) Ld[tid][j] = (tid < pw && j < pw && tid >= j) ? G[(k0 + tid) + (k0 + j) * f] : (T)0;
  __syncwarp();
  const T eps = (T)eps_d, delta = (T)delta_d;
  for (int kk = 0; kk < pw; ++kk) {
    if (tid == 0) {
      bool hit;
      T d = regularise(Ld[kk][kk], (int)dsg[k0 + kk], eps, delta, &hit);
      if (hit) atomicAdd(dyn_hits, 1);
      Ld[kk][kk] = d;
      dd[kk] = d;
    }
    __syncwarp();
    const T inv = (T)1 / dd[kk];
    if (tid > kk && tid < pw) {
      const T lik = Ld[tid][kk];
      for (int j = kk + 1; j <= tid; ++j) Ld[tid][j] -= lik * Ld[j][kk] * inv;
    }
    __syncwarp();
    if (tid > kk && tid < pw) Ld[tid][kk] *= inv;
    __syncwarp();
  }
  for (int j = 0; j < pw; ++j)
    if (tid >= j && tid < pw) G[(k0 + tid) + (k0 + j) * f] = Ld[tid][j];
  if (tid < pw) Dp[k0 + tid] = dd[tid];
}

// k_big_trsm: rows r0 = k0+pw+32 b ... of L21 = F21 L11^{-T} D^{-1}, one row per thread,
// reading the factored diagonal block written by k_big_diag.
template <typename T>
__global__ void k_big_trsm(T* __restrict__ G, int64_t f, int64_t k0, int pw, const T* __restrict__ Dp,
                           const int* skip) {
  if (skip && *skip) return;
  __shared__ T Ld[32][33];
  __shared__ T dd[32];
  const int tid = threadIdx.x;  // blockDim.x == 32
  for (int j = 0; j < 32; ++j) Ld[tid][j] = (tid < pw && j < pw && tid > j) ? G[(k0 + tid) + (k0 + j) * f] : (T)0;
  if (tid < pw) dd[tid] = Dp[k0 + tid];
  __syncwarp();
  const int64_t r = k0 + pw + (int64_t)blockIdx.x * 32 + tid;
  if (r >= f) return;
  T x[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (j < pw) {
      T v = G[r + (k0 + j) * f];
      for (int l = 0; l < j; ++l) v -= x[l] * dd[l] * Ld[j][l];
      x[j] = v / dd[j];
    }
  }
#pragma unroll
  for (int j = 0; j < 32; ++j)
    if (j < pw) G[r + (k0 + j) * f] = x[j];
}

// Trailing update of a large front: C(i, j) -= sum_l L(i, l) d_l L(j, l) over
// the panel columns, lower tiles of 64 x 64 (256 threads, 4 x 4 per thread).
template <typename T>
__global__ void k_big_update(T* __restrict__ G, int64_t f, int64_t k0, int pw, const T* __restrict__ Dp, int64_t t0,
                             const int* skip) {
  if (skip && *skip) return;
  constexpr int TS = 64;
  __shared__ T As[TS][33];
  __shared__ T Bs[TS][33];
  // lower-tile index -> (bi, bj), bi >= bj
  const int64_t bid = blockIdx.x;
  int64_t bi = (int64_t)((sqrt(8.0 * (double)bid + 1.0) - 1.0) / 2.0);
  while (bi * (bi + 1) / 2 > bid) --bi;
  while ((bi + 1) * (bi + 2) / 2 <= bid) ++bi;
  const int64_t bj = bid - bi * (bi + 1) / 2;
  const int64_t i0 = t0 + bi * TS, j0 = t0 + bj * TS;
  const int tid = threadIdx.x;
  for (int q = tid; q < TS * 32; q += blockDim.x) {
    const int rr = q % TS, l = q / TS;
    const int64_t ia = i0 + rr, ib = j0 + rr;
    As[rr][l] = (l < pw && ia < f) ? G[ia + (k0 + l) * f] : (T)0;
    Bs[rr][l] = (l < pw && ib < f) ? G[ib + (k0 + l) * f] * Dp[k0 + l] : (T)0;
  }
  __syncthreads();
  const int tr = tid % 16, tc = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
  for (int l = 0; l < pw; ++l) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[tr + 16 * a][l];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[tc + 16 * b][l];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int64_t j = j0 + tc + 16 * b;
    if (j >= f) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t i = i0 + tr + 16 * a;
      if (i < f && i >= j) G[i + j * f] -= acc[a][b];
    }
  }
}

// ------------------------------------------------------------------ solve
template <typename T>
__global__ void k_init_w(T* __restrict__ w, const int32_t* __restrict__ w_init, const double* __restrict__ rhs,
                         int64_t wtot, const int* skip) {
  if (skip && *skip) return;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < wtot; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = w_init[q];
    w[q] = (i >= 0) ? (T)rhs[i] : (T)0;
  }
}

// Forward sweep of one front per CTA: unit lower solve of the c x c diagonal
// block in 32-column blocks (warp 0), then the rows below each block.
template <typename T>
__global__ void k_fwd_front(const T* __restrict__ F, T* __restrict__ w, const int64_t* __restrict__ fronts,
                            const int64_t* __restrict__ sn_ptr, const int64_t* __restrict__ row_ptr,
                            const int64_t* __restrict__ front_off, const int64_t* __restrict__ upd_off,
                            const int* skip) {
  if (skip && *skip) return;
  __shared__ T xb[32];
  const int64_t J = fronts[blockIdx.x];
  const int64_t c = sn_ptr[J + 1] - sn_ptr[J];
  const int64_t f = row_ptr[J + 1] - row_ptr[J];
  const T* G = F + front_off[J];
  T* wj = w + upd_off[J];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t j0 = 0; j0 < c; j0 += 32) {
    const int jb = (int)min((int64_t)32, c - j0);
    if (wid == 0) {
      T xi = (lane < jb) ? wj[j0 + lane] : (T)0;
      for (int jj = 0; jj < jb; ++jj) {
        const T xj = __shfl_sync(0xffffffffu, xi, jj);
        if (lane > jj && lane < jb) xi -= G[(j0 + lane) + (j0 + jj) * f] * xj;
      }
      if (lane < jb) {
        wj[j0 + lane] = xi;
        xb[lane] = xi;
      }
    }
    __syncthreads();
    for (int64_t i = j0 + jb + threadIdx.x; i < f; i += blockDim.x) {
      T s = (T)0;
      for (int jj = 0; jj < jb; ++jj) s += G[i + (j0 + jj) * f] * xb[jj];
      wj[i] -= s;
    }
    __syncthreads();
  }
}

// Backward sweep of one front per CTA: v = y / D, then L^T x = v with the
// solution of the ancestors (rows c .. f-1) gathered from xs by KKT index.
template <typename T>
__global__ void k_bwd_front(const T* __restrict__ F, const T* __restrict__ Dp, T* __restrict__ w, T* __restrict__ xs,
                            const int64_t* __restrict__ fronts, const int64_t* __restrict__ sn_ptr,
                            const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ front_off,
                            const int64_t* __restrict__ upd_off, const int32_t* __restrict__ rows_kkt,
                            const int* skip) {
  if (skip && *skip) return;
  const int64_t J = fronts[blockIdx.x];
  const int64_t c = sn_ptr[J + 1] - sn_ptr[J];
  const int64_t f = row_ptr[J + 1] - row_ptr[J];
  const T* G = F + front_off[J];
  T* X = w + upd_off[J];
  const int32_t* rk = rows_kkt + row_ptr[J];
  const T* D = Dp + sn_ptr[J];
  for (int64_t i = threadIdx.x; i < f; i += blockDim.x) X[i] = (i < c) ? X[i] / D[i] : xs[rk[i]];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t j1 = c; j1 > 0; j1 -= 32) {
    const int64_t j0 = max((int64_t)0, j1 - 32);
    // v[k] -= sum_{i >= j1} L(i, k) x_i for k in [j0, j1): one warp per column
    for (int64_t k = j0 + wid; k < j1; k += nw) {
      T s = (T)0;
      for (int64_t i = j1 + lane; i < f; i += 32) s += G[i + k * f] * X[i];
      s = warp_sum(s);
      if (lane == 0) X[k] -= s;
    }
    __syncthreads();
    if (wid == 0) {
      const int jb = (int)(j1 - j0);
      T vi = (lane < jb) ? X[j0 + lane] : (T)0;
      for (int kk = jb - 1; kk >= 0; --kk) {
        const T xk = __shfl_sync(0xffffffffu, vi, kk);
        if (lane < kk) vi -= G[(j0 + kk) + (j0 + lane) * f] * xk;
      }
      if (lane < jb) X[j0 + lane] = vi;
    }
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < c; i += blockDim.x) xs[rk[i]] = X[i];
}

// ------------------------------------------------------------------ host side
namespace {
template <typename T>
T* up(DeviceArena& ar, const std::vector<T>& v) {
  return ar.upload(v.data(), (int64_t)v.size());
}
}  // namespace

int ldl_structure_upload(DeviceArena& ar, const Symbolic& sy, const NumericMaps& mp, const std::vector<int8_t>& dsign,
                         int small_max, LdlStructure& st) {
  st.N = sy.N;
  st.nsn = sy.nsn;
  st.nlev = sy.nlev;
  st.pool = sy.pool;
  st.wtot = sy.upd_total;
  st.nk = (int64_t)mp.kdest.size();
  st.small_max = small_max;
  st.max_front = sy.max_front;
  st.h_lev_ptr = sy.lev_ptr;
  st.h_lev_sn = sy.lev_sn;
  st.h_fa_lev_ptr = mp.fa_lev_ptr;
  st.h_sv_lev_ptr = mp.sv_lev_ptr;
  st.h_sn_ptr = sy.sn_ptr;
  st.h_row_ptr = sy.row_ptr;
  st.h_front_off = sy.front_off;
  std::vector<int32_t> w_init(sy.upd_total, -1);
  for (int64_t J = 0; J < sy.nsn; ++J) {
    const int64_t c = sy.sn_ptr[J + 1] - sy.sn_ptr[J];
    for (int64_t k = 0; k < c; ++k) w_init[sy.upd_off[J] + k] = mp.rows_kkt[sy.row_ptr[J] + k];
  }
  st.lev_small_maxf.assign(sy.nlev, 0);
  st.lev_big.assign(sy.nlev, {});
  for (int64_t l = 0; l < sy.nlev; ++l)
    for (int64_t t = sy.lev_ptr[l]; t < sy.lev_ptr[l + 1]; ++t) {
      const int64_t J = sy.lev_sn[t];
      const int64_t f = sy.row_ptr[J + 1] - sy.row_ptr[J];
      if (f > small_max) st.lev_big[l].push_back(J);
      else st.lev_small_maxf[l] = std::max(st.lev_small_maxf[l], (int)f);
    }
  st.sn_ptr = up(ar, sy.sn_ptr);
  st.row_ptr = up(ar, sy.row_ptr);
  st.front_off = up(ar, sy.front_off);
  st.upd_off = up(ar, sy.upd_off);
  st.lev_sn = up(ar, sy.lev_sn);
  st.rows_kkt = up(ar, mp.rows_kkt);
  st.w_init = up(ar, w_init);
  st.dsign = up(ar, dsign);
  st.kdest = up(ar, mp.kdest);
  st.diag_pos = up(ar, mp.diag_pos);
  st.fa_tgt = up(ar, mp.fa_tgt);
  st.fa_ptr = up(ar, mp.fa_ptr);
  st.fa_src = up(ar, mp.fa_src);
  st.sv_tgt = up(ar, mp.sv_tgt);
  st.sv_ptr = up(ar, mp.sv_ptr);
  st.sv_src = up(ar, mp.sv_src);
  if (!st.sn_ptr || !st.row_ptr || !st.front_off || !st.upd_off || !st.lev_sn || !st.rows_kkt || !st.w_init ||
      !st.dsign || !st.kdest || !st.diag_pos || !st.fa_tgt || !st.fa_ptr || !st.fa_src || !st.sv_tgt ||
      !st.sv_ptr || !st.sv_src)
    return CLR_E_OOM;
  return CLR_OK;
}

template <typename T>
int LdlFactor<T>::alloc(DeviceArena& ar, const LdlStructure& st) {
  s = &st;
  F = ar.alloc_n<T>(st.pool);
  Dp = ar.alloc_n<T>(st.N);
  w = ar.alloc_n<T>(st.wtot);
  xs = ar.alloc_n<T>(st.N);
  dyn_hits = ar.alloc_n<int>(1);
  if (!F || !Dp || !w || !xs || !dyn_hits) return CLR_E_OOM;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_factor_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  return CLR_OK;
}

template <typename T>
int LdlFactor<T>::factor(cudaStream_t stm, const double* kval, const double* delta, double dyn_eps, double dyn_delta,
                         const int* skip) const {
  const LdlStructure& S = *s;
  CLR_CUDA(cudaMemsetAsync(dyn_hits, 0, sizeof(int), stm));
  CLR_CUDA(cudaMemsetAsync(F, 0, sizeof(T) * (size_t)S.pool, stm));
  k_scatter_kval<T><<<grid_for(S.nk, 256), 256, 0, stm>>>(F, kval, S.kdest, S.nk, skip);
  k_add_reg<T><<<grid_for(S.N, 256), 256, 0, stm>>>(F, S.diag_pos, S.dsign, S.N, delta, skip);
  CLR_CHECK_LAUNCH();
  for (int64_t l = 0; l < S.nlev; ++l) {
    const int64_t t0 = S.h_fa_lev_ptr[l], t1 = S.h_fa_lev_ptr[l + 1];
    if (t1 > t0) k_pull<T><<<grid_for(t1 - t0, 256), 256, 0, stm>>>(F, S.fa_tgt, S.fa_ptr, S.fa_src, t0, t1, skip);
    const int64_t nf = S.h_lev_ptr[l + 1] - S.h_lev_ptr[l];
    if ((int64_t)S.lev_big[l].size() < nf) {
      const int mf = S.lev_small_maxf[l];
      const size_t smem = sizeof(T) * (size_t)mf * (size_t)mf;
      const int threads = mf <= 16 ? 64 : (mf <= 48 ? 128 : 256);
      k_factor_small<T><<<(unsigned)nf, threads, smem, stm>>>(F, Dp, S.lev_sn + S.h_lev_ptr[l], S.sn_ptr, S.row_ptr,
                                                               S.front_off, S.dsign, S.small_max, dyn_eps, dyn_delta,
                                                               dyn_hits, skip);
    }
    for (int64_t J : S.lev_big[l]) {
      const int64_t c = S.h_sn_ptr[J + 1] - S.h_sn_ptr[J];
      const int64_t f = S.h_row_ptr[J + 1] - S.h_row_ptr[J];
      T* G = F + S.h_front_off[J];
      T* DpJ = Dp + S.h_sn_ptr[J];
      const int8_t* dsJ = S.dsign + S.h_sn_ptr[J];
      for (int64_t k0 = 0; k0 < c; k0 += 32) {
        const int pw = (int)std::min<int64_t>(32, c - k0);
        const int64_t below = f - k0 - pw;
        k_big_diag<T><<<1, 32, 0, stm>>>(G, f, k0, pw, DpJ, dsJ, dyn_eps, dyn_delta, dyn_hits, skip);
        if (below > 0) {
          k_big_trsm<T><<<(unsigned)((below + 31) / 32), 32, 0, stm>>>(G, f, k0, pw, DpJ, skip);
          const int64_t nt = (below + 63) / 64;
          k_big_update<T><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, stm>>>(G, f, k0, pw, DpJ, k0 + pw, skip);
        }
      }
    }
    CLR_CHECK_LAUNCH();
  }
  return CLR_OK;
}

template <typename T>
int LdlFactor<T>::solve(cudaStream_t stm, const double* rhs, const int* skip) const {
  const LdlStructure& S = *s;
  k_init_w<T><<<grid_for(S.wtot, 256), 256, 0, stm>>>(w, S.w_init, rhs, S.wtot, skip);
  for (int64_t l = 0; l < S.nlev; ++l) {
    const int64_t t0 = S.h_sv_lev_ptr[l], t1 = S.h_sv_lev_ptr[l + 1];
    if (t1 > t0) k_pull<T><<<grid_for(t1 - t0, 256), 256, 0, stm>>>(w, S.sv_tgt, S.sv_ptr, S.sv_src, t0, t1, skip);
    const int64_t nf = S.h_lev_ptr[l + 1] - S.h_lev_ptr[l];
    k_fwd_front<T><<<(unsigned)nf, 256, 0, stm>>>(F, w, S.lev_sn + S.h_lev_ptr[l], S.sn_ptr, S.row_ptr, S.front_off,
                                                   S.upd_off, skip);
  }
  for (int64_t l = S.nlev - 1; l >= 0; --l) {
    const int64_t nf = S.h_lev_ptr[l + 1] - S.h_lev_ptr[l];
    k_bwd_front<T><<<(unsigned)nf, 256, 0, stm>>>(F, Dp, w, xs, S.lev_sn + S.h_lev_ptr[l], S.sn_ptr, S.row_ptr,
                                                  S.front_off, S.upd_off, S.rows_kkt, skip);
  }
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

template struct LdlFactor<double>;
template struct LdlFactor<float>;

}  // namespace clr
