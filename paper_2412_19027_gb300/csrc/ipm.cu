// Per-iteration device step of Algorithm 1 (arXiv:2412.19027) and the solver
// object.  Every step of an iteration runs in the kernels below or in
// cones.cu / ldl.cu; the host only launches them (replaying one captured CUDA
// graph per iteration) and reads back the status words.
//
// A solver holds a cohort of B >= 1 problems merged block-diagonally
// (cohort.cpp): x = [x_1; ...; x_B], the constraint rows family-major (all
// zero rows, all nonneg rows, SOCs, exp, pow, PSD cones; each problem's rows in
// problem order inside a family).  Every scalar of the method is per problem
// (IterScal[B]); vector reductions run over chunks that never straddle two
// problems and are summed per problem in a fixed order, so a problem's
// iterates do not depend on the rest of its cohort.
//
// Scaled space: the device holds P^ = c D P D, q^ = c D q, A^ = E A D,
// b^ = E b (setup.cpp) and iterates x^, s^, z^, tau, kappa; residuals and the
// termination tests (Eq. residuals-objectives, termination-check,
// infeasibility-check) are evaluated on the unscaled quantities
// x = D x^, s = s^ / E, z = E z^ / c.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ipm.cuh"

namespace clr {

// ------------------------------------------------------------------ slots
enum SumSlot { S_XPX = 0, S_QX, S_BZ, S_SZ, S_D0, S_D1, S_D2, S_NSLOT };
enum MaxSlot { M_RD = 0, M_X, M_RP, M_S, M_Z, M_ATZ, M_PX, M_AXS, M_GS, M_NMAX };

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// Launch geometry of the chunked kernels: one block per chunk, x chunks first.
struct ChunkGrid {
  const Chunk* ck;
  int64_t nckx, pst, n;  // pst: stride of a partial-sum slot
  int64_t zaux = INT64_MAX;  // first auxiliary row of the expanded SOCs (kernels that keep them at 0)
};
// KKT index range of block b's chunk: [i0, i0 + len); z chunks start at n.
__device__ __forceinline__ void chunk_range(const ChunkGrid& g, int64_t* i0, int64_t* len, int* pid, bool* zpart) {
  const Chunk c = g.ck[blockIdx.x];
  *zpart = blockIdx.x >= g.nckx;
  *i0 = *zpart ? g.n + c.begin : c.begin;
  *len = c.len;
  *pid = c.pid;
}
// index of block b's chunk inside its own (x or z) list
__device__ __forceinline__ int64_t chunk_slot(const ChunkGrid& g) {
  return blockIdx.x >= g.nckx ? blockIdx.x - g.nckx : blockIdx.x;
}

// ------------------------------------------------------------------ K products
// G lanes per row of the full (both triangles) KKT CSR; values through kvi into kval.
// mode 0: lo[i] = sum_{col < n} K_ij v_j, hi[i] = sum_{col >= n} K_ij v_j
// mode 1: out[i] = rhs[i] - (K v)_i and max |out| of each problem -> sc[p].rnorm_bits
// mode 2 (rows n..N-1): out[i-n] = -rhs[i-n] + hi   (Delta s = -d_s - H Delta z; K_zz = -H)
// The sum of a row is formed in one fixed order whatever G is (32 partial sums,
// entry e of the row going to partial e mod 32, then the pairwise tree t += t+16,
// t += t+8, ...), so a row gives the same bits in every cohort it belongs to.
// Rows longer than this go to k_kmv_long (a CTA per row); each row's sum is taken
// in an order fixed by its length alone, so a problem's K products are the same
// alone and in a cohort.
constexpr int64_t kLongRow = 512;

template <int G>
__global__ void k_kmv(int mode, int64_t r0, int64_t r1, int64_t n, const int64_t* __restrict__ kptr,
                      const int32_t* __restrict__ kcol, const int32_t* __restrict__ kvi, const double* __restrict__ kval,
                      const double* __restrict__ kfv,
                      const double* __restrict__ v, double* __restrict__ lo, double* __restrict__ hi,
                      const double* __restrict__ rhs, double* __restrict__ out, const int32_t* __restrict__ pid,
                      IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  constexpr int NU = 32 / G;  // partial sums per lane: t = lane + G u
  const int lane = threadIdx.x % G;
  // the G lanes of a row group share its trip count: shuffles name only their own group
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t gstride = ((int64_t)gridDim.x * blockDim.x) / G;
  RunExt<true> mx;
  for (int64_t i = r0 + gid; i < r1; i += gstride) {
    double a[NU], b[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) a[u] = b[u] = 0.0;
    const int64_t p0 = kptr[i], p1 = kptr[i + 1];
    if (p1 - p0 > kLongRow) continue;  // k_kmv_long (the whole G-lane group skips)
    // four 32-entry steps per pass: all loads of the pass issued before the adds,
    // which keep the order of the plain one-step loop (partial t sums entries
    // p = p0 + t (mod 32) in increasing p)
    for (int64_t base = p0; base < p1; base += 128) {
      double tv[4][NU];
      bool tx[4][NU];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int64_t p = base + 32 * k + lane + G * u;
          tv[k][u] = 0.0;
          tx[k][u] = true;
          if (p < p1) {
            const int32_t c = kcol[p];
            tv[k][u] = (i < n ? kfv[p] : kval[kvi[p]]) * v[c];
            tx[k][u] = c < n;
          }
        }
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          if (base + 32 * k + lane + G * u >= p1) continue;
          if (tx[k][u]) a[u] += tv[k][u];
          else b[u] += tv[k][u];
        }
    }
#pragma unroll
    for (int off = 16; off >= G; off >>= 1)
#pragma unroll
      for (int u = 0; u < off / G; ++u) {
        a[u] += a[u + off / G];
        b[u] += b[u + off / G];
      }
#pragma unroll
    for (int off = (G == 32 ? 16 : G / 2); off > 0; off >>= 1) {
      a[0] += __shfl_xor_sync(gmask, a[0], off, G);
      b[0] += __shfl_xor_sync(gmask, b[0], off, G);
    }
    if (lane == 0) {
      if (mode == 0) {
        lo[i] = a[0];
        hi[i] = b[0];
      } else if (mode == 1) {
        const double r = rhs[i] - (a[0] + b[0]);
        out[i] = r;
        mx.add(sc, &IterScal::rnorm_bits, pid[i], dbits(fabs(r)));
      } else {
        out[i - n] = -rhs[i - n] + b[0];
      }
    }
  }
  if (mode == 1) mx.flush(sc, &IterScal::rnorm_bits);
}

// The long rows: 8 warps per row, warp w sums the w-th of 8 contiguous segments of
// 32-entry steps (lane t: entries p = p0 + t (mod 32)), the 8 partials of a lane are
// added in warp order, then the 32 lanes by the same butterfly as k_kmv.  Outputs
// as k_kmv for the modes.
__global__ void __launch_bounds__(256)
    k_kmv_long(int mode, const int64_t* __restrict__ rows, int64_t nrows, int64_t n, const int64_t* __restrict__ kptr,
               const int32_t* __restrict__ kcol, const int32_t* __restrict__ kvi, const double* __restrict__ kval,
               const double* __restrict__ kfv,
               const double* __restrict__ v, double* __restrict__ lo, double* __restrict__ hi,
               const double* __restrict__ rhs, double* __restrict__ out, const int32_t* __restrict__ pid,
               IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  __shared__ double pa[8][32], pb[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  RunExt<true> mx;
  for (int64_t t = blockIdx.x; t < nrows; t += gridDim.x) {
    const int64_t i = rows[t];
    const int64_t p0 = kptr[i], p1 = kptr[i + 1];
    const int64_t S = ((p1 - p0 + 255) / 256) * 32;  // segment length, a multiple of 32
    const int64_t s0 = p0 + w * S, s1 = min(p1, s0 + S);
    double a = 0.0, b = 0.0;
    for (int64_t base = s0; base < s1; base += 128) {
      double tv[4];
      bool tx[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t p = base + 32 * k + lane;
        tv[k] = 0.0;
        tx[k] = true;
        if (p < s1) {
          const int32_t c = kcol[p];
          tv[k] = (i < n ? kfv[p] : kval[kvi[p]]) * v[c];
          tx[k] = c < n;
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (base + 32 * k + lane >= s1) continue;
        if (tx[k]) a += tv[k];
        else b += tv[k];
      }
    }
    pa[w][lane] = a;
    pb[w][lane] = b;
    __syncthreads();
    if (w == 0) {
      a = pa[0][lane];
      b = pb[0][lane];
#pragma unroll
      for (int q = 1; q < 8; ++q) {
        a += pa[q][lane];
        b += pb[q][lane];
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
      }
      if (lane == 0) {
        if (mode == 0) {
          lo[i] = a;
          hi[i] = b;
        } else if (mode == 1) {
          const double r = rhs[i] - (a + b);
          out[i] = r;
          mx.add(sc, &IterScal::rnorm_bits, pid[i], dbits(fabs(r)));
        } else {
          out[i - n] = -rhs[i - n] + b;
        }
      }
    }
    __syncthreads();
  }
  if (mode == 1 && w == 0) mx.flush(sc, &IterScal::rnorm_bits);
}

// launch k_kmv_long for the long rows in [r0, r1)
void kmv_long(cudaStream_t s, int mode, int64_t r0, int64_t r1, int64_t n, const VecDev& v,
              const std::vector<int64_t>& h_long, const double* x, double* lo, double* hi, const double* rhs,
              double* out, IterScal* sc, const int* skip) {
  if (h_long.empty()) return;
  const int64_t a = std::lower_bound(h_long.begin(), h_long.end(), r0) - h_long.begin();
  const int64_t b = std::lower_bound(h_long.begin(), h_long.end(), r1) - h_long.begin();
  if (b <= a) return;
  const unsigned g = (unsigned)std::min<int64_t>(b - a, 16 * kSMs);  // a row per CTA, up to 16 CTAs per SM
  k_kmv_long<<<g, 256, 0, s>>>(mode, v.long_rows + a, b - a, n, v.kptr, v.kcol, v.kvi, v.kval, v.kfv, x, lo, hi, rhs,
                               out, v.pid, sc, skip);
}

// ------------------------------------------------------------------ residuals
// x chunks: G1 = -(P x + A' z + q tau), qp = q + 2 P x / tau, sums x'Px, q'x and maxima;
// z chunks: G2 = s + A x - b tau, sums b'z, s'z and maxima.
__global__ void k_resid(ChunkGrid g, const double* __restrict__ xz, const double* __restrict__ s,
                        const double* __restrict__ lo, const double* __restrict__ hi, const double* __restrict__ q,
                        const double* __restrict__ b, const double* __restrict__ D, const double* __restrict__ E,
                        const IterScal* sc, double* __restrict__ G, double* __restrict__ qp, double* part,
                        unsigned long long* maxb, const int* skip) {
  if (skip && *skip) return;
  __shared__ double sh[32];
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  const int64_t slot = chunk_slot(g);
  const double tau = sc[pid].tau;
  unsigned long long* mb = maxb + (int64_t)M_NMAX * pid;
  double s0 = 0, s1 = 0, m0 = 0, m1 = 0, m2 = 0, m3 = 0, m4 = 0;
  if (!zp) {
    for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x) {
      const double x = xz[i], px = lo[i], atz = hi[i], qi = q[i], di = D[i];
      const double g1 = -(px + atz + qi * tau);
      G[i] = g1;
      qp[i] = qi + 2.0 * px / tau;
      s0 += x * px;
      s1 += qi * x;
      m0 = fmax(m0, fabs(g1) / di);
      m1 = fmax(m1, fabs(di * x));
      m2 = fmax(m2, fabs(atz) / di);
      m3 = fmax(m3, fabs(px) / di);
      m4 = fmax(m4, fabs(g1));
    }
  } else {
    const int64_t n = g.n;
    for (int64_t k = i0 + threadIdx.x; k < i0 + len; k += blockDim.x) {
      const int64_t i = k - n;
      const double zi = xz[k], si = s[i], ax = lo[k], bi = b[i], ei = E[i];
      const double g2 = si + ax - bi * tau;
      G[k] = g2;
      s0 += bi * zi;
      s1 += si * zi;
      m0 = fmax(m0, fabs(g2) / ei);
      m1 = fmax(m1, fabs(si) / ei);
      m2 = fmax(m2, fabs(ei * zi));
      m3 = fmax(m3, fabs(ax + si) / ei);
      m4 = fmax(m4, fabs(g2));
    }
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  m0 = block_max(m0, sh);
  m1 = block_max(m1, sh);
  m2 = block_max(m2, sh);
  m3 = block_max(m3, sh);
  m4 = block_max(m4, sh);
  if (threadIdx.x == 0) {
    atomicMax(mb + M_GS, dbits(m4));
    part[(zp ? S_BZ : S_XPX) * g.pst + slot] = s0;
    part[(zp ? S_SZ : S_QX) * g.pst + slot] = s1;
    if (!zp) {
      atomicMax(mb + M_RD, dbits(m0));
      atomicMax(mb + M_X, dbits(m1));
      atomicMax(mb + M_ATZ, dbits(m2));
      atomicMax(mb + M_PX, dbits(m3));
    } else {
      atomicMax(mb + M_RP, dbits(m0));
      atomicMax(mb + M_S, dbits(m1));
      atomicMax(mb + M_Z, dbits(m2));
      atomicMax(mb + M_AXS, dbits(m3));
    }
  }
}

// Sum of slot `slot` over chunks [c0, c1) of one problem, in a fixed order; valid in thread 0.
__device__ double fin_sum(const double* part, int slot, int64_t pst, int64_t c0, int64_t c1) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) v += part[slot * pst + c];
  v = block_sum(v, sh);
  __syncthreads();
  return v;
}

// Transition of problem p to "stopped": the last one to stop raises all_halt.
__device__ void halt_problem(IterScal& q, BatchFlags* bf) {
  if (q.halt) return;
  q.halt = 1;
  if (atomicSub(&bf->n_running, 1) == 1) bf->all_halt = 1;
}

struct TermParams {
  double eps_feas, eps_inf;
  int max_iter;
  int hist_cap;
};

// Residuals, objectives, mu and the termination / infeasibility tests; one block per problem.
__global__ void k_fin_resid(IterScal* scs, const ProbConst* pcs, const double* part, int64_t pst,
                            const int64_t* ckx_ptr, const int64_t* ckz_ptr, const unsigned long long* maxb,
                            TermParams tp, double* hist, BatchFlags* bf, const int* skip) {
  if (skip && *skip) return;
  const int64_t p = blockIdx.x;
  IterScal& sc = scs[p];
  if (sc.halt) return;
  const double xpx = fin_sum(part, S_XPX, pst, ckx_ptr[p], ckx_ptr[p + 1]);
  const double qx = fin_sum(part, S_QX, pst, ckx_ptr[p], ckx_ptr[p + 1]);
  const double bz = fin_sum(part, S_BZ, pst, ckz_ptr[p], ckz_ptr[p + 1]);
  const double sz = fin_sum(part, S_SZ, pst, ckz_ptr[p], ckz_ptr[p + 1]);
  if (threadIdx.x != 0) return;
  const ProbConst pc = pcs[p];
  const unsigned long long* mb = maxb + (int64_t)M_NMAX * p;
  const double tau = sc.tau, kappa = sc.kappa, c = pc.c;
  const double mu = (sz + kappa * tau) / (double)(pc.nu + 1);
  const double nrp = bitsd(mb[M_RP]) / tau;
  const double nrd = bitsd(mb[M_RD]) / (c * tau);
  const double nx = bitsd(mb[M_X]) / tau, ns = bitsd(mb[M_S]) / tau, nz = bitsd(mb[M_Z]) / (c * tau);
  const double gp = (0.5 * xpx / (tau * tau) + qx / tau) / c;
  const double gd = (-0.5 * xpx / (tau * tau) - bz / tau) / c;
  const double gap = fabs(gp - gd);
  sc.mu = mu;
  sc.g_scaled = bitsd(mb[M_GS]);
  sc.xPx = xpx;
  sc.qx = qx;
  sc.bz = bz;
  sc.sz = sz;
  sc.G3 = kappa + qx + bz + xpx / tau;
  sc.pcost = gp;
  sc.dcost = gd;
  sc.res_p = nrp;
  sc.res_d = nrd;
  sc.gap_abs = gap;
  sc.gap_rel = gap / fmax(1.0, fmin(fabs(gp), fabs(gd)));
  int status = 0;
  if (!isfinite(mu) || !isfinite(nrp) || !isfinite(nrd) || !isfinite(gp) || !isfinite(gd) || !isfinite(tau) ||
      !isfinite(kappa)) {
    status = CLR_NUMERICAL_ERROR;
  } else if (nrp < tp.eps_feas * fmax(1.0, pc.bnorm + nx + ns) && nrd < tp.eps_feas * fmax(1.0, pc.qnorm + nx + nz) &&
             gap < tp.eps_feas * fmax(1.0, fmin(fabs(gp), fabs(gd)))) {
    status = CLR_SOLVED;
  } else {
    // infeasibility on the unnormalised unscaled iterates
    const double btz = bz / c, qtx = qx / c;
    const double nxu = bitsd(mb[M_X]), nzu = bitsd(mb[M_Z]) / c, nsu = bitsd(mb[M_S]);
    const double natz = bitsd(mb[M_ATZ]) / c, npx = bitsd(mb[M_PX]) / c, naxs = bitsd(mb[M_AXS]);
    if (btz < -tp.eps_inf && natz < -tp.eps_inf * fmax(1.0, nxu + nzu) * btz) status = CLR_PRIMAL_INFEASIBLE;
    else if (qtx < -tp.eps_inf && npx < -tp.eps_inf * fmax(1.0, nxu) * qtx &&
             naxs < -tp.eps_inf * fmax(1.0, nxu + nsu) * qtx)
      status = CLR_DUAL_INFEASIBLE;
    else if (sc.iter >= tp.max_iter)
      status = CLR_MAX_ITER;
  }
  sc.status = status;
  sc.feas_ratio = fmax(nrp / (tp.eps_feas * fmax(1.0, pc.bnorm + nx + ns)),
                       nrd / (tp.eps_feas * fmax(1.0, pc.qnorm + nx + nz)));
  if (status == 0) {
    // the complementarity gap still falls while the residuals stay: with a
    // low-precision factor, the accuracy of the KKT solves is what holds them up
    const double feas = sc.feas_ratio;
    if (sc.feas_best == 0.0 || feas < 0.5 * sc.feas_best) {
      sc.feas_best = feas;
      sc.mu_at_best = mu;
      sc.feas_stall = 0;
    } else if (feas < 1e6 && mu < 0.1 * sc.mu_at_best) {
      sc.feas_stall += 1;
    }
  }
  if (sc.iter < tp.hist_cap) {
    double* h = hist + (int64_t)12 * tp.hist_cap * p + 12 * sc.iter;
    h[0] = sc.iter;
    h[1] = mu;
    h[2] = gp;
    h[3] = gd;
    h[4] = nrp;
    h[5] = nrd;
    h[6] = gap;
    h[7] = h[8] = h[9] = h[10] = 0.0;
    h[11] = tau;
  }
  if (status != 0) halt_problem(sc, bf);
}

// ------------------------------------------------------------------ per-problem small kernels
// problems p = tid, tid + stride, ...
#define FOR_PROBLEMS(B) \
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < (B); p += (int64_t)gridDim.x * blockDim.x)

__global__ void k_hmax_reset(IterScal* sc, int64_t B, const int* skip) {
  if (skip && *skip) return;
  FOR_PROBLEMS(B) {
    sc[p].hmax_bits = 0ull;
    sc[p].ir_fail = 0;
    sc[p].escalate = 0;
    sc[p].ir_worst = 0.0;
  }
}

// static + proportional regularisation
__global__ void k_fin_delta(IterScal* sc, const ProbConst* pc, int64_t B, double static_reg, double static_reg_dyn,
                            const int* skip) {
  if (skip && *skip) return;
  FOR_PROBLEMS(B)
  sc[p].delta = static_reg * fmax(1.0, sc[p].reg_boost) + static_reg_dyn * fmax(pc[p].maxPdiag, bitsd(sc[p].hmax_bits));
}

// ------------------------------------------------------------------ solves / refinement
// per-problem max |v| over the chunks -> sc[p].rnorm_bits
__global__ void k_inf_norm(ChunkGrid g, const double* __restrict__ v, IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  __shared__ double sh[32];
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  double mx = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x) {
    const double a = fabs(v[i]);
    mx = (a == a) ? fmax(mx, a) : INFINITY;  // a NaN entry makes the norm infinite (fmax would drop it)
  }
  mx = block_max(mx, sh);
  if (threadIdx.x == 0) atomicMax(&sc[pid].rnorm_bits, dbits(mx));
}

__global__ void k_ir_begin(IterScal* sc, int64_t B, BatchFlags* bf) {
  FOR_PROBLEMS(B) {
    IterScal& q = sc[p];
    q.ir_skip = q.halt;
    q.ir_cur = 0;
    q.rhs_norm = bitsd(q.rnorm_bits);
    q.rnorm_bits = 0ull;
    q.ir_prev = INFINITY;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) bf->ir_none = bf->all_halt;
}

// dst (+)= src on the chunks of problems still refining (add) or of every problem (set)
template <typename T>
__global__ void k_set_from(ChunkGrid g, double* __restrict__ dst, const T* __restrict__ src, int add,
                           const IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  if (add && sc[pid].ir_skip) return;
  for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x)
    dst[i] = add ? dst[i] + (double)src[i] : (double)src[i];
}

// Refinement test of one problem (Sec. 3.6): stop at the tolerance, or after
// max_steps steps, or, when stop_ratio > 0 and ||r||_inf is already below the
// acceptance bar fail_tol = 1e-4 max(1, ||rhs||_inf), as soon as a step has
// reduced ||r||_inf by less than stop_ratio (the last correction is kept).  A
// step that made ||r||_inf larger is undone (k_ir_revert) and ends the
// refinement: the regularised factor is not a contraction for K there.
// A refinement that ends above fail_tol marks the iteration (ir_fail = 1; 2 if
// the residual is not finite): with a low-precision factor it is then redone in
// FP64; in FP64 a non-finite solve stops the solve at the current iterate.
__device__ bool ir_step_due(IterScal& q, double abstol, double reltol, double stop_ratio, int max_steps) {
  const double r = bitsd(q.rnorm_bits);
  q.rnorm_bits = 0ull;
  q.ir_revert = 0;
  if (q.ir_skip) return false;
  const double fail_tol = 1e-4 * fmax(1.0, q.rhs_norm);
  const double tol = abstol + reltol * q.rhs_norm;
  if (r > q.ir_prev) {
    q.ir_revert = 1;
    q.ir_skip = 1;
    if (!(q.ir_prev <= fail_tol)) q.ir_fail = max(q.ir_fail, isfinite(q.ir_prev) ? 1 : 2);
    if (q.ir_prev > tol) q.ir_worst = fmax(q.ir_worst, q.ir_prev);
    return false;
  }
  const bool stalled = stop_ratio > 0 && r <= fail_tol && !(r * stop_ratio < q.ir_prev);
  q.ir_prev = r;
  if (!(r > tol) || stalled || q.ir_cur >= max_steps) {  // NaN also stops
    q.ir_skip = 1;
    if (!(r <= fail_tol)) q.ir_fail = max(q.ir_fail, isfinite(r) ? 1 : 2);  // 2: a non-finite solve
    if (r > tol) q.ir_worst = fmax(q.ir_worst, r);
    return false;
  }
  q.ir_cur += 1;
  q.ir_total += 1;
  return true;
}

// Undo the last correction of the problems whose residual it made larger.
template <typename T>
__global__ void k_ir_revert(ChunkGrid g, double* __restrict__ dst, const T* __restrict__ src, const IterScal* sc,
                            const int* skip) {
  if (skip && *skip) return;
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  if (!sc[pid].ir_revert) return;
  for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x) dst[i] -= (double)src[i];
}

// Unrolled loop (no graph): per-problem test, ir_none = no problem continues.
__global__ void k_ir_check(IterScal* sc, int64_t B, BatchFlags* bf, double abstol, double reltol, double stop_ratio,
                           int max_steps) {
  int go = 0;
  for (int64_t p = threadIdx.x; p < B; p += blockDim.x)
    go |= ir_step_due(sc[p], abstol, reltol, stop_ratio, max_steps) ? 1 : 0;
  go = __syncthreads_or(go);
  if (threadIdx.x == 0) bf->ir_none = go ? 0 : 1;
}

// Graph WHILE loop: the same test; the body runs again iff some problem continues.
__global__ void k_ir_check_cond(IterScal* sc, int64_t B, BatchFlags* bf, double abstol, double reltol,
                                double stop_ratio, int max_steps, cudaGraphConditionalHandle h) {
  int go = 0;
  for (int64_t p = threadIdx.x; p < B; p += blockDim.x)
    go |= ir_step_due(sc[p], abstol, reltol, stop_ratio, max_steps) ? 1 : 0;
  go = __syncthreads_or(go);
  if (threadIdx.x == 0) {
    bf->ir_none = go ? 0 : 1;
    cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

// ------------------------------------------------------------------ direction
// Up to three dot products; product k runs over the x chunks (xs[k] = 1) or the z
// chunks, with a[k], b[k] indexed by the chunk's local index (x index or row).
struct DotArgs {
  const double* a[3];
  const double* b[3];
  int xs[3];
  int np;
};
__global__ void k_dots(ChunkGrid g, DotArgs d, double* part, int slot0, const int* skip) {
  if (skip && *skip) return;
  __shared__ double sh[32];
  const bool zp = blockIdx.x >= g.nckx;
  const Chunk c = g.ck[blockIdx.x];
  const int64_t slot = chunk_slot(g);
  for (int k = 0; k < d.np; ++k) {
    if ((d.xs[k] != 0) == zp) continue;
    double v = 0.0;
    for (int64_t i = c.begin + threadIdx.x; i < c.begin + c.len; i += blockDim.x) v += d.a[k][i] * d.b[k][i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) part[(slot0 + k) * g.pst + slot] = v;
  }
}

__global__ void k_fin_const(IterScal* sc, const double* part, int64_t pst, const int64_t* ckx_ptr,
                            const int64_t* ckz_ptr, const int* skip) {
  if (skip && *skip) return;
  const int64_t p = blockIdx.x;
  const double a = fin_sum(part, S_D0, pst, ckx_ptr[p], ckx_ptr[p + 1]);
  const double b = fin_sum(part, S_D1, pst, ckz_ptr[p], ckz_ptr[p + 1]);
  if (threadIdx.x == 0) {
    sc[p].qp_dx2 = a;
    sc[p].b_dz2 = b;
  }
}

// Delta tau (first form of Eq. step-direction) and Delta kappa.
__global__ void k_fin_dtau(IterScal* sc, const double* part, int64_t pst, const int64_t* ckx_ptr,
                           const int64_t* ckz_ptr, const int* skip) {
  if (skip && *skip) return;
  const int64_t p = blockIdx.x;
  const double qpdx1 = fin_sum(part, S_D0, pst, ckx_ptr[p], ckx_ptr[p + 1]);
  const double bdz1 = fin_sum(part, S_D1, pst, ckz_ptr[p], ckz_ptr[p + 1]);
  if (threadIdx.x != 0) return;
  IterScal& q = sc[p];
  const double tau = q.tau, kappa = q.kappa;
  const double num = q.d_tau - q.d_kap / tau + qpdx1 + bdz1;
  const double den = kappa / tau + q.xPx / (tau * tau) - q.qp_dx2 - q.b_dz2;
  const double dtau = num / den;
  q.dtau = dtau;
  q.dkap = -(q.d_kap + kappa * dtau) / tau;
}

__global__ void k_recover(ChunkGrid g, double* __restrict__ dir, const double* __restrict__ sol1,
                          const double* __restrict__ sol2, const IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  const double dtau = sc[pid].dtau;
  for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x) dir[i] = sol1[i] + dtau * sol2[i];
}

// right-hand side [d_x; -(d_z - d_s)] with (d_x, d_z, d_tau) = f G, d_s given, d_kappa given
__global__ void k_rhs(ChunkGrid g, double* __restrict__ rhs, const double* __restrict__ G,
                      const double* __restrict__ ds, IterScal* sc, int64_t B, int affine, const int* skip) {
  if (skip && *skip) return;
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  const double f = affine ? 1.0 : (1.0 - sc[pid].sigma);
  if (!zp) {
    for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x) rhs[i] = f * G[i];
  } else {
    for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x) rhs[i] = -(f * G[i] - ds[i - g.n]);
  }
  // the per-problem part, once per problem (every problem has >= 1 chunk and the grid has >= B threads)
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < B) {
    IterScal& q = sc[t];
    const double ft = affine ? 1.0 : (1.0 - q.sigma);
    q.d_tau = ft * q.G3;
    q.d_kap = affine ? q.kappa * q.tau : q.kappa * q.tau + q.dkap_a * q.dtau_a - q.sigma_mu;
  }
}

// ------------------------------------------------------------------ step length
struct StepParams {
  double backtrack, min_step, beta, step_fraction;
  int nonsym;
  int hist_cap;
  int escalate_on;  // a failed refinement holds the iteration back for a redo in FP64
  int boost_on;     // FP64 factor: a non-finite solve holds the iteration back for a redo
                    // with a larger static regularisation
  double escalate_ratio;  // escalate when a refinement ended above its tolerance with
                          // ||r|| > escalate_ratio max|G| (0: off)
};
constexpr double kRegBoostStep = 100.0, kRegBoostMax = 1e4;

__global__ void k_step_begin(IterScal* sc, int64_t B, const int* skip) {
  if (skip && *skip) return;
  FOR_PROBLEMS(B) sc[p].amin_bits = dbits(INFINITY);
}

__global__ void k_fin_step_sym(IterScal* sc, int64_t B, const int* skip) {
  if (skip && *skip) return;
  FOR_PROBLEMS(B) {
    IterScal& q = sc[p];
    double a = fmin(1.0, bitsd(q.amin_bits));
    if (q.dtau < 0) a = fmin(a, -q.tau / q.dtau);
    if (q.dkap < 0) a = fmin(a, -q.kappa / q.dkap);
    q.alpha_sym = a;
  }
}

__global__ void k_mu_coef(IterScal* sc, const ProbConst* pc, const double* part, int64_t pst, const int64_t* ckz_ptr,
                          const int* skip) {
  if (skip && *skip) return;
  const int64_t p = blockIdx.x;
  const int64_t c0 = ckz_ptr[p], c1 = ckz_ptr[p + 1];
  const double sdz = fin_sum(part, S_D0, pst, c0, c1), dsz = fin_sum(part, S_D1, pst, c0, c1),
               dsdz = fin_sum(part, S_D2, pst, c0, c1);
  if (threadIdx.x != 0) return;
  IterScal& q = sc[p];
  const double k = 1.0 / (double)(pc[p].nu + 1);
  q.mu_coef[0] = (q.sz + q.tau * q.kappa) * k;
  q.mu_coef[1] = (sdz + dsz + q.tau * q.dkap + q.kappa * q.dtau) * k;
  q.mu_coef[2] = (dsdz + q.dtau * q.dkap) * k;
}

__global__ void k_fin_step(IterScal* sc, int64_t B, StepParams sp, int combined, double* hist, BatchFlags* bf,
                           const int* skip) {
  if (skip && *skip) return;
  FOR_PROBLEMS(B) {
    IterScal& q = sc[p];
    if (q.halt) continue;
    double a = q.alpha_sym;
    if (sp.nonsym) {
      int j = q.ns.jint;
      if (combined && q.ns.fail) {
        const unsigned long long m = q.ns.mask;
        j = (m == 0ull) ? -1 : j + __ffsll((long long)m);  // first common pass after jint
      }
      a = (j < 0) ? 0.0 : a * pow(sp.backtrack, (double)j);
    }
    double* h = (q.iter < sp.hist_cap) ? hist + (int64_t)12 * sp.hist_cap * p + 12 * q.iter : nullptr;
    if (!combined) {
      q.alpha_a = a;
      const double om = 1.0 - a;
      q.sigma = om * om * om;
      q.sigma_mu = q.sigma * q.mu;
      q.dtau_a = q.dtau;
      q.dkap_a = q.dkap;
      if (h) {
        h[7] = a;
        h[8] = q.sigma;
      }
    } else {
      // the direction is too inexact to reduce feasibility residuals still far (100x)
      // above their termination tolerance
      const bool inexact = sp.escalate_ratio > 0 && q.ir_worst > sp.escalate_ratio * q.g_scaled && q.feas_ratio > 100.0;
      if ((q.ir_fail || q.feas_stall >= 3 || inexact) && sp.escalate_on) {
        q.alpha_c = 0.0;
        q.escalate = 1;  // redo the iteration with the FP64 factor
        continue;
      }
      if (q.ir_fail == 2 && sp.boost_on && fmax(1.0, q.reg_boost) < kRegBoostMax) {
        // the unpivoted FP64 factor broke down (a pivot near zero made it overflow):
        // redo the iteration with the static regularisation raised; refinement on
        // the unregularised K recovers the solution of K
        q.reg_boost = fmax(1.0, q.reg_boost) * kRegBoostStep;
        q.alpha_c = 0.0;
        q.escalate = 1;
        continue;
      }
      if (q.ir_fail == 2) {
        // a KKT solve of this iteration gave a non-finite value even in FP64 with
        // the largest regularisation: stop at the current, finite iterate
        q.alpha_c = 0.0;
        q.status = CLR_NUMERICAL_ERROR;
        halt_problem(q, bf);
        continue;
      }
      q.alpha_c = a;
      if (h) {
        h[9] = a;
        h[10] = q.ir_total;
      }
      if (!(a >= sp.min_step)) {
        q.status = CLR_INSUFFICIENT_PROGRESS;
        halt_problem(q, bf);
      }
    }
  }
}

__global__ void k_update(ChunkGrid g, double* __restrict__ xz, double* __restrict__ s, const double* __restrict__ dir,
                         const double* __restrict__ ds, const IterScal* sc, double frac, const int* skip) {
  if (skip && *skip) return;
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  if (sc[pid].halt || sc[pid].escalate) return;
  const double a = frac * sc[pid].alpha_c;
  for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x) {
    if (zp && i - g.n >= g.zaux) continue;  // auxiliary rows: s = z = 0
    xz[i] += a * dir[i];
    if (zp) s[i - g.n] += a * ds[i - g.n];
  }
}

// dyn_hits[1]: a tensor-core wait of the factorization ran out (its result is unusable)
__global__ void k_fin_update(IterScal* sc, int64_t B, double frac, const int* dyn_hits, BatchFlags* bf,
                             const int* skip) {
  if (skip && *skip) return;
  FOR_PROBLEMS(B) {
    IterScal& q = sc[p];
    if (q.halt || q.escalate) continue;
    if (dyn_hits[1]) {
      q.status = CLR_NUMERICAL_ERROR;
      halt_problem(q, bf);
      continue;
    }
    const double a = frac * q.alpha_c;
    q.tau += a * q.dtau;
    q.kappa += a * q.dkap;
    q.iter += 1;
    q.dyn_hits = *dyn_hits;
  }
}

// ------------------------------------------------------------------ init helpers
__global__ void k_init_scal(IterScal* sc, int64_t B, BatchFlags* bf) {
  FOR_PROBLEMS(B) {
    memset(&sc[p], 0, sizeof(IterScal));
    sc[p].tau = 1.0;
    sc[p].kappa = 1.0;
    sc[p].reg_boost = 1.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    bf->all_halt = 0;
    bf->n_running = (int)B;
    bf->ir_none = 0;
  }
}

__global__ void k_init_delta(IterScal* sc, const ProbConst* pc, int64_t B, double static_reg, double static_reg_dyn) {
  FOR_PROBLEMS(B) sc[p].delta = static_reg + static_reg_dyn * fmax(pc[p].maxPdiag, 1.0);
}

// which 0: [0; b], which 1: [-q; 0], which 2: [-q; b]
__global__ void k_build_rhs(ChunkGrid g, double* __restrict__ rhs, const double* __restrict__ q,
                            const double* __restrict__ b, int which, const int* skip) {
  if (skip && *skip) return;
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x)
    rhs[i] = zp ? (which == 1 ? 0.0 : b[i - g.n]) : (which == 0 ? 0.0 : -q[i]);
}

// symmetric initial point of the problems with symmetric cones only
__global__ void k_init_take(ChunkGrid g, double* __restrict__ xz, double* __restrict__ s,
                            const double* __restrict__ sol, const ProbConst* pc, int which) {
  int64_t i0, len;
  int pid;
  bool zp;
  chunk_range(g, &i0, &len, &pid, &zp);
  if (!pc[pid].sym) return;
  for (int64_t i = i0 + threadIdx.x; i < i0 + len; i += blockDim.x) {
    const bool aux = zp && i - g.n >= g.zaux;  // auxiliary rows: s = z = 0
    if (which == 0) {
      if (!zp) xz[i] = sol[i];
      else s[i - g.n] = aux ? 0.0 : -sol[i];
    } else if (zp) {
      xz[i] = aux ? 0.0 : sol[i];
    }
  }
}

// ------------------------------------------------------------------ host side
namespace {
thread_local std::string g_cuda_err;
struct AllocHook {
  clr_alloc_fn a = nullptr;
  clr_free_fn f = nullptr;
  void* ctx = nullptr;
} g_alloc;
}  // namespace

void set_cuda_error(cudaError_t e, const char* where) {
  if (g_cuda_err.empty()) g_cuda_err = std::string(cudaGetErrorString(e)) + " at " + where;
}

void* DeviceArena::alloc(size_t bytes) {
  void* p = nullptr;
  bytes = (bytes + 255) & ~(size_t)255;
  if (g_alloc.a) p = g_alloc.a(bytes, g_alloc.ctx);
  else if (async_) {
    if (cudaMallocAsync(&p, bytes, async_) != cudaSuccess) p = nullptr;
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (!p) return nullptr;
  if (nblocks_ == cap_) {
    size_t nc = cap_ ? 2 * cap_ : 64;
    Block* nb = new Block[nc];
    for (size_t i = 0; i < nblocks_; ++i) nb[i] = blocks_[i];
    delete[] blocks_;
    blocks_ = nb;
    cap_ = nc;
  }
  blocks_[nblocks_++] = Block{p, bytes};
  total_ += bytes;
  return p;
}

void DeviceArena::release() {
  for (size_t i = 0; i < nblocks_; ++i) {
    if (g_alloc.f) g_alloc.f(blocks_[i].p, blocks_[i].n, g_alloc.ctx);
    else if (async_) cudaFreeAsync(blocks_[i].p, async_);
    else cudaFree(blocks_[i].p);
  }
  delete[] blocks_;
  blocks_ = nullptr;
  nblocks_ = cap_ = total_ = 0;
}

namespace {
std::mutex g_pin_mu;
std::vector<std::pair<size_t, void*>> g_pin_free;  // (size class, block)
size_t pin_class(size_t bytes) {
  size_t c = 256;
  while (c < bytes) c <<= 1;
  return c;
}
}  // namespace

void* pinned_get(size_t bytes) {
  const size_t c = pin_class(bytes);
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (size_t i = 0; i < g_pin_free.size(); ++i)
      if (g_pin_free[i].first == c) {
        void* p = g_pin_free[i].second;
        g_pin_free[i] = g_pin_free.back();
        g_pin_free.pop_back();
        return p;
      }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, c) != cudaSuccess) return nullptr;
  return p;
}

void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.emplace_back(pin_class(bytes), p);
}

void Solver::drop_graphs() {
  for (int k = 0; k < 2; ++k) {
    if (gexec_[k]) cudaGraphExecDestroy(gexec_[k]);
    if (graph_[k]) cudaGraphDestroy(graph_[k]);
    gexec_[k] = nullptr;
    graph_[k] = nullptr;
  }
  if (igexec_) cudaGraphExecDestroy(igexec_);
  if (igraph_) cudaGraphDestroy(igraph_);
  igexec_ = nullptr;
  igraph_ = nullptr;
}

// Event marks: 0/1 bracket the initialisation, 2 = iteration start, 3 = before the
// factorization, 4 = after it, 5 = iteration end.
void Solver::mark(int i) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(stream_, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev_[i], stream_, cudaEventRecordExternal);
  else cudaEventRecord(ev_[i], stream_);
}

namespace {
int64_t count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  int64_t k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}
double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

Solver::~Solver() {
  if (stream_) cudaStreamSynchronize(stream_);  // nothing of ours in flight before buffers go back
  drop_graphs();
  ar_.release();
  for (cudaEvent_t e : ev_)
    if (e) cudaEventDestroy(e);
  if (step_ev_) cudaEventDestroy(step_ev_);
  pinned_put(sc_host_, sizeof(IterScal) * (size_t)lay.B);
  pinned_put(bf_host_, sizeof(BatchFlags));
  if (own_stream_ && stream_) cudaStreamDestroy(stream_);
  if (body_stream_) cudaStreamDestroy(body_stream_);
}

int Solver::analyze(const clr_csc* P, const double* q, const clr_csc* A, const double* b, const clr_cone* cones,
                    int32_t ncones, const clr_settings& s) {
  st = s;
  const double t0 = now_s();
  std::vector<HostProblem> ps(1);
  int rc = build_problem(ps[0], P, q, A, b, cones, ncones, st, err);
  if (rc != CLR_OK) return rc;
  if (st.verbose) std::fprintf(stderr, "[clr] setup: validate, reorder, equilibrate, KKT layout %.3f s\n", now_s() - t0);
  rc = analyze_cohort(std::move(ps), {}, s);
  setup_s = now_s() - t0;
  return rc;
}

int Solver::analyze_cohort(std::vector<HostProblem>&& ps, const std::vector<std::vector<int64_t>>& orders,
                           const clr_settings& s) {
  st = s;
  const double t0 = now_s();
  probs = std::move(ps);
  int rc = build_cohort(probs, orders, hp, lay, sy, err, st.verbose, st.amalgamation);
  if (rc != CLR_OK) return rc;
  const double t1 = now_s();
  build_numeric_maps(sy, hp.kcol_ptr, hp.krow, mp, st.pull_lists_direct != 0);
  if (st.verbose)
    std::fprintf(stderr, "[clr] setup: ordering + symbolic %.3f s, numeric maps %.3f s (N %lld, nnz(L) %lld, %.3g flops)\n",
                 t1 - t0, now_s() - t1, (long long)sy.N, (long long)sy.l_nnz, sy.flops);
  setup_s += now_s() - t0;
  return CLR_OK;
}

int Solver::upload() {
  const double t0 = now_s();
  const int64_t n = hp.n, m = hp.m, N = n + m, B = lay.B;
  if (!stream_) {
    CLR_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
    own_stream_ = true;
  }
  sc_host_ = static_cast<IterScal*>(pinned_get(sizeof(IterScal) * (size_t)B));
  bf_host_ = static_cast<BatchFlags*>(pinned_get(sizeof(BatchFlags)));
  if (!sc_host_ || !bf_host_) return CLR_E_OOM;
  CLR_CUDA(cudaStreamCreateWithFlags(&body_stream_, cudaStreamNonBlocking));
  for (cudaEvent_t& e : ev_) CLR_CUDA(cudaEventCreate(&e));
  CLR_CUDA(cudaEventCreateWithFlags(&step_ev_, cudaEventDisableTiming));
  // expected pivot sign and problem by elimination position
  std::vector<int8_t> dsign(N);
  std::vector<int32_t> pos_pid(N);
  for (int64_t k = 0; k < N; ++k) {
    const int64_t v = sy.perm[k], r = v - n;
    // x rows +1, constraint rows -1, except the first auxiliary row (p) of each expanded SOC: +1
    const bool aux_p = r >= hp.cl.aux_begin && r < hp.cl.aux_begin + hp.cl.n_aux && (r - hp.cl.aux_begin) % 2 == 0;
    dsign[k] = (v < n || aux_p) ? 1 : -1;
    pos_pid[k] = lay.pid[sy.perm[k]];
  }
  const int small_max = st.small_front_max > 0 ? st.small_front_max : (st.factor_bits == 64 ? 96 : 128);
  int rc = ldl_structure_upload(ar_, sy, mp, dsign, small_max, ls_, &pos_pid);
  if (rc != CLR_OK) return rc;
  f32_.tc16 = st.factor_bits == 16;
  f32_.flow = f64_.flow = st.big_front_schedule != 0;
  f32_.flow_tc = st.big_front_schedule == 1 ? 1 : (st.big_front_schedule == 3 ? 2 : 0);
  rc = (st.factor_bits == 64) ? f64_.alloc(ar_, ls_) : f32_.alloc(ar_, ls_);
  if (rc != CLR_OK) return rc;
  // full-K CSR with value indices
  {
    std::vector<int64_t> cnt(N + 1, 0);
    for (int64_t j = 0; j < N; ++j)
      for (int64_t p = hp.kcol_ptr[j]; p < hp.kcol_ptr[j + 1]; ++p) {
        const int64_t i = hp.krow[p];
        cnt[i + 1]++;
        if (i != j) cnt[j + 1]++;
      }
    for (int64_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> col(cnt[N]), vi(cnt[N]);
    std::vector<int64_t> next(cnt.begin(), cnt.end() - 1);
    // rows get entries from columns j (lower part, row i >= j) and their own column's entries
    for (int64_t j = 0; j < N; ++j)
      for (int64_t p = hp.kcol_ptr[j]; p < hp.kcol_ptr[j + 1]; ++p) {
        const int64_t i = hp.krow[p];
        if (i != j) {
          col[next[i]] = (int32_t)j;
          vi[next[i]++] = (int32_t)p;
        }
      }
    for (int64_t j = 0; j < N; ++j)
      for (int64_t p = hp.kcol_ptr[j]; p < hp.kcol_ptr[j + 1]; ++p) {
        const int64_t i = hp.krow[p];
        col[next[j]] = (int32_t)i;
        vi[next[j]++] = (int32_t)p;
      }
    std::vector<std::pair<int32_t, int32_t>> row;
    for (int64_t i = 0; i < N; ++i) {
      // sort each row by column (entries may interleave)
      row.clear();
      for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) row.emplace_back(col[p], vi[p]);
      std::sort(row.begin(), row.end());
      for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) {
        col[p] = row[p - cnt[i]].first;
        vi[p] = row[p - cnt[i]].second;
      }
    }
    h_long_.clear();
    for (int64_t i = 0; i < N; ++i)
      if (cnt[i + 1] - cnt[i] > kLongRow) h_long_.push_back(i);
    v_.nlong = (int64_t)h_long_.size();
    v_.long_rows = h_long_.empty() ? nullptr : ar_.upload(h_long_.data(), v_.nlong);
    if (!h_long_.empty() && !v_.long_rows) return CLR_E_OOM;
    v_.kptr = ar_.upload(cnt.data(), N + 1);
    v_.kcol = ar_.upload(col.data(), (int64_t)col.size());
    v_.kvi = ar_.upload(vi.data(), (int64_t)vi.size());
    {
      // the x rows' values in full-CSR order (P and A are constant through the solve):
      // contiguous loads instead of gathers through the value index
      std::vector<double> fv(cnt[hp.n], 0.0);
      for (int64_t p = 0; p < cnt[hp.n]; ++p) fv[p] = hp.kval[vi[p]];
      h_kfv_src_.assign(vi.begin(), vi.begin() + cnt[hp.n]);
      v_.kfv = fv.empty() ? nullptr : ar_.upload(fv.data(), (int64_t)fv.size());
      if (!fv.empty() && !v_.kfv) return CLR_E_OOM;
    }
    const double avg = N ? (double)cnt[N] / (double)N : 1.0;
    csr_group_ = avg > 24 ? 32 : (avg > 12 ? 16 : (avg > 6 ? 8 : 4));
  }
  // cohort layout
  nckx_ = (int64_t)lay.ckx.size();
  nckz_ = (int64_t)lay.ckz.size();
  pst_ = std::max<int64_t>(1, std::max(nckx_, nckz_));
  {
    std::vector<Chunk> ck(lay.ckx);
    ck.insert(ck.end(), lay.ckz.begin(), lay.ckz.end());
    v_.ck = ar_.upload(ck.data(), (int64_t)ck.size());
  }
  v_.ckx_ptr = ar_.upload(lay.ckx_ptr.data(), B + 1);
  v_.ckz_ptr = ar_.upload(lay.ckz_ptr.data(), B + 1);
  v_.pid = ar_.upload(lay.pid.data(), N);
  v_.pc = ar_.upload(lay.pc.data(), B);
  hist_rows_ = st.max_iter + 2;
  v_.kval = ar_.upload(hp.kval.data(), (int64_t)hp.kval.size());
  v_.q = ar_.upload(hp.q.data(), n);
  v_.b = ar_.upload(hp.b.data(), m);
  v_.D = ar_.upload(hp.D.data(), n);
  v_.E = ar_.upload(hp.E.data(), m);
  v_.xz = ar_.alloc_n<double>(N);
  v_.s = ar_.alloc_n<double>(m);
  v_.lo = ar_.alloc_n<double>(N);
  v_.hi = ar_.alloc_n<double>(N);
  v_.G = ar_.alloc_n<double>(N);
  v_.qp = ar_.alloc_n<double>(n);
  v_.rhs = ar_.alloc_n<double>(N);
  v_.sol1 = ar_.alloc_n<double>(N);
  v_.sol2 = ar_.alloc_n<double>(N);
  v_.dir_a = ar_.alloc_n<double>(N);
  v_.dsa = ar_.alloc_n<double>(m);
  v_.dir = ar_.alloc_n<double>(N);
  v_.ds = ar_.alloc_n<double>(m);
  // Delta s of the auxiliary rows is never written: zero for good
  if (v_.dsa && v_.ds) {
    CLR_CUDA(cudaMemsetAsync(v_.dsa, 0, sizeof(double) * (size_t)std::max<int64_t>(m, 1), stream_));
    CLR_CUDA(cudaMemsetAsync(v_.ds, 0, sizeof(double) * (size_t)std::max<int64_t>(m, 1), stream_));
  }
  v_.dsrhs = ar_.alloc_n<double>(m);
  v_.r = ar_.alloc_n<double>(N);
  v_.solb = ar_.alloc_n<double>(N);
  v_.part = ar_.alloc_n<double>((int64_t)S_NSLOT * pst_);
  v_.maxb = ar_.alloc_n<unsigned long long>((int64_t)M_NMAX * B);
  v_.hist = ar_.alloc_n<double>(12 * (int64_t)hist_rows_ * B);
  sc_ = ar_.alloc_n<IterScal>(B);
  bf_ = ar_.alloc_n<BatchFlags>(1);
  // cone layout
  const ConeLayout& cl = hp.cl;
  cd_ = ConeDev();
  cd_.m = m;
  cd_.m_zero = cl.m_zero;
  cd_.m_nonneg = cl.m_nonneg;
  cd_.kvz = v_.kval + hp.kval_x;
  cd_.nkz = cl.kval_z;
  cd_.nprob = B;
  cd_.row_pid = v_.pid + n;
  cd_.pc = v_.pc;
  cd_.scratch = ar_.alloc_n<double>(m);
  cd_.nn_w = ar_.alloc_n<double>(cl.m_nonneg);
  cd_.nn_lam = ar_.alloc_n<double>(cl.m_nonneg);
  cd_.n_soc = cl.soc_end - cl.soc_begin;
  {
    std::vector<int64_t> off, kb, aux;
    std::vector<int32_t> dim;
    for (int64_t c = cl.soc_begin; c < cl.soc_end; ++c) {
      off.push_back(cl.cones[c].off);
      dim.push_back((int32_t)cl.cones[c].dim);
      cd_.soc_dmax = std::max<int>(cd_.soc_dmax, (int)cl.cones[c].dim);
      kb.push_back(cl.cones[c].kbase);
      aux.push_back(cl.cones[c].aux);
      if (cl.cones[c].dim <= 8 && cl.cones[c].aux < 0) cd_.soc_nsmall++;  // a thread per cone
    }
    cd_.soc_split = (cd_.soc_nsmall > 0 && cd_.soc_nsmall < cd_.n_soc) ? 1 : 0;
    cd_.soc_off = ar_.upload(off.data(), (int64_t)off.size());
    cd_.soc_dim = ar_.upload(dim.data(), (int64_t)dim.size());
    cd_.soc_kb = ar_.upload(kb.data(), (int64_t)kb.size());
    if (cl.n_aux > 0) cd_.soc_aux = ar_.upload(aux.data(), (int64_t)aux.size());
    cd_.aux_begin = cl.aux_begin;
    cd_.n_aux = cl.n_aux;
  }
  cd_.soc_eta = ar_.alloc_n<double>(cd_.n_soc);
  cd_.soc_wb = ar_.alloc_n<double>(m);
  cd_.soc_lam = ar_.alloc_n<double>(m);
  cd_.n_exp = cl.exp_end - cl.exp_begin;
  cd_.exp_row0 = cd_.n_exp ? cl.cones[cl.exp_begin].off : 0;
  cd_.exp_kb0 = cd_.n_exp ? cl.cones[cl.exp_begin].kbase : 0;
  cd_.n_pow = cl.pow_end - cl.pow_begin;
  cd_.pow_row0 = cd_.n_pow ? cl.cones[cl.pow_begin].off : 0;
  cd_.pow_kb0 = cd_.n_pow ? cl.cones[cl.pow_begin].kbase : 0;
  {
    std::vector<double> al;
    for (int64_t c = cl.pow_begin; c < cl.pow_end; ++c) al.push_back(cl.cones[c].alpha);
    cd_.pow_alpha = ar_.upload(al.data(), (int64_t)al.size());
  }
  {
    std::vector<int64_t> dims, rows, kbs;
    for (int64_t c = cl.psd_begin; c < cl.psd_end; ++c) {
      dims.push_back(cl.cones[c].dim);
      rows.push_back(cl.cones[c].off);
      kbs.push_back(cl.cones[c].kbase);
    }
    if (!cones_psd_setup(ar_, cd_, dims, rows, kbs)) return CLR_E_OOM;
  }
  cd_.ep_zt = ar_.alloc_n<double>(3 * (cd_.n_exp + cd_.n_pow));
  exp_central_point_host(cd_.exp_center);
  if (!v_.kptr || !v_.kcol || !v_.kvi || !v_.kval || !v_.xz || !v_.part || !sc_ || !bf_ || !cd_.scratch || !v_.ck ||
      !v_.pid || !v_.pc || !v_.hist || !v_.maxb)
    return CLR_E_OOM;
  CLR_CUDA(cudaStreamSynchronize(stream_));
  device_ready = true;
  setup_s += now_s() - t0;
  return CLR_OK;
}

int Solver::use_stream_ordered(cudaStream_t stream) {
  if (device_ready || !stream) return CLR_E_STATE;
  stream_ = stream;
  own_stream_ = false;
  ar_.set_stream_ordered(stream);
  return CLR_OK;
}

int Solver::set_stream(void* stream) {
  drop_graphs();
  if (own_stream_ && stream_) cudaStreamDestroy(stream_);
  own_stream_ = false;
  stream_ = (cudaStream_t)stream;
  if (!stream_) {
    CLR_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
    own_stream_ = true;
  }
  return CLR_OK;
}

double Solver::reg_static() const { return escalated_ ? 1e-8 : st.static_reg; }
double Solver::reg_dyn_eps() const { return escalated_ ? 1e-13 : st.dyn_reg_eps; }
double Solver::reg_dyn_delta() const { return escalated_ ? 2e-7 : st.dyn_reg_delta; }

int Solver::factor() {
  const int* halt = &bf_->all_halt;
  if (use64()) return f64_.factor(stream_, v_.kval, sc_, reg_dyn_eps(), reg_dyn_delta(), halt);
  return f32_.factor(stream_, v_.kval, sc_, reg_dyn_eps(), reg_dyn_delta(), halt);
}

// sol = K^{-1} rhs by the factor plus iterative refinement on the unregularised K (FP64),
// per problem.  While a graph is being captured the refinement loop is a conditional
// WHILE node (its body runs only while some problem needs another step); otherwise it
// is unrolled to ir_max_steps steps whose kernels return at once after convergence.
int Solver::kkt_solve(const double* rhs, double* sol) {
  const int64_t N = hp.n + hp.m, B = lay.B;
  cudaStream_t s = stream_;
  const int* halt = &bf_->all_halt;
  const int* irs = &bf_->ir_none;
  const ChunkGrid cg{v_.ck, nckx_, pst_, hp.n};
  const unsigned nck = (unsigned)(nckx_ + nckz_);
  const int pg = grid_for(B, 128);
  k_inf_norm<<<nck, 256, 0, s>>>(cg, rhs, sc_, halt);
  k_ir_begin<<<pg, 128, 0, s>>>(sc_, B, bf_);
  auto revert = [&](cudaStream_t ss) {
    if (use64()) k_ir_revert<double><<<nck, 256, 0, ss>>>(cg, sol, f64_.xs, sc_, halt);
    else k_ir_revert<float><<<nck, 256, 0, ss>>>(cg, sol, f32_.xs, sc_, halt);
  };
  auto ldl_solve_add = [&](cudaStream_t ss, const double* b, int add) -> int {
    if (use64()) {
      int rc = f64_.solve(ss, b, irs);
      if (rc) return rc;
      k_set_from<double><<<nck, 256, 0, ss>>>(cg, sol, f64_.xs, add, sc_, irs);
    } else {
      int rc = f32_.solve(ss, b, irs);
      if (rc) return rc;
      k_set_from<float><<<nck, 256, 0, ss>>>(cg, sol, f32_.xs, add, sc_, irs);
    }
    return CLR_OK;
  };
  const int G = csr_group_;
  const int kg = grid_for(N * G, 256, 16 * kSMs);
  auto residual = [&](cudaStream_t ss) {
    switch (G) {
      case 32: k_kmv<32><<<kg, 256, 0, ss>>>(1, 0, N, hp.n, v_.kptr, v_.kcol, v_.kvi, v_.kval, v_.kfv, sol, nullptr, nullptr, rhs, v_.r, v_.pid, sc_, irs); break;
      case 16: k_kmv<16><<<kg, 256, 0, ss>>>(1, 0, N, hp.n, v_.kptr, v_.kcol, v_.kvi, v_.kval, v_.kfv, sol, nullptr, nullptr, rhs, v_.r, v_.pid, sc_, irs); break;
      case 8: k_kmv<8><<<kg, 256, 0, ss>>>(1, 0, N, hp.n, v_.kptr, v_.kcol, v_.kvi, v_.kval, v_.kfv, sol, nullptr, nullptr, rhs, v_.r, v_.pid, sc_, irs); break;
      default: k_kmv<4><<<kg, 256, 0, ss>>>(1, 0, N, hp.n, v_.kptr, v_.kcol, v_.kvi, v_.kval, v_.kfv, sol, nullptr, nullptr, rhs, v_.r, v_.pid, sc_, irs); break;
    }
    kmv_long(ss, 1, 0, N, hp.n, v_, h_long_, sol, nullptr, nullptr, rhs, v_.r, sc_, irs);
  };
  const int cb = (int)std::min<int64_t>(1024, std::max<int64_t>(32, ((B + 31) / 32) * 32));
  int rc = ldl_solve_add(s, rhs, 0);
  if (rc) return rc;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CLR_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusActive || st.ir_max_steps == 0) {
    for (int it = 0; it <= st.ir_max_steps; ++it) {  // the last pass only checks the last step
      residual(s);
      k_ir_check<<<1, cb, 0, s>>>(sc_, B, bf_, st.ir_abstol, st.ir_reltol, st.ir_stop_ratio, st.ir_max_steps);
      if (it > 0) revert(s);
      if (it == st.ir_max_steps) break;
      rc = ldl_solve_add(s, v_.r, 1);
      if (rc) return rc;
    }
    CLR_CHECK_LAUNCH();
    return CLR_OK;
  }
  // graph capture: condition set by the check before the node and at the end of each body pass
  cudaGraph_t cgraph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  cudaGraphConditionalHandle h;
  residual(s);
  CLR_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cgraph, nullptr, nullptr, nullptr));
  CLR_CUDA(cudaGraphConditionalHandleCreate(&h, cgraph, 0, 0));
  k_ir_check_cond<<<1, cb, 0, s>>>(sc_, B, bf_, st.ir_abstol, st.ir_reltol, st.ir_stop_ratio, st.ir_max_steps, h);
  CLR_CHECK_LAUNCH();
  CLR_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cgraph, &deps, &edata, &ndeps));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CLR_CUDA(cudaGraphAddNode(&node, cgraph, deps, edata, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CLR_CUDA(cudaStreamBeginCaptureToGraph(body_stream_, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  rc = ldl_solve_add(body_stream_, v_.r, 1);
  residual(body_stream_);
  k_ir_check_cond<<<1, cb, 0, body_stream_>>>(sc_, B, bf_, st.ir_abstol, st.ir_reltol, st.ir_stop_ratio,
                                              st.ir_max_steps, h);
  revert(body_stream_);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(body_stream_, &out);
  if (rc) return rc;
  if (e != cudaSuccess) {
    set_cuda_error(e, "cudaStreamEndCapture(body)");
    return CLR_E_CUDA;
  }
  CLR_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  ir_nodes_.push_back(body);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

namespace {
template <int G>
void launch_kmv_split(cudaStream_t s, int mode, int64_t r0, int64_t r1, int64_t n, const VecDev& v, const double* x,
                      double* lo, double* hi, const double* rhs, double* out, IterScal* sc, const int* skip) {
  const int kg = grid_for((r1 - r0) * G, 256, 16 * kSMs);
  k_kmv<G><<<kg, 256, 0, s>>>(mode, r0, r1, n, v.kptr, v.kcol, v.kvi, v.kval, v.kfv, x, lo, hi, rhs, out, v.pid, sc,
                              skip);
}
void kmv(int G, cudaStream_t s, int mode, int64_t r0, int64_t r1, int64_t n, const VecDev& v,
         const std::vector<int64_t>& h_long, const double* x, double* lo, double* hi, const double* rhs, double* out,
         IterScal* sc, const int* skip) {
  if (r1 <= r0) return;
  switch (G) {
    case 32: launch_kmv_split<32>(s, mode, r0, r1, n, v, x, lo, hi, rhs, out, sc, skip); break;
    case 16: launch_kmv_split<16>(s, mode, r0, r1, n, v, x, lo, hi, rhs, out, sc, skip); break;
    case 8: launch_kmv_split<8>(s, mode, r0, r1, n, v, x, lo, hi, rhs, out, sc, skip); break;
    default: launch_kmv_split<4>(s, mode, r0, r1, n, v, x, lo, hi, rhs, out, sc, skip); break;
  }
  kmv_long(s, mode, r0, r1, n, v, h_long, x, lo, hi, rhs, out, sc, skip);
}
}  // namespace

// One search direction: solve with the current right-hand side (rhs built by
// k_rhs), Delta tau, Delta x/z, Delta s = -d_s - H Delta z (PSD blocks of H in
// factored form).
int Solver::direction(bool affine) {
  const int64_t n = hp.n, m = hp.m, N = n + m, B = lay.B;
  cudaStream_t s = stream_;
  const int* halt = &bf_->all_halt;
  const ChunkGrid cg{v_.ck, nckx_, pst_, n};
  const unsigned nck = (unsigned)(nckx_ + nckz_);
  double* dir = affine ? v_.dir_a : v_.dir;
  double* ds = affine ? v_.dsa : v_.ds;
  int rc = kkt_solve(v_.rhs, v_.sol1);
  if (rc) return rc;
  DotArgs da{{v_.qp, v_.b, nullptr}, {v_.sol1, v_.sol1 + n, nullptr}, {1, 0, 0}, 2};
  k_dots<<<nck, 256, 0, s>>>(cg, da, v_.part, S_D0, halt);
  k_fin_dtau<<<(unsigned)B, 128, 0, s>>>(sc_, v_.part, pst_, v_.ckx_ptr, v_.ckz_ptr, halt);
  k_recover<<<nck, 256, 0, s>>>(cg, dir, v_.sol1, v_.sol2, sc_, halt);
  // (the auxiliary rows of expanded SOCs, the last rows, keep Delta s = 0)
  kmv(csr_group_, s, 2, n, N - hp.cl.n_aux, n, v_, h_long_, dir, nullptr, nullptr, v_.dsrhs, ds, sc_, halt);
  // PSD rows again, with H in factored form (the assembled block loses the small
  // eigen-directions of S near convergence)
  cones_psd_ds_from_dz(s, cd_, dir + n, v_.dsrhs, ds, halt);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

int Solver::step_length(bool combined) {
  const int64_t n = hp.n, B = lay.B;
  cudaStream_t s = stream_;
  const int* halt = &bf_->all_halt;
  const ChunkGrid cg{v_.ck, nckx_, pst_, n};
  const unsigned nck = (unsigned)(nckx_ + nckz_);
  const int pg = grid_for(B, 128);
  const double* dir = combined ? v_.dir : v_.dir_a;
  const double* ds = combined ? v_.ds : v_.dsa;
  k_step_begin<<<pg, 128, 0, s>>>(sc_, B, halt);
  int rc = cones_step_symmetric(s, cd_, v_.s, ds, v_.xz + n, dir + n, sc_, halt);
  if (rc) return rc;
  k_fin_step_sym<<<pg, 128, 0, s>>>(sc_, B, halt);
  const bool nonsym = (cd_.n_exp + cd_.n_pow) > 0;
  if (nonsym) {
    if (combined) {
      DotArgs da{{v_.s, ds, ds}, {dir + n, v_.xz + n, dir + n}, {0, 0, 0}, 3};
      k_dots<<<nck, 256, 0, s>>>(cg, da, v_.part, S_D0, halt);
      k_mu_coef<<<(unsigned)B, 128, 0, s>>>(sc_, v_.pc, v_.part, pst_, v_.ckz_ptr, halt);
    }
    rc = cones_step_nonsym(s, cd_, v_.s, ds, v_.xz + n, dir + n, sc_, st.backtrack, combined ? 1 : 0, st.nbhd_beta,
                           halt);
    if (rc) return rc;
  }
  StepParams sp{st.backtrack, st.min_step, st.nbhd_beta, st.step_fraction, nonsym ? 1 : 0, hist_rows_,
                (st.fp64_escalation && !use64()) ? 1 : 0, use64() ? 1 : 0, st.escalate_ratio};
  k_fin_step<<<pg, 128, 0, s>>>(sc_, B, sp, combined ? 1 : 0, v_.hist, bf_, halt);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

// Algorithm 1, one pass of steps 12 (residuals, here at the top), 4-11.
int Solver::iteration() {
  const int64_t n = hp.n, m = hp.m, N = n + m, B = lay.B;
  cudaStream_t s = stream_;
  const int* halt = &bf_->all_halt;
  const ChunkGrid cg{v_.ck, nckx_, pst_, n, hp.cl.n_aux ? hp.cl.aux_begin : INT64_MAX};
  const unsigned nck = (unsigned)(nckx_ + nckz_);
  const int pg = grid_for(B, 128);
  int rc;
  mark(2);
  // ---- residuals, objectives, mu, termination ----
  kmv(csr_group_, s, 0, 0, N, n, v_, h_long_, v_.xz, v_.lo, v_.hi, nullptr, nullptr, sc_, halt);
  CLR_CUDA(cudaMemsetAsync(v_.maxb, 0, sizeof(unsigned long long) * M_NMAX * (size_t)B, s));
  k_resid<<<nck, 256, 0, s>>>(cg, v_.xz, v_.s, v_.lo, v_.hi, v_.q, v_.b, v_.D, v_.E, sc_, v_.G, v_.qp, v_.part,
                              v_.maxb, halt);
  TermParams tp{st.eps_feas, st.eps_inf, st.max_iter, hist_rows_};
  k_fin_resid<<<(unsigned)B, 128, 0, s>>>(sc_, v_.pc, v_.part, pst_, v_.ckx_ptr, v_.ckz_ptr, v_.maxb, tp, v_.hist,
                                          bf_, halt);
  // ---- step 4: scaling H, KKT values; static + proportional regularisation ----
  k_hmax_reset<<<pg, 128, 0, s>>>(sc_, B, halt);
  rc = cones_scaling(s, cd_, v_.s, v_.xz + n, sc_, halt);
  if (rc) return rc;
  k_fin_delta<<<pg, 128, 0, s>>>(sc_, v_.pc, B, reg_static(), st.static_reg_dyn, halt);
  // ---- step 5: factor ----
  mark(3);
  rc = factor();
  if (rc) return rc;
  mark(4);
  // ---- constant right-hand side [-q; b] ----
  k_build_rhs<<<nck, 256, 0, s>>>(cg, v_.rhs, v_.q, v_.b, 2, halt);
  rc = kkt_solve(v_.rhs, v_.sol2);
  if (rc) return rc;
  DotArgs da{{v_.qp, v_.b, nullptr}, {v_.sol2, v_.sol2 + n, nullptr}, {1, 0, 0}, 2};
  k_dots<<<nck, 256, 0, s>>>(cg, da, v_.part, S_D0, halt);
  k_fin_const<<<(unsigned)B, 128, 0, s>>>(sc_, v_.part, pst_, v_.ckx_ptr, v_.ckz_ptr, halt);
  // ---- step 6: affine direction, d = (G, d_s = s, d_kappa = kappa tau) ----
  CLR_CUDA(cudaMemcpyAsync(v_.dsrhs, v_.s, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, s));
  k_rhs<<<nck, 256, 0, s>>>(cg, v_.rhs, v_.G, v_.dsrhs, sc_, B, 1, halt);
  rc = direction(true);
  if (rc) return rc;
  // ---- steps 7-8: affine step length, sigma ----
  rc = step_length(false);
  if (rc) return rc;
  // ---- step 9: combined direction ----
  rc = cones_combined_ds(s, cd_, v_.s, v_.xz + n, v_.dsa, v_.dir_a + n, sc_, v_.dsrhs, halt);
  if (rc) return rc;
  k_rhs<<<nck, 256, 0, s>>>(cg, v_.rhs, v_.G, v_.dsrhs, sc_, B, 0, halt);
  rc = direction(false);
  if (rc) return rc;
  // ---- step 10: combined step length with the neighbourhood check ----
  rc = step_length(true);
  if (rc) return rc;
  // ---- step 11: update ----
  k_update<<<nck, 256, 0, s>>>(cg, v_.xz, v_.s, v_.dir, v_.ds, sc_, st.step_fraction, halt);
  const int* dh = use64() ? f64_.dyn_hits : f32_.dyn_hits;
  k_fin_update<<<pg, 128, 0, s>>>(sc_, B, st.step_fraction, dh, bf_, halt);
  mark(5);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

int Solver::initialise() {
  const int64_t n = hp.n, m = hp.m, N = n + m, B = lay.B;
  cudaStream_t s = stream_;
  const ChunkGrid cg{v_.ck, nckx_, pst_, n, hp.cl.n_aux ? hp.cl.aux_begin : INT64_MAX};
  const unsigned nck = (unsigned)(nckx_ + nckz_);
  const int pg = grid_for(B, 128);
  bool any_sym = false, any_nonsym = false;
  for (const ProbConst& p : lay.pc) (p.sym ? any_sym : any_nonsym) = true;
  mark(0);
  k_init_scal<<<pg, 128, 0, s>>>(sc_, B, bf_);
  CLR_CUDA(cudaMemsetAsync(v_.xz, 0, sizeof(double) * (size_t)N, s));
  CLR_CUDA(cudaMemsetAsync(v_.s, 0, sizeof(double) * (size_t)m, s));
  if (any_sym) {
    int rc = cones_identity_H(s, cd_, nullptr);
    if (rc) return rc;
    k_init_delta<<<pg, 128, 0, s>>>(sc_, v_.pc, B, st.static_reg, st.static_reg_dyn);
    rc = factor();
    if (rc) return rc;
    k_build_rhs<<<nck, 256, 0, s>>>(cg, v_.rhs, v_.q, v_.b, 0, nullptr);
    rc = kkt_solve(v_.rhs, v_.sol1);
    if (rc) return rc;
    k_init_take<<<nck, 256, 0, s>>>(cg, v_.xz, v_.s, v_.sol1, v_.pc, 0);
    k_build_rhs<<<nck, 256, 0, s>>>(cg, v_.rhs, v_.q, v_.b, 1, nullptr);
    rc = kkt_solve(v_.rhs, v_.sol1);
    if (rc) return rc;
    k_init_take<<<nck, 256, 0, s>>>(cg, v_.xz, v_.s, v_.sol1, v_.pc, 1);
    rc = cones_shift_init(s, cd_, v_.s, sc_, nullptr);
    if (rc) return rc;
    rc = cones_shift_init(s, cd_, v_.xz + n, sc_, nullptr);
    if (rc) return rc;
  }
  if (any_nonsym) {
    int rc = cones_unit_init(s, cd_, v_.s, nullptr);
    if (rc) return rc;
    rc = cones_init_shadow(s, cd_, nullptr);
    if (rc) return rc;
    rc = cones_unit_init(s, cd_, v_.xz + n, nullptr);
    if (rc) return rc;
  }
  k_init_scal<<<pg, 128, 0, s>>>(sc_, B, bf_);  // tau = kappa = 1, counters reset (ir_total of the init dropped)
  mark(1);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

int Solver::launch_iteration() {
  if (!st.use_graph) return iteration();
  const int k = (use64() && st.factor_bits != 64) ? 1 : 0;
  if (!gexec_[k]) {
    CLR_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
    int rc = iteration();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(stream_, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) {
      set_cuda_error(e, "cudaStreamEndCapture");
      return CLR_E_CUDA;
    }
    graph_[k] = g;
    iter_kernels_[k] = count_kernel_nodes(graph_[k]);
    body_kernels_[k] = ir_nodes_.empty() ? 0 : count_kernel_nodes(ir_nodes_.back());
    ir_nodes_.clear();
    CLR_CUDA(cudaGraphInstantiate(&gexec_[k], graph_[k], 0));
  }
  CLR_CUDA(cudaGraphLaunch(gexec_[k], stream_));
  return CLR_OK;
}

int Solver::launch_init() {
  if (!st.use_graph) return initialise();
  if (!igexec_) {
    CLR_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
    int rc = initialise();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(stream_, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) {
      set_cuda_error(e, "cudaStreamEndCapture");
      return CLR_E_CUDA;
    }
    igraph_ = g;
    init_kernels_ = count_kernel_nodes(igraph_);
    ir_nodes_.clear();
    CLR_CUDA(cudaGraphInstantiate(&igexec_, igraph_, 0));
  }
  CLR_CUDA(cudaGraphLaunch(igexec_, stream_));
  return CLR_OK;
}

int Solver::solve_begin() {
  if (!device_ready) return CLR_E_STATE;
  t_begin_ = now_s();
  perf = clr_perf{};
  it_ = 0;
  first_step_ = true;
  escalated_ = false;
  esc_iter_.assign(lay.B, -1);
  for (int64_t p = 0; p < lay.B; ++p) sc_host_[p].iter = 0;  // host mirror: no iteration of this solve yet
  int rc = launch_init();
  if (rc) return rc;
  perf.kernel_launches += init_kernels_;
  bool any_sym = false;
  for (const ProbConst& p : lay.pc) any_sym = any_sym || p.sym;
  perf.factorizations += any_sym ? 1 : 0;
  return CLR_OK;
}

int Solver::step_launch() {
  step64_ = use64();
  int rc = launch_iteration();
  if (rc) return rc;
  perf.kernel_launches += iter_kernels_[(use64() && st.factor_bits != 64) ? 1 : 0];
  CLR_CUDA(cudaMemcpyAsync(sc_host_, sc_, sizeof(IterScal) * (size_t)lay.B, cudaMemcpyDeviceToHost, stream_));
  CLR_CUDA(cudaMemcpyAsync(bf_host_, bf_, sizeof(BatchFlags), cudaMemcpyDeviceToHost, stream_));
  CLR_CUDA(cudaEventRecord(step_ev_, stream_));
  ++it_;
  return CLR_OK;
}

int Solver::step_poll(bool* ready) {
  cudaError_t e = cudaEventQuery(step_ev_);
  if (e == cudaErrorNotReady) {
    *ready = false;
    return CLR_OK;
  }
  if (e != cudaSuccess) {
    set_cuda_error(e, "cudaEventQuery");
    return CLR_E_CUDA;
  }
  *ready = true;
  return finish_step();
}

// Switch the rest of this solve to the FP64 factor (allocated on first use).
int Solver::escalate_to_fp64() {
  if (!f64_ready_ && st.factor_bits != 64) {
    int rc = f64_.alloc(ar_, ls_);
    if (rc != CLR_OK) return rc;
    f64_ready_ = true;
  }
  escalated_ = true;
  for (int64_t p = 0; p < lay.B; ++p)
    if (esc_iter_[p] < 0) esc_iter_[p] = sc_host_[p].iter;
  if (st.verbose)
    std::fprintf(stderr, "[clr] refinement failed with the low-precision factor: continuing with the FP64 factor "
                         "and its regularisation\n");
  return CLR_OK;
}

// bookkeeping once a launched step has finished
int Solver::finish_step() {
  if (!use64() && st.fp64_escalation) {
    for (int64_t p = 0; p < lay.B; ++p)
      if (sc_host_[p].escalate) {
        int rc = escalate_to_fp64();
        if (rc != CLR_OK) return rc;
        break;
      }
  }
  float ms = 0.f;
  if (first_step_) {
    if (cudaEventElapsedTime(&ms, ev_[0], ev_[1]) == cudaSuccess) perf.init_ms += ms;
    first_step_ = false;
  }
  // a full iteration ran unless every problem stopped at its residual stage
  bool full = false;
  for (int64_t p = 0; p < lay.B && !full; ++p) {
    const int stt = sc_host_[p].status;
    full = (stt == 0 || stt == CLR_INSUFFICIENT_PROGRESS);
  }
  if (full || !bf_host_->all_halt) {
    if (cudaEventElapsedTime(&ms, ev_[2], ev_[3]) == cudaSuccess) perf.resid_cones_ms += ms;
    if (cudaEventElapsedTime(&ms, ev_[3], ev_[4]) == cudaSuccess) {
      perf.factor_ms += ms;
      if (step64_) {
        perf.factor64_ms += ms;
        perf.factorizations64 += 1;
      }
    }
    if (cudaEventElapsedTime(&ms, ev_[4], ev_[5]) == cudaSuccess) perf.solve_step_ms += ms;
    perf.factorizations += 1;
  } else if (cudaEventElapsedTime(&ms, ev_[2], ev_[5]) == cudaSuccess) {
    perf.resid_cones_ms += ms;  // the terminating pass only evaluates the residuals
  }
  return CLR_OK;
}

bool Solver::all_halted() const { return bf_host_->all_halt != 0 || it_ > st.max_iter + 1; }
int Solver::problem_status(int64_t p) const { return sc_host_[p].status; }

int Solver::solve_end() {
  CLR_CUDA(cudaStreamSynchronize(stream_));
  int iters = 0, irt = 0;
  for (int64_t p = 0; p < lay.B; ++p) {
    iters = std::max(iters, sc_host_[p].iter);
    irt += sc_host_[p].ir_total;
  }
  perf.iterations = iters;
  if (st.use_graph) perf.kernel_launches += (int64_t)irt * body_kernels_[escalated_ ? 1 : 0];  // loop bodies (upper bound)
  perf.factor_flops = sy.flops;
  solve_s = now_s() - t_begin_;
  infos.assign(lay.B, clr_info{});
  history.assign(lay.B, {});
  std::vector<double> hall(12 * (size_t)hist_rows_ * (size_t)lay.B);
  CLR_CUDA(cudaMemcpy(hall.data(), v_.hist, sizeof(double) * hall.size(), cudaMemcpyDeviceToHost));
  for (int64_t p = 0; p < lay.B; ++p) {
    const IterScal& h = sc_host_[p];
    infos[p] = info_now(p);
    infos[p].solve_s = solve_s;
    const int rows = std::min(h.iter + 1, hist_rows_);
    const double* src = hall.data() + 12 * (size_t)hist_rows_ * (size_t)p;
    history[p].assign(src, src + 12 * (size_t)rows);
  }
  solved_once = true;
  return CLR_OK;
}

int Solver::step_wait(bool* ready) {
  CLR_CUDA(cudaEventSynchronize(step_ev_));
  return step_poll(ready);
}

int Solver::solve() {
  int rc = solve_begin();
  if (rc) return rc;
  for (int it = 0; it <= st.max_iter + 1; ++it) {
    rc = step_launch();
    if (rc) return rc;
    bool ready = false;
    rc = step_wait(&ready);
    if (rc) return rc;
    if (bf_host_->all_halt) break;
  }
  return solve_end();
}

clr_info Solver::info_now(int64_t p) const {
  const IterScal& h = sc_host_[p];
  clr_info info{};
  info.fp64_from_iter = (p < (int64_t)esc_iter_.size()) ? esc_iter_[p] : -1;
  info.status = h.status;
  info.iterations = h.iter;
  info.ir_steps_total = h.ir_total;
  info.dyn_reg_hits = h.dyn_hits;
  info.obj_primal = h.pcost;
  info.obj_dual = h.dcost;
  info.res_primal = h.res_p;
  info.res_dual = h.res_d;
  info.gap_abs = h.gap_abs;
  info.gap_rel = h.gap_rel;
  info.mu = h.mu;
  info.tau = h.tau;
  info.kappa = h.kappa;
  info.setup_s = setup_s;
  info.solve_s = now_s() - t_begin_;
  return info;
}

int Solver::get_solution_now(int64_t p, double* x, double* sl, double* z, clr_info* out) {
  if (p < 0 || p >= lay.B) return CLR_E_INVALID;
  if (infos.size() != (size_t)lay.B) infos.assign(lay.B, clr_info{});
  infos[p] = info_now(p);
  return unscale_solution(p, x, sl, z, out);
}

int Solver::get_solution(int64_t p, double* x, double* sl, double* z, clr_info* out) {
  if (!solved_once) return CLR_E_STATE;
  if (p < 0 || p >= lay.B) return CLR_E_INVALID;
  return unscale_solution(p, x, sl, z, out);
}

int Solver::unscale_solution(int64_t p, double* x, double* sl, double* z, clr_info* out) {
  const HostProblem& pr = probs[p];
  const int64_t n = pr.n, m = pr.m, N = hp.n + hp.m;
  (void)N;
  std::vector<double> xs(n), zs(m), ss(m);
  if (n) CLR_CUDA(cudaMemcpy(xs.data(), v_.xz + lay.xo[p], sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));
  if (m) {
    // the problem's rows sit in up to six family runs of the cohort rows
    const std::vector<int64_t>& zr = lay.zrow[p];
    int64_t r = 0;
    while (r < m) {
      int64_t e = r + 1;
      while (e < m && zr[e] == zr[e - 1] + 1) ++e;
      CLR_CUDA(cudaMemcpy(zs.data() + r, v_.xz + hp.n + zr[r], sizeof(double) * (size_t)(e - r),
                          cudaMemcpyDeviceToHost));
      CLR_CUDA(cudaMemcpy(ss.data() + r, v_.s + zr[r], sizeof(double) * (size_t)(e - r), cudaMemcpyDeviceToHost));
      r = e;
    }
  }
  const clr_info& info = infos[p];
  const double tau = info.tau, c = pr.c;
  // unscale: x = D x^, s = s^ / E, z = E z^ / c
  std::vector<double> xu(n), su(m), zu(m);
  for (int64_t j = 0; j < n; ++j) xu[j] = pr.D[j] * xs[j];
  for (int64_t r = 0; r < m; ++r) {
    su[r] = ss[r] / pr.E[r];
    zu[r] = pr.E[r] * zs[r] / c;
  }
  double fx = 1.0 / tau, fs = 1.0 / tau, fz = 1.0 / tau;
  const double nan = std::nan("");
  if (info.status == CLR_PRIMAL_INFEASIBLE) {
    double btz = 0;
    for (int64_t r = 0; r < m; ++r) btz += (pr.b[r] / pr.E[r]) * zu[r];
    fx = fs = nan;
    fz = -1.0 / btz;
  } else if (info.status == CLR_DUAL_INFEASIBLE) {
    double qtx = 0;
    for (int64_t j = 0; j < n; ++j) qtx += (pr.q[j] / (c * pr.D[j])) * xu[j];
    fx = fs = -1.0 / qtx;
    fz = nan;
  }
  if (x)
    for (int64_t j = 0; j < n; ++j) x[j] = xu[j] * fx;
  for (int64_t r = 0; r < m; ++r) {
    const int64_t orig = pr.row_perm[r];
    if (orig < 0) continue;  // auxiliary row of an expanded SOC
    if (sl) sl[orig] = su[r] * fs;
    if (z) z[orig] = zu[r] * fz;
  }
  if (out) *out = info;
  return CLR_OK;
}

int Solver::update_qb(int64_t p, const double* q, const double* b) {
  if (p < 0 || p >= lay.B) return CLR_E_INVALID;
  HostProblem& pr = probs[p];
  int rc = set_qb(pr, q, b);
  if (rc) return rc;
  for (int64_t j = 0; j < pr.n; ++j) hp.q[lay.xo[p] + j] = pr.q[j];
  for (int64_t r = 0; r < pr.m; ++r) hp.b[lay.zrow[p][r]] = pr.b[r];
  lay.pc[p].bnorm = pr.bnorm;
  lay.pc[p].qnorm = pr.qnorm;
  if (device_ready) {
    CLR_CUDA(cudaMemcpyAsync(v_.q, hp.q.data(), sizeof(double) * (size_t)hp.n, cudaMemcpyHostToDevice, stream_));
    CLR_CUDA(cudaMemcpyAsync(v_.b, hp.b.data(), sizeof(double) * (size_t)hp.m, cudaMemcpyHostToDevice, stream_));
    CLR_CUDA(cudaMemcpyAsync(v_.pc, lay.pc.data(), sizeof(ProbConst) * (size_t)lay.B, cudaMemcpyHostToDevice,
                             stream_));
    CLR_CUDA(cudaStreamSynchronize(stream_));
  }
  return CLR_OK;
}

// New values of P and/or A for problem p (same pattern): the x part of the KKT
// values and its full-CSR copy are rewritten; the symbolic analysis, the order
// and every device buffer are kept (parametric programming, Sec. 4.6).
int Solver::update_PA(int64_t p, const double* Px, const double* Ax) {
  if (p < 0 || p >= lay.B) return CLR_E_INVALID;
  if (!Px && !Ax) return CLR_OK;
  HostProblem& pr = probs[p];
  int rc = set_PA(pr, Px, Ax, hp.kval);
  if (rc) return rc;
  lay.pc[p].maxPdiag = pr.maxPdiag;
  if (device_ready) {
    std::vector<double> fv(h_kfv_src_.size());
    for (size_t k = 0; k < fv.size(); ++k) fv[k] = hp.kval[h_kfv_src_[k]];
    CLR_CUDA(cudaMemcpyAsync(v_.kval, hp.kval.data(), sizeof(double) * (size_t)hp.kval_x, cudaMemcpyHostToDevice,
                             stream_));
    if (!fv.empty())
      CLR_CUDA(cudaMemcpyAsync(const_cast<double*>(v_.kfv), fv.data(), sizeof(double) * fv.size(),
                               cudaMemcpyHostToDevice, stream_));
    CLR_CUDA(cudaMemcpyAsync(v_.pc, lay.pc.data(), sizeof(ProbConst) * (size_t)lay.B, cudaMemcpyHostToDevice,
                             stream_));
    CLR_CUDA(cudaStreamSynchronize(stream_));
  }
  return CLR_OK;
}

const char* last_cuda_error() { return g_cuda_err.c_str(); }
void set_allocator(clr_alloc_fn a, clr_free_fn f, void* ctx) {
  g_alloc.a = a;
  g_alloc.f = f;
  g_alloc.ctx = ctx;
}

}  // namespace clr
