// Per-iteration device step of Algorithm 1 (arXiv:2412.19027) and the solver
// object.  Every step of an iteration runs in the kernels below or in
// cones.cu / ldl.cu; the host only launches them (replaying one captured CUDA
// graph per iteration) and reads back the status word.
//
// Scaled space: the device holds P^ = c D P D, q^ = c D q, A^ = E A D,
// b^ = E b (setup.cpp) and iterates x^, s^, z^, tau, kappa; residuals and the
// termination tests (Eq. residuals-objectives, termination-check,
// infeasibility-check) are evaluated on the unscaled quantities
// x = D x^, s = s^ / E, z = E z^ / c.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "ipm.cuh"

namespace clr {

// ------------------------------------------------------------------ slots
enum SumSlot { S_XPX = 0, S_QX, S_BZ, S_SZ, S_D0, S_D1, S_D2, S_D3, S_NSLOT };
enum MaxSlot { M_RD = 0, M_X, M_RP, M_S, M_Z, M_ATZ, M_PX, M_AXS, M_NMAX };

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// ------------------------------------------------------------------ K products
// G lanes per row of the full (both triangles) KKT CSR; values through kvi into kval.
// mode 0: lo[i] = sum_{col < n} K_ij v_j, hi[i] = sum_{col >= n} K_ij v_j
// mode 1: out[i] = rhs[i] - (K v)_i and max |out| -> *maxb
// mode 2 (rows n..N-1): out[i-n] = -rhs[i-n] + hi   (Delta s = -d_s - H Delta z; K_zz = -H)
template <int G>
__global__ void k_kmv(int mode, int64_t r0, int64_t r1, int64_t n, const int64_t* __restrict__ kptr,
                      const int32_t* __restrict__ kcol, const int32_t* __restrict__ kvi, const double* __restrict__ kval,
                      const double* __restrict__ v, double* __restrict__ lo, double* __restrict__ hi,
                      const double* __restrict__ rhs, double* __restrict__ out, unsigned long long* maxb,
                      const int* skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x % G;
  const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int64_t gstride = ((int64_t)gridDim.x * blockDim.x) / G;
  double mx = 0.0;
  for (int64_t i = r0 + gid; i < r1; i += gstride) {
    double a = 0.0, b = 0.0;
    for (int64_t p = kptr[i] + lane; p < kptr[i + 1]; p += G) {
      const int32_t c = kcol[p];
      const double t = kval[kvi[p]] * v[c];
      if (c < n) a += t;
      else b += t;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o, G);
      b += __shfl_xor_sync(0xffffffffu, b, o, G);
    }
    if (lane == 0) {
      if (mode == 0) {
        lo[i] = a;
        hi[i] = b;
      } else if (mode == 1) {
        const double r = rhs[i] - (a + b);
        out[i] = r;
        mx = fmax(mx, fabs(r));
      } else {
        out[i - n] = -rhs[i - n] + b;
      }
    }
  }
  if (mode == 1) {
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) atomicMax(maxb, dbits(mx));
  }
}

// ------------------------------------------------------------------ residuals
__device__ void block_write_sum(double v, double* part, int slot) {
  __shared__ double sh[32];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) part[slot * kRedBlocks + blockIdx.x] = v;
}

__global__ void k_resid_x(int64_t n, const double* __restrict__ xz, const double* __restrict__ lo,
                          const double* __restrict__ hi, const double* __restrict__ q, const double* __restrict__ D,
                          IterScal* sc, double* __restrict__ G, double* __restrict__ qp, double* part,
                          unsigned long long* maxb, const int* skip) {
  if (skip && *skip) return;
  const double tau = sc->tau;
  double xpx = 0, qx = 0, mrd = 0, mx = 0, matz = 0, mpx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = xz[i], px = lo[i], atz = hi[i], qi = q[i], di = D[i];
    const double g1 = -(px + atz + qi * tau);
    G[i] = g1;
    qp[i] = qi + 2.0 * px / tau;
    xpx += x * px;
    qx += qi * x;
    mrd = fmax(mrd, fabs(g1) / di);
    mx = fmax(mx, fabs(di * x));
    matz = fmax(matz, fabs(atz) / di);
    mpx = fmax(mpx, fabs(px) / di);
  }
  block_write_sum(xpx, part, S_XPX);
  block_write_sum(qx, part, S_QX);
  mrd = warp_max(mrd);
  mx = warp_max(mx);
  matz = warp_max(matz);
  mpx = warp_max(mpx);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(maxb + M_RD, dbits(mrd));
    atomicMax(maxb + M_X, dbits(mx));
    atomicMax(maxb + M_ATZ, dbits(matz));
    atomicMax(maxb + M_PX, dbits(mpx));
  }
}

__global__ void k_resid_z(int64_t n, int64_t m, const double* __restrict__ xz, const double* __restrict__ s,
                          const double* __restrict__ lo, const double* __restrict__ b, const double* __restrict__ E,
                          IterScal* sc, double* __restrict__ G, double* part, unsigned long long* maxb,
                          const int* skip) {
  if (skip && *skip) return;
  const double tau = sc->tau;
  double bz = 0, sz = 0, mrp = 0, ms = 0, mz = 0, maxs = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = xz[n + i], si = s[i], ax = lo[n + i], bi = b[i], ei = E[i];
    const double g2 = si + ax - bi * tau;
    G[n + i] = g2;
    bz += bi * zi;
    sz += si * zi;
    mrp = fmax(mrp, fabs(g2) / ei);
    ms = fmax(ms, fabs(si) / ei);
    mz = fmax(mz, fabs(ei * zi));
    maxs = fmax(maxs, fabs(ax + si) / ei);
  }
  block_write_sum(bz, part, S_BZ);
  block_write_sum(sz, part, S_SZ);
  mrp = warp_max(mrp);
  ms = warp_max(ms);
  mz = warp_max(mz);
  maxs = warp_max(maxs);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(maxb + M_RP, dbits(mrp));
    atomicMax(maxb + M_S, dbits(ms));
    atomicMax(maxb + M_Z, dbits(mz));
    atomicMax(maxb + M_AXS, dbits(maxs));
  }
}

__device__ double fin_sum(const double* part, int slot) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) v += part[slot * kRedBlocks + b];
  v = block_sum(v, sh);
  __syncthreads();
  return v;  // valid in thread 0
}

struct TermParams {
  double c, bnorm, qnorm, eps_feas, eps_inf;
  int64_t nu;
  int max_iter;
  int hist_cap;
};

// Residuals, objectives, mu and the termination / infeasibility tests.
__global__ void k_fin_resid(IterScal* sc, const double* part, const unsigned long long* maxb, TermParams tp,
                            double* hist, const int* skip) {
  if (skip && *skip) return;
  const double xpx = fin_sum(part, S_XPX), qx = fin_sum(part, S_QX), bz = fin_sum(part, S_BZ),
               sz = fin_sum(part, S_SZ);
  if (threadIdx.x != 0) return;
  const double tau = sc->tau, kappa = sc->kappa, c = tp.c;
  const double mu = (sz + kappa * tau) / (double)(tp.nu + 1);
  const double nrp = bitsd(maxb[M_RP]) / tau;
  const double nrd = bitsd(maxb[M_RD]) / (c * tau);
  const double nx = bitsd(maxb[M_X]) / tau, ns = bitsd(maxb[M_S]) / tau, nz = bitsd(maxb[M_Z]) / (c * tau);
  const double gp = (0.5 * xpx / (tau * tau) + qx / tau) / c;
  const double gd = (-0.5 * xpx / (tau * tau) - bz / tau) / c;
  const double gap = fabs(gp - gd);
  sc->mu = mu;
  sc->xPx = xpx;
  sc->qx = qx;
  sc->bz = bz;
  sc->sz = sz;
  sc->G3 = kappa + qx + bz + xpx / tau;
  sc->pcost = gp;
  sc->dcost = gd;
  sc->res_p = nrp;
  sc->res_d = nrd;
  sc->gap_abs = gap;
  sc->gap_rel = gap / fmax(1.0, fmin(fabs(gp), fabs(gd)));
  int status = 0;
  if (!isfinite(mu) || !isfinite(nrp) || !isfinite(nrd) || !isfinite(gp) || !isfinite(gd) || !isfinite(tau) ||
      !isfinite(kappa)) {
    status = CLR_NUMERICAL_ERROR;
  } else if (nrp < tp.eps_feas * fmax(1.0, tp.bnorm + nx + ns) && nrd < tp.eps_feas * fmax(1.0, tp.qnorm + nx + nz) &&
             gap < tp.eps_feas * fmax(1.0, fmin(fabs(gp), fabs(gd)))) {
    status = CLR_SOLVED;
  } else {
    // infeasibility on the unnormalised unscaled iterates
    const double btz = bz / c, qtx = qx / c;
    const double nxu = bitsd(maxb[M_X]), nzu = bitsd(maxb[M_Z]) / c, nsu = bitsd(maxb[M_S]);
    const double natz = bitsd(maxb[M_ATZ]) / c, npx = bitsd(maxb[M_PX]) / c, naxs = bitsd(maxb[M_AXS]);
    if (btz < -tp.eps_inf && natz < -tp.eps_inf * fmax(1.0, nxu + nzu) * btz) status = CLR_PRIMAL_INFEASIBLE;
    else if (qtx < -tp.eps_inf && npx < -tp.eps_inf * fmax(1.0, nxu) * qtx &&
             naxs < -tp.eps_inf * fmax(1.0, nxu + nsu) * qtx)
      status = CLR_DUAL_INFEASIBLE;
    else if (sc->iter >= tp.max_iter)
      status = CLR_MAX_ITER;
  }
  sc->status = status;
  if (status != 0) sc->halt = 1;
  if (sc->iter < tp.hist_cap) {
    double* h = hist + 12 * sc->iter;
    h[0] = sc->iter;
    h[1] = mu;
    h[2] = gp;
    h[3] = gd;
    h[4] = nrp;
    h[5] = nrd;
    h[6] = gap;
    h[7] = h[8] = h[9] = h[10] = 0.0;
    h[11] = tau;
  }
}

// ------------------------------------------------------------------ regularisation
__global__ void k_fin_delta(IterScal* sc, double static_reg, double static_reg_dyn, double maxPdiag,
                            const int* skip) {
  if (skip && *skip) return;
  const double hm = bitsd(sc->hmax_bits);
  sc->delta = static_reg + static_reg_dyn * fmax(maxPdiag, hm);
}

// ------------------------------------------------------------------ solves / refinement
__global__ void k_inf_norm(const double* __restrict__ v, int64_t N, unsigned long long* maxb, const int* skip) {
  if (skip && *skip) return;
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(v[i]));
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) atomicMax(maxb, dbits(mx));
}

__global__ void k_ir_begin(IterScal* sc, const unsigned long long* rhsmax) {
  sc->ir_skip = sc->halt;
  sc->ir_cur = 0;
  sc->rhs_norm = bitsd(*rhsmax);
  sc->ir_prev = INFINITY;
}

template <typename T>
__global__ void k_set_from(double* __restrict__ dst, const T* __restrict__ src, int64_t N, int add, const int* skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = add ? dst[i] + (double)src[i] : (double)src[i];
}

// Refinement stops at the tolerance (Sec. 3.6), or, when stop_ratio > 0, as soon as a
// step has reduced ||r||_inf by less than stop_ratio (the last correction is kept).
__global__ void k_ir_check(IterScal* sc, unsigned long long* rmax, double abstol, double reltol, double stop_ratio) {
  if (sc->ir_skip) return;
  const double r = bitsd(*rmax);
  *rmax = 0ull;
  const bool stalled = stop_ratio > 0 && !(r * stop_ratio < sc->ir_prev);
  sc->ir_prev = r;
  if (!(r > abstol + reltol * sc->rhs_norm) || stalled) sc->ir_skip = 1;  // converged (NaN also stops)
  else {
    sc->ir_cur += 1;
    sc->ir_total += 1;
  }
}

// The same test for the graph WHILE loop: continue (condition 1) iff another
// refinement step is due; at most max_steps steps.
__global__ void k_ir_check_cond(IterScal* sc, unsigned long long* rmax, double abstol, double reltol,
                                double stop_ratio, int max_steps, cudaGraphConditionalHandle h) {
  unsigned int go = 0;
  if (!sc->ir_skip) {
    const double r = bitsd(*rmax);
    const bool stalled = stop_ratio > 0 && !(r * stop_ratio < sc->ir_prev);
    sc->ir_prev = r;
    if (!(r > abstol + reltol * sc->rhs_norm) || stalled || sc->ir_cur >= max_steps) {
      sc->ir_skip = 1;
    } else {
      sc->ir_cur += 1;
      sc->ir_total += 1;
      go = 1;
    }
  }
  *rmax = 0ull;
  cudaGraphSetConditional(h, go);
}

// ------------------------------------------------------------------ direction
__global__ void k_dots(const double* __restrict__ a0, const double* __restrict__ b0, int64_t n0,
                       const double* __restrict__ a1, const double* __restrict__ b1, int64_t n1,
                       const double* __restrict__ a2, const double* __restrict__ b2, int64_t n2, double* part,
                       int slot0, const int* skip) {
  if (skip && *skip) return;
  double s0 = 0, s1 = 0, s2 = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t i = t; i < n0; i += stride) s0 += a0[i] * b0[i];
  for (int64_t i = t; i < n1; i += stride) s1 += a1[i] * b1[i];
  for (int64_t i = t; i < n2; i += stride) s2 += a2[i] * b2[i];
  block_write_sum(s0, part, slot0);
  block_write_sum(s1, part, slot0 + 1);
  block_write_sum(s2, part, slot0 + 2);
}

__global__ void k_fin_const(IterScal* sc, const double* part, const int* skip) {
  if (skip && *skip) return;
  const double a = fin_sum(part, S_D0), b = fin_sum(part, S_D1);
  if (threadIdx.x == 0) {
    sc->qp_dx2 = a;
    sc->b_dz2 = b;
  }
}

// Delta tau (first form of Eq. step-direction) and Delta kappa.
__global__ void k_fin_dtau(IterScal* sc, const double* part, const int* skip) {
  if (skip && *skip) return;
  const double qpdx1 = fin_sum(part, S_D0), bdz1 = fin_sum(part, S_D1);
  if (threadIdx.x != 0) return;
  const double tau = sc->tau, kappa = sc->kappa;
  const double num = sc->d_tau - sc->d_kap / tau + qpdx1 + bdz1;
  const double den = kappa / tau + sc->xPx / (tau * tau) - sc->qp_dx2 - sc->b_dz2;
  const double dtau = num / den;
  sc->dtau = dtau;
  sc->dkap = -(sc->d_kap + kappa * dtau) / tau;
}

__global__ void k_recover(double* __restrict__ dir, const double* __restrict__ sol1, const double* __restrict__ sol2,
                          int64_t N, const IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  const double dtau = sc->dtau;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    dir[i] = sol1[i] + dtau * sol2[i];
}

// right-hand side [d_x; -(d_z - d_s)] with (d_x, d_z, d_tau) = f G, d_s given, d_kappa given
__global__ void k_rhs(double* __restrict__ rhs, const double* __restrict__ G, const double* __restrict__ ds,
                      int64_t n, int64_t m, double f_dummy, IterScal* sc, int affine, const int* skip) {
  if (skip && *skip) return;
  const double f = affine ? 1.0 : (1.0 - sc->sigma);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)gridDim.x * blockDim.x)
    rhs[i] = (i < n) ? f * G[i] : -(f * G[i] - ds[i - n]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->d_tau = f * sc->G3;
    sc->d_kap = affine ? sc->kappa * sc->tau : sc->kappa * sc->tau + sc->dkap_a * sc->dtau_a - sc->sigma_mu;
  }
  (void)f_dummy;
}

// ------------------------------------------------------------------ step length
struct StepParams {
  double backtrack, min_step, beta, step_fraction;
  int nonsym;
  int64_t nu;
  int hist_cap;
};

__global__ void k_step_begin(IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  sc->amin_bits = dbits(INFINITY);
}

__global__ void k_fin_step_sym(IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  double a = fmin(1.0, bitsd(sc->amin_bits));
  if (sc->dtau < 0) a = fmin(a, -sc->tau / sc->dtau);
  if (sc->dkap < 0) a = fmin(a, -sc->kappa / sc->dkap);
  sc->alpha_sym = a;
}

__global__ void k_mu_coef(IterScal* sc, const double* part, int64_t nu, const int* skip) {
  if (skip && *skip) return;
  const double sdz = fin_sum(part, S_D0), dsz = fin_sum(part, S_D1), dsdz = fin_sum(part, S_D2);
  if (threadIdx.x != 0) return;
  const double k = 1.0 / (double)(nu + 1);
  sc->mu_coef[0] = (sc->sz + sc->tau * sc->kappa) * k;
  sc->mu_coef[1] = (sdz + dsz + sc->tau * sc->dkap + sc->kappa * sc->dtau) * k;
  sc->mu_coef[2] = (dsdz + sc->dtau * sc->dkap) * k;
}

__global__ void k_fin_step(IterScal* sc, StepParams sp, int combined, double* hist, const int* skip) {
  if (skip && *skip) return;
  double a = sc->alpha_sym;
  if (sp.nonsym) {
    int j = sc->ns.jint;
    if (combined && sc->ns.fail) {
      const unsigned long long m = sc->ns.mask;
      j = (m == 0ull) ? -1 : j + __ffsll((long long)m);  // first common pass after jint
    }
    a = (j < 0) ? 0.0 : a * pow(sp.backtrack, (double)j);
  }
  double* h = (sc->iter < sp.hist_cap) ? hist + 12 * sc->iter : nullptr;
  if (!combined) {
    sc->alpha_a = a;
    const double om = 1.0 - a;
    sc->sigma = om * om * om;
    sc->sigma_mu = sc->sigma * sc->mu;
    sc->dtau_a = sc->dtau;
    sc->dkap_a = sc->dkap;
    if (h) {
      h[7] = a;
      h[8] = sc->sigma;
    }
  } else {
    sc->alpha_c = a;
    if (h) {
      h[9] = a;
      h[10] = sc->ir_total;
    }
    if (!(a >= sp.min_step)) {
      sc->status = CLR_INSUFFICIENT_PROGRESS;
      sc->halt = 1;
    }
  }
}

__global__ void k_update(double* __restrict__ xz, double* __restrict__ s, const double* __restrict__ dir,
                         const double* __restrict__ ds, int64_t N, int64_t m, const IterScal* sc, double frac,
                         const int* skip) {
  if (skip && *skip) return;
  const double a = frac * sc->alpha_c;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    xz[i] += a * dir[i];
    if (i < m) s[i] += a * ds[i];
  }
}

__global__ void k_fin_update(IterScal* sc, double frac, const int* dyn_hits, const int* skip) {
  if (skip && *skip) return;
  const double a = frac * sc->alpha_c;
  sc->tau += a * sc->dtau;
  sc->kappa += a * sc->dkap;
  sc->iter += 1;
  sc->dyn_hits = *dyn_hits;
}

// ------------------------------------------------------------------ init helpers
__global__ void k_init_scal(IterScal* sc) {
  memset(sc, 0, sizeof(IterScal));
  sc->tau = 1.0;
  sc->kappa = 1.0;
}

__global__ void k_init_delta(IterScal* sc, double static_reg, double static_reg_dyn, double maxPdiag) {
  sc->delta = static_reg + static_reg_dyn * fmax(maxPdiag, 1.0);
}

__global__ void k_build_rhs_init(double* __restrict__ rhs, const double* __restrict__ q, const double* __restrict__ b,
                                 int64_t n, int64_t m, int which) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)gridDim.x * blockDim.x)
    rhs[i] = (which == 0) ? (i < n ? 0.0 : b[i - n]) : (i < n ? -q[i] : 0.0);
}

__global__ void k_init_take(double* __restrict__ xz, double* __restrict__ s, const double* __restrict__ sol,
                            int64_t n, int64_t m, int which) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)gridDim.x * blockDim.x) {
    if (which == 0) {
      if (i < n) xz[i] = sol[i];
      else s[i - n] = -sol[i];
    } else if (i >= n) {
      xz[i] = sol[i];
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
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
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
    else cudaFree(blocks_[i].p);
  }
  delete[] blocks_;
  blocks_ = nullptr;
  nblocks_ = cap_ = total_ = 0;
}

void Solver::drop_graphs() {
  if (gexec_) cudaGraphExecDestroy(gexec_);
  if (graph_) cudaGraphDestroy(graph_);
  if (igexec_) cudaGraphExecDestroy(igexec_);
  if (igraph_) cudaGraphDestroy(igraph_);
  gexec_ = nullptr;
  graph_ = nullptr;
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
}  // namespace

Solver::~Solver() {
  drop_graphs();
  for (cudaEvent_t e : ev_)
    if (e) cudaEventDestroy(e);
  if (sc_host_) cudaFreeHost(sc_host_);
  if (own_stream_ && stream_) cudaStreamDestroy(stream_);
  if (body_stream_) cudaStreamDestroy(body_stream_);
}

int Solver::analyze(const clr_csc* P, const double* q, const clr_csc* A, const double* b, const clr_cone* cones,
                    int32_t ncones, const clr_settings& s) {
  st = s;
  auto t0 = std::chrono::steady_clock::now();
  int rc = build_problem(hp, P, q, A, b, cones, ncones, st, err);
  if (rc != CLR_OK) return rc;
  rc = symbolic_analyze(hp.n + hp.m, hp.kcol_ptr, hp.krow, nullptr, sy);
  if (rc != CLR_OK) return rc;
  build_numeric_maps(sy, hp.kcol_ptr, hp.krow, mp);
  setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return CLR_OK;
}

int Solver::upload() {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t n = hp.n, m = hp.m, N = n + m;
  if (!stream_) {
    CLR_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
    own_stream_ = true;
  }
  CLR_CUDA(cudaMallocHost(&sc_host_, sizeof(IterScal)));
  CLR_CUDA(cudaStreamCreateWithFlags(&body_stream_, cudaStreamNonBlocking));
  for (cudaEvent_t& e : ev_) CLR_CUDA(cudaEventCreate(&e));
  // expected pivot sign by elimination position: + for x, - for z
  std::vector<int8_t> dsign(N);
  for (int64_t k = 0; k < N; ++k) dsign[k] = sy.perm[k] < n ? 1 : -1;
  int rc = ldl_structure_upload(ar_, sy, mp, dsign, st.factor_bits == 64 ? 96 : 128, ls_);
  if (rc != CLR_OK) return rc;
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
    // fill row by row in increasing column order: rows get entries from columns j (lower part,
    // row i >= j) visited in increasing j, and their own column's entries (upper part) after
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
    for (int64_t i = 0; i < N; ++i) {
      // sort each row by column (entries may interleave)
      std::vector<std::pair<int32_t, int32_t>> row;
      for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) row.emplace_back(col[p], vi[p]);
      std::sort(row.begin(), row.end());
      for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) {
        col[p] = row[p - cnt[i]].first;
        vi[p] = row[p - cnt[i]].second;
      }
    }
    v_.kptr = ar_.upload(cnt.data(), N + 1);
    v_.kcol = ar_.upload(col.data(), (int64_t)col.size());
    v_.kvi = ar_.upload(vi.data(), (int64_t)vi.size());
    const double avg = N ? (double)cnt[N] / (double)N : 1.0;
    csr_group_ = avg > 24 ? 32 : (avg > 12 ? 16 : (avg > 6 ? 8 : 4));
  }
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
  v_.dsrhs = ar_.alloc_n<double>(m);
  v_.r = ar_.alloc_n<double>(N + 16);  // also holds 8 residual-stage maxima
  v_.solb = ar_.alloc_n<double>(N);
  v_.part = ar_.alloc_n<double>((int64_t)S_NSLOT * kRedBlocks);
  v_.hist = ar_.alloc_n<double>(12 * (int64_t)(st.max_iter + 2));
  sc_ = ar_.alloc_n<IterScal>(1);
  // cone layout
  const ConeLayout& cl = hp.cl;
  cd_ = ConeDev();
  cd_.m = m;
  cd_.m_zero = cl.m_zero;
  cd_.m_nonneg = cl.m_nonneg;
  cd_.kvz = v_.kval + hp.kval_x;
  cd_.nkz = cl.kval_z;
  cd_.scratch = ar_.alloc_n<double>(m);
  cd_.nn_w = ar_.alloc_n<double>(cl.m_nonneg);
  cd_.nn_lam = ar_.alloc_n<double>(cl.m_nonneg);
  cd_.n_soc = cl.soc_end - cl.soc_begin;
  {
    std::vector<int64_t> off, kb;
    std::vector<int32_t> dim;
    for (int64_t c = cl.soc_begin; c < cl.soc_end; ++c) {
      off.push_back(cl.cones[c].off);
      dim.push_back((int32_t)cl.cones[c].dim);
      kb.push_back(cl.cones[c].kbase);
    }
    cd_.soc_off = ar_.upload(off.data(), (int64_t)off.size());
    cd_.soc_dim = ar_.upload(dim.data(), (int64_t)dim.size());
    cd_.soc_kb = ar_.upload(kb.data(), (int64_t)kb.size());
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
  cd_.n_psd = cl.psd_end - cl.psd_begin;
  cd_.psd_k = cl.psd_k;
  cd_.psd_d = cl.psd_k * (cl.psd_k + 1) / 2;
  cd_.psd_row0 = cd_.n_psd ? cl.cones[cl.psd_begin].off : 0;
  cd_.psd_kb0 = cd_.n_psd ? cl.cones[cl.psd_begin].kbase : 0;
  cd_.psd_R = ar_.alloc_n<double>(cd_.n_psd * cl.psd_k * cl.psd_k);
  cd_.psd_Ri = ar_.alloc_n<double>(cd_.n_psd * cl.psd_k * cl.psd_k);
  cd_.psd_lam = ar_.alloc_n<double>(cd_.n_psd * cl.psd_k);
  cd_.ep_zt = ar_.alloc_n<double>(3 * (cd_.n_exp + cd_.n_pow));
  exp_central_point_host(cd_.exp_center);
  if (!v_.kptr || !v_.kcol || !v_.kvi || !v_.kval || !v_.xz || !v_.part || !sc_ || !cd_.scratch) return CLR_E_OOM;
  CLR_CUDA(cudaStreamSynchronize(stream_));
  device_ready = true;
  setup_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
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

int Solver::factor() {
  const int* halt = &sc_->halt;
  if (st.factor_bits == 64)
    return f64_.factor(stream_, v_.kval, &sc_->delta, st.dyn_reg_eps, st.dyn_reg_delta, halt);
  return f32_.factor(stream_, v_.kval, &sc_->delta, st.dyn_reg_eps, st.dyn_reg_delta, halt);
}

// sol = K^{-1} rhs by the factor plus iterative refinement on the unregularised K (FP64).
// While a graph is being captured the refinement loop is a conditional WHILE
// node (its body runs only as often as needed); otherwise it is unrolled to
// ir_max_steps steps whose kernels return at once after convergence.
int Solver::kkt_solve(const double* rhs, double* sol) {
  const int64_t N = hp.n + hp.m;
  cudaStream_t s = stream_;
  const int* halt = &sc_->halt;
  const int* irs = &sc_->ir_skip;
  unsigned long long* rmax = &sc_->rnorm_bits;
  CLR_CUDA(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long), s));
  k_inf_norm<<<grid_for(N, 256, kRedBlocks), 256, 0, s>>>(rhs, N, rmax, halt);
  k_ir_begin<<<1, 1, 0, s>>>(sc_, rmax);
  CLR_CUDA(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long), s));
  const int g = grid_for(N, 256);
  auto ldl_solve_add = [&](cudaStream_t ss, const double* b, int add) -> int {
    if (st.factor_bits == 64) {
      int rc = f64_.solve(ss, b, irs);
      if (rc) return rc;
      k_set_from<double><<<g, 256, 0, ss>>>(sol, f64_.xs, N, add, irs);
    } else {
      int rc = f32_.solve(ss, b, irs);
      if (rc) return rc;
      k_set_from<float><<<g, 256, 0, ss>>>(sol, f32_.xs, N, add, irs);
    }
    return CLR_OK;
  };
  const int G = csr_group_;
  const int kg = grid_for(N * G, 256, 16 * kSMs);
  auto residual = [&](cudaStream_t ss) {
    switch (G) {
      case 32: k_kmv<32><<<kg, 256, 0, ss>>>(1, 0, N, hp.n, v_.kptr, v_.kcol, v_.kvi, v_.kval, sol, nullptr, nullptr, rhs, v_.r, rmax, irs); break;
      case 16: k_kmv<16><<<kg, 256, 0, ss>>>(1, 0, N, hp.n, v_.kptr, v_.kcol, v_.kvi, v_.kval, sol, nullptr, nullptr, rhs, v_.r, rmax, irs); break;
      case 8: k_kmv<8><<<kg, 256, 0, ss>>>(1, 0, N, hp.n, v_.kptr, v_.kcol, v_.kvi, v_.kval, sol, nullptr, nullptr, rhs, v_.r, rmax, irs); break;
      default: k_kmv<4><<<kg, 256, 0, ss>>>(1, 0, N, hp.n, v_.kptr, v_.kcol, v_.kvi, v_.kval, sol, nullptr, nullptr, rhs, v_.r, rmax, irs); break;
    }
  };
  int rc = ldl_solve_add(s, rhs, 0);
  if (rc) return rc;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CLR_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusActive || st.ir_max_steps == 0) {
    for (int it = 0; it < st.ir_max_steps; ++it) {
      residual(s);
      k_ir_check<<<1, 1, 0, s>>>(sc_, rmax, st.ir_abstol, st.ir_reltol, st.ir_stop_ratio);
      rc = ldl_solve_add(s, v_.r, 1);
      if (rc) return rc;
    }
    CLR_CHECK_LAUNCH();
    return CLR_OK;
  }
  // graph capture: condition set by the check before the node and at the end of each body pass
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  cudaGraphConditionalHandle h;
  residual(s);
  CLR_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
  CLR_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 0, 0));
  k_ir_check_cond<<<1, 1, 0, s>>>(sc_, rmax, st.ir_abstol, st.ir_reltol, st.ir_stop_ratio, st.ir_max_steps, h);
  CLR_CHECK_LAUNCH();
  CLR_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, &edata, &ndeps));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CLR_CUDA(cudaGraphAddNode(&node, cg, deps, edata, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CLR_CUDA(cudaStreamBeginCaptureToGraph(body_stream_, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  rc = ldl_solve_add(body_stream_, v_.r, 1);
  residual(body_stream_);
  k_ir_check_cond<<<1, 1, 0, body_stream_>>>(sc_, rmax, st.ir_abstol, st.ir_reltol, st.ir_stop_ratio,
                                             st.ir_max_steps, h);
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
                      double* lo, double* hi, const double* rhs, double* out, const int* skip) {
  const int kg = grid_for((r1 - r0) * G, 256, 16 * kSMs);
  k_kmv<G><<<kg, 256, 0, s>>>(mode, r0, r1, n, v.kptr, v.kcol, v.kvi, v.kval, x, lo, hi, rhs, out, nullptr, skip);
}
void kmv(int G, cudaStream_t s, int mode, int64_t r0, int64_t r1, int64_t n, const VecDev& v, const double* x,
         double* lo, double* hi, const double* rhs, double* out, const int* skip) {
  if (r1 <= r0) return;
  switch (G) {
    case 32: launch_kmv_split<32>(s, mode, r0, r1, n, v, x, lo, hi, rhs, out, skip); break;
    case 16: launch_kmv_split<16>(s, mode, r0, r1, n, v, x, lo, hi, rhs, out, skip); break;
    case 8: launch_kmv_split<8>(s, mode, r0, r1, n, v, x, lo, hi, rhs, out, skip); break;
    default: launch_kmv_split<4>(s, mode, r0, r1, n, v, x, lo, hi, rhs, out, skip); break;
  }
}
}  // namespace

// One search direction: solve with the current right-hand side (rhs built by
// k_rhs), Delta tau, Delta x/z, Delta s = -d_s - H Delta z.
int Solver::direction(bool affine) {
  const int64_t n = hp.n, m = hp.m, N = n + m;
  cudaStream_t s = stream_;
  const int* halt = &sc_->halt;
  double* dir = affine ? v_.dir_a : v_.dir;
  double* ds = affine ? v_.dsa : v_.ds;
  int rc = kkt_solve(v_.rhs, v_.sol1);
  if (rc) return rc;
  k_dots<<<kRedBlocks, kRedThreads, 0, s>>>(v_.qp, v_.sol1, n, v_.b, v_.sol1 + n, m, nullptr, nullptr, 0, v_.part,
                                            S_D0, halt);
  k_fin_dtau<<<1, 256, 0, s>>>(sc_, v_.part, halt);
  k_recover<<<grid_for(N, 256), 256, 0, s>>>(dir, v_.sol1, v_.sol2, N, sc_, halt);
  kmv(csr_group_, s, 2, n, N, n, v_, dir, nullptr, nullptr, v_.dsrhs, ds, halt);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

int Solver::step_length(bool combined) {
  const int64_t n = hp.n, m = hp.m;
  cudaStream_t s = stream_;
  const int* halt = &sc_->halt;
  const double* dir = combined ? v_.dir : v_.dir_a;
  const double* ds = combined ? v_.ds : v_.dsa;
  k_step_begin<<<1, 1, 0, s>>>(sc_, halt);
  int rc = cones_step_symmetric(s, cd_, v_.s, ds, v_.xz + n, dir + n, &sc_->amin_bits, halt);
  if (rc) return rc;
  k_fin_step_sym<<<1, 1, 0, s>>>(sc_, halt);
  const bool nonsym = (cd_.n_exp + cd_.n_pow) > 0;
  if (nonsym) {
    if (combined) {
      k_dots<<<kRedBlocks, kRedThreads, 0, s>>>(v_.s, dir + n, m, ds, v_.xz + n, m, ds, dir + n, m, v_.part, S_D0,
                                                halt);
      k_mu_coef<<<1, 256, 0, s>>>(sc_, v_.part, hp.cl.nu, halt);
    }
    rc = cones_step_nonsym(s, cd_, v_.s, ds, v_.xz + n, dir + n, &sc_->alpha_sym, st.backtrack, combined ? 1 : 0,
                           st.nbhd_beta, sc_->mu_coef, &sc_->ns, halt);
    if (rc) return rc;
  }
  StepParams sp{st.backtrack, st.min_step, st.nbhd_beta, st.step_fraction, nonsym ? 1 : 0, hp.cl.nu,
                st.max_iter + 1};
  k_fin_step<<<1, 1, 0, s>>>(sc_, sp, combined ? 1 : 0, v_.hist, halt);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

// Algorithm 1, one pass of steps 12 (residuals, here at the top), 4-11.
int Solver::iteration() {
  const int64_t n = hp.n, m = hp.m, N = n + m;
  cudaStream_t s = stream_;
  const int* halt = &sc_->halt;
  unsigned long long* maxb = reinterpret_cast<unsigned long long*>(v_.r);  // r is free here; 8 slots
  int rc;
  mark(2);
  // ---- residuals, objectives, mu, termination ----
  kmv(csr_group_, s, 0, 0, N, n, v_, v_.xz, v_.lo, v_.hi, nullptr, nullptr, halt);
  CLR_CUDA(cudaMemsetAsync(maxb, 0, sizeof(unsigned long long) * M_NMAX, s));
  k_resid_x<<<kRedBlocks, kRedThreads, 0, s>>>(n, v_.xz, v_.lo, v_.hi, v_.q, v_.D, sc_, v_.G, v_.qp, v_.part, maxb,
                                               halt);
  k_resid_z<<<kRedBlocks, kRedThreads, 0, s>>>(n, m, v_.xz, v_.s, v_.lo, v_.b, v_.E, sc_, v_.G, v_.part, maxb, halt);
  TermParams tp{hp.c, hp.bnorm, hp.qnorm, st.eps_feas, st.eps_inf, hp.cl.nu, st.max_iter, st.max_iter + 1};
  k_fin_resid<<<1, 256, 0, s>>>(sc_, v_.part, maxb, tp, v_.hist, halt);
  // ---- step 4: scaling H, KKT values; static + proportional regularisation ----
  CLR_CUDA(cudaMemsetAsync(&sc_->hmax_bits, 0, sizeof(unsigned long long), s));
  rc = cones_scaling(s, cd_, v_.s, v_.xz + n, &sc_->mu, &sc_->hmax_bits, halt);
  if (rc) return rc;
  k_fin_delta<<<1, 1, 0, s>>>(sc_, st.static_reg, st.static_reg_dyn, hp.maxPdiag, halt);
  // ---- step 5: factor ----
  mark(3);
  rc = factor();
  if (rc) return rc;
  mark(4);
  // ---- constant right-hand side [-q; b] ----
  k_build_rhs_init<<<grid_for(N, 256), 256, 0, s>>>(v_.rhs, v_.q, v_.b, n, m, 1);
  // k_build_rhs_init(which=1) gives [-q; 0]; add b on the z part
  k_set_from<double><<<grid_for(m, 256), 256, 0, s>>>(v_.rhs + n, v_.b, m, 1, halt);
  rc = kkt_solve(v_.rhs, v_.sol2);
  if (rc) return rc;
  k_dots<<<kRedBlocks, kRedThreads, 0, s>>>(v_.qp, v_.sol2, n, v_.b, v_.sol2 + n, m, nullptr, nullptr, 0, v_.part,
                                            S_D0, halt);
  k_fin_const<<<1, 256, 0, s>>>(sc_, v_.part, halt);
  // ---- step 6: affine direction, d = (G, d_s = s, d_kappa = kappa tau) ----
  CLR_CUDA(cudaMemcpyAsync(v_.dsrhs, v_.s, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, s));
  k_rhs<<<grid_for(N, 256), 256, 0, s>>>(v_.rhs, v_.G, v_.dsrhs, n, m, 0.0, sc_, 1, halt);
  rc = direction(true);
  if (rc) return rc;
  // ---- steps 7-8: affine step length, sigma ----
  rc = step_length(false);
  if (rc) return rc;
  // ---- step 9: combined direction ----
  rc = cones_combined_ds(s, cd_, v_.s, v_.xz + n, v_.dsa, v_.dir_a + n, &sc_->sigma_mu, v_.dsrhs, halt);
  if (rc) return rc;
  k_rhs<<<grid_for(N, 256), 256, 0, s>>>(v_.rhs, v_.G, v_.dsrhs, n, m, 0.0, sc_, 0, halt);
  rc = direction(false);
  if (rc) return rc;
  // ---- step 10: combined step length with the neighbourhood check ----
  rc = step_length(true);
  if (rc) return rc;
  // ---- step 11: update ----
  k_update<<<grid_for(N, 256), 256, 0, s>>>(v_.xz, v_.s, v_.dir, v_.ds, N, m, sc_, st.step_fraction, halt);
  const int* dh = (st.factor_bits == 64) ? f64_.dyn_hits : f32_.dyn_hits;
  k_fin_update<<<1, 1, 0, s>>>(sc_, st.step_fraction, dh, halt);
  mark(5);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

int Solver::initialise() {
  const int64_t n = hp.n, m = hp.m, N = n + m;
  cudaStream_t s = stream_;
  mark(0);
  k_init_scal<<<1, 1, 0, s>>>(sc_);
  CLR_CUDA(cudaMemsetAsync(v_.xz, 0, sizeof(double) * (size_t)N, s));
  CLR_CUDA(cudaMemsetAsync(v_.s, 0, sizeof(double) * (size_t)m, s));
  if (hp.cl.symmetric_only) {
    int rc = cones_identity_H(s, cd_, nullptr);
    if (rc) return rc;
    k_init_delta<<<1, 1, 0, s>>>(sc_, st.static_reg, st.static_reg_dyn, hp.maxPdiag);
    rc = factor();
    if (rc) return rc;
    k_build_rhs_init<<<grid_for(N, 256), 256, 0, s>>>(v_.rhs, v_.q, v_.b, n, m, 0);
    rc = kkt_solve(v_.rhs, v_.sol1);
    if (rc) return rc;
    k_init_take<<<grid_for(N, 256), 256, 0, s>>>(v_.xz, v_.s, v_.sol1, n, m, 0);
    k_build_rhs_init<<<grid_for(N, 256), 256, 0, s>>>(v_.rhs, v_.q, v_.b, n, m, 1);
    rc = kkt_solve(v_.rhs, v_.sol1);
    if (rc) return rc;
    k_init_take<<<grid_for(N, 256), 256, 0, s>>>(v_.xz, v_.s, v_.sol1, n, m, 1);
    rc = cones_shift_init(s, cd_, v_.s, v_.r, nullptr);
    if (rc) return rc;
    rc = cones_shift_init(s, cd_, v_.xz + n, v_.r, nullptr);
    if (rc) return rc;
  } else {
    int rc = cones_unit_init(s, cd_, v_.s, nullptr);
    if (rc) return rc;
    rc = cones_init_shadow(s, cd_, nullptr);
    if (rc) return rc;
    rc = cones_unit_init(s, cd_, v_.xz + n, nullptr);
    if (rc) return rc;
  }
  k_init_scal<<<1, 1, 0, s>>>(sc_);  // tau = kappa = 1, counters reset (ir_total of the init dropped)
  mark(1);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

int Solver::launch_iteration() {
  if (!st.use_graph) return iteration();
  if (!gexec_) {
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
    graph_ = g;
    iter_kernels_ = count_kernel_nodes(graph_);
    body_kernels_ = ir_nodes_.empty() ? 0 : count_kernel_nodes(ir_nodes_.back());
    ir_nodes_.clear();
    CLR_CUDA(cudaGraphInstantiate(&gexec_, graph_, 0));
  }
  CLR_CUDA(cudaGraphLaunch(gexec_, stream_));
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

int Solver::solve() {
  if (!device_ready) return CLR_E_STATE;
  auto t0 = std::chrono::steady_clock::now();
  perf = clr_perf{};
  int rc = launch_init();
  if (rc) return rc;
  perf.kernel_launches += init_kernels_;
  perf.factorizations += hp.cl.symmetric_only ? 1 : 0;
  bool first = true;
  int status = 0;
  for (int it = 0; it <= st.max_iter + 1; ++it) {
    rc = launch_iteration();
    if (rc) return rc;
    perf.kernel_launches += iter_kernels_;
    CLR_CUDA(cudaMemcpyAsync(sc_host_, sc_, sizeof(IterScal), cudaMemcpyDeviceToHost, stream_));
    CLR_CUDA(cudaStreamSynchronize(stream_));
    float ms = 0.f;
    if (first) {
      if (cudaEventElapsedTime(&ms, ev_[0], ev_[1]) == cudaSuccess) perf.init_ms += ms;
      first = false;
    }
    status = sc_host_->status;
    if (status == 0 || status == CLR_INSUFFICIENT_PROGRESS) {
      // a full iteration ran (or stopped at its step-length test, after the factorization)
      if (cudaEventElapsedTime(&ms, ev_[2], ev_[3]) == cudaSuccess) perf.resid_cones_ms += ms;
      if (cudaEventElapsedTime(&ms, ev_[3], ev_[4]) == cudaSuccess) perf.factor_ms += ms;
      if (cudaEventElapsedTime(&ms, ev_[4], ev_[5]) == cudaSuccess) perf.solve_step_ms += ms;
      perf.factorizations += 1;
    } else if (cudaEventElapsedTime(&ms, ev_[2], ev_[5]) == cudaSuccess) {
      perf.resid_cones_ms += ms;  // the terminating pass only evaluates the residuals
    }
    if (status != 0) break;
  }
  perf.iterations = sc_host_->iter;
  if (st.use_graph) perf.kernel_launches += (int64_t)sc_host_->ir_total * body_kernels_;  // executed loop bodies
  perf.factor_flops = sy.flops;
  CLR_CUDA(cudaStreamSynchronize(stream_));
  solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  const IterScal& h = *sc_host_;
  info = clr_info{};
  info.status = status;
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
  info.solve_s = solve_s;
  const int rows = std::min(h.iter + 1, st.max_iter + 1);
  history.assign(12 * (size_t)rows, 0.0);
  CLR_CUDA(cudaMemcpy(history.data(), v_.hist, sizeof(double) * history.size(), cudaMemcpyDeviceToHost));
  solved_once = true;
  last_status = status;
  return CLR_OK;
}

int Solver::get_solution(double* x, double* sl, double* z, clr_info* out) {
  if (!solved_once) return CLR_E_STATE;
  const int64_t n = hp.n, m = hp.m;
  std::vector<double> xz(n + m), s(m);
  CLR_CUDA(cudaMemcpy(xz.data(), v_.xz, sizeof(double) * (size_t)(n + m), cudaMemcpyDeviceToHost));
  CLR_CUDA(cudaMemcpy(s.data(), v_.s, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost));
  const double tau = info.tau, c = hp.c;
  // unscale: x = D x^, s = s^ / E, z = E z^ / c
  std::vector<double> xu(n), su(m), zu(m);
  for (int64_t j = 0; j < n; ++j) xu[j] = hp.D[j] * xz[j];
  for (int64_t r = 0; r < m; ++r) {
    su[r] = s[r] / hp.E[r];
    zu[r] = hp.E[r] * xz[n + r] / c;
  }
  double fx = 1.0 / tau, fs = 1.0 / tau, fz = 1.0 / tau;
  const double nan = std::nan("");
  if (last_status == CLR_PRIMAL_INFEASIBLE) {
    double btz = 0;
    for (int64_t r = 0; r < m; ++r) btz += (hp.b[r] / hp.E[r]) * zu[r];
    fx = fs = nan;
    fz = -1.0 / btz;
  } else if (last_status == CLR_DUAL_INFEASIBLE) {
    double qtx = 0;
    for (int64_t j = 0; j < n; ++j) qtx += (hp.q[j] / (c * hp.D[j])) * xu[j];
    fx = fs = -1.0 / qtx;
    fz = nan;
  }
  if (x)
    for (int64_t j = 0; j < n; ++j) x[j] = xu[j] * fx;
  for (int64_t r = 0; r < m; ++r) {
    const int64_t orig = hp.row_perm[r];
    if (sl) sl[orig] = su[r] * fs;
    if (z) z[orig] = zu[r] * fz;
  }
  if (out) *out = info;
  return CLR_OK;
}

int Solver::update_qb(const double* q, const double* b) {
  int rc = set_qb(hp, q, b);
  if (rc) return rc;
  if (device_ready) {
    CLR_CUDA(cudaMemcpyAsync(v_.q, hp.q.data(), sizeof(double) * (size_t)hp.n, cudaMemcpyHostToDevice, stream_));
    CLR_CUDA(cudaMemcpyAsync(v_.b, hp.b.data(), sizeof(double) * (size_t)hp.m, cudaMemcpyHostToDevice, stream_));
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
