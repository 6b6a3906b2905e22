// Cone kernels (see cones.cuh).  FP64 throughout.
//
// Readings shared with the rest of the solver: f is the barrier of the dual
// cone K* (Sec. 2.2), the central path is s = -mu grad f(z); the scaling H in
// Eq. linsys_4x4 satisfies H z = s; for SOC and PSD it is the Nesterov-Todd
// scaling H = W^T W with W z = W^{-T} s = lambda (Appendix A); for exp/pow
// it is the rank-4 BFGS matrix of Appendix A with S = [s, s~], Z = [z, z~],
// s~ = -grad f(z), z~ = -grad f*(s), H_a = mu Hess f(z), falling back to H_a
// when 1 - 9 / ((s'z)(s~'z~)) <= 1e-6.  PSD cones use svec (upper triangle by
// columns, off-diagonals times sqrt(2)).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "cones.cuh"
#include "psd_step.cuh"

namespace clr {

namespace {

constexpr double kSqrt2 = 1.4142135623730951;
constexpr double kBfgsDegeneracy = 1e-6;

// ------------------------------------------------------------------ exp / pow
struct Psi {
  double psi, g[3], h[3][3], sep1[3], sep2[3], sep3[3];
};

// f(z) = -log psi(z) + sum_i sep_i(z_i) for the dual exp / dual pow barrier.
__device__ void psi_parts(bool is_exp, const double* z, double a, Psi& P) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P.h[i][j] = 0.0;
  if (is_exp) {
    const double r = z[0], s = z[1], t = z[2];
    P.psi = s - r - r * log(t / (-r));
    P.g[0] = log(-r / t);
    P.g[1] = 1.0;
    P.g[2] = -r / t;
    P.h[0][0] = 1.0 / r;
    P.h[0][2] = P.h[2][0] = -1.0 / t;
    P.h[2][2] = r / (t * t);
    P.sep1[0] = -1.0 / r; P.sep1[1] = 0.0; P.sep1[2] = -1.0 / t;
    P.sep2[0] = 1.0 / (r * r); P.sep2[1] = 0.0; P.sep2[2] = 1.0 / (t * t);
    P.sep3[0] = -2.0 / (r * r * r); P.sep3[1] = 0.0; P.sep3[2] = -2.0 / (t * t * t);
  } else {
    const double u = z[0], v = z[1], w = z[2];
    const double pa = 2.0 * a, pb = 2.0 * (1.0 - a);
    const double phi = exp(pa * log(u / a) + pb * log(v / (1.0 - a)));
    P.psi = phi - w * w;
    P.g[0] = pa * phi / u;
    P.g[1] = pb * phi / v;
    P.g[2] = -2.0 * w;
    P.h[0][0] = pa * (pa - 1.0) * phi / (u * u);
    P.h[0][1] = P.h[1][0] = pa * pb * phi / (u * v);
    P.h[1][1] = pb * (pb - 1.0) * phi / (v * v);
    P.h[2][2] = -2.0;
    P.sep1[0] = -(1.0 - a) / u; P.sep1[1] = -a / v; P.sep1[2] = 0.0;
    P.sep2[0] = (1.0 - a) / (u * u); P.sep2[1] = a / (v * v); P.sep2[2] = 0.0;
    P.sep3[0] = -2.0 * (1.0 - a) / (u * u * u); P.sep3[1] = -2.0 * a / (v * v * v); P.sep3[2] = 0.0;
  }
}

// third derivatives of psi
__device__ double psi3(bool is_exp, const double* z, double a, int i, int j, int k, double phi_or_zero) {
  if (is_exp) {
    const double r = z[0], t = z[2];
    const int n0 = (i == 0) + (j == 0) + (k == 0), n1 = (i == 1) + (j == 1) + (k == 1), n2 = 3 - n0 - n1;
    if (n1) return 0.0;
    if (n0 == 3) return -1.0 / (r * r);
    if (n0 == 1 && n2 == 2) return 1.0 / (t * t);
    if (n2 == 3) return -2.0 * r / (t * t * t);
    return 0.0;
  }
  if (i == 2 || j == 2 || k == 2) return 0.0;
  const double u = z[0], v = z[1];
  const double pa = 2.0 * a, pb = 2.0 * (1.0 - a);
  const int nu = (i == 0) + (j == 0) + (k == 0), nv = 3 - nu;
  double cu = 1.0, cv = 1.0;
  for (int q = 0; q < nu; ++q) cu *= (pa - q);
  for (int q = 0; q < nv; ++q) cv *= (pb - q);
  double den = 1.0;
  for (int q = 0; q < nu; ++q) den *= u;
  for (int q = 0; q < nv; ++q) den *= v;
  return cu * cv * phi_or_zero / den;
}

__device__ void barrier_grad(bool is_exp, const double* z, double a, double* g) {
  Psi P;
  psi_parts(is_exp, z, a, P);
  for (int i = 0; i < 3; ++i) g[i] = -P.g[i] / P.psi + P.sep1[i];
}

__device__ void barrier_hess(bool is_exp, const double* z, double a, double H[3][3]) {
  Psi P;
  psi_parts(is_exp, z, a, P);
  const double ip = 1.0 / P.psi, ip2 = ip * ip;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) H[i][j] = P.g[i] * P.g[j] * ip2 - P.h[i][j] * ip + (i == j ? P.sep2[i] : 0.0);
}

// x = H^{-1} b for a symmetric positive definite 3x3 H (Cholesky).
__device__ bool spd3_solve(const double H[3][3], const double* b, double* x) {
  double L00 = H[0][0];
  if (!(L00 > 0)) return false;
  L00 = sqrt(L00);
  const double L10 = H[1][0] / L00, L20 = H[2][0] / L00;
  double L11 = H[1][1] - L10 * L10;
  if (!(L11 > 0)) return false;
  L11 = sqrt(L11);
  const double L21 = (H[2][1] - L20 * L10) / L11;
  double L22 = H[2][2] - L20 * L20 - L21 * L21;
  if (!(L22 > 0)) return false;
  L22 = sqrt(L22);
  const double y0 = b[0] / L00, y1 = (b[1] - L10 * y0) / L11, y2 = (b[2] - L20 * y0 - L21 * y1) / L22;
  x[2] = y2 / L22;
  x[1] = (y1 - L21 * x[2]) / L11;
  x[0] = (y0 - L10 * x[1] - L20 * x[2]) / L00;
  return true;
}

__device__ bool in_int_primal(bool is_exp, const double* s, double a) {
  if (is_exp) {
    const double x = s[0], y = s[1], z = s[2];
    return y > 0 && z > 0 && y * log(z / y) - x > 0;
  }
  const double x = s[0], y = s[1], z = s[2];
  return x > 0 && y > 0 && exp(a * log(x) + (1.0 - a) * log(y)) - fabs(z) > 0;
}

__device__ bool in_int_dual(bool is_exp, const double* z, double a) {
  if (is_exp) {
    const double u = z[0], v = z[1], w = z[2];
    return u < 0 && w > 0 && 1.0 + log(w) - log(-u) - v / u > 0;
  }
  const double u = z[0], v = z[1], w = z[2];
  return u > 0 && v > 0 && exp(a * log(u / a) + (1.0 - a) * log(v / (1.0 - a))) - fabs(w) > 0;
}

__device__ void central_point(bool is_exp, double a, const double* exp_c, double* u) {
  if (is_exp) {
    u[0] = exp_c[0];
    u[1] = exp_c[1];
    u[2] = exp_c[2];
  } else {
    u[0] = sqrt(1.0 + a);
    u[1] = sqrt(2.0 - a);
    u[2] = 0.0;
  }
}

// z~ = -grad f*(s): damped Newton on f(u) + <s, u> from `start` (a point of int K*).
__device__ bool dual_shadow(bool is_exp, const double* s, double a, const double* start, double* u) {
  u[0] = start[0];
  u[1] = start[1];
  u[2] = start[2];
  for (int it = 0; it < 100; ++it) {
    double g[3], H[3][3], du[3], mg[3];
    barrier_grad(is_exp, u, a, g);
    for (int i = 0; i < 3; ++i) {
      g[i] += s[i];
      mg[i] = -g[i];
    }
    barrier_hess(is_exp, u, a, H);
    if (!spd3_solve(H, mg, du)) return false;
    const double lam2 = -(g[0] * du[0] + g[1] * du[1] + g[2] * du[2]);
    if (lam2 < 1e-28) {
      for (int i = 0; i < 3; ++i) u[i] += du[i];
      return true;
    }
    const double lam = sqrt(fmax(lam2, 0.0));
    const double step = lam < 0.25 ? 1.0 : 1.0 / (1.0 + lam);
    for (int i = 0; i < 3; ++i) u[i] += step * du[i];
  }
  return true;
}

__device__ void inv2(const double M[2][2], double R[2][2]) {
  const double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
  R[0][0] = M[1][1] / det;
  R[1][1] = M[0][0] / det;
  R[0][1] = -M[0][1] / det;
  R[1][0] = -M[1][0] / det;
}

__device__ void bfgs_H(bool is_exp, const double* s, const double* z, double mu, double a, const double* start,
                       double H[3][3], double* zt) {
  double g[3], Ha[3][3], st[3];
  barrier_grad(is_exp, z, a, g);
  for (int i = 0; i < 3; ++i) st[i] = -g[i];
  barrier_hess(is_exp, z, a, Ha);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Ha[i][j] *= mu;
  const bool ok = dual_shadow(is_exp, s, a, start, zt);
  const double sz = s[0] * z[0] + s[1] * z[1] + s[2] * z[2];
  const double stzt = st[0] * zt[0] + st[1] * zt[1] + st[2] * zt[2];
  if (!ok || !(1.0 - 9.0 / (sz * stzt) > kBfgsDegeneracy)) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) H[i][j] = Ha[i][j];
    return;
  }
  const double* Sc[2] = {s, st};
  const double* Zc[2] = {z, zt};
  double SZ[2][2], SZi[2][2];
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q) SZ[p][q] = Sc[p][0] * Zc[q][0] + Sc[p][1] * Zc[q][1] + Sc[p][2] * Zc[q][2];
  inv2(SZ, SZi);
  double HaZ[3][2];
  for (int i = 0; i < 3; ++i)
    for (int q = 0; q < 2; ++q) HaZ[i][q] = Ha[i][0] * Zc[q][0] + Ha[i][1] * Zc[q][1] + Ha[i][2] * Zc[q][2];
  double ZHZ[2][2], ZHZi[2][2];
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q) ZHZ[p][q] = Zc[p][0] * HaZ[0][q] + Zc[p][1] * HaZ[1][q] + Zc[p][2] * HaZ[2][q];
  inv2(ZHZ, ZHZi);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t1 = 0.0, t2 = 0.0;
      for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
          t1 += Sc[p][i] * SZi[p][q] * Sc[q][j];
          t2 += HaZ[i][p] * ZHZi[p][q] * HaZ[j][q];
        }
      H[i][j] = t1 + Ha[i][j] - t2;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) {
      const double v = 0.5 * (H[i][j] + H[j][i]);
      H[i][j] = H[j][i] = v;
    }
}

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }


// ------------------------------------------------------------------ SOC helpers
// Warp-cooperative: lanes stride over the d entries of one cone.
struct SocScal {
  double eta, wb0, w1z1;
};

}  // namespace

// ====================================================================== scaling
__global__ void k_scale_nonneg(ConeDev cd, const double* __restrict__ s, const double* __restrict__ z, IterScal* sc,
                               const int* skip) {
  if (skip && *skip) return;
  RunExt<true> mx;
  const int64_t nz = cd.m_zero, nn = cd.m_nonneg;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nz + nn; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nz) {
      cd.kvz[i] = 0.0;  // zero cone: H = 0
      continue;
    }
    // lambda = sqrt(s z), w = s / lambda = sqrt(s / z), H = w^2 (one square root and
    // one division: FP64 division and square root dominate this pass on GB300)
    const double si = s[i], zi = z[i];
    const double lam = sqrt(si * zi);
    const double wi = si / lam;
    const double h = wi * wi;
    cd.kvz[i] = -h;
    cd.nn_w[i - nz] = wi;
    cd.nn_lam[i - nz] = lam;
    if (h > 0) mx.add(sc, &IterScal::hmax_bits, cd.row_pid[i], dbits(h));
  }
  mx.flush(sc, &IterScal::hmax_bits);
}

// Lanes per SOC: groups of G lanes of a warp (G = 8 when every SOC has at most 8
// rows, else 32) each take one cone at a time; reductions are G-lane butterflies.
template <int G>
__device__ __forceinline__ double gsum(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int G>
__device__ __forceinline__ double gmax(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// A SOC of at most kSocT rows in dense form: the thread-per-cone kernels take it.
// In a cohort that also holds larger (or expanded) SOCs each kernel family takes
// its own cones (ConeDev::soc_split), so that a cone's arithmetic does not depend
// on which other problems share the launch.
constexpr int kSocT = 8;
__device__ __forceinline__ bool soc_small(const ConeDev& cd, int64_t c) {
  return cd.soc_dim[c] <= kSocT && !(cd.soc_aux && cd.soc_aux[c] >= 0);
}
// The cones of a warp in pass k: (w + k nw) 32/G + g, g the lane group.  Every
// lane of a warp runs the same passes (shuffles need the whole warp); a group
// past the last cone works on an empty cone (d = 0) and writes nothing.
#define SOC_GROUP_LOOP(G)                                                                \
  constexpr int PG = 32 / (G);                                                           \
  const int lane = threadIdx.x & ((G) - 1);                                              \
  const int64_t w_ = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;              \
  const int64_t nw_ = ((int64_t)gridDim.x * blockDim.x) >> 5;                            \
  for (int64_t base = w_ * PG; base < cd.n_soc; base += nw_ * PG)

// blocks of 256 threads for the SOC kernels: one pass over the cones when that
// takes at most 16 blocks per SM, else grid-stride passes
inline unsigned soc_grid(const ConeDev& cd, int G) {
  const int64_t warps = (cd.n_soc * G + 31) / 32;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 16 * kSMs));
}

// Launch shape of the thread-per-cone exp/pow kernels: their FP64 transcendental
// work (logs, exponentials, Newton steps) is bound by the SM's FP64 pipe (~2 DFMA
// per clock on a GB300), so few cones are spread over as many SMs as possible
// (blocks of ceil(n / 152) threads, at most 128) rather than packed into few.
struct EpLaunch {
  unsigned blocks;
  int threads;
};
inline EpLaunch ep_launch(int64_t nc) {
  const int64_t t = std::min<int64_t>(128, std::max<int64_t>(1, (nc + kSMs - 1) / kSMs));
  return EpLaunch{(unsigned)((nc + t - 1) / t), (int)t};
}

template <int G>
__global__ void k_scale_soc(ConeDev cd, const double* __restrict__ s, const double* __restrict__ z, IterScal* sc,
                            const int* skip) {
  if (skip && *skip) return;
  RunExt<true> run;
  SOC_GROUP_LOOP(G) {
    const int64_t cone = base + (threadIdx.x & 31) / G;
    const bool valid = cone < cd.n_soc && !(cd.soc_split && soc_small(cd, cone));
    const int64_t off = valid ? cd.soc_off[cone] : 0;
    const int d = valid ? cd.soc_dim[cone] : 0;
    const double* sv = s + off;
    const double* zc = z + off;
    double s1 = 0, z1 = 0, sz = 0;
    for (int j = lane; j < d; j += G) {
      const double a = sv[j], b = zc[j];
      if (j > 0) {
        s1 += a * a;
        z1 += b * b;
      }
      sz += a * b;
    }
    s1 = gsum<G>(s1);
    z1 = gsum<G>(z1);
    sz = gsum<G>(sz);
    const double s0 = valid ? sv[0] : 1.0, z0 = valid ? zc[0] : 1.0;
    const double ns1 = sqrt(s1), nz1 = sqrt(z1);
    const double ns = sqrt((s0 - ns1) * (s0 + ns1)), nzj = sqrt((z0 - nz1) * (z0 + nz1));
    const double sbzb = sz / (ns * nzj);
    const double gamma = sqrt(0.5 * (1.0 + sbzb));
    const double eta = sqrt(ns / nzj);
    const double inv2g = 1.0 / (2.0 * gamma);
    // w-bar and the products needed for lambda = eta W-bar z
    double wz = 0, w1z1 = 0;
    for (int j = lane; j < d; j += G) {
      const double wb = (j == 0) ? (s0 / ns + z0 / nzj) * inv2g : (sv[j] / ns - zc[j] / nzj) * inv2g;
      cd.soc_wb[off + j] = wb;
      wz += wb * zc[j];
      if (j > 0) w1z1 += wb * zc[j];
    }
    wz = gsum<G>(wz);
    w1z1 = gsum<G>(w1z1);
    __syncwarp();
    const double wb0 = valid ? cd.soc_wb[off] : 1.0;
    const double coef = z0 + w1z1 / (1.0 + wb0);
    for (int j = lane; j < d; j += G) {
      const double lam = (j == 0) ? eta * wz : eta * (zc[j] + coef * cd.soc_wb[off + j]);
      cd.soc_lam[off + j] = lam;
    }
    if (lane == 0 && valid) cd.soc_eta[cone] = eta;
    // H = eta^2 (2 wb wb' - J), packed lower, column-major; KKT value is -H
    const double e2 = eta * eta;
    double* kb = cd.kvz + (valid ? cd.soc_kb[cone] : 0);
    double mx = 0.0;
    const int64_t aux = (valid && cd.soc_aux) ? cd.soc_aux[cone] : -1;  // uniform over the group
    if (aux >= 0) {
      // sparse form of a large SOC (Sec. 3.3 names cones of thousands of rows, whose dense H
      // block would hold d (d + 1) / 2 KKT values): 2 wb wb' - J = I + 2 (wb wb' - e0 e0'),
      // and the rank-two part has, in the basis e0, w^ = (0, wb_1) / r (r = ||wb_1||, wb0^2 - r^2 = 1),
      // the matrix 2 [r^2, wb0 r; wb0 r, r^2]: eigenvectors (e0 +- w^) / sqrt 2, eigenvalues
      // 2 r (r +- wb0).  So H = eta^2 (I + u u' - v v') with u = sqrt(r (r + wb0)) (e0 + w^) and
      // v = sqrt(r / (r + wb0)) (e0 - w^), v'v = 2 r / (r + wb0) < 1 (the matrix with the two
      // extra rows stays quasi-definite).  Column i: -eta^2 on the diagonal, eta u_i and
      // eta v_i in the two auxiliary rows.
      double r2 = 0.0;
      for (int j = lane; j < d; j += G)
        if (j > 0) r2 += cd.soc_wb[off + j] * cd.soc_wb[off + j];
      r2 = gsum<G>(r2);
      const double r = sqrt(r2);
      const double cu = r > 0.0 ? sqrt(r * (r + wb0)) : 0.0, cv = r > 0.0 ? sqrt(r / (r + wb0)) : 0.0;
      const double ir = r > 0.0 ? 1.0 / r : 0.0;
      for (int j = lane; j < d; j += G) {
        const double wj = cd.soc_wb[off + j];
        const double uj = (j == 0) ? cu : cu * wj * ir, vj = (j == 0) ? cv : -cv * wj * ir;
        kb[3 * j] = -e2;
        kb[3 * j + 1] = eta * uj;
        kb[3 * j + 2] = eta * vj;
        mx = fmax(mx, fabs(e2 * (2.0 * wj * wj + ((j == 0) ? -1.0 : 1.0))));  // H_jj
      }
    } else {
      int64_t kbase = 0;
      for (int c = 0; c < d; ++c) {
        const double wc = cd.soc_wb[off + c];
        for (int r = c + lane; r < d; r += G) {
          double h = 2.0 * e2 * cd.soc_wb[off + r] * wc;
          if (r == c) {
            h += (c == 0) ? -e2 : e2;
            mx = fmax(mx, fabs(h));
          }
          kb[kbase + (r - c)] = -h;
        }
        kbase += d - c;
      }
    }
    mx = gmax<G>(mx);
    if (lane == 0 && valid) run.add(sc, &IterScal::hmax_bits, cd.row_pid[off], dbits(mx));
    __syncwarp();
  }
  run.flush(sc, &IterScal::hmax_bits);
}

// ---------------------------------------------------------------- small SOCs, a thread per cone
// When every SOC has at most kSocT rows (the common case: SOC(3..8) in MPC, portfolio
// and the mixed-cone QP) one thread holds a cone's rows in registers.  The per-cone
// scalars -- J-norms, gamma, eta and their square roots and divisions -- are then
// computed once per cone, where a lane group computed them once per lane; these passes
// are bound by the FP64 pipe (~2 DFMA per clock per SM), so the redundant work was
// what they spent their time on.  The formulas are those of the lane-group kernels.
inline unsigned soc_t_grid(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16 * kSMs));
}
#define SOC_THREAD_LOOP \
  for (int64_t cone = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cone < cd.n_soc; \
       cone += (int64_t)gridDim.x * blockDim.x) \
    if (!cd.soc_split || soc_small(cd, cone))

__global__ void __launch_bounds__(256) k_scale_soc_t(ConeDev cd, const double* __restrict__ s,
                                                     const double* __restrict__ z, IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  RunExt<true> run;
  SOC_THREAD_LOOP {
    const int64_t off = cd.soc_off[cone];
    const int d = cd.soc_dim[cone];
    double sv[kSocT], zv[kSocT], wb[kSocT];
#pragma unroll
    for (int j = 0; j < kSocT; ++j) {
      sv[j] = j < d ? s[off + j] : 0.0;
      zv[j] = j < d ? z[off + j] : 0.0;
    }
    double s1 = 0, z1 = 0, sz = sv[0] * zv[0];
#pragma unroll
    for (int j = 1; j < kSocT; ++j) {
      s1 += sv[j] * sv[j];
      z1 += zv[j] * zv[j];
      sz += sv[j] * zv[j];
    }
    const double ns1 = sqrt(s1), nz1 = sqrt(z1);
    const double ns = sqrt((sv[0] - ns1) * (sv[0] + ns1)), nzj = sqrt((zv[0] - nz1) * (zv[0] + nz1));
    const double sbzb = sz / (ns * nzj);
    const double gamma = sqrt(0.5 * (1.0 + sbzb));
    const double eta = sqrt(ns / nzj);
    const double inv2g = 1.0 / (2.0 * gamma);
    const double rs = 1.0 / ns, rz = 1.0 / nzj;
    double wz = 0, w1z1 = 0;
#pragma unroll
    for (int j = 0; j < kSocT; ++j) {
      wb[j] = (j == 0) ? (sv[0] * rs + zv[0] * rz) * inv2g : (sv[j] * rs - zv[j] * rz) * inv2g;
      wz += wb[j] * zv[j];
      if (j > 0) w1z1 += wb[j] * zv[j];
    }
    const double coef = zv[0] + w1z1 / (1.0 + wb[0]);
#pragma unroll
    for (int j = 0; j < kSocT; ++j) {
      if (j >= d) continue;
      cd.soc_wb[off + j] = wb[j];
      cd.soc_lam[off + j] = (j == 0) ? eta * wz : eta * (zv[j] + coef * wb[j]);
    }
    cd.soc_eta[cone] = eta;
    // H = eta^2 (2 wb wb' - J), packed lower, column-major; KKT value is -H
    const double e2 = eta * eta;
    double* kb = cd.kvz + cd.soc_kb[cone];
    double mx = 0.0;
    int q = 0;
#pragma unroll
    for (int c = 0; c < kSocT; ++c) {
#pragma unroll
      for (int r = c; r < kSocT; ++r) {
        if (r >= d || c >= d) continue;
        double h = 2.0 * e2 * wb[r] * wb[c];
        if (r == c) {
          h += (c == 0) ? -e2 : e2;
          mx = fmax(mx, fabs(h));
        }
        kb[q++] = -h;
      }
    }
    run.add(sc, &IterScal::hmax_bits, cd.row_pid[off], dbits(mx));
  }
  run.flush(sc, &IterScal::hmax_bits);
}

__device__ __forceinline__ double soc_step_t(const double* x, const double* dx) {
  double a2 = 0, b2 = 0, c2 = 0;
#pragma unroll
  for (int j = 1; j < kSocT; ++j) {
    a2 += dx[j] * dx[j];
    b2 += x[j] * dx[j];
    c2 += x[j] * x[j];
  }
  const double A = dx[0] * dx[0] - a2;
  const double B = x[0] * dx[0] - b2;
  const double C = x[0] * x[0] - c2;
  double r = INFINITY;
  if (A == 0.0) {
    if (B < 0) r = -C / (2.0 * B);
  } else {
    const double disc = B * B - A * C;
    if (disc >= 0) {
      const double sq = sqrt(disc);
      const double r1 = (-B - sq) / A, r2 = (-B + sq) / A;
      if (r1 > 0) r = fmin(r, r1);
      if (r2 > 0) r = fmin(r, r2);
    }
  }
  if (dx[0] < 0) r = fmin(r, -x[0] / dx[0]);
  return r;
}

__global__ void __launch_bounds__(256) k_step_soc_t(ConeDev cd, const double* __restrict__ s,
                                                    const double* __restrict__ ds, const double* __restrict__ z,
                                                    const double* __restrict__ dz, IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  RunExt<false> run;
  SOC_THREAD_LOOP {
    const int64_t off = cd.soc_off[cone];
    const int d = cd.soc_dim[cone];
    double x[kSocT], dx[kSocT], y[kSocT], dy[kSocT];
#pragma unroll
    for (int j = 0; j < kSocT; ++j) {
      x[j] = j < d ? s[off + j] : 0.0;
      dx[j] = j < d ? ds[off + j] : 0.0;
      y[j] = j < d ? z[off + j] : 0.0;
      dy[j] = j < d ? dz[off + j] : 0.0;
    }
    const double a = d > 0 ? fmin(soc_step_t(x, dx), soc_step_t(y, dy)) : INFINITY;
    if (a < INFINITY) run.add(sc, &IterScal::amin_bits, cd.row_pid[off], dbits(a));
  }
  run.flush(sc, &IterScal::amin_bits);
}

// y = W-bar x, or J W-bar J x (jconj), for one cone in registers
__device__ __forceinline__ void soc_wbar_t(const double* wb, const double* x, double* y, bool jconj) {
  double w1x1 = 0;
#pragma unroll
  for (int j = 1; j < kSocT; ++j) w1x1 += wb[j] * x[j];
  const double w0 = wb[0], x0 = x[0];
  if (!jconj) {
    const double coef = x0 + w1x1 / (1.0 + w0);
    y[0] = w0 * x0 + w1x1;
#pragma unroll
    for (int j = 1; j < kSocT; ++j) y[j] = x[j] + coef * wb[j];
  } else {
    const double coef = x0 - w1x1 / (1.0 + w0);
    y[0] = w0 * x0 - w1x1;
#pragma unroll
    for (int j = 1; j < kSocT; ++j) y[j] = x[j] - coef * wb[j];
  }
}

// d_s = W (lambda \ (lambda o lambda + (W^{-1} ds_a) o (W dz_a) - sigma mu e)), W = eta W-bar
__global__ void __launch_bounds__(256) k_ds_soc_t(ConeDev cd, const double* __restrict__ dsa,
                                                  const double* __restrict__ dza, const IterScal* sc,
                                                  double* __restrict__ out, const int* skip) {
  if (skip && *skip) return;
  SOC_THREAD_LOOP {
    const int64_t off = cd.soc_off[cone];
    const int d = cd.soc_dim[cone];
    const double eta = cd.soc_eta[cone];
    double wb[kSocT], lam[kSocT], a[kSocT], b[kSocT], u[kSocT], v[kSocT];
#pragma unroll
    for (int j = 0; j < kSocT; ++j) {
      wb[j] = j < d ? cd.soc_wb[off + j] : 0.0;
      lam[j] = j < d ? cd.soc_lam[off + j] : 0.0;
      a[j] = j < d ? dsa[off + j] : 0.0;
      b[j] = j < d ? dza[off + j] : 0.0;
    }
    soc_wbar_t(wb, a, u, true);   // W-bar^{-1} ds_a = J W-bar J ds_a
    soc_wbar_t(wb, b, v, false);  // W-bar dz_a
    double uv = 0, ll = 0;
#pragma unroll
    for (int j = 0; j < kSocT; ++j) {
      u[j] /= eta;
      v[j] *= eta;
      uv += u[j] * v[j];
      ll += lam[j] * lam[j];
    }
    const double smu = sc[cd.row_pid[off]].sigma_mu;
    // w = lam o lam + u o v - sigma mu e  (into a)
    a[0] = ll + uv - smu;
#pragma unroll
    for (int j = 1; j < kSocT; ++j) a[j] = 2.0 * lam[0] * lam[j] + u[0] * v[j] + v[0] * u[j];
    double l1v = 0, l1sq = 0;
#pragma unroll
    for (int j = 1; j < kSocT; ++j) {
      l1v += lam[j] * a[j];
      l1sq += lam[j] * lam[j];
    }
    const double l0 = lam[0];
    const double x0 = (l0 * a[0] - l1v) / (l0 * l0 - l1sq);
    b[0] = x0;
#pragma unroll
    for (int j = 1; j < kSocT; ++j) b[j] = (a[j] - x0 * lam[j]) / l0;
    soc_wbar_t(wb, b, u, false);
#pragma unroll
    for (int j = 0; j < kSocT; ++j)
      if (j < d) out[off + j] = eta * u[j];
  }
}

__global__ void k_scale_exppow(ConeDev cd, const double* __restrict__ s, const double* __restrict__ z, IterScal* sc,
                               const int* skip) {
  if (skip && *skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cd.n_exp + cd.n_pow) return;
  const bool is_exp = t < cd.n_exp;
  const int64_t i = is_exp ? t : t - cd.n_exp;
  const int64_t row = is_exp ? cd.exp_row0 + 3 * i : cd.pow_row0 + 3 * i;
  const int64_t kb = is_exp ? cd.exp_kb0 + 6 * i : cd.pow_kb0 + 6 * i;
  const double a = is_exp ? 0.0 : cd.pow_alpha[i];
  double sv[3] = {s[row], s[row + 1], s[row + 2]}, zv[3] = {z[row], z[row + 1], z[row + 2]};
  double H[3][3], zt[3];
  double* zs = cd.ep_zt + 3 * t;
  const double start[3] = {zs[0], zs[1], zs[2]};
  const int pid = cd.row_pid[row];
  bfgs_H(is_exp, sv, zv, sc[pid].mu, a, start, H, zt);
  if (isfinite(zt[0]) && isfinite(zt[1]) && isfinite(zt[2]) && in_int_dual(is_exp, zt, a)) {
    zs[0] = zt[0];
    zs[1] = zt[1];
    zs[2] = zt[2];
  }
  int q = 0;
  double mx = 0.0;
  for (int c = 0; c < 3; ++c)
    for (int r = c; r < 3; ++r) {
      cd.kvz[kb + q++] = -H[r][c];
      if (r == c) mx = fmax(mx, fabs(H[r][c]));
    }
  atomicMax(&sc[pid].hmax_bits, dbits(mx));
}

// ---------------------------------------------------------------- PSD helpers
// All run with the whole block; matrices k x k in shared memory with leading dimension 33.
namespace {
constexpr int LDP = 33;

__device__ int smat_index(int i, int j) {  // svec index of (i, j), i <= j
  return j * (j + 1) / 2 + i;
}

__device__ void load_smat(const double* v, int k, double* M) {
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    const int a = min(i, j), b = max(i, j);
    const double x = v[smat_index(a, b)];
    M[i + j * LDP] = (i == j) ? x : x / kSqrt2;
  }
  __syncthreads();
}

// In-place lower Cholesky of M (upper part left untouched).  Sets *bad if not PD.
__device__ void chol(double* M, int k, int* bad) {
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = M[j + j * LDP];
      if (!(d > 0)) *bad = 1;
      M[j + j * LDP] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    const double ljj = M[j + j * LDP];
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) M[i + j * LDP] /= ljj;
    __syncthreads();
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
      const int i = q % k, l = q / k;
      if (l > j && i >= l) M[i + l * LDP] -= M[i + j * LDP] * M[l + j * LDP];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, l = q / k;
    if (i < l) M[i + l * LDP] = 0.0;
  }
  __syncthreads();
}

// Round-robin pairing of k' = k + (k odd) players: pair p of round r.
__device__ void rr_pair(int kk, int r, int p, int* a, int* b) {
  // player 0 fixed, others rotate
  auto pos = [&](int x) -> int { return x == 0 ? 0 : 1 + ((x - 1 + r) % (kk - 1)); };
  *a = pos(p);
  *b = pos(kk - 1 - p);
}

// One-sided Jacobi SVD of M (k x k): on exit M = U Sigma (columns), V
// accumulated, sig = column norms.  Warp w handles pair w of each round.
__device__ void jacobi_svd(double* M, double* V, double* sig, int k, int* flag) {
  const int kk = k + (k & 1);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) V[(q % k) + (q / k) * LDP] = (q % k == q / k) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < kk - 1; ++r) {
      for (int p = wid; p < kk / 2; p += nw) {
        int a, b;
        rr_pair(kk, r, p, &a, &b);
        if (a >= k || b >= k) continue;
        double al = 0, be = 0, ga = 0;
        for (int i = lane; i < k; i += 32) {
          const double x = M[i + a * LDP], y = M[i + b * LDP];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (fabs(ga) > 1e-15 * sqrt(al * be) && fabs(ga) > 1e-300) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
          for (int i = lane; i < k; i += 32) {
            const double x = M[i + a * LDP], y = M[i + b * LDP];
            M[i + a * LDP] = c * x - sn * y;
            M[i + b * LDP] = sn * x + c * y;
            const double vx = V[i + a * LDP], vy = V[i + b * LDP];
            V[i + a * LDP] = c * vx - sn * vy;
            V[i + b * LDP] = sn * vx + c * vy;
          }
          if (lane == 0) *flag = 1;
        }
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double nrm = 0;
    for (int i = 0; i < k; ++i) nrm += M[i + j * LDP] * M[i + j * LDP];
    sig[j] = sqrt(nrm);
  }
  __syncthreads();
}

// Parallel two-sided Jacobi (Brent-Luk) eigenvalues of the symmetric A (k x k);
// returns the smallest eigenvalue (valid in all threads).
__device__ double jacobi_eigmin(double* A, int k, double* cs_buf, int* flag) {
  const int kk = k + (k & 1);
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < kk - 1; ++r) {
      for (int p = threadIdx.x; p < kk / 2; p += blockDim.x) {
        int a, b;
        rr_pair(kk, r, p, &a, &b);
        double c = 1.0, sn = 0.0;
        if (a < k && b < k) {
          const double apq = A[a + b * LDP], app = A[a + a * LDP], aqq = A[b + b * LDP];
          if (fabs(apq) > 1e-15 * sqrt(fabs(app * aqq)) && fabs(apq) > 1e-300) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = c * t;
            *flag = 1;
          }
        }
        cs_buf[2 * p] = c;
        cs_buf[2 * p + 1] = sn;
      }
      __syncthreads();
      // rows: A <- J^T A  (pair rows a, b)
      for (int q = threadIdx.x; q < (kk / 2) * k; q += blockDim.x) {
        const int p = q / k, col = q % k;
        int a, b;
        rr_pair(kk, r, p, &a, &b);
        if (a >= k || b >= k) continue;
        const double c = cs_buf[2 * p], sn = cs_buf[2 * p + 1];
        const double x = A[a + col * LDP], y = A[b + col * LDP];
        A[a + col * LDP] = c * x - sn * y;
        A[b + col * LDP] = sn * x + c * y;
      }
      __syncthreads();
      // columns: A <- A J
      for (int q = threadIdx.x; q < (kk / 2) * k; q += blockDim.x) {
        const int p = q / k, row = q % k;
        int a, b;
        rr_pair(kk, r, p, &a, &b);
        if (a >= k || b >= k) continue;
        const double c = cs_buf[2 * p], sn = cs_buf[2 * p + 1];
        const double x = A[row + a * LDP], y = A[row + b * LDP];
        A[row + a * LDP] = c * x - sn * y;
        A[row + b * LDP] = sn * x + c * y;
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
  double mn = INFINITY;
  for (int i = 0; i < k; ++i) mn = fmin(mn, A[i + i * LDP]);
  return mn;
}
}  // namespace

// PSD scaling: L_s L_s' = S, L_z L_z' = Z, L_z' L_s = U Lambda V', R = L_s V Lambda^{-1/2},
// R^{-1} = Lambda^{-1/2} U' L_z', H(X) = (R R') X (R R') written as the svec block.
// PSD cone holding row r (r >= psd_row0): binary search over the cones' first rows
__device__ __forceinline__ int64_t psd_cone_of(const ConeDev& cd, int64_t r) {
  int64_t lo = 0, hi = cd.n_psd - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (cd.psd_crow[mid] <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_scale_psd(ConeDev cd, const int32_t* __restrict__ list, const double* __restrict__ s,
                            const double* __restrict__ z, IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  __shared__ double Ls[32 * LDP], Lz[32 * LDP], M[32 * LDP], V[32 * LDP], sig[32];
  __shared__ int bad, flag;
  const int64_t cone = list[blockIdx.x];
  const int k = cd.psd_ck[cone], d = k * (k + 1) / 2;
  const int64_t row = cd.psd_crow[cone];
  if (threadIdx.x == 0) bad = 0;
  load_smat(s + row, k, Ls);
  load_smat(z + row, k, Lz);
  chol(Ls, k, &bad);
  chol(Lz, k, &bad);
  // M = Lz' Ls
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += Lz[l + i * LDP] * Ls[l + j * LDP];
    M[i + j * LDP] = acc;
  }
  __syncthreads();
  jacobi_svd(M, V, sig, k, &flag);
  double* R = cd.psd_R + cd.psd_cR[cone];
  double* Ri = cd.psd_Ri + cd.psd_cR[cone];
  double* lam = cd.psd_lam + cd.psd_cl[cone];
  for (int j = threadIdx.x; j < k; j += blockDim.x) lam[j] = bad ? NAN : sig[j];
  // R = Ls V diag(sig^-1/2); Ri = diag(sig^-1/2) U' Lz' with U = M / sig (columns)
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += Ls[i + l * LDP] * V[l + j * LDP];
    R[i + j * k] = acc / sqrt(sig[j]);
    double acc2 = 0;  // (U' Lz')_{ij} = sum_l U_{li} Lz_{jl}
    for (int l = 0; l < k; ++l) acc2 += (M[l + i * LDP] / sig[i]) * Lz[j + l * LDP];
    Ri[i + j * k] = acc2 / sqrt(sig[i]);
  }
  __syncthreads();
  // Mrr = R R' (reuse Ls)
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += R[i + l * k] * R[j + l * k];
    V[i + j * LDP] = acc;
  }
  __syncthreads();
  // H_{(i,j),(p,q)} = c_ij c_pq (M_ip M_jq + M_iq M_jp), c = 1/sqrt(2) on diagonal pairs;
  // packed lower over svec indices (row index >= column index), column-major.
  double* kb = cd.kvz + cd.psd_ckb[cone];
  double mx = 0.0;
  const int64_t npk = (int64_t)d * (d + 1) / 2;
  for (int64_t t = threadIdx.x; t < npk; t += blockDim.x) {
    // packed column-major lower: find column cidx with start(c) <= t < start(c+1), start(c) = c d - c(c-1)/2
    int cidx = 0;
    {
      int lo = 0, hi = d - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        const int64_t st = (int64_t)mid * d - (int64_t)mid * (mid - 1) / 2;
        if (st <= t) lo = mid;
        else hi = mid - 1;
      }
      cidx = lo;
    }
    const int64_t start = (int64_t)cidx * d - (int64_t)cidx * (cidx - 1) / 2;
    const int ridx = cidx + (int)(t - start);
    // svec index -> (i, j), i <= j: j = largest with j(j+1)/2 <= idx
    auto decode = [&](int idx, int* ii, int* jj) {
      int j = (int)((sqrt(8.0 * idx + 1.0) - 1.0) / 2.0);
      while (j * (j + 1) / 2 > idx) --j;
      while ((j + 1) * (j + 2) / 2 <= idx) ++j;
      *jj = j;
      *ii = idx - j * (j + 1) / 2;
    };
    int i, j, p, q;
    decode(ridx, &i, &j);
    decode(cidx, &p, &q);
    const double cij = (i == j) ? 1.0 / kSqrt2 : 1.0, cpq = (p == q) ? 1.0 / kSqrt2 : 1.0;
    const double h = cij * cpq *
                     (V[i + p * LDP] * V[j + q * LDP] + V[i + q * LDP] * V[j + p * LDP]);
    kb[t] = -h;
    if (ridx == cidx) mx = fmax(mx, fabs(h));
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) atomicMax(&sc[cd.row_pid[row]].hmax_bits, dbits(mx));
}

// PSD scaling of the cones of order k <= KM (KM = 4, 8 or 16): a group of KM lanes
// per cone, lane j holding column j of each k x k matrix in registers, so that the
// scalar work of a Jacobi rotation (two norms, the angle, cos and sin) is done once
// per column pair by its two lanes instead of once per pair by a whole warp (an
// FP64 warp instruction occupies the FP64 pipe of its sub-partition whatever the
// number of active lanes).  The same steps as k_scale_psd: Cholesky factors of S
// and Z, M = Lz' Ls, one-sided cyclic Jacobi on M with the same round-robin pair
// order, R = Ls V Lambda^{-1/2}, R^{-1} = Lambda^{-1/2} U' Lz', and the packed -H
// block from W = R R'.  Differences in rounding only: the Cholesky scales a column
// by the reciprocal of its pivot, and the column sums run over rows, not lanes.
// Every loop that shuffles runs the warp's largest trip count; the extra rounds,
// steps and sweeps are no-ops for a smaller cone, so a cone's result does not
// depend on the cones sharing its warp.
template <int KM>
__global__ void __launch_bounds__(128, 1) k_scale_psd_lane(ConeDev cd, const int32_t* __restrict__ list, int64_t nlist,
                                                        const double* __restrict__ s, const double* __restrict__ z,
                                                        IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  constexpr int LD = KM + 1;           // column stride in shared memory (column writes on distinct banks)
  constexpr int MAT = KM * LD;         // one k x k matrix
  constexpr int PER = 2 * MAT + 1;     // two per cone, odd stride between the cones of a warp
  constexpr int CPB = 128 / KM;        // cones per block
  constexpr int DM = KM * (KM + 1) / 2;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ double sm[CPB * PER];
  __shared__ unsigned char tab_i[DM], tab_j[DM];  // svec index -> (i, j), i <= j
  for (int t = threadIdx.x; t < DM; t += blockDim.x) {
    int j = 0;
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    tab_j[t] = (unsigned char)j;
    tab_i[t] = (unsigned char)(t - j * (j + 1) / 2);
  }
  __syncthreads();
  const int c = threadIdx.x % KM;  // my column
  const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / KM;
  const bool live = slot < nlist;
  const int64_t cone = live ? list[slot] : 0;
  const int k = live ? cd.psd_ck[cone] : 0;
  const int64_t row = live ? cd.psd_crow[cone] : 0;
  double* A = sm + (threadIdx.x / KM) * PER;  // Ls, later R
  double* B = A + MAT;                        // Lz, later W
  int kw = k;  // the warp's largest order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kw = max(kw, __shfl_xor_sync(FULL, kw, o));

  // ---- Cholesky factors of S (into A) and Z (into B), column c in registers
  int bad = 0;
  double col[KM];
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    const double* v = (pass == 0 ? s : z) + row;
#pragma unroll
    for (int i = 0; i < KM; ++i) {
      double x = 0.0;
      if (c < k && i < k) {
        const int a = min(i, c), b = max(i, c);
        x = v[b * (b + 1) / 2 + a];
        if (i != c) x /= kSqrt2;
      }
      col[i] = x;
    }
#pragma unroll 1
    for (int p = 0; p < kw; ++p) {  // (kw: uniform over the warp)
      if (c == p && p < k) {
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < KM; ++i)
          if (i == p) d = col[i];
        if (!(d > 0)) bad = 1;
        const double l = sqrt(fmax(d, 1e-300));
        const double rl = 1.0 / l;
#pragma unroll
        for (int i = 0; i < KM; ++i) {
          if (i == p) col[i] = l;
          else if (i > p) col[i] *= rl;
        }
      }
      // column p of L, from its owner; my own row's entry of it
      double lpc = 0.0;
      double lp[KM];
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        lp[i] = __shfl_sync(FULL, col[i], p, KM);
        if (i == c) lpc = lp[i];
      }
      if (c > p && c < k) {
#pragma unroll
        for (int i = 0; i < KM; ++i)
          if (i > p && i >= c && i < k) col[i] -= lp[i] * lpc;
      }
    }
    double* X = pass == 0 ? A : B;
#pragma unroll
    for (int i = 0; i < KM; ++i) X[i + c * LD] = (i >= c) ? col[i] : 0.0;
  }
  const unsigned seg_bits = ((1u << KM) - 1u) << ((threadIdx.x & 31) & ~(KM - 1));  // my cone's lanes
  const bool cone_bad = (__ballot_sync(FULL, bad) & seg_bits) != 0;
  __syncwarp();

  // ---- M = Lz' Ls (column c), V = I
  double mc[KM], vc[KM];
#pragma unroll
  for (int i = 0; i < KM; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < KM; ++l)
      if (l >= i && l >= c && l < k) acc += B[l + i * LD] * A[l + c * LD];
    mc[i] = (i < k && c < k) ? acc : 0.0;
    vc[i] = (i == c && c < k) ? 1.0 : 0.0;
  }

  // ---- one-sided cyclic Jacobi: round r pairs the columns as the round-robin
  // tournament of kk = k + (k odd) players (column 0 fixed, the others rotating)
  const int kk = k + (k & 1), kkw = kw + (kw & 1);
  for (int sweep = 0; sweep < 40; ++sweep) {
    int rot = 0;
    for (int r = 0; r < kkw - 1; ++r) {
      int partner = -1;
      bool first = false;
      if (c < k && r < kk - 1) {
        const int x = (c == 0) ? 0 : 1 + ((c - 1 - r) % (kk - 1) + (kk - 1)) % (kk - 1);
        const int y = kk - 1 - x;
        partner = (y == 0) ? 0 : 1 + ((y - 1 + r) % (kk - 1));
        first = x < kk / 2;
        if (partner >= k) partner = -1;
      }
      const int src = partner >= 0 ? partner : c;
      // rows k.. of a cone's columns are zero and stay zero, so the row loops run to
      // the warp's largest order (a uniform exit) without changing any sum
      double so = 0.0, sp = 0.0, ga = 0.0;
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        if (i >= kw) break;
        const double o = __shfl_sync(FULL, mc[i], src, KM);
        so += mc[i] * mc[i];
        sp += o * o;
        ga += mc[i] * o;
      }
      double cs = 1.0, sg = 0.0;
      if (partner >= 0) {
        const double al = first ? so : sp, be = first ? sp : so;  // the pair's (a, b) norms, same on both lanes
        if (fabs(ga) > 1e-15 * sqrt(al * be) && fabs(ga) > 1e-300) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          cs = 1.0 / sqrt(1.0 + t * t);
          const double sn = cs * t;
          sg = first ? -sn : sn;  // a' = c a - s b,  b' = s a + c b
          rot = 1;
        }
      }
      // (cs, sg) = (1, 0) leaves a column that does not rotate unchanged
#pragma unroll
      for (int i = 0; i < KM; ++i) {
        if (i >= kw) break;
        const double om = __shfl_sync(FULL, mc[i], src, KM);
        const double ov = __shfl_sync(FULL, vc[i], src, KM);
        mc[i] = cs * mc[i] + sg * om;
        vc[i] = cs * vc[i] + sg * ov;
      }
    }
    if (!__any_sync(FULL, rot)) break;
  }

  // ---- Lambda, R = Ls V Lambda^{-1/2} (column c), R^{-1} = Lambda^{-1/2} U' Lz' (row c)
  double nrm = 0.0;
#pragma unroll
  for (int i = 0; i < KM; ++i)
    if (i < k) nrm += mc[i] * mc[i];
  const double sig = sqrt(nrm), rs = sqrt(sig);
  double* Rg = live ? cd.psd_R + cd.psd_cR[cone] : nullptr;
  double* Rig = live ? cd.psd_Ri + cd.psd_cR[cone] : nullptr;
  if (c < k) cd.psd_lam[cd.psd_cl[cone] + c] = cone_bad ? NAN : sig;
#pragma unroll
  for (int i = 0; i < KM; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < KM; ++l)
      if (l <= i && l < k) acc += A[i + l * LD] * vc[l];
    col[i] = acc / rs;
    if (c < k && i < k) Rg[i + c * k] = col[i];
  }
#pragma unroll
  for (int l = 0; l < KM; ++l) mc[l] = (l < k) ? mc[l] / sig : 0.0;  // column c of U
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < KM; ++l)
      if (l <= j && l < k) acc += mc[l] * B[j + l * LD];
    if (c < k && j < k) Rig[c + j * k] = acc / rs;
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < KM; ++i) A[i + c * LD] = (c < k && i < k) ? col[i] : 0.0;  // R
  __syncwarp();
  // W = R R' (row c), then the packed lower -H over svec indices, column-major:
  // H_{(i,j),(p,q)} = c_ij c_pq (W_ip W_jq + W_iq W_jp), c = 1/sqrt(2) on diagonal pairs
#pragma unroll
  for (int l = 0; l < KM; ++l) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) acc += A[c + j * LD] * A[l + j * LD];
    B[c + l * LD] = acc;
  }
  __syncwarp();
  const int d = k * (k + 1) / 2;
  double* kb = live ? cd.kvz + cd.psd_ckb[cone] : nullptr;
  double mx = 0.0;
  for (int cc = 0; cc < d; ++cc) {
    const int p = tab_i[cc], q = tab_j[cc];
    const double cpq = (p == q) ? 1.0 / kSqrt2 : 1.0;
    const int64_t start = (int64_t)cc * d - (int64_t)cc * (cc - 1) / 2;
    for (int rr = cc + c; rr < d; rr += KM) {
      const int i = tab_i[rr], j = tab_j[rr];
      const double cij = (i == j) ? 1.0 / kSqrt2 : 1.0;
      const double h = cij * cpq * (B[i + p * LD] * B[j + q * LD] + B[i + q * LD] * B[j + p * LD]);
      kb[start + (rr - cc)] = -h;
      if (rr == cc) mx = fmax(mx, fabs(h));
    }
  }
#pragma unroll
  for (int o = KM / 2; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o, KM));
  if (live && c == 0) atomicMax(&sc[cd.row_pid[row]].hmax_bits, dbits(mx));
}

int cones_scaling(cudaStream_t st, const ConeDev& cd, const double* s, const double* z, IterScal* sc,
                  const int* skip) {
  if (cd.m_zero + cd.m_nonneg > 0)
    k_scale_nonneg<<<grid_for(cd.m_zero + cd.m_nonneg, 256), 256, 0, st>>>(cd, s, z, sc, skip);
  if (cd.n_soc > 0) {
    // small dense SOCs a thread per cone; larger and expanded ones (sparse KKT form) a warp per cone
    if (cd.soc_nsmall > 0) k_scale_soc_t<<<soc_t_grid(cd.n_soc), 256, 0, st>>>(cd, s, z, sc, skip);
    if (cd.soc_nsmall < cd.n_soc) k_scale_soc<32><<<soc_grid(cd, 32), 256, 0, st>>>(cd, s, z, sc, skip);
  }
  if (cd.n_exp + cd.n_pow > 0)
    k_scale_exppow<<<ep_launch(cd.n_exp + cd.n_pow).blocks, ep_launch(cd.n_exp + cd.n_pow).threads, 0, st>>>(
        cd, s, z, sc, skip);
  if (cd.n_psd > 0) {
    // orders up to 16: a lane per column (4, 8 or 16 lanes per cone); larger: a block per cone
    if (cd.psd_nlist[0] > 0)
      k_scale_psd_lane<4><<<grid_for(cd.psd_nlist[0] * 4, 128, 1 << 30), 128, 0, st>>>(cd, cd.psd_list[0],
                                                                                      cd.psd_nlist[0], s, z, sc, skip);
    if (cd.psd_nlist[1] > 0)
      k_scale_psd_lane<8><<<grid_for(cd.psd_nlist[1] * 8, 128, 1 << 30), 128, 0, st>>>(cd, cd.psd_list[1],
                                                                                      cd.psd_nlist[1], s, z, sc, skip);
    if (cd.psd_nlist[2] > 0)
      k_scale_psd_lane<16><<<grid_for(cd.psd_nlist[2] * 16, 128, 1 << 30), 128, 0, st>>>(
          cd, cd.psd_list[2], cd.psd_nlist[2], s, z, sc, skip);
    if (cd.psd_nlist[3] > 0) {
      const int threads = 32 * ((cd.psd_kmax + 1) / 2 > 0 ? (cd.psd_kmax + 1) / 2 : 1);
      k_scale_psd<<<(unsigned)cd.psd_nlist[3], threads < 64 ? 64 : threads, 0, st>>>(cd, cd.psd_list[3], s, z, sc,
                                                                                   skip);
    }
  }
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

// ---------------------------------------------------------------- H = I
__global__ void k_identity_diag(ConeDev cd, const int* skip) {
  if (skip && *skip) return;
  const int64_t total = cd.m;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
    // locate the packed diagonal entry of row r
    if (r < cd.m_zero + cd.m_nonneg) {
      cd.kvz[r] = -1.0;
      continue;
    }
    // SOC: binary search the cone
    int64_t lo = 0, hi = cd.n_soc - 1;
    if (cd.n_soc > 0 && r < cd.soc_off[cd.n_soc - 1] + cd.soc_dim[cd.n_soc - 1]) {
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (cd.soc_off[mid] <= r) lo = mid;
        else hi = mid - 1;
      }
      const int64_t c = r - cd.soc_off[lo];
      const int64_t d = cd.soc_dim[lo];
      const bool expanded = cd.soc_aux && cd.soc_aux[lo] >= 0;  // its couplings stay 0 (u = v = 0)
      cd.kvz[cd.soc_kb[lo] + (expanded ? 3 * c : c * d - c * (c - 1) / 2)] = -1.0;
      continue;
    }
    if (cd.n_aux > 0 && r >= cd.aux_begin) {  // auxiliary rows: their constant diagonals
      const int64_t k = r - cd.aux_begin;
      cd.kvz[cd.nkz - cd.n_aux + k] = (k % 2 == 0) ? 1.0 : -1.0;
      continue;
    }
    if (r >= cd.exp_row0 && r < cd.exp_row0 + 3 * cd.n_exp) {
      const int64_t i = (r - cd.exp_row0) / 3, c = (r - cd.exp_row0) % 3;
      cd.kvz[cd.exp_kb0 + 6 * i + c * 3 - c * (c - 1) / 2] = -1.0;
      continue;
    }
    if (r >= cd.pow_row0 && r < cd.pow_row0 + 3 * cd.n_pow) {
      const int64_t i = (r - cd.pow_row0) / 3, c = (r - cd.pow_row0) % 3;
      cd.kvz[cd.pow_kb0 + 6 * i + c * 3 - c * (c - 1) / 2] = -1.0;
      continue;
    }
    if (cd.n_psd > 0 && r >= cd.psd_row0) {
      const int64_t i = psd_cone_of(cd, r);
      const int64_t kk = cd.psd_ck[i], d = kk * (kk + 1) / 2, c = r - cd.psd_crow[i];
      cd.kvz[cd.psd_ckb[i] + c * d - c * (c - 1) / 2] = -1.0;
    }
  }
}

int cones_identity_H(cudaStream_t st, const ConeDev& cd, const int* skip) {
  CLR_CUDA(cudaMemsetAsync(cd.kvz, 0, sizeof(double) * (size_t)cd.nkz, st));
  k_identity_diag<<<grid_for(cd.m, 256), 256, 0, st>>>(cd, skip);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

// ====================================================================== step length
__global__ void k_step_nonneg(ConeDev cd, const double* __restrict__ s, const double* __restrict__ ds,
                              const double* __restrict__ z, const double* __restrict__ dz, IterScal* sc,
                              const int* skip) {
  if (skip && *skip) return;
  // a ratio -x / dx is divided out only when it can beat the thread's running
  // minimum (x <= best (-dx) (1 + 1e-15) covers every quotient that rounds to at
  // most best): the FP64 divisions, not the loads, bounded this pass
  RunExt<false> mn;
  const int64_t b0 = cd.m_zero, b1 = cd.m_zero + cd.m_nonneg;
  double best = INFINITY;
  int bpid = -1;
  for (int64_t i = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b1; i += (int64_t)gridDim.x * blockDim.x) {
    const double dsi = ds[i], dzi = dz[i];
    if (!(dsi < 0) && !(dzi < 0)) continue;
    const int pid = cd.row_pid[i];
    if (pid != bpid) {
      best = INFINITY;
      bpid = pid;
    }
    if (dsi < 0) {
      const double num = s[i], den = -dsi;
      if (num <= best * den * (1.0 + 1e-15)) {
        const double a = num / den;
        best = fmin(best, a);
        mn.add(sc, &IterScal::amin_bits, pid, dbits(a));
      }
    }
    if (dzi < 0) {
      const double num = z[i], den = -dzi;
      if (num <= best * den * (1.0 + 1e-15)) {
        const double a = num / den;
        best = fmin(best, a);
        mn.add(sc, &IterScal::amin_bits, pid, dbits(a));
      }
    }
  }
  mn.flush(sc, &IterScal::amin_bits);
}

namespace {
// Largest alpha with x + alpha dx in the closed SOC (smallest positive root of
// the J-norm quadratic, and t + alpha dt >= 0); G-lane cooperative, result in all
// lanes of the group (d = 0: no limit).
template <int G>
__device__ double soc_step(const double* x, const double* dx, int d) {
  const int lane = threadIdx.x & (G - 1);
  double a2 = 0, b2 = 0, c2 = 0;
  for (int j = lane; j < d; j += G) {
    if (j == 0) continue;
    a2 += dx[j] * dx[j];
    b2 += x[j] * dx[j];
    c2 += x[j] * x[j];
  }
  a2 = gsum<G>(a2);
  b2 = gsum<G>(b2);
  c2 = gsum<G>(c2);
  if (d == 0) return INFINITY;
  const double A = dx[0] * dx[0] - a2;
  const double B = x[0] * dx[0] - b2;
  const double C = x[0] * x[0] - c2;
  double r = INFINITY;
  if (A == 0.0) {
    if (B < 0) r = -C / (2.0 * B);
  } else {
    const double disc = B * B - A * C;
    if (disc >= 0) {
      const double sq = sqrt(disc);
      const double r1 = (-B - sq) / A, r2 = (-B + sq) / A;
      if (r1 > 0) r = fmin(r, r1);
      if (r2 > 0) r = fmin(r, r2);
    }
  }
  if (dx[0] < 0) r = fmin(r, -x[0] / dx[0]);
  return r;
}
}  // namespace

template <int G>
__global__ void k_step_soc(ConeDev cd, const double* __restrict__ s, const double* __restrict__ ds,
                           const double* __restrict__ z, const double* __restrict__ dz, IterScal* sc,
                           const int* skip) {
  if (skip && *skip) return;
  RunExt<false> run;
  SOC_GROUP_LOOP(G) {
    const int64_t cone = base + (threadIdx.x & 31) / G;
    const bool valid = cone < cd.n_soc && !(cd.soc_split && soc_small(cd, cone));
    const int64_t off = valid ? cd.soc_off[cone] : 0;
    const int d = valid ? cd.soc_dim[cone] : 0;
    const double a = fmin(soc_step<G>(s + off, ds + off, d), soc_step<G>(z + off, dz + off, d));
    if (lane == 0 && valid && a < INFINITY) run.add(sc, &IterScal::amin_bits, cd.row_pid[off], dbits(a));
  }
  run.flush(sc, &IterScal::amin_bits);
}

// Step length of the PSD cones of order k <= KM, a thread per cone (the order-16
// arithmetic fills every lane of an FP64 warp instruction); one atomic per warp
// when the warp's cones belong to one problem.
template <int KM>
__global__ void __launch_bounds__(128) k_step_psd_thread(ConeDev cd, const int32_t* __restrict__ list, int64_t nlist,
                                                         const double* __restrict__ s, const double* __restrict__ ds,
                                                         const double* __restrict__ z, const double* __restrict__ dz,
                                                         IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  constexpr unsigned FULL = 0xffffffffu;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = t < nlist;
  double amax = INFINITY;
  int pid = -1;
  if (live) {
    const int64_t cone = list[t];
    const int k = cd.psd_ck[cone];
    const int64_t row = cd.psd_crow[cone];
    pid = cd.row_pid[row];
    amax = fmin(psd_step_side<KM>(s + row, ds + row, k), psd_step_side<KM>(z + row, dz + row, k));
  }
  const int pid0 = __shfl_sync(FULL, pid, 0);  // (dead lanes are the warp's last)
  if (__all_sync(FULL, !live || pid == pid0)) {
    double m = amax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0 && live && m < INFINITY) atomicMin(&sc[pid0].amin_bits, dbits(m));
  } else if (live && amax < INFINITY) {
    atomicMin(&sc[pid].amin_bits, dbits(amax));
  }
}

__global__ void k_step_psd(ConeDev cd, const int32_t* __restrict__ list, const double* __restrict__ s,
                           const double* __restrict__ ds, const double* __restrict__ z, const double* __restrict__ dz,
                           IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  __shared__ double L[32 * LDP], X[32 * LDP], Y[32 * LDP], csb[64];
  __shared__ int bad, flag;
  const int64_t cone = list[blockIdx.x];
  const int k = cd.psd_ck[cone];
  const int64_t row = cd.psd_crow[cone];
  double amax = INFINITY;
  for (int side = 0; side < 2; ++side) {
    const double* v = side == 0 ? s + row : z + row;
    const double* dv = side == 0 ? ds + row : dz + row;
    if (threadIdx.x == 0) bad = 0;
    load_smat(v, k, L);
    load_smat(dv, k, X);
    chol(L, k, &bad);
    // Y = L^{-1} dX (forward substitution per column, thread per column)
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      for (int i = 0; i < k; ++i) {
        double acc = X[i + j * LDP];
        for (int l = 0; l < i; ++l) acc -= L[i + l * LDP] * Y[l + j * LDP];
        Y[i + j * LDP] = acc / L[i + i * LDP];
      }
    __syncthreads();
    // X = L^{-1} Y' (Y' = dX L^{-T}); result symmetric
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      for (int i = 0; i < k; ++i) {
        double acc = Y[j + i * LDP];
        for (int l = 0; l < i; ++l) acc -= L[i + l * LDP] * X[l + j * LDP];
        X[i + j * LDP] = acc / L[i + i * LDP];
      }
    __syncthreads();
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
      const int i = q % k, j = q / k;
      if (i < j) {
        const double avg = 0.5 * (X[i + j * LDP] + X[j + i * LDP]);
        X[i + j * LDP] = avg;
        X[j + i * LDP] = avg;
      }
    }
    __syncthreads();
    const double lmin = jacobi_eigmin(X, k, csb, &flag);
    if (lmin < 0) amax = fmin(amax, -1.0 / lmin);
    if (bad || !(lmin == lmin)) amax = 0.0;  // not positive definite in floating point, or NaN: no step
    __syncthreads();
  }
  if (threadIdx.x == 0 && amax < INFINITY) atomicMin(&sc[cd.row_pid[row]].amin_bits, dbits(amax));
}

int cones_step_symmetric(cudaStream_t st, const ConeDev& cd, const double* s, const double* ds, const double* z,
                         const double* dz, IterScal* sc, const int* skip) {
  if (cd.m_nonneg > 0) k_step_nonneg<<<grid_for(cd.m_nonneg, 256), 256, 0, st>>>(cd, s, ds, z, dz, sc, skip);
  if (cd.n_soc > 0) {
    if (cd.soc_nsmall > 0) k_step_soc_t<<<soc_t_grid(cd.n_soc), 256, 0, st>>>(cd, s, ds, z, dz, sc, skip);
    if (cd.soc_nsmall < cd.n_soc) k_step_soc<32><<<soc_grid(cd, 32), 256, 0, st>>>(cd, s, ds, z, dz, sc, skip);
  }
  if (cd.n_psd > 0) {
    // orders up to 16: a thread per cone (tridiagonalisation and Sturm bisection);
    // larger: a block per cone (two-sided Jacobi)
    if (cd.psd_nlist[0] > 0)
      k_step_psd_thread<4><<<grid_for(cd.psd_nlist[0], 128, 1 << 30), 128, 0, st>>>(cd, cd.psd_list[0],
                                                                                   cd.psd_nlist[0], s, ds, z, dz, sc,
                                                                                   skip);
    if (cd.psd_nlist[1] > 0)
      k_step_psd_thread<8><<<grid_for(cd.psd_nlist[1], 128, 1 << 30), 128, 0, st>>>(cd, cd.psd_list[1],
                                                                                   cd.psd_nlist[1], s, ds, z, dz, sc,
                                                                                   skip);
    if (cd.psd_nlist[2] > 0)
      k_step_psd_thread<16><<<grid_for(cd.psd_nlist[2], 128, 1 << 30), 128, 0, st>>>(cd, cd.psd_list[2],
                                                                                    cd.psd_nlist[2], s, ds, z, dz, sc,
                                                                                    skip);
    if (cd.psd_nlist[3] > 0) {
      const int threads = std::max(64, 32 * ((cd.psd_kmax + 1) / 2));
      k_step_psd<<<(unsigned)cd.psd_nlist[3], threads, 0, st>>>(cd, cd.psd_list[3], s, ds, z, dz, sc, skip);
    }
  }
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

namespace {
struct NsCone {
  bool is_exp;
  int pid;
  double a, sv[3], zv[3], dsv[3], dzv[3];
  const double* zt0;
};
__device__ NsCone load_cone(const ConeDev& cd, int64_t t, const double* s, const double* ds, const double* z,
                            const double* dz) {
  NsCone c;
  c.is_exp = t < cd.n_exp;
  const int64_t i = c.is_exp ? t : t - cd.n_exp;
  const int64_t row = c.is_exp ? cd.exp_row0 + 3 * i : cd.pow_row0 + 3 * i;
  c.a = c.is_exp ? 0.0 : cd.pow_alpha[i];
  c.pid = cd.row_pid[row];
  for (int q = 0; q < 3; ++q) {
    c.sv[q] = s[row + q];
    c.zv[q] = z[row + q];
    c.dsv[q] = ds[row + q];
    c.dzv[q] = dz[row + q];
  }
  c.zt0 = cd.ep_zt + 3 * t;
  return c;
}
__device__ bool ns_interior(const NsCone& c, double alpha) {
  double sc[3], zc[3];
  for (int q = 0; q < 3; ++q) {
    sc[q] = c.sv[q] + alpha * c.dsv[q];
    zc[q] = c.zv[q] + alpha * c.dzv[q];
  }
  return in_int_primal(c.is_exp, sc, c.a) && in_int_dual(c.is_exp, zc, c.a);
}
// nu <grad f*(s), grad f(z)>^{-1} >= beta mu at the trial point (nu = 3)
__device__ bool ns_nbhd(const NsCone& c, double alpha, const double* mu_coef, double beta) {
  double sc[3], zc[3], zt[3], g[3];
  for (int q = 0; q < 3; ++q) {
    sc[q] = c.sv[q] + alpha * c.dsv[q];
    zc[q] = c.zv[q] + alpha * c.dzv[q];
  }
  const double mu_t = mu_coef[0] + alpha * (mu_coef[1] + alpha * mu_coef[2]);
  const double start[3] = {c.zt0[0], c.zt0[1], c.zt0[2]};
  // a trial point whose grad f*(s) cannot be evaluated counts as outside N(beta)
  if (!dual_shadow(c.is_exp, sc, c.a, start, zt)) return false;
  barrier_grad(c.is_exp, zc, c.a, g);
  const double dot = -(zt[0] * g[0] + zt[1] * g[1] + zt[2] * g[2]);  // <z~, s~>, s~ = -grad f(z)
  return isfinite(dot) && dot > 0.0 && 3.0 / dot >= beta * mu_t;
}
}  // namespace

__global__ void k_ns_reset(IterScal* sc, int64_t nprob, const int* skip) {
  if (skip && *skip) return;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nprob; p += (int64_t)gridDim.x * blockDim.x) {
    sc[p].ns.jint = 0;
    sc[p].ns.fail = 0;
    sc[p].ns.mask = ~0ull;
  }
}

__global__ void k_ns_interior(ConeDev cd, const double* __restrict__ s, const double* __restrict__ ds,
                              const double* __restrict__ z, const double* __restrict__ dz, IterScal* sc,
                              double backtrack, const int* skip) {
  if (skip && *skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cd.n_exp + cd.n_pow) return;
  const NsCone c = load_cone(cd, t, s, ds, z, dz);
  double alpha = sc[c.pid].alpha_sym;
  int j = 0;
  while (j < 120 && !ns_interior(c, alpha)) {
    alpha *= backtrack;
    ++j;
  }
  atomicMax(&sc[c.pid].ns.jint, j);
}

__global__ void k_ns_first(ConeDev cd, const double* __restrict__ s, const double* __restrict__ ds,
                           const double* __restrict__ z, const double* __restrict__ dz, IterScal* sc,
                           double backtrack, double beta, const int* skip) {
  if (skip && *skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cd.n_exp + cd.n_pow) return;
  const NsCone c = load_cone(cd, t, s, ds, z, dz);
  IterScal& q = sc[c.pid];
  const double alpha = q.alpha_sym * pow(backtrack, (double)q.ns.jint);
  if (!ns_nbhd(c, alpha, q.mu_coef, beta)) atomicOr(&q.ns.fail, 1);
}

__global__ void k_ns_window(ConeDev cd, const double* __restrict__ s, const double* __restrict__ ds,
                            const double* __restrict__ z, const double* __restrict__ dz, IterScal* sc,
                            double backtrack, double beta, const int* skip) {
  if (skip && *skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cd.n_exp + cd.n_pow) return;
  const NsCone c = load_cone(cd, t, s, ds, z, dz);
  IterScal& q = sc[c.pid];
  if (!q.ns.fail) return;
  double alpha = q.alpha_sym * pow(backtrack, (double)(q.ns.jint + 1));
  unsigned long long bits = 0ull;
  for (int k = 0; k < 64; ++k) {
    if (ns_nbhd(c, alpha, q.mu_coef, beta)) bits |= (1ull << k);
    alpha *= backtrack;
  }
  atomicAnd(&q.ns.mask, bits);
}

int cones_step_nonsym(cudaStream_t st, const ConeDev& cd, const double* s, const double* ds, const double* z,
                      const double* dz, IterScal* sc, double backtrack, int nbhd, double beta, const int* skip) {
  k_ns_reset<<<grid_for(cd.nprob, 128), 128, 0, st>>>(sc, cd.nprob, skip);
  const int64_t nc = cd.n_exp + cd.n_pow;
  if (nc == 0) return CLR_OK;
  const EpLaunch el = ep_launch(nc);
  k_ns_interior<<<el.blocks, el.threads, 0, st>>>(cd, s, ds, z, dz, sc, backtrack, skip);
  if (nbhd) {
    k_ns_first<<<el.blocks, el.threads, 0, st>>>(cd, s, ds, z, dz, sc, backtrack, beta, skip);
    k_ns_window<<<el.blocks, el.threads, 0, st>>>(cd, s, ds, z, dz, sc, backtrack, beta, skip);
  }
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

__global__ void k_init_shadow(ConeDev cd, const int* skip) {
  if (skip && *skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cd.n_exp + cd.n_pow) return;
  const bool is_exp = t < cd.n_exp;
  const double a = is_exp ? 0.0 : cd.pow_alpha[t - cd.n_exp];
  central_point(is_exp, a, cd.exp_center, cd.ep_zt + 3 * t);
}

int cones_init_shadow(cudaStream_t st, const ConeDev& cd, const int* skip) {
  const int64_t nc = cd.n_exp + cd.n_pow;
  if (nc == 0) return CLR_OK;
  k_init_shadow<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(cd, skip);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

// ====================================================================== combined d_s
__global__ void k_ds_nonneg(ConeDev cd, const double* __restrict__ dsa, const double* __restrict__ dza,
                            const IterScal* sc, double* __restrict__ out, const int* skip) {
  if (skip && *skip) return;
  const int64_t nz = cd.m_zero, nn = cd.m_nonneg;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nz + nn; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nz) {
      out[i] = 0.0;
      continue;
    }
    const double w = cd.nn_w[i - nz], lam = cd.nn_lam[i - nz];
    const double eta = (dsa[i] / w) * (w * dza[i]);
    const double v = lam * lam + eta - sc[cd.row_pid[i]].sigma_mu;
    out[i] = w * (v / lam);
  }
}

namespace {
// y = W-bar x (warp), x, y of length d indexed by lane stride; wb in global.
template <int G>
__device__ void soc_wbar(const double* wb, const double* x, double* y, int d, bool jconj) {
  // jconj: y = J W-bar J x
  const int lane = threadIdx.x & (G - 1);
  double w1x1 = 0, w0 = d > 0 ? wb[0] : 1.0;
  for (int j = lane; j < d; j += G)
    if (j > 0) w1x1 += wb[j] * x[j];
  w1x1 = gsum<G>(w1x1);
  const double x0 = d > 0 ? x[0] : 0.0;
  __syncwarp();
  if (!jconj) {
    const double coef = x0 + w1x1 / (1.0 + w0);
    for (int j = lane; j < d; j += G) y[j] = (j == 0) ? w0 * x0 + w1x1 : x[j] + coef * wb[j];
  } else {
    const double coef = x0 - w1x1 / (1.0 + w0);
    for (int j = lane; j < d; j += G) y[j] = (j == 0) ? w0 * x0 - w1x1 : x[j] - coef * wb[j];
  }
  __syncwarp();
}
}  // namespace

// SOC: d_s = W (lambda \ (lambda o lambda + (W^{-1} ds_a) o (W dz_a) - sigma mu e)); W symmetric.
// Uses `out` on the cone's rows as scratch.
template <int G>
__global__ void k_ds_soc(ConeDev cd, const double* __restrict__ dsa, const double* __restrict__ dza,
                         const IterScal* sc, double* __restrict__ out, double* __restrict__ scratch,
                         const int* skip) {
  if (skip && *skip) return;
  SOC_GROUP_LOOP(G) {
    const int64_t cone = base + (threadIdx.x & 31) / G;
    const bool valid = cone < cd.n_soc && !(cd.soc_split && soc_small(cd, cone));
    const int64_t off = valid ? cd.soc_off[cone] : 0;
    const int d = valid ? cd.soc_dim[cone] : 0;
    const double eta = valid ? cd.soc_eta[cone] : 1.0;
    const double* wb = cd.soc_wb + off;
    const double* lam = cd.soc_lam + off;
    double* u = scratch + off;  // W^{-1} ds_a
    double* v = out + off;      // W dz_a, then the Jordan quotient
    soc_wbar<G>(wb, dsa + off, u, d, true);
    soc_wbar<G>(wb, dza + off, v, d, false);
    for (int j = lane; j < d; j += G) {
      u[j] /= eta;
      v[j] *= eta;
    }
    __syncwarp();
    // eta_c = u o v = (u'v, u0 v1 + v0 u1);  lambda o lambda = (|lam|^2, 2 lam0 lam1)
    double uv = 0, ll = 0, l1v = 0, l1sq = 0;
    for (int j = lane; j < d; j += G) {
      uv += u[j] * v[j];
      ll += lam[j] * lam[j];
    }
    uv = gsum<G>(uv);
    ll = gsum<G>(ll);
    const double u0 = valid ? u[0] : 0.0, v0 = valid ? v[0] : 0.0, l0 = valid ? lam[0] : 1.0;
    const double smu = valid ? sc[cd.row_pid[off]].sigma_mu : 0.0;
    __syncwarp();
    // w = lam o lam + eta_c - sigma mu e
    for (int j = lane; j < d; j += G) {
      const double wj = (j == 0) ? ll + uv - smu : 2.0 * l0 * lam[j] + u0 * v[j] + v0 * u[j];
      u[j] = wj;  // reuse u for w
    }
    __syncwarp();
    for (int j = lane; j < d; j += G)
      if (j > 0) {
        l1v += lam[j] * u[j];
        l1sq += lam[j] * lam[j];
      }
    l1v = gsum<G>(l1v);
    l1sq = gsum<G>(l1sq);
    const double w0 = valid ? u[0] : 0.0;
    const double x0 = (l0 * w0 - l1v) / (l0 * l0 - l1sq);
    __syncwarp();
    for (int j = lane; j < d; j += G) v[j] = (j == 0) ? x0 : (u[j] - x0 * lam[j]) / l0;
    __syncwarp();
    // out = W x = eta W-bar x (write through u as scratch)
    soc_wbar<G>(wb, v, u, d, false);
    for (int j = lane; j < d; j += G) out[off + j] = eta * u[j];
    __syncwarp();
  }
}

__global__ void k_ds_exppow(ConeDev cd, const double* __restrict__ s, const double* __restrict__ z,
                            const double* __restrict__ dsa, const double* __restrict__ dza, const IterScal* sc,
                            double* __restrict__ out, const int* skip) {
  if (skip && *skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cd.n_exp + cd.n_pow) return;
  const bool is_exp = t < cd.n_exp;
  const int64_t i = is_exp ? t : t - cd.n_exp;
  const int64_t row = is_exp ? cd.exp_row0 + 3 * i : cd.pow_row0 + 3 * i;
  const double a = is_exp ? 0.0 : cd.pow_alpha[i];
  const double zv[3] = {z[row], z[row + 1], z[row + 2]};
  double g[3], H[3][3], u[3] = {0.0, 0.0, 0.0};
  barrier_grad(is_exp, zv, a, g);
  barrier_hess(is_exp, zv, a, H);
  const double dsv[3] = {dsa[row], dsa[row + 1], dsa[row + 2]}, dzv[3] = {dza[row], dza[row + 1], dza[row + 2]};
  // a Hessian that is not positive definite in floating point (z at the boundary of
  // the dual cone to rounding) leaves u = 0: the third-order term is dropped
  spd3_solve(H, dsv, u);
  // eta = -1/2 sum_jk T_ijk dz_j u_k with T the third derivative of f
  Psi P;
  psi_parts(is_exp, zv, a, P);
  const double phi = is_exp ? 0.0 : P.psi + zv[2] * zv[2];
  const double ip = 1.0 / P.psi, ip2 = ip * ip, ip3 = ip2 * ip;
  const double smu = sc[cd.row_pid[row]].sigma_mu;
  for (int r = 0; r < 3; ++r) {
    double acc = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        double T = -psi3(is_exp, zv, a, r, j, k, phi) * ip +
                   (P.h[r][j] * P.g[k] + P.h[r][k] * P.g[j] + P.h[j][k] * P.g[r]) * ip2 -
                   2.0 * P.g[r] * P.g[j] * P.g[k] * ip3;
        if (r == j && j == k) T += P.sep3[r];
        acc += T * dzv[j] * u[k];
      }
    out[row + r] = s[row + r] + smu * g[r] - 0.5 * acc;
  }
}

// PSD: d_s = R (Lambda \ (Lambda^2 + eta - sigma mu I)) R', eta = (R^{-1} dS R^{-T}) o (R' dZ R).
__global__ void k_ds_psd(ConeDev cd, const double* __restrict__ dsa, const double* __restrict__ dza,
                         const IterScal* sc, double* __restrict__ out, const int* skip) {
  if (skip && *skip) return;
  __shared__ double A[32 * LDP], B[32 * LDP], T[32 * LDP];
  const int64_t cone = blockIdx.x;
  const int k = cd.psd_ck[cone];
  const int64_t row = cd.psd_crow[cone];
  const double* R = cd.psd_R + cd.psd_cR[cone];
  const double* Ri = cd.psd_Ri + cd.psd_cR[cone];
  const double* lam = cd.psd_lam + cd.psd_cl[cone];
  const double smu = sc[cd.row_pid[row]].sigma_mu;
  // A = Ri dS Ri'
  load_smat(dsa + row, k, A);
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += Ri[i + l * k] * A[l + j * LDP];
    T[i + j * LDP] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += T[i + l * LDP] * Ri[j + l * k];
    A[i + j * LDP] = acc;
  }
  __syncthreads();
  // B = R' dZ R
  load_smat(dza + row, k, B);
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += R[l + i * k] * B[l + j * LDP];
    T[i + j * LDP] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += T[i + l * LDP] * R[l + j * k];
    B[i + j * LDP] = acc;
  }
  __syncthreads();
  // V = Lambda^2 + (A B + B A)/2 - sigma mu I; X_ij = 2 V_ij / (lam_i + lam_j)  -> T
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double ab = 0, ba = 0;
    for (int l = 0; l < k; ++l) {
      ab += A[i + l * LDP] * B[l + j * LDP];
      ba += B[i + l * LDP] * A[l + j * LDP];
    }
    double v = 0.5 * (ab + ba);
    if (i == j) v += lam[i] * lam[i] - smu;
    T[i + j * LDP] = 2.0 * v / (lam[i] + lam[j]);
  }
  __syncthreads();
  // out = svec(R X R')
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += R[i + l * k] * T[l + j * LDP];
    A[i + j * LDP] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    if (i > j) continue;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += A[i + l * LDP] * R[j + l * k];
    // symmetric part of R X R' at (i, j)
    double acc2 = 0;
    for (int l = 0; l < k; ++l) acc2 += A[j + l * LDP] * R[i + l * k];
    const double val = 0.5 * (acc + acc2);
    out[row + smat_index(i, j)] = (i == j) ? val : val * kSqrt2;
  }
}

// Delta s = -d_s - H Delta z on the rows of each PSD cone, with H = W^T W applied
// in factored form: Delta S = -D_s - R (R^T Delta Z R) R^T (Appendix A, W(X) = R^T X R).
// Near convergence the assembled svec block of H has entries up to ~1/mu, and its
// product with Delta z loses the small eigen-directions of S to cancellation; each
// factor R carries only the square root of that range.  R (R^T dZ R) R^T is
// symmetrised by averaging the (i, j) and (j, i) entries.  Overwrites the PSD rows
// of out (written before by the K product of the assembled blocks).
__global__ void k_psd_ds_from_dz(ConeDev cd, const double* __restrict__ dz, const double* __restrict__ dsrhs,
                                 double* __restrict__ out, const int* skip) {
  if (skip && *skip) return;
  __shared__ double B[32 * LDP], T[32 * LDP];
  const int64_t cone = blockIdx.x;
  const int k = cd.psd_ck[cone];
  const int64_t row = cd.psd_crow[cone];
  const double* R = cd.psd_R + cd.psd_cR[cone];
  load_smat(dz + row, k, B);
  // T = R' dZ
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += R[l + i * k] * B[l + j * LDP];
    T[i + j * LDP] = acc;
  }
  __syncthreads();
  // B = T R = R' dZ R
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += T[i + l * LDP] * R[l + j * k];
    B[i + j * LDP] = acc;
  }
  __syncthreads();
  // T = R B
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    double acc = 0;
    for (int l = 0; l < k; ++l) acc += R[i + l * k] * B[l + j * LDP];
    T[i + j * LDP] = acc;
  }
  __syncthreads();
  // (T R')_{ij} and (T R')_{ji}, averaged; out = -d_s - svec
  for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
    const int i = q % k, j = q / k;
    if (i > j) continue;
    double acc = 0, acc2 = 0;
    for (int l = 0; l < k; ++l) {
      acc += T[i + l * LDP] * R[j + l * k];
      acc2 += T[j + l * LDP] * R[i + l * k];
    }
    const double val = 0.5 * (acc + acc2);
    const int64_t r = row + smat_index(i, j);
    out[r] = -dsrhs[r] - ((i == j) ? val : val * kSqrt2);
  }
}

int cones_psd_ds_from_dz(cudaStream_t st, const ConeDev& cd, const double* dz, const double* dsrhs, double* ds_out,
                         const int* skip) {
  if (cd.n_psd == 0) return CLR_OK;
  const int threads = std::max(64, 32 * ((cd.psd_kmax + 1) / 2));
  k_psd_ds_from_dz<<<(unsigned)cd.n_psd, threads, 0, st>>>(cd, dz, dsrhs, ds_out, skip);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

int cones_combined_ds(cudaStream_t st, const ConeDev& cd, const double* s, const double* z, const double* dsa,
                      const double* dza, IterScal* sc, double* ds_out, const int* skip) {
  if (cd.m_zero + cd.m_nonneg > 0)
    k_ds_nonneg<<<grid_for(cd.m_zero + cd.m_nonneg, 256), 256, 0, st>>>(cd, dsa, dza, sc, ds_out, skip);
  if (cd.n_soc > 0) {
    if (cd.soc_nsmall > 0) k_ds_soc_t<<<soc_t_grid(cd.n_soc), 256, 0, st>>>(cd, dsa, dza, sc, ds_out, skip);
    if (cd.soc_nsmall < cd.n_soc)
      k_ds_soc<32><<<soc_grid(cd, 32), 256, 0, st>>>(cd, dsa, dza, sc, ds_out, cd.scratch, skip);
  }
  if (cd.n_exp + cd.n_pow > 0)
    k_ds_exppow<<<ep_launch(cd.n_exp + cd.n_pow).blocks, ep_launch(cd.n_exp + cd.n_pow).threads, 0, st>>>(
        cd, s, z, dsa, dza, sc, ds_out,
                                                                               skip);
  if (cd.n_psd > 0) {
    const int threads = std::max(64, 32 * ((cd.psd_kmax + 1) / 2));
    k_ds_psd<<<(unsigned)cd.n_psd, threads, 0, st>>>(cd, dsa, dza, sc, ds_out, skip);
  }
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

// ====================================================================== initial point
__global__ void k_nn_min_reset(IterScal* sc, int64_t nprob, const int* skip) {
  if (skip && *skip) return;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nprob; p += (int64_t)gridDim.x * blockDim.x)
    sc[p].nn_min_bits = ~0ull;
}

// least nonneg entry of each problem, as order-preserving bits of a double of any sign
__global__ void k_nn_min(ConeDev cd, const double* __restrict__ v, IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  RunExt<false> mn;
  for (int64_t i = cd.m_zero + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cd.m_zero + cd.m_nonneg;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long b = dbits(v[i]);
    b = (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
    mn.add(sc, &IterScal::nn_min_bits, cd.row_pid[i], b);
  }
  mn.flush(sc, &IterScal::nn_min_bits);
}

__global__ void k_shift_nonneg(ConeDev cd, double* __restrict__ v, const IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cd.m_zero + cd.m_nonneg;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < cd.m_zero) {
      v[i] = 0.0;
      continue;
    }
    unsigned long long b = sc[cd.row_pid[i]].nn_min_bits;
    b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
    const double a = __longlong_as_double((long long)b);
    if (a < 1.4901161193847656e-08) v[i] += 1.0 - a;  // sqrt(eps_64)
  }
}

__global__ void k_shift_soc(ConeDev cd, double* __restrict__ v, const int* skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int64_t cone = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (cone >= cd.n_soc) return;
  const int64_t off = cd.soc_off[cone];
  const int d = cd.soc_dim[cone];
  double x1 = 0;
  for (int j = lane; j < d; j += 32)
    if (j > 0) x1 += v[off + j] * v[off + j];
  x1 = warp_sum(x1);
  const double a = v[off] - sqrt(x1);
  if (lane == 0 && a < 1.4901161193847656e-08) v[off] += 1.0 - a;
}

__global__ void k_shift_psd(ConeDev cd, double* __restrict__ v, const int* skip) {
  if (skip && *skip) return;
  __shared__ double X[32 * LDP], csb[64];
  __shared__ int flag;
  const int k = cd.psd_ck[blockIdx.x];
  const int64_t row = cd.psd_crow[blockIdx.x];
  load_smat(v + row, k, X);
  const double a = jacobi_eigmin(X, k, csb, &flag);
  __syncthreads();
  if (a < 1.4901161193847656e-08)
    for (int j = threadIdx.x; j < k; j += blockDim.x) v[row + smat_index(j, j)] += 1.0 - a;
}

int cones_shift_init(cudaStream_t st, const ConeDev& cd, double* v, IterScal* sc, const int* skip) {
  if (cd.m_zero + cd.m_nonneg > 0) {
    k_nn_min_reset<<<grid_for(cd.nprob, 128), 128, 0, st>>>(sc, cd.nprob, skip);
    if (cd.m_nonneg > 0) k_nn_min<<<grid_for(cd.m_nonneg, 256), 256, 0, st>>>(cd, v, sc, skip);
    k_shift_nonneg<<<grid_for(cd.m_zero + cd.m_nonneg, 256), 256, 0, st>>>(cd, v, sc, skip);
  }
  if (cd.n_soc > 0) k_shift_soc<<<(unsigned)((cd.n_soc * 32 + 255) / 256), 256, 0, st>>>(cd, v, skip);
  if (cd.n_psd > 0) {
    const int threads = std::max(64, 32 * ((cd.psd_kmax + 1) / 2));
    k_shift_psd<<<(unsigned)cd.n_psd, threads, 0, st>>>(cd, v, skip);
  }
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

__global__ void k_unit_init(ConeDev cd, double* __restrict__ v, const int* skip) {
  if (skip && *skip) return;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < cd.m; r += (int64_t)gridDim.x * blockDim.x) {
    if (cd.pc[cd.row_pid[r]].sym) continue;  // symmetric problems keep their symmetric initial point
    double val = 0.0;
    if (r < cd.m_zero || (cd.n_aux > 0 && r >= cd.aux_begin)) val = 0.0;  // zero cone, auxiliary rows
    else if (r < cd.m_zero + cd.m_nonneg) val = 1.0;
    else if (cd.n_soc > 0 && r < cd.soc_off[cd.n_soc - 1] + cd.soc_dim[cd.n_soc - 1]) {
      int64_t lo = 0, hi = cd.n_soc - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (cd.soc_off[mid] <= r) lo = mid;
        else hi = mid - 1;
      }
      val = (r == cd.soc_off[lo]) ? 1.0 : 0.0;
    } else if (r >= cd.exp_row0 && r < cd.exp_row0 + 3 * cd.n_exp) {
      val = cd.exp_center[(r - cd.exp_row0) % 3];
    } else if (r >= cd.pow_row0 && r < cd.pow_row0 + 3 * cd.n_pow) {
      const int64_t i = (r - cd.pow_row0) / 3, c = (r - cd.pow_row0) % 3;
      const double a = cd.pow_alpha[i];
      val = (c == 0) ? sqrt(1.0 + a) : (c == 1 ? sqrt(2.0 - a) : 0.0);
    } else if (cd.n_psd > 0 && r >= cd.psd_row0) {
      const int64_t c = r - cd.psd_crow[psd_cone_of(cd, r)];
      int j = (int)((sqrt(8.0 * c + 1.0) - 1.0) / 2.0);
      while ((int64_t)j * (j + 1) / 2 > c) --j;
      while ((int64_t)(j + 1) * (j + 2) / 2 <= c) ++j;
      const int i = (int)(c - (int64_t)j * (j + 1) / 2);
      val = (i == j) ? 1.0 : 0.0;
    }
    v[r] = val;
  }
}

int cones_unit_init(cudaStream_t st, const ConeDev& cd, double* v, const int* skip) {
  k_unit_init<<<grid_for(cd.m, 256), 256, 0, st>>>(cd, v, skip);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

// Newton on u + grad f(u) = 0 for the exp cone (host, FP64, at setup).
double exp_central_point_host(double out[3]) {
  double u[3] = {-1.0, 0.5, 1.2};
  for (int it = 0; it < 100; ++it) {
    const double r = u[0], s = u[1], t = u[2];
    const double psi = s - r - r * std::log(t / (-r));
    const double g[3] = {std::log(-r / t), 1.0, -r / t};
    const double h[3][3] = {{1.0 / r, 0.0, -1.0 / t}, {0.0, 0.0, 0.0}, {-1.0 / t, 0.0, r / (t * t)}};
    const double sep1[3] = {-1.0 / r, 0.0, -1.0 / t}, sep2[3] = {1.0 / (r * r), 0.0, 1.0 / (t * t)};
    double F[3], J[3][3];
    for (int i = 0; i < 3; ++i) {
      F[i] = u[i] + (-g[i] / psi + sep1[i]);
      for (int j = 0; j < 3; ++j)
        J[i][j] = (i == j ? 1.0 : 0.0) + g[i] * g[j] / (psi * psi) - h[i][j] / psi + (i == j ? sep2[i] : 0.0);
    }
    // solve J du = -F (Gaussian elimination with partial pivoting)
    double A[3][4];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) A[i][j] = J[i][j];
      A[i][3] = -F[i];
    }
    for (int c = 0; c < 3; ++c) {
      int p = c;
      for (int r2 = c + 1; r2 < 3; ++r2)
        if (std::fabs(A[r2][c]) > std::fabs(A[p][c])) p = r2;
      for (int j = 0; j < 4; ++j) std::swap(A[c][j], A[p][j]);
      for (int r2 = c + 1; r2 < 3; ++r2) {
        const double f = A[r2][c] / A[c][c];
        for (int j = c; j < 4; ++j) A[r2][j] -= f * A[c][j];
      }
    }
    double du[3];
    for (int i = 2; i >= 0; --i) {
      double acc = A[i][3];
      for (int j = i + 1; j < 3; ++j) acc -= A[i][j] * du[j];
      du[i] = acc / A[i][i];
    }
    double mx = 0;
    for (int i = 0; i < 3; ++i) {
      u[i] += du[i];
      mx = std::fmax(mx, std::fabs(du[i]));
    }
    if (mx < 1e-15) break;
  }
  for (int i = 0; i < 3; ++i) out[i] = u[i];
  return u[0];
}

}  // namespace clr
