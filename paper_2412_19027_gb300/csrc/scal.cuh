// Per-problem iteration scalars and batch bookkeeping shared by the kernels
// of the per-iteration device step.  A solver holds B >= 1 independent
// problems merged block-diagonally (a "cohort"); every scalar of Algorithm 1
// (tau, kappa, mu, step lengths, sigma, ...) exists once per problem, and a
// problem's result does not depend on the other problems of its cohort.
#pragma once

#include <cstdint>

namespace clr {

// Result of the exp/pow backtracking of one problem (see cones_step_nonsym).
struct NonsymStep {
  int jint;                 // smallest j with every cone interior at a0 * backtrack^j
  int fail;                 // some cone fails N(beta) at jint
  unsigned long long mask;  // bit k: every cone passes N(beta) at jint + 1 + k
};

// Scalars of one problem shared by the kernels of one iteration (device memory).
struct IterScal {
  double tau, kappa;
  // residual stage (scaled quantities unless noted)
  double mu, pcost, dcost, res_p, res_d, gap_abs, gap_rel;  // pcost..gap unscaled
  double xPx, qx, bz, sz, G3;
  int status, iter, halt, pad0;
  // regularisation
  unsigned long long hmax_bits;
  double delta;
  // constant-RHS part of Delta tau
  double qp_dx2, b_dz2;
  // current direction
  double d_tau, d_kap, dtau, dkap;
  double dtau_a, dkap_a;
  // step length
  unsigned long long amin_bits;
  NonsymStep ns;
  double alpha_sym, alpha_a, alpha_c, sigma, sigma_mu;
  double mu_coef[3];
  // iterative refinement
  int ir_skip, ir_steps, ir_total, ir_cur;
  double rhs_norm, ir_prev;
  unsigned long long rnorm_bits;
  int dyn_hits, ir_revert;  // ir_revert: the last refinement step is being undone
  // initial point: order-preserving bits of the least nonneg entry
  unsigned long long nn_min_bits;
  // precision escalation: a refinement of this iteration stopped short (ir_fail);
  // the iteration is not taken (escalate) and is redone with the FP64 factor
  int ir_fail, escalate;
  // feasibility stall (low-precision factor): the best termination ratio of the
  // residuals so far, mu when it was reached, and the iterations since then in
  // which mu stood ten times lower; three of them also escalate
  double feas_best, mu_at_best;
  int feas_stall, pad1;
  // FP64 factor breakdown: a KKT solve of the iteration gave a non-finite value
  // (the unpivoted factor overflowed); the iteration is redone (escalate) with the
  // static regularisation multiplied by reg_boost (x100 per breakdown, at most 1e4)
  double reg_boost;
  // largest scaled residual |G| of the iterate, and the largest final refinement
  // residual of this iteration's KKT solves that ended above the tolerance
  double g_scaled, ir_worst;
  // max of the two feasibility termination ratios r/(eps (1 + norms)) of the iterate
  double feas_ratio;
};

// Constants of one problem (device memory, written at setup).
struct ProbConst {
  double c, bnorm, qnorm, maxPdiag;  // cost scaling, unscaled ||b||_inf, ||q||_inf, max |P^_ii|
  int64_t nu;                        // barrier degree
  int32_t sym;                       // 1: symmetric cones only (symmetric initial point)
  int32_t pad;
};

// Cohort-wide flags.
struct BatchFlags {
  int all_halt;   // every problem has stopped: the remaining kernels return at once
  int n_running;  // problems still iterating
  int ir_none;    // no problem wants another refinement step
  int pad;
};

// A contiguous run of at most kChunk entries of one problem's x or z segment.
// Reductions sum each chunk in one block and then the chunks of a problem in
// list order, so a problem's sums do not depend on the rest of the cohort.
struct Chunk {
  int64_t begin;
  int32_t len, pid;
};
constexpr int kChunk = 2048;

#ifdef __CUDACC__
// Per-problem extremum of a flat row kernel.  Each thread keeps a running value
// for the problem of its current row and flushes it with an atomic when the
// problem changes (batches only); at the end all 32 lanes call warp_flush, which
// reduces across the warp first when every lane with data has the same problem.
// `b` holds order-preserving bits; lanes without data pass pid < 0.
template <bool IsMax>
__device__ __forceinline__ void atomic_ext(unsigned long long* a, unsigned long long b) {
  if (IsMax) atomicMax(a, b);
  else atomicMin(a, b);
}
template <bool IsMax>
__device__ void warp_flush(IterScal* sc, unsigned long long IterScal::*f, int pid, unsigned long long b) {
  const unsigned full = 0xffffffffu;
  int lo = pid >= 0 ? pid : 0x7fffffff, hi = pid;
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(full, lo, o));
    hi = max(hi, __shfl_xor_sync(full, hi, o));
  }
  if (hi < 0) return;
  if (lo == hi) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(full, b, o);
      b = IsMax ? (t > b ? t : b) : (t < b ? t : b);
    }
    if ((threadIdx.x & 31) == 0) atomic_ext<IsMax>(&(sc[hi].*f), b);
  } else if (pid >= 0) {
    atomic_ext<IsMax>(&(sc[pid].*f), b);
  }
}
template <bool IsMax>
struct RunExt {
  int pid = -1;
  unsigned long long b = IsMax ? 0ull : ~0ull;
  __device__ void add(IterScal* sc, unsigned long long IterScal::*f, int p, unsigned long long v) {
    if (p != pid) {
      if (pid >= 0) atomic_ext<IsMax>(&(sc[pid].*f), b);
      pid = p;
      b = IsMax ? 0ull : ~0ull;
    }
    b = IsMax ? (v > b ? v : b) : (v < b ? v : b);
  }
  __device__ void flush(IterScal* sc, unsigned long long IterScal::*f) { warp_flush<IsMax>(sc, f, pid, b); }
};
#endif

}  // namespace clr
