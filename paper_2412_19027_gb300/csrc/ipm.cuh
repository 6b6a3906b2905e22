// The per-iteration device step of Algorithm 1 and the solver object behind
// the C ABI.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "cones.cuh"
#include "device.cuh"
#include "internal.h"
#include "ldl.cuh"
#include "symbolic.h"

// Scalars shared by the kernels of one iteration (device memory).
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
  clr::NonsymStep ns;
  double alpha_sym, alpha_a, alpha_c, sigma, sigma_mu;
  double mu_coef[3];
  // iterative refinement
  int ir_skip, ir_steps, ir_total, ir_cur;
  double rhs_norm, ir_prev;
  unsigned long long rnorm_bits;
  int dyn_hits, pad1;
};

namespace clr {

struct VecDev {
  double *xz, *s;            // iterate: [x; z] (N), s (m)
  double *lo, *hi;           // split K products (N each)
  double *G;                 // [G1; G2] (N)
  double *qp;                // q + 2 P x / tau (n)
  double *rhs, *sol2, *sol1; // N each
  double *dir_a, *dsa;       // affine direction [dx; dz] (N), ds (m)
  double *dir, *ds;          // current / combined direction
  double *dsrhs;             // d_s of the current right-hand side (m)
  double *r, *solb;          // refinement residual and accumulated solution (N)
  double *part;              // reduction partials
  double *hist;              // history rows
  double *q, *b, *D, *E;     // scaled data and scalings
  double *kval;              // KKT values (x part constant, z part = -H)
  int64_t *kptr;             // full-K CSR (both triangles), values through kvi
  int32_t *kcol, *kvi;
};

class Solver {
 public:
  clr_settings st{};
  HostProblem hp;
  Symbolic sy;
  NumericMaps mp;
  bool device_ready = false;
  bool solved_once = false;
  double setup_s = 0, solve_s = 0;
  int last_status = 0, last_iters = 0;
  clr_info info{};
  clr_perf perf{};
  std::vector<double> history;  // rows of 12
  std::string err;

  ~Solver();
  int analyze(const clr_csc* P, const double* q, const clr_csc* A, const double* b, const clr_cone* cones,
              int32_t ncones, const clr_settings& s);
  int upload();
  int solve();
  int get_solution(double* x, double* s, double* z, clr_info* out);
  int update_qb(const double* q, const double* b);
  int set_stream(void* stream);

 private:
  DeviceArena ar_;
  cudaStream_t stream_ = nullptr;
  bool own_stream_ = false;
  LdlStructure ls_;
  LdlFactor<double> f64_;
  LdlFactor<float> f32_;
  ConeDev cd_;
  VecDev v_{};
  IterScal* sc_ = nullptr;       // device
  IterScal* sc_host_ = nullptr;  // pinned
  int csr_group_ = 32;
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t gexec_ = nullptr;
  cudaGraph_t igraph_ = nullptr;
  cudaGraphExec_t igexec_ = nullptr;
  int64_t iter_kernels_ = 0, init_kernels_ = 0, body_kernels_ = 0;
  cudaStream_t body_stream_ = nullptr;
  std::vector<cudaGraph_t> ir_nodes_;  // refinement loop bodies captured in the current graph
  cudaEvent_t ev_[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void mark(int i);
  void drop_graphs();
  int launch_init();

  int factor();
  int kkt_solve(const double* rhs, double* sol);
  int iteration();
  int initialise();
  int direction(bool affine);
  int step_length(bool combined);
  int launch_iteration();
};

}  // namespace clr
