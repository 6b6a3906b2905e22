// The per-iteration device step of Algorithm 1 and the solver object behind
// the C ABI.  One Solver holds a cohort of B >= 1 independent problems merged
// block-diagonally: one captured CUDA graph per iteration advances all of
// them, and every scalar of the method is kept per problem.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "cones.cuh"
#include "device.cuh"
#include "internal.h"
#include "ldl.cuh"
#include "scal.cuh"
#include "symbolic.h"

namespace clr {

struct VecDev {
  const int64_t* long_rows = nullptr;  // KKT rows with more than kLongRow entries (sorted)
  const double* kfv = nullptr;         // values of the x rows of the full KKT CSR (constant), CSR order
  int64_t nlong = 0;
  double *xz, *s;            // iterate: [x; z] (N), s (m)
  double *lo, *hi;           // split K products (N each)
  double *G;                 // [G1; G2] (N)
  double *qp;                // q + 2 P x / tau (n)
  double *rhs, *sol2, *sol1; // N each
  double *dir_a, *dsa;       // affine direction [dx; dz] (N), ds (m)
  double *dir, *ds;          // current / combined direction
  double *dsrhs;             // d_s of the current right-hand side (m)
  double *r, *solb;          // refinement residual and accumulated solution (N)
  double *part;              // chunk partial sums (S_NSLOT x pst)
  unsigned long long* maxb;  // residual-stage maxima (8 per problem)
  double *hist;              // history rows (per problem)
  double *q, *b, *D, *E;     // scaled data and scalings
  double *kval;              // KKT values (x part constant, z part = -H)
  int64_t *kptr;             // full-K CSR (both triangles), values through kvi
  int32_t *kcol, *kvi;
  int32_t* pid;              // KKT index -> problem
  Chunk* ck;                 // x chunks then z chunks (z begins are row indices)
  int64_t *ckx_ptr, *ckz_ptr;
  ProbConst* pc;
};

class Solver {
 public:
  clr_settings st{};
  std::vector<HostProblem> probs;  // per problem (small arrays kept: row order, scalings, q, b)
  HostProblem hp;                  // the cohort problem
  CohortLayout lay;
  Symbolic sy;
  NumericMaps mp;
  bool device_ready = false;
  bool solved_once = false;
  double setup_s = 0, solve_s = 0;
  clr_perf perf{};
  std::vector<clr_info> infos;          // per problem, after a solve
  std::vector<std::vector<double>> history;  // per problem, rows of 12
  std::string err;

  ~Solver();
  // One problem.
  int analyze(const clr_csc* P, const double* q, const clr_csc* A, const double* b, const clr_cone* cones,
              int32_t ncones, const clr_settings& s);
  // A cohort from problems already through build_problem (moved in) with their orders.
  int analyze_cohort(std::vector<HostProblem>&& ps, const std::vector<std::vector<int64_t>>& orders,
                     const clr_settings& s);
  int upload();
  int solve();
  // Asynchronous driving (serving): begin, then step until step_poll says done.
  int solve_begin();
  int step_launch();           // one iteration + status copy to pinned memory, no wait
  int step_poll(bool* ready);  // has the last launched step finished?
  int step_wait(bool* ready);  // wait for the last launched step, then as step_poll
  int problem_iter(int64_t p) const { return sc_host_[p].iter; }  // valid after a step finished
  bool all_halted() const;     // valid after a step finished
  int problem_status(int64_t p) const;  // from the last finished step
  int solve_end();
  int get_solution(int64_t p, double* x, double* s, double* z, clr_info* out);
  // Problem p as of the last finished step (it must have stopped; used to hand
  // out results while the rest of the cohort goes on).
  int get_solution_now(int64_t p, double* x, double* s, double* z, clr_info* out);
  // Build on caller-owned `stream` with stream-ordered device memory (before upload).
  int use_stream_ordered(cudaStream_t stream);
  int update_qb(int64_t p, const double* q, const double* b);
  int update_PA(int64_t p, const double* Px, const double* Ax);
  int set_stream(void* stream);
  size_t device_bytes() const { return ar_.bytes(); }
  int64_t nprob() const { return lay.B; }

 private:
  DeviceArena ar_;
  cudaStream_t stream_ = nullptr;
  bool own_stream_ = false;
  LdlStructure ls_;
  LdlFactor<double> f64_;
  LdlFactor<float> f32_;
  ConeDev cd_;
  VecDev v_{};
  IterScal* sc_ = nullptr;        // device, B entries
  IterScal* sc_host_ = nullptr;   // pinned, B entries
  BatchFlags* bf_ = nullptr;      // device
  BatchFlags* bf_host_ = nullptr; // pinned
  int64_t nckx_ = 0, nckz_ = 0, pst_ = 1;
  int hist_rows_ = 0;
  int csr_group_ = 32;
  std::vector<int64_t> h_long_;  // KKT rows handled by k_kmv_long
  std::vector<int32_t> h_kfv_src_;  // kval index of each entry of the x rows' full-CSR values (kfv)
  // iteration graphs per factor precision (0: configured, 1: FP64 after an escalation)
  cudaGraph_t graph_[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec_[2] = {nullptr, nullptr};
  cudaGraph_t igraph_ = nullptr;
  cudaGraphExec_t igexec_ = nullptr;
  int64_t iter_kernels_[2] = {0, 0}, init_kernels_ = 0, body_kernels_[2] = {0, 0};
  bool escalated_ = false;       // this solve continues with the FP64 factor
  bool step64_ = false;          // the last launched iteration factored in FP64
  bool f64_ready_ = false;       // f64_ allocated
  std::vector<int> esc_iter_;    // per problem: iteration of the escalation, -1
  bool use64() const { return st.factor_bits == 64 || escalated_; }
  // regularisation constants of the factor in use (FP64 defaults after an escalation)
  double reg_static() const;
  double reg_dyn_eps() const;
  double reg_dyn_delta() const;
  int escalate_to_fp64();
  cudaStream_t body_stream_ = nullptr;
  std::vector<cudaGraph_t> ir_nodes_;  // refinement loop bodies captured in the current graph
  cudaEvent_t ev_[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t step_ev_ = nullptr;
  // asynchronous solve state
  int it_ = 0;
  bool first_step_ = true;
  double t_begin_ = 0;
  void mark(int i);
  void drop_graphs();
  int launch_init();
  int finish_step();
  clr_info info_now(int64_t p) const;
  int unscale_solution(int64_t p, double* x, double* s, double* z, clr_info* out);

  int factor();
  int kkt_solve(const double* rhs, double* sol);
  int iteration();
  int initialise();
  int direction(bool affine);
  int step_length(bool combined);
  int launch_iteration();
};

}  // namespace clr
