// extern "C" entry points declared in include/clr.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>

#include "ipm.cuh"

struct clr_solver {
  clr::Solver impl;
};

namespace clr {
const char* last_cuda_error();
void set_allocator(clr_alloc_fn a, clr_free_fn f, void* ctx);
}  // namespace clr

using clr::Solver;

extern "C" {

int clr_default_settings(clr_settings* out, int32_t factor_bits) {
  if (!out || (factor_bits != 64 && factor_bits != 32 && factor_bits != 16)) return CLR_E_INVALID;
  const bool low = factor_bits != 64;
  const double eps64 = 2.220446049250313e-16;
  const double eps32 = 1.1920928955078125e-07;
  clr_settings s{};
  s.eps_feas = 1e-8;
  s.eps_inf = 1e-8;
  s.max_iter = 200;
  s.factor_bits = factor_bits;
  s.static_reg = low ? std::sqrt(eps32) : 1e-8;
  s.static_reg_dyn = eps64 * eps64;
  s.dyn_reg_eps = low ? 1e-6 : 1e-13;
  s.dyn_reg_delta = low ? 1e-4 : 2e-7;
  s.ir_max_steps = 10;
  s.ir_abstol = 1e-12;
  s.ir_reltol = 1e-12;
  s.ir_stop_ratio = 0.0;
  s.equilibrate = 1;
  s.ruiz_passes = 10;
  s.scale_min = 1e-4;
  s.scale_max = 1e4;
  s.step_fraction = 0.99;
  s.backtrack = 0.8;
  s.nbhd_beta = 1e-6;
  s.min_step = 1e-10;
  s.use_graph = 1;
  s.verbose = 0;
  s.fp64_escalation = 1;
  s.big_front_schedule = 1;
  s.small_front_max = 0;
  s.amalgamation = 1;
  s.escalate_ratio = 0.1;
  s.soc_expand_dim = 33;
  s.pull_lists_direct = 1;
  *out = s;
  return CLR_OK;
}

static int check_settings(const clr_settings& s) {
  if (s.factor_bits != 64 && s.factor_bits != 32 && s.factor_bits != 16) return CLR_E_INVALID;
  if (!(s.eps_feas > 0) || !(s.eps_inf > 0) || s.max_iter < 0 || s.ir_max_steps < 0 || s.ruiz_passes < 0 ||
      !(s.ir_stop_ratio >= 0) || s.big_front_schedule < 0 || s.big_front_schedule > 3)
    return CLR_E_INVALID;
  if (s.small_front_max < 0 || s.small_front_max > (s.factor_bits == 64 ? 160 : 224) || s.amalgamation < 0 ||
      s.amalgamation > 2)
    return CLR_E_INVALID;
  if (!(s.scale_min > 0) || !(s.scale_max >= s.scale_min)) return CLR_E_INVALID;
  if (!(s.escalate_ratio >= 0) || s.soc_expand_dim < 0) return CLR_E_INVALID;
  if (s.pull_lists_direct != 0 && s.pull_lists_direct != 1) return CLR_E_INVALID;
  if (!(s.step_fraction > 0 && s.step_fraction <= 1) || !(s.backtrack > 0 && s.backtrack < 1)) return CLR_E_INVALID;
  return CLR_OK;
}

static int make(clr_solver** out, const clr_csc* P, const double* q, const clr_csc* A, const double* b,
                const clr_cone* cones, int32_t ncones, const clr_settings* st, bool device) {
  if (!out) return CLR_E_INVALID;
  *out = nullptr;
  clr_settings s;
  if (st) s = *st;
  else clr_default_settings(&s, 64);
  int rc = check_settings(s);
  if (rc) return rc;
  clr_solver* h = new (std::nothrow) clr_solver;
  if (!h) return CLR_E_OOM;
  try {
    rc = h->impl.analyze(P, q, A, b, cones, ncones, s);
    if (rc == CLR_OK && device) rc = h->impl.upload();
  } catch (const std::bad_alloc&) {
    rc = CLR_E_OOM;
  }
  if (rc != CLR_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return CLR_OK;
}

int clr_setup(clr_solver** out, const clr_csc* P_upper, const double* q, const clr_csc* A, const double* b,
              const clr_cone* cones, int32_t ncones, const clr_settings* st) {
  return make(out, P_upper, q, A, b, cones, ncones, st, true);
}

int clr_analyze(clr_solver** out, const clr_csc* P_upper, const double* q, const clr_csc* A, const double* b,
                const clr_cone* cones, int32_t ncones, const clr_settings* st) {
  return make(out, P_upper, q, A, b, cones, ncones, st, false);
}

int clr_solve(clr_solver* s) {
  if (!s) return CLR_E_INVALID;
  return s->impl.solve();
}

int clr_solve_begin(clr_solver* s) {
  if (!s) return CLR_E_INVALID;
  return s->impl.solve_begin();
}

int clr_solve_iterate(clr_solver* s, int32_t k, int32_t* done, int32_t* iters_run) {
  if (!s || k < 0) return CLR_E_INVALID;
  clr::Solver& v = s->impl;
  if (!v.device_ready) return CLR_E_STATE;
  int64_t before = 0;
  for (int64_t p = 0; p < v.lay.B; ++p) before = std::max<int64_t>(before, v.problem_iter(p));
  int32_t finished = 0;
  for (int32_t i = 0; i < k; ++i) {
    int rc = v.step_launch();
    if (rc) return rc;
    bool ready = false;
    rc = v.step_wait(&ready);
    if (rc) return rc;
    if (v.all_halted()) {
      finished = 1;
      break;
    }
  }
  int64_t after = 0;
  for (int64_t p = 0; p < v.lay.B; ++p) after = std::max<int64_t>(after, v.problem_iter(p));
  if (done) *done = finished;
  if (iters_run) *iters_run = (int32_t)(after - before);
  return CLR_OK;
}

int clr_solve_end(clr_solver* s) {
  if (!s) return CLR_E_INVALID;
  return s->impl.solve_end();
}

int clr_get_solution(const clr_solver* s, double* x, double* sl, double* z, clr_info* info) {
  if (!s) return CLR_E_INVALID;
  return const_cast<clr_solver*>(s)->impl.get_solution(0, x, sl, z, info);
}

int clr_update_qb(clr_solver* s, const double* q, const double* b) {
  if (!s) return CLR_E_INVALID;
  return s->impl.update_qb(0, q, b);
}

int clr_update_PA(clr_solver* s, const double* Px, const double* Ax) {
  if (!s) return CLR_E_INVALID;
  return s->impl.update_PA(0, Px, Ax);
}

// ---- cohorts ----
static int make_batch(clr_solver** out, int32_t nprob, const clr_problem* probs, const clr_settings* st,
                      bool device) {
  if (!out || nprob < 1 || !probs) return CLR_E_INVALID;
  *out = nullptr;
  clr_settings s;
  if (st) s = *st;
  else clr_default_settings(&s, 64);
  int rc = check_settings(s);
  if (rc) return rc;
  clr_solver* h = new (std::nothrow) clr_solver;
  if (!h) return CLR_E_OOM;
  try {
    // host setup of every problem (validation, equilibration, KKT layout, AMD) on worker threads
    std::vector<clr::HostProblem> hps(nprob);
    std::vector<std::vector<int64_t>> orders(nprob);
    std::vector<int> rcs(nprob, CLR_OK);
    std::vector<std::string> errs(nprob);
    std::atomic<int32_t> next{0};
    auto work = [&]() {
      for (int32_t i = next++; i < nprob; i = next++) {
        const clr_problem& pr = probs[i];
        rcs[i] = clr::build_problem(hps[i], pr.P_upper, pr.q, pr.A, pr.b, pr.cones, pr.ncones, s, errs[i]);
        if (rcs[i] == CLR_OK) {
          int64_t nd = 0;
          int which = 0;
          clr::choose_kkt_order(hps[i], orders[i], nd, &which);
        }
      }
    };
    const int nt = (int)std::max<unsigned>(1, std::min<unsigned>(std::thread::hardware_concurrency(), 16));
    std::vector<std::thread> pool;
    for (int t = 1; t < std::min<int>(nt, nprob); ++t) pool.emplace_back(work);
    work();
    for (std::thread& t : pool) t.join();
    for (int32_t i = 0; i < nprob && rc == CLR_OK; ++i) rc = rcs[i];
    if (rc == CLR_OK) rc = h->impl.analyze_cohort(std::move(hps), orders, s);
    if (rc == CLR_OK && device) rc = h->impl.upload();
  } catch (const std::bad_alloc&) {
    rc = CLR_E_OOM;
  }
  if (rc != CLR_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return CLR_OK;
}

int clr_batch_setup(clr_solver** out, int32_t nprob, const clr_problem* probs, const clr_settings* st) {
  return make_batch(out, nprob, probs, st, true);
}

int clr_batch_analyze(clr_solver** out, int32_t nprob, const clr_problem* probs, const clr_settings* st) {
  return make_batch(out, nprob, probs, st, false);
}

// ---- autotuner ----
static std::string tune_key(int32_t nprob, const clr_problem* probs, const clr_settings& st) {
  int64_t n = 0, m = 0, nnzp = 0, nnza = 0, cnt[6] = {0, 0, 0, 0, 0, 0};
  for (int32_t i = 0; i < nprob; ++i) {
    const clr_problem& p = probs[i];
    if (p.A) {
      n += p.A->ncols;
      m += p.A->nrows;
      nnza += p.A->nnz;
    }
    if (p.P_upper) nnzp += p.P_upper->nnz;
    for (int32_t c = 0; c < p.ncones && p.cones; ++c)
      if (p.cones[c].type >= 0 && p.cones[c].type < 6) cnt[p.cones[c].type] += p.cones[c].type <= 1 ? p.cones[c].dim : 1;
  }
  char buf[256];
  std::snprintf(buf, sizeof(buf), "bits=%d;B=%d;n=%lld;m=%lld;nnzP=%lld;nnzA=%lld;cones=%lld,%lld,%lld,%lld,%lld,%lld",
                st.factor_bits, nprob, (long long)n, (long long)m, (long long)nnzp, (long long)nnza, (long long)cnt[0],
                (long long)cnt[1], (long long)cnt[2], (long long)cnt[3], (long long)cnt[4], (long long)cnt[5]);
  return buf;
}

// device ms per IPM iteration of a cohort with settings s (iters iterations)
static int tune_time(int32_t nprob, const clr_problem* probs, const clr_settings& s, double* ms) {
  clr_solver* h = nullptr;
  int rc = make_batch(&h, nprob, probs, &s, true);
  if (rc) return rc;
  rc = h->impl.solve();
  if (rc == CLR_OK) {
    const clr_perf& p = h->impl.perf;
    const double tot = p.resid_cones_ms + p.factor_ms + p.solve_step_ms;
    *ms = tot / std::max(1, p.iterations);
  }
  clr_free(h);
  return rc;
}

int clr_autotune(int32_t nprob, const clr_problem* probs, const clr_settings* base, int32_t iters,
                 const char* cache_path, clr_tune_result* out) {
  if (!out || !base || iters < 1 || nprob < 1 || !probs) return CLR_E_INVALID;
  int rc = check_settings(*base);
  if (rc) return rc;
  *out = clr_tune_result{};
  const std::string key = tune_key(nprob, probs, *base);
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[512];
      while (std::fgets(line, sizeof(line), f)) {
        char k[300];
        int sm = 0, am = 0, sc = 0;
        double ms = 0;
        if (std::sscanf(line, "%299s %d %d %d %lf", k, &sm, &am, &sc, &ms) == 5 && key == k) {
          out->small_front_max = sm;
          out->amalgamation = am;
          out->big_front_schedule = sc;
          out->ms_per_iter = ms;
          out->base_ms_per_iter = -1;
          out->from_cache = 1;
        }
      }
      std::fclose(f);
      if (out->from_cache) return CLR_OK;
    }
  }
  clr_settings s = *base;
  s.max_iter = iters;
  s.verbose = 0;
  double ms = 0;
  rc = tune_time(nprob, probs, s, &ms);  // warm-up (module load, allocator pools)
  if (rc) return rc;
  rc = tune_time(nprob, probs, s, &ms);
  if (rc) return rc;
  out->base_ms_per_iter = ms;
  out->small_front_max = s.small_front_max;
  out->amalgamation = s.amalgamation;
  out->big_front_schedule = s.big_front_schedule;
  out->ms_per_iter = ms;
  const int fronts64[] = {64, 96, 128, 160};
  const int fronts32[] = {64, 96, 128, 160, 192};
  const bool f64 = base->factor_bits == 64;
  const int* fr = f64 ? fronts64 : fronts32;
  const int nfr = f64 ? 4 : 5;
  for (int a = 0; a <= 2; ++a)
    for (int i = 0; i < nfr; ++i)
      for (int sc = 0; sc <= (f64 ? 1 : 2); ++sc) {  // 2 = 1 for the FP64 factor
        s.small_front_max = fr[i];
        s.amalgamation = a;
        s.big_front_schedule = sc;
        rc = tune_time(nprob, probs, s, &ms);
        if (rc) return rc;
        out->candidates += 1;
        if (ms < out->ms_per_iter) {
          out->ms_per_iter = ms;
          out->small_front_max = fr[i];
          out->amalgamation = a;
          out->big_front_schedule = sc;
        }
      }
  if (cache_path)
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), out->small_front_max, out->amalgamation,
                   out->big_front_schedule, out->ms_per_iter);
      std::fclose(f);
    }
  return CLR_OK;
}

int32_t clr_batch_size(const clr_solver* s) { return s ? (int32_t)s->impl.nprob() : 0; }

int clr_batch_get(const clr_solver* s, int32_t i, double* x, double* sl, double* z, clr_info* info) {
  if (!s) return CLR_E_INVALID;
  return const_cast<clr_solver*>(s)->impl.get_solution(i, x, sl, z, info);
}

int clr_batch_update_qb(clr_solver* s, int32_t i, const double* q, const double* b) {
  if (!s) return CLR_E_INVALID;
  return s->impl.update_qb(i, q, b);
}

int clr_batch_update_PA(clr_solver* s, int32_t i, const double* Px, const double* Ax) {
  if (!s) return CLR_E_INVALID;
  return s->impl.update_PA(i, Px, Ax);
}

int clr_get_symbolic_stats(const clr_solver* s, clr_symbolic_stats* out) {
  if (!s || !out) return CLR_E_INVALID;
  const Solver& v = s->impl;
  clr_symbolic_stats r{};
  r.n = v.hp.n;
  r.m = v.hp.m;
  r.kkt_dim = v.hp.n + v.hp.m;
  r.kkt_nnz_lower = (int64_t)v.hp.krow.size();
  r.l_nnz = v.sy.l_nnz;
  r.factor_flops = v.sy.flops;
  r.n_supernodes = v.sy.nsn;
  r.n_levels = v.sy.nlev;
  r.max_front = v.sy.max_front;
  r.front_pool_entries = v.sy.pool;
  r.n_dense_rows = v.sy.n_dense;
  r.ordering = v.sy.ordering;
  r.l_nnz_exact = v.sy.l_nnz_exact;
  r.l_nnz_counted = v.sy.pred_nnz;
  r.factor_flops_stored = v.sy.flops_stored;
  r.maps_digest = maps_digest(v.sy, v.mp);
  *out = r;
  return CLR_OK;
}

int clr_get_perf(const clr_solver* s, clr_perf* out) {
  if (!s || !out) return CLR_E_INVALID;
  if (!s->impl.solved_once) return CLR_E_STATE;
  *out = s->impl.perf;
  return CLR_OK;
}

int clr_get_symbolic(const clr_solver* s, int64_t* perm, int64_t* sn_ptr, int64_t* sn_parent, int64_t* row_ptr,
                     int64_t* rows, int64_t* rows_len, int64_t* row_perm) {
  if (!s) return CLR_E_INVALID;
  const Solver& v = s->impl;
  if (perm) std::copy(v.sy.perm.begin(), v.sy.perm.end(), perm);
  if (sn_ptr) std::copy(v.sy.sn_ptr.begin(), v.sy.sn_ptr.end(), sn_ptr);
  if (sn_parent) std::copy(v.sy.sn_parent.begin(), v.sy.sn_parent.end(), sn_parent);
  if (row_ptr) std::copy(v.sy.row_ptr.begin(), v.sy.row_ptr.end(), row_ptr);
  if (rows) std::copy(v.sy.rows.begin(), v.sy.rows.end(), rows);
  if (rows_len) *rows_len = (int64_t)v.sy.rows.size();
  // the caller's rows (the auxiliary rows of expanded SOCs come last and have none)
  if (row_perm) std::copy(v.hp.row_perm.begin(), v.hp.row_perm.end() - v.hp.cl.n_aux, row_perm);
  return CLR_OK;
}

int clr_get_scaling(const clr_solver* s, double* D, double* E, double* c) {
  if (!s) return CLR_E_INVALID;
  const Solver& v = s->impl;
  if (D) std::copy(v.hp.D.begin(), v.hp.D.end(), D);
  if (E) std::copy(v.hp.E.begin(), v.hp.E.end() - v.hp.cl.n_aux, E);
  if (c) *c = v.hp.c;
  return CLR_OK;
}

int clr_get_history(const clr_solver* s, double* out, int32_t cap, int32_t* rows) {
  if (!s) return CLR_E_INVALID;
  const Solver& v = s->impl;
  if (v.history.empty()) {
    if (rows) *rows = 0;
    return CLR_OK;
  }
  const std::vector<double>& h = v.history[0];
  const int32_t have = (int32_t)(h.size() / 12);
  const int32_t k = std::min(have, std::max(cap, 0));
  if (out) std::copy(h.begin(), h.begin() + 12 * (size_t)k, out);
  if (rows) *rows = k;
  return CLR_OK;
}

int clr_set_stream(clr_solver* s, void* cuda_stream) {
  if (!s) return CLR_E_INVALID;
  return s->impl.set_stream(cuda_stream);
}

int clr_set_allocator(clr_alloc_fn alloc_fn, clr_free_fn free_fn, void* ctx) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return CLR_E_INVALID;
  clr::set_allocator(alloc_fn, free_fn, ctx);
  return CLR_OK;
}

void clr_free(clr_solver* s) { delete s; }

const char* clr_error_string(int code) {
  switch (code) {
    case CLR_OK: return "ok";
    case CLR_E_INVALID: return "invalid input";
    case CLR_E_DIM: return "dimension mismatch";
    case CLR_E_UNSUPPORTED: return "unsupported problem";
    case CLR_E_OOM: return "out of memory";
    case CLR_E_CUDA: return "CUDA error";
    case CLR_E_TIMEOUT: return "device wait timed out";
    case CLR_E_AGAIN: return "not ready";
    case CLR_E_STATE: return "call out of order";
    default: return "unknown error";
  }
}

const char* clr_status_string(int status) {
  switch (status) {
    case CLR_UNSOLVED: return "UNSOLVED";
    case CLR_SOLVED: return "SOLVED";
    case CLR_PRIMAL_INFEASIBLE: return "PRIMAL_INFEASIBLE";
    case CLR_DUAL_INFEASIBLE: return "DUAL_INFEASIBLE";
    case CLR_MAX_ITER: return "MAX_ITER";
    case CLR_INSUFFICIENT_PROGRESS: return "INSUFFICIENT_PROGRESS";
    case CLR_NUMERICAL_ERROR: return "NUMERICAL_ERROR";
    default: return "UNKNOWN";
  }
}

const char* clr_last_cuda_error(void) { return clr::last_cuda_error(); }

}  // extern "C"
