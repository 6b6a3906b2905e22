// Serving loop: continuous batching of independent solves.
//
// Requests are deep-copied on submit and analysed on the host by worker
// threads (validation, equilibration, KKT layout, AMD order).  A builder
// thread forms a cohort from every analysed request waiting (up to
// max_cohort) whenever a slot (one of max_active CUDA streams) and the device
// budget allow it, uploads it with stream-ordered memory and captures its
// iteration graph.  The stepper thread interleaves the IPM iterations of all
// active cohorts -- it launches the next iteration of every cohort whose last
// one has finished, so the cohorts' work overlaps on the device -- and hands
// each problem's result out as soon as that problem stops, while the rest of
// its cohort goes on.  A cohort's memory and slot are released when its last
// problem stops; requests that arrived meanwhile are admitted into the freed
// slot.  No step of a solve runs on the host.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "ipm.cuh"

namespace clr {
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  // deep copy of the inputs
  int64_t n = 0, m = 0, p_nrows = 0, p_ncols = 0;
  std::vector<int64_t> pcol, acol;
  std::vector<int32_t> prow, arow;
  std::vector<double> pval, aval, q, b;
  std::vector<clr_cone> cones;
  // analysis
  HostProblem hp;
  std::vector<int64_t> order;
  // result
  int rc = CLR_OK;
  bool done = false;
  std::vector<double> x, s, z;
  clr_info info{};
  double t_submit = 0, t_analysed = 0, t_done = 0;
};

struct Cohort {
  std::unique_ptr<Solver> solver;
  std::vector<std::shared_ptr<Request>> reqs;
  std::vector<char> delivered;
  int slot = -1;
  size_t bytes = 0;
  bool stepping = false;
};

}  // namespace

class Server {
 public:
  Server(size_t budget, int max_cohort, int max_active, const clr_settings& st)
      : budget_(budget), max_cohort_(max_cohort), max_active_(max_active), st_(st) {}
  ~Server() { stop(); }

  int start() {
    streams_.resize(max_active_, nullptr);
    slot_free_.assign(max_active_, 1);
    for (cudaStream_t& s : streams_) CLR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    // keep freed device memory in the pool while the server runs (cohorts come and
    // go); the pool's previous release threshold is restored by stop()
    int dev = 0;
    CLR_CUDA(cudaGetDevice(&dev));
    CLR_CUDA(cudaDeviceGetDefaultMemPool(&pool_, dev));
    CLR_CUDA(cudaMemPoolGetAttribute(pool_, cudaMemPoolAttrReleaseThreshold, &pool_thr_old_));
    uint64_t thr = UINT64_MAX;
    CLR_CUDA(cudaMemPoolSetAttribute(pool_, cudaMemPoolAttrReleaseThreshold, &thr));
    pool_set_ = true;
    const int nw = (int)std::max<unsigned>(1, std::min<unsigned>(std::thread::hardware_concurrency(), 8));
    for (int i = 0; i < nw; ++i) workers_.emplace_back([this] { worker(); });
    builder_ = std::thread([this] { build_loop(); });
    stepper_ = std::thread([this] { step_loop(); });
    return CLR_OK;
  }

  void stop() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (stopping_) return;
      stopping_ = true;
    }
    cv_work_.notify_all();
    cv_build_.notify_all();
    cv_step_.notify_all();
    cv_done_.notify_all();
    for (std::thread& t : workers_)
      if (t.joinable()) t.join();
    if (builder_.joinable()) builder_.join();
    if (stepper_.joinable()) stepper_.join();
    active_.clear();  // solvers synchronise their own streams and release memory
    for (cudaStream_t s : streams_)
      if (s) cudaStreamDestroy(s);
    streams_.clear();
    if (pool_set_) {
      cudaMemPoolSetAttribute(pool_, cudaMemPoolAttrReleaseThreshold, &pool_thr_old_);
      pool_set_ = false;
    }
  }

  int submit(const clr_problem* p, uint64_t* ticket) {
    if (!p || !ticket || !p->A || !p->P_upper) return CLR_E_INVALID;
    auto r = std::make_shared<Request>();
    const clr_csc* A = p->A;
    const clr_csc* P = p->P_upper;
    if (A->ncols < 0 || A->nrows < 0 || A->nnz < 0 || P->ncols < 0 || P->nnz < 0 || (A->ncols > 0 && !A->colptr) ||
        (P->ncols > 0 && !P->colptr) || (A->nnz > 0 && (!A->rowind || !A->val)) ||
        (P->nnz > 0 && (!P->rowind || !P->val)) || (A->nrows > 0 && !p->b) || (A->ncols > 0 && !p->q) ||
        (p->ncones > 0 && !p->cones) || p->ncones < 0)
      return CLR_E_INVALID;
    r->n = A->ncols;
    r->m = A->nrows;
    r->p_nrows = P->nrows;
    r->p_ncols = P->ncols;
    if (A->colptr) r->acol.assign(A->colptr, A->colptr + (A->ncols + 1));
    else r->acol.assign(1, 0);
    r->arow.assign(A->rowind, A->rowind + A->nnz);
    r->aval.assign(A->val, A->val + A->nnz);
    if (P->colptr) r->pcol.assign(P->colptr, P->colptr + (P->ncols + 1));
    else r->pcol.assign(1, 0);
    r->prow.assign(P->rowind, P->rowind + P->nnz);
    r->pval.assign(P->val, P->val + P->nnz);
    r->q.assign(p->q, p->q + r->n);
    r->b.assign(p->b, p->b + r->m);
    r->cones.assign(p->cones, p->cones + p->ncones);
    r->t_submit = now_s();
    {
      std::lock_guard<std::mutex> lk(mu_);
      r->ticket = ++next_ticket_;
      all_[r->ticket] = r;
      todo_.push_back(r);
      ++stats_.submitted;
    }
    *ticket = r->ticket;
    cv_work_.notify_one();
    return CLR_OK;
  }

  // CLR_E_AGAIN until done; then copies the result and forgets the ticket.
  int poll(uint64_t ticket, double* x, double* s, double* z, clr_info* info, double wait_s) {
    std::unique_lock<std::mutex> lk(mu_);
    auto it = all_.find(ticket);
    if (it == all_.end()) return CLR_E_INVALID;
    std::shared_ptr<Request> r = it->second;
    if (!r->done && wait_s > 0) {
      cv_done_.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return r->done || stopping_; });
    }
    if (!r->done) return CLR_E_AGAIN;
    all_.erase(it);
    lk.unlock();
    if (r->rc != CLR_OK) return r->rc;
    if (x) std::copy(r->x.begin(), r->x.end(), x);
    if (s) std::copy(r->s.begin(), r->s.end(), s);
    if (z) std::copy(r->z.begin(), r->z.end(), z);
    if (info) *info = r->info;
    return CLR_OK;
  }

  void stats(clr_server_stats* out) {
    std::lock_guard<std::mutex> lk(mu_);
    *out = stats_;
    out->bytes_in_use = bytes_in_use_;
  }

 private:
  // ---- host analysis ----
  void worker() {
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_work_.wait(lk, [&] { return stopping_ || !todo_.empty(); });
        if (stopping_) return;
        r = todo_.front();
        todo_.pop_front();
      }
      clr_csc A{r->m, r->n, (int64_t)r->aval.size(), r->acol.data(), r->arow.data(), r->aval.data()};
      clr_csc P{r->p_nrows, r->p_ncols, (int64_t)r->pval.size(), r->pcol.data(), r->prow.data(), r->pval.data()};
      std::string err;
      if (r->rc == CLR_OK)
        r->rc = build_problem(r->hp, &P, r->q.data(), &A, r->b.data(), r->cones.data(), (int32_t)r->cones.size(),
                              st_, err);
      if (r->rc == CLR_OK) {
        int64_t nd = 0;
        int which = 0;
        choose_kkt_order(r->hp, r->order, nd, &which);
      }
      // inputs no longer needed
      std::vector<int64_t>().swap(r->pcol);
      std::vector<int64_t>().swap(r->acol);
      std::vector<int32_t>().swap(r->prow);
      std::vector<int32_t>().swap(r->arow);
      std::vector<double>().swap(r->pval);
      std::vector<double>().swap(r->aval);
      r->t_analysed = now_s();
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (r->rc != CLR_OK) {
          r->done = true;
          r->t_done = now_s();
          ++stats_.failed;
          cv_done_.notify_all();
          continue;
        }
        ready_.push_back(r);
      }
      cv_build_.notify_one();
    }
  }

  // ---- cohort formation and upload ----
  void build_loop() {
    for (;;) {
      std::vector<std::shared_ptr<Request>> take;
      int slot = -1;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_build_.wait(lk, [&] {
          if (stopping_) return true;
          if (ready_.empty()) return false;
          for (int i = 0; i < max_active_; ++i)
            if (slot_free_[i]) return bytes_in_use_ < budget_ || n_active_ == 0;
          return false;
        });
        if (stopping_) return;
        for (int i = 0; i < max_active_; ++i)
          if (slot_free_[i]) {
            slot = i;
            break;
          }
        slot_free_[slot] = 0;
        while (!ready_.empty() && (int)take.size() < max_cohort_) {
          take.push_back(ready_.front());
          ready_.pop_front();
        }
      }
      auto c = std::make_unique<Cohort>();
      c->slot = slot;
      c->reqs = take;
      c->delivered.assign(take.size(), 0);
      c->solver = std::make_unique<Solver>();
      Solver& sv = *c->solver;
      std::vector<HostProblem> hps;
      std::vector<std::vector<int64_t>> orders;
      hps.reserve(take.size());
      for (auto& r : take) {
        hps.push_back(std::move(r->hp));
        orders.push_back(std::move(r->order));
      }
      int rc = sv.use_stream_ordered(streams_[slot]);
      if (rc == CLR_OK) rc = sv.analyze_cohort(std::move(hps), orders, st_);
      if (rc == CLR_OK) rc = sv.upload();
      if (rc == CLR_OK) rc = sv.solve_begin();
      if (rc == CLR_OK) rc = sv.step_launch();  // captures the iteration graph
      c->bytes = sv.device_bytes();
      std::lock_guard<std::mutex> lk(mu_);
      if (rc != CLR_OK) {
        for (auto& r : take) {
          r->rc = rc;
          r->done = true;
          r->t_done = now_s();
          ++stats_.failed;
        }
        c.reset();
        slot_free_[slot] = 1;
        cv_done_.notify_all();
        continue;
      }
      c->stepping = true;
      bytes_in_use_ += c->bytes;
      stats_.peak_bytes = std::max(stats_.peak_bytes, (int64_t)bytes_in_use_);
      ++stats_.cohorts;
      stats_.admitted += (int64_t)take.size();
      stats_.max_cohort_seen = std::max<int64_t>(stats_.max_cohort_seen, (int64_t)take.size());
      incoming_.push_back(std::move(c));
      ++n_active_;
      cv_step_.notify_one();
    }
  }

  // ---- interleaved iterations and hand-out ----
  void deliver(Cohort& c, int64_t p, bool final_step) {
    Request& r = *c.reqs[p];
    r.x.resize(r.n);
    r.s.resize(r.m);
    r.z.resize(r.m);
    Solver& sv = *c.solver;
    int rc = final_step ? sv.get_solution(p, r.x.data(), r.s.data(), r.z.data(), &r.info)
                        : sv.get_solution_now(p, r.x.data(), r.s.data(), r.z.data(), &r.info);
    r.t_done = now_s();
    r.info.setup_s = r.t_analysed - r.t_submit;  // host analysis incl. queueing for a worker
    r.info.solve_s = r.t_done - r.t_submit;      // latency: submit -> result readable
    std::lock_guard<std::mutex> lk(mu_);
    r.rc = rc;
    r.done = true;
    c.delivered[p] = 1;
    ++stats_.completed;
  }

  void step_loop() {
    std::vector<std::unique_ptr<Cohort>> active;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        if (active.empty())
          cv_step_.wait(lk, [&] { return stopping_ || !incoming_.empty(); });
        if (stopping_) {
          active_ = std::move(active);
          for (auto& c : incoming_) active_.push_back(std::move(c));
          incoming_.clear();
          return;
        }
        for (auto& c : incoming_) active.push_back(std::move(c));
        incoming_.clear();
      }
      bool progressed = false;
      for (size_t i = 0; i < active.size();) {
        Cohort& c = *active[i];
        Solver& sv = *c.solver;
        bool ready = false;
        int rc = sv.step_poll(&ready);
        if (rc == CLR_OK && !ready) {
          ++i;
          continue;
        }
        progressed = true;
        bool finished = rc != CLR_OK || sv.all_halted();
        if (rc == CLR_OK && !finished) {
          for (int64_t p = 0; p < (int64_t)c.reqs.size(); ++p)
            if (!c.delivered[p] && sv.problem_status(p) != 0) deliver(c, p, false);
          rc = sv.step_launch();
          finished = rc != CLR_OK;
        }
        if (finished) {
          if (rc == CLR_OK) rc = sv.solve_end();
          for (int64_t p = 0; p < (int64_t)c.reqs.size(); ++p) {
            if (c.delivered[p]) continue;
            if (rc == CLR_OK) {
              deliver(c, p, true);
            } else {
              std::lock_guard<std::mutex> lk(mu_);
              c.reqs[p]->rc = rc;
              c.reqs[p]->done = true;
              c.reqs[p]->t_done = now_s();
              ++stats_.failed;
            }
          }
          const int slot = c.slot;
          const size_t bytes = c.bytes;
          active[i].reset();  // frees the cohort (stream-ordered)
          active.erase(active.begin() + (long)i);
          {
            std::lock_guard<std::mutex> lk(mu_);
            slot_free_[slot] = 1;
            bytes_in_use_ -= bytes;
            --n_active_;
          }
          cv_build_.notify_one();
        } else {
          ++i;
        }
        cv_done_.notify_all();
      }
      if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }

  cudaMemPool_t pool_ = nullptr;  // the device's default pool (stream-ordered allocations)
  uint64_t pool_thr_old_ = 0;      // its release threshold before start()
  bool pool_set_ = false;
  size_t budget_;
  int max_cohort_, max_active_;
  clr_settings st_;
  std::mutex mu_;
  std::condition_variable cv_work_, cv_build_, cv_step_, cv_done_;
  bool stopping_ = false;
  uint64_t next_ticket_ = 0;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> all_;
  std::deque<std::shared_ptr<Request>> todo_, ready_;
  std::vector<std::unique_ptr<Cohort>> incoming_, active_;
  std::vector<cudaStream_t> streams_;
  std::vector<char> slot_free_;
  size_t bytes_in_use_ = 0;
  int n_active_ = 0;
  clr_server_stats stats_{};
  std::vector<std::thread> workers_;
  std::thread builder_, stepper_;
};

}  // namespace clr

struct clr_server {
  std::unique_ptr<clr::Server> impl;
};

extern "C" {

int clr_server_create(clr_server** out, size_t device_bytes, int32_t max_cohort, int32_t max_active,
                      const clr_settings* st) {
  if (!out || max_cohort < 1 || max_active < 1 || device_bytes == 0) return CLR_E_INVALID;
  *out = nullptr;
  clr_settings s;
  if (st) s = *st;
  else clr_default_settings(&s, 64);
  if (s.factor_bits != 64 && s.factor_bits != 32 && s.factor_bits != 16) return CLR_E_INVALID;
  s.use_graph = 1;
  auto* h = new (std::nothrow) clr_server;
  if (!h) return CLR_E_OOM;
  h->impl = std::make_unique<clr::Server>(device_bytes, max_cohort, max_active, s);
  int rc = h->impl->start();
  if (rc != CLR_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return CLR_OK;
}

int clr_server_submit(clr_server* sv, const clr_problem* p, uint64_t* ticket) {
  if (!sv) return CLR_E_INVALID;
  return sv->impl->submit(p, ticket);
}

int clr_server_poll(clr_server* sv, uint64_t ticket, double* x, double* sl, double* z, clr_info* info) {
  if (!sv) return CLR_E_INVALID;
  return sv->impl->poll(ticket, x, sl, z, info, 0.0);
}

int clr_server_wait(clr_server* sv, uint64_t ticket, double timeout_s, double* x, double* sl, double* z,
                    clr_info* info) {
  if (!sv || !(timeout_s >= 0)) return CLR_E_INVALID;
  int rc = sv->impl->poll(ticket, x, sl, z, info, timeout_s);
  return rc == CLR_E_AGAIN ? CLR_E_TIMEOUT : rc;
}

int clr_server_get_stats(clr_server* sv, clr_server_stats* out) {
  if (!sv || !out) return CLR_E_INVALID;
  sv->impl->stats(out);
  return CLR_OK;
}

int clr_server_destroy(clr_server* sv) {
  if (!sv) return CLR_E_INVALID;
  sv->impl->stop();
  delete sv;
  return CLR_OK;
}

}  // extern "C"
