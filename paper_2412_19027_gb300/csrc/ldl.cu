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
#include <queue>
#include <unordered_map>

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
                          const int32_t* __restrict__ pos_pid, int64_t N, const IterScal* sc, const int* skip) {
  if (skip && *skip) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
    F[diag_pos[k]] += (T)(dsign[k] * sc[pos_pid[k]].delta);
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

// Extend-add of large update blocks by relative indices, one child per front per
// launch: 32 x 32 tiles of the lower update block U_J (rows/cols c_J .. f_J-1 of
// front J) added into the parent front at (rel[a], rel[b]).
template <typename T>
__global__ void k_push(T* __restrict__ F, WorkList wl, const int64_t* __restrict__ sn_ptr,
                       const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ front_off,
                       const int64_t* __restrict__ sn_parent, const int64_t* __restrict__ rel_off,
                       const int32_t* __restrict__ rel, const int* skip) {
  if (skip && *skip) return;
  int64_t lo = 0, hi = wl.nfront - 1;
  const int64_t bid = blockIdx.x;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (wl.pref[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  const int64_t J = wl.front[lo], q = bid - wl.pref[lo];
  const int64_t c = sn_ptr[J + 1] - sn_ptr[J], f = row_ptr[J + 1] - row_ptr[J], r = f - c;
  int64_t ti = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) / 2.0);
  while (ti * (ti + 1) / 2 > q) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= q) ++ti;
  const int64_t tj = q - ti * (ti + 1) / 2;
  const int64_t P = sn_parent[J];
  const int64_t fP = row_ptr[P + 1] - row_ptr[P];
  const T* U = F + front_off[J];
  T* FP = F + front_off[P];
  const int32_t* rl = rel + rel_off[J];
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int64_t a = ti * 32 + (e & 31), b = tj * 32 + (e >> 5);
    if (a < r && b < r && a >= b) FP[rl[a] + (int64_t)rl[b] * fP] += U[(c + a) + (c + b) * f];
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
                            int small_max, const int* skip) {
  if (skip && *skip) return;
  __shared__ T xb[32];
  const int64_t J = fronts[blockIdx.x];
  const int64_t c = sn_ptr[J + 1] - sn_ptr[J];
  const int64_t f = row_ptr[J + 1] - row_ptr[J];
  if (f > small_max) return;
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
                            int small_max, const int* skip) {
  if (skip && *skip) return;
  const int64_t J = fronts[blockIdx.x];
  const int64_t c = sn_ptr[J + 1] - sn_ptr[J];
  const int64_t f = row_ptr[J + 1] - row_ptr[J];
  if (f > small_max) return;
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

// Order the tasks [t0, end) of one level for the counter of k_bf_flow.  A CTA
// takes the next ticket as soon as it is free and then waits until the task's
// inputs are there, so a ticket handed out long before its task can run keeps a
// CTA idle.  The order is therefore that of a list schedule simulated on the
// host: `workers` CTAs, each task taking its typical duration (FP32 times per
// kind measured on a GB300, 64 x 64 tiles) plus a notification delay after each
// input; a free CTA starts, among the tasks whose inputs are done, the one with
// the largest bottom level (longest weighted path to the end), and the tickets
// follow the simulated start times.  The fused chain task DX(p) publishes the L
// rows of block p early (its trsm word), so the updates that only read those
// rows count from that point.  Start times never decrease along the order and
// each task starts after its inputs finish, so the order is topological: every
// wait is for a smaller ticket.  Returns false if the graph has a cycle (a bug:
// the caller then fails the setup).  The caller schedules each level twice --
// two CTAs per SM, or one CTA per SM whose tasks run faster without a second
// CTA beside them -- and keeps the shorter.
//   deps: D(0) -; DX(p) D/DX(p-1), U(p-2, p, p-1), U(p-2, p, p);
//   T(p, i) D/DX(p), U(p-1, i, p); Efin(p, e) D/DX(p), EU(p-1, p, e);
//   U(p, i, j) T~(p, i), T~(p, j), U(p-1, i, j);
//   EU(p, i, e) T~(p, i), Efin(p, e) or D/DX(p) (e = p), EU(p-1, i, e);
// T~(p, i) is DX(p+1) when i = p + 1 is a pivot block (folded), else T(p, i).
// dur: typical durations (microseconds) by kind D, T, Efin, U, EU, DX; span: the
// simulated duration of the level.
static bool flow_schedule_order(std::vector<FlowTask>& tasks, int64_t t0, const std::vector<int64_t>& P_of,
                                int workers, const double* dur, double* span, bool split = false) {
  const int64_t n = (int64_t)tasks.size() - t0;
  *span = 0.0;
  if (n <= 1) return true;
  // DX publishes its L rows this long after it starts; delay of a notification
  const double kMid = 6.0, kLat = 2.5;
  auto key = [](int64_t b, int kind, int64_t p, int64_t i, int64_t j) -> uint64_t {
    return ((uint64_t)b << 43) ^ ((uint64_t)kind << 40) ^ ((uint64_t)p << 28) ^ ((uint64_t)i << 14) ^ (uint64_t)j;
  };
  std::unordered_map<uint64_t, int64_t> idx;
  idx.reserve((size_t)n * 2);
  for (int64_t t = 0; t < n; ++t) {
    const FlowTask& k = tasks[t0 + t];
    idx[key(k.bf, k.kind, k.p, k.i, k.j)] = t;
  }
  auto find = [&](int64_t b, int kind, int64_t p, int64_t i, int64_t j) -> int64_t {
    auto it = idx.find(key(b, kind, p, i, j));
    return it == idx.end() ? -1 : it->second;
  };
  // split: FP64 chain tasks TX(p, q), UX(p, q), D(p) in place of DX(p) (bigfront.cuh)
  auto dd = [&](int64_t b, int64_t p) {
    return (p == 0 || split) ? find(b, 0, p, p, p) : find(b, 5, p, p, p);
  };
  auto folded = [&](int64_t b, int64_t p, int64_t i) { return i == p + 1 && i < P_of[b]; };
  struct Edge {
    int64_t to;
    bool mid;  // the successor needs only the early-published rows of a DX task
  };
  std::vector<std::vector<Edge>> succ(n);
  std::vector<int> indeg(n, 0);
  std::vector<std::pair<int64_t, bool>> d;  // predecessors of one task (index, mid)
  // the producer(s) of L_IK, block row i of panel p: T(p, i), DX(p + 1) when folded
  // (its early-published rows), or the four parts TX(p + 1, q) when split
  auto add_tt = [&](int64_t b, int64_t p, int64_t i) {
    if (!folded(b, p, i)) d.emplace_back(find(b, 1, p, i, p), false);
    else if (!split) d.emplace_back(find(b, 5, i, i, i), true);
    else
      for (int64_t q = 0; q < 4; ++q) d.emplace_back(find(b, 6, i, q, 0), false);
  };
  for (int64_t t = 0; t < n; ++t) {
    const FlowTask& k = tasks[t0 + t];
    d.clear();
    const int64_t p = k.p, i = k.i, j = k.j, b = k.bf;
    switch (k.kind) {
      case 0:
        if (split && p >= 1)
          for (int64_t q = 0; q < 4; ++q) d.emplace_back(find(b, 7, p, q, 0), false);
        break;
      case 5:
        d.emplace_back(dd(b, p - 1), false);
        if (p >= 2) {
          d.emplace_back(find(b, 3, p - 2, p, p - 1), false);
          d.emplace_back(find(b, 3, p - 2, p, p), false);
        }
        break;
      case 6:
        d.emplace_back(dd(b, p - 1), false);
        if (p >= 2) d.emplace_back(find(b, 3, p - 2, p, p - 1), false);
        break;
      case 7:
        for (int64_t q = 0; q < 4; ++q) d.emplace_back(find(b, 6, p, q, 0), false);
        if (p >= 2) d.emplace_back(find(b, 3, p - 2, p, p), false);
        break;
      case 1:
        d.emplace_back(dd(b, p), false);
        if (p > 0) d.emplace_back(find(b, 3, p - 1, i, p), false);
        break;
      case 2:
        d.emplace_back(dd(b, p), false);
        if (p - 1 >= j) d.emplace_back(find(b, 4, p - 1, p, j), false);
        break;
      case 3:
        add_tt(b, p, i);
        add_tt(b, p, j);
        if (p > 0) d.emplace_back(find(b, 3, p - 1, i, j), false);
        break;
      default:
        add_tt(b, p, i);
        d.emplace_back(j < p ? find(b, 2, p, p, j) : dd(b, p), false);
        if (p - 1 >= j) d.emplace_back(find(b, 4, p - 1, i, j), false);
        break;
    }
    for (size_t q = 0; q < d.size(); ++q) {
      if (d[q].first < 0) continue;
      bool dup = false;
      for (size_t r = 0; r < q; ++r) dup = dup || d[r].first == d[q].first;
      if (dup) continue;
      succ[d[q].first].push_back(Edge{t, d[q].second});
      ++indeg[t];
    }
  }
  // a topological order (FIFO Kahn), then bottom levels in its reverse
  std::vector<int64_t> topo;
  topo.reserve((size_t)n);
  {
    std::vector<int> deg = indeg;
    for (int64_t t = 0; t < n; ++t)
      if (deg[t] == 0) topo.push_back(t);
    for (size_t h = 0; h < topo.size(); ++h)
      for (const Edge& e : succ[topo[h]])
        if (--deg[e.to] == 0) topo.push_back(e.to);
  }
  if ((int64_t)topo.size() != n) return false;
  std::vector<double> bl(n, 0.0);
  for (int64_t h = n - 1; h >= 0; --h) {
    const int64_t t = topo[h];
    double m = 0.0;
    for (const Edge& e : succ[t]) m = std::max(m, bl[e.to]);
    bl[t] = m + dur[tasks[t0 + t].kind];
  }
  // the list schedule
  using TimeTask = std::pair<double, int64_t>;
  std::priority_queue<TimeTask, std::vector<TimeTask>, std::greater<TimeTask>> pending;  // (ready time, task)
  std::priority_queue<std::pair<double, int64_t>> avail;                                 // (bottom level, -task)
  std::priority_queue<double, std::vector<double>, std::greater<double>> cta;           // free times
  for (int w = 0; w < std::max(1, workers); ++w) cta.push(0.0);
  std::vector<double> ready(n, 0.0);
  for (int64_t t = 0; t < n; ++t)
    if (indeg[t] == 0) pending.emplace(0.0, t);
  std::vector<FlowTask> out;
  out.reserve((size_t)n);
  while ((int64_t)out.size() < n) {
    const double now = cta.top();
    cta.pop();
    while (!pending.empty() && pending.top().first <= now) {
      avail.emplace(bl[pending.top().second], -pending.top().second);
      pending.pop();
    }
    if (avail.empty()) {
      if (pending.empty()) return false;
      cta.push(pending.top().first);  // idle until the next task is ready
      continue;
    }
    const int64_t t = -avail.top().second;
    avail.pop();
    out.push_back(tasks[t0 + t]);
    const double fin = now + dur[tasks[t0 + t].kind];
    *span = std::max(*span, fin);
    cta.push(fin);
    for (const Edge& e : succ[t]) {
      ready[e.to] = std::max(ready[e.to], (e.mid ? now + kMid : fin) + kLat);
      if (--indeg[e.to] == 0) pending.emplace(ready[e.to], e.to);
    }
  }
  std::copy(out.begin(), out.end(), tasks.begin() + t0);
  return true;
}

int ldl_structure_upload(DeviceArena& ar, const Symbolic& sy, const NumericMaps& mp, const std::vector<int8_t>& dsign,
                         int small_max, LdlStructure& st, const std::vector<int32_t>* pos_pid) {
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
  // ---- extend-add rounds by relative indices ----
  {
    st.rel = up(ar, mp.rel);
    st.rel_off = up(ar, mp.rel_off);
    st.sn_parent = up(ar, sy.sn_parent);
    std::vector<int64_t> buf;
    std::vector<std::pair<size_t, size_t>> where;  // (front offset, prefix offset) in buf per list
    st.push_rounds.assign(sy.nlev, {});
    for (int64_t l = 0; l < sy.nlev; ++l)
      for (int64_t k = mp.px_lev_ptr[l]; k < mp.px_lev_ptr[l + 1]; ++k) {
        WorkList wl;
        const size_t fo = buf.size();
        for (int64_t t = mp.px_round_ptr[k]; t < mp.px_round_ptr[k + 1]; ++t) buf.push_back(mp.px_child[t]);
        const size_t po = buf.size();
        int64_t nb = 0;
        for (int64_t t = mp.px_round_ptr[k]; t < mp.px_round_ptr[k + 1]; ++t) {
          const int64_t J = mp.px_child[t];
          const int64_t r = (sy.row_ptr[J + 1] - sy.row_ptr[J]) - (sy.sn_ptr[J + 1] - sy.sn_ptr[J]);
          const int64_t T = (r + 31) / 32;
          buf.push_back(nb);
          nb += T * (T + 1) / 2;
        }
        buf.push_back(nb);
        wl.nfront = mp.px_round_ptr[k + 1] - mp.px_round_ptr[k];
        wl.nblocks = nb;
        st.push_rounds[l].push_back(wl);
        where.emplace_back(fo, po);
      }
    int64_t* dbuf = buf.empty() ? nullptr : ar.upload(buf.data(), (int64_t)buf.size());
    if (!buf.empty() && !dbuf) return CLR_E_OOM;
    size_t w = 0;
    for (int64_t l = 0; l < sy.nlev; ++l)
      for (WorkList& wl : st.push_rounds[l]) {
        wl.front = dbuf + where[w].first;
        wl.pref = dbuf + where[w].second;
        ++w;
      }
    if ((!mp.rel.empty() && !st.rel) || !st.rel_off || !st.sn_parent) return CLR_E_OOM;
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
  // ---- big fronts: arrays, E / y pools, launch plans per level ----
  {
    std::vector<int64_t> bf_f, bf_c, bf_goff, bf_eoff, bf_k0, bf_woff, bf_yoff, bf_rk, bf_pk;
    std::vector<int64_t> bid_of(sy.nsn, -1);
    int64_t epool = 0, ypool = 0;
    st.pk_tiles = 0;
    for (int64_t l = 0; l < sy.nlev; ++l) {
      int64_t pk_level = 0;  // packed tiles are scratch of one level's launch: offsets restart per level
      for (int64_t J : st.lev_big[l]) {
        const int64_t f = sy.row_ptr[J + 1] - sy.row_ptr[J], c = sy.sn_ptr[J + 1] - sy.sn_ptr[J];
        bid_of[J] = (int64_t)bf_f.size();
        bf_f.push_back(f);
        bf_c.push_back(c);
        bf_goff.push_back(sy.front_off[J]);
        bf_eoff.push_back(epool);
        bf_k0.push_back(sy.sn_ptr[J]);
        bf_woff.push_back(sy.upd_off[J]);
        bf_yoff.push_back(ypool);
        bf_rk.push_back(sy.row_ptr[J]);
        bf_pk.push_back(pk_level);
        pk_level += flow_pk_tiles(f, c);
        epool += f * c;
        ypool += c;
      }
      st.pk_tiles = std::max(st.pk_tiles, pk_level);
    }
    BigFrontDev& bd = st.bfd;
    bd.n = (int64_t)bf_f.size();
    bd.epool = epool;
    bd.ypool = ypool;
    bd.f = up(ar, bf_f);
    bd.c = up(ar, bf_c);
    bd.goff = up(ar, bf_goff);
    bd.eoff = up(ar, bf_eoff);
    bd.k0pos = up(ar, bf_k0);
    bd.woff = up(ar, bf_woff);
    bd.yoff = up(ar, bf_yoff);
    bd.rk = up(ar, bf_rk);
    bd.pkoff = up(ar, bf_pk);
    // work lists: host-built (front ids, prefix sums), uploaded in one buffer
    std::vector<int64_t> buf;
    struct Pending {
      WorkList* wl;
      size_t fo, po;
    };
    std::vector<Pending> pend;
    st.bplans.assign(sy.nlev, BigLevelPlan());
    auto add_list = [&](WorkList& wl, const std::vector<int64_t>& fronts, const std::vector<int64_t>& counts) {
      wl.nfront = 0;
      wl.nblocks = 0;
      std::vector<int64_t> fr, pr;
      for (size_t i = 0; i < fronts.size(); ++i)
        if (counts[i] > 0) {
          fr.push_back(fronts[i]);
          pr.push_back(wl.nblocks);
          wl.nblocks += counts[i];
        }
      pr.push_back(wl.nblocks);
      wl.nfront = (int64_t)fr.size();
      if (wl.nfront == 0) return;
      Pending pd{&wl, buf.size(), 0};
      buf.insert(buf.end(), fr.begin(), fr.end());
      pd.po = buf.size();
      buf.insert(buf.end(), pr.begin(), pr.end());
      pend.push_back(pd);
    };
    for (int64_t l = 0; l < sy.nlev; ++l) {
      if (st.lev_big[l].empty()) continue;
      BigLevelPlan& pl = st.bplans[l];
      std::vector<int64_t> ids;
      int maxp = 0;
      for (int64_t J : st.lev_big[l]) {
        ids.push_back(bid_of[J]);
        maxp = std::max<int>(maxp, (int)((bf_c[bid_of[J]] + kBfNB - 1) / kBfNB));
      }
      pl.A.resize(maxp + 1);
      pl.B.resize(maxp + 1);
      pl.C.resize(maxp + 1);
      pl.Ctc.resize(maxp + 1);
      for (int p = 0; p <= maxp; ++p) {
        std::vector<int64_t> ca, cb, cc, ct;
        for (int64_t b : ids) {
          const int64_t f = bf_f[b], c = bf_c[b];
          ca.push_back((int64_t)p * kBfNB < c ? 1 : 0);
          cb.push_back(bf_trsm_blocks(f, c, p) + bf_fin_blocks(c, p));
          cc.push_back(bf_update_tiles(f, c, p));
          ct.push_back(bf_tc_tiles(f, c, p));
        }
        add_list(pl.A[p], ids, ca);
        add_list(pl.B[p], ids, cb);
        add_list(pl.C[p], ids, cc);
        add_list(pl.Ctc[p], ids, ct);
      }
      std::vector<int64_t> cf, cbw;
      for (int64_t b : ids) {
        cf.push_back((bf_f[b] + 31) / 32);
        cbw.push_back((bf_c[b] + 7) / 8);
      }
      add_list(pl.fwd, ids, cf);
      add_list(pl.bwd, ids, cbw);
    }
    int64_t* dbuf = buf.empty() ? nullptr : ar.upload(buf.data(), (int64_t)buf.size());
    if (!buf.empty() && !dbuf) return CLR_E_OOM;
    for (Pending& pd : pend) {
      pd.wl->front = dbuf + pd.fo;
      pd.wl->pref = dbuf + pd.po;
    }
    // dataflow task tables (bigfront.cuh), per level: every task of every big front
    // of the level, then ordered by flow_schedule_order.  A pivot block p >= 1
    // has the fused task DX(p) instead of D(p), T(p-1, p) and U(p-1, p, p).
    std::vector<FlowTask> tasks;
    std::vector<int64_t> soff(bf_f.size(), 0), P_of(bf_f.size(), 0);
    // SMs of the device: a launch of k_bf_flow runs one or two CTAs on each
    int flow_sms = 152, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        sms > 0)
      flow_sms = sms;
    st.flow_one.assign(sy.nlev, 0);
    st.flow_tc.assign(sy.nlev, 0);
    int64_t words = 0;
    st.flow_t0.assign(sy.nlev, 0);
    st.flow_nt.assign(sy.nlev, 0);
    st.flow_head.assign(sy.nlev, 0);
    for (int64_t l = 0; l < sy.nlev; ++l) {
      if (st.lev_big[l].empty()) continue;
      st.flow_head[l] = words++;
      st.flow_t0[l] = (int64_t)tasks.size();
      auto add = [&](int64_t b, int kind, int64_t p, int64_t i, int64_t j) {
        tasks.push_back(FlowTask{(int32_t)b, (int16_t)kind, (int16_t)p, (int32_t)i, (int32_t)j});
      };
      for (int64_t J : st.lev_big[l]) {
        const int64_t b = bid_of[J];
        soff[b] = words;
        words += flow_words(bf_f[b], bf_c[b]);
        const int64_t P = (bf_c[b] + kBfNB - 1) / kBfNB, nb = flow_nbf(bf_f[b], bf_c[b]);
        P_of[b] = P;
        for (int64_t p = 0; p < P; ++p) {
          add(b, p == 0 ? 0 : 5, p, p, p);
          for (int64_t i = p + 1; i < nb; ++i)
            if (!(i == p + 1 && i < P)) add(b, 1, p, i, p);
          for (int64_t e = 0; e < p; ++e) add(b, 2, p, p, e);
          for (int64_t j = p + 1; j < nb; ++j)
            for (int64_t i = j; i < nb; ++i)
              if (!(i == p + 1 && j == p + 1 && i < P)) add(b, 3, p, i, j);
          for (int64_t i = p + 1; i < nb; ++i)
            for (int64_t e = 0; e <= p; ++e) add(b, 4, p, i, e);
        }
      }
      st.flow_nt[l] = (int64_t)tasks.size() - st.flow_t0[l];
      // FP32 task times (microseconds; D, T, Efin, U, EU, DX) measured on a GB300
      // with two CTAs per SM and with one (no second CTA competing for the SM),
      // and of the tensor-core launch (two CTAs per SM; per-task timestamps on the
      // mixed-cone QP's root front: U and EU ~0.8x, the diagonal tasks ~1.1x and
      // the panel tasks ~1.08x those of the CUDA-core launch)
      static const double dur2[8] = {22.0, 7.0, 5.5, 8.0, 8.0, 27.0, 0.0, 0.0};
      static const double dur1[8] = {20.0, 6.5, 5.3, 5.8, 6.1, 25.0, 0.0, 0.0};
      static const double dur2tc[8] = {25.2, 7.6, 5.9, 6.5, 5.9, 29.8, 0.0, 0.0};
      std::vector<FlowTask> one(tasks.begin() + st.flow_t0[l], tasks.end()), tco(one);
      double span2 = 0.0, span1 = 0.0, spantc = 0.0;
      if (!flow_schedule_order(tasks, st.flow_t0[l], P_of, 2 * flow_sms, dur2, &span2) ||
          !flow_schedule_order(one, 0, P_of, flow_sms, dur1, &span1) ||
          !flow_schedule_order(tco, 0, P_of, 2 * flow_sms, dur2tc, &spantc))
        return CLR_E_INVALID;
      // the launch of the level: the shortest simulated schedule (the one-CTA and
      // tensor-core launches only when at least 3 % shorter); the tensor-core
      // launch applies to FP32 factors only -- an FP64 factor runs its CUDA-core
      // launch in the order simulated for that choice (any of the orders is valid)
      const double best_cc = std::min(span2, span1 < 0.97 * span2 ? span1 : span2);
      st.flow_tc[l] = spantc < 0.97 * best_cc ? 1 : 0;
      st.flow_one[l] = (!st.flow_tc[l] && span1 < 0.97 * span2) ? 1 : 0;
      if (st.flow_tc[l]) std::copy(tco.begin(), tco.end(), tasks.begin() + st.flow_t0[l]);
      else if (st.flow_one[l]) std::copy(one.begin(), one.end(), tasks.begin() + st.flow_t0[l]);
    }
    st.flow_words = words;
    // the FP64 factor's table: the same levels, fronts and version words, with the
    // fused chain task split into TX(p, q), UX(p, q) and D(p) (bigfront.cuh)
    std::vector<FlowTask> tasks64;
    st.flow_t0_64.assign(sy.nlev, 0);
    st.flow_nt_64.assign(sy.nlev, 0);
    st.flow_one64.assign(sy.nlev, 0);
    for (int64_t l = 0; l < sy.nlev; ++l) {
      if (st.lev_big[l].empty()) continue;
      st.flow_t0_64[l] = (int64_t)tasks64.size();
      auto add = [&](int64_t b, int kind, int64_t p, int64_t i, int64_t j) {
        tasks64.push_back(FlowTask{(int32_t)b, (int16_t)kind, (int16_t)p, (int32_t)i, (int32_t)j});
      };
      for (int64_t J : st.lev_big[l]) {
        const int64_t b = bid_of[J];
        const int64_t P = P_of[b], nb = flow_nbf(bf_f[b], bf_c[b]);
        for (int64_t p = 0; p < P; ++p) {
          if (p >= 1) {
            for (int64_t q = 0; q < 4; ++q) add(b, 6, p, q, 0);
            for (int64_t q = 0; q < 4; ++q) add(b, 7, p, q, 0);
          }
          add(b, 0, p, p, p);
          for (int64_t i = p + 1; i < nb; ++i)
            if (!(i == p + 1 && i < P)) add(b, 1, p, i, p);
          for (int64_t e = 0; e < p; ++e) add(b, 2, p, p, e);
          for (int64_t j = p + 1; j < nb; ++j)
            for (int64_t i = j; i < nb; ++i)
              if (!(i == p + 1 && j == p + 1 && i < P)) add(b, 3, p, i, j);
          for (int64_t i = p + 1; i < nb; ++i)
            for (int64_t e = 0; e <= p; ++e) add(b, 4, p, i, e);
        }
      }
      st.flow_nt_64[l] = (int64_t)tasks64.size() - st.flow_t0_64[l];
      // FP64 task times (microseconds; D, T, Efin, U, EU, -, TX, UX) from per-task
      // timestamps on a GB300 at two CTAs per SM (banded LP generator), and estimates
      // for one CTA per SM (a task then has the SM's FP64 pipe to itself)
      static const double dur64_2[8] = {95.0, 41.0, 57.0, 57.0, 57.0, 204.0, 12.0, 14.0};
      static const double dur64_1[8] = {70.0, 28.0, 38.0, 36.0, 36.0, 150.0, 8.0, 9.0};
      std::vector<FlowTask> one(tasks64.begin() + st.flow_t0_64[l], tasks64.end());
      double span2 = 0.0, span1 = 0.0;
      if (!flow_schedule_order(tasks64, st.flow_t0_64[l], P_of, 2 * flow_sms, dur64_2, &span2, true) ||
          !flow_schedule_order(one, 0, P_of, flow_sms, dur64_1, &span1, true))
        return CLR_E_INVALID;
      st.flow_one64[l] = span1 < 0.97 * span2 ? 1 : 0;
      if (st.flow_one64[l]) std::copy(one.begin(), one.end(), tasks64.begin() + st.flow_t0_64[l]);
    }
    if (!tasks.empty()) {
      st.flow_task = ar.upload(tasks.data(), (int64_t)tasks.size());
      st.flow_task64 = ar.upload(tasks64.data(), (int64_t)tasks64.size());
      st.flow_soff = ar.upload(soff.data(), (int64_t)soff.size());
      if (!st.flow_task || !st.flow_task64 || !st.flow_soff) return CLR_E_OOM;
    }
  }
  st.sn_ptr = up(ar, sy.sn_ptr);
  st.row_ptr = up(ar, sy.row_ptr);
  st.front_off = up(ar, sy.front_off);
  st.upd_off = up(ar, sy.upd_off);
  st.lev_sn = up(ar, sy.lev_sn);
  st.rows_kkt = up(ar, mp.rows_kkt);
  st.w_init = up(ar, w_init);
  st.dsign = up(ar, dsign);
  {
    std::vector<int32_t> zeros;
    if (!pos_pid) zeros.assign(sy.N, 0);
    st.pos_pid = up(ar, pos_pid ? *pos_pid : zeros);
  }
  st.kdest = up(ar, mp.kdest);
  st.diag_pos = up(ar, mp.diag_pos);
  st.fa_tgt = up(ar, mp.fa_tgt);
  st.fa_ptr = up(ar, mp.fa_ptr);
  st.fa_src = up(ar, mp.fa_src);
  st.sv_tgt = up(ar, mp.sv_tgt);
  st.sv_ptr = up(ar, mp.sv_ptr);
  st.sv_src = up(ar, mp.sv_src);
  if (!st.sn_ptr || !st.row_ptr || !st.front_off || !st.upd_off || !st.lev_sn || !st.rows_kkt || !st.w_init ||
      !st.dsign || !st.pos_pid || !st.kdest || !st.diag_pos || !st.fa_tgt || !st.fa_ptr || !st.fa_src || !st.sv_tgt ||
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
  dyn_hits = ar.alloc_n<int>(2);
  tc_err = dyn_hits ? dyn_hits + 1 : nullptr;
  E = ar.alloc_n<T>(st.bfd.epool);
  ybuf = ar.alloc_n<T>(st.bfd.ypool);
  Linv = ar.alloc_n<T>(st.bfd.n * 2 * kBfNB * kBfNB);
  if (!F || !Dp || !w || !xs || !dyn_hits || !E || !ybuf || !Linv) return CLR_E_OOM;
  if (BigFrontOps<T>::setup_attributes() != CLR_OK) return CLR_E_CUDA;
  if (st.flow_words > 0) {
    flow_state = ar.alloc_n<int>(st.flow_words);
    if (!flow_state) return CLR_E_OOM;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return CLR_E_CUDA;
    const bool tc = use_flow_tc();
    if (tc) {
      tcs.tiles = st.pk_tiles;
      tcs.pk = ar.alloc_n<float>(st.pk_tiles * kPkWords);
      if (!tcs.pk) return CLR_E_OOM;
      const int rc = flow_tc_encode(&tcs);
      if (rc != CLR_OK) return rc;
    }
    const int occ = BigFrontOps<T>::flow_occupancy(tc);
    if (occ < 0) return CLR_E_CUDA;
    flow_sms = sms;
    flow_occ = occ;
  }
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_factor_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  return CLR_OK;
}

template <typename T>
int LdlFactor<T>::factor(cudaStream_t stm, const double* kval, const IterScal* sc, double dyn_eps, double dyn_delta,
                         const int* skip) const {
  const LdlStructure& S = *s;
  CLR_CUDA(cudaMemsetAsync(dyn_hits, 0, 2 * sizeof(int), stm));  // dynamic-regularisation hits, big-front error
  const bool use_flow = flow && !tc16 && flow_state != nullptr;
  if (use_flow) CLR_CUDA(cudaMemsetAsync(flow_state, 0, sizeof(int) * (size_t)S.flow_words, stm));
  CLR_CUDA(cudaMemsetAsync(F, 0, sizeof(T) * (size_t)S.pool, stm));
  if (S.bfd.epool > 0) CLR_CUDA(cudaMemsetAsync(E, 0, sizeof(T) * (size_t)S.bfd.epool, stm));
  k_scatter_kval<T><<<grid_for(S.nk, 256), 256, 0, stm>>>(F, kval, S.kdest, S.nk, skip);
  k_add_reg<T><<<grid_for(S.N, 256), 256, 0, stm>>>(F, S.diag_pos, S.dsign, S.pos_pid, S.N, sc, skip);
  CLR_CHECK_LAUNCH();
  for (int64_t l = 0; l < S.nlev; ++l) {
    const int64_t t0 = S.h_fa_lev_ptr[l], t1 = S.h_fa_lev_ptr[l + 1];
    if (t1 > t0) k_pull<T><<<grid_for(t1 - t0, 256), 256, 0, stm>>>(F, S.fa_tgt, S.fa_ptr, S.fa_src, t0, t1, skip);
    for (const WorkList& wl : S.push_rounds[l])
      if (wl.nblocks > 0)
        k_push<T><<<(unsigned)wl.nblocks, 256, 0, stm>>>(F, wl, S.sn_ptr, S.row_ptr, S.front_off, S.sn_parent,
                                                          S.rel_off, S.rel, skip);
    const int64_t nf = S.h_lev_ptr[l + 1] - S.h_lev_ptr[l];
    if ((int64_t)S.lev_big[l].size() < nf) {
      const int mf = S.lev_small_maxf[l];
      const size_t smem = sizeof(T) * (size_t)mf * (size_t)mf;
      const int threads = mf <= 16 ? 64 : (mf <= 48 ? 128 : 256);
      k_factor_small<T><<<(unsigned)nf, threads, smem, stm>>>(F, Dp, S.lev_sn + S.h_lev_ptr[l], S.sn_ptr, S.row_ptr,
                                                               S.front_off, S.dsign, S.small_max, dyn_eps, dyn_delta,
                                                               dyn_hits, skip);
    }
    if (!S.lev_big[l].empty()) {
      // FP64: the table with the split chain task; FP32: the fused one
      const bool f64 = sizeof(T) == 8;
      const FlowTask* tab = f64 ? S.flow_task64 : S.flow_task;
      const int64_t ft0 = f64 ? S.flow_t0_64[l] : S.flow_t0[l], fnt = f64 ? S.flow_nt_64[l] : S.flow_nt[l];
      const bool one = f64 ? S.flow_one64[l] != 0 : S.flow_one[l] != 0;
      int rc = use_flow ? BigFrontOps<T>::flow_level(stm, S.bfd, tab, ft0, fnt, flow_state,
                                                     S.flow_head[l], S.flow_soff,
                                                     one ? flow_sms : flow_sms * flow_occ, one,
                                                     F, E, Dp, S.dsign, dyn_eps, dyn_delta, dyn_hits, tc_err, skip,
                                                     (use_flow_tc() && tcs.pk && (S.flow_tc[l] || flow_tc == 2)) ? &tcs : nullptr)
                        : BigFrontOps<T>::factor_level(stm, S.bfd, S.bplans[l], F, E, Dp, Linv, S.dsign, dyn_eps,
                                                       dyn_delta, dyn_hits, skip, tc16, tc_err);
      if (rc) return rc;
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
    if ((int64_t)S.lev_big[l].size() < nf)
      k_fwd_front<T><<<(unsigned)nf, 256, 0, stm>>>(F, w, S.lev_sn + S.h_lev_ptr[l], S.sn_ptr, S.row_ptr,
                                                     S.front_off, S.upd_off, S.small_max, skip);
    if (!S.lev_big[l].empty()) {
      int rc = BigFrontOps<T>::fwd(stm, S.bfd, S.bplans[l].fwd, E, Dp, w, ybuf, skip);
      if (rc) return rc;
    }
  }
  for (int64_t l = S.nlev - 1; l >= 0; --l) {
    const int64_t nf = S.h_lev_ptr[l + 1] - S.h_lev_ptr[l];
    if ((int64_t)S.lev_big[l].size() < nf)
      k_bwd_front<T><<<(unsigned)nf, 256, 0, stm>>>(F, Dp, w, xs, S.lev_sn + S.h_lev_ptr[l], S.sn_ptr, S.row_ptr,
                                                    S.front_off, S.upd_off, S.rows_kkt, S.small_max, skip);
    if (!S.lev_big[l].empty()) {
      int rc = BigFrontOps<T>::bwd(stm, S.bfd, S.bplans[l].bwd, E, Dp, ybuf, xs, S.rows_kkt, skip);
      if (rc) return rc;
    }
  }
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

template struct LdlFactor<double>;
template struct LdlFactor<float>;

}  // namespace clr
