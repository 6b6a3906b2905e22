// Dataflow factorization of the big fronts of one level: one persistent launch
// in which CTAs take 64 x 64 tile tasks from a counter in a topological order
// of the task graph and wait (bounded) for the version words of the tiles they
// read.  The arithmetic of each task is that of the per-panel kernels
// (bigfront.cu); only the scheduling differs: the diagonal block of panel p + 1
// starts as soon as its own tile has received panel p's update, while the rest
// of panel p's updates are still running.
#include "bfdiag.cuh"
#include "bigfront.cuh"

namespace clr {
namespace {
constexpr int NB = kBfNB;
constexpr int LD = NB + 1;   // odd stride: column accesses free of bank conflicts
constexpr int LDK = NB + 4;  // 16-byte aligned rows of the K-major operand tiles
constexpr int NT = kFlowThreads;
constexpr uint32_t kSpin = 1u << 21;  // polls of one wait (about 2 s) before it gives up

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait until *p >= v.  False if the wait ran out (err := 2) or another
// CTA has given up (err != 0).
__device__ bool wait_ge(const int* p, int v, int* err) {
  for (uint32_t it = 0; it < kSpin; ++it) {
    if (ld_acquire(p) >= v) return true;
    if (it >= 16) {
      if (ld_acquire(err) != 0) return false;
      __nanosleep(64);
    }
  }
  atomicExch(err, 2);
  return false;
}

struct Geo {
  int64_t f, c, P, nbf;
};
__device__ __forceinline__ int64_t brow0(const Geo& g, int64_t b) { return b < g.P ? NB * b : g.c + NB * (b - g.P); }
__device__ __forceinline__ int bnrow(const Geo& g, int64_t b) {
  return (int)(b < g.P ? min((int64_t)NB, g.c - NB * b) : min((int64_t)NB, g.f - g.c - NB * (b - g.P)));
}
struct Words {
  int *tile, *etile, *diag, *trsm;
  int64_t P;
  __device__ int* t(int64_t i, int64_t j) const { return tile + i * (i + 1) / 2 + j; }
  __device__ int* e(int64_t i, int64_t c) const { return etile + i * P + c; }
};
__device__ __forceinline__ Words words_of(int* base, const Geo& g) {
  Words w;
  w.P = g.P;
  w.tile = base;
  w.etile = base + g.nbf * (g.nbf + 1) / 2;
  w.diag = w.etile + g.nbf * g.P;
  w.trsm = w.diag + g.P;
  return w;
}

// element r of K-row k of a K-major operand tile: 4-element units XOR-swizzled by k
__device__ __forceinline__ int swz(int k, int r) { return k * LDK + (((r >> 2) ^ (k & 7)) << 2) + (r & 3); }
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// D(p): LDL^T of the pw x pw diagonal block with dynamic regularisation (see
// bfdiag.cuh); L and the pivots written back, Linv = L_KK^{-1} written into
// E_KK, which it equals (the zeros above its diagonal are the E pool's).
template <typename T>
__device__ void task_diag(const BigFrontDev& bf, int64_t b, const Geo& g, int p, T* F, T* E, T* Dp,
                          const int8_t* dsign, T eps, T delta, int* hits, T* sm, DiagScratch<T>& sh) {
  const int64_t f = g.f, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);
  const int64_t kp = bf.k0pos[b] + k0;
  T* G = F + bf.goff[b] + k0 + k0 * f;
  T* Li = E + bf.eoff[b] + k0 + k0 * f;
  const int nhit = bf_diag_block<T>(G, f, pw, Dp + kp, Li, f, false, dsign + kp, eps, delta, sm, sh);
  if (threadIdx.x == 0 && nhit) atomicAdd(hits, nhit);
}

// DX(p), 1 <= p < P: the three links of the critical chain in one task, kept in
// shared memory between them -- the panel row T(p-1, p) (its L rows stored and
// published through the trsm word of block p as soon as they are written), the
// update of the diagonal tile (p, p) by panel p-1, and D(p).  Same arithmetic,
// in the same order, as the three separate tasks.
template <typename T>
__device__ int task_dx(const BigFrontDev& bf, int64_t b, const Geo& g, int p, T* F, T* E, T* Dp, const int8_t* dsign,
                       T eps, T delta, T* sm, DiagScratch<T>& sh, T* dl, int* trsm_word) {
  T* Bk = sm;                // K-major Linv of panel p - 1 (row j, k = l); work space of the factorization afterwards
  T* Xk = sm + NB * LDK;     // K-major F_{p,p-1} (row i, k = l), then L_{p,p-1}
  T* A = sm + 2 * NB * LDK;  // the diagonal tile (p, p), lower triangle, row stride LD
  const int64_t f = g.f, kq = (int64_t)(p - 1) * NB, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);  // panel p - 1 is a full 64-column panel (p - 1 < P - 1)
  T* G = F + bf.goff[b];
  T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
  {  // all loads in one batch, then into shared memory
    T ra[16], rb[16], rc[16];
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      ra[it] = __ldcg(Eb + (kq + i) + (kq + l) * f);
      rb[it] = (i < pw) ? __ldcg(G + (k0 + i) + (kq + l) * f) : (T)0;
      rc[it] = (i < pw && l < pw && i >= l) ? __ldcg(G + (k0 + i) + (k0 + l) * f) : (T)0;
    }
    if (tid < NB) dl[tid] = __ldcg(Dp + bf.k0pos[b] + kq + tid);
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      Bk[swz(l, i)] = ra[it];
      Xk[swz(l, i)] = rb[it];
      A[i * LD + l] = rc[it];
    }
  }
  __syncthreads();
  const int tr = tid % 16, tc = tid / 16;  // rows 4 tr .. 4 tr + 3, columns 4 tc .. 4 tc + 3
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  for (int l = 0; l < NB; ++l) {
    T av[4], bv[4];
    ld4<T>(Xk + swz(l, 4 * tr), av);
    ld4<T>(Bk + swz(l, 4 * tc), bv);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
  __syncthreads();  // every thread has read F_{p,p-1}
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    const int j = 4 * tc + bb;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = 4 * tr + a;
      Xk[swz(j, i)] = (i < pw) ? acc[a][bb] / dl[j] : (T)0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int idx = tid; idx < NB * NB; idx += NT) {
    const int i = idx % NB, j = idx / NB;
    if (i < pw) G[(k0 + i) + (kq + j) * f] = Xk[swz(j, i)];
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    st_release(trsm_word, p);
  }
  // A_ij -= sum_l L_il (L_jl d_l), i >= j
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  for (int l = 0; l < NB; ++l) {
    T av[4], bv[4];
    ld4<T>(Xk + swz(l, 4 * tr), av);
    ld4<T>(Xk + swz(l, 4 * tc), bv);
    const T dlv = dl[l];
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) bv[bb] *= dlv;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    const int j = 4 * tc + bb;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = 4 * tr + a;
      if (i < pw && i >= j) A[i * LD + j] -= acc[a][bb];
    }
  }
  __syncthreads();
  const int64_t kp = bf.k0pos[b] + k0;
  return bf_diag_factor<T>(A, Bk, G + k0 + k0 * f, f, pw, Dp + kp, Eb + k0 + k0 * f, f, false, dsign + kp, eps, delta,
                           sh);
}

// T(p, i): L_IK = F_IK Linv^T D_K^{-1} for the rows of block i (each thread 4 x 4).
template <typename T>
__device__ void task_trsm(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int64_t bi, T* F, const T* E,
                          const T* Dp, T* sm, T* dl) {
  T* Bk = sm;             // K-major Linv (row j, k = l)
  T* Xk = sm + NB * LDK;  // K-major F_IK (row i, k = l), then L_IK (row i, k = j)
  const int64_t f = g.f, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);
  const int64_t r0 = brow0(g, bi);
  const int nr = bnrow(g, bi);
  T* G = F + bf.goff[b];
  const T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
  {  // all loads in one batch, then into shared memory
    T ra[16], rb[16];
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      ra[it] = (i < pw && l < pw) ? __ldcg(Eb + (k0 + i) + (k0 + l) * f) : (T)0;
      rb[it] = (i < nr && l < pw) ? __ldcg(G + (r0 + i) + (k0 + l) * f) : (T)0;
    }
    if (tid < pw) dl[tid] = __ldcg(Dp + bf.k0pos[b] + k0 + tid);
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int idx = tid + NT * it;
      const int i = idx % NB, l = idx / NB;
      Bk[swz(l, i)] = ra[it];
      Xk[swz(l, i)] = rb[it];
    }
  }
  __syncthreads();
  const int tr = tid % 16, tc = tid / 16;  // rows 4 tr .. 4 tr + 3, columns 4 tc .. 4 tc + 3
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  for (int l = 0; l < pw; ++l) {
    T av[4], bv[4];
    ld4<T>(Xk + swz(l, 4 * tr), av);
    ld4<T>(Bk + swz(l, 4 * tc), bv);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
  __syncthreads();  // every thread has read F_IK
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    const int j = 4 * tc + bb;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = 4 * tr + a;
      if (j < pw) Xk[swz(j, i)] = acc[a][bb] / dl[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int idx = tid; idx < NB * NB; idx += NT) {
    const int i = idx % NB, j = idx / NB;
    if (i < nr && j < pw) G[(r0 + i) + (k0 + j) * f] = Xk[swz(j, i)];
  }
}

// Efin(p, e): E_KC <- Linv E_KC for the E rows of panel p and column block e < p.
template <typename T>
__device__ void task_efin(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int64_t e, T* E, T* sm) {
  T* Ls = sm;
  T* Xs = sm + NB * LD;
  const int64_t f = g.f, k0 = (int64_t)p * NB, cb = (int64_t)e * NB;
  const int pw = bnrow(g, p);
  T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
#pragma unroll
  for (int idx = tid; idx < NB * NB; idx += NT) {
    const int i = idx % NB, j = idx / NB;
    Ls[i * LD + j] = (i < pw && j < pw) ? __ldcg(Eb + (k0 + i) + (k0 + j) * f) : (T)0;
    Xs[i * LD + j] = (i < pw) ? __ldcg(Eb + (k0 + i) + (cb + j) * f) : (T)0;
  }
  __syncthreads();
  const int tr = tid % 16, tc = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  for (int l = 0; l < pw; ++l) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = Ls[(tr + 16 * a) * LD + l];
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) bv[bb] = Xs[l * LD + tc + 16 * bb];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = tr + 16 * a;
    if (i >= pw) continue;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) Eb[(k0 + i) + (cb + tc + 16 * bb) * f] = acc[a][bb];
  }
}

// U(p, i, j): F_IJ -= L_IK (D_K L_JK^T) (lower part only on a diagonal tile);
// EU(p, i, e): E_IC -= L_IK E_KC.  4 x 4 outputs per thread from K-major tiles.
template <typename T>
__device__ void task_update(const BigFrontDev& bf, int64_t b, const Geo& g, int p, int64_t bi, int64_t bj,
                            bool etile, T* F, T* E, const T* Dp, T* sm, T* dl) {
  T* Ak = sm;
  T* Bk = sm + NB * LDK;
  const int64_t f = g.f, k0 = (int64_t)p * NB;
  const int pw = bnrow(g, p);
  const int64_t i0 = brow0(g, bi);
  const int ni = bnrow(g, bi);
  T* G = F + bf.goff[b];
  T* Eb = E + bf.eoff[b];
  const int tid = threadIdx.x;
  const int64_t c0 = etile ? bj * NB : brow0(g, bj);
  const int nc = bnrow(g, bj);
  const bool diag = !etile && bi == bj;
  T* base = etile ? Eb : G;
  const int tr = tid % 16, tc = tid / 16;  // rows 4 tr .. 4 tr + 3, columns 4 tc .. 4 tc + 3
  // every global load of the task in one batch: both operand tiles, the pivots
  // and this thread's 4 x 4 outputs of the target tile (its inputs are complete
  // once the task runs), so the task pays one round trip to L2
  T ra[16], rb[16], tv[4][4];
#pragma unroll
  for (int it = 0; it < 16; ++it) {
    const int idx = tid + NT * it;
    const int r = idx % NB, k = idx / NB;
    ra[it] = (k < pw && r < ni) ? __ldcg(G + (i0 + r) + (k0 + k) * f) : (T)0;
    if (!etile)
      rb[it] = (k < pw && r < nc) ? __ldcg(G + (c0 + r) + (k0 + k) * f) : (T)0;
    else  // E_KC: consecutive threads read consecutive rows k0 + kk of column c0 + cc
      rb[it] = (r < pw && k < nc) ? __ldcg(Eb + (k0 + r) + (c0 + k) * f) : (T)0;
  }
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    const int cc = 4 * tc + bb;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = 4 * tr + a;
      tv[a][bb] = (r < ni && cc < nc && (!diag || r >= cc)) ? __ldcg(base + (i0 + r) + (c0 + cc) * f) : (T)0;
    }
  }
  if (!etile && tid < NB) dl[tid] = tid < pw ? __ldcg(Dp + bf.k0pos[b] + k0 + tid) : (T)0;
  if (!etile) __syncthreads();
#pragma unroll
  for (int it = 0; it < 16; ++it) {
    const int idx = tid + NT * it;
    const int r = idx % NB, k = idx / NB;
    Ak[swz(k, r)] = ra[it];
    if (!etile)
      Bk[swz(k, r)] = rb[it] * dl[k];
    else
      Bk[swz(r, k)] = rb[it];
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) acc[a][bb] = (T)0;
  for (int k = 0; k < pw; ++k) {
    T av[4], bv[4];
    ld4<T>(Ak + swz(k, 4 * tr), av);
    ld4<T>(Bk + swz(k, 4 * tc), bv);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[a][bb] += av[a] * bv[bb];
  }
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    const int cc = 4 * tc + bb;
    if (cc >= nc) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = 4 * tr + a;
      if (r < ni && (!diag || r >= cc)) base[(i0 + r) + (c0 + cc) * f] = tv[a][bb] - acc[a][bb];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT, 2)
    k_bf_flow(BigFrontDev bf, const FlowTask* __restrict__ task, int64_t t0, int64_t nt, int* __restrict__ state,
              int64_t head_off, const int64_t* __restrict__ soff, T* F, T* E, T* Dp, const int8_t* __restrict__ dsign,
              double eps_d, double delta_d, int* hits, int* err, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ DiagScratch<T> dsh;
  __shared__ T dl[NB];
  __shared__ FlowTask s_task;
  __shared__ int s_go;
  int* head = state + head_off;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      // The next ticket is taken only once this CTA is free: a ticket reserved
      // while the current task still waits for its inputs would be held back
      // for the whole wait, although another CTA could run it at once.
      const int cur = atomicAdd(head, 1);
      int go = 0;
      if (cur < nt) {
        const FlowTask tk = task[t0 + cur];
        s_task = tk;
        const int64_t b = tk.bf;
        const Geo g{bf.f[b], bf.c[b], (bf.c[b] + NB - 1) / NB, flow_nbf(bf.f[b], bf.c[b])};
        const Words w = words_of(state + soff[b], g);
        const int p = tk.p;
        // the version words this task reads and the versions it needs
        const int* wp[3];
        int wv[3];
        int nw;
        switch (tk.kind) {
          case 0:
            wp[0] = w.t(p, p), wv[0] = p;
            nw = 1;
            break;
          case 5:
            wp[0] = w.diag + p - 1, wv[0] = 1;
            wp[1] = w.t(p, p - 1), wv[1] = p - 1;
            wp[2] = w.t(p, p), wv[2] = p - 1;
            nw = 3;
            break;
          case 1:
            wp[0] = w.diag + p, wv[0] = 1;
            wp[1] = w.t(tk.i, p), wv[1] = p;
            nw = 2;
            break;
          case 2:
            wp[0] = w.diag + p, wv[0] = 1;
            wp[1] = w.e(p, tk.j), wv[1] = p - tk.j;
            nw = 2;
            break;
          case 3:
            wp[0] = w.trsm + tk.i, wv[0] = p + 1;
            wp[1] = w.trsm + tk.j, wv[1] = p + 1;
            wp[2] = w.t(tk.i, tk.j), wv[2] = p;
            nw = 3;
            break;
          default:
            wp[0] = w.trsm + tk.i, wv[0] = p + 1;
            if (tk.j < p)
              wp[1] = w.e(p, tk.j), wv[1] = p - tk.j + 1;
            else
              wp[1] = w.diag + p, wv[1] = 1;
            wp[2] = w.e(tk.i, tk.j), wv[2] = p - tk.j;
            nw = 3;
            break;
        }
        // one round trip when the inputs are already there (the loads are issued
        // together; the fence below orders them before the task's reads), else
        // bounded waits word by word
        int got[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < nw) got[q] = ld_relaxed(wp[q]);
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < nw && got[q] < wv[q]) ok = ok && wait_ge(wp[q], wv[q], err);
        go = ok ? 1 : 0;
        if (ok) __threadfence();
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const FlowTask tk = s_task;
    const int64_t b = tk.bf;
    const Geo g{bf.f[b], bf.c[b], (bf.c[b] + NB - 1) / NB, flow_nbf(bf.f[b], bf.c[b])};
    switch (tk.kind) {
      case 0:
        task_diag<T>(bf, b, g, tk.p, F, E, Dp, dsign, (T)eps_d, (T)delta_d, hits, sm, dsh);
        break;
      case 5: {
        const Words w = words_of(state + soff[b], g);
        const int nhit = task_dx<T>(bf, b, g, tk.p, F, E, Dp, dsign, (T)eps_d, (T)delta_d, sm, dsh, dl, w.trsm + tk.p);
        if (tid == 0 && nhit) atomicAdd(hits, nhit);
        break;
      }
      case 1:
        task_trsm<T>(bf, b, g, tk.p, tk.i, F, E, Dp, sm, dl);
        break;
      case 2:
        task_efin<T>(bf, b, g, tk.p, tk.j, E, sm);
        break;
      case 3:
        task_update<T>(bf, b, g, tk.p, tk.i, tk.j, false, F, E, Dp, sm, dl);
        break;
      default:
        task_update<T>(bf, b, g, tk.p, tk.i, tk.j, true, F, E, Dp, sm, dl);
        break;
    }
    __syncthreads();
    if (tid == 0) {
      const Words w = words_of(state + soff[b], g);
      const int p = tk.p;
      __threadfence();
      switch (tk.kind) {
        case 0:
          st_release(w.diag + p, 1);
          break;
        case 5:
          st_release(w.t(p, p), p);
          st_release(w.diag + p, 1);
          break;
        case 1:
          st_release(w.trsm + tk.i, p + 1);
          break;
        case 2:
          st_release(w.e(p, tk.j), p - tk.j + 1);
          break;
        case 3:
          st_release(w.t(tk.i, tk.j), p + 1);
          break;
        default:
          st_release(w.e(tk.i, tk.j), p - tk.j + 1);
          break;
      }
    }
  }
}

template <typename T>
size_t flow_smem() {  // the fused chain task's three blocks; the others need less
  constexpr int n = 2 * NB * LDK + NB * LD;
  static_assert(n >= kDiagSmem && NB * LDK >= NB * kDiagLD && LD == kDiagLD, "shared memory of the flow tasks");
  return n * sizeof(T);
}
}  // namespace

// dynamic shared memory of a launch with one CTA per SM (more than half an SM's)
template <typename T>
size_t flow_smem_one() {
  return flow_smem<T>() > (size_t)120 * 1024 ? flow_smem<T>() : (size_t)120 * 1024;
}

template <typename T>
int BigFrontOps<T>::flow_occupancy() {
  CLR_CUDA(cudaFuncSetAttribute(k_bf_flow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)flow_smem_one<T>()));
  int n = 0;
  CLR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bf_flow<T>, NT, flow_smem<T>()));
  return n > 0 ? n : 1;
}

template <typename T>
int BigFrontOps<T>::flow_level(cudaStream_t st, const BigFrontDev& bf, const FlowTask* task, int64_t t0, int64_t nt,
                               int* state, int64_t head_off, const int64_t* soff, int grid, bool one_per_sm, T* F,
                               T* E, T* Dp, const int8_t* dsign, double eps, double delta, int* hits, int* err,
                               const int* skip) {
  if (nt <= 0) return CLR_OK;
  const unsigned g = (unsigned)(nt < grid ? nt : grid);
  const size_t smem = one_per_sm ? flow_smem_one<T>() : flow_smem<T>();
  k_bf_flow<T><<<g, NT, smem, st>>>(bf, task, t0, nt, state, head_off, soff, F, E, Dp, dsign, eps, delta, hits, err,
                                    skip);
  CLR_CHECK_LAUNCH();
  return CLR_OK;
}

#define CLR_FLOW_INST(T)                                                                                         \
  template int BigFrontOps<T>::flow_occupancy();                                                                   \
  template int BigFrontOps<T>::flow_level(cudaStream_t, const BigFrontDev&, const FlowTask*, int64_t, int64_t, int*, \
                                          int64_t, const int64_t*, int, bool, T*, T*, T*, const int8_t*, double,     \
                                          double,                                                                    \
                                          int*, int*, const int*);
CLR_FLOW_INST(double)
CLR_FLOW_INST(float)
#undef CLR_FLOW_INST

}  // namespace clr
