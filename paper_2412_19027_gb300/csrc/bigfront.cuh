// Large frontal matrices of the multifrontal LDL^T (fronts too big for one
// CTA's shared memory): blocked factorization in 64-column panels that also
// builds E = L^{-1} [I; 0] = [L11^{-1}; -L21 L11^{-1}], so that each triangular
// solve with the front is one matrix-vector product with E (forward) and one
// with E^T (backward), parallel over all rows / columns.
#pragma once

#include <vector>

#include "device.cuh"

namespace clr {

constexpr int kBfNB = 64;
constexpr int kTrsmRows = 64;  // rows of L21 per CTA of the panel kernel

// Device arrays indexed by big-front id.
struct BigFrontDev {
  int64_t n = 0;
  const int64_t* f = nullptr;     // front order
  const int64_t* c = nullptr;     // pivots
  const int64_t* goff = nullptr;  // front offset in the frontal pool (f x f, column-major)
  const int64_t* eoff = nullptr;  // offset of E (f x c, column-major) in the E pool
  const int64_t* k0pos = nullptr; // elimination position of the first pivot (pivot array offset)
  const int64_t* woff = nullptr;  // offset of the front's solve slots
  const int64_t* yoff = nullptr;  // offset of its forward result y (c entries)
  const int64_t* rk = nullptr;    // offset of its rows in rows_kkt
  const int64_t* pkoff = nullptr; // first packed operand tile of the front in its level's tiles (tensor-core flow)
  int64_t epool = 0, ypool = 0;
};

// CTAs of one launch: front ids and the prefix sum of their CTA counts.
struct WorkList {
  const int64_t* front = nullptr;
  const int64_t* pref = nullptr;
  int64_t nfront = 0, nblocks = 0;
};

// Host description of the big-front launches of one level.
struct BigLevelPlan {
  std::vector<WorkList> A, B, C;  // per panel step p (B/C may be empty lists)
  std::vector<WorkList> Ctc;      // C as 128 x 64 tensor-core tiles (16-bit products)
  WorkList fwd, bwd;
};

// ---------------------------------------------------------------------------
// Dataflow factorization of the big fronts of one level in ONE launch.
// A front with c pivots and f rows is cut into blocks of 64: P = ceil(c/64)
// pivot blocks [64b, min(64b+64, c)), then the update rows [c, f) in blocks of
// 64 from c, nbf blocks in all.  Tasks (64 x 64 tiles):
//   D(p)        diagonal block of panel p: LDL^T, pivots, Linv = L_KK^{-1}
//               (written into E_KK, which it equals); for 1 <= p < P the task
//               DX(p) does T(p-1, p), U(p-1, p, p) and D(p) in one, in shared memory;
//   T(p, i)     block row i > p of panel p: L_IK = F_IK Linv^T D_K^{-1};
//   Efin(p, e)  E rows of panel p, column block e < p: E_KC <- Linv E_KC;
//   U(p, i, j)  trailing tile i >= j > p: F_IJ -= L_IK D_K L_JK^T;
//   EU(p, i, e) E tile i > p, e <= p: E_IC -= L_IK E_KC.
// Persistent CTAs take tasks from one counter in a fixed topological order of
// the task graph (with the next panel's diagonal block ahead of the bulk of the
// current panel's updates); a task waits (bounded) on per-front version words
// set by the tasks it depends on.  Every task it waits on was taken earlier by a
// CTA that is running, so the launch needs no co-residency guarantee.
// FP64 factors split the fused chain task (an FP64 warp instruction holds a
// sub-partition's FP64 pipe ~64 cycles, so DX(p) alone takes ~200 us on one SM):
// for 1 <= p < P, TX(p, q) (q = 0..3: rows 16 q .. 16 q + 15 of T(p-1, p)), then
// UX(p, q) (four row slabs of equal area of the update of the diagonal tile (p, p)
// by panel p-1), then D(p).  The last part of TX(p) (of UX(p)) to finish releases
// the word the consumers of T(p-1, p) (of the tile) wait on.  Same arithmetic, in
// the same order, as DX(p).
struct FlowTask {
  int32_t bf;    // big-front id
  int16_t kind;  // 0 D, 1 T, 2 Efin, 3 U, 4 EU, 5 DX, 6 TX, 7 UX
  int16_t p;     // panel
  int32_t i, j;  // block row; block column (Efin: e; EU: e; TX, UX: the part q in i)
};
// version words of one front: tile[tri(i, j)], etile[i * P + e], diag[P], trsm[nbf],
// pe[P] (tensor-core flow: the packed E_KK tile of panel p is stored), txc[P] and
// uxc[P] (FP64 split chain: parts of TX(p) and UX(p) done)
__host__ __device__ inline int64_t flow_nbf(int64_t f, int64_t c) {
  return (c + kBfNB - 1) / kBfNB + (f - c + kBfNB - 1) / kBfNB;
}
__host__ __device__ inline int64_t flow_words(int64_t f, int64_t c) {
  const int64_t P = (c + kBfNB - 1) / kBfNB, n = flow_nbf(f, c);
  return n * (n + 1) / 2 + n * P + P + n + 3 * P;
}
constexpr int kFlowThreads = 256;

// Tensor-core products of the dataflow factorization (FP32 factor).  The tasks
// that produce an L tile (T, DX) or an E_KC tile (D, DX, Efin) also store it as
// a packed FP32 operand tile: 64 rows x 64 k in K-major core matrices of 8 rows
// x 16 bytes without swizzle (element (row, k) at word (k / 4) * 256 + row * 4
// + k % 4), the layout one TMA tensor copy lands in shared memory.  The U and EU
// tasks copy their two operand tiles into shared memory with TMA, split them
// there into high and low TF32 parts (the U task's B operand scaled by D_K on
// the way) and multiply them on the tensor cores with FP32 accumulation in
// tensor memory.  Per front (P pivot blocks, nbf blocks): PL(p, i), i > p
// (L_IK), then PE(p, e), e <= p (E_KC, stored with rows = the C columns).
constexpr int64_t kPkWords = kBfNB * kBfNB;  // floats of one packed tile (16 KB)
__host__ __device__ inline int64_t flow_pk_nl(int64_t f, int64_t c) {
  const int64_t P = (c + kBfNB - 1) / kBfNB, n = flow_nbf(f, c);
  return P * (n - 1) - P * (P - 1) / 2;
}
__host__ __device__ inline int64_t flow_pk_tiles(int64_t f, int64_t c) {
  const int64_t P = (c + kBfNB - 1) / kBfNB;
  return flow_pk_nl(f, c) + P * (P + 1) / 2;
}
// The packed tiles of one level and the TMA tensor map over them (a
// CUtensorMap, kept opaque here): rows of 256 floats, a tile is 16 rows.
struct FlowTc {
  float* pk = nullptr;
  int64_t tiles = 0;
  unsigned char tmap[128] = {};
};
// Host: encode the tensor map over tc->pk (tc->tiles packed tiles).  CLR_E_CUDA
// if the driver entry point is missing or rejects the map.
int flow_tc_encode(FlowTc* tc);

template <typename T>
struct BigFrontOps {
  static int setup_attributes();
  // tc16: trailing and E updates on the tensor cores with BF16 operands and FP32
  // accumulation (T = float only); err: set to 1 if a tensor-core wait ran out.
  static int factor_level(cudaStream_t st, const BigFrontDev& bf, const BigLevelPlan& plan, T* F, T* E, T* Dp,
                          T* Linv, const int8_t* dsign, double eps, double delta, int* hits, const int* skip,
                          bool tc16 = false, int* err = nullptr);
  static int fwd(cudaStream_t st, const BigFrontDev& bf, const WorkList& wl, const T* E, const T* Dp, T* w,
                 T* ybuf, const int* skip);
  static int bwd(cudaStream_t st, const BigFrontDev& bf, const WorkList& wl, const T* E, const T* Dp, const T* ybuf,
                 T* xs, const int32_t* rows_kkt, const int* skip);
  // Dataflow factorization of one level: tasks [t0, t0 + nt) of the task table;
  // state: zeroed words holding the level's task counter (at head_off) and, at
  // soff[b], the version words of each big front b of the level.  err: set to 2
  // if a wait ran out (the factor is then unusable).  one_per_sm: enough shared
  // memory is requested that a single CTA fits on an SM.
  // tc (T = float only; null: CUDA-core products): trailing and E updates on
  // the tensor cores from packed operand tiles (see FlowTc).
  static int flow_level(cudaStream_t st, const BigFrontDev& bf, const FlowTask* task, int64_t t0, int64_t nt,
                        int* state, int64_t head_off, const int64_t* soff, int grid, bool one_per_sm, T* F, T* E, T* Dp,
                        const int8_t* dsign, double eps, double delta, int* hits, int* err, const int* skip,
                        const FlowTc* tc = nullptr);
  static int flow_occupancy(bool tc = false);  // resident CTAs per SM of the flow kernel
};


// CTA counts per front used to build the plans (must match the kernels).
__host__ __device__ inline int64_t bf_trsm_blocks(int64_t f, int64_t c, int p) {
  const int64_t k0 = (int64_t)p * kBfNB;
  if (k0 >= c) return 0;
  const int64_t pw = (c - k0 < kBfNB) ? c - k0 : kBfNB;
  return (f - k0 - pw + kTrsmRows - 1) / kTrsmRows;
}
__host__ __device__ inline int64_t bf_fin_blocks(int64_t c, int p) {  // finalisation of the E rows of panel p (same launch)
  if (p < 0 || (int64_t)p * kBfNB >= c) return 0;
  return p + 1;
}
// 128 x 64 tensor-core tiles of panel p: trailing tiles (row block bi of 128,
// column block bj of 64, bi >= bj / 2 so that the tile meets the lower
// triangle) and E tiles (row blocks of 128 x the p + 1 column blocks of 64).
__host__ __device__ inline int64_t bf_tc_tiles(int64_t f, int64_t c, int p) {
  const int64_t k0 = (int64_t)p * kBfNB;
  if (k0 >= c) return 0;
  const int64_t pw = (c - k0 < kBfNB) ? c - k0 : kBfNB;
  const int64_t nr = f - k0 - pw;
  const int64_t n128 = (nr + 127) / 128, n64 = (nr + 63) / 64;
  int64_t t = 0;
  for (int64_t bj = 0; bj < n64; ++bj) t += n128 - bj / 2;
  return t + n128 * (p + 1);
}
__host__ __device__ inline int64_t bf_update_tiles(int64_t f, int64_t c, int p) {
  const int64_t k0 = (int64_t)p * kBfNB;
  if (k0 >= c) return 0;
  const int64_t pw = (c - k0 < kBfNB) ? c - k0 : kBfNB;
  const int64_t nt = (f - k0 - pw + kBfNB - 1) / kBfNB;
  return nt * (nt + 1) / 2 + nt * (p + 1);
}

}  // namespace clr
