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
