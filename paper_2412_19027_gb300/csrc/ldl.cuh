// Numeric supernodal (multifrontal) LDL^T of the quasi-definite KKT matrix
// and its level-scheduled triangular solves (Sec. 3.6 of the paper, Alg. 1
// steps 5, 6 and 9).  T is the factor precision (double or float).
#pragma once

#include <vector>

#include "bigfront.cuh"
#include "device.cuh"
#include "internal.h"
#include "scal.cuh"
#include "symbolic.h"

namespace clr {

// Device arrays of the symbolic structure and the index maps (shared by the
// FP64 and FP32 factors).
struct LdlStructure {
  int64_t N = 0, nsn = 0, nlev = 0, pool = 0, wtot = 0, nk = 0;
  int64_t *sn_ptr = nullptr, *row_ptr = nullptr, *front_off = nullptr, *upd_off = nullptr, *lev_sn = nullptr;
  int32_t* rows_kkt = nullptr;
  int32_t* w_init = nullptr;   // solve slot -> KKT index of the right-hand side, or -1
  int8_t* dsign = nullptr;     // expected pivot sign by position
  int32_t* pos_pid = nullptr;  // problem of each elimination position (cohorts)
  int64_t *kdest = nullptr, *diag_pos = nullptr;
  int64_t *fa_tgt = nullptr, *fa_ptr = nullptr, *fa_src = nullptr;
  int64_t *sv_tgt = nullptr, *sv_ptr = nullptr, *sv_src = nullptr;
  // host copies used to configure launches
  std::vector<int64_t> h_lev_ptr, h_lev_sn, h_fa_lev_ptr, h_sv_lev_ptr;
  std::vector<int64_t> h_sn_ptr, h_row_ptr, h_front_off;
  std::vector<int> lev_small_maxf;               // largest small front of each level
  std::vector<std::vector<int64_t>> lev_big;     // big fronts of each level
  BigFrontDev bfd;                               // big-front arrays (device)
  std::vector<BigLevelPlan> bplans;              // per level
  // extend-add by relative indices: per level, the rounds' work lists (children
  // and prefix sums of their 32 x 32 tile counts)
  int32_t* rel = nullptr;
  int64_t* rel_off = nullptr;
  int64_t* sn_parent = nullptr;
  std::vector<std::vector<WorkList>> push_rounds;
  // dataflow factorization of the big fronts: task table (device), per level
  // its task range and the offset of its task counter in the state words;
  // per big-front id the offset of its version words
  FlowTask* flow_task = nullptr;
  int64_t* flow_soff = nullptr;
  std::vector<int64_t> flow_t0, flow_nt, flow_head;
  std::vector<int8_t> flow_one;  // per level: launch one CTA per SM (else two)
  std::vector<int8_t> flow_tc;   // per level: FP32 factors use the tensor-core launch
  // the FP64 factor's task table (the fused chain task split, bigfront.cuh), per level
  FlowTask* flow_task64 = nullptr;
  std::vector<int64_t> flow_t0_64, flow_nt_64;
  std::vector<int8_t> flow_one64;
  int64_t flow_words = 0;
  int64_t pk_tiles = 0;  // packed operand tiles of the largest level (tensor-core flow, FP32 factor)
  int small_max = 0;
  int64_t max_front = 0;
};

// pos_pid: problem of each elimination position (null: one problem).
int ldl_structure_upload(DeviceArena& ar, const Symbolic& sy, const NumericMaps& mp, const std::vector<int8_t>& dsign,
                         int small_max, LdlStructure& st, const std::vector<int32_t>* pos_pid = nullptr);

template <typename T>
struct LdlFactor {
  const LdlStructure* s = nullptr;
  T* F = nullptr;   // frontal-matrix pool
  T* Dp = nullptr;  // pivots by elimination position
  T* w = nullptr;   // forward-solve slots
  T* xs = nullptr;  // solution in KKT order
  T* E = nullptr;     // augmented inverse blocks of the big fronts
  T* ybuf = nullptr;  // forward results of the big fronts
  T* Linv = nullptr;  // per big front, two 64 x 64 diagonal-block inverses
  int* dyn_hits = nullptr;
  int* tc_err = nullptr;  // set if a wait of the big-front kernels ran out (the factor is unusable)
  bool tc16 = false;      // big-front updates with BF16 products on the tensor cores (float only)
  bool flow = true;       // big fronts by the dataflow kernel (one launch per level); else per-panel launches
  int flow_tc = 1;        // FP32 dataflow, trailing and E updates on the tensor cores (TF32 hi/lo parts):
                          // 0 never, 1 on the levels whose simulated schedule is shorter that way, 2 always
  FlowTc tcs;             // its packed operand tiles and their tensor map (allocated when used)
  int* flow_state = nullptr;
  int flow_sms = 0, flow_occ = 0;  // SMs of the device, resident flow CTAs per SM
  int alloc(DeviceArena& ar, const LdlStructure& st);
  // the FP32 dataflow factorization with tensor-core updates is in use
  bool use_flow_tc() const { return sizeof(T) == 4 && flow && flow_tc != 0 && !tc16 && s && s->pk_tiles > 0; }
  // Factor K: kval (FP64, lower triangle entries in kval order) scattered into
  // the fronts, +/- delta added on the diagonal (x rows +, z rows -), with
  // delta = sc[p].delta of the position's problem p.
  int factor(cudaStream_t st, const double* kval, const IterScal* sc, double dyn_eps, double dyn_delta,
             const int* skip) const;
  // xs = (L D L^T)^{-1} rhs (rhs FP64 in KKT order).
  int solve(cudaStream_t st, const double* rhs, const int* skip) const;
};

}  // namespace clr
