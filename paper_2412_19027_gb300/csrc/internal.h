// Internal data structures of the solver library (host side).
//
// Numbering used throughout:
//   KKT index i in [0, N), N = n + m:  i < n is x_i, i = n + r is constraint
//   row r of the REORDERED constraint block (zero, nonneg, SOC, exp, pow, PSD;
//   Sec. 3.3 and 3.5 of the paper), then the auxiliary rows of the expanded
//   SOCs (two per cone, p then q; no caller row, empty A row, b = 0, s = z = 0
//   throughout; their KKT rows carry the low-rank part of the cone's H).  The
//   KKT matrix is Eq. linsys_2x2: K = [P A^T; A -H].
//   Elimination position k in [0, N): perm[k] = KKT index eliminated k-th.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/clr.h"
#include "scal.cuh"

namespace clr {

enum Family { F_ZERO = 0, F_NONNEG = 1, F_SOC = 2, F_EXP = 3, F_POW = 4, F_PSD = 5 };

struct Cone {
  int type;
  int64_t dim;
  double alpha;
  int64_t off;    // first reordered constraint row
  int64_t kbase;  // offset of its packed lower H block in the z part of kval
  int64_t aux = -1;  // expanded SOC: its first auxiliary row (q = aux + 1); its z columns then
                     // hold 3 values each (diagonal -eta^2, eta u_i, eta v_i) from kbase on
};

// Compressed sparse row (or column) matrix with int64 pointers.
struct Sparse {
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> idx;
  std::vector<double> val;
  int64_t nnz() const { return (int64_t)idx.size(); }
};

// Reordered, merged cone list and family ranges.
struct ConeLayout {
  std::vector<Cone> cones;  // merged, in row order
  int64_t m_zero = 0, m_nonneg = 0;
  int64_t soc_begin = 0, soc_end = 0;  // cone index range in `cones`
  int64_t exp_begin = 0, exp_end = 0;
  int64_t pow_begin = 0, pow_end = 0;
  int64_t psd_begin = 0, psd_end = 0;
  int psd_k = 0;  // largest PSD order (cones of different orders are allowed)
  int64_t nu = 0;            // barrier degree of K
  int64_t soc_max_dim = 0;
  int64_t kval_z = 0;        // entries of the z part of kval
  bool symmetric_only = true;
  int64_t aux_begin = 0, n_aux = 0;  // auxiliary rows of the expanded SOCs: [aux_begin, aux_begin + n_aux),
                                     // the last rows; p rows at even offsets (KKT diagonal +1), q rows -1
};

// Symbolic supernodal factorization of the permuted KKT matrix.
struct Symbolic {
  int64_t N = 0;
  std::vector<int64_t> perm, iperm;        // elimination order
  int64_t n_dense = 0;
  // supernodes (in postorder: children before parents)
  int64_t nsn = 0;
  std::vector<int64_t> sn_ptr;             // columns (positions) of supernode J
  std::vector<int64_t> sn_parent;
  std::vector<int64_t> row_ptr;            // rows of front J (positions), own columns first
  std::vector<int64_t> rows;
  std::vector<int64_t> front_off;          // offset of front J in the pool (f_J^2 entries)
  int64_t pool = 0;
  std::vector<int64_t> upd_off;            // offset of J's update vector (r_J entries) for the solve
  int64_t upd_total = 0;
  // level schedule (level 0 = leaves)
  int64_t nlev = 0;
  std::vector<int64_t> lev_ptr, lev_sn;    // supernodes of each level
  // statistics
  int64_t l_nnz = 0;        // entries of L as stored (explicit zeros of merged supernodes included)
  int64_t l_nnz_exact = 0;  // entries of the exact factor pattern
  double flops = 0;         // flops of the exact factor (algorithmic)
  double flops_stored = 0;  // flops the supernodal factorization performs (explicit zeros included)
  int ordering = 0;         // 0 AMD, 1 cone rows first, -1 given by the caller
  int64_t pred_nnz = 0;     // nnz(L) and flops from column counts of the order (equal to the above)
  double pred_flops = 0;
  int64_t max_front = 0;
};

struct HostProblem {
  int64_t n = 0, m = 0;
  ConeLayout cl;
  std::vector<int64_t> row_perm;  // reordered row r = caller row row_perm[r]
  // unscaled reordered data (for norms and for q/b updates)
  Sparse P_full_u;   // unused after scaling, kept empty
  // scaled data
  Sparse Pf;         // full symmetric P (CSR == CSC), scaled
  Sparse A;          // CSR m x n, scaled
  Sparse At;         // CSR n x m, scaled (CSC of A)
  std::vector<double> q, b;        // scaled
  std::vector<double> D, E;        // equilibration
  double c = 1.0;
  double bnorm = 0, qnorm = 0;     // unscaled infinity norms
  double maxPdiag = 0;             // max |P_ii| (scaled)
  // KKT lower-triangle values kval: x columns (P lower, A column), then z blocks
  std::vector<double> kval;        // constant part filled (P, A, zero-cone H = 0)
  std::vector<int64_t> kcol_ptr;   // CSC of the lower triangle of K (KKT indices)
  std::vector<int64_t> krow;       // row KKT index of each kval entry
  std::vector<int64_t> kdiag;      // kval index of the diagonal of each KKT column
  int64_t kval_x = 0;              // entries of the x part of kval
  // value updates of P and A (clr_update_PA): for each stored value of the
  // caller's P (upper triangle) and A, in their CSC order, its kval index (x
  // part of this problem) and equilibration factor (c D_i D_j for P, E_r D_j
  // for A); the caller indices of P's diagonal entries; the offset of this
  // problem's x part in the cohort's kval (set by build_cohort)
  int64_t nnzP = 0, nnzA = 0;
  std::vector<int64_t> p_kv, a_kv, p_diag;
  std::vector<double> p_scale, a_scale;
  int64_t kx_off = 0;
};

// Where the problems of a cohort live in the merged vectors (host side).
struct CohortLayout {
  int64_t B = 1;
  std::vector<int64_t> xo;                 // B + 1: x_p = x[xo[p] .. xo[p+1])
  std::vector<std::vector<int64_t>> zrow;  // per problem: its reordered row r -> cohort row
  std::vector<Chunk> ckx, ckz;             // chunk lists; a problem's chunks are contiguous
  std::vector<int64_t> ckx_ptr, ckz_ptr;   // B + 1
  std::vector<int32_t> pid;                // KKT index -> problem (N)
  std::vector<ProbConst> pc;
};

// Merge the problems (each already through build_problem and with its own
// fill-reducing order `orders[p]`, or none) into one cohort problem `hp` and
// its symbolic factorization.  The big per-problem arrays are released.
int build_cohort(std::vector<HostProblem>& probs, const std::vector<std::vector<int64_t>>& orders, HostProblem& hp,
                 CohortLayout& lay, Symbolic& sy, std::string& err, int verbose = 0, int relax = 1);

// ---- host routines (setup.cpp / amd.cpp / symbolic.cpp) ----
int build_problem(HostProblem& hp, const clr_csc* P, const double* q, const clr_csc* A, const double* b,
                  const clr_cone* cones, int32_t ncones, const clr_settings& st, std::string& err);
int set_qb(HostProblem& hp, const double* q, const double* b);
// New values of P (upper, nnzP entries) and/or A (nnzA entries) in the caller's
// CSC order (either may be NULL): written, scaled by the setup's equilibration,
// into kval (at kx_off + the problem's index); maxPdiag updated.
int set_PA(HostProblem& pr, const double* Px, const double* Ax, std::vector<double>& kval);
void amd_order(int64_t N, const std::vector<int64_t>& ptr, const std::vector<int64_t>& idx,
               std::vector<int64_t>& perm, int64_t& n_dense);
// relax: merge supernodes with few explicit zeros (relaxed amalgamation):
// 0 off, 1 column thresholds 4 / 16 / 48, 2 thresholds 8 / 32 / 96.
int symbolic_analyze(int64_t N, const std::vector<int64_t>& colptr, const std::vector<int64_t>& rowidx,
                     const std::vector<int64_t>* user_order, Symbolic& sy, int relax = 1);
// The fill-reducing order symbolic_analyze uses when given none (AMD on the KKT pattern).
void kkt_amd_order(int64_t N, const std::vector<int64_t>& colptr, const std::vector<int64_t>& rowidx,
                   std::vector<int64_t>& order, int64_t& n_dense);
// nnz(L) (diagonal included) and factor flops of the KKT pattern in `order`, from column counts.
void kkt_factor_counts(int64_t N, const std::vector<int64_t>& colptr, const std::vector<int64_t>& rowidx,
                       const std::vector<int64_t>& order, int64_t* nnz, double* flops);
// The order used for a problem: AMD, or cone rows first when that needs fewer flops
// (*which = 0 or 1).
int choose_kkt_order(const HostProblem& hp, std::vector<int64_t>& order, int64_t& n_dense, int* which);

}  // namespace clr
