// Cone kernels of the per-iteration device step (Alg. 1 steps 4, 7, 8, 10 of
// the paper): scaling H written into the KKT values, step lengths, and the
// combined-step d_s.  Families are handled as Sec. 3.3 proposes, mapped to
// GB300: zero/nonneg one flat pass, SOC a thread per cone up to 8 rows and a
// warp per cone above (shuffle reductions), exp/pow a thread per cone, PSD
// scaling a group of 4-16 lanes per cone up to order 16 (a lane per column) and a
// block per cone above, the other PSD kernels a block per cone.
#pragma once

#include <algorithm>
#include <vector>

#include "device.cuh"
#include "scal.cuh"

namespace clr {

// Device view of the reordered cone layout and the per-cone scaling data.
struct ConeDev {
  int64_t m = 0, m_zero = 0, m_nonneg = 0;
  // SOC cones: row offset, dimension, offset of the packed H block in kval
  int64_t n_soc = 0;
  const int64_t* soc_off = nullptr;
  const int32_t* soc_dim = nullptr;
  const int64_t* soc_kb = nullptr;
  // expanded SOCs (null: none): per cone its first auxiliary row, or -1 for a dense
  // block.  An expanded cone's kval holds 3 values per row from soc_kb on (the
  // diagonal -eta^2, then eta u_i and eta v_i in its two auxiliary rows); the
  // auxiliary rows [aux_begin, aux_begin + n_aux) are the last rows, their
  // diagonals (+1, -1 alternating) the last n_aux entries of kvz
  const int64_t* soc_aux = nullptr;
  int64_t aux_begin = 0, n_aux = 0;
  int soc_dmax = 0;  // largest SOC dimension
  // dense SOCs of at most 8 rows (a thread per cone; the others a warp per cone);
  // soc_split: both kinds are present, each kernel family skips the other's cones
  int64_t soc_nsmall = 0;
  int soc_split = 0;
  // exp / pow cones: rows row0 + 3 i, packed H at kb0 + 6 i
  int64_t n_exp = 0, exp_row0 = 0, exp_kb0 = 0;
  int64_t n_pow = 0, pow_row0 = 0, pow_kb0 = 0;
  const double* pow_alpha = nullptr;
  // PSD cones, of mixed orders k <= 32: per cone its order, first row, packed-H
  // offset in kvz and offset of its k x k blocks in psd_R / psd_Ri (its k entries
  // of psd_lam at psd_cl); psd_row0 = the first PSD row, psd_kmax = the largest k
  int64_t n_psd = 0, psd_row0 = 0;
  int psd_kmax = 0;
  const int32_t* psd_ck = nullptr;
  const int64_t* psd_crow = nullptr;
  const int64_t* psd_ckb = nullptr;
  const int64_t* psd_cR = nullptr;
  const int64_t* psd_cl = nullptr;
  // PSD cones by scaling-kernel class: orders 1-4, 5-8 and 9-16 (psd_list[0..2]; a
  // group of 4, 8 or 16 lanes per cone, lane j holding column j) and 17-32
  // (psd_list[3]; a block per cone)
  const int32_t* psd_list[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t psd_nlist[4] = {0, 0, 0, 0};
  int64_t nn_kb = 0;  // packed offset of the first nonneg diagonal (after the zero cone)
  double* kvz = nullptr;  // z part of the KKT values (-H blocks)
  int64_t nkz = 0;        // number of entries of kvz
  double* scratch = nullptr;  // m doubles of work space for the SOC corrector
  // scaling data written by the scaling kernels
  double* nn_w = nullptr;     // sqrt(s/z) per nonneg row
  double* nn_lam = nullptr;   // sqrt(s z)
  double* soc_eta = nullptr;  // per SOC cone
  double* soc_wb = nullptr;   // w-bar, indexed by row (m entries, used on SOC rows)
  double* soc_lam = nullptr;  // lambda, indexed by row
  double* psd_R = nullptr;    // k*k per cone (column-major)
  double* psd_Ri = nullptr;   // R^{-1}
  double* psd_lam = nullptr;  // k per cone
  double* ep_zt = nullptr;   // 3 per exp/pow cone: z~ = -grad f*(s) at the current s (Newton warm start)
  double exp_center[3] = {0, 0, 0};  // central point of the exp cone (u = -grad f(u))
  // cohort: problem of every (reordered, family-major) row and per-problem constants
  int64_t nprob = 1;
  const int32_t* row_pid = nullptr;
  const ProbConst* pc = nullptr;
};

// Per-cone PSD data on the device from each PSD cone's svec dimension, first row
// and packed-H offset (in cone order); allocates psd_R, psd_Ri, psd_lam.  False
// on a dimension that is not k(k+1)/2 with k <= 32, or on allocation failure.
inline bool cones_psd_setup(DeviceArena& ar, ConeDev& cd, const std::vector<int64_t>& dims,
                            const std::vector<int64_t>& rows, const std::vector<int64_t>& kbs) {
  const int64_t n = (int64_t)dims.size();
  std::vector<int32_t> ck(n);
  std::vector<int64_t> cR(n), cl(n);
  int64_t nR = 0, nl = 0;
  int kmax = 0;
  for (int64_t i = 0; i < n; ++i) {
    int k = 0;
    while ((int64_t)(k + 1) * (k + 2) / 2 <= dims[i]) ++k;
    if ((int64_t)k * (k + 1) / 2 != dims[i] || k < 1 || k > 32) return false;
    ck[i] = k;
    cR[i] = nR;
    cl[i] = nl;
    nR += (int64_t)k * k;
    nl += k;
    kmax = std::max(kmax, k);
  }
  cd.n_psd = n;
  cd.psd_kmax = kmax;
  cd.psd_row0 = n ? rows[0] : 0;
  if (n == 0) return true;
  cd.psd_ck = ar.upload(ck.data(), n);
  cd.psd_crow = ar.upload(rows.data(), n);
  cd.psd_ckb = ar.upload(kbs.data(), n);
  cd.psd_cR = ar.upload(cR.data(), n);
  cd.psd_cl = ar.upload(cl.data(), n);
  cd.psd_R = ar.alloc_n<double>(nR);
  cd.psd_Ri = ar.alloc_n<double>(nR);
  cd.psd_lam = ar.alloc_n<double>(nl);
  std::vector<int32_t> lists[4];
  for (int64_t i = 0; i < n; ++i) lists[ck[i] <= 4 ? 0 : ck[i] <= 8 ? 1 : ck[i] <= 16 ? 2 : 3].push_back((int32_t)i);
  for (int c = 0; c < 4; ++c) {
    cd.psd_nlist[c] = (int64_t)lists[c].size();
    cd.psd_list[c] = nullptr;
    if (!lists[c].empty() && !(cd.psd_list[c] = ar.upload(lists[c].data(), cd.psd_nlist[c]))) return false;
  }
  return cd.psd_ck && cd.psd_crow && cd.psd_ckb && cd.psd_cR && cd.psd_cl && cd.psd_R && cd.psd_Ri && cd.psd_lam;
}

// Per-problem scalars are read from and written to sc[row_pid[row]]; `skip`
// (when non-null and set) makes every kernel return at once.

// Scaling H (-H into kvz) for every cone (exp/pow use the problem's mu); max |H_ii| of
// each problem into sc[p].hmax_bits (atomicMax on the bit pattern; caller zeroes it).
int cones_scaling(cudaStream_t st, const ConeDev& cd, const double* s, const double* z, IterScal* sc,
                  const int* skip);
// H = I on every cone block (initialisation solves), zero cone included.
int cones_identity_H(cudaStream_t st, const ConeDev& cd, const int* skip);
// Symmetric-cone step length over s/ds and z/dz -> atomicMin into sc[p].amin_bits.
int cones_step_symmetric(cudaStream_t st, const ConeDev& cd, const double* s, const double* ds, const double* z,
                         const double* dz, IterScal* sc, const int* skip);
// exp/pow backtracking from a0 = sc[p].alpha_sym (Sec. 2.2: ratio 0.8): the
// candidates are a_j = a0 backtrack^j.  Interior-ness is monotone along the
// ray, so the joint first interior candidate is the largest per-cone one
// (jint).  With nbhd != 0 the N(beta) test (trial mu from sc[p].mu_coef =
// {c0, c1, c2}: mu(a) = c0 + a c1 + a^2 c2) is evaluated at jint and, only if
// some cone of the problem fails there, on the 64 candidates after it; the
// step is the first candidate every cone of the problem passes.  Result in sc[p].ns.
int cones_step_nonsym(cudaStream_t st, const ConeDev& cd, const double* s, const double* ds, const double* z,
                      const double* dz, IterScal* sc, double backtrack, int nbhd, double beta, const int* skip);
// z~ of every exp/pow cone set to its central point (start of a solve).
int cones_init_shadow(cudaStream_t st, const ConeDev& cd, const int* skip);
// Combined-step d_s (Eq. ds-correction-step) for every cone, with the problem's sigma mu.
int cones_combined_ds(cudaStream_t st, const ConeDev& cd, const double* s, const double* z, const double* dsa,
                      const double* dza, IterScal* sc, double* ds_out, const int* skip);
// Delta s = -d_s - H Delta z on the PSD rows with H applied in factored form
// (R (R^T Delta Z R) R^T); overwrites those rows of ds_out (z-row indexing).
int cones_psd_ds_from_dz(cudaStream_t st, const ConeDev& cd, const double* dz, const double* dsrhs, double* ds_out,
                         const int* skip);
// Initial point shift (symmetric init): v += (1 - a) e where a = least Jordan eigenvalue < sqrt(eps).
// Zero-cone entries are set to 0; the merged nonneg cone of each problem shifts by its own
// minimum (sc[p].nn_min_bits is scratch).
int cones_shift_init(cudaStream_t st, const ConeDev& cd, double* v, IterScal* sc, const int* skip);
// Unit initialisation: v = central point of each cone (0 on the zero cone), on the rows of
// problems whose ProbConst::sym is 0 (problems with exp/pow cones); other rows untouched.
int cones_unit_init(cudaStream_t st, const ConeDev& cd, double* v, const int* skip);

__host__ double exp_central_point_host(double out[3]);

}  // namespace clr
