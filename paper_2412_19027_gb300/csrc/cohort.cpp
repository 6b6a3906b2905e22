// Cohorts: B independent problems merged into one block-diagonal problem so
// that one pass of the per-iteration device step advances all of them.
//
// Layout of the merged problem:
//   x = [x_1; ...; x_B];
//   constraint rows family-major (zero, nonneg, SOC, exp, pow, PSD), each
//   family holding its rows of problem 1, then problem 2, ...; so the zero and
//   nonnegative rows of the whole cohort are one flat range and the cone lists
//   stay contiguous per family, as the cone kernels expect;
//   the KKT values in the column order of the merged KKT matrix.
// Each problem keeps its own equilibration, cost scaling and fill-reducing
// order (the merged order is the concatenation), so its supernodes, fronts
// and arithmetic are those it has alone.
#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <numeric>

#include "internal.h"

namespace clr {

namespace {

void chunk_run(std::vector<Chunk>& out, int64_t begin, int64_t len, int32_t pid) {
  for (int64_t o = 0; o < len; o += kChunk) out.push_back(Chunk{begin + o, (int32_t)std::min<int64_t>(kChunk, len - o), pid});
}

// rows of family f (0 zero, 1 nonneg, 2 SOC, 3 exp, 4 pow, 5 PSD) in a problem's reordered rows
void family_ranges(const HostProblem& p, int64_t start[7], int64_t size[7]) {
  const ConeLayout& cl = p.cl;
  auto rows_of = [&](int64_t c0, int64_t c1, int64_t* st, int64_t* sz) {
    *sz = 0;
    *st = (c0 < c1) ? cl.cones[c0].off : 0;
    for (int64_t c = c0; c < c1; ++c) *sz += cl.cones[c].dim;
  };
  start[0] = 0;
  size[0] = cl.m_zero;
  start[1] = cl.m_zero;
  size[1] = cl.m_nonneg;
  rows_of(cl.soc_begin, cl.soc_end, &start[2], &size[2]);
  rows_of(cl.exp_begin, cl.exp_end, &start[3], &size[3]);
  rows_of(cl.pow_begin, cl.pow_end, &start[4], &size[4]);
  rows_of(cl.psd_begin, cl.psd_end, &start[5], &size[5]);
  start[6] = cl.aux_begin;  // the auxiliary rows of the expanded SOCs
  size[6] = cl.n_aux;
}

void release_big(HostProblem& p) {
  std::vector<int64_t>().swap(p.Pf.ptr);
  std::vector<int32_t>().swap(p.Pf.idx);
  std::vector<double>().swap(p.Pf.val);
  std::vector<int64_t>().swap(p.A.ptr);
  std::vector<int32_t>().swap(p.A.idx);
  std::vector<double>().swap(p.A.val);
  std::vector<int64_t>().swap(p.At.ptr);
  std::vector<int32_t>().swap(p.At.idx);
  std::vector<double>().swap(p.At.val);
  std::vector<double>().swap(p.kval);
  std::vector<int64_t>().swap(p.kcol_ptr);
  std::vector<int64_t>().swap(p.krow);
  std::vector<int64_t>().swap(p.kdiag);
}

ProbConst prob_const(const HostProblem& p) {
  ProbConst c{};
  c.c = p.c;
  c.bnorm = p.bnorm;
  c.qnorm = p.qnorm;
  c.maxPdiag = p.maxPdiag;
  c.nu = p.cl.nu;
  c.sym = p.cl.symmetric_only ? 1 : 0;
  return c;
}

}  // namespace

int build_cohort(std::vector<HostProblem>& probs, const std::vector<std::vector<int64_t>>& orders, HostProblem& hp,
                 CohortLayout& lay, Symbolic& sy, std::string& err, int verbose, int relax) {
  const int64_t B = (int64_t)probs.size();
  if (B == 0) {
    err = "a cohort needs at least one problem";
    return CLR_E_INVALID;
  }
  if (!orders.empty() && (int64_t)orders.size() != B) {
    err = "one order per problem";
    return CLR_E_DIM;
  }
  int psd_k = 0;  // the largest PSD order (cones of every order <= 32 are handled per cone)
  for (const HostProblem& p : probs) psd_k = std::max(psd_k, p.cl.psd_k);
  lay = CohortLayout();
  lay.B = B;
  lay.pc.resize(B);
  lay.zrow.resize(B);
  lay.ckx_ptr.assign(B + 1, 0);
  lay.ckz_ptr.assign(B + 1, 0);

  if (B == 1) {
    // the cohort problem is the problem itself; the per-problem copy keeps the small arrays
    hp = std::move(probs[0]);
    HostProblem& p = probs[0];
    p = HostProblem();
    p.n = hp.n;
    p.m = hp.m;
    p.cl = hp.cl;
    p.row_perm = hp.row_perm;
    p.q = hp.q;
    p.b = hp.b;
    p.D = hp.D;
    p.E = hp.E;
    p.c = hp.c;
    p.bnorm = hp.bnorm;
    p.qnorm = hp.qnorm;
    p.maxPdiag = hp.maxPdiag;
    p.nnzP = hp.nnzP;
    p.nnzA = hp.nnzA;
    p.p_kv = std::move(hp.p_kv);
    p.a_kv = std::move(hp.a_kv);
    p.p_diag = std::move(hp.p_diag);
    p.p_scale = std::move(hp.p_scale);
    p.a_scale = std::move(hp.a_scale);
    p.kx_off = 0;
    const int64_t n = hp.n, m = hp.m, N = n + m;
    lay.xo = {0, n};
    lay.zrow[0].resize(m);
    std::iota(lay.zrow[0].begin(), lay.zrow[0].end(), 0);
    lay.pid.assign(N, 0);
    lay.pc[0] = prob_const(hp);
    chunk_run(lay.ckx, 0, n, 0);
    if (lay.ckx.empty()) lay.ckx.push_back(Chunk{0, 0, 0});
    int64_t fs[7], fz[7];
    family_ranges(hp, fs, fz);
    for (int f = 0; f < 7; ++f) chunk_run(lay.ckz, fs[f], fz[f], 0);
    if (lay.ckz.empty()) lay.ckz.push_back(Chunk{0, 0, 0});
    lay.ckx_ptr[1] = (int64_t)lay.ckx.size();
    lay.ckz_ptr[1] = (int64_t)lay.ckz.size();
    std::vector<int64_t> own;
    int64_t nd = 0;
    int which = 0;
    const std::vector<int64_t>* use = nullptr;
    if (!orders.empty() && !orders[0].empty()) {
      use = &orders[0];
      which = -1;
    } else {
      const auto t0 = std::chrono::steady_clock::now();
      choose_kkt_order(hp, own, nd, &which);
      if (verbose)
        std::fprintf(stderr, "[clr] setup: ordering %.3f s (%s)\n",
                     std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(),
                     which ? "cone rows first" : "AMD");
      use = &own;
    }
    const auto t1 = std::chrono::steady_clock::now();
    int rc = symbolic_analyze(N, hp.kcol_ptr, hp.krow, use, sy, relax);
    if (verbose)
      std::fprintf(stderr, "[clr] setup: symbolic %.3f s\n",
                   std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count());
    if (rc != CLR_OK) {
      err = "symbolic analysis failed";
      return rc;
    }
    sy.n_dense = nd;
    sy.ordering = which;
    kkt_factor_counts(N, hp.kcol_ptr, hp.krow, *use, &sy.pred_nnz, &sy.pred_flops);
    return CLR_OK;
  }

  // ---- x segments and family-major rows ----
  lay.xo.assign(B + 1, 0);
  for (int64_t p = 0; p < B; ++p) lay.xo[p + 1] = lay.xo[p] + probs[p].n;
  const int64_t n = lay.xo[B];
  constexpr int NF = 7;  // zero, nonneg, SOC, exp, pow, PSD, auxiliary rows
  std::vector<std::array<int64_t, NF>> fstart(B), fsize(B);
  int64_t ftot[NF] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t p = 0; p < B; ++p) {
    family_ranges(probs[p], fstart[p].data(), fsize[p].data());
    for (int f = 0; f < NF; ++f) ftot[f] += fsize[p][f];
  }
  int64_t cstart[NF + 1] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int f = 0; f < NF; ++f) cstart[f + 1] = cstart[f] + ftot[f];
  const int64_t m = cstart[NF];
  const int64_t N = n + m;
  std::vector<std::array<int64_t, NF>> pref(B);  // start of problem p's run inside family f
  {
    int64_t run[NF];
    for (int f = 0; f < NF; ++f) run[f] = cstart[f];
    for (int64_t p = 0; p < B; ++p)
      for (int f = 0; f < NF; ++f) {
        pref[p][f] = run[f];
        run[f] += fsize[p][f];
      }
  }
  std::vector<int32_t> zinv_p(m);
  std::vector<int64_t> zinv_r(m);
  for (int64_t p = 0; p < B; ++p) {
    lay.zrow[p].assign(probs[p].m, -1);
    for (int f = 0; f < NF; ++f)
      for (int64_t k = 0; k < fsize[p][f]; ++k) {
        const int64_t r = fstart[p][f] + k, R = pref[p][f] + k;
        lay.zrow[p][r] = R;
        zinv_p[R] = (int32_t)p;
        zinv_r[R] = r;
      }
  }
  lay.pid.assign(N, 0);
  for (int64_t p = 0; p < B; ++p) {
    for (int64_t j = lay.xo[p]; j < lay.xo[p + 1]; ++j) lay.pid[j] = (int32_t)p;
    for (int64_t R : lay.zrow[p]) lay.pid[n + R] = (int32_t)p;
    lay.pc[p] = prob_const(probs[p]);
  }
  // ---- chunks ----
  for (int64_t p = 0; p < B; ++p) {
    const size_t x0 = lay.ckx.size(), z0 = lay.ckz.size();
    chunk_run(lay.ckx, lay.xo[p], probs[p].n, (int32_t)p);
    if (lay.ckx.size() == x0) lay.ckx.push_back(Chunk{lay.xo[p], 0, (int32_t)p});
    for (int f = 0; f < NF; ++f) chunk_run(lay.ckz, pref[p][f], fsize[p][f], (int32_t)p);
    if (lay.ckz.size() == z0) lay.ckz.push_back(Chunk{0, 0, (int32_t)p});
    lay.ckx_ptr[p + 1] = (int64_t)lay.ckx.size();
    lay.ckz_ptr[p + 1] = (int64_t)lay.ckz.size();
  }
  // ---- merged problem: data vectors ----
  hp = HostProblem();
  hp.n = n;
  hp.m = m;
  hp.q.assign(n, 0.0);
  hp.D.assign(n, 1.0);
  hp.b.assign(m, 0.0);
  hp.E.assign(m, 1.0);
  hp.row_perm.resize(m);
  std::iota(hp.row_perm.begin(), hp.row_perm.end(), 0);
  for (int64_t p = 0; p < B; ++p) {
    const HostProblem& pr = probs[p];
    std::copy(pr.q.begin(), pr.q.end(), hp.q.begin() + lay.xo[p]);
    std::copy(pr.D.begin(), pr.D.end(), hp.D.begin() + lay.xo[p]);
    for (int64_t r = 0; r < pr.m; ++r) {
      hp.b[lay.zrow[p][r]] = pr.b[r];
      hp.E[lay.zrow[p][r]] = pr.E[r];
    }
    hp.maxPdiag = std::max(hp.maxPdiag, pr.maxPdiag);
  }
  // ---- merged KKT lower triangle (CSC over merged KKT indices) ----
  auto map_idx = [&](int64_t p, int64_t v) -> int64_t {
    return v < probs[p].n ? lay.xo[p] + v : n + lay.zrow[p][v - probs[p].n];
  };
  hp.kcol_ptr.assign(N + 1, 0);
  hp.kdiag.assign(N, -1);
  int64_t nnz = 0;
  for (const HostProblem& pr : probs) nnz += (int64_t)pr.krow.size();
  hp.krow.reserve(nnz);
  hp.kval.reserve(nnz);
  auto copy_col = [&](int64_t p, int64_t lc, int64_t col) {
    const HostProblem& pr = probs[p];
    for (int64_t e = pr.kcol_ptr[lc]; e < pr.kcol_ptr[lc + 1]; ++e) {
      const int64_t row = map_idx(p, pr.krow[e]);
      if (row == col) hp.kdiag[col] = (int64_t)hp.kval.size();
      hp.krow.push_back(row);
      hp.kval.push_back(pr.kval[e]);
    }
    hp.kcol_ptr[col + 1] = (int64_t)hp.kval.size();
  };
  for (int64_t p = 0; p < B; ++p) {
    probs[p].kx_off = (int64_t)hp.kval.size();  // the problem's x columns are copied whole, in order
    for (int64_t j = 0; j < probs[p].n; ++j) copy_col(p, j, lay.xo[p] + j);
  }
  hp.kval_x = (int64_t)hp.kval.size();
  std::vector<int64_t> zcol_start(m);  // kval z-part offset of each merged z column
  for (int64_t R = 0; R < m; ++R) {
    const int64_t p = zinv_p[R];
    zcol_start[R] = (int64_t)hp.kval.size() - hp.kval_x;
    copy_col(p, probs[p].n + zinv_r[R], n + R);
  }
  // ---- merged cone list ----
  ConeLayout& cl = hp.cl;
  cl = ConeLayout();
  cl.m_zero = ftot[0];
  cl.m_nonneg = ftot[1];
  cl.psd_k = psd_k;
  if (ftot[0] > 0) cl.cones.push_back(Cone{CLR_ZERO, ftot[0], 0.0, 0, 0});
  if (ftot[1] > 0) cl.cones.push_back(Cone{CLR_NONNEG, ftot[1], 0.0, cstart[1], zcol_start[cstart[1]]});
  auto add_family = [&](int64_t ConeLayout::*b0, int64_t ConeLayout::*b1, int64_t* begin, int64_t* end) {
    *begin = (int64_t)cl.cones.size();
    for (int64_t p = 0; p < B; ++p) {
      const ConeLayout& pl = probs[p].cl;
      for (int64_t c = pl.*b0; c < pl.*b1; ++c) {
        Cone k = pl.cones[c];
        k.off = lay.zrow[p][k.off];
        k.kbase = zcol_start[k.off];
        if (k.aux >= 0) k.aux = lay.zrow[p][k.aux];
        cl.cones.push_back(k);
        if (k.type == CLR_SOC) cl.soc_max_dim = std::max(cl.soc_max_dim, k.dim);
      }
    }
    *end = (int64_t)cl.cones.size();
  };
  add_family(&ConeLayout::soc_begin, &ConeLayout::soc_end, &cl.soc_begin, &cl.soc_end);
  add_family(&ConeLayout::exp_begin, &ConeLayout::exp_end, &cl.exp_begin, &cl.exp_end);
  add_family(&ConeLayout::pow_begin, &ConeLayout::pow_end, &cl.pow_begin, &cl.pow_end);
  add_family(&ConeLayout::psd_begin, &ConeLayout::psd_end, &cl.psd_begin, &cl.psd_end);
  cl.aux_begin = cstart[6];
  cl.n_aux = ftot[6];
  cl.kval_z = (int64_t)hp.kval.size() - hp.kval_x;
  cl.nu = 0;
  cl.symmetric_only = true;
  for (const HostProblem& pr : probs) {
    cl.nu += pr.cl.nu;
    cl.symmetric_only = cl.symmetric_only && pr.cl.symmetric_only;
  }
  // ---- merged fill-reducing order: each problem's own, concatenated ----
  std::vector<int64_t> order;
  order.reserve(N);
  int64_t n_dense = 0;
  for (int64_t p = 0; p < B; ++p) {
    const HostProblem& pr = probs[p];
    std::vector<int64_t> own;
    const std::vector<int64_t>* use = nullptr;
    if (!orders.empty() && !orders[p].empty()) {
      use = &orders[p];
    } else {
      int64_t nd = 0;
      int which = 0;
      choose_kkt_order(pr, own, nd, &which);
      n_dense += nd;
      use = &own;
    }
    if ((int64_t)use->size() != pr.n + pr.m) {
      err = "order has the wrong length";
      return CLR_E_DIM;
    }
    for (int64_t v : *use) {
      if (v < 0 || v >= pr.n + pr.m) {
        err = "order entry out of range";
        return CLR_E_INVALID;
      }
      order.push_back(map_idx(p, v));
    }
  }
  for (HostProblem& pr : probs) release_big(pr);
  int rc = symbolic_analyze(N, hp.kcol_ptr, hp.krow, &order, sy, relax);
  if (rc != CLR_OK) {
    err = "symbolic analysis failed";
    return rc;
  }
  sy.n_dense = n_dense;
  sy.ordering = -1;
  kkt_factor_counts(N, hp.kcol_ptr, hp.krow, order, &sy.pred_nnz, &sy.pred_flops);
  return CLR_OK;
}

}  // namespace clr
