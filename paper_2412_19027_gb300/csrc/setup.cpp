// Setup phase, host side: validation, cone reordering and merging, modified
// Ruiz equilibration, scaled CSR copies of P, A, A^T and the value layout of
// the KKT matrix K = [P A^T; A -H] (Algorithm 1 steps 1-2 of the paper).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace clr {

namespace {

bool finite_all(const double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

int check_csc(const clr_csc* M, int64_t nrows, int64_t ncols, bool upper, std::string& err, const char* name) {
  if (!M) {
    err = std::string(name) + " is NULL";
    return CLR_E_INVALID;
  }
  if (M->nrows != nrows || M->ncols != ncols) {
    err = std::string(name) + " has the wrong shape";
    return CLR_E_DIM;
  }
  if (M->nnz < 0 || (M->nnz > 0 && (!M->colptr || !M->rowind || !M->val)) || (ncols > 0 && !M->colptr)) {
    err = std::string(name) + ": missing arrays";
    return CLR_E_INVALID;
  }
  if (ncols > 0 && (M->colptr[0] != 0 || M->colptr[ncols] != M->nnz)) {
    err = std::string(name) + ": colptr[0] must be 0 and colptr[ncols] == nnz";
    return CLR_E_INVALID;
  }
  for (int64_t j = 0; j < ncols; ++j) {
    if (M->colptr[j + 1] < M->colptr[j]) {
      err = std::string(name) + ": colptr not monotone";
      return CLR_E_INVALID;
    }
    for (int64_t p = M->colptr[j]; p < M->colptr[j + 1]; ++p) {
      int64_t i = M->rowind[p];
      if (i < 0 || i >= nrows || (p > M->colptr[j] && i <= M->rowind[p - 1])) {
        err = std::string(name) + ": row indices out of range or not increasing";
        return CLR_E_INVALID;
      }
      if (upper && i > j) {
        err = std::string(name) + ": entry below the diagonal (pass the upper triangle)";
        return CLR_E_INVALID;
      }
    }
  }
  if (!finite_all(M->val, M->nnz)) {
    err = std::string(name) + " has a NaN or Inf";
    return CLR_E_INVALID;
  }
  return CLR_OK;
}

int psd_order_of(int64_t d) {
  int k = (int)std::lround((std::sqrt(8.0 * (double)d + 1.0) - 1.0) / 2.0);
  return ((int64_t)k * (k + 1) / 2 == d) ? k : -1;
}

int64_t packed(int64_t d) { return d * (d + 1) / 2; }

double scale_factor(double norm, const clr_settings& st) {
  if (norm < 1e-8) return 1.0;
  double f = 1.0 / std::sqrt(norm);
  return std::min(std::max(f, st.scale_min), st.scale_max);
}

}  // namespace

int build_problem(HostProblem& hp, const clr_csc* P, const double* q, const clr_csc* A, const double* b,
                  const clr_cone* cones, int32_t ncones, const clr_settings& st, std::string& err) {
  if (!A || !P) {
    err = "P or A is NULL";
    return CLR_E_INVALID;
  }
  const int64_t n = A->ncols, m = A->nrows;
  if (n < 0 || m < 0) return CLR_E_DIM;
  int rc;
  if ((rc = check_csc(P, n, n, true, err, "P")) != CLR_OK) return rc;
  if ((rc = check_csc(A, m, n, false, err, "A")) != CLR_OK) return rc;
  if ((n > 0 && !q) || (m > 0 && !b) || (ncones > 0 && !cones) || ncones < 0) {
    err = "q, b or cones is NULL";
    return CLR_E_INVALID;
  }
  if (!finite_all(q, n) || !finite_all(b, m)) {
    err = "q or b has a NaN or Inf";
    return CLR_E_INVALID;
  }
  // ---- cones (Sec. 2.1) ----
  int64_t total = 0;
  int psd_k = 0;
  for (int32_t i = 0; i < ncones; ++i) {
    const clr_cone& c = cones[i];
    if (c.type < CLR_ZERO || c.type > CLR_PSD_TRI || c.dim < 0) {
      err = "bad cone type or dimension";
      return CLR_E_INVALID;
    }
    if ((c.type == CLR_EXP || c.type == CLR_POW) && c.dim != 3) {
      err = "exponential and power cones have dimension 3";
      return CLR_E_INVALID;
    }
    if (c.type == CLR_POW && !(c.alpha > 0.0 && c.alpha < 1.0)) {
      err = "power cone exponent must lie in (0, 1)";
      return CLR_E_INVALID;
    }
    if (c.type == CLR_SOC && c.dim < 1) {
      err = "second-order cone dimension must be >= 1";
      return CLR_E_INVALID;
    }
    if (c.type == CLR_PSD_TRI) {
      int k = psd_order_of(c.dim);
      if (k < 1) {
        err = "PSD cone dimension is not k(k+1)/2";
        return CLR_E_INVALID;
      }
      if (k > 32) {
        err = "PSD cones of order <= 32 only";
        return CLR_E_UNSUPPORTED;
      }
      psd_k = std::max(psd_k, k);
    }
    total += c.dim;
  }
  if (total != m) {
    err = "cone dimensions do not add up to the rows of A";
    return CLR_E_DIM;
  }
  hp.n = n;
  hp.m = m;

  // ---- reorder: zero, nonneg, SOC, exp, pow, PSD; merge zero and nonneg ----
  std::vector<int64_t> coff(ncones + 1, 0);
  for (int32_t i = 0; i < ncones; ++i) coff[i + 1] = coff[i] + cones[i].dim;
  ConeLayout& cl = hp.cl;
  cl = ConeLayout();
  hp.row_perm.clear();
  hp.row_perm.reserve(m);
  const int fam_order[6] = {CLR_ZERO, CLR_NONNEG, CLR_SOC, CLR_EXP, CLR_POW, CLR_PSD_TRI};
  for (int fi = 0; fi < 6; ++fi) {
    const int fam = fam_order[fi];
    if (fam == CLR_SOC) cl.soc_begin = (int64_t)cl.cones.size();
    if (fam == CLR_EXP) cl.exp_begin = (int64_t)cl.cones.size();
    if (fam == CLR_POW) cl.pow_begin = (int64_t)cl.cones.size();
    if (fam == CLR_PSD_TRI) cl.psd_begin = (int64_t)cl.cones.size();
    if (fam == CLR_ZERO || fam == CLR_NONNEG) {
      int64_t start = (int64_t)hp.row_perm.size();
      for (int32_t i = 0; i < ncones; ++i)
        if (cones[i].type == fam)
          for (int64_t r = coff[i]; r < coff[i + 1]; ++r) hp.row_perm.push_back(r);
      int64_t d = (int64_t)hp.row_perm.size() - start;
      if (fam == CLR_ZERO) cl.m_zero = d;
      else cl.m_nonneg = d;
      if (d > 0) cl.cones.push_back(Cone{fam, d, 0.0, start, 0});
    } else {
      for (int32_t i = 0; i < ncones; ++i) {
        if (cones[i].type != fam || cones[i].dim == 0) continue;
        cl.cones.push_back(Cone{fam, cones[i].dim, cones[i].alpha, (int64_t)hp.row_perm.size(), 0});
        for (int64_t r = coff[i]; r < coff[i + 1]; ++r) hp.row_perm.push_back(r);
      }
    }
    if (fam == CLR_SOC) cl.soc_end = (int64_t)cl.cones.size();
    if (fam == CLR_EXP) cl.exp_end = (int64_t)cl.cones.size();
    if (fam == CLR_POW) cl.pow_end = (int64_t)cl.cones.size();
    if (fam == CLR_PSD_TRI) cl.psd_end = (int64_t)cl.cones.size();
  }
  cl.psd_k = psd_k;
  // ---- large SOCs (Sec. 3.3: thousands of rows) in sparse form: H = eta^2 (I + u u' - v v'), the
  // rank-two part carried by two auxiliary KKT rows per cone, appended after
  // every cone row (rows m .. m + 2L - 1; no caller row) ----
  int64_t n_expanded = 0;
  for (int64_t c = cl.soc_begin; c < cl.soc_end; ++c)
    if (st.soc_expand_dim > 0 && cl.cones[c].dim >= st.soc_expand_dim) cl.cones[c].aux = m + 2 * n_expanded++;
  cl.aux_begin = m;
  cl.n_aux = 2 * n_expanded;
  const int64_t mi = m + cl.n_aux;  // internal constraint rows
  for (int64_t k = 0; k < cl.n_aux; ++k) hp.row_perm.push_back(-1);
  hp.m = mi;
  cl.nu = 0;
  cl.kval_z = 0;
  for (Cone& c : cl.cones) {
    c.kbase = cl.kval_z;
    switch (c.type) {
      case CLR_ZERO: cl.kval_z += c.dim; break;
      case CLR_NONNEG: cl.kval_z += c.dim; cl.nu += c.dim; break;
      case CLR_SOC:
        cl.kval_z += c.aux >= 0 ? 3 * c.dim : packed(c.dim);
        cl.nu += 1;
        cl.soc_max_dim = std::max(cl.soc_max_dim, c.dim);
        break;
      case CLR_EXP: case CLR_POW: cl.kval_z += 6; cl.nu += 3; cl.symmetric_only = false; break;
      case CLR_PSD_TRI: cl.kval_z += packed(c.dim); cl.nu += psd_order_of(c.dim); break;
    }
  }
  cl.kval_z += cl.n_aux;  // the auxiliary rows' diagonals

  // ---- reordered A as CSR (unscaled) and full P as CSR ----
  std::vector<int64_t> inv_row(m);
  for (int64_t r = 0; r < m; ++r) inv_row[hp.row_perm[r]] = r;
  Sparse& Ar = hp.A;
  Ar = Sparse();
  Ar.nrows = mi;  // the auxiliary rows are empty
  Ar.ncols = n;
  Ar.ptr.assign(mi + 1, 0);
  for (int64_t p = 0; p < A->nnz; ++p) Ar.ptr[inv_row[A->rowind[p]] + 1]++;
  for (int64_t r = 0; r < mi; ++r) Ar.ptr[r + 1] += Ar.ptr[r];
  Ar.idx.resize(A->nnz);
  Ar.val.resize(A->nnz);
  std::vector<int64_t> ar_src(A->nnz);  // caller index of each Ar entry
  {
    std::vector<int64_t> next(Ar.ptr.begin(), Ar.ptr.end() - 1);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = A->colptr[j]; p < A->colptr[j + 1]; ++p) {
        int64_t r = inv_row[A->rowind[p]];
        Ar.idx[next[r]] = (int32_t)j;
        ar_src[next[r]] = p;
        Ar.val[next[r]++] = A->val[p];
      }
  }
  // full symmetric P: upper entries (i <= j) plus their mirror
  Sparse& Pf = hp.Pf;
  Pf = Sparse();
  Pf.nrows = Pf.ncols = n;
  Pf.ptr.assign(n + 1, 0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = P->colptr[j]; p < P->colptr[j + 1]; ++p) {
      int64_t i = P->rowind[p];
      Pf.ptr[j + 1]++;
      if (i != j) Pf.ptr[i + 1]++;
    }
  for (int64_t j = 0; j < n; ++j) Pf.ptr[j + 1] += Pf.ptr[j];
  Pf.idx.resize(Pf.ptr[n]);
  Pf.val.resize(Pf.ptr[n]);
  std::vector<int64_t> pf_src(Pf.ptr[n]);  // caller index of each Pf entry
  {
    // row j of the full matrix: entries (j, i) for i < j come from column j's upper part mirrored
    // (P(i, j) stored in column j gives row i col j and row j col i).  Fill rows in column order so
    // every row comes out sorted.
    std::vector<int64_t> next(Pf.ptr.begin(), Pf.ptr.end() - 1);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = P->colptr[j]; p < P->colptr[j + 1]; ++p) {
        int64_t i = P->rowind[p];  // i <= j
        // row i gets column j (j >= i: appended in increasing j order)
        Pf.idx[next[i]] = (int32_t)j;
        pf_src[next[i]] = p;
        Pf.val[next[i]++] = P->val[p];
        if (i != j) {
          // row j gets column i; columns i < j arrive in increasing i order for fixed j, and
          // before any entry (j, j') with j' >= j is appended, since those come from column j' >= j.
          Pf.idx[next[j]] = (int32_t)i;
          pf_src[next[j]] = p;
          Pf.val[next[j]++] = P->val[p];
        }
      }
  }

  // ---- modified Ruiz equilibration (reading of Alg. 1 step 1) ----
  hp.D.assign(n, 1.0);
  hp.E.assign(mi, 1.0);
  hp.c = 1.0;
  std::vector<double> colx(n), rowz(mi);
  if (st.equilibrate) {
    for (int pass = 0; pass < st.ruiz_passes; ++pass) {
      std::fill(colx.begin(), colx.end(), 0.0);
      std::fill(rowz.begin(), rowz.end(), 0.0);
      for (int64_t i = 0; i < n; ++i)
        for (int64_t p = Pf.ptr[i]; p < Pf.ptr[i + 1]; ++p) {
          double v = std::fabs(hp.D[i] * Pf.val[p] * hp.D[Pf.idx[p]]);
          colx[i] = std::max(colx[i], v);
        }
      for (int64_t r = 0; r < mi; ++r)
        for (int64_t p = Ar.ptr[r]; p < Ar.ptr[r + 1]; ++p) {
          int64_t j = Ar.idx[p];
          double v = std::fabs(hp.E[r] * Ar.val[p] * hp.D[j]);
          colx[j] = std::max(colx[j], v);
          rowz[r] = std::max(rowz[r], v);
        }
      for (const Cone& c : cl.cones) {
        if (c.type == CLR_ZERO || c.type == CLR_NONNEG) continue;
        double mx = 0.0;
        for (int64_t r = c.off; r < c.off + c.dim; ++r) mx = std::max(mx, rowz[r]);
        for (int64_t r = c.off; r < c.off + c.dim; ++r) rowz[r] = mx;
      }
      for (int64_t j = 0; j < n; ++j)
        hp.D[j] = std::min(std::max(hp.D[j] * scale_factor(colx[j], st), st.scale_min), st.scale_max);
      for (int64_t r = 0; r < mi; ++r)
        hp.E[r] = std::min(std::max(hp.E[r] * scale_factor(rowz[r], st), st.scale_min), st.scale_max);
    }
    // cost scaling
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double mx = 0.0;
      for (int64_t p = Pf.ptr[i]; p < Pf.ptr[i + 1]; ++p)
        mx = std::max(mx, std::fabs(hp.D[i] * Pf.val[p] * hp.D[Pf.idx[p]]));
      sum += mx;
    }
    double mean = n ? sum / (double)n : 0.0;
    double qn = 0.0;
    for (int64_t j = 0; j < n; ++j) qn = std::max(qn, std::fabs(hp.D[j] * q[j]));
    double gamma = std::max(mean, qn);
    hp.c = (gamma < 1e-8) ? 1.0 : 1.0 / std::min(std::max(gamma, st.scale_min), st.scale_max);
  }
  // ---- scale P, A; build A^T ----
  hp.maxPdiag = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = Pf.ptr[i]; p < Pf.ptr[i + 1]; ++p) {
      Pf.val[p] *= hp.c * hp.D[i] * hp.D[Pf.idx[p]];
      if (Pf.idx[p] == i) hp.maxPdiag = std::max(hp.maxPdiag, std::fabs(Pf.val[p]));
    }
  for (int64_t r = 0; r < mi; ++r)
    for (int64_t p = Ar.ptr[r]; p < Ar.ptr[r + 1]; ++p) Ar.val[p] *= hp.E[r] * hp.D[Ar.idx[p]];
  Sparse& At = hp.At;
  At = Sparse();
  At.nrows = n;
  At.ncols = mi;
  At.ptr.assign(n + 1, 0);
  for (int64_t p = 0; p < Ar.nnz(); ++p) At.ptr[Ar.idx[p] + 1]++;
  for (int64_t j = 0; j < n; ++j) At.ptr[j + 1] += At.ptr[j];
  At.idx.resize(Ar.nnz());
  At.val.resize(Ar.nnz());
  std::vector<int64_t> at_src(Ar.nnz());  // caller index of each At entry
  {
    std::vector<int64_t> next(At.ptr.begin(), At.ptr.end() - 1);
    for (int64_t r = 0; r < mi; ++r)
      for (int64_t p = Ar.ptr[r]; p < Ar.ptr[r + 1]; ++p) {
        int64_t j = Ar.idx[p];
        At.idx[next[j]] = (int32_t)r;
        at_src[next[j]] = ar_src[p];
        At.val[next[j]++] = Ar.val[p];
      }
  }
  int rcq = set_qb(hp, q, b);
  if (rcq != CLR_OK) return rcq;

  // ---- KKT lower triangle (CSC over KKT indices) and the kval layout ----
  // x column j: P(i, j) for i >= j with an explicit diagonal, then A(:, j) as rows n + r.
  // z block of each cone: packed lower triangle of its H block (column-major);
  // an expanded SOC: per column its diagonal and its two auxiliary rows; the
  // auxiliary columns: their diagonal (+1 for p, -1 for q; constant).
  const int64_t N = n + mi;
  // value-update maps: equilibration factor of each caller value, P's diagonal
  hp.nnzP = P->nnz;
  hp.nnzA = A->nnz;
  hp.p_kv.assign(P->nnz, -1);
  hp.a_kv.assign(A->nnz, -1);
  hp.p_scale.resize(P->nnz);
  hp.a_scale.resize(A->nnz);
  hp.p_diag.clear();
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = P->colptr[j]; p < P->colptr[j + 1]; ++p) {
      const int64_t i = P->rowind[p];
      hp.p_scale[p] = hp.c * hp.D[i] * hp.D[j];
      if (i == j) hp.p_diag.push_back(p);
    }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t p = A->colptr[j]; p < A->colptr[j + 1]; ++p)
      hp.a_scale[p] = hp.E[inv_row[A->rowind[p]]] * hp.D[j];
  hp.kx_off = 0;
  hp.kcol_ptr.assign(N + 1, 0);
  hp.krow.clear();
  hp.kval.clear();
  hp.kdiag.assign(N, -1);
  for (int64_t j = 0; j < n; ++j) {
    // P row j == column j (symmetric); entries with index >= j
    bool has_diag = false;
    for (int64_t p = Pf.ptr[j]; p < Pf.ptr[j + 1]; ++p)
      if (Pf.idx[p] == j) has_diag = true;
    if (!has_diag) {
      hp.kdiag[j] = (int64_t)hp.kval.size();
      hp.krow.push_back(j);
      hp.kval.push_back(0.0);
    }
    for (int64_t p = Pf.ptr[j]; p < Pf.ptr[j + 1]; ++p) {
      int64_t i = Pf.idx[p];
      if (i < j) continue;
      if (i == j) hp.kdiag[j] = (int64_t)hp.kval.size();
      hp.p_kv[pf_src[p]] = (int64_t)hp.kval.size();
      hp.krow.push_back(i);
      hp.kval.push_back(Pf.val[p]);
    }
    for (int64_t p = At.ptr[j]; p < At.ptr[j + 1]; ++p) {
      hp.a_kv[at_src[p]] = (int64_t)hp.kval.size();
      hp.krow.push_back(n + At.idx[p]);
      hp.kval.push_back(At.val[p]);
    }
    hp.kcol_ptr[j + 1] = (int64_t)hp.kval.size();
  }
  hp.kval_x = (int64_t)hp.kval.size();
  // z columns: for each cone, columns off..off+dim-1; column c of a dense block has rows c..dim-1
  for (const Cone& c : cl.cones) {
    const bool dense = (c.type != CLR_ZERO && c.type != CLR_NONNEG && c.aux < 0);
    for (int64_t a = 0; a < c.dim; ++a) {
      const int64_t col = n + c.off + a;
      hp.kdiag[col] = (int64_t)hp.kval.size();
      int64_t last = dense ? c.dim : a + 1;
      for (int64_t r = a; r < last; ++r) {
        hp.krow.push_back(n + c.off + r);
        hp.kval.push_back(0.0);
      }
      if (c.aux >= 0)
        for (int64_t t = 0; t < 2; ++t) {  // eta u_a, eta v_a (written by the scaling)
          hp.krow.push_back(n + c.aux + t);
          hp.kval.push_back(0.0);
        }
      hp.kcol_ptr[col + 1] = (int64_t)hp.kval.size();
    }
  }
  for (int64_t k = 0; k < cl.n_aux; ++k) {
    const int64_t col = n + cl.aux_begin + k;
    hp.kdiag[col] = (int64_t)hp.kval.size();
    hp.krow.push_back(col);
    hp.kval.push_back((k % 2 == 0) ? 1.0 : -1.0);
    hp.kcol_ptr[col + 1] = (int64_t)hp.kval.size();
  }
  return CLR_OK;
}

// q, b in the caller's order -> scaled, reordered copies and unscaled norms.
int set_qb(HostProblem& hp, const double* q, const double* b) {
  const int64_t m_caller = hp.m - hp.cl.n_aux;  // b has the caller's rows only
  if ((hp.n && !q) || (m_caller && !b)) return CLR_E_INVALID;
  if (!finite_all(q, hp.n) || !finite_all(b, m_caller)) return CLR_E_INVALID;
  hp.q.resize(hp.n);
  hp.b.resize(hp.m);
  hp.qnorm = 0.0;
  hp.bnorm = 0.0;
  for (int64_t j = 0; j < hp.n; ++j) {
    hp.q[j] = hp.c * hp.D[j] * q[j];
    hp.qnorm = std::max(hp.qnorm, std::fabs(q[j]));
  }
  for (int64_t r = 0; r < hp.m; ++r) {
    const double v = hp.row_perm[r] >= 0 ? b[hp.row_perm[r]] : 0.0;  // auxiliary rows: b = 0
    hp.b[r] = hp.E[r] * v;
    hp.bnorm = std::max(hp.bnorm, std::fabs(v));
  }
  return CLR_OK;
}

// New values of P and/or A in the caller's CSC order, scaled with the setup's
// equilibration (the parametric update keeps D, E and c, as clr_update_qb does).
int set_PA(HostProblem& pr, const double* Px, const double* Ax, std::vector<double>& kval) {
  if ((Px && !finite_all(Px, pr.nnzP)) || (Ax && !finite_all(Ax, pr.nnzA))) return CLR_E_INVALID;
  if ((Px && (int64_t)pr.p_kv.size() != pr.nnzP) || (Ax && (int64_t)pr.a_kv.size() != pr.nnzA)) return CLR_E_STATE;
  if (Px) {
    for (int64_t k = 0; k < pr.nnzP; ++k) kval[pr.kx_off + pr.p_kv[k]] = Px[k] * pr.p_scale[k];
    pr.maxPdiag = 0.0;
    for (int64_t k : pr.p_diag) pr.maxPdiag = std::max(pr.maxPdiag, std::fabs(Px[k] * pr.p_scale[k]));
  }
  if (Ax)
    for (int64_t k = 0; k < pr.nnzA; ++k) kval[pr.kx_off + pr.a_kv[k]] = Ax[k] * pr.a_scale[k];
  return CLR_OK;
}

}  // namespace clr
