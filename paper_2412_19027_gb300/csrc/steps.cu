// Step-level entry points of the C ABI: the cone kernels and the sparse
// LDL^T run on their own, on host arrays (see include/clr.h).
#include <algorithm>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cones.cuh"
#include "internal.h"
#include "ldl.cuh"
#include "symbolic.h"

namespace clr {
namespace {

// Reordered layout of a bare cone list plus device buffers for the cone kernels.
struct ConeBench {
  DeviceArena ar;
  ConeDev cd;
  std::vector<int64_t> perm;            // reordered row -> caller row
  std::vector<int> fam;                 // caller cone -> family
  std::vector<int64_t> layout_index;    // caller cone -> index of its dense block in the layout
  std::vector<int64_t> kbase;           // caller cone -> packed kvz offset (dense families)
  std::vector<int64_t> caller_off;      // caller cone -> first caller row
  int64_t m = 0;
  int rc = CLR_OK;
  IterScal* sc = nullptr;  // the per-problem scalars of the single problem

  ConeBench(const clr_cone* cones, int32_t ncones) {
    int64_t total = 0;
    caller_off.resize(ncones);
    for (int32_t i = 0; i < ncones; ++i) {
      caller_off[i] = total;
      total += cones[i].dim;
      if (cones[i].type < CLR_ZERO || cones[i].type > CLR_PSD_TRI || cones[i].dim < 0) rc = CLR_E_INVALID;
      if ((cones[i].type == CLR_EXP || cones[i].type == CLR_POW) && cones[i].dim != 3) rc = CLR_E_INVALID;
      if (cones[i].type == CLR_PSD_TRI) {
        int k = (int)std::lround((std::sqrt(8.0 * cones[i].dim + 1.0) - 1.0) / 2.0);
        if (k * (k + 1) / 2 != cones[i].dim || k > 32) rc = CLR_E_UNSUPPORTED;
      }
    }
    if (rc) return;
    m = total;
    fam.resize(ncones);
    layout_index.assign(ncones, -1);
    kbase.assign(ncones, -1);
    int64_t mz = 0, mn = 0;
    for (int32_t i = 0; i < ncones; ++i) {
      fam[i] = cones[i].type;
      if (cones[i].type == CLR_ZERO) mz += cones[i].dim;
      if (cones[i].type == CLR_NONNEG) mn += cones[i].dim;
    }
    // zero rows, nonneg rows, then SOC, exp, pow, PSD cones in caller order
    for (int f : {CLR_ZERO, CLR_NONNEG})
      for (int32_t i = 0; i < ncones; ++i)
        if (cones[i].type == f)
          for (int64_t r = 0; r < cones[i].dim; ++r) perm.push_back(caller_off[i] + r);
    std::vector<int64_t> soc_off, soc_kb, psd_dim, psd_row, psd_kb;
    std::vector<int32_t> soc_dim;
    std::vector<double> alpha;
    int64_t kz = mz + mn;
    int64_t counts[6] = {0, 0, 0, 0, 0, 0};
    int64_t row0[6] = {0, 0, 0, 0, 0, 0}, kb0[6] = {0, 0, 0, 0, 0, 0};
    for (int f : {CLR_SOC, CLR_EXP, CLR_POW, CLR_PSD_TRI}) {
      row0[f] = (int64_t)perm.size();
      kb0[f] = kz;
      for (int32_t i = 0; i < ncones; ++i) {
        if (cones[i].type != f || cones[i].dim == 0) continue;
        const int64_t d = cones[i].dim;
        layout_index[i] = counts[f]++;
        kbase[i] = kz;
        if (f == CLR_SOC) {
          soc_off.push_back((int64_t)perm.size());
          soc_dim.push_back((int32_t)d);
          cd.soc_dmax = std::max<int>(cd.soc_dmax, (int)d);
          if (d <= 8) cd.soc_nsmall++;  // a thread per cone
          soc_kb.push_back(kz);
        }
        if (f == CLR_POW) alpha.push_back(cones[i].alpha);
        if (f == CLR_PSD_TRI) {
          psd_dim.push_back(d);
          psd_row.push_back((int64_t)perm.size());
          psd_kb.push_back(kz);
        }
        kz += (f == CLR_EXP || f == CLR_POW) ? 6 : d * (d + 1) / 2;
        for (int64_t r = 0; r < d; ++r) perm.push_back(caller_off[i] + r);
      }
    }
    cd.m = m;
    cd.m_zero = mz;
    cd.m_nonneg = mn;
    cd.n_soc = counts[CLR_SOC];
    cd.soc_split = (cd.soc_nsmall > 0 && cd.soc_nsmall < cd.n_soc) ? 1 : 0;
    cd.soc_off = ar.upload(soc_off.data(), (int64_t)soc_off.size());
    cd.soc_dim = ar.upload(soc_dim.data(), (int64_t)soc_dim.size());
    cd.soc_kb = ar.upload(soc_kb.data(), (int64_t)soc_kb.size());
    cd.n_exp = counts[CLR_EXP];
    cd.exp_row0 = row0[CLR_EXP];
    cd.exp_kb0 = kb0[CLR_EXP];
    cd.n_pow = counts[CLR_POW];
    cd.pow_row0 = row0[CLR_POW];
    cd.pow_kb0 = kb0[CLR_POW];
    cd.pow_alpha = ar.upload(alpha.data(), (int64_t)alpha.size());
    if (!cones_psd_setup(ar, cd, psd_dim, psd_row, psd_kb)) {
      rc = CLR_E_OOM;
      return;
    }
    cd.nkz = kz;
    cd.kvz = ar.alloc_n<double>(kz);
    cd.scratch = ar.alloc_n<double>(m);
    cd.nn_w = ar.alloc_n<double>(mn);
    cd.nn_lam = ar.alloc_n<double>(mn);
    cd.soc_eta = ar.alloc_n<double>(cd.n_soc);
    cd.soc_wb = ar.alloc_n<double>(m);
    cd.soc_lam = ar.alloc_n<double>(m);

    cd.ep_zt = ar.alloc_n<double>(3 * (cd.n_exp + cd.n_pow));
    exp_central_point_host(cd.exp_center);
    // one problem: every row belongs to problem 0
    std::vector<int32_t> pid(m, 0);
    ProbConst pc{};
    pc.sym = (cd.n_exp + cd.n_pow) == 0 ? 1 : 0;
    cd.nprob = 1;
    cd.row_pid = ar.upload(pid.data(), m);
    cd.pc = ar.upload(&pc, 1);
    sc = ar.alloc_n<IterScal>(1);
    if (cones_init_shadow(nullptr, cd, nullptr) != CLR_OK) rc = CLR_E_CUDA;
    if (!cd.kvz || !cd.scratch || !cd.soc_wb || !cd.row_pid || !cd.pc || !sc) rc = CLR_E_OOM;
  }

  double* upload_perm(const double* v) {
    std::vector<double> t(m);
    for (int64_t r = 0; r < m; ++r) t[r] = v[perm[r]];
    return ar.upload(t.data(), m);
  }
  int download_unperm(const double* d, double* out) {
    std::vector<double> t(m);
    if (m > 0) CLR_CUDA(cudaMemcpy(t.data(), d, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost));
    for (int64_t r = 0; r < m; ++r) out[perm[r]] = t[r];
    return CLR_OK;
  }
};

}  // namespace
}  // namespace clr

using namespace clr;

extern "C" {

int clr_cones_scaling(const clr_cone* cones, int32_t ncones, const double* s, const double* z, double mu,
                      double* H_out) {
  if ((ncones && !cones) || !H_out) return CLR_E_INVALID;
  ConeBench cb(cones, ncones);
  if (cb.rc) return cb.rc;
  if (cb.m == 0) return CLR_OK;
  if (!s || !z) return CLR_E_INVALID;
  double* ds = cb.upload_perm(s);
  double* dz = cb.upload_perm(z);
  if (!ds || !dz) return CLR_E_OOM;
  IterScal h{};
  h.mu = mu;
  CLR_CUDA(cudaMemcpy(cb.sc, &h, sizeof(IterScal), cudaMemcpyHostToDevice));
  int rc = cones_scaling(nullptr, cb.cd, ds, dz, cb.sc, nullptr);
  if (rc) return rc;
  std::vector<double> kv(cb.cd.nkz);
  CLR_CUDA(cudaDeviceSynchronize());
  CLR_CUDA(cudaMemcpy(kv.data(), cb.cd.kvz, sizeof(double) * kv.size(), cudaMemcpyDeviceToHost));
  // inverse row permutation
  std::vector<int64_t> iperm(cb.m);
  for (int64_t r = 0; r < cb.m; ++r) iperm[cb.perm[r]] = r;
  int64_t hoff = 0;
  for (int32_t i = 0; i < ncones; ++i) {
    const int64_t d = cones[i].dim;
    double* H = H_out + hoff;
    std::fill(H, H + d * d, 0.0);
    if (cones[i].type == CLR_NONNEG)
      for (int64_t a = 0; a < d; ++a) H[a * d + a] = -kv[iperm[cb.caller_off[i] + a]];
    else if (cones[i].type != CLR_ZERO) {
      const double* kb = kv.data() + cb.kbase[i];
      int64_t q = 0;
      for (int64_t c = 0; c < d; ++c)
        for (int64_t r = c; r < d; ++r) {
          H[r * d + c] = H[c * d + r] = -kb[q];
          ++q;
        }
    }
    hoff += d * d;
  }
  return CLR_OK;
}

int clr_cones_step_length(const clr_cone* cones, int32_t ncones, const double* s, const double* z, const double* ds,
                          const double* dz, double alpha_max, double* alpha_out) {
  if ((ncones && !cones) || !alpha_out) return CLR_E_INVALID;
  ConeBench cb(cones, ncones);
  if (cb.rc) return cb.rc;
  if (cb.m == 0) {
    *alpha_out = alpha_max;
    return CLR_OK;
  }
  double *d_s = cb.upload_perm(s), *d_z = cb.upload_perm(z), *d_ds = cb.upload_perm(ds), *d_dz = cb.upload_perm(dz);
  if (!d_s || !d_z || !d_ds || !d_dz) return CLR_E_OOM;
  IterScal h{};
  const double inf = INFINITY;
  std::memcpy(&h.amin_bits, &inf, 8);
  CLR_CUDA(cudaMemcpy(cb.sc, &h, sizeof(IterScal), cudaMemcpyHostToDevice));
  int rc = cones_step_symmetric(nullptr, cb.cd, d_s, d_ds, d_z, d_dz, cb.sc, nullptr);
  if (rc) return rc;
  CLR_CUDA(cudaMemcpy(&h, cb.sc, sizeof(IterScal), cudaMemcpyDeviceToHost));
  double amin_v;
  std::memcpy(&amin_v, &h.amin_bits, 8);
  double a = std::min(alpha_max, amin_v);
  if (cb.cd.n_exp + cb.cd.n_pow > 0) {
    h.alpha_sym = a;
    CLR_CUDA(cudaMemcpy(cb.sc, &h, sizeof(IterScal), cudaMemcpyHostToDevice));
    rc = cones_step_nonsym(nullptr, cb.cd, d_s, d_ds, d_z, d_dz, cb.sc, 0.8, 0, 1e-6, nullptr);
    if (rc) return rc;
    CLR_CUDA(cudaMemcpy(&h, cb.sc, sizeof(IterScal), cudaMemcpyDeviceToHost));
    a = a * std::pow(0.8, (double)h.ns.jint);
  }
  *alpha_out = a;
  return CLR_OK;
}

int clr_cones_combined_ds(const clr_cone* cones, int32_t ncones, const double* s, const double* z,
                          const double* ds_a, const double* dz_a, double sigma_mu, double* ds_out) {
  if ((ncones && !cones) || !ds_out) return CLR_E_INVALID;
  ConeBench cb(cones, ncones);
  if (cb.rc) return cb.rc;
  if (cb.m == 0) return CLR_OK;
  double *d_s = cb.upload_perm(s), *d_z = cb.upload_perm(z), *d_dsa = cb.upload_perm(ds_a),
         *d_dza = cb.upload_perm(dz_a);
  double* out = cb.ar.alloc_n<double>(cb.m);
  if (!d_s || !d_z || !d_dsa || !d_dza || !out) return CLR_E_OOM;
  IterScal h{};
  h.mu = 1.0;
  h.sigma_mu = sigma_mu;
  CLR_CUDA(cudaMemcpy(cb.sc, &h, sizeof(IterScal), cudaMemcpyHostToDevice));
  int rc = cones_scaling(nullptr, cb.cd, d_s, d_z, cb.sc, nullptr);
  if (rc) return rc;
  rc = cones_combined_ds(nullptr, cb.cd, d_s, d_z, d_dsa, d_dza, cb.sc, out, nullptr);
  if (rc) return rc;
  CLR_CUDA(cudaDeviceSynchronize());
  return cb.download_unperm(out, ds_out);
}

int clr_cones_time(const clr_cone* cones, int32_t ncones, const double* s, const double* z, const double* ds,
                   const double* dz, double mu, int32_t reps, clr_cone_times* out) {
  if ((ncones && !cones) || !out || !s || !z || !ds || !dz || reps < 1) return CLR_E_INVALID;
  *out = clr_cone_times{-1.0, -1.0, -1.0, 0, 0};
  ConeBench cb(cones, ncones);
  if (cb.rc) return cb.rc;
  out->rows = cb.m;
  out->kkt_values = cb.cd.nkz;
  if (cb.m == 0) return CLR_OK;
  double *d_s = cb.upload_perm(s), *d_z = cb.upload_perm(z), *d_ds = cb.upload_perm(ds), *d_dz = cb.upload_perm(dz);
  double* dsout = cb.ar.alloc_n<double>(cb.m);
  if (!d_s || !d_z || !d_ds || !d_dz || !dsout) return CLR_E_OOM;
  IterScal h{};
  h.mu = mu;
  h.sigma_mu = 0.1 * mu;
  const double inf = INFINITY;
  std::memcpy(&h.amin_bits, &inf, 8);
  CLR_CUDA(cudaMemcpy(cb.sc, &h, sizeof(IterScal), cudaMemcpyHostToDevice));
  cudaEvent_t e0, e1;
  CLR_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CLR_E_CUDA;
  }
  int rc = CLR_OK;
  // 0: scaling (+ KKT block), 1: symmetric step-length ratio tests, 2: combined-step d_s
  for (int which = 0; which < 3 && rc == CLR_OK; ++which) {
    for (int r = 0; r <= reps && rc == CLR_OK; ++r) {
      if (r == 1 && cudaEventRecord(e0, nullptr) != cudaSuccess) rc = CLR_E_CUDA;
      if (rc) break;
      if (which == 0) rc = cones_scaling(nullptr, cb.cd, d_s, d_z, cb.sc, nullptr);
      else if (which == 1) rc = cones_step_symmetric(nullptr, cb.cd, d_s, d_ds, d_z, d_dz, cb.sc, nullptr);
      else rc = cones_combined_ds(nullptr, cb.cd, d_s, d_z, d_ds, d_dz, cb.sc, dsout, nullptr);
    }
    float ms = 0.f;
    if (rc == CLR_OK && (cudaEventRecord(e1, nullptr) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = CLR_E_CUDA;
    if (rc == CLR_OK) (which == 0 ? out->scaling_ms : which == 1 ? out->step_ms : out->combined_ds_ms) = ms / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int clr_ldl_solve(const clr_csc* K, const double* signs, const int64_t* order, int32_t factor_bits,
                  double dyn_reg_eps, double dyn_reg_delta, const double* rhs, double* x_out, double* D_out,
                  int32_t* dyn_hits_out, int32_t big_front_schedule) {
  if (!K || !signs || !rhs || !x_out || (factor_bits != 64 && factor_bits != 32 && factor_bits != 16) ||
      big_front_schedule < 0 || big_front_schedule > 3)
    return CLR_E_INVALID;
  const int64_t N = K->ncols;
  if (K->nrows != N) return CLR_E_DIM;
  if (N == 0) return CLR_OK;
  std::vector<int64_t> colptr(K->colptr, K->colptr + N + 1), row(K->nnz);
  for (int64_t j = 0; j < N; ++j) {
    bool diag = false;
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      row[p] = K->rowind[p];
      if (row[p] < j || row[p] >= N) return CLR_E_INVALID;
      if (row[p] == j) diag = true;
      if (!std::isfinite(K->val[p])) return CLR_E_INVALID;
    }
    if (!diag) return CLR_E_INVALID;
  }
  Symbolic sy;
  std::vector<int64_t> ord;
  if (order) ord.assign(order, order + N);
  int rc = symbolic_analyze(N, colptr, row, order ? &ord : nullptr, sy);
  if (rc) return rc;
  NumericMaps mp;
  build_numeric_maps(sy, colptr, row, mp);
  std::vector<int8_t> dsign(N);
  for (int64_t k = 0; k < N; ++k) dsign[k] = signs[sy.perm[k]] > 0 ? 1 : -1;
  DeviceArena ar;
  LdlStructure ls;
  rc = ldl_structure_upload(ar, sy, mp, dsign, factor_bits == 64 ? 96 : 128, ls);
  if (rc) return rc;
  double* kv = ar.upload(K->val, K->nnz);
  double* drhs = ar.upload(rhs, N);
  IterScal hsc{};  // delta = 0: K is factored as given
  IterScal* ddelta = ar.upload(&hsc, 1);
  if (!kv || !drhs || !ddelta) return CLR_E_OOM;
  std::vector<double> xs(N), Dpos(N);
  int hits = 0;
  if (factor_bits == 64) {
    LdlFactor<double> f;
    f.flow = big_front_schedule != 0;
    if ((rc = f.alloc(ar, ls))) return rc;
    if ((rc = f.factor(nullptr, kv, ddelta, dyn_reg_eps, dyn_reg_delta, nullptr))) return rc;
    if ((rc = f.solve(nullptr, drhs, nullptr))) return rc;
    CLR_CUDA(cudaDeviceSynchronize());
    CLR_CUDA(cudaMemcpy(xs.data(), f.xs, sizeof(double) * N, cudaMemcpyDeviceToHost));
    CLR_CUDA(cudaMemcpy(Dpos.data(), f.Dp, sizeof(double) * N, cudaMemcpyDeviceToHost));
    CLR_CUDA(cudaMemcpy(&hits, f.dyn_hits, sizeof(int), cudaMemcpyDeviceToHost));
  } else {
    LdlFactor<float> f;
    f.tc16 = factor_bits == 16;
    f.flow = big_front_schedule != 0;
    f.flow_tc = big_front_schedule == 1 ? 1 : (big_front_schedule == 3 ? 2 : 0);
    if ((rc = f.alloc(ar, ls))) return rc;
    if ((rc = f.factor(nullptr, kv, ddelta, dyn_reg_eps, dyn_reg_delta, nullptr))) return rc;
    if ((rc = f.solve(nullptr, drhs, nullptr))) return rc;
    CLR_CUDA(cudaDeviceSynchronize());
    std::vector<float> xf(N), df(N);
    CLR_CUDA(cudaMemcpy(xf.data(), f.xs, sizeof(float) * N, cudaMemcpyDeviceToHost));
    CLR_CUDA(cudaMemcpy(df.data(), f.Dp, sizeof(float) * N, cudaMemcpyDeviceToHost));
    CLR_CUDA(cudaMemcpy(&hits, f.dyn_hits, sizeof(int), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < N; ++i) {
      xs[i] = xf[i];
      Dpos[i] = df[i];
    }
  }
  for (int64_t i = 0; i < N; ++i) x_out[i] = xs[i];
  if (D_out)
    for (int64_t k = 0; k < N; ++k) D_out[sy.perm[k]] = Dpos[k];
  if (dyn_hits_out) *dyn_hits_out = hits;
  return CLR_OK;
}

}  // extern "C"
