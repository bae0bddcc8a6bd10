// sign(Q) and the Neuberger-Dirac operator (Sec. 2.2, 2.3) on the GPU.
//
//   D_N = (1 + gamma5 sign(Q)) / abar, abar = 1/(1 + s);  D_N^m = (1 - abar m_q/2) D_N + m_q.
//   sign(Q) ~ P_+ - P_- + (1 - P) X R(X^2) (1 - P),  X = Q / sqrt(lambda_max),
// with R(x) = x sum_l b_l / (x^2 + sigma_l) the Zolotarev approximation on [sqrt(eps), 1]
// (the paper's polynomial X P_n(X^2) replaced by the rational minmax function) and P the
// projector on the context's low modes.  Two-sided projection keeps the approximation
// hermitian; left_only = 1 gives the paper's literal (1 - P) X R(X^2) eta.
// The shifted inverses come from the multi-shift CG: pure FP64 (only y = sum_l b_l x_l is
// accumulated), or sloppy FP32/FP16 Krylov iterations with FP64 defect correction per shift.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "solver.h"

namespace nd {
nd_status lambda_max_estimate(nd_ctx* c, int iters, double* lam);
}

using namespace nd;

static nd_status sign_impl(nd_ctx* c, const double* in, const nd_dn_params* p, nd_dn_info* info, void** sign64,
                           void** eta64) {
  if (!c || !p) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (!in || p->n_poles < 1 || p->n_poles > CG_NMAX || !(p->tol > 0) || p->maxit < 1 || p->inner_prec < ND_FP64 ||
      p->inner_prec > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "sign(Q): bad parameters (1 <= n_poles <= 32, tol > 0)");
  if (!c->links[0] || !c->links[p->inner_prec] || (p->inner_prec != ND_FP64 && !c->links[1]))
    return fail(c, ND_ERR_STATE, "sign(Q): links must be set in FP64, the inner precision and (mixed) FP32");
  auto t0 = std::chrono::steady_clock::now();
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  const int l = c->nlow;
  double lam = p->lambda_max;
  if (!(lam > 0)) {
    if (!(c->lam_max > 0)) ND_TRY(lambda_max_estimate(c, 40, &c->lam_max));
    lam = 1.01 * c->lam_max;
  }
  double eps = p->eps;
  if (!(eps > 0)) {
    if (l == 0 || !(c->lam_next > 0))
      return fail(c, ND_ERR_INVALID_ARG, "sign(Q): eps must be given when no low modes are set");
    eps = 0.99 * c->lam_next / lam;
  }
  if (!(eps < 1.0)) return fail(c, ND_ERR_INVALID_ARG, "sign(Q): eps must be below 1");
  const int n = p->n_poles;
  std::vector<double> sigma(n), bw(n);
  double delta = 0.0;
  if (nd_zolotarev(n, eps, sigma.data(), bw.data(), &delta) != ND_OK)
    return fail(c, ND_ERR_INVALID_ARG, "sign(Q): Zolotarev coefficients");
  void* eta = field(c, "dn_eta", 0);
  void* src = field(c, "dn_src", 0);
  void* y = field(c, "dn_y", 0);
  void* z = field(c, "dn_z", 0);
  double* cdev = static_cast<double*>(workspace(c, "dn_c", sizeof(double) * 4 * 64));
  if (!eta || !src || !y || !z || !cdev) return fail(c, ND_ERR_OOM, "sign(Q): workspace");
  ND_TRY(nd_pack_spinor(c, eta, in, ND_FP64, 1));
  // low-mode coefficients c_k = (u_k, eta) and eta_perp = eta - sum_k c_k u_k
  std::vector<double> ck(2 * std::max(l, 1), 0.0);
  if (l) {
    ND_TRY_CUDA(c, blas_multidot(c->g, c->evecs, fs, l, eta, slot(c, cdev), c->stream));
    ND_TRY(read_back(c, cdev, ck.data(), 2 * l));
  }
  const bool two_sided = !p->left_only || l == 0;
  if (l && two_sided) {
    std::vector<double> neg(2 * l);
    for (int i = 0; i < 2 * l; ++i) neg[i] = -ck[i];
    ND_TRY_CUDA(c, cudaMemcpyAsync(cdev + 2 * 64, neg.data(), sizeof(double) * 2 * l, cudaMemcpyHostToDevice, c->stream));
    ND_TRY_CUDA(c, blas_lincomb(c->g, src, 1.0, eta, c->evecs, fs, l, cdev + 2 * 64, c->stream));
  } else {
    ND_TRY_CUDA(c, cudaMemcpyAsync(src, eta, fs, cudaMemcpyDeviceToDevice, c->stream));
  }
  double bn2;
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, src, 1.0, src, 0.0, nullptr, true, slot(c, c->red_scratch), c->stream));
  ND_TRY(read_back(c, c->red_scratch, &bn2, 1));
  if (!std::isfinite(bn2)) return fail(c, ND_ERR_NAN, "sign(Q): source has NaN or Inf");
  // per-shift residual targets bounding ||sum_l b_l (x_l - x_l*)|| <= tol ||src||
  double lam_min = eps;
  if (!two_sided) {
    lam_min = 1e300;
    for (int k = 0; k < l; ++k) lam_min = std::min(lam_min, c->nu[k] * c->nu[k] / lam);
  }
  std::vector<double> tol(n);
  for (int k = 0; k < n; ++k) tol[k] = p->tol * (lam_min + sigma[k]) / (n * std::fabs(bw[k]));
  nd_dn_info inf{};
  const double ascale = 1.0 / lam;
  if (bn2 == 0.0) {
    ND_TRY_CUDA(c, cudaMemsetAsync(y, 0, fs, c->stream));
  } else if (p->inner_prec == ND_FP64) {
    MsResult ms;
    nd_status s = mscg_run(c, 0, 0, true, src, y, sigma, tol, bw, ascale, p->maxit, &ms);
    if (s != ND_OK) return s;
    inf.iters = inf.sloppy_iters = ms.iters;
    for (int k = 0; k < n; ++k) inf.max_resid = std::max(inf.max_resid, ms.res[k]);
  } else {
    MixedStats ms;
    ND_TRY_CUDA(c, cudaMemsetAsync(y, 0, fs, c->stream));
    auto sink = [&](int k, void* x64) -> nd_status {
      ND_TRY_CUDA(c, blas_axpby(c->g, 0, y, 1.0, y, bw[k], x64, false, slot(c, nullptr), c->stream));
      return ND_OK;
    };
    nd_status s = mixed_solve(c, (int)p->inner_prec, src, bn2, sigma, tol, ascale, p->maxit, &ms, sink);
    if (s != ND_OK) return s;
    inf.iters = ms.iters;
    inf.sloppy_iters = ms.sloppy_iters;
    inf.outer = ms.outer;
    inf.max_resid = ms.max_resid;
  }
  // z = X y = Q y / sqrt(lambda_max); then z <- z - P z + sum_k sgn(nu_k) c_k u_k
  ND_TRY(q_apply(c, 0, z, y, 1.0 / std::sqrt(lam)));
  if (l) {
    std::vector<double> dk(2 * l);
    ND_TRY_CUDA(c, blas_multidot(c->g, c->evecs, fs, l, z, slot(c, cdev), c->stream));
    ND_TRY(read_back(c, cdev, dk.data(), 2 * l));
    std::vector<double> coef(2 * l);
    for (int k = 0; k < l; ++k) {
      const double sg = c->nu[k] > 0 ? 1.0 : -1.0;
      coef[2 * k] = -dk[2 * k] + sg * ck[2 * k];
      coef[2 * k + 1] = -dk[2 * k + 1] + sg * ck[2 * k + 1];
    }
    ND_TRY_CUDA(c, cudaMemcpyAsync(cdev + 2 * 64, coef.data(), sizeof(double) * 2 * l, cudaMemcpyHostToDevice, c->stream));
    ND_TRY_CUDA(c, blas_lincomb(c->g, z, 1.0, z, c->evecs, fs, l, cdev + 2 * 64, c->stream));
  }
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  inf.n_low = l;
  inf.delta = delta;
  inf.eps = eps;
  inf.lambda_max = lam;
  inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  *sign64 = z;
  *eta64 = eta;
  return ND_OK;
}

extern "C" nd_status nd_apply_sign(nd_ctx* c, double* out, const double* in, const nd_dn_params* p, nd_dn_info* info) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (!out || out == in) return fail(c, ND_ERR_INVALID_ARG, "nd_apply_sign: bad output pointer");
  void *sg, *eta;
  ND_TRY(sign_impl(c, in, p, info, &sg, &eta));
  ND_TRY(nd_unpack_spinor(c, out, sg, ND_FP64, 1));
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  return ND_OK;
}

extern "C" nd_status nd_apply_DN(nd_ctx* c, double* out, const double* in, const nd_dn_params* p, nd_dn_info* info) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (!out || out == in) return fail(c, ND_ERR_INVALID_ARG, "nd_apply_DN: bad output pointer");
  auto t0 = std::chrono::steady_clock::now();
  void *sg, *eta;
  ND_TRY(sign_impl(c, in, p, info, &sg, &eta));
  // D_N^m eta = (1 - abar m_q/2)(1 + s)(eta + gamma5 sign eta) + m_q eta
  const double abar = 1.0 / (1.0 + c->s);
  const double f = (1.0 - 0.5 * abar * p->m_q) / abar;
  void* o = field(c, "dn_out", 0);
  if (!o) return fail(c, ND_ERR_OOM, "nd_apply_DN: workspace");
  ND_TRY_CUDA(c, blas_g5_axpby(c->g, o, f + p->m_q, eta, f, sg, c->stream));
  ND_TRY(nd_unpack_spinor(c, out, o, ND_FP64, 1));
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  if (info) info->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return ND_OK;
}
