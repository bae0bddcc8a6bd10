// sign(Q) and the Neuberger-Dirac operator (Sec. 2.2, 2.3) on the GPU.
//
//   D_N = (1 + gamma5 sign(Q)) / abar, abar = 1/(1 + s);  D_N^m = (1 - abar m_q/2) D_N + m_q.
//   sign(Q) ~ P_+ - P_- + (1 - P) X R(X^2) (1 - P),  X = Q / sqrt(lambda_max),
// with R(x) = x sum_l b_l / (x^2 + sigma_l) the Zolotarev approximation on [sqrt(eps), 1]
// (the rational minmax function), or the paper's own minmax polynomial R(x) = x P_n(x^2) by the
// Clenshaw recurrence (approx = ND_SIGN_CHEBYSHEV), and P the projector on the context's low
// modes.  Two-sided projection keeps the approximation hermitian; left_only = 1 gives the
// paper's literal (1 - P) X R(X^2) eta.
// The shifted inverses of R come from the multi-shift CG: pure FP64 (only y = sum_l b_l x_l is
// accumulated), or sloppy FP32/FP16 Krylov iterations with FP64 defect correction per shift.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "solver.h"

namespace nd {
nd_status lambda_max_estimate(nd_ctx* c, int iters, double* lam);
}

using namespace nd;

// y = P_n(X^2) s by the Clenshaw recurrence (Sec. 2.2), every vector in storage precision ps:
//   b_n = c_n s,  b_k = c_k s + 2 A b_{k+1} - b_{k+2},  P_n(X^2) s = c_0 s + A b_1 - b_2,
//   A = (2 X^2 - 1 - eps) / (1 - eps),  X^2 = Q^2 / lambda,  so 2 A = alpha Q^2 + beta with
//   alpha = 4 / (lambda (1 - eps)),  beta = -2 (1 + eps) / (1 - eps).
// A step is two launches: t = Q b_{k+1}, then b_k = alpha Q t + beta b_{k+1} - b_{k+2} + c_k s
// written over b_{k+2} (two b buffers rotate).
static nd_status clenshaw(nd_ctx* c, int ps, const void* src64, void* y64, const std::vector<double>& co, double lam,
                          double eps) {
  NvtxRange range("nd.clenshaw");
  const int n = (int)co.size() - 1;
  const double alpha = 4.0 / (lam * (1.0 - eps)), beta = -2.0 * (1.0 + eps) / (1.0 - eps);
  if (n == 0) {
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, y64, co[0], src64, 0.0, nullptr, false, slot(c, nullptr), c->stream));
    return ND_OK;
  }
  const void* s = src64;
  if (ps != 0) {
    void* s_ps = field(c, "ch_s", ps);
    if (!s_ps) return fail(c, ND_ERR_OOM, "Clenshaw: workspace");
    ND_TRY_CUDA(c, blas_convert(c->g, ps, s_ps, 0, src64, c->stream));
    s = s_ps;
  }
  void* b1 = field(c, "ch_b0", ps);
  void* b2 = field(c, "ch_b1", ps);
  void* t = field(c, "ch_t", ps);
  if (!b1 || !b2 || !t) return fail(c, ND_ERR_OOM, "Clenshaw: workspace");
  ND_TRY_CUDA(c, blas_axpby(c->g, ps, b1, co[n], s, 0.0, nullptr, false, slot(c, nullptr), c->stream));  // b_n
  // k = n - 1 (b_{n+1} = 0), or the final step when n = 1
  const double h1 = n == 1 ? 0.5 : 1.0;
  ND_TRY(q_apply(c, ps, t, b1));
  ND_TRY(q_apply(c, ps, b2, t, h1 * alpha, h1 * beta, b1, nullptr, nullptr, s, co[n - 1]));
  std::swap(b1, b2);  // b1 = b_{n-1}, b2 = b_n
  for (int k = n - 2; k >= 0; --k) {
    const double hk = k == 0 ? 0.5 : 1.0;
    ND_TRY(q_apply(c, ps, t, b1));
    ND_TRY(q_apply(c, ps, b2, t, hk * alpha, hk * beta, b1, nullptr, nullptr, b2, -1.0, s, co[k]));
    std::swap(b1, b2);
  }
  // b1 holds P_n(X^2) s
  if (ps != 0)
    ND_TRY_CUDA(c, blas_convert(c->g, 0, y64, ps, b1, c->stream));
  else
    ND_TRY_CUDA(c, cudaMemcpyAsync(y64, b1, (size_t)spinor_bytes(0, c->Vh), cudaMemcpyDeviceToDevice, c->stream));
  return ND_OK;
}

// in: canonical FP64 (packed here), or the internal FP64 layout when `internal`.
static nd_status sign_impl(nd_ctx* c, const double* in, const nd_dn_params* p, nd_dn_info* info, void** sign64,
                           void** eta64, bool internal = false) {
  NvtxRange range("nd.sign");
  if (!c || !p) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  const bool poly = p->approx == ND_SIGN_CHEBYSHEV;
  if (p->approx != ND_SIGN_ZOLOTAREV && !poly) return fail(c, ND_ERR_INVALID_ARG, "sign(Q): unknown approximation");
  if (!in || (!poly && (p->n_poles < 1 || p->n_poles > CG_NMAX || p->maxit < 1)) || !(p->tol > 0) ||
      p->inner_prec < ND_FP64 || p->inner_prec > ND_FP16 || (poly && (p->degree < 0 || p->degree > 2048)))
    return fail(c, ND_ERR_INVALID_ARG, "sign(Q): bad parameters (1 <= n_poles <= 32, 0 <= degree <= 2048, tol > 0)");
  if (!c->links[0] || !c->links[p->inner_prec] || (!poly && p->inner_prec != ND_FP64 && !c->links[1]))
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
  const int n = poly ? 0 : p->n_poles;
  std::vector<double> sigma(n), bw(n), cheb;
  double delta = 0.0;
  int degree = 0;
  if (poly) {
    degree = p->degree;
    if (degree == 0 && nd_chebyshev_degree(eps, p->tol, &degree) != ND_OK)
      return fail(c, ND_ERR_INVALID_ARG, "sign(Q): no polynomial degree <= 2048 reaches tol on [eps, 1]");
    cheb.resize(degree + 1);
    const nd_status st = nd_chebyshev(degree, eps, cheb.data(), &delta);
    if (st != ND_OK) return fail(c, st, "sign(Q): minmax polynomial coefficients");
  } else if (nd_zolotarev(n, eps, sigma.data(), bw.data(), &delta) != ND_OK) {
    return fail(c, ND_ERR_INVALID_ARG, "sign(Q): Zolotarev coefficients");
  }
  void* eta = internal ? const_cast<double*>(in) : field(c, "dn_eta", 0);
  void* src = field(c, "dn_src", 0);
  void* y = field(c, "dn_y", 0);
  void* z = field(c, "dn_z", 0);
  double* cdev = static_cast<double*>(workspace(c, "dn_c", sizeof(double) * 4 * 64));
  if (!eta || !src || !y || !z || !cdev) return fail(c, ND_ERR_OOM, "sign(Q): workspace");
  if (!internal) ND_TRY(nd_pack_spinor(c, eta, in, ND_FP64, 1));
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
  } else if (poly) {
    ND_TRY(clenshaw(c, (int)p->inner_prec, src, y, cheb, lam, eps));
    inf.degree = degree;
  } else if (p->inner_prec == ND_FP64) {
    MsResult ms;
    nd_status s = mscg_run(c, 0, 0, true, src, y, sigma, tol, bw, ascale, p->maxit, &ms);
    if (s != ND_OK) return s;
    inf.iters = inf.sloppy_iters = ms.iters;
    for (int k = 0; k < n; ++k) inf.max_resid = std::max(inf.max_resid, ms.res[k]);
    inf.krylov_ms = ms.ms;
    inf.krylov_live_shifts = (int)ms.live;
    inf.krylov_active_shifts = (int)ms.active;
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
    inf.krylov_ms = ms.krylov_ms;
    inf.krylov_live_shifts = (int)ms.live;
    inf.krylov_active_shifts = (int)ms.active;
    inf.residuals64 = ms.residuals64;
    inf.correction_iters = ms.correction_iters;
    inf.refine_ms = ms.refine_ms;
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

namespace nd {
nd_status sign_internal(nd_ctx* c, const void* in64, const nd_dn_params* p, nd_dn_info* info, void** sign64) {
  void* eta;
  return sign_impl(c, static_cast<const double*>(in64), p, info, sign64, &eta, true);
}
}  // namespace nd

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

// D_N^m^dagger eta = gamma5 D_N^m gamma5 eta (Sec. 2.2: D_N^dagger = gamma5 D_N gamma5 because sign(Q) is
// hermitian; the two-sided deflated approximation keeps it so).  With f = (1 - abar m_q/2)(1 + s):
//   gamma5 [f (gamma5 eta + gamma5 sign(Q) gamma5 eta) + m_q gamma5 eta] = (f + m_q) eta + f sign(Q) gamma5 eta,
// so one sign(Q) application on gamma5 eta and one combination.
extern "C" nd_status nd_apply_DN_dagger(nd_ctx* c, double* out, const double* in, const nd_dn_params* p,
                                        nd_dn_info* info) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (!out || out == in || !p) return fail(c, ND_ERR_INVALID_ARG, "nd_apply_DN_dagger: bad argument");
  if (p->left_only)
    return fail(c, ND_ERR_INVALID_ARG, "nd_apply_DN_dagger: gamma5 D_N gamma5 is the adjoint only of the two-sided form");
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  auto t0 = std::chrono::steady_clock::now();
  void* eta = field(c, "dnd_eta", 0);
  void* g5eta = field(c, "dnd_g5eta", 0);
  void* o = field(c, "dn_out", 0);
  if (!eta || !g5eta || !o) return fail(c, ND_ERR_OOM, "nd_apply_DN_dagger: workspace");
  ND_TRY(nd_pack_spinor(c, eta, in, ND_FP64, 1));
  ND_TRY_CUDA(c, blas_g5(c->g, 0, g5eta, eta, c->stream));
  void *sg, *e2;
  ND_TRY(sign_impl(c, static_cast<const double*>(g5eta), p, info, &sg, &e2, true));
  const double abar = 1.0 / (1.0 + c->s);
  const double f = (1.0 - 0.5 * abar * p->m_q) / abar;
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, o, f + p->m_q, eta, f, sg, false, slot(c, nullptr), c->stream));
  ND_TRY(nd_unpack_spinor(c, out, o, ND_FP64, 1));
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  if (info) info->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return ND_OK;
}
