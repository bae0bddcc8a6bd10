// Propagators of the massive overlap operator: x = (D_N^m)^{-1} b (Sec. 2.2 operator; the
// paper's stated next use of it).
//
// D^m = alpha (1 + gamma5 eps) + m with eps = sign(Q), alpha = (1 + s)(1 - abar m / 2).  With
// eps^2 = 1 and eps hermitian, D^m is normal and
//   H = D^m D^m^dagger = D^m^dagger D^m = k (2 + gamma5 eps + eps gamma5) + m^2,  k = alpha^2 + alpha m,
// which commutes with gamma5.  On a vector of one chirality (gamma5 v = c v, c = +-1)
//   H v = (2k + m^2) v + 2 c k P_c eps v = (2k + m^2) v + k (c z + gamma5 z),  z = eps v,
// so every CG iteration costs one sign(Q) application.  b is split into its two chiral parts
// (a point source has one), each part is solved by CG on H to ||b_c - H y_c|| <= tol ||b_c||,
// and x = D^m^dagger y = gamma5 D^m gamma5 y.  With an approximate sign(Q), eps^2 = 1 holds only to
// the accuracy of the approximation and of the low modes, so H and D^m D^m^dagger differ by that
// much: an outer defect correction on D^m x = b (true residual after each pass, one more sign(Q)
// application) brings the residual of D^m x = b itself below tol.
#include <chrono>
#include <cmath>

#include "solver.h"

using namespace nd;

namespace {

// w = H v for v of chirality c (internal FP64 fields)
nd_status apply_H(nd_ctx* c, void* w, const void* v, int chir, double k, double m, const nd_dn_params* p,
                  int* sign_iters) {
  nd_dn_info inf{};
  void* z;
  ND_TRY(sign_internal(c, v, p, &inf, &z));
  *sign_iters += inf.iters + inf.degree;
  ND_TRY_CUDA(c, blas_g5_axpby(c->g, w, chir * k, z, k, z, c->stream));
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, w, 1.0, w, 2.0 * k + m * m, v, false, slot(c, nullptr), c->stream));
  return ND_OK;
}

double dot_re(nd_ctx* c, const void* x, const void* y, nd_status* st) {
  double h[3] = {0, 0, 0};
  cudaError_t e = blas_dot(c->g, 0, x, y, slot(c, c->red_scratch), c->stream);
  if (e != cudaSuccess) {
    *st = fail_cuda(c, e, "propagator: dot");
    return 0.0;
  }
  *st = read_back(c, c->red_scratch, h, 3);
  return h[0];
}

}  // namespace

extern "C" nd_status nd_propagator(nd_ctx* c, double* x_out, const double* b_in, const nd_dn_params* p, double tol,
                                   int maxit, nd_prop_info* info) {
  NvtxRange range("nd.propagator");
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (!p || !x_out || !b_in || x_out == b_in || !(tol > 0) || maxit < 1)
    return fail(c, ND_ERR_INVALID_ARG, "nd_propagator: bad arguments");
  if (p->left_only)
    return fail(c, ND_ERR_INVALID_ARG, "nd_propagator: needs the hermitian (two-sided) approximation of sign(Q)");
  auto t0 = std::chrono::steady_clock::now();
  const double abar = 1.0 / (1.0 + c->s), m = p->m_q;
  const double alpha = (1.0 + c->s) * (1.0 - 0.5 * abar * m);
  const double k = alpha * alpha + alpha * m;
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  void* b = field(c, "pr_b", 0);
  void* res = field(c, "pr_res", 0);
  void* x = field(c, "pr_x", 0);
  void* bc = field(c, "pr_bc", 0);
  void* y = field(c, "pr_y", 0);
  void* yc = field(c, "pr_yc", 0);
  void* r = field(c, "pr_r", 0);
  void* q = field(c, "pr_p", 0);
  void* w = field(c, "pr_w", 0);
  if (!b || !res || !x || !bc || !y || !yc || !r || !q || !w) return fail(c, ND_ERR_OOM, "nd_propagator: workspace");
  ND_TRY(nd_pack_spinor(c, b, b_in, ND_FP64, 1));
  ND_TRY_CUDA(c, cudaMemsetAsync(x, 0, fs, c->stream));
  ND_TRY_CUDA(c, cudaMemcpyAsync(res, b, fs, cudaMemcpyDeviceToDevice, c->stream));
  nd_status st = ND_OK;
  const double bn2 = dot_re(c, b, b, &st);
  if (st != ND_OK) return st;
  if (!std::isfinite(bn2)) return fail(c, ND_ERR_NAN, "nd_propagator: source has NaN or Inf");
  nd_prop_info inf{};
  double rel = bn2 > 0 ? 1.0 : 0.0, prev = 1e300;
  for (int sweep = 0; rel > tol; ++sweep) {
    if (sweep >= 20 || rel > 0.5 * prev) {
      ND_TRY(nd_unpack_spinor(c, x_out, x, ND_FP64, 1));
      inf.resid = rel;
      if (info) *info = inf;
      return fail(c, ND_ERR_NOT_CONVERGED, "nd_propagator: defect correction stagnates (sign(Q) too inaccurate for tol)");
    }
    prev = rel;
    // y = H^{-1} res, chirality by chirality; each CG reduces its part by tin, which takes the
    // residual of D^m x = b from rel to about tol / 2
    const double tin = 0.5 * tol / rel;
    ND_TRY_CUDA(c, cudaMemsetAsync(y, 0, fs, c->stream));
    for (int chir = 1; chir >= -1; chir -= 2) {
      // bc = P_c res = (res + c gamma5 res) / 2
      ND_TRY_CUDA(c, blas_g5_axpby(c->g, bc, 0.5, res, 0.5 * chir, res, c->stream));
      const double bc2 = dot_re(c, bc, bc, &st);
      if (st != ND_OK) return st;
      if (bc2 == 0.0) continue;
      ND_TRY_CUDA(c, cudaMemsetAsync(yc, 0, fs, c->stream));
      ND_TRY_CUDA(c, cudaMemcpyAsync(r, bc, fs, cudaMemcpyDeviceToDevice, c->stream));
      ND_TRY_CUDA(c, cudaMemcpyAsync(q, bc, fs, cudaMemcpyDeviceToDevice, c->stream));
      double rr = bc2;
      int it = 0;
      while (rr > tin * tin * bc2) {
        if (it >= maxit) {
          ND_TRY(nd_unpack_spinor(c, x_out, x, ND_FP64, 1));
          inf.iters += it;
          inf.resid = rel;
          if (info) *info = inf;
          return fail(c, ND_ERR_NOT_CONVERGED, "nd_propagator: CG iteration limit");
        }
        ND_TRY(apply_H(c, w, q, chir, k, m, p, &inf.sign_iters));
        const double pw = dot_re(c, q, w, &st);
        if (st != ND_OK) return st;
        if (!(pw > 0)) return fail(c, pw == pw ? ND_ERR_BREAKDOWN : ND_ERR_NAN, "nd_propagator: (p, H p) <= 0");
        const double a = rr / pw;
        ND_TRY_CUDA(c, blas_axpby(c->g, 0, yc, 1.0, yc, a, q, false, slot(c, nullptr), c->stream));
        ND_TRY_CUDA(c, blas_axpby(c->g, 0, r, 1.0, r, -a, w, true, slot(c, c->red_scratch), c->stream));
        double rr_new;
        ND_TRY(read_back(c, c->red_scratch, &rr_new, 1));
        ND_TRY_CUDA(c, blas_axpby(c->g, 0, q, 1.0, r, rr_new / rr, q, false, slot(c, nullptr), c->stream));
        rr = rr_new;
        ++it;
      }
      inf.iters += it;
      ND_TRY_CUDA(c, blas_axpby(c->g, 0, y, 1.0, y, 1.0, yc, false, slot(c, nullptr), c->stream));
    }
    // x += gamma5 D^m gamma5 y,  D^m v = alpha (v + gamma5 eps v) + m v
    void* z;
    nd_dn_info dinf{};
    ND_TRY_CUDA(c, blas_g5_axpby(c->g, w, 0.0, y, 1.0, y, c->stream));  // w = gamma5 y
    ND_TRY(sign_internal(c, w, p, &dinf, &z));
    inf.sign_iters += dinf.iters + dinf.degree;
    ND_TRY_CUDA(c, blas_g5_axpby(c->g, q, alpha + m, w, alpha, z, c->stream));  // q = D^m gamma5 y
    ND_TRY_CUDA(c, blas_g5_axpby(c->g, x, 1.0, x, 1.0, q, c->stream));         // x += gamma5 q
    // res = b - D^m x
    ND_TRY(sign_internal(c, x, p, &dinf, &z));
    inf.sign_iters += dinf.iters + dinf.degree;
    ND_TRY_CUDA(c, blas_g5_axpby(c->g, w, alpha + m, x, alpha, z, c->stream));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, res, 1.0, b, -1.0, w, true, slot(c, c->red_scratch), c->stream));
    double res2;
    ND_TRY(read_back(c, c->red_scratch, &res2, 1));
    rel = std::sqrt(res2 / bn2);
    ++inf.outer;
  }
  inf.resid = rel;
  ND_TRY(nd_unpack_spinor(c, x_out, x, ND_FP64, 1));
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return ND_OK;
}
