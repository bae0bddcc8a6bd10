// Even-odd (Schur complement) preconditioned Wilson operator and its use for (Q^2)^{-1}.
//
// The hopping term of D_W connects even and odd sites only (Sec. 2.1), so with D_ee = D_oo = 4 + m
//   Dhat = (4 + m) - D_eo D_oe / (4 + m)    (even sites),   Qhat = gamma5 Dhat   (hermitian),
//   D_W x = b  <=>  Dhat x_e = b_e - D_eo b_o / (4 + m),   x_o = (b_o - D_oe x_e) / (4 + m).
// Qhat is two one-parity launches of the stencil:
//   t_o = -D_oe in_e               (gamma5 left out, a = -1, diag 0)
//   out_e = gamma5 ((4+m)^2 in_e - 1/2 hop(t_o)) / (4 + m) = gamma5 ((4+m) in_e - D_eo D_oe in_e / (4+m))
// (the diagonal term reads in_e through a separate pointer, the hop reads the odd half of t).
// (Q^2)^{-1} phi = D_W^{-1} gamma5 D_W^{-1} gamma5 phi (Q^2 = D_W^dagger D_W); each D_W^{-1} is CG on
// Qhat^2 x_e = Qhat gamma5 bhat_e over the even sites (BLAS on half-size fields), in FP64 or with
// FP32 / FP16 correction solves refined in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "solver.h"

using namespace nd;

namespace {

Geom even_geom(const nd_ctx* c) {
  Geom g = c->g;
  g.even_only = 1;
  return g;
}

// One-parity stencil launch: out_p = a * [gamma5] (diag * din_p - 1/2 hop(in_{1-p})).
nd_status parity_launch(nd_ctx* c, int prec, int parity, void* out, const void* in, const void* din, double diag,
                        double a, bool g5) {
  if (!c->links[prec]) return fail(c, ND_ERR_STATE, "links are not set in the precision this call needs");
  QLaunch L{};
  L.prec = prec;
  L.recon = c->recon[prec];
  L.mode = Q_PLAIN;
  L.links = c->links[prec];
  L.in = in;
  L.din = din;
  L.out = out;
  L.diag = diag;
  L.a = a;
  L.no_g5 = g5 ? 0 : 1;
  L.parity0 = parity;
  L.nsites = (int)c->Vh;
  ND_TRY_CUDA(c, launch_q(c->g, L, c->stream));
  return ND_OK;
}

}  // namespace

namespace nd {

// out_e = Qhat in_e (fields of precision prec; odd halves of in and out are not touched).  With
// norms != null the second launch also reduces norms[0] = ||out_e||^2, norms[1] = ||in_e||^2.
nd_status qhat_apply(nd_ctx* c, int prec, void* out, const void* in, double* norms = nullptr) {
  void* t = field(c, "eo_t", prec);
  if (!t) return fail(c, ND_ERR_OOM, "Qhat: workspace");
  if (!c->links[prec]) return fail(c, ND_ERR_STATE, "links are not set in the precision this call needs");
  const double d = 4.0 + c->m;
  ND_TRY(parity_launch(c, prec, 1, t, in, nullptr, 0.0, -1.0, false));
  QLaunch L{};
  L.prec = prec;
  L.recon = c->recon[prec];
  L.mode = Q_PLAIN;
  L.reduce = norms != nullptr;
  L.links = c->links[prec];
  L.in = t;
  L.din = in;
  L.out = out;
  L.diag = d * d;
  L.a = 1.0 / d;
  L.parity0 = 0;
  L.nsites = (int)c->Vh;
  if (norms) L.slot = slot(c, norms);
  ND_TRY_CUDA(c, launch_q(c->g, L, c->stream));
  return ND_OK;
}

// x_e = (Qhat^2)^{-1} b_e by CG from x = 0 in precision prec, to ||b - Qhat^2 x|| <= tol ||b||.
// (p, Qhat^2 p) = ||Qhat p||^2 comes fused out of the first Qhat of each iteration.
nd_status cg_qhat2(nd_ctx* c, int prec, void* x, const void* b, double tol, int maxit, int* iters) {
  const Geom ge = even_geom(c);
  void* r = field(c, "eo_r", prec);
  void* p = field(c, "eo_p", prec);
  void* w = field(c, "eo_w", prec);
  void* q = field(c, "eo_q", prec);
  if (!r || !p || !w || !q) return fail(c, ND_ERR_OOM, "Qhat CG: workspace");
  double* red = c->red_scratch + 16;
  ND_TRY_CUDA(c, blas_axpby(ge, prec, x, 0.0, nullptr, 0.0, nullptr, false, slot(c, nullptr), c->stream));
  ND_TRY_CUDA(c, blas_axpby(ge, prec, r, 1.0, b, 0.0, nullptr, true, slot(c, red), c->stream));
  ND_TRY_CUDA(c, blas_axpby(ge, prec, p, 1.0, r, 0.0, nullptr, false, slot(c, nullptr), c->stream));
  double rr;
  ND_TRY(read_back(c, red, &rr, 1));
  if (!std::isfinite(rr)) return fail(c, ND_ERR_NAN, "Qhat CG: right-hand side has NaN or Inf");
  const double stop = tol * tol * rr;
  int it = 0;
  while (rr > stop) {
    if (it >= maxit) {
      *iters += it;
      return fail(c, ND_ERR_NOT_CONVERGED, "Qhat CG: iteration limit");
    }
    double nq[2];
    ND_TRY(qhat_apply(c, prec, q, p, red));
    ND_TRY(qhat_apply(c, prec, w, q));
    ND_TRY(read_back(c, red, nq, 2));
    if (!(nq[0] > 0)) return fail(c, nq[0] == nq[0] ? ND_ERR_BREAKDOWN : ND_ERR_NAN, "Qhat CG: (p, Qhat^2 p) <= 0");
    const double a = rr / nq[0];
    ND_TRY_CUDA(c, blas_axpby(ge, prec, x, 1.0, x, a, p, false, slot(c, nullptr), c->stream));
    ND_TRY_CUDA(c, blas_axpby(ge, prec, r, 1.0, r, -a, w, true, slot(c, red), c->stream));
    double rr_new;
    ND_TRY(read_back(c, red, &rr_new, 1));
    ND_TRY_CUDA(c, blas_axpby(ge, prec, p, 1.0, r, rr_new / rr, p, false, slot(c, nullptr), c->stream));
    rr = rr_new;
    ++it;
  }
  *iters += it;
  return ND_OK;
}

// out = D_W^{-1} v (whole-lattice fields of precision prec): Schur complement on the even sites.
nd_status dw_inverse(nd_ctx* c, int prec, void* out, const void* v, double tol, int maxit, int* iters) {
  const double d = 4.0 + c->m;
  void* gb = field(c, "eo_gb", prec);
  void* rhs = field(c, "eo_rhs", prec);
  if (!gb || !rhs) return fail(c, ND_ERR_OOM, "D_W solve: workspace");
  // gamma5 bhat_e = gamma5 (v_e - D_eo v_o / (4 + m)) = (-1/(4+m)) gamma5 (-(4+m) v_e - 1/2 hop(v_o))
  ND_TRY(parity_launch(c, prec, 0, gb, v, v, -d, -1.0 / d, true));
  ND_TRY(qhat_apply(c, prec, rhs, gb));  // Qhat gamma5 bhat_e: Qhat^2 x_e = rhs <=> Dhat x_e = bhat_e
  ND_TRY(cg_qhat2(c, prec, out, rhs, tol, maxit, iters));
  // x_o = (v_o - D_oe x_e) / (4 + m) = (-1/(4+m)) (-v_o - 1/2 hop(x_e))
  ND_TRY(parity_launch(c, prec, 1, out, out, v, -1.0, -1.0 / d, false));
  return ND_OK;
}

}  // namespace nd

extern "C" nd_status nd_apply_Qhat(nd_ctx* c, void* out, const void* in, nd_prec prec) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (!out || !in || out == in || prec < ND_FP64 || prec > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Qhat: bad arguments (out and in must differ)");
  if (!(4.0 + c->m != 0.0)) return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Qhat: 4 + m must not vanish");
  return qhat_apply(c, (int)prec, out, in);
}

extern "C" nd_status nd_solve_Q2_eo(nd_ctx* c, double* x_out, const double* b_in, double tol, int maxit, nd_prec inner,
                                    nd_solve_info* info) {
  NvtxRange range("nd.solve_q2_eo");
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (!x_out || !b_in || x_out == b_in || !(tol > 0) || maxit < 1 || inner < ND_FP64 || inner > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_solve_Q2_eo: bad arguments");
  if (!c->links[0] || !c->links[inner]) return fail(c, ND_ERR_STATE, "nd_solve_Q2_eo: links not set (FP64 and inner)");
  auto t0 = std::chrono::steady_clock::now();
  const int ps = (int)inner;
  void* b = field(c, "eo_b64", 0);
  void* x = field(c, "eo_x64", 0);
  void* r = field(c, "eo_r64", 0);
  void* vs = field(c, "eo_vs", ps);
  void* ys = field(c, "eo_ys", ps);
  void* es = field(c, "eo_es", ps);
  if (!b || !x || !r || !vs || !ys || !es) return fail(c, ND_ERR_OOM, "nd_solve_Q2_eo: workspace");
  ND_TRY(nd_pack_spinor(c, b, b_in, ND_FP64, 1));
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, b, 1.0, b, 0.0, nullptr, true, slot(c, c->red_scratch), c->stream));
  double bn2;
  ND_TRY(read_back(c, c->red_scratch, &bn2, 1));
  if (!std::isfinite(bn2)) return fail(c, ND_ERR_NAN, "nd_solve_Q2_eo: source has NaN or Inf");
  nd_solve_info inf{};
  ND_TRY_CUDA(c, cudaMemsetAsync(x, 0, (size_t)spinor_bytes(0, c->Vh), c->stream));
  // FP64 defect correction on Q^2: r = b - Q^2 x; e = D_W^{-1} gamma5 D_W^{-1} gamma5 r in the inner
  // precision (each D_W^{-1} to tin relative on its normal equations); x += e
  const double floor_in = ps == 0 ? 0.0 : (ps == 1 ? 1e-5 : 1e-3);
  double rel = bn2 > 0 ? 1.0 : 0.0, prev = 1e300;
  ND_TRY_CUDA(c, cudaMemcpyAsync(r, b, (size_t)spinor_bytes(0, c->Vh), cudaMemcpyDeviceToDevice, c->stream));
  for (int sweep = 0; rel > tol; ++sweep) {
    if (sweep >= 40 || rel > 0.5 * prev) {
      ND_TRY(nd_unpack_spinor(c, x_out, x, ND_FP64, 1));
      inf.max_resid = rel;
      if (info) *info = inf;
      return fail(c, ND_ERR_NOT_CONVERGED, "nd_solve_Q2_eo: defect correction stagnates");
    }
    prev = rel;
    const double tin = std::max(0.1 * tol / rel, floor_in);
    // r <- gamma5 r / ||r||: unit norm before the inner precision (no subnormal products there)
    const double rn = rel * std::sqrt(bn2);
    ND_TRY_CUDA(c, blas_g5_axpby(c->g, r, 0.0, r, 1.0 / rn, r, c->stream));
    ND_TRY_CUDA(c, blas_convert(c->g, ps, vs, 0, r, c->stream));
    ND_TRY(dw_inverse(c, ps, ys, vs, tin, maxit, &inf.iters));
    ND_TRY_CUDA(c, blas_g5(c->g, ps, ys, ys, c->stream));
    ND_TRY(dw_inverse(c, ps, es, ys, tin, maxit, &inf.iters));
    ND_TRY_CUDA(c, blas_convert(c->g, 0, r, ps, es, c->stream));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, x, 1.0, x, rn, r, false, slot(c, nullptr), c->stream));
    ND_TRY(residual64(c, r, b, x, 0.0, 1.0, bn2, &rel));
    ++inf.outer;
  }
  inf.max_resid = rel;
  inf.sloppy_iters = ps == 0 ? 0 : inf.iters;
  ND_TRY(nd_unpack_spinor(c, x_out, x, ND_FP64, 1));
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return ND_OK;
}
