// Force of the pseudofermion action S = phi^dagger (Q^2)^{-1} phi with respect to the links.
//
// With X = (Q^2)^{-1} phi and Y = Q X, dS = -2 Re(Y^dagger dQ X), and dQ = -1/2 gamma5 dH follows
// from the definition of D_W (Sec. 2.1).  For U_mu(x) -> exp(i w T^a) U_mu(x), T^a = lambda^a/2:
//   dS/dw = -Im tr[T^a (A1 - A2)],
//   A1 = U_mu(x) sum_alpha [(1 - gamma_mu) X(x+mu)]_alpha [gamma5 Y(x)]_alpha^dagger,
//   A2 = sum_alpha [(1 + gamma_mu) X(x)]_alpha [U_mu(x) gamma5 Y(x+mu)]_alpha^dagger.
// One FP64 thread per link; the spin projections use the same half-spinor algebra as the
// stencil.  X comes from a CG solve that is recomputed for every force evaluation.
#include <chrono>
#include <cmath>

#include "dslash.cuh"
#include "solver.h"

namespace nd {

template <int MU>
__device__ __forceinline__ void force_link(const Geom& g, const Site& s, int p, int h, const char* links,
                                           const void* X, const void* Y, double* F) {
  using T = double;
  bool crossed;
  const int hf = neighbour_h<MU, true>(g, s, &crossed);
  const T sgn = (g.apbc && crossed) ? -1.0 : 1.0;
  Spinor<T> xf, xx, yx, yf;
  SpinorIO<P64>::load(xf, X, g.Vh, 1 - p, hf);
  SpinorIO<P64>::load(xx, X, g.Vh, p, h);
  SpinorIO<P64>::load(yx, Y, g.Vh, p, h);
  SpinorIO<P64>::load(yf, Y, g.Vh, 1 - p, hf);
  LinkRaw<P64, 18> raw;
  load_raw<P64, 18>(raw, links, g.Vh, p, MU, h);
  Su3<T> U;
  reconstruct<P64, 18>(U, raw);
  // a = (1 - gamma_mu) X(x+mu) (times the boundary sign), c = (1 + gamma_mu) X(x)
  cx<T> hs[2][3];
  Spinor<T> a, cc;
  spin_project<MU, true>(xf, hs);
#pragma unroll
  for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
    for (int i = 0; i < 3; ++i) a.s[a2][i] = mk(0.0, 0.0);
  spin_accumulate<MU, true>(a, hs);
  spin_project<MU, false>(xx, hs);
#pragma unroll
  for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
    for (int i = 0; i < 3; ++i) cc.s[a2][i] = mk(0.0, 0.0);
  spin_accumulate<MU, false>(cc, hs);
  // gamma5 Y
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    yx.s[2][i] = -yx.s[2][i];
    yx.s[3][i] = -yx.s[3][i];
    yf.s[2][i] = -yf.s[2][i];
    yf.s[3][i] = -yf.s[3][i];
  }
  // d_alpha = U (gamma5 Y(x+mu))_alpha
  Spinor<T> d;
#pragma unroll
  for (int al = 0; al < 4; ++al)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      cx<T> v = mk(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < 3; ++j) cfma(v, U.e[i][j], yf.s[al][j]);
      d.s[al][i] = v;
    }
  // B = sum_alpha a_alpha (g5 Y(x))_alpha^dagger; A2 = sum_alpha c_alpha d_alpha^dagger (both times sgn)
  cx<T> B[3][3], M[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> b = mk(0.0, 0.0), a2 = mk(0.0, 0.0);
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        cfmac(b, yx.s[al][j], a.s[al][i]);   // a_i conj(g_j)
        cfmac(a2, d.s[al][j], cc.s[al][i]);  // c_i conj(d_j)
      }
      B[i][j] = sgn * b;
      M[i][j] = -(sgn * a2);
    }
  // M = U B - A2
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> v = M[i][j];
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma(v, U.e[i][k], B[k][j]);
      M[i][j] = v;
    }
  // F^a = -Im tr[(lambda^a / 2) M],  tr[lambda M] = sum_ij lambda_ij M_ji
  const double r3 = 0.57735026918962576451;
  double f[8];
  f[0] = M[1][0].im + M[0][1].im;                                    // lambda1
  f[1] = -M[1][0].re + M[0][1].re;                                   // lambda2: Im(-i M10 + i M01)
  f[2] = M[0][0].im - M[1][1].im;                                    // lambda3
  f[3] = M[2][0].im + M[0][2].im;                                    // lambda4
  f[4] = -M[2][0].re + M[0][2].re;                                   // lambda5
  f[5] = M[2][1].im + M[1][2].im;                                    // lambda6
  f[6] = -M[2][1].re + M[1][2].re;                                   // lambda7
  f[7] = r3 * (M[0][0].im + M[1][1].im - 2.0 * M[2][2].im);          // lambda8
  double* o = F + ((int64_t)MU * 2 * g.Vh + s.lex) * 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) o[k] = -0.5 * f[k];
}

// Euclidean gradient of S with respect to the complex link matrix (U treated as a general 3x3
// matrix, U^dagger in the backward hops as its conjugate transpose):
//   dS = Re sum_{x,mu} tr(dU_mu(x) K_mu(x)),  K = M1 + M2^dagger,
//   M1 = sum_alpha [(1 - gamma_mu) X(x+mu)]_alpha [gamma5 Y(x)]_alpha^dagger,
//   M2 = sum_alpha [(1 + gamma_mu) X(x)]_alpha [gamma5 Y(x+mu)]_alpha^dagger,
// (from dS = -2 Re Y^dagger dQ X, dQ = -1/2 gamma5 dH).  Stored as G = K^dagger / 2 = dS/dU^*,
// the conjugate Wirtinger derivative: dS = 2 Re sum conj(G_ij) dU_ij.
template <int MU>
__device__ __forceinline__ void gradient_link(const Geom& g, const Site& s, int p, int h, const void* X, const void* Y,
                                              double* G) {
  using T = double;
  bool crossed;
  const int hf = neighbour_h<MU, true>(g, s, &crossed);
  const T sgn = (g.apbc && crossed) ? -1.0 : 1.0;
  Spinor<T> xf, xx, yx, yf;
  SpinorIO<P64>::load(xf, X, g.Vh, 1 - p, hf);
  SpinorIO<P64>::load(xx, X, g.Vh, p, h);
  SpinorIO<P64>::load(yx, Y, g.Vh, p, h);
  SpinorIO<P64>::load(yf, Y, g.Vh, 1 - p, hf);
  cx<T> hs[2][3];
  Spinor<T> a, cc;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a.s[k][i] = mk(0.0, 0.0);
      cc.s[k][i] = mk(0.0, 0.0);
    }
  spin_project<MU, true>(xf, hs);
  spin_accumulate<MU, true>(a, hs);
  spin_project<MU, false>(xx, hs);
  spin_accumulate<MU, false>(cc, hs);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    yx.s[2][i] = -yx.s[2][i];
    yx.s[3][i] = -yx.s[3][i];
    yf.s[2][i] = -yf.s[2][i];
    yf.s[3][i] = -yf.s[3][i];
  }
  double* o = G + ((int64_t)MU * 2 * g.Vh + s.lex) * 18;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // K_ij = (M1)_ij + conj((M2)_ji);  G_ij = conj(K_ji) / 2
      //      => G_ij = (conj(M1_ji) + M2_ij) / 2
      cx<T> m1ji = mk(0.0, 0.0), m2ij = mk(0.0, 0.0);
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        cfmac(m1ji, yx.s[al][i], a.s[al][j]);   // a_j conj(g5Y(x)_i)
        cfmac(m2ij, yf.s[al][j], cc.s[al][i]);  // c_i conj(g5Y(x+mu)_j)
      }
      o[2 * (3 * i + j)] = 0.5 * sgn * (m1ji.re + m2ij.re);
      o[2 * (3 * i + j) + 1] = 0.5 * sgn * (-m1ji.im + m2ij.im);
    }
}

__global__ void __launch_bounds__(128) gradient_kernel(const Geom g, const void* X, const void* Y, double* G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh * 4) return;
  const int mu = i & 3, site = i >> 2;
  const int p = site & 1, h = site >> 1;
  const Site s = site_of(g, p, h);
  switch (mu) {
    case 0: gradient_link<0>(g, s, p, h, X, Y, G); break;
    case 1: gradient_link<1>(g, s, p, h, X, Y, G); break;
    case 2: gradient_link<2>(g, s, p, h, X, Y, G); break;
    case 3: gradient_link<3>(g, s, p, h, X, Y, G); break;
  }
}

__global__ void __launch_bounds__(128) force_kernel(const Geom g, const char* links, const void* X, const void* Y,
                                                    double* F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh * 4) return;
  const int mu = i & 3, site = i >> 2;
  const int p = site & 1, h = site >> 1;
  const Site s = site_of(g, p, h);
  switch (mu) {
    case 0: force_link<0>(g, s, p, h, links, X, Y, F); break;
    case 1: force_link<1>(g, s, p, h, links, X, Y, F); break;
    case 2: force_link<2>(g, s, p, h, links, X, Y, F); break;
    case 3: force_link<3>(g, s, p, h, links, X, Y, F); break;
  }
}

}  // namespace nd

using namespace nd;

// X = (Q^2)^{-1} phi (FP64 or mixed), Y = Q X, and S = Re phi^dagger X; fields in the context's
// workspaces "fo_X", "fo_Y".
static nd_status solve_action(nd_ctx* c, const double* phi, double tol, int maxit, nd_prec inner, void** Xo, void** Yo,
                              double* S, nd_solve_info* info) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (!phi || !(tol > 0) || maxit < 1 || inner < ND_FP64 || inner > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "force: bad argument");
  if (c->recon[0] != 18 || !c->links[inner] || (inner != ND_FP64 && !c->links[1]))
    return fail(c, ND_ERR_STATE, "force: needs FP64 links with 18 reals (and the inner precision)");
  auto t0 = std::chrono::steady_clock::now();
  void* b64 = field(c, "fo_b", 0);
  void* X = field(c, "fo_X", 0);
  void* Y = field(c, "fo_Y", 0);
  if (!b64 || !X || !Y) return fail(c, ND_ERR_OOM, "force: workspace");
  ND_TRY(nd_pack_spinor(c, b64, phi, ND_FP64, 1));
  double bn2;
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, b64, 1.0, b64, 0.0, nullptr, true, slot(c, c->red_scratch), c->stream));
  ND_TRY(read_back(c, c->red_scratch, &bn2, 1));
  if (!std::isfinite(bn2)) return fail(c, ND_ERR_NAN, "force: source has NaN or Inf");
  nd_solve_info inf{};
  if (bn2 == 0.0) {
    ND_TRY_CUDA(c, cudaMemsetAsync(X, 0, (size_t)spinor_bytes(0, c->Vh), c->stream));
  } else if (inner == ND_FP64) {
    MsResult ms;
    ND_TRY(mscg_run(c, 0, 0, false, b64, X, {0.0}, {tol}, {}, 1.0, maxit, &ms));
    inf.iters = inf.sloppy_iters = ms.iters;
    double rel;
    ND_TRY(residual64(c, Y, b64, X, 0.0, 1.0, bn2, &rel));
    inf.max_resid = rel;
  } else {
    MixedStats ms;
    auto sink = [&](int, void* x64) -> nd_status {
      ND_TRY_CUDA(c, cudaMemcpyAsync(X, x64, (size_t)spinor_bytes(0, c->Vh), cudaMemcpyDeviceToDevice, c->stream));
      return ND_OK;
    };
    ND_TRY(mixed_solve(c, (int)inner, b64, bn2, {0.0}, {tol}, 1.0, maxit, &ms, sink));
    inf.iters = ms.iters;
    inf.sloppy_iters = ms.sloppy_iters;
    inf.outer = ms.outer;
    inf.max_resid = ms.max_resid;
  }
  ND_TRY(q_apply(c, 0, Y, X));
  if (S) {
    ND_TRY_CUDA(c, blas_dot(c->g, 0, b64, X, slot(c, c->red_scratch), c->stream));
    double d[3];
    ND_TRY(read_back(c, c->red_scratch, d, 3));
    *S = d[0];
  }
  inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  *Xo = X;
  *Yo = Y;
  return ND_OK;
}

extern "C" nd_status nd_force(nd_ctx* c, double* F, const double* phi, double tol, int maxit, nd_prec inner,
                              nd_solve_info* info) {
  NvtxRange range("nd.force");
  if (c && !F) return fail(c, ND_ERR_INVALID_ARG, "nd_force: null output");
  void *X, *Y;
  ND_TRY(solve_action(c, phi, tol, maxit, inner, &X, &Y, nullptr, info));
  const int n = (int)(4 * c->V);
  force_kernel<<<(n + 127) / 128, 128, 0, c->stream>>>(c->g, static_cast<const char*>(c->links[0]), X, Y, F);
  ND_TRY_CUDA(c, cudaGetLastError());
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  return ND_OK;
}

extern "C" nd_status nd_link_gradient(nd_ctx* c, double* G, double* Xout, double* S, const double* phi, double tol,
                                      int maxit, nd_prec inner, nd_solve_info* info) {
  NvtxRange range("nd.link_gradient");
  if (c && !G) return fail(c, ND_ERR_INVALID_ARG, "nd_link_gradient: null output");
  void *X, *Y;
  ND_TRY(solve_action(c, phi, tol, maxit, inner, &X, &Y, S, info));
  if (Xout) ND_TRY(nd_unpack_spinor(c, Xout, X, ND_FP64, 1));
  const int n = (int)(4 * c->V);
  gradient_kernel<<<(n + 127) / 128, 128, 0, c->stream>>>(c->g, X, Y, G);
  ND_TRY_CUDA(c, cudaGetLastError());
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  return ND_OK;
}
