// Device side of the multi-shift conjugate gradient (B. Jegerlehner, hep-lat/9612014):
// the scalar recurrences run in a one-warp kernel on device-resident state, so an iteration
// is four launches with no host round trip:
//   K1  t = Q p_0                         (Q kernel, fused ||t||^2, ||p_0||^2)
//   K2  r -= alpha (ascale Q t + sigma_0 p_0)  (Q kernel in CG mode, fused ||r||^2)
//   K3  zeta, alpha_l, beta_l, convergence  (mscg_scalar_kernel)
//   K4  x_l += alpha_l p_l, p_l = zeta_l r + beta_l p_l for every live shift  (mscg_update_kernel)
// with alpha = (r, r) / (p_0, (A + sigma_0) p_0), (p_0, A p_0) = ascale ||Q p_0||^2 since Q is
// hermitian, and the shifted recurrence
//   zeta_l' = zeta_l zeta_l^- alpha^- / [alpha beta^- (zeta_l^- - zeta_l) + zeta_l^- alpha^- (1 + (sigma_l - sigma_0) alpha)],
//   alpha_l = alpha zeta_l' / zeta_l,  beta_l = beta (zeta_l' / zeta_l)^2.
// Shift 0 is the smallest shift (the base system); it stays live until the run ends.
// Stopping: shift l freezes once |zeta_l'| ||r|| <= tol_l ||b||; the run ends after the
// iteration in which the last shift froze (CG_PENDING), or at once on a breakdown / NaN
// (CG_DONE), or after maxit iterations (CG_PENDING with ND_ERR_NOT_CONVERGED).
#include <math.h>

#include "../../include/nd.h"
#include "fields.cuh"
#include "kernels.h"

namespace nd {

__global__ void mscg_init_kernel(double* s, int n) {
  const int l = threadIdx.x;
  if (l < CG_NMAX) {
    const bool on = l < n;
    s[sh(SH_ZETA, l)] = 1.0;
    s[sh(SH_ZETAP, l)] = 1.0;
    s[sh(SH_ACTIVE, l)] = on ? 1.0 : 0.0;
    s[sh(SH_LIVE, l)] = on ? 1.0 : 0.0;
    s[sh(SH_UPD, l)] = 0.0;
    s[sh(SH_COEFX, l)] = 0.0;
    s[sh(SH_RES, l)] = 1.0;
  }
  if (l == 0) {
    s[CG_DONE] = 0.0;
    s[CG_PENDING] = 0.0;
    s[CG_STATUS] = (double)ND_OK;
    s[CG_ITER] = 0.0;
    s[CG_ALPHA_PREV] = 1.0;
    s[CG_BETA_PREV] = 0.0;
    s[CG_BNORM2] = s[CG_RR];
    s[CG_SIGMA0] = s[sh(SH_SIGMA, 0)];
    if (!(s[CG_RR] > 0.0)) {  // zero (or NaN) source: nothing to do
      s[CG_PENDING] = 1.0;
      if (s[CG_RR] != 0.0) {
        s[CG_DONE] = 1.0;
        s[CG_STATUS] = (double)ND_ERR_NAN;
      }
    }
  }
}

template <bool GRAPH>
__global__ void mscg_scalar_kernel(double* s, int n, int maxit, cudaGraphConditionalHandle h) {
  if (s[CG_DONE] != 0.0 || s[CG_PENDING] != 0.0) {
    // the update of the iteration that set PENDING has been applied: stop everything now,
    // so the update kernels of further (already launched) iterations skip as well
    if (threadIdx.x == 0) {
      s[CG_DONE] = 1.0;
      if (GRAPH) cudaGraphSetConditional(h, 0);
    }
    return;
  }
  const int l = threadIdx.x;
  const double rr = s[CG_RR], rrn = s[CG_RRNEW];
  const double den = s[CG_ASCALE] * s[CG_TT] + s[CG_SIGMA0] * s[CG_PP];
  const double alpha = rr / den;
  const double beta = rrn / rr;
  const double ap = s[CG_ALPHA_PREV], bp = s[CG_BETA_PREV];
  const double s0 = s[CG_SIGMA0];
  const double rnorm_rel = sqrt(rrn / s[CG_BNORM2]);
  int active_after = 0;
  if (l < n) {
    const bool active = s[sh(SH_ACTIVE, l)] != 0.0;
    const bool live = active || l == 0;
    s[sh(SH_UPD, l)] = active ? 1.0 : 0.0;
    s[sh(SH_LIVE, l)] = live ? 1.0 : 0.0;
    if (live) {
      const double z = s[sh(SH_ZETA, l)], zp = s[sh(SH_ZETAP, l)];
      const double ds = s[sh(SH_SIGMA, l)] - s0;
      const double zn = z * zp * ap / (alpha * bp * (zp - z) + zp * ap * (1.0 + ds * alpha));
      const double q = zn / z;
      s[sh(SH_COEFX, l)] = active ? alpha * q : 0.0;
      s[sh(SH_COEFR, l)] = zn;
      s[sh(SH_COEFP, l)] = beta * q * q;
      s[sh(SH_ZETAP, l)] = z;
      s[sh(SH_ZETA, l)] = zn;
      if (active) {
        const double res = fabs(zn) * rnorm_rel;
        s[sh(SH_RES, l)] = res;
        if (res <= s[sh(SH_TOL, l)]) s[sh(SH_ACTIVE, l)] = 0.0;
        else active_after = 1;
      }
    }
  }
  active_after = __syncthreads_or(active_after);
  if (l == 0) {
    const double it = s[CG_ITER] + 1.0;
    s[CG_ITER] = it;
    s[CG_ALPHA_PREV] = alpha;
    s[CG_BETA_PREV] = beta;
    s[CG_RR] = rrn;
    if (!(den > 0.0) || !isfinite(den)) {
      s[CG_DONE] = 1.0;
      s[CG_STATUS] = isfinite(den) ? (double)ND_ERR_BREAKDOWN : (double)ND_ERR_NAN;
    } else if (!isfinite(rrn)) {
      s[CG_DONE] = 1.0;
      s[CG_STATUS] = (double)ND_ERR_NAN;
    } else if (!active_after || rrn == 0.0) {
      s[CG_PENDING] = 1.0;
    } else if (it >= (double)maxit) {
      s[CG_PENDING] = 1.0;
      s[CG_STATUS] = (double)ND_ERR_NOT_CONVERGED;
    }
    // in a graph the while-loop ends after this iteration's update kernel
    if (GRAPH && (s[CG_DONE] != 0.0 || s[CG_PENDING] != 0.0)) cudaGraphSetConditional(h, 0);
  }
}

template <int PS, int PX, bool YMODE>
__global__ void __launch_bounds__(256) mscg_update_kernel(const Geom g, const void* r, char* p_all, size_t pstride,
                                                          char* x_all, size_t xstride, void* y, const double* s,
                                                          int n) {
  using T = typename Traits<PS>::real;
  using TX = typename Traits<PX>::real;
  if (s[CG_DONE] != 0.0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh) return;
  const int p = i >= g.Vh ? 1 : 0, h = i - p * g.Vh;
  Spinor<T> vr;
  SpinorIO<PS>::load(vr, r, g.Vh, p, h);
  Spinor<TX> vy;
  if (YMODE) SpinorIO<PX>::load(vy, y, g.Vh, p, h);
  for (int l = 0; l < n; ++l) {
    if (s[sh(SH_LIVE, l)] == 0.0) continue;
    Spinor<T> vp;
    void* pl = p_all + l * pstride;
    SpinorIO<PS>::load(vp, pl, g.Vh, p, h);
    if (s[sh(SH_UPD, l)] != 0.0) {
      const double ax = s[sh(SH_COEFX, l)];
      if (YMODE) {
        const TX c = (TX)(ax * s[sh(SH_W, l)]);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int k = 0; k < 3; ++k)
            vy.s[a][k] = vy.s[a][k] + c * mk((TX)vp.s[a][k].re, (TX)vp.s[a][k].im);
      } else {
        void* xl = x_all + l * xstride;
        Spinor<TX> vx;
        SpinorIO<PX>::load(vx, xl, g.Vh, p, h);
        const TX c = (TX)ax;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int k = 0; k < 3; ++k)
            vx.s[a][k] = vx.s[a][k] + c * mk((TX)vp.s[a][k].re, (TX)vp.s[a][k].im);
        SpinorIO<PX>::store(vx, xl, g.Vh, p, h);
      }
    }
    const T cr = (T)s[sh(SH_COEFR, l)], cp = (T)s[sh(SH_COEFP, l)];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) vp.s[a][k] = cr * vr.s[a][k] + cp * vp.s[a][k];
    SpinorIO<PS>::store(vp, pl, g.Vh, p, h);
  }
  if (YMODE) SpinorIO<PX>::store(vy, y, g.Vh, p, h);
}

cudaError_t mscg_init(double* state, int n, cudaStream_t st) {
  mscg_init_kernel<<<1, CG_NMAX, 0, st>>>(state, n);
  return cudaGetLastError();
}

cudaError_t mscg_scalar(double* state, int n, int maxit, cudaStream_t st) {
  mscg_scalar_kernel<false><<<1, CG_NMAX, 0, st>>>(state, n, maxit, cudaGraphConditionalHandle{});
  return cudaGetLastError();
}

cudaError_t mscg_scalar_graph(double* state, int n, int maxit, cudaGraphConditionalHandle h, cudaStream_t st) {
  mscg_scalar_kernel<true><<<1, CG_NMAX, 0, st>>>(state, n, maxit, h);
  return cudaGetLastError();
}

cudaError_t mscg_update(const Geom& g, int ps, int px, bool ymode, const void* r, void* p_all, size_t pstride,
                        void* x_all, size_t xstride, void* y, const double* state, int n, cudaStream_t st) {
  const int blocks = (2 * g.Vh + 255) / 256;
  char* pa = static_cast<char*>(p_all);
  char* xa = static_cast<char*>(x_all);
#define UPD(A, B, Y)                                                                                     \
  if (ps == A && px == B && ymode == Y) {                                                                \
    mscg_update_kernel<A, B, Y><<<blocks, 256, 0, st>>>(g, r, pa, pstride, xa, xstride, y, state, n);    \
    return cudaGetLastError();                                                                           \
  }
  UPD(P64, P64, false) UPD(P64, P64, true) UPD(P32, P32, false) UPD(P32, P32, true) UPD(P16, P32, false)
  UPD(P16, P32, true) UPD(P16, P16, false)
#undef UPD
  return cudaErrorInvalidValue;
}

}  // namespace nd
