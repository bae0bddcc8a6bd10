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
#include <algorithm>
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
    s[CG_LIVE_SUM] = 0.0;
    s[CG_ACTIVE_SUM] = 0.0;
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
  const bool active = l < n && s[sh(SH_ACTIVE, l)] != 0.0;
  const bool live = l < n && (active || l == 0);
  // work counters of this iteration's update kernel (read by the host for the byte count)
  const int n_live = __syncthreads_count(live), n_active = __syncthreads_count(active);
  if (l < n) {
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
    s[CG_LIVE_SUM] += (double)n_live;
    s[CG_ACTIVE_SUM] += (double)n_active;
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

// ---------------------------------------------------------------- batched CG
// nsys independent systems (A + sigma_s) x_s = b_s, each with its own scalar block laid out as
// the multi-shift state with one shift.  The recurrences are those of plain CG (zeta = 1):
// alpha = (r, r) / (p, (A + sigma) p), beta = (r, r)_new / (r, r).

namespace nd {

__global__ void bcg_init_kernel(double* states, int nsys) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  double* st = states + (int64_t)s * CG_STATE_DOUBLES;
  st[sh(SH_ZETA, 0)] = 1.0;
  st[sh(SH_ZETAP, 0)] = 1.0;
  st[sh(SH_ACTIVE, 0)] = 1.0;
  st[sh(SH_RES, 0)] = 1.0;
  st[CG_DONE] = 0.0;
  st[CG_PENDING] = 0.0;
  st[CG_STATUS] = (double)ND_OK;
  st[CG_ITER] = 0.0;
  st[CG_BNORM2] = st[CG_RR];
  st[CG_SIGMA0] = st[sh(SH_SIGMA, 0)];
  if (!(st[CG_RR] > 0.0)) {
    st[CG_PENDING] = 1.0;
    if (st[CG_RR] != 0.0) {
      st[CG_DONE] = 1.0;
      st[CG_STATUS] = (double)ND_ERR_NAN;
    }
  }
}

template <bool GRAPH>
__global__ void bcg_scalar_kernel(double* states, int nsys, int maxit, cudaGraphConditionalHandle h) {
  const int s = threadIdx.x;
  int running = 0;
  if (s < nsys) {
    double* st = states + (int64_t)s * CG_STATE_DOUBLES;
    if (st[CG_DONE] != 0.0 || st[CG_PENDING] != 0.0) {
      st[CG_DONE] = 1.0;  // its last update has been applied
    } else {
      const double rr = st[CG_RR], rrn = st[CG_RRNEW];
      const double den = st[CG_ASCALE] * st[CG_TT] + st[CG_SIGMA0] * st[CG_PP];
      const double alpha = rr / den, beta = rrn / rr;
      st[sh(SH_UPD, 0)] = 1.0;
      st[sh(SH_COEFX, 0)] = alpha;
      st[sh(SH_COEFR, 0)] = 1.0;
      st[sh(SH_COEFP, 0)] = beta;
      const double res = sqrt(rrn / st[CG_BNORM2]);
      st[sh(SH_RES, 0)] = res;
      const double it = st[CG_ITER] + 1.0;
      st[CG_ITER] = it;
      st[CG_RR] = rrn;
      if (!(den > 0.0) || !isfinite(den)) {
        st[CG_DONE] = 1.0;
        st[CG_STATUS] = isfinite(den) ? (double)ND_ERR_BREAKDOWN : (double)ND_ERR_NAN;
      } else if (!isfinite(rrn)) {
        st[CG_DONE] = 1.0;
        st[CG_STATUS] = (double)ND_ERR_NAN;
      } else if (res <= st[sh(SH_TOL, 0)] || rrn == 0.0) {
        st[CG_PENDING] = 1.0;
      } else if (it >= (double)maxit) {
        st[CG_PENDING] = 1.0;
        st[CG_STATUS] = (double)ND_ERR_NOT_CONVERGED;
      }
      running = st[CG_DONE] == 0.0 && st[CG_PENDING] == 0.0;
    }
  }
  running = __syncthreads_or(running);
  // the while-loop ends after the update kernel of the iteration in which the last system
  // stopped
  if (GRAPH && threadIdx.x == 0 && !running) cudaGraphSetConditional(h, 0);
}

// x += alpha p, p = r + beta p for every system that has not stopped.  A grid of resident blocks
// strides over the (site block, running system) items.
template <int PS>
__global__ void __launch_bounds__(256) bcg_update_kernel(const Geom g, const char* r, char* p, char* x, size_t fstride,
                                                         const double* states, int nsys) {
  using T = typename Traits<PS>::real;
  // the systems still updating (CG_DONE does not change during the launch), listed once per block
  __shared__ short running[ND_BATCH_MAX_SYSTEMS];
  __shared__ int nrun;
  if (threadIdx.x < 32) {
    int base = 0;
    for (int c = 0; c < nsys; c += 32) {
      const int sys = c + (int)threadIdx.x;
      const bool go = sys < nsys && states[(int64_t)sys * CG_STATE_DOUBLES + CG_DONE] == 0.0;
      const unsigned m = __ballot_sync(0xffffffffu, go);
      if (go) running[base + __popc(m & ((1u << threadIdx.x) - 1u))] = (short)sys;
      base += __popc(m);
    }
    if (threadIdx.x == 0) nrun = base;
  }
  __syncthreads();
  const int bps = (2 * g.Vh + 255) / 256, nr = nrun;
  for (int item = blockIdx.x; item < bps * nr; item += gridDim.x) {
    const int sys = running[item % nr], blk = item / nr;
    const double* st = states + (int64_t)sys * CG_STATE_DOUBLES;
    const int i = blk * 256 + threadIdx.x;
    if (i >= 2 * g.Vh) continue;
    const int pp = i >= g.Vh ? 1 : 0, h = i - pp * g.Vh;
    const size_t off = (size_t)sys * fstride;
    Spinor<T> vr, vp, vx;
    SpinorIO<PS>::load(vr, r + off, g.Vh, pp, h);
    SpinorIO<PS>::load(vp, p + off, g.Vh, pp, h);
    SpinorIO<PS>::load(vx, x + off, g.Vh, pp, h);
    const T a = (T)st[sh(SH_COEFX, 0)], b = (T)st[sh(SH_COEFP, 0)];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vx.s[s][c] = vx.s[s][c] + a * vp.s[s][c];
        vp.s[s][c] = vr.s[s][c] + b * vp.s[s][c];
      }
    SpinorIO<PS>::store(vx, x + off, g.Vh, pp, h);
    SpinorIO<PS>::store(vp, p + off, g.Vh, pp, h);
  }
}

cudaError_t bcg_init(double* states, int nsys, cudaStream_t st) {
  bcg_init_kernel<<<(nsys + 31) / 32, 32, 0, st>>>(states, nsys);
  return cudaGetLastError();
}

cudaError_t bcg_scalar(double* states, int nsys, int maxit, const cudaGraphConditionalHandle* h, cudaStream_t st) {
  if (nsys > 1024) return cudaErrorInvalidValue;
  const int threads = ((nsys + 31) / 32) * 32;
  if (h)
    bcg_scalar_kernel<true><<<1, threads, 0, st>>>(states, nsys, maxit, *h);
  else
    bcg_scalar_kernel<false><<<1, threads, 0, st>>>(states, nsys, maxit, cudaGraphConditionalHandle{});
  return cudaGetLastError();
}

cudaError_t bcg_update(const Geom& g, int ps, const void* r, void* p, void* x, size_t fstride, const double* states,
                       int nsys, cudaStream_t st) {
  // one wave of resident 256-thread blocks (4 per SM), capped by the number of items
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && sms[dev] == 0) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  const int64_t items = (int64_t)((2 * g.Vh + 255) / 256) * nsys;
  const int grid = (int)std::min<int64_t>(items, 4 * (int64_t)std::max(1, dev < 64 ? sms[dev] : 152));
  const char* rr = static_cast<const char*>(r);
  char* pp = static_cast<char*>(p);
  char* xx = static_cast<char*>(x);
  switch (ps) {
    case P64: bcg_update_kernel<P64><<<grid, 256, 0, st>>>(g, rr, pp, xx, fstride, states, nsys); break;
    case P32: bcg_update_kernel<P32><<<grid, 256, 0, st>>>(g, rr, pp, xx, fstride, states, nsys); break;
    case P16: bcg_update_kernel<P16><<<grid, 256, 0, st>>>(g, rr, pp, xx, fstride, states, nsys); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace nd
