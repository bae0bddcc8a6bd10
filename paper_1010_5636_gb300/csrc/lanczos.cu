// Low modes of Q (Sec. 2.3): the paper finds the lowest modes of Q^2 by minimising the Ritz
// functional; here a Chebyshev-filtered subspace iteration on Q^2 (FP32 or FP64 filter, FP64
// orthonormalisation and Rayleigh-Ritz) plays that role, followed by the Rayleigh-Ritz step of
// Q on the found space V:
//   u_k in V with P Q u_k = nu_k u_k,  rho_k = ||(Q - nu_k) u_k||,
//   kappa_+-^2 = sum_{+-nu_k > 0} rho_k^2 / d_k^2.
// d_k (distance of nu_k from the exact spectrum on the complement of the exact projector of
// its sign; the paper gives no estimator) is estimated as
//   d_k = min(|nu_k| + m_opp, sqrt(lambda_{l+1}) - |nu_k|),
// m_opp = smallest |nu_j| of the opposite sign in V (sqrt(lambda_{l+1}) if there is none).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>

#include "solver.h"

namespace nd {

namespace {

// w = Q^2 v in FP64 (two launches through the scratch field t)
nd_status apply_q2(nd_ctx* c, void* w, const void* v) {
  void* t = field(c, "lz_t", 0);
  if (!t) return fail(c, ND_ERR_OOM, "Q^2: workspace");
  ND_TRY(q_apply(c, 0, t, v));
  ND_TRY(q_apply(c, 0, w, t));
  return ND_OK;
}

nd_status norm2_64(nd_ctx* c, const void* v, double* out) {
  void* junk = field(c, "lz_junk", 0);
  ND_TRY_CUDA(c, blas_dot(c->g, 0, v, v, slot(c, c->red_scratch), c->stream));
  double h[3];
  ND_TRY(read_back(c, c->red_scratch, h, 3));
  (void)junk;
  *out = h[2];
  return ND_OK;
}

// h[0..2K) = (v_k, w) for the K vectors at base
nd_status dots(nd_ctx* c, const char* base, size_t stride, int K, const void* w, std::vector<double>& h) {
  double* dev = static_cast<double*>(workspace(c, "lz_dots", sizeof(double) * 2 * 128));
  if (!dev) return fail(c, ND_ERR_OOM, "dots: workspace");
  h.assign(2 * K, 0.0);
  for (int k0 = 0; k0 < K; k0 += 64) {
    const int kk = std::min(64, K - k0);
    ND_TRY_CUDA(c, blas_multidot(c->g, base + k0 * stride, stride, kk, w, slot(c, dev), c->stream));
    ND_TRY(read_back(c, dev, h.data() + 2 * k0, 2 * kk));
  }
  return ND_OK;
}

// out = beta * y + sum_k coef_k v_k (coef host, complex)
nd_status lincomb(nd_ctx* c, void* out, double beta, const void* y, const char* base, size_t stride, int K,
                  const std::vector<double>& coef) {
  double* dev = static_cast<double*>(workspace(c, "lz_coef", sizeof(double) * 2 * 256));
  if (!dev) return fail(c, ND_ERR_OOM, "lincomb: workspace");
  for (int k0 = 0; k0 < K; k0 += 256) {
    const int kk = std::min(256, K - k0);
    ND_TRY_CUDA(c, cudaMemcpyAsync(dev, coef.data() + 2 * k0, sizeof(double) * 2 * kk, cudaMemcpyHostToDevice,
                                   c->stream));
    ND_TRY_CUDA(c, blas_lincomb(c->g, out, k0 == 0 ? beta : 1.0, k0 == 0 ? y : out, base + k0 * stride, stride, kk,
                                dev, c->stream));
    // the coefficient buffer is reused: wait before the next upload
    ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return ND_OK;
}

}  // namespace

// Plain Lanczos on Q^2 for the largest eigenvalue (iters steps, full reorthogonalisation).
nd_status lambda_max_estimate(nd_ctx* c, int iters, double* lam) {
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  iters = std::max(2, std::min(iters, 100));
  char* V = static_cast<char*>(field(c, "lm_V", 0, iters + 1));
  if (!V) return fail(c, ND_ERR_OOM, "lambda_max: workspace");
  ND_TRY_CUDA(c, blas_random(c->g, V, 12345, c->stream));
  double n2;
  ND_TRY(norm2_64(c, V, &n2));
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, V, 1.0 / std::sqrt(n2), V, 0.0, nullptr, false, slot(c, nullptr), c->stream));
  std::vector<double> T(2 * iters * iters, 0.0);
  int m = iters;
  for (int j = 0; j < iters; ++j) {
    void* w = V + (j + 1) * fs;
    ND_TRY(apply_q2(c, w, V + j * fs));
    std::vector<double> h, h2;
    ND_TRY(dots(c, V, fs, j + 1, w, h));
    std::vector<double> neg(2 * (j + 1));
    for (int i = 0; i < 2 * (j + 1); ++i) neg[i] = -h[i];
    ND_TRY(lincomb(c, w, 1.0, w, V, fs, j + 1, neg));
    ND_TRY(dots(c, V, fs, j + 1, w, h2));
    for (int i = 0; i < 2 * (j + 1); ++i) neg[i] = -h2[i];
    ND_TRY(lincomb(c, w, 1.0, w, V, fs, j + 1, neg));
    for (int i = 0; i <= j; ++i) {
      T[2 * (i * iters + j)] = h[2 * i] + h2[2 * i];
      T[2 * (i * iters + j) + 1] = h[2 * i + 1] + h2[2 * i + 1];
      T[2 * (j * iters + i)] = T[2 * (i * iters + j)];
      T[2 * (j * iters + i) + 1] = -T[2 * (i * iters + j) + 1];
    }
    double b2;
    ND_TRY(norm2_64(c, w, &b2));
    if (b2 <= 1e-28 * std::max(1.0, std::fabs(T[2 * (j * iters + j)]))) {
      m = j + 1;
      break;
    }
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, w, 1.0 / std::sqrt(b2), w, 0.0, nullptr, false, slot(c, nullptr), c->stream));
  }
  std::vector<double> Tm(2 * m * m), ev, evec;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      Tm[2 * (i * m + j)] = T[2 * (i * iters + j)];
      Tm[2 * (i * m + j) + 1] = T[2 * (i * iters + j) + 1];
    }
  hermitian_eig(m, Tm, ev, evec);
  *lam = ev[m - 1];
  return ND_OK;
}

// Rayleigh-Ritz of Q on the l FP64 fields at U (overwritten by the rotated u_k, ordered by
// |nu| ascending); fills nu, rho.
nd_status ritz_of_Q(nd_ctx* c, char* U, int l, std::vector<double>& nu, std::vector<double>& rho) {
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  char* QU = static_cast<char*>(field(c, "rr_QU", 0, l));
  char* U2 = static_cast<char*>(field(c, "rr_U2", 0, 2 * l));
  if (!QU || !U2) return fail(c, ND_ERR_OOM, "Rayleigh-Ritz: workspace");
  for (int j = 0; j < l; ++j) ND_TRY(q_apply(c, 0, QU + j * fs, U + j * fs));
  std::vector<double> M(2 * l * l), h;
  for (int j = 0; j < l; ++j) {
    ND_TRY(dots(c, U, fs, l, QU + j * fs, h));
    for (int i = 0; i < l; ++i) {
      M[2 * (i * l + j)] = h[2 * i];
      M[2 * (i * l + j) + 1] = h[2 * i + 1];
    }
  }
  // symmetrise (M is hermitian up to rounding)
  for (int i = 0; i < l; ++i)
    for (int j = i; j < l; ++j) {
      const double re = 0.5 * (M[2 * (i * l + j)] + M[2 * (j * l + i)]);
      const double im = 0.5 * (M[2 * (i * l + j) + 1] - M[2 * (j * l + i) + 1]);
      M[2 * (i * l + j)] = re;
      M[2 * (i * l + j) + 1] = im;
      M[2 * (j * l + i)] = re;
      M[2 * (j * l + i) + 1] = -im;
    }
  std::vector<double> ev, W;
  hermitian_eig(l, M, ev, W);
  std::vector<int> order(l);
  for (int k = 0; k < l; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(ev[a]) < std::fabs(ev[b]); });
  nu.assign(l, 0.0);
  rho.assign(l, 0.0);
  double* res = c->red_scratch + 16;
  for (int k = 0; k < l; ++k) {
    const int kk = order[k];
    nu[k] = ev[kk];
    std::vector<double> coef(2 * l);
    for (int j = 0; j < l; ++j) {
      coef[2 * j] = W[2 * (j * l + kk)];
      coef[2 * j + 1] = W[2 * (j * l + kk) + 1];
    }
    ND_TRY(lincomb(c, U2 + k * fs, 0.0, nullptr, U, fs, l, coef));
    ND_TRY(lincomb(c, U2 + (l + k) * fs, 0.0, nullptr, QU, fs, l, coef));
    // rho_k = ||Q u_k - nu_k u_k||
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, U2 + (l + k) * fs, 1.0, U2 + (l + k) * fs, -nu[k], U2 + k * fs, true,
                              slot(c, res), c->stream));
    double r2;
    ND_TRY(read_back(c, res, &r2, 1));
    rho[k] = std::sqrt(std::max(0.0, r2));
  }
  ND_TRY_CUDA(c, cudaMemcpyAsync(U, U2, fs * l, cudaMemcpyDeviceToDevice, c->stream));
  return ND_OK;
}

void kappas(const std::vector<double>& nu, const std::vector<double>& rho, double lam_next, double* kp, double* km) {
  const double top = std::sqrt(std::max(0.0, lam_next));
  double sp = 0.0, sm = 0.0;
  const int l = (int)nu.size();
  for (int k = 0; k < l; ++k) {
    double m_opp = top;
    for (int j = 0; j < l; ++j)
      if ((nu[j] > 0) != (nu[k] > 0)) m_opp = std::min(m_opp, std::fabs(nu[j]));
    const double d = std::min(std::fabs(nu[k]) + m_opp, top - std::fabs(nu[k]));
    const double q = d > 0 ? rho[k] / d : INFINITY;
    if (nu[k] > 0)
      sp += q * q;
    else
      sm += q * q;
  }
  *kp = std::sqrt(sp);
  *km = std::sqrt(sm);
}

// Store l modes (FP64 internal fields at src) in the context.
nd_status store_modes(nd_ctx* c, const void* src, int l) {
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  if ((size_t)l * fs > c->evecs_cap) {
    if (c->evecs) cudaFree(c->evecs);
    c->evecs = nullptr;
    c->evecs_cap = 0;
    if (cudaMalloc(&c->evecs, (size_t)l * fs) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, ND_ERR_OOM, "low modes: cudaMalloc");
    }
    c->evecs_cap = (size_t)l * fs;
  }
  if (l) ND_TRY_CUDA(c, cudaMemcpyAsync(c->evecs, src, (size_t)l * fs, cudaMemcpyDeviceToDevice, c->stream));
  c->nlow = l;
  return ND_OK;
}

}  // namespace nd

using namespace nd;

extern "C" nd_status nd_lambda_max(nd_ctx* c, int iters, double* lam) {
  if (!c || !lam) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (!c->links[0]) return fail(c, ND_ERR_STATE, "nd_lambda_max: FP64 links not set");
  ND_TRY(lambda_max_estimate(c, iters, lam));
  c->lam_max = *lam;
  return ND_OK;
}

namespace nd {

// Chebyshev filter x <- C_d(Q^2) x with C_d(t) = T_d(L(t)) / T_d(L(0)), L mapping [lo, hi] onto
// [-1, 1]: modes below lo are amplified relative to the damped interval, and the normalisation
// at t = 0 (Q^2 >= 0) keeps every value in [-1, 1], so no precision overflows.  Scaled
// three-term recurrence with s_1 = e / (0 - c), s_{k+1} = 1 / (2 / s_1 - s_k):
//   C_1 = (s_1 / e) (A - c),  C_{k+1} = (2 s_{k+1} / e) (A - c) C_k - s_k s_{k+1} C_{k-1},
// e = (hi - lo) / 2, c = (hi + lo) / 2.  Evaluated in precision prec on the FP64 field x
// (converted in and out); every step is two Q launches, the second carrying the recurrence
// terms in its epilogue.
nd_status cheb_filter(nd_ctx* c, int prec, void* x64, int deg, double lo, double hi) {
  const double e = 0.5 * (hi - lo), cc = 0.5 * (hi + lo);
  const double s1 = e / (0.0 - cc), tau = 2.0 / s1;
  void* ya = field(c, prec == 0 ? "cf_ya64" : "cf_ya32", prec);
  void* yb = field(c, prec == 0 ? "cf_yb64" : "cf_yb32", prec);
  void* t = field(c, prec == 0 ? "cf_t64" : "cf_t32", prec);
  if (!ya || !yb || !t) return fail(c, ND_ERR_OOM, "Chebyshev filter: workspace");
  ND_TRY_CUDA(c, blas_convert(c->g, prec, ya, 0, x64, c->stream));  // C_0 x
  ND_TRY(q_apply(c, prec, t, ya));
  ND_TRY(q_apply(c, prec, yb, t, s1 / e, -cc * s1 / e, ya));  // C_1 x
  void* prev = ya;
  void* cur = yb;
  double s = s1;
  for (int k = 1; k < deg; ++k) {
    const double sn = 1.0 / (tau - s);
    ND_TRY(q_apply(c, prec, t, cur));
    // C_{k+1} x = (2 sn / e)(Q^2 - c) C_k x - s sn C_{k-1} x, written over C_{k-1} x
    ND_TRY(q_apply(c, prec, prev, t, 2.0 * sn / e, -2.0 * sn * cc / e, cur, nullptr, nullptr, prev, -s * sn));
    std::swap(prev, cur);
    s = sn;
  }
  ND_TRY_CUDA(c, blas_convert(c->g, 0, x64, prec, cur, c->stream));
  return ND_OK;
}

// Classical Gram-Schmidt with one reorthogonalisation pass over the k FP64 fields at X.
nd_status orthonormalise(nd_ctx* c, char* X, int k, size_t fs) {
  for (int j = 0; j < k; ++j) {
    void* x = X + j * fs;
    for (int attempt = 0; attempt < 3; ++attempt) {
      for (int pass = 0; pass < 2 && j > 0; ++pass) {
        std::vector<double> h;
        ND_TRY(dots(c, X, fs, j, x, h));
        for (auto& v : h) v = -v;
        ND_TRY(lincomb(c, x, 1.0, x, X, fs, j, h));
      }
      double n2;
      ND_TRY(norm2_64(c, x, &n2));
      if (n2 > 1e-200 && std::isfinite(n2)) {
        ND_TRY_CUDA(c, blas_axpby(c->g, 0, x, 1.0 / std::sqrt(n2), x, 0.0, nullptr, false, slot(c, nullptr), c->stream));
        break;
      }
      if (attempt == 2) return fail(c, ND_ERR_BREAKDOWN, "low modes: basis lost rank");
      ND_TRY_CUDA(c, blas_random(c->g, x, 1000003ull * (j + 1) + attempt, c->stream));
    }
  }
  return ND_OK;
}

// Rayleigh-Ritz of Q^2 on the orthonormal FP64 basis X (k fields): X <- X W, AX <- Q^2 X W,
// theta ascending, res_i = ||Q^2 x_i - theta_i x_i||.
nd_status rayleigh_ritz_q2(nd_ctx* c, char*& X, char*& AX, char*& Y, int k, size_t fs, std::vector<double>& theta,
                           std::vector<double>& res) {
  for (int j = 0; j < k; ++j) ND_TRY(apply_q2(c, AX + j * fs, X + j * fs));
  std::vector<double> H(2 * k * k), h;
  for (int j = 0; j < k; ++j) {
    ND_TRY(dots(c, X, fs, k, AX + j * fs, h));
    for (int i = 0; i < k; ++i) {
      H[2 * (i * k + j)] = h[2 * i];
      H[2 * (i * k + j) + 1] = h[2 * i + 1];
    }
  }
  for (int i = 0; i < k; ++i)
    for (int j = i; j < k; ++j) {
      const double re = 0.5 * (H[2 * (i * k + j)] + H[2 * (j * k + i)]);
      const double im = 0.5 * (H[2 * (i * k + j) + 1] - H[2 * (j * k + i) + 1]);
      H[2 * (i * k + j)] = re;
      H[2 * (i * k + j) + 1] = im;
      H[2 * (j * k + i)] = re;
      H[2 * (j * k + i) + 1] = -im;
    }
  std::vector<double> W;
  hermitian_eig(k, H, theta, W);
  // rotated basis into Y, rotated Q^2 X into X's old storage via a second pass
  for (int j = 0; j < k; ++j) {
    std::vector<double> coef(2 * k);
    for (int i = 0; i < k; ++i) {
      coef[2 * i] = W[2 * (i * k + j)];
      coef[2 * i + 1] = W[2 * (i * k + j) + 1];
    }
    ND_TRY(lincomb(c, Y + j * fs, 0.0, nullptr, X, fs, k, coef));
  }
  std::swap(X, Y);  // X = rotated basis; Y = old basis (free)
  for (int j = 0; j < k; ++j) {
    std::vector<double> coef(2 * k);
    for (int i = 0; i < k; ++i) {
      coef[2 * i] = W[2 * (i * k + j)];
      coef[2 * i + 1] = W[2 * (i * k + j) + 1];
    }
    ND_TRY(lincomb(c, Y + j * fs, 0.0, nullptr, AX, fs, k, coef));
  }
  std::swap(AX, Y);  // AX = rotated Q^2 X; Y free
  res.assign(k, 0.0);
  double* rs = c->red_scratch + 24;
  void* tmp = field(c, "cf_res", 0);
  if (!tmp) return fail(c, ND_ERR_OOM, "low modes: workspace");
  for (int j = 0; j < k; ++j) {
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, tmp, 1.0, AX + j * fs, -theta[j], X + j * fs, true, slot(c, rs), c->stream));
    double r2;
    ND_TRY(read_back(c, rs, &r2, 1));
    res[j] = std::sqrt(std::max(0.0, r2));
  }
  return ND_OK;
}

}  // namespace nd

// One step of the filtered subspace iteration on the block X (k FP64 fields): filter every vector
// but the `locked` lowest with T_d(L(Q^2)) damping [lo, hi], lo = the largest Ritz value of the
// block, then re-orthonormalise and Rayleigh-Ritz project.  FP32 filtering reaches residuals of about 1e-7 lambda_max; once the
// worst wanted residual is below 1e-6 lambda_max the filter runs in FP64.
nd_status filter_step(nd_ctx* c, char*& X, char*& AX, char*& Y, int k, size_t fs, double hi, double worst,
                      std::vector<double>& theta, std::vector<double>& res, int* apps, int locked = 0) {
  const double lo = std::min(theta[k - 1], 0.5 * hi);
  const int prec = (c->links[1] && worst > 1e-6 * hi) ? 1 : 0;
  const int deg = prec == 1 ? 100 : 40;
  // the lowest `locked` Ritz vectors have converged: they stay in the basis (orthogonalisation and
  // Rayleigh-Ritz) but are not filtered again
  for (int j = locked; j < k; ++j) ND_TRY(cheb_filter(c, prec, X + j * fs, deg, lo, hi));
  *apps += (k - locked) * deg;
  ND_TRY(orthonormalise(c, X, k, fs));
  ND_TRY(rayleigh_ritz_q2(c, X, AX, Y, k, fs, theta, res));
  *apps += k;
  return ND_OK;
}

// The l in [l_min, l_max] with the largest relative gap (sqrt(theta_l) - sqrt(theta_{l-1})) / sqrt(theta_l)
// between the last kept (theta_{l-1}) and the first remaining (theta_l) Ritz value of Q^2, the
// smallest l on ties; *gap receives that gap.
static int choose_l_by_gap(const std::vector<double>& theta, int l_min, int l_max, double* gap) {
  int l = l_min;
  double best = -1.0;
  for (int j = l_min; j <= l_max; ++j) {
    const double a = std::sqrt(std::max(theta[j - 1], 0.0)), b = std::sqrt(std::max(theta[j], 0.0));
    const double g = b > 0 ? (b - a) / b : 0.0;
    if (g > best) {
      best = g;
      l = j;
    }
  }
  *gap = best;
  return l;
}

// Keep l modes (FP64 fields at U) in the context and fill the caller's outputs.
static nd_status finish_lowmodes(nd_ctx* c, const void* U, int l, const std::vector<double>& nu,
                                 const std::vector<double>& rho, const std::vector<double>& theta, double lam_max,
                                 int apps, std::chrono::steady_clock::time_point t0, int* l_out, double* nu_out,
                                 double* rho_out, double* evq2_out, nd_lowmode_info* info) {
  c->lam_next = theta[l];
  ND_TRY(store_modes(c, U, l));
  c->nu = nu;
  c->rho = rho;
  double kp, km;
  kappas(nu, rho, c->lam_next, &kp, &km);
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  if (l_out) *l_out = l;
  if (nu_out) std::copy(nu.begin(), nu.end(), nu_out);
  if (rho_out) std::copy(rho.begin(), rho.end(), rho_out);
  if (evq2_out) std::copy(theta.begin(), theta.begin() + l + 1, evq2_out);
  if (info) {
    info->l = l;
    info->iters = apps;
    info->lambda_max = lam_max;
    info->lambda_next = c->lam_next;
    info->kappa_plus = kp;
    info->kappa_minus = km;
    info->max_rho = *std::max_element(rho.begin(), rho.end());
    info->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  c->lam_max = lam_max;
  return ND_OK;
}

// Low modes by Chebyshev-filtered subspace iteration on Q^2: a block of k = l+1+buffer FP64
// vectors is filtered with T_d(L(Q^2)) (damping [lo, lambda_max], lo = the largest Ritz value
// of the block), re-orthonormalised in FP64 and Rayleigh-Ritz projected with FP64 Q^2.  The
// filter runs in FP32 while the residuals are above 1e-5 lambda_max, then in FP64.
extern "C" nd_status nd_lowmodes(nd_ctx* c, int l, double tol, int maxit, double* nu_out, double* rho_out,
                                 double* evq2_out, nd_lowmode_info* info) {
  NvtxRange range("nd.lowmodes");
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (l < 1 || l > 64 || !(tol > 0) || maxit < 1) return fail(c, ND_ERR_INVALID_ARG, "nd_lowmodes: 1 <= l <= 64");
  if (!c->links[0]) return fail(c, ND_ERR_STATE, "nd_lowmodes: FP64 links not set");
  auto t0 = std::chrono::steady_clock::now();
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  double lam_max;
  ND_TRY(lambda_max_estimate(c, 40, &lam_max));
  const double hi = 1.01 * lam_max;
  const int nwant = l + 1;
  // a block twice the wanted size keeps the damped interval away from the wanted modes when
  // the low spectrum is a dense band (the gap between mode l+1 and the block edge sets the rate)
  const int k = std::min(std::max(nwant + 8, 2 * nwant), 130);
  char* X = static_cast<char*>(field(c, "cf_X", 0, k));
  char* AX = static_cast<char*>(field(c, "cf_AX", 0, k));
  char* Y = static_cast<char*>(field(c, "cf_Y", 0, k));
  if (!X || !AX || !Y) return fail(c, ND_ERR_OOM, "nd_lowmodes: workspace");
  for (int j = 0; j < k; ++j) ND_TRY_CUDA(c, blas_random(c->g, X + j * fs, 777 + 7919ull * j, c->stream));
  ND_TRY(orthonormalise(c, X, k, fs));
  std::vector<double> theta, res;
  ND_TRY(rayleigh_ritz_q2(c, X, AX, Y, k, fs, theta, res));
  int apps = k;
  const bool trace = std::getenv("ND_TRACE") != nullptr;  // per-iteration progress on stderr
  bool converged = false;
  for (int it = 0; it < 1000; ++it) {
    double worst = 0.0;
    int nconv = 0;
    for (int i = 0; i < nwant; ++i) {
      worst = std::max(worst, res[i]);
      if (res[i] <= tol * hi) ++nconv;
    }
    if (nconv == nwant) {
      converged = true;
      break;
    }
    if (apps >= maxit) break;
    // lock the leading wanted vectors that already meet a tenth of the target
    int locked = 0;
    while (locked < nwant && res[locked] <= 0.1 * tol * hi) ++locked;
    if (trace)
      std::fprintf(stderr, "nd_lowmodes: it %d apps %d hi %.6g theta0 %.6g theta_l %.6g worst %.3g nconv %d locked %d\n",
                   it, apps, hi, theta[0], theta[l], worst, nconv, locked);
    ND_TRY(filter_step(c, X, AX, Y, k, fs, hi, worst, theta, res, &apps, locked));
    lam_max = std::max(lam_max, theta[k - 1]);
  }
  // keep the workspace registry pointing at the right buffers after the swaps
  c->ws["cf_X"].first = X;
  c->ws["cf_AX"].first = AX;
  c->ws["cf_Y"].first = Y;
  if (!converged) return fail(c, ND_ERR_NOT_CONVERGED, "nd_lowmodes: filtered subspace iteration did not converge");
  std::vector<double> nu, rho;
  ND_TRY(ritz_of_Q(c, X, l, nu, rho));
  return finish_lowmodes(c, X, l, nu, rho, theta, lam_max, apps, t0, nullptr, nu_out, rho_out, evq2_out, info);
}

extern "C" nd_status nd_set_lowmodes(nd_ctx* c, int l, const double* evecs, const double* nu, double lambda_next,
                                     nd_lowmode_info* info) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (l < 0 || l > 64 || (l > 0 && (!evecs || !nu)) || !(lambda_next > 0))
    return fail(c, ND_ERR_INVALID_ARG, "nd_set_lowmodes: bad argument");
  if (!c->links[0]) return fail(c, ND_ERR_STATE, "nd_set_lowmodes: FP64 links not set");
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  char* U = static_cast<char*>(field(c, "sl_U", 0, std::max(l, 1)));
  void* t = field(c, "sl_t", 0);
  if (!U || !t) return fail(c, ND_ERR_OOM, "nd_set_lowmodes: workspace");
  std::vector<double> nuv(nu, nu + l), rho(l, 0.0);
  double* res = c->red_scratch + 16;
  for (int k = 0; k < l; ++k) {
    ND_TRY(nd_pack_spinor(c, U + k * fs, evecs + (size_t)k * 24 * c->V, ND_FP64, 1));
    ND_TRY(q_apply(c, 0, t, U + k * fs));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, t, 1.0, t, -nuv[k], U + k * fs, true, slot(c, res), c->stream));
    double r2;
    ND_TRY(read_back(c, res, &r2, 1));
    rho[k] = std::sqrt(std::max(0.0, r2));
  }
  ND_TRY(store_modes(c, U, l));
  c->nu = nuv;
  c->rho = rho;
  c->lam_next = lambda_next;
  if (info) {
    double kp = 0, km = 0;
    kappas(nuv, rho, lambda_next, &kp, &km);
    info->l = l;
    info->lambda_next = lambda_next;
    info->lambda_max = c->lam_max;
    info->kappa_plus = kp;
    info->kappa_minus = km;
    info->max_rho = l ? *std::max_element(rho.begin(), rho.end()) : 0.0;
  }
  return ND_OK;
}

extern "C" nd_status nd_get_lowmodes(nd_ctx* c, double* evecs, double* nu) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  for (int k = 0; k < c->nlow; ++k) {
    if (evecs)
      ND_TRY(nd_unpack_spinor(c, evecs + (size_t)k * 24 * c->V, static_cast<char*>(c->evecs) + k * fs, ND_FP64, 1));
    if (nu) nu[k] = c->nu[k];
  }
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  return ND_OK;
}

extern "C" nd_status nd_lowmode_state(nd_ctx* c, int* l, double* lambda_next, double* lambda_max) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (l) *l = c->nlow;
  if (lambda_next) *lambda_next = c->lam_next;
  if (lambda_max) *lambda_max = c->lam_max;
  return ND_OK;
}

// Low modes with the number l chosen dynamically and kappa_+- driving the stopping (Sec. 2.3).
// The block iteration above runs for l_max + 1 wanted modes.  After each step the candidate l in
// [l_min, l_max] with the largest relative gap (sqrt(theta_{l+1}) - sqrt(theta_l)) / sqrt(theta_{l+1})
// between the last kept and the first remaining Ritz value of Q^2 is taken (smallest l on ties), so
// that the spectral distance d_k entering kappa is not small by chance.  Once the l + 1 lowest
// Q^2 residuals are below 1e-4 lambda_max, the Rayleigh-Ritz pairs of Q on the first l vectors give
// rho_k and kappa_+- (d_k as in nd_lowmodes, lambda_{l+1} ~ theta_{l+1}); the iteration stops when
// both kappas are at most kappa_target.  Once all candidates' Ritz values have settled, l is
// fixed and the block shrinks to the vectors needed for the kept modes.
extern "C" nd_status nd_lowmodes_dynamic(nd_ctx* c, int l_min, int l_max, double kappa_target, int maxit, int* l_out,
                                         double* nu_out, double* rho_out, double* evq2_out, nd_lowmode_info* info) {
  NvtxRange range("nd.lowmodes_dynamic");
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (l_min < 1 || l_max < l_min || l_max > 64 || !(kappa_target > 0) || maxit < 1)
    return fail(c, ND_ERR_INVALID_ARG, "nd_lowmodes_dynamic: need 1 <= l_min <= l_max <= 64, kappa_target > 0");
  if (!c->links[0]) return fail(c, ND_ERR_STATE, "nd_lowmodes_dynamic: FP64 links not set");
  auto t0 = std::chrono::steady_clock::now();
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  double lam_max;
  ND_TRY(lambda_max_estimate(c, 40, &lam_max));
  const double hi = 1.01 * lam_max;
  const int nwant = l_max + 1;
  const int k = std::min(std::max(nwant + 8, 2 * nwant), 130);
  char* X = static_cast<char*>(field(c, "cf_X", 0, k));
  char* AX = static_cast<char*>(field(c, "cf_AX", 0, k));
  char* Y = static_cast<char*>(field(c, "cf_Y", 0, k));
  char* Z = static_cast<char*>(field(c, "cf_Z", 0, l_max));
  if (!X || !AX || !Y || !Z) return fail(c, ND_ERR_OOM, "nd_lowmodes_dynamic: workspace");
  for (int j = 0; j < k; ++j) ND_TRY_CUDA(c, blas_random(c->g, X + j * fs, 777 + 7919ull * j, c->stream));
  ND_TRY(orthonormalise(c, X, k, fs));
  std::vector<double> theta, res, nu, rho;
  ND_TRY(rayleigh_ritz_q2(c, X, AX, Y, k, fs, theta, res));
  int apps = k, l = l_min;
  double kp = INFINITY, km = INFINITY;
  const bool trace = std::getenv("ND_TRACE") != nullptr;
  bool converged = false;
  bool fixed = false;
  double lock_frac = 0.1;
  int kb = k;  // current block size
  double best = -1.0;
  for (int it = 0; it < 1000; ++it) {
    if (!fixed) {
      l = choose_l_by_gap(theta, l_min, l_max, &best);
      // once every candidate's Ritz value is settled (residual <= 1e-3 lambda_max bounds its error
      // by ~1e-6 lambda_max^2 / gap), l is fixed and the block shrinks to the lowest
      // max(l + 9, 2 (l + 1)) Ritz vectors: the rest of the work only refines the kept modes
      double worst_all = 0.0;
      for (int i = 0; i <= l_max; ++i) worst_all = std::max(worst_all, res[i]);
      if (worst_all <= 1e-3 * hi) {
        fixed = true;
        kb = std::min(kb, std::max(l + 9, 2 * (l + 1)));
        theta.resize(kb);
        res.resize(kb);
      }
    }
    double worst = 0.0;
    for (int i = 0; i <= l; ++i) worst = std::max(worst, res[i]);
    if (worst <= 1e-4 * hi) {
      ND_TRY_CUDA(c, cudaMemcpyAsync(Z, X, fs * l, cudaMemcpyDeviceToDevice, c->stream));
      ND_TRY(ritz_of_Q(c, Z, l, nu, rho));
      apps += (l + 1) / 2;
      kappas(nu, rho, theta[l], &kp, &km);
      if (trace)
        std::fprintf(stderr, "nd_lowmodes_dynamic: it %d apps %d l %d gap %.3g worst %.3g kappa+ %.3g kappa- %.3g\n", it,
                     apps, l, best, worst, kp, km);
      if (kp <= kappa_target && km <= kappa_target) {
        converged = true;
        break;
      }
    }
    if (apps >= maxit) break;
    // once l is fixed, lock the leading kept vectors whose residual already implies their share of
    // the kappa target: rho_k ~ res_k / (2 sqrt(theta_k)) and d_k >= g = sqrt(theta_l) - sqrt(theta_{l-1}),
    // so res_k <= 2 sqrt(theta_k) kappa g / sqrt(l) suffices; lock at lock_frac of that
    int locked = 0;
    if (fixed) {
      const double g = std::sqrt(std::max(theta[l], 0.0)) - std::sqrt(std::max(theta[l - 1], 0.0));
      while (locked < l &&
             res[locked] <= lock_frac * 2.0 * std::sqrt(std::max(theta[locked], 0.0)) * kappa_target * g / std::sqrt((double)l))
        ++locked;
      if (locked == l && !(kp <= kappa_target && km <= kappa_target) && worst <= 1e-4 * hi) {
        lock_frac *= 0.1;  // the estimate was too loose: tighten and filter everything again
        locked = 0;
      }
    }
    ND_TRY(filter_step(c, X, AX, Y, kb, fs, hi, worst, theta, res, &apps, locked));
    if (!fixed) lam_max = std::max(lam_max, theta[kb - 1]);
  }
  c->ws["cf_X"].first = X;
  c->ws["cf_AX"].first = AX;
  c->ws["cf_Y"].first = Y;
  if (!converged)
    return fail(c, ND_ERR_NOT_CONVERGED, "nd_lowmodes_dynamic: kappa target not reached within maxit Q^2 applications");
  return finish_lowmodes(c, Z, l, nu, rho, theta, lam_max, apps, t0, l_out, nu_out, rho_out, evq2_out, info);
}

namespace {

// Project v onto the complement of the k orthonormal FP64 fields at U (two passes).
nd_status project_out(nd_ctx* c, const char* U, int k, size_t fs, void* v) {
  for (int pass = 0; pass < 2 && k > 0; ++pass) {
    std::vector<double> h;
    ND_TRY(dots(c, U, fs, k, v, h));
    for (auto& e : h) e = -e;
    ND_TRY(lincomb(c, v, 1.0, v, U, fs, k, h));
  }
  return ND_OK;
}

// Complex (x, y) from the FP64 dot kernel.
nd_status cdot(nd_ctx* c, const void* x, const void* y, double* re, double* im) {
  double h[3];
  ND_TRY_CUDA(c, blas_dot(c->g, 0, x, y, slot(c, c->red_scratch), c->stream));
  ND_TRY(read_back(c, c->red_scratch, h, 3));
  *re = h[0];
  *im = h[1];
  return ND_OK;
}

// v <- (cre + i cim) v  (complex scale, FP64 field)
nd_status cscale(nd_ctx* c, void* v, double cre, double cim) {
  std::vector<double> coef = {cre, cim};
  return lincomb(c, v, 0.0, nullptr, static_cast<const char*>(v), 0, 1, coef);
}

}  // namespace

// Minimise the Ritz functional mu(x) = (x, A x) / (x, x) of A = Q^2 / hi over x orthogonal to the k
// orthonormal fields at U, starting from x (Sec. 2.3: the low modes are found by minimising the
// Ritz functional of Q^2).  Nonlinear conjugate gradients in the form of Kalkreuter and Simma: the
// search direction p is made orthogonal to x, and each step takes the exact minimum of mu on
// span{x, p} (the lower eigenpair of the 2 x 2 projected matrix), so no line search is needed and
// A x is carried along without an extra application.  Stops when ||A x - mu x|| <= tol.
static nd_status ritz_cg(nd_ctx* c, const char* U, int k, size_t fs, void* x, double hi, double tol, int maxit,
                         double* mu_out, double* gn_out, int* apps) {
  void* y = field(c, "rf_y", 0);
  void* g = field(c, "rf_g", 0);
  void* p = field(c, "rf_p", 0);
  void* q = field(c, "rf_q", 0);
  void* z = field(c, "rf_z", 0);
  if (!y || !g || !p || !q || !z) return fail(c, ND_ERR_OOM, "Ritz functional: workspace");
  const double s = 1.0 / hi;
  ND_TRY(project_out(c, U, k, fs, x));
  double n2;
  ND_TRY(norm2_64(c, x, &n2));
  if (!(n2 > 0)) return fail(c, ND_ERR_BREAKDOWN, "Ritz functional: start vector lies in the found space");
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, x, 1.0 / std::sqrt(n2), x, 0.0, nullptr, false, slot(c, nullptr), c->stream));
  double mu = 0.0, gg = 0.0;
  auto refresh = [&]() -> nd_status {
    ND_TRY(apply_q2(c, y, x));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, y, s, y, 0.0, nullptr, false, slot(c, nullptr), c->stream));
    ++*apps;
    double im;
    ND_TRY(cdot(c, x, y, &mu, &im));
    return ND_OK;
  };
  auto gradient = [&]() -> nd_status {
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, g, 1.0, y, -mu, x, false, slot(c, nullptr), c->stream));
    ND_TRY(project_out(c, U, k, fs, g));
    return norm2_64(c, g, &gg);
  };
  ND_TRY(refresh());
  ND_TRY(gradient());
  ND_TRY_CUDA(c, cudaMemcpyAsync(p, g, fs, cudaMemcpyDeviceToDevice, c->stream));
  for (int it = 0; it < maxit && std::sqrt(gg) > tol; ++it) {
    // q = p - (x, p) x on the complement of U, normalised
    double are, aim;
    ND_TRY(cdot(c, x, p, &are, &aim));
    ND_TRY_CUDA(c, cudaMemcpyAsync(q, p, fs, cudaMemcpyDeviceToDevice, c->stream));
    std::vector<double> coef = {-are, -aim};
    ND_TRY(lincomb(c, q, 1.0, q, static_cast<const char*>(x), 0, 1, coef));
    ND_TRY(project_out(c, U, k, fs, q));
    double nq2;
    ND_TRY(norm2_64(c, q, &nq2));
    if (!(nq2 > 1e-300)) break;
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, q, 1.0 / std::sqrt(nq2), q, 0.0, nullptr, false, slot(c, nullptr), c->stream));
    ND_TRY(apply_q2(c, z, q));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, z, s, z, 0.0, nullptr, false, slot(c, nullptr), c->stream));
    ++*apps;
    double bre, bim, d, dim;
    ND_TRY(cdot(c, x, z, &bre, &bim));
    ND_TRY(cdot(c, q, z, &d, &dim));
    // lower eigenpair of [[mu, b], [conj(b), d]]: m and the vector (b, m - mu)
    const double half = 0.5 * (mu - d), bb = bre * bre + bim * bim;
    const double m = 0.5 * (mu + d) - std::sqrt(half * half + bb);
    const double nv = std::sqrt(bb + (m - mu) * (m - mu));
    if (!(nv > 0)) break;
    const double cxr = bre / nv, cxi = bim / nv, cq = (m - mu) / nv;
    // x <- cx x + cq q,  y <- cx y + cq z
    ND_TRY(cscale(c, x, cxr, cxi));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, x, 1.0, x, cq, q, false, slot(c, nullptr), c->stream));
    ND_TRY(cscale(c, y, cxr, cxi));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, y, 1.0, y, cq, z, false, slot(c, nullptr), c->stream));
    mu = m;
    if ((it + 1) % 25 == 0) {
      // renormalise and recompute A x against drift
      ND_TRY(norm2_64(c, x, &n2));
      ND_TRY_CUDA(c, blas_axpby(c->g, 0, x, 1.0 / std::sqrt(n2), x, 0.0, nullptr, false, slot(c, nullptr), c->stream));
      ND_TRY(refresh());
    }
    const double gg_old = gg;
    ND_TRY(gradient());
    // p <- g + beta (p - (x, p) x), Fletcher-Reeves beta
    ND_TRY(cdot(c, x, p, &are, &aim));
    coef = {-are, -aim};
    ND_TRY(lincomb(c, p, 1.0, p, static_cast<const char*>(x), 0, 1, coef));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, p, 1.0, g, gg / gg_old, p, false, slot(c, nullptr), c->stream));
  }
  *mu_out = mu * hi;
  *gn_out = std::sqrt(gg) * hi;
  return ND_OK;
}

// The paper's own low-mode method (Sec. 2.3): l_max + 1 vectors, each minimising the Ritz
// functional of Q^2 on the complement of the ones before it (ritz_cg), then a Rayleigh-Ritz
// step of Q^2 on all of them; l in [l_min, l_max] at the largest relative gap as in
// nd_lowmodes_dynamic; if kappa_+- exceed the target, every vector is minimised again with a
// ten times smaller gradient tolerance, until kappa_+- <= kappa_target.
extern "C" nd_status nd_lowmodes_ritz(nd_ctx* c, int l_min, int l_max, double kappa_target, int maxit, int* l_out,
                                      double* nu_out, double* rho_out, double* evq2_out, nd_lowmode_info* info) {
  NvtxRange range("nd.lowmodes_ritz");
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (l_min < 1 || l_max < l_min || l_max > 64 || !(kappa_target > 0) || maxit < 1)
    return fail(c, ND_ERR_INVALID_ARG, "nd_lowmodes_ritz: need 1 <= l_min <= l_max <= 64, kappa_target > 0");
  if (!c->links[0]) return fail(c, ND_ERR_STATE, "nd_lowmodes_ritz: FP64 links not set");
  auto t0 = std::chrono::steady_clock::now();
  const size_t fs = (size_t)spinor_bytes(0, c->Vh);
  double lam_max;
  ND_TRY(lambda_max_estimate(c, 40, &lam_max));
  const double hi = 1.01 * lam_max;
  const int K = l_max + 1;
  char* X = static_cast<char*>(field(c, "rf_X", 0, K));
  char* AX = static_cast<char*>(field(c, "rf_AX", 0, K));
  char* Y = static_cast<char*>(field(c, "rf_Y", 0, K));
  char* Z = static_cast<char*>(field(c, "cf_Z", 0, l_max));
  if (!X || !AX || !Y || !Z) return fail(c, ND_ERR_OOM, "nd_lowmodes_ritz: workspace");
  for (int j = 0; j < K; ++j) ND_TRY_CUDA(c, blas_random(c->g, X + j * fs, 4242 + 7919ull * j, c->stream));
  std::vector<double> theta, res, nu, rho;
  int apps = 0, l = l_min;
  double kp = INFINITY, km = INFINITY, tol = 1e-4;
  const bool trace = std::getenv("ND_TRACE") != nullptr;
  bool converged = false;
  for (int round = 0; round < 12 && apps < maxit; ++round, tol *= 0.1) {
    for (int j = 0; j < K && apps < maxit; ++j) {
      double mu, gn;
      ND_TRY(ritz_cg(c, X, j, fs, X + j * fs, hi, tol, maxit - apps, &mu, &gn, &apps));
    }
    ND_TRY(orthonormalise(c, X, K, fs));
    ND_TRY(rayleigh_ritz_q2(c, X, AX, Y, K, fs, theta, res));
    apps += K;
    double best;
    l = choose_l_by_gap(theta, l_min, l_max, &best);
    ND_TRY_CUDA(c, cudaMemcpyAsync(Z, X, fs * l, cudaMemcpyDeviceToDevice, c->stream));
    ND_TRY(ritz_of_Q(c, Z, l, nu, rho));
    kappas(nu, rho, theta[l], &kp, &km);
    if (trace)
      std::fprintf(stderr, "nd_lowmodes_ritz: round %d tol %.1e apps %d l %d kappa+ %.3g kappa- %.3g\n", round, tol,
                   apps, l, kp, km);
    if (kp <= kappa_target && km <= kappa_target) {
      converged = true;
      break;
    }
  }
  c->ws["rf_X"].first = X;
  c->ws["rf_AX"].first = AX;
  c->ws["rf_Y"].first = Y;
  if (!converged) return fail(c, ND_ERR_NOT_CONVERGED, "nd_lowmodes_ritz: kappa target not reached");
  return finish_lowmodes(c, Z, l, nu, rho, theta, lam_max, apps, t0, l_out, nu_out, rho_out, evq2_out, info);
}
