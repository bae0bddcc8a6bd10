// Zolotarev optimal rational approximation of sign(x) on sqrt(eps) <= |x| <= 1 (host code).
//
// The paper approximates sign(Q) by a minmax polynomial with uniform error delta on
// sqrt(eps) <= |x| <= 1 (Sec. 2.2); the rational minmax solution of the same problem is
// Zolotarev's.  In t = x / sqrt(eps) in [1, 1/sqrt(eps)], with kappa'^2 = 1 - eps and
// K' = K(kappa'^2):
//   c_l = sn^2 / cn^2 (l K'/(2n); kappa'^2),  l = 1 .. 2n-1,
//   Rhat(t) = t prod_{i<n} (t^2 + c_{2i}) / prod_{l<=n} (t^2 + c_{2l-1}),
//   R = d0 Rhat with d0 = 2 / (max Rhat + min Rhat) over the interval (symmetric
//   equioscillation), delta = (max - min) / (max + min);
//   R(t) = t sum_l B_l / (t^2 + c_{2l-1}), B_l = d0 prod_i (c_{2i} - c_{2l-1}) / prod_{j!=l} (c_{2j-1} - c_{2l-1});
//   in x: sigma_l = eps c_{2l-1}, b_l = sqrt(eps) B_l.
// Jacobi functions by the arithmetic-geometric mean (Abramowitz & Stegun 16.4), started from
// the complementary parameter eps itself so that kappa' close to 1 loses no digits; long
// double throughout.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/nd.h"

namespace {

typedef long double ld;

// sn and cn of (u | m) with m1 = 1 - m given directly.
void jacobi_sn_cn(ld u, ld m, ld m1, ld* sn, ld* cn) {
  ld a[64], c[64];
  a[0] = 1.0L;
  ld b = sqrtl(m1);
  c[0] = sqrtl(m);
  int n = 0;
  while (n < 60 && fabsl(c[n]) > 1e-30L * a[n]) {
    a[n + 1] = 0.5L * (a[n] + b);
    c[n + 1] = 0.5L * (a[n] - b);
    b = sqrtl(a[n] * b);
    ++n;
  }
  ld phi = ldexpl(a[n] * u, n);
  for (int k = n; k >= 1; --k) phi = 0.5L * (phi + asinl(c[k] / a[k] * sinl(phi)));
  *sn = sinl(phi);
  *cn = cosl(phi);
}

// Complete elliptic integral K(m) with m1 = 1 - m given directly: pi / (2 AGM(1, sqrt(m1))).
ld ellip_k(ld m1) {
  ld a = 1.0L, b = sqrtl(m1);
  for (int k = 0; k < 60 && fabsl(a - b) > 1e-30L * a; ++k) {
    ld an = 0.5L * (a + b);
    b = sqrtl(a * b);
    a = an;
  }
  return 3.14159265358979323846264338327950288L / (2.0L * a);
}

ld rhat(ld t, const std::vector<ld>& c, int n) {
  ld num = t, den = 1.0L;
  for (int i = 1; i < n; ++i) num *= t * t + c[2 * i];
  for (int l = 1; l <= n; ++l) den *= t * t + c[2 * l - 1];
  return num / den;
}

}  // namespace

namespace {
// Tables already computed in this process, keyed by (n, eps bits): the extended-precision
// computation is slow on hosts whose long double is emulated in software, and D_N asks for the
// same table on every application.
struct ZoloEntry {
  std::vector<double> sigma, b;
  double delta;
};
std::mutex g_zmutex;
std::map<std::pair<int, uint64_t>, ZoloEntry> g_zcache;
}  // namespace

static nd_status zolotarev_compute(int n, double eps, double* sigma, double* b, double* delta);

extern "C" nd_status nd_zolotarev(int n, double eps, double* sigma, double* b, double* delta) {
  if (n < 1 || n > 64 || !(eps > 0.0 && eps < 1.0) || !sigma || !b) return ND_ERR_INVALID_ARG;
  uint64_t bits;
  std::memcpy(&bits, &eps, sizeof(bits));
  const auto key = std::make_pair(n, bits);
  {
    std::lock_guard<std::mutex> lock(g_zmutex);
    auto it = g_zcache.find(key);
    if (it != g_zcache.end()) {
      std::copy(it->second.sigma.begin(), it->second.sigma.end(), sigma);
      std::copy(it->second.b.begin(), it->second.b.end(), b);
      if (delta) *delta = it->second.delta;
      return ND_OK;
    }
  }
  double d = 0.0;
  const nd_status st = zolotarev_compute(n, eps, sigma, b, &d);
  if (st != ND_OK) return st;
  if (delta) *delta = d;
  std::lock_guard<std::mutex> lock(g_zmutex);
  ZoloEntry e;
  e.sigma.assign(sigma, sigma + n);
  e.b.assign(b, b + n);
  e.delta = d;
  if (g_zcache.size() > 256) g_zcache.clear();
  g_zcache[key] = e;
  return ND_OK;
}

static nd_status zolotarev_compute(int n, double eps, double* sigma, double* b, double* delta) {
  const ld e = (ld)eps;
  const ld m = 1.0L - e;
  const ld Kp = ellip_k(e);
  std::vector<ld> c(2 * n + 1, 0.0L);
  for (int l = 1; l < 2 * n; ++l) {
    ld sn, cn;
    jacobi_sn_cn((ld)l * Kp / (2.0L * n), m, e, &sn, &cn);
    c[l] = (sn / cn) * (sn / cn);
  }
  // Extrema of Rhat on [1, 1/sqrt(eps)]: endpoints plus local extrema located on a log grid
  // and refined by golden-section search in log t.
  const ld la = 0.0L, lb = -0.5L * logl(e);
  const int S = 20000;
  std::vector<ld> v(S + 1);
  for (int k = 0; k <= S; ++k) v[k] = rhat(expl(la + (lb - la) * k / S), c, n);
  ld vmax = std::max(v[0], v[S]), vmin = std::min(v[0], v[S]);
  const ld gr = 0.61803398874989484820458683436563811L;
  for (int k = 1; k < S; ++k) {
    if ((v[k] - v[k - 1]) * (v[k + 1] - v[k]) > 0) continue;
    const ld sg = v[k] >= v[k - 1] ? 1.0L : -1.0L;
    ld lo = la + (lb - la) * (k - 1) / S, hi = la + (lb - la) * (k + 1) / S;
    ld x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    ld f1 = sg * rhat(expl(x1), c, n), f2 = sg * rhat(expl(x2), c, n);
    for (int it = 0; it < 100; ++it) {
      if (f1 > f2) {
        hi = x2; x2 = x1; f2 = f1;
        x1 = hi - gr * (hi - lo);
        f1 = sg * rhat(expl(x1), c, n);
      } else {
        lo = x1; x1 = x2; f1 = f2;
        x2 = lo + gr * (hi - lo);
        f2 = sg * rhat(expl(x2), c, n);
      }
    }
    const ld val = rhat(expl(0.5L * (lo + hi)), c, n);
    vmax = std::max(vmax, val);
    vmin = std::min(vmin, val);
  }
  const ld d0 = 2.0L / (vmax + vmin);
  if (delta) *delta = (double)((vmax - vmin) / (vmax + vmin));
  const ld se = sqrtl(e);
  for (int l = 1; l <= n; ++l) {
    ld num = d0, den = 1.0L;
    for (int i = 1; i < n; ++i) num *= c[2 * i] - c[2 * l - 1];
    for (int j = 1; j <= n; ++j)
      if (j != l) den *= c[2 * j - 1] - c[2 * l - 1];
    sigma[l - 1] = (double)(e * c[2 * l - 1]);
    b[l - 1] = (double)(se * num / den);
  }
  return ND_OK;
}
