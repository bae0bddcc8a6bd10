// Minmax polynomial approximation of sign(x) (host code), Sec. 2.2.
//
// sign(Q) ~ X P_n(X^2), X = Q / ||Q||, with P_n(y) = sum_{k<=n} c_k T_k(z(y)) a Chebyshev series in
// z(y) = (2y - 1 - eps) / (1 - eps), which maps [eps, 1] onto [-1, 1].  The coefficients minimise
// delta = max_{eps <= y <= 1} |h(y)|, h(y) = 1 - sqrt(y) P(y): the weighted best approximation of
// 1/sqrt(y) with weight sqrt(y).  By the alternation theorem the optimum is the polynomial whose
// error reaches its largest modulus with alternating signs at n + 2 points; the Remez exchange
// finds it: solve sqrt(y_i) P(y_i) + (-1)^i E = 1 on a reference y_0 < ... < y_{n+1}, locate the
// n + 1 zeros of h between reference points, take the extremum of |h| between consecutive zeros
// (and the interval ends) as the next reference, and stop when the extrema are level.
// Tables are cached per (n, eps); degree searches per (eps, target).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/nd.h"

namespace {

constexpr int kMaxDegree = 2048;

struct Series {
  int n;
  double eps;
  const std::vector<double>& c;
  double z(double y) const { return (2.0 * y - 1.0 - eps) / (1.0 - eps); }
  // P(y) by the Clenshaw recurrence
  double p(double y) const {
    const double t = z(y);
    double b1 = 0.0, b2 = 0.0;
    for (int k = n; k >= 1; --k) {
      const double b0 = c[k] + 2.0 * t * b1 - b2;
      b2 = b1;
      b1 = b0;
    }
    return c[0] + t * b1 - b2;
  }
  double h(double y) const { return 1.0 - std::sqrt(y) * p(y); }
};

// Solve A x = r in place (row-major m x m) by Gaussian elimination with partial pivoting.
bool solve_dense(std::vector<double>& A, std::vector<double>& r, int m) {
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int i = col + 1; i < m; ++i)
      if (std::fabs(A[(size_t)i * m + col]) > std::fabs(A[(size_t)piv * m + col])) piv = i;
    if (A[(size_t)piv * m + col] == 0.0) return false;
    if (piv != col) {
      for (int j = 0; j < m; ++j) std::swap(A[(size_t)piv * m + j], A[(size_t)col * m + j]);
      std::swap(r[piv], r[col]);
    }
    const double inv = 1.0 / A[(size_t)col * m + col];
    for (int i = col + 1; i < m; ++i) {
      const double f = A[(size_t)i * m + col] * inv;
      if (f == 0.0) continue;
      double* ri = &A[(size_t)i * m];
      const double* rc = &A[(size_t)col * m];
      for (int j = col; j < m; ++j) ri[j] -= f * rc[j];
      r[i] -= f * r[col];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < m; ++j) s -= A[(size_t)i * m + j] * r[j];
    r[i] = s / A[(size_t)i * m + i];
  }
  return true;
}

// Coefficients levelling the error on the reference: sqrt(y_i) P(y_i) + (-1)^i E = 1.
bool level(const std::vector<double>& yref, int n, double eps, std::vector<double>& c) {
  const int m = n + 2;
  std::vector<double> A((size_t)m * m), r(m, 1.0);
  for (int i = 0; i < m; ++i) {
    const double y = yref[i], t = (2.0 * y - 1.0 - eps) / (1.0 - eps), sy = std::sqrt(y);
    double tkm1 = 1.0, tk = t;
    for (int k = 0; k <= n; ++k) {
      double v;
      if (k == 0) {
        v = 1.0;
      } else if (k == 1) {
        v = t;
      } else {
        v = 2.0 * t * tk - tkm1;
        tkm1 = tk;
        tk = v;
      }
      A[(size_t)i * m + k] = sy * v;
    }
    A[(size_t)i * m + n + 1] = (i & 1) ? -1.0 : 1.0;
  }
  if (!solve_dense(A, r, m)) return false;
  c.assign(r.begin(), r.begin() + n + 1);
  return true;
}

// Zero of h in (a, b) where h(a), h(b) have opposite signs (bisection to the last bit).
double zero_between(const Series& S, double a, double b) {
  double ha = S.h(a);
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (a + b);
    if (m <= a || m >= b) break;
    const double hm = S.h(m);
    if (hm == 0.0) return m;
    if ((hm > 0) == (ha > 0)) {
      a = m;
      ha = hm;
    } else {
      b = m;
    }
  }
  return 0.5 * (a + b);
}

// Point of largest |h| on [lo, hi]: sampling, then golden-section search around the best sample.
double extremum(const Series& S, double lo, double hi) {
  constexpr int NS = 32;
  double ys[NS], best = -1.0;
  int j = 0;
  for (int i = 0; i < NS; ++i) {
    ys[i] = lo + (hi - lo) * i / (NS - 1);
    const double v = std::fabs(S.h(ys[i]));
    if (v > best) {
      best = v;
      j = i;
    }
  }
  const double sg = S.h(ys[j]) >= 0 ? 1.0 : -1.0;
  double a = ys[std::max(j - 1, 0)], b = ys[std::min(j + 1, NS - 1)];
  const double gr = 0.6180339887498949;
  double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
  double f1 = sg * S.h(x1), f2 = sg * S.h(x2);
  for (int it = 0; it < 100 && b - a > 1e-16 * b; ++it) {
    if (f1 > f2) {
      b = x2;
      x2 = x1;
      f2 = f1;
      x1 = b - gr * (b - a);
      f1 = sg * S.h(x1);
    } else {
      a = x1;
      x1 = x2;
      f1 = f2;
      x2 = a + gr * (b - a);
      f2 = sg * S.h(x2);
    }
  }
  const double xm = 0.5 * (a + b);
  return sg * S.h(xm) > best ? xm : ys[j];
}

nd_status remez(int n, double eps, std::vector<double>& c, double* delta) {
  const int m = n + 2;
  const double pi = 3.14159265358979323846;
  std::vector<double> yref(m), edges(m + 1), ynew(m);
  for (int i = 0; i < m; ++i) yref[i] = 0.5 * (1.0 + eps) - 0.5 * (1.0 - eps) * std::cos(pi * i / (n + 1));
  for (int it = 0; it < 200; ++it) {
    if (!level(yref, n, eps, c)) return ND_ERR_BREAKDOWN;
    const Series S{n, eps, c};
    bool alternates = true;
    double hprev = S.h(yref[0]), emax = std::fabs(hprev);
    for (int i = 1; i < m; ++i) {
      const double hi = S.h(yref[i]);
      alternates = alternates && hi * hprev < 0;
      emax = std::max(emax, std::fabs(hi));
      hprev = hi;
    }
    if (!alternates) {
      // the levelled error is at the rounding level of h in FP64 and its alternation can no longer
      // be resolved: report the largest |h| on a fine grid (Chebyshev angles) as delta
      if (emax > 1e-12) return ND_ERR_NOT_CONVERGED;
      const int ng = 20 * m;
      double d = 0.0;
      for (int i = 0; i < ng; ++i)
        d = std::max(d, std::fabs(S.h(0.5 * (1.0 + eps) - 0.5 * (1.0 - eps) * std::cos(pi * i / (ng - 1)))));
      *delta = d;
      return ND_OK;
    }
    edges[0] = eps;
    edges[m] = 1.0;
    for (int i = 0; i + 1 < m; ++i) edges[i + 1] = zero_between(S, yref[i], yref[i + 1]);
    double hmax = 0.0, hmin = 1e300;
    for (int i = 0; i < m; ++i) {
      ynew[i] = extremum(S, edges[i], edges[i + 1]);
      const double v = std::fabs(S.h(ynew[i]));
      hmax = std::max(hmax, v);
      hmin = std::min(hmin, v);
    }
    yref = ynew;
    // h is known to a few 1e-15 in FP64, which limits how level small errors can be made
    if (hmax - hmin <= std::max(1e-9 * hmax, 2e-14)) {
      if (!level(yref, n, eps, c)) return ND_ERR_BREAKDOWN;
      const Series F{n, eps, c};
      double d = 0.0;
      for (int i = 0; i < m; ++i) d = std::max(d, std::fabs(F.h(yref[i])));
      *delta = d;
      return ND_OK;
    }
  }
  return ND_ERR_NOT_CONVERGED;
}

struct Entry {
  std::vector<double> c;
  double delta;
};
std::mutex g_mutex;
std::map<std::pair<int, uint64_t>, Entry> g_tables;
std::map<std::pair<uint64_t, uint64_t>, int> g_degrees;

uint64_t bits_of(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
}

nd_status table(int n, double eps, std::vector<double>& c, double* delta) {
  const auto key = std::make_pair(n, bits_of(eps));
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_tables.find(key);
    if (it != g_tables.end()) {
      c = it->second.c;
      *delta = it->second.delta;
      return ND_OK;
    }
  }
  const nd_status st = remez(n, eps, c, delta);
  if (st != ND_OK) return st;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_tables.size() > 256) g_tables.clear();
  g_tables[key] = Entry{c, *delta};
  return ND_OK;
}

}  // namespace

extern "C" nd_status nd_chebyshev(int degree, double eps, double* c, double* delta) {
  if (degree < 0 || degree > kMaxDegree || !(eps > 0.0 && eps < 1.0) || !c) return ND_ERR_INVALID_ARG;
  std::vector<double> cv;
  double d = 0.0;
  const nd_status st = table(degree, eps, cv, &d);
  if (st != ND_OK) return st;
  std::copy(cv.begin(), cv.end(), c);
  if (delta) *delta = d;
  return ND_OK;
}

extern "C" nd_status nd_chebyshev_degree(double eps, double delta_target, int* degree) {
  if (!(eps > 0.0 && eps < 1.0) || !(delta_target > 0.0) || !degree) return ND_ERR_INVALID_ARG;
  const auto key = std::make_pair(bits_of(eps), bits_of(delta_target));
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_degrees.find(key);
    if (it != g_degrees.end()) {
      *degree = it->second;
      return ND_OK;
    }
  }
  std::vector<double> c;
  double d;
  auto delta_of = [&](int n, double* out) { return table(n, eps, c, out); };
  nd_status st = delta_of(0, &d);
  if (st != ND_OK) return st;
  int n = 0;
  if (d > delta_target) {
    // delta(n) does not increase with n, so double, then bisect
    int lo = 0, hi = 1;
    for (;;) {
      if ((st = delta_of(hi, &d)) != ND_OK) return st;
      if (d <= delta_target) break;
      lo = hi;
      hi *= 2;
      if (hi > kMaxDegree) {
        hi = kMaxDegree;
        if ((st = delta_of(hi, &d)) != ND_OK) return st;
        if (d > delta_target) return ND_ERR_INVALID_ARG;
        break;
      }
    }
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if ((st = delta_of(mid, &d)) != ND_OK) return st;
      if (d > delta_target)
        lo = mid;
      else
        hi = mid;
    }
    n = hi;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  g_degrees[key] = n;
  *degree = n;
  return ND_OK;
}
