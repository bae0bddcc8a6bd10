"""Zolotarev optimal rational approximation of sign(x), evaluated with mpmath at 40 digits.

Test infrastructure only.  The paper approximates sign(Q) by X P_n(X^2) with a minmax
polynomial and states the uniform error bound delta on sqrt(eps) <= |x| <= 1 (Sec. 2.2,
definition of delta and h(y)).  The hot path replaces the polynomial by the optimal
rational function of the same minmax kind (Zolotarev's solution; see van den Eshof et al.,
Comput. Phys. Commun. 146 (2002) 203, and Chiu et al., Phys. Rev. D 66 (2002) 114502):

  in the scaled variable t = x / sqrt(eps) in [1, 1/sqrt(eps)], with kappa'^2 = 1 - eps and
  K' = K(kappa'^2) the complete elliptic integral,
     c_l = sn^2(l K'/(2n); kappa'^2) / cn^2(l K'/(2n); kappa'^2),    l = 1 .. 2n-1,
     Rhat(t) = t prod_{i=1}^{n-1} (t^2 + c_{2i}) / prod_{i=1}^{n} (t^2 + c_{2i-1}),
     R(t) = d0 Rhat(t), with d0 fixed so that 1 - R equioscillates symmetrically:
     d0 = 2 / (max Rhat + min Rhat),  delta = (max Rhat - min Rhat) / (max Rhat + min Rhat);
  partial fractions  R(t) = t sum_l B_l / (t^2 + c_{2l-1}),
     B_l = d0 prod_{i=1}^{n-1} (c_{2i} - c_{2l-1}) / prod_{j != l} (c_{2j-1} - c_{2l-1});
  back in x = sqrt(eps) t:  R(x) = x sum_l b_l / (x^2 + sigma_l),
     sigma_l = eps c_{2l-1},  b_l = sqrt(eps) B_l.

"n poles" means n denominator factors, i.e. n shifted systems.  Pinned in
tests/test_oracle_zolotarev.py by the Chebyshev alternation property (2n+1 extrema of
1 - R of equal magnitude delta and alternating sign), which characterises the minmax
solution independently of the formula above.
"""
import mpmath as mp

DPS = 40


def _rhat(t, c, n):
    num = t
    for i in range(1, n):
        num *= t * t + c[2 * i]
    den = mp.mpf(1)
    for l in range(1, n + 1):
        den *= t * t + c[2 * l - 1]
    return num / den


def _extrema(f, a, b, samples=4000):
    """Endpoints plus every interior local extremum of f on [a, b], located on a log grid
    and refined by golden-section search on log t."""
    la, lb = mp.log(a), mp.log(b)
    grid = [la + (lb - la) * k / samples for k in range(samples + 1)]
    vals = [f(mp.e ** g) for g in grid]
    pts = [(a, f(a))]
    gr = (mp.sqrt(5) - 1) / 2
    for k in range(1, samples):
        if (vals[k] - vals[k - 1]) * (vals[k + 1] - vals[k]) <= 0:
            sgn = 1 if vals[k] >= vals[k - 1] else -1  # +1: maximum
            lo, hi = grid[k - 1], grid[k + 1]
            x1 = hi - gr * (hi - lo)
            x2 = lo + gr * (hi - lo)
            f1, f2 = sgn * f(mp.e ** x1), sgn * f(mp.e ** x2)
            for _ in range(120):
                if f1 > f2:
                    hi, x2, f2 = x2, x1, f1
                    x1 = hi - gr * (hi - lo)
                    f1 = sgn * f(mp.e ** x1)
                else:
                    lo, x1, f1 = x1, x2, f2
                    x2 = lo + gr * (hi - lo)
                    f2 = sgn * f(mp.e ** x2)
            tm = mp.e ** ((lo + hi) / 2)
            pts.append((tm, f(tm)))
    pts.append((b, f(b)))
    return pts


def zolotarev(n, eps, dps=DPS):
    """Coefficients of R(x) = x sum_l b_l/(x^2 + sigma_l) approximating sign(x) on sqrt(eps) <= |x| <= 1.

    Returns a dict with float lists ``sigma`` (ascending) and ``b``, plus ``d0``, ``delta``
    and the high-precision extrema of 1 - R in x (for the alternation pin).
    """
    with mp.workdps(dps):
        eps_m = mp.mpf(eps)
        m = 1 - eps_m  # parameter kappa'^2
        Kp = mp.ellipk(m)
        c = [None] * (2 * n)
        for l in range(1, 2 * n):
            u = l * Kp / (2 * n)
            sn = mp.ellipfun("sn", u, m=m)
            cn = mp.ellipfun("cn", u, m=m)
            c[l] = (sn / cn) ** 2
        tmax = 1 / mp.sqrt(eps_m)
        pts = _extrema(lambda t: _rhat(t, c, n), mp.mpf(1), tmax)
        vals = [v for _, v in pts]
        vmax, vmin = max(vals), min(vals)
        d0 = 2 / (vmax + vmin)
        delta = (vmax - vmin) / (vmax + vmin)
        B = []
        for l in range(1, n + 1):
            num = d0
            for i in range(1, n):
                num *= c[2 * i] - c[2 * l - 1]
            den = mp.mpf(1)
            for j in range(1, n + 1):
                if j != l:
                    den *= c[2 * j - 1] - c[2 * l - 1]
            B.append(num / den)
        se = mp.sqrt(eps_m)
        sigma = [eps_m * c[2 * l - 1] for l in range(1, n + 1)]
        b = [se * Bl for Bl in B]
        ext_x = [t * se for t, _ in pts]
        ext_err = [1 - d0 * v for _, v in pts]
        return {
            "n": n,
            "eps": float(eps),
            "sigma": [float(s) for s in sigma],
            "b": [float(x) for x in b],
            "d0": float(d0),
            "delta": float(delta),
            "sigma_mp": sigma,
            "b_mp": b,
            "extrema_x": ext_x,
            "extrema_err": ext_err,
        }


def evaluate(coef, x):
    """R(x) = x sum_l b_l / (x^2 + sigma_l) in mpmath (scalar x)."""
    with mp.workdps(DPS):
        x = mp.mpf(x)
        return x * mp.fsum(bl / (x * x + sl) for bl, sl in zip(coef["b_mp"], coef["sigma_mp"]))
