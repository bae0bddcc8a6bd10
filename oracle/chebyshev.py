"""Minmax polynomial approximation of sign(x) and its Clenshaw evaluation (plain numpy, FP64).

Test infrastructure only.  Sec. 2.2 approximates sign(Q) ~ X P_n(X^2), X = Q / ||Q||, with
P_n(y) = sum_{k=0}^{n} c_k T_k a Chebyshev series, its coefficients chosen to minimise
    delta = max_{eps <= y <= 1} |h(y)|,   h(y) = 1 - sqrt(y) P(y),
so that x P(x^2) approximates sign(x) on sqrt(eps) <= |x| <= 1 with uniform error delta, and
evaluates the series with the Clenshaw recurrence.

Readings (the paper is silent on them):
  * T_k acts on the variable of [eps, 1] mapped to [-1, 1]:  z(y) = (2 y - 1 - eps) / (1 - eps).
  * The minmax coefficients are found by the Remez exchange algorithm.  It rests on the
    Chebyshev alternation theorem for the weighted approximation of 1/sqrt(y) by polynomials of
    degree n with weight sqrt(y): the best P is the unique one for which h takes its maximum
    modulus, with alternating signs, at n + 2 points of [eps, 1].  Each exchange step solves
    sqrt(y_i) P(y_i) + (-1)^i E = 1 on the current reference y_0 < ... < y_{n+1}, then moves the
    reference to the extrema of h between the zeros of h.

Pinned in tests/test_oracle_chebyshev.py: n = 0 closed form, a linear-programming solution of the
discretised minimax problem at small n, convexity (no perturbation improves), the alternation
property, the uniform bound against dense sign(Q) = V sgn(Lambda) V^dagger, and
the Clenshaw recurrence against numpy's Chebyshev series evaluation on the eigenvalues.
"""
import numpy as np
from numpy.polynomial import chebyshev as npcheb
from scipy.optimize import brentq, minimize_scalar


def z_of(y, eps):
    """Map [eps, 1] onto [-1, 1]."""
    return (2.0 * np.asarray(y, dtype=np.float64) - 1.0 - eps) / (1.0 - eps)


def p_eval(c, y, eps):
    """P(y) = sum_k c_k T_k(z(y))."""
    return npcheb.chebval(z_of(y, eps), c)


def h_eval(c, y, eps):
    """h(y) = 1 - sqrt(y) P(y)."""
    y = np.asarray(y, dtype=np.float64)
    return 1.0 - np.sqrt(y) * p_eval(c, y, eps)


def _solve_reference(yref, n, eps):
    """Coefficients c_0..c_n and levelled error E with sqrt(y_i) P(y_i) + (-1)^i E = 1."""
    m = n + 2
    A = np.zeros((m, m))
    T = npcheb.chebvander(z_of(yref, eps), n)  # T_k(z_i)
    A[:, : n + 1] = np.sqrt(yref)[:, None] * T
    A[:, n + 1] = (-1.0) ** np.arange(m)
    sol = np.linalg.solve(A, np.ones(m))
    return sol[: n + 1], sol[n + 1]


def _extremum(c, eps, lo, hi, samples=48):
    """Point of largest |h| on [lo, hi] (dense sampling, then bounded refinement)."""
    ys = np.linspace(lo, hi, samples)
    hs = h_eval(c, ys, eps)
    j = int(np.argmax(np.abs(hs)))
    s = 1.0 if hs[j] >= 0 else -1.0
    a = ys[max(j - 1, 0)]
    b = ys[min(j + 1, samples - 1)]
    best_y, best_v = ys[j], abs(hs[j])
    if b > a:
        r = minimize_scalar(lambda t: -s * float(h_eval(c, t, eps)), bounds=(a, b), method="bounded",
                            options={"xatol": 1e-15 * max(1.0, b)})
        if r.success and s * float(h_eval(c, r.x, eps)) > best_v:
            best_y = r.x
    return best_y


def minmax(n, eps, rtol=1e-9, atol=2e-14, maxiter=200):
    """Minmax coefficients of degree n on [eps, 1]: returns dict(c=array[n+1], delta, ref, iters,
    resolved).  Stops when the extrema of |h| agree to rtol relative or atol absolute (h itself is
    only known to a few 1e-15 in FP64, which bounds the levelling of small delta).  When delta is
    at that rounding level the alternation cannot be resolved: resolved = False and delta is the
    largest |h| on a fine grid (an upper estimate, not the minmax value)."""
    if n < 0 or not (0.0 < eps < 1.0):
        raise ValueError("need n >= 0 and 0 < eps < 1")
    # start from the Chebyshev extrema of degree n + 1 mapped onto [eps, 1]
    yref = 0.5 * (1.0 + eps) - 0.5 * (1.0 - eps) * np.cos(np.pi * np.arange(n + 2) / (n + 1))
    for it in range(1, maxiter + 1):
        c, E = _solve_reference(yref, n, eps)
        hr = h_eval(c, yref, eps)
        if np.any(hr[1:] * hr[:-1] >= 0):
            # the levelled error is at the rounding level of h: the alternation can no longer be
            # resolved in FP64; report the largest |h| on a fine grid as delta
            if abs(E) > 1e-12:
                raise RuntimeError("Remez exchange lost the alternation")
            grid = 0.5 * (1 + eps) - 0.5 * (1 - eps) * np.cos(np.linspace(0, np.pi, 20 * (n + 2)))
            return {"c": c, "delta": float(np.max(np.abs(h_eval(c, grid, eps)))), "ref": yref, "iters": it,
                    "resolved": False}
        # zeros of h between consecutive reference points (h alternates there by construction)
        roots = [brentq(lambda t: float(h_eval(c, t, eps)), yref[i], yref[i + 1], xtol=1e-16, rtol=1e-15)
                 for i in range(n + 1)]
        edges = [eps] + roots + [1.0]
        ynew = np.array([_extremum(c, eps, edges[i], edges[i + 1]) for i in range(n + 2)])
        hv = np.abs(h_eval(c, ynew, eps))
        yref = ynew
        if hv.max() - hv.min() <= max(rtol * hv.max(), atol):
            c, E = _solve_reference(yref, n, eps)
            return {"c": c, "delta": float(np.abs(h_eval(c, yref, eps)).max()), "ref": yref, "iters": it,
                    "resolved": True}
    raise RuntimeError("Remez exchange did not converge")


def degree_for(eps, delta_target, nmax=4000):
    """Smallest degree n with minmax delta(n) <= delta_target.  delta(n) does not increase
    with n (degree-n polynomials are among those of degree n + 1), so bisection applies."""
    if minmax(0, eps)["delta"] <= delta_target:
        return 0
    lo, hi = 0, 1
    while minmax(hi, eps)["delta"] > delta_target:
        lo, hi = hi, 2 * hi
        if hi > nmax:
            raise ValueError("degree above nmax")
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if minmax(mid, eps)["delta"] > delta_target:
            lo = mid
        else:
            hi = mid
    return hi


def clenshaw(apply_A, c, v):
    """sum_k c_k T_k(A) v by the Clenshaw recurrence (A maps into [-1, 1]):
    b_k = c_k v + 2 A b_{k+1} - b_{k+2} (k = n .. 1, b_{n+1} = b_{n+2} = 0), result
    c_0 v + A b_1 - b_2."""
    b1 = np.zeros_like(v)
    b2 = np.zeros_like(v)
    for k in range(len(c) - 1, 0, -1):
        b0 = c[k] * v + 2.0 * apply_A(b1) - b2
        b2, b1 = b1, b0
    return c[0] * v + apply_A(b1) - b2


def poly_apply(apply_X2, c, eps, v):
    """P_n(X^2) v with A = z(X^2) = (2 X^2 - 1 - eps) / (1 - eps)."""
    A = lambda w: (2.0 * apply_X2(w) - (1.0 + eps) * w) / (1.0 - eps)
    return clenshaw(A, c, v)
