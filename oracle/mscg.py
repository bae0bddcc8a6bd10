"""Multi-shift conjugate gradient of the oracle (plain numpy, FP64).

Test infrastructure only.  Solves (A + sigma_l) x_l = b for all shifts from one Krylov
space (B. Jegerlehner, hep-lat/9612014).  The paper evaluates its sign approximation with
a Clenshaw recurrence (Sec. 2.2); the rational (Zolotarev) form needs these shifted
inverses instead.  Steps, with sigma_0 the smallest shift as the base system:

  x_l = 0, r = p_l = b, zeta_l^{-1} = zeta_l^{0} = 1, alpha_{-1} = 1, beta_{-1} = 0
  repeat j = 0, 1, ...:
    w = (A + sigma_0) p_0,  alpha_j = (r, r) / (p_0, w)
    zeta_l^{j+1} = zeta_l^j zeta_l^{j-1} alpha_{j-1}
                   / [alpha_j beta_{j-1} (zeta_l^{j-1} - zeta_l^j) + zeta_l^{j-1} alpha_{j-1} (1 + (sigma_l - sigma_0) alpha_j)]
    alpha_l = alpha_j zeta_l^{j+1} / zeta_l^j,   x_l += alpha_l p_l
    r -= alpha_j w,  beta_j = (r, r)_new / (r, r)_old
    beta_l = beta_j (zeta_l^{j+1} / zeta_l^j)^2, p_l = zeta_l^{j+1} r + beta_l p_l

The residual of shift l is zeta_l r (collinear residuals).  Stopping: shift l is frozen
(no further updates of x_l, p_l) once |zeta_l| ||r|| <= tol_l ||b||; the iteration ends
when every shift is frozen.  ``rational_tolerances`` gives the per-shift targets that bound
the error of sum_l b_l x_l (see its docstring).
"""
import numpy as np


class NotConverged(RuntimeError):
    pass


def rational_tolerances(b, sigma, lam_min, tol):
    """Per-shift residual targets for y = sum_l b_l x_l.

    With A >= lam_min on the space solved in, ||x_l - x_l*|| <= ||r_l|| / (lam_min + sigma_l),
    so requiring |b_l| ||r_l|| / (lam_min + sigma_l) <= tol ||b|| / n for every l bounds
    ||y - y*|| <= tol ||b||.  Returns tol_l = tol (lam_min + sigma_l) / (n |b_l|).
    """
    n = len(sigma)
    return [tol * (lam_min + s) / (n * abs(bl)) for bl, s in zip(b, sigma)]


def multishift_cg(apply_A, b, sigma, tol, maxit=100000):
    """Solve (A + sigma_l) x_l = b for every l.

    apply_A: callable v -> A v (A Hermitian positive semi-definite, sigma_0 + A > 0).
    sigma:   shifts (any order; the smallest is the base system).
    tol:     scalar or per-shift list of relative residual targets.
    Returns (x [n, *b.shape], info dict with iterations and final per-shift residual estimates).
    """
    sigma = [float(s) for s in sigma]
    n = len(sigma)
    tols = [float(tol)] * n if np.isscalar(tol) else [float(t) for t in tol]
    base = int(np.argmin(sigma))
    s0 = sigma[base]
    bnorm = np.sqrt(np.vdot(b, b).real)
    x = np.zeros((n,) + b.shape, dtype=b.dtype)
    if bnorm == 0.0:
        return x, {"iters": 0, "res": [0.0] * n}
    r = b.copy()
    p = [b.copy() for _ in range(n)]
    zeta_prev = [1.0] * n
    zeta = [1.0] * n
    alpha_prev, beta_prev = 1.0, 0.0
    rr = np.vdot(r, r).real
    active = [True] * n
    res = [1.0] * n
    it = 0
    while any(active):
        if it >= maxit:
            raise NotConverged(f"multi-shift CG: {it} iterations")
        w = apply_A(p[base]) + s0 * p[base]
        alpha = rr / np.vdot(p[base], w).real
        # the base system keeps driving the recurrence even after its own x is final
        live = [l for l in range(n) if active[l] or l == base]
        zeta_next = [0.0] * n
        for l in live:
            ds = sigma[l] - s0
            zeta_next[l] = (zeta[l] * zeta_prev[l] * alpha_prev
                            / (alpha * beta_prev * (zeta_prev[l] - zeta[l]) + zeta_prev[l] * alpha_prev * (1.0 + ds * alpha)))
            if active[l]:
                x[l] += (alpha * zeta_next[l] / zeta[l]) * p[l]
        r = r - alpha * w
        rr_new = np.vdot(r, r).real
        beta = rr_new / rr
        for l in live:
            beta_l = beta * (zeta_next[l] / zeta[l]) ** 2
            p[l] = zeta_next[l] * r + beta_l * p[l]
            zeta_prev[l], zeta[l] = zeta[l], zeta_next[l]
        alpha_prev, beta_prev = alpha, beta
        rr = rr_new
        it += 1
        rnorm = np.sqrt(rr)
        for l in range(n):
            if active[l]:
                res[l] = abs(zeta[l]) * rnorm / bnorm
                if res[l] <= tols[l]:
                    active[l] = False
    return x, {"iters": it, "res": res}
