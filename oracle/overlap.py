"""Deflated sign(Q) and the Neuberger-Dirac operator D_N of the oracle (plain numpy, FP64).

Test infrastructure only.
  D_N = (1 + gamma5 sign(Q)) / abar  (Sec. 2.2), with abar = a / (1 + s), a = 1, so
  1/abar = 1 + s; Q = gamma5 D_W with D_W's mass m = -1 - s gives the paper's
  Q = gamma5 (a D_W - 1 - s).  (abar is not defined in the paper itself; this value is the
  one for which the paper's error bound (2/abar)(1 - abar m/2) equals (2/a)(1 + s - am/2).)
  Massive operator: D_N^m = (1 - abar m_q / 2) D_N + m_q.
  Deflated sign (Sec. 2.3, the formula replacing the polynomial approximation):
     sign(Q) ~ P_+ - P_- + (1 - P_+ - P_-) X R(X^2),  X = Q / ||Q||,
  with R the Zolotarev rational function (oracle/zolotarev.py) in place of P_n.
  Reading: the projector is applied on both sides, (1 - P) X R(X^2) (1 - P), which equals
  the paper's form when V is an exact invariant subspace and keeps the approximation
  Hermitian; ``two_sided=False`` gives the paper's literal left-only form.
  ||Q||^2 is passed in as lam_max (an upper estimate of lambda_max(Q^2)); eps is the lower
  end of the approximation interval of X^2.
  ``sign_apply_poly`` is the same deflated operator with the paper's own minmax polynomial
  X P_n(X^2) evaluated by the Clenshaw recurrence (oracle/chebyshev.py) in place of R.
"""
import numpy as np

from . import chebyshev, mscg, wilson, zolotarev

_zcache = {}


def zolo(npoles, eps):
    key = (int(npoles), float(eps))
    if key not in _zcache:
        _zcache[key] = zolotarev.zolotarev(int(npoles), float(eps))
    return _zcache[key]


def gamma5(psi):
    out = psi.copy()
    out[..., 2:, :] *= -1.0
    return out


def sign_apply(U, dims, m, eta, lam_max, eps, npoles, tol, u=None, nu=None, two_sided=True,
               antiperiodic_t=False, maxit=100000):
    """sign(Q) eta with l = len(nu) deflated modes (u orthonormal, Q u_k ~ nu_k u_k)."""
    Q = lambda v: wilson.apply_Q(U, np.ascontiguousarray(v), dims, m, antiperiodic_t)
    coef = zolo(npoles, eps)
    l = 0 if nu is None else len(nu)
    if l:
        c = np.array([np.vdot(u[k], eta) for k in range(l)])
        eta_perp = eta - np.einsum("k,k...->...", c, u)
    else:
        c = np.zeros(0, dtype=np.complex128)
        eta_perp = eta
    src = eta_perp if (two_sided or not l) else eta
    lam_min = eps if (two_sided or not l) else float(np.min(np.asarray(nu) ** 2)) / lam_max
    tols = mscg.rational_tolerances(coef["b"], coef["sigma"], lam_min, tol)
    x, info = mscg.multishift_cg(lambda v: Q(Q(v)) / lam_max, src, coef["sigma"], tols, maxit=maxit)
    y = np.einsum("l,l...->...", np.asarray(coef["b"]), x)
    z = Q(y) / np.sqrt(lam_max)
    if l:
        cz = np.array([np.vdot(u[k], z) for k in range(l)])
        z = z - np.einsum("k,k...->...", cz, u) + np.einsum("k,k...->...", np.sign(nu) * c, u)
    info = dict(info)
    info["delta"] = coef["delta"]
    return z, info


_ccache = {}


def cheb(degree, eps):
    key = (int(degree), float(eps))
    if key not in _ccache:
        _ccache[key] = chebyshev.minmax(int(degree), float(eps))
    return _ccache[key]


def sign_apply_poly(U, dims, m, eta, lam_max, eps, degree, u=None, nu=None, two_sided=True, antiperiodic_t=False):
    """sign(Q) eta ~ P_+ - P_- + (1 - P) X P_n(X^2) (1 - P) eta (two-sided) with the minmax
    polynomial of the given degree on [eps, 1]; ``two_sided=False`` drops the right projector."""
    Q = lambda v: wilson.apply_Q(U, np.ascontiguousarray(v), dims, m, antiperiodic_t)
    coef = cheb(degree, eps)
    l = 0 if nu is None else len(nu)
    if l:
        c = np.array([np.vdot(u[k], eta) for k in range(l)])
        eta_perp = eta - np.einsum("k,k...->...", c, u)
    else:
        c = np.zeros(0, dtype=np.complex128)
        eta_perp = eta
    src = eta_perp if (two_sided or not l) else eta
    y = chebyshev.poly_apply(lambda v: Q(Q(v)) / lam_max, coef["c"], eps, src)
    z = Q(y) / np.sqrt(lam_max)
    if l:
        cz = np.array([np.vdot(u[k], z) for k in range(l)])
        z = z - np.einsum("k,k...->...", cz, u) + np.einsum("k,k...->...", np.sign(nu) * c, u)
    return z, {"delta": coef["delta"], "degree": int(degree)}


def dn_from_sign(eta, sign_eta, s, m_q=0.0):
    """D_N^m eta from eta and sign(Q) eta (Sec. 2.2): D_N = (1 + gamma5 sign(Q)) / abar,
    abar = 1 / (1 + s), and D_N^m = (1 - abar m_q/2) D_N + m_q."""
    abar = 1.0 / (1.0 + s)
    dn = (eta + gamma5(sign_eta)) / abar
    return (1.0 - abar * m_q / 2.0) * dn + m_q * eta


def dn_apply(U, dims, m, s, eta, lam_max, eps, npoles, tol, u=None, nu=None, m_q=0.0, two_sided=True,
             antiperiodic_t=False, degree=None):
    """D_N^m eta = (1 - abar m_q/2) (1 + s) (eta + gamma5 sign(Q) eta) + m_q eta.  With ``degree``
    given, sign(Q) uses the minmax polynomial of that degree instead of the Zolotarev function."""
    if degree is None:
        sg, info = sign_apply(U, dims, m, eta, lam_max, eps, npoles, tol, u, nu, two_sided, antiperiodic_t)
    else:
        sg, info = sign_apply_poly(U, dims, m, eta, lam_max, eps, degree, u, nu, two_sided, antiperiodic_t)
    return dn_from_sign(eta, sg, s, m_q), info


def propagator(U, dims, m, s, b, lam_max, eps, npoles, tol_inner, u=None, nu=None, m_q=0.1, tol=1e-10,
               maxit=10000, degree=None):
    """x = (D_N^m)^{-1} b by CG on the normal equations D D^dagger y = b, x = D^dagger y, with
    D^dagger = gamma5 D gamma5 (exact for the two-sided, hermitian approximation of sign(Q)).
    Stops at ||b - D D^dagger y|| <= tol ||b||.  Returns x and dict(iters, resid) with resid the
    true relative residual ||b - D x|| / ||b||."""
    D = lambda v: dn_apply(U, dims, m, s, v, lam_max, eps, npoles, tol_inner, u, nu, m_q, degree=degree)[0]
    Dd = lambda v: gamma5(D(gamma5(v)))
    DDd = lambda v: D(Dd(v))
    y = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bn = np.sqrt(np.vdot(b, b).real)
    it = 0
    while np.sqrt(rr) > tol * bn:
        if it >= maxit:
            raise RuntimeError("propagator CG did not converge")
        w = DDd(p)
        alpha = rr / np.vdot(p, w).real
        y = y + alpha * p
        r = r - alpha * w
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    x = Dd(y)
    res = np.linalg.norm(b - D(x)) / bn
    return x, {"iters": it, "resid": float(res)}
