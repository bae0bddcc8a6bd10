"""Pseudofermion action S = phi^dagger (Q^2)^{-1} phi and its force (plain numpy + oracle C).

Test infrastructure only.  The force formula is derived in oracle/wilson.c from the
definition of D_W (Sec. 2.1); X = (Q^2)^{-1} phi comes from the oracle's CG.
"""
import numpy as np

from . import mscg, wilson


def solve_Q2(U, dims, m, phi, tol=1e-13, antiperiodic_t=False):
    x, info = mscg.multishift_cg(lambda v: wilson.apply_Q2(U, v, dims, m, antiperiodic_t), phi, [0.0], tol)
    return x[0], info


def action(U, dims, m, phi, tol=1e-13, antiperiodic_t=False):
    X, _ = solve_Q2(U, dims, m, phi, tol, antiperiodic_t)
    return float(np.vdot(phi, X).real)


def force(U, dims, m, phi, tol=1e-13, antiperiodic_t=False):
    """F[mu, lex, a] = dS / d omega^a_mu(x) for U_mu(x) -> exp(i omega^a T^a) U_mu(x)."""
    X, _ = solve_Q2(U, dims, m, phi, tol, antiperiodic_t)
    Y = wilson.apply_Q(U, X, dims, m, antiperiodic_t)
    return wilson.force(U, X, Y, dims, antiperiodic_t)


def exp_i_omega_T(omega):
    """exp(i omega^a T^a) for omega[..., 8] (T^a = lambda^a/2), via eigendecomposition."""
    lam = np.stack([wilson.gellmann(a) for a in range(1, 9)])
    H = np.einsum("...a,aij->...ij", omega, lam) / 2.0
    w, v = np.linalg.eigh(H)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), v.conj())


def rotate_links(U, omega, h):
    """U_mu(x) -> exp(i h omega^a_mu(x) T^a) U_mu(x) for every link."""
    return np.ascontiguousarray(np.einsum("...ij,...jk->...ik", exp_i_omega_T(h * omega), U))
