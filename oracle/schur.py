"""Even-odd (Schur complement) preconditioned Wilson operator of the oracle (plain numpy, FP64).

Test infrastructure only.  Sec. 2.1 splits the lattice into even and odd sites (the hopping
term of D_W only connects the two), so that

    D_W = [[D_ee, D_eo], [D_oe, D_oo]],   D_ee = D_oo = (4 + m),   D_eo, D_oe = the hopping blocks.

The Schur complement on the even sites,  Dhat = (4 + m) - D_eo D_oe / (4 + m),  and
Qhat = gamma5 Dhat (hermitian, as Q is) give D_W x = b by
    Dhat x_e = b_e - D_eo b_o / (4 + m),   x_o = (b_o - D_oe x_e) / (4 + m).
With Q = gamma5 D_W and Q^2 = D_W^dagger D_W, (Q^2)^{-1} phi = D_W^{-1} gamma5 D_W^{-1} gamma5 phi; each
D_W^{-1} is one even-site solve, here by CG on the normal equations Qhat^2 x_e = Qhat gamma5 bhat_e.

Fields are full-lattice spinors in the oracle's lex layout [V][4][3]; "even" fields are zero on odd
sites.  The blocks are taken from the oracle's D_W applied to fields supported on one parity.
Pinned in tests/test_oracle_schur.py by the block-LDU determinant identity
det D_W = (4 + m)^{12 V/2} det Dhat, hermiticity of Qhat, and dense LAPACK solves.
"""
import numpy as np

from . import wilson


def parity_mask(dims):
    """1.0 on even sites, 0.0 on odd sites, shape [V, 1, 1]."""
    V = int(np.prod(dims))
    x = np.array(np.unravel_index(np.arange(V), dims)).T
    return ((x.sum(axis=1) % 2) == 0).astype(np.float64)[:, None, None]


def _g5(v):
    out = v.copy()
    out[..., 2:, :] *= -1.0
    return out


def blocks(U, dims, m, antiperiodic_t=False):
    """Functions P_e D_W P_o and P_o D_W P_e (the hopping blocks) and the masks."""
    even = parity_mask(dims)
    odd = 1.0 - even
    DW = lambda v: wilson.apply_DW(U, np.ascontiguousarray(v), dims, m, antiperiodic_t)
    D_eo = lambda v: even * DW(odd * v)
    D_oe = lambda v: odd * DW(even * v)
    return D_eo, D_oe, even, odd


def qhat_apply(U, dims, m, v, antiperiodic_t=False):
    """Qhat v_e = gamma5 ((4 + m) v_e - D_eo D_oe v_e / (4 + m)) for v supported on even sites."""
    D_eo, D_oe, even, _ = blocks(U, dims, m, antiperiodic_t)
    ve = even * v
    return _g5((4.0 + m) * ve - D_eo(D_oe(ve)) / (4.0 + m))


def _cg(apply_A, b, tol, maxit):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bn = np.sqrt(rr)
    it = 0
    while np.sqrt(rr) > tol * bn:
        if it >= maxit:
            raise RuntimeError("CG did not converge")
        w = apply_A(p)
        a = rr / np.vdot(p, w).real
        x = x + a * p
        r = r - a * w
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def dw_solve(U, dims, m, b, tol=1e-12, maxit=100000, antiperiodic_t=False):
    """x = D_W^{-1} b through the even-site Schur complement (CG on Qhat^2)."""
    D_eo, D_oe, even, odd = blocks(U, dims, m, antiperiodic_t)
    Qh = lambda v: qhat_apply(U, dims, m, v, antiperiodic_t)
    bhat = even * b - D_eo(odd * b) / (4.0 + m)
    rhs = Qh(_g5(bhat))
    xe, it = _cg(lambda v: Qh(Qh(v)), rhs, tol, maxit)
    xo = (odd * b - D_oe(xe)) / (4.0 + m)
    return xe + xo, it


def q2_solve(U, dims, m, phi, tol=1e-12, maxit=100000, antiperiodic_t=False):
    """(Q^2)^{-1} phi = D_W^{-1} gamma5 D_W^{-1} gamma5 phi by two Schur-complement solves."""
    y, it1 = dw_solve(U, dims, m, _g5(phi), tol, maxit, antiperiodic_t)
    x, it2 = dw_solve(U, dims, m, _g5(y), tol, maxit, antiperiodic_t)
    return x, it1 + it2
