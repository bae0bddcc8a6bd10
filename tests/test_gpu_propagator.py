"""GPU parity of the massive overlap propagator x = (D_N^m)^{-1} b (nd_propagator, chiral-sector
CG with one sign(Q) per iteration) against the oracle (CG on the normal equations D D^dagger,
oracle/overlap.py) and against the dense LAPACK solve of D_N^m built from the exact sign(Q), on
the 4^4 Haar lattice with its 8 exact low modes injected."""
import numpy as np
import pytest

import synth
from oracle import chebyshev, lowmodes, overlap
from tests.gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu
M, S = -1.4, 0.4


@pytest.fixture(scope="module")
def nd():
    import paper_1010_5636_gb300 as nd
    nd.lib()
    return nd


@pytest.fixture(scope="module")
def cfg1():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    lm = lowmodes.lowmodes_dense(U, dims, M, 8)
    lam_max = 1.01 * lm["lam_max"]
    eps = 0.99 * lm["lam_next"] / lam_max
    return dims, U, lm, lam_max, eps


def _ctx(nd, dims, U, lm):
    ctx = nd.nd_create(dims, antiperiodic_t=False, m=M, s=S)
    nd.nd_set_links(ctx, dev(U), (18, 12, 12))
    nd.nd_set_lowmodes(ctx, dev(lm["u"]), list(lm["nu"]), lm["lam_next"])
    return ctx


def _sources(dims):
    V = int(np.prod(dims))
    point = np.zeros((V, 4, 3), dtype=np.complex128)
    point[0, 1, 2] = 1.0  # spin 1: gamma5 = +1, one chirality
    return {"point": point, "gauss": synth.spinor(dims, seed=9)}


@pytest.mark.parametrize("inner", [0, 1])
@pytest.mark.parametrize("source", ["point", "gauss"])
@pytest.mark.parametrize("m_q", [0.2, 0.05])
def test_vs_oracle(nd, cfg1, inner, source, m_q):
    import torch
    dims, U, lm, lam_max, eps = cfg1
    b = _sources(dims)[source]
    ref, rinfo = overlap.propagator(U, dims, M, S, b, lam_max, eps, 16, 1e-12, lm["u"], lm["nu"], m_q=m_q,
                                    tol=1e-11)
    ctx = _ctx(nd, dims, U, lm)
    try:
        # sign(Q) to 1e-12: the mixed-precision refinement reaches about that far in FP64
        p = nd.dn_params(16, eps, lam_max, 1e-12, 20000, inner, m_q, False)
        x = torch.empty_like(dev(b))
        info = nd.nd_propagator(ctx, x, dev(b), p, tol=1e-11, maxit=5000)
        err = rel(host(x), ref)
        print(f"{source} m_q {m_q} inner {inner}: iters {info.iters} sign_iters {info.sign_iters} "
              f"resid {info.resid:.2e} err {err:.2e}")
        assert info.resid <= 5e-11
        # both sides reach a relative residual ~1e-11 of operators that differ by the sign(Q)
        # solver tolerance (1e-12 relative, times 1 + s), and ||D^-1|| <= 1/m_q
        assert err <= (5e-11 + (1 + S) * 2e-12) / m_q
        if source == "point":
            # one chirality only: the other sector costs nothing
            assert info.iters <= rinfo["iters"] + 5
    finally:
        nd.nd_destroy(ctx)


def test_vs_dense_and_chebyshev(nd, cfg1):
    """Against LAPACK on the dense D_N^m from the exact sign, with both approximations of sign(Q)."""
    import torch
    dims, U, lm, lam_max, eps = cfg1
    m_q = 0.1
    b = synth.spinor(dims, seed=10)
    w, v = lm["spectrum"], lm["eigvecs"]
    S_ex = (v * np.sign(w)) @ v.conj().T
    n = b.size
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), n // 12)
    abar = 1.0 / (1.0 + S)
    D_ex = (1.0 - abar * m_q / 2.0) * (1.0 + S) * (np.eye(n) + g5[:, None] * S_ex) + m_q * np.eye(n)
    x_ex = np.linalg.solve(D_ex, b.reshape(-1))
    degree = chebyshev.degree_for(eps, 1e-12)
    ctx = _ctx(nd, dims, U, lm)
    try:
        for p in (nd.dn_params(16, eps, lam_max, 1e-13, 20000, 0, m_q, False),
                  nd.dn_params(0, eps, lam_max, 1e-12, 1, 0, m_q, False, approx=nd.ND_SIGN_CHEBYSHEV, degree=degree)):
            x = torch.empty_like(dev(b))
            info = nd.nd_propagator(ctx, x, dev(b), p, tol=1e-11, maxit=5000)
            xh = host(x).reshape(-1)
            # ||x - x_ex|| <= (||b - D x|| + ||D - D_ex|| ||x||) / m_q, ||D - D_ex|| <= (1 + s)(delta + solver error)
            bound = (info.resid * np.linalg.norm(b) + (1 + S) * 2e-12 * np.linalg.norm(xh)) / m_q
            assert np.linalg.norm(xh - x_ex) <= bound
    finally:
        nd.nd_destroy(ctx)


def test_edge_cases(nd, cfg1):
    import torch
    dims, U, lm, lam_max, eps = cfg1
    b = synth.spinor(dims, seed=11)
    ctx = _ctx(nd, dims, U, lm)
    try:
        x = torch.empty_like(dev(b))
        info = nd.nd_propagator(ctx, x, torch.zeros_like(dev(b)), nd.dn_params(16, eps, lam_max, 1e-12, 20000, 0, 0.1))
        assert info.iters == 0 and float(x.abs().max()) == 0.0
        with pytest.raises(nd.NdError) as e:
            nd.nd_propagator(ctx, x, dev(b), nd.dn_params(16, eps, lam_max, 1e-12, 20000, 0, 0.1, True))
        assert e.value.status == nd.ND_ERR_INVALID_ARG
        with pytest.raises(nd.NdError) as e:
            nd.nd_propagator(ctx, x, dev(b), nd.dn_params(16, eps, lam_max, 1e-12, 20000, 0, 0.1), tol=1e-11, maxit=2)
        assert e.value.status == nd.ND_ERR_NOT_CONVERGED
        # the context stays usable after the failure
        info = nd.nd_propagator(ctx, x, dev(b), nd.dn_params(16, eps, lam_max, 1e-12, 20000, 0, 0.1), tol=1e-9)
        assert info.resid <= 5e-9
    finally:
        nd.nd_destroy(ctx)


def test_inexact_sign_needs_outer_passes(nd, cfg1):
    """With a sign(Q) accurate to ~1e-6 only (a low-degree polynomial), H = D D^dagger no longer holds
    to the solve tolerance; the defect correction still brings ||b - D x|| below tol."""
    import torch
    dims, U, lm, lam_max, eps = cfg1
    b = synth.spinor(dims, seed=12)
    degree = chebyshev.degree_for(eps, 1e-6)
    ctx = _ctx(nd, dims, U, lm)
    try:
        p = nd.dn_params(0, eps, lam_max, 1e-6, 1, 0, 0.1, False, approx=nd.ND_SIGN_CHEBYSHEV, degree=degree)
        x = torch.empty_like(dev(b))
        info = nd.nd_propagator(ctx, x, dev(b), p, tol=1e-10, maxit=5000)
        print(f"degree {degree}: passes {info.outer}, CG iterations {info.iters}, resid {info.resid:.2e}")
        assert info.resid <= 1e-10
        assert info.outer >= 2
    finally:
        nd.nd_destroy(ctx)
