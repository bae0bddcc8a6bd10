"""GPU parity of sign(Q) and D_N with the paper's minmax polynomial X P_n(X^2) evaluated by the
Clenshaw recurrence (Sec. 2.2) against the oracle's Remez table and Clenshaw evaluation, through
the C-ABI: deflated (two-sided and left-only) and undeflated, FP64 / FP32 / FP16 recurrences,
degrees 0, 1 and 2 (the special branches of the recurrence) and the zero source."""
import numpy as np
import pytest

import synth
from oracle import chebyshev, lowmodes, overlap
from tests.gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu
M, S = -1.4, 0.4
CHEB = 1
# Relative agreement with the FP64 oracle.  FP64: both sides evaluate the same polynomial (their
# coefficient tables agree to ~1e-14) with different rounding order.  FP32 / FP16: the recurrence
# runs in that storage precision; rounding grows about linearly with the degree (measured at
# degree 145 on 4^4: FP64 2.6e-15, FP32 7.9e-7, FP16 1.4e-3).
TOL = {0: 1e-10, 1: 1e-5, 2: 1e-2}


@pytest.fixture(scope="module")
def nd():
    import paper_1010_5636_gb300 as nd
    nd.lib()
    return nd


@pytest.fixture(scope="module")
def cfg1():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    eta = synth.spinor(dims, seed=1)
    lm = lowmodes.lowmodes_dense(U, dims, M, 8)
    lam_max = 1.01 * lm["lam_max"]
    eps = 0.99 * lm["lam_next"] / lam_max
    degree = chebyshev.degree_for(eps, 1e-10)
    return dims, U, eta, lm, lam_max, eps, degree


def _ctx(nd, dims, U, recon=(18, 12, 12)):
    ctx = nd.nd_create(dims, antiperiodic_t=False, m=M, s=S)
    nd.nd_set_links(ctx, dev(U), recon)
    return ctx


@pytest.mark.parametrize("inner", [0, 1, 2])
@pytest.mark.parametrize("left_only", [False, True])
def test_sign_and_dn_vs_oracle(nd, cfg1, inner, left_only):
    import torch
    dims, U, eta, lm, lam_max, eps, degree = cfg1
    ref_sign, rinfo = overlap.sign_apply_poly(U, dims, M, eta, lam_max, eps, degree, lm["u"], lm["nu"],
                                              two_sided=not left_only)
    ref_dn, _ = overlap.dn_apply(U, dims, M, S, eta, lam_max, eps, 0, 0, lm["u"], lm["nu"], two_sided=not left_only,
                                 degree=degree)
    ctx = _ctx(nd, dims, U)
    try:
        nd.nd_set_lowmodes(ctx, dev(lm["u"]), list(lm["nu"]), lm["lam_next"])
        p = nd.dn_params(0, eps, lam_max, 1e-10, 1, inner, 0.0, left_only, approx=CHEB, degree=degree)
        out = torch.empty_like(dev(eta))
        info = nd.nd_apply_sign(ctx, out, dev(eta), p)
        err_s = rel(host(out), ref_sign)
        info = nd.nd_apply_DN(ctx, out, dev(eta), p)
        err_d = rel(host(out), ref_dn)
        print(f"inner {inner} left_only {left_only} degree {degree}: sign {err_s:.3e} D_N {err_d:.3e}")
        assert err_s <= TOL[inner] and err_d <= TOL[inner]
        assert info.degree == degree and info.n_low == 8
        assert info.delta == pytest.approx(rinfo["delta"], rel=1e-6, abs=5e-14)
    finally:
        nd.nd_destroy(ctx)


def test_auto_degree_and_exact_bound(nd, cfg1):
    """degree = 0 picks the smallest degree with delta <= tol; the result stays within delta of
    the exact sign(Q) from the dense eigendecomposition (exact low modes injected)."""
    import torch
    dims, U, eta, lm, lam_max, eps, degree = cfg1
    w, v = lm["spectrum"], lm["eigvecs"]
    exact = ((v * np.sign(w)) @ v.conj().T) @ eta.reshape(-1)
    ctx = _ctx(nd, dims, U)
    try:
        nd.nd_set_lowmodes(ctx, dev(lm["u"]), list(lm["nu"]), lm["lam_next"])
        out = torch.empty_like(dev(eta))
        info = nd.nd_apply_sign(ctx, out, dev(eta), nd.dn_params(0, eps, lam_max, 1e-10, 1, 0, approx=CHEB))
        assert info.degree == degree
        assert info.delta <= 1e-10
        err = np.linalg.norm(host(out).reshape(-1) - exact) / np.linalg.norm(eta)
        assert err <= info.delta + 1e-11
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("degree", [0, 1, 2, 7])
def test_low_degrees_undeflated(nd, cfg1, degree):
    """The n = 0, 1, 2 branches of the recurrence, no low modes, eps below the spectrum."""
    import torch
    dims, U, eta, lm, lam_max, _, _ = cfg1
    eps = 0.99 * float(np.min(lm["spectrum"] ** 2)) / lam_max
    if degree == 0:
        # degree 0 is not asked for by value (0 means automatic): take the n = 0 table through tol
        tol = chebyshev.minmax(0, eps)["delta"] * (1 + 1e-9)
        assert chebyshev.degree_for(eps, tol) == 0
    else:
        tol = 1e-10
    ref, _ = overlap.sign_apply_poly(U, dims, M, eta, lam_max, eps, degree)
    ctx = _ctx(nd, dims, U)
    try:
        out = torch.empty_like(dev(eta))
        info = nd.nd_apply_sign(ctx, out, dev(eta), nd.dn_params(0, eps, lam_max, tol, 1, 0, approx=CHEB,
                                                                  degree=degree))
        assert info.degree == degree
        assert rel(host(out), ref) <= 1e-12
    finally:
        nd.nd_destroy(ctx)


def test_massive_dn_and_zero_source(nd, cfg1):
    import torch
    dims, U, eta, lm, lam_max, eps, degree = cfg1
    ref, _ = overlap.dn_apply(U, dims, M, S, eta, lam_max, eps, 0, 0, lm["u"], lm["nu"], m_q=0.07, degree=degree)
    ctx = _ctx(nd, dims, U)
    try:
        nd.nd_set_lowmodes(ctx, dev(lm["u"]), list(lm["nu"]), lm["lam_next"])
        p = nd.dn_params(0, eps, lam_max, 1e-10, 1, 0, 0.07, False, approx=CHEB, degree=degree)
        out = torch.empty_like(dev(eta))
        nd.nd_apply_DN(ctx, out, dev(eta), p)
        assert rel(host(out), ref) <= 1e-10
        zero = torch.zeros_like(dev(eta))
        nd.nd_apply_sign(ctx, out, zero, p)
        assert float(out.abs().max()) == 0.0
    finally:
        nd.nd_destroy(ctx)


def test_bad_parameters(nd, cfg1):
    import torch
    dims, U, eta, lm, lam_max, eps, _ = cfg1
    ctx = _ctx(nd, dims, U)
    try:
        out = torch.empty_like(dev(eta))
        for p in [nd.dn_params(0, eps, lam_max, 1e-10, 1, 0, approx=7),
                  nd.dn_params(0, eps, lam_max, 1e-10, 1, 0, approx=CHEB, degree=-3),
                  nd.dn_params(0, eps, lam_max, 1e-10, 1, 0, approx=CHEB, degree=4096)]:
            with pytest.raises(nd.NdError) as e:
                nd.nd_apply_sign(ctx, out, dev(eta), p)
            assert e.value.status == nd.ND_ERR_INVALID_ARG
    finally:
        nd.nd_destroy(ctx)
