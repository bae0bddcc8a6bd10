"""GPU parity of the multi-shift solver, the low modes, sign(Q), D_N and the force against
the oracle (dense LAPACK at 4^4, the oracle's CG / multi-shift CG elsewhere), through the
C-ABI, plus the host-visible failure paths (iteration limit, NaN source, bad arguments)."""
import numpy as np
import pytest

import synth
from oracle import force as oforce
from oracle import lowmodes, overlap, wilson
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
    """4^4 Haar lattice (seed 0), source seed 1, dense spectrum of Q, 8 exact low modes."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    eta = synth.spinor(dims, seed=1)
    lm = lowmodes.lowmodes_dense(U, dims, M, 8)
    return dims, U, eta, lm


def _ctx(nd, dims, U, recon=(18, 12, 12), antiperiodic=False):
    ctx = nd.nd_create(dims, antiperiodic_t=antiperiodic, m=M, s=S)
    nd.nd_set_links(ctx, dev(U), recon)
    return ctx


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_solve_vs_dense(nd, cfg1, inner):
    import torch
    dims, U, eta, lm = cfg1
    w = lm["spectrum"]
    vecs = lm["eigvecs"]
    shifts = [0.02, 0.3, 2.5, 0.0]
    tol = 1e-11
    ctx = _ctx(nd, dims, U)
    try:
        xs = [torch.empty_like(dev(eta)) for _ in shifts]
        info = nd.nd_solve(ctx, xs, dev(eta), shifts, tol, 20000, inner)
        torch.cuda.synchronize()
        assert info.max_resid <= tol
        b = eta.reshape(-1)
        for x, s in zip(xs, shifts):
            ex = vecs @ ((vecs.conj().T @ b) / (w ** 2 + s))
            bound = tol * np.linalg.norm(b) / (np.min(w ** 2) + s)
            assert np.linalg.norm(host(x).reshape(-1) - ex) <= 1.5 * bound
    finally:
        nd.nd_destroy(ctx)


def test_solve_failure_paths(nd, cfg1):
    import torch
    dims, U, eta, lm = cfg1
    ctx = _ctx(nd, dims, U)
    try:
        x = [torch.empty_like(dev(eta))]
        with pytest.raises(nd.NdError) as e:
            nd.nd_solve(ctx, x, dev(eta), [0.0], 1e-12, 3, 0)
        assert e.value.status == nd.ND_ERR_NOT_CONVERGED
        with pytest.raises(nd.NdError) as e:
            nd.nd_solve(ctx, x, dev(eta), [-1.0], 1e-12, 100, 0)
        assert e.value.status == nd.ND_ERR_INVALID_ARG
        bad = eta.copy()
        bad[3, 1, 2] = np.nan
        with pytest.raises(nd.NdError) as e:
            nd.nd_solve(ctx, x, dev(bad), [0.0], 1e-12, 100, 0)
        assert e.value.status == nd.ND_ERR_NAN
        # the context stays usable after host-visible failures
        info = nd.nd_solve(ctx, x, dev(eta), [0.5], 1e-10, 5000, 0)
        assert info.max_resid <= 1e-10
    finally:
        nd.nd_destroy(ctx)


def test_lowmodes_vs_dense(nd, cfg1):
    dims, U, eta, lm = cfg1
    l = 8
    ctx = _ctx(nd, dims, U)
    try:
        nu, rho, ev, info = nd.nd_lowmodes(ctx, l, 1e-12, 20000)
        assert np.allclose(np.sort(ev), np.sort(lm["eval_Q2"]), rtol=1e-9, atol=0)
        assert np.allclose(np.sort(nu), np.sort(lm["nu"]), rtol=1e-9, atol=1e-12)
        # a Ritz value from below; sign(Q) pads it by 1 %
        assert lm["lam_max"] * (1 - 2e-3) <= info.lambda_max <= lm["lam_max"] * (1 + 1e-12)
        assert max(rho) < 1e-9 and info.kappa_plus < 1e-6 and info.kappa_minus < 1e-6
        import torch
        ev_dev = torch.empty((l,) + eta.shape, dtype=torch.complex128, device="cuda")
        nu2 = nd.nd_get_lowmodes(ctx, ev_dev, l)
        u = host(ev_dev).reshape(l, -1)
        assert np.allclose(u.conj() @ u.T, np.eye(l), atol=1e-12)
        ue = lm["u"].reshape(l, -1)
        for seed in range(3):
            v = synth.spinor(dims, seed=40 + seed).reshape(-1)
            pv = u.T @ (u.conj() @ v)
            pe = ue.T @ (ue.conj() @ v)
            assert np.linalg.norm(pv - pe) <= 1e-9 * np.linalg.norm(v)
        assert nu2 == nu
    finally:
        nd.nd_destroy(ctx)


def _oracle_params(lm):
    lam_max = 1.01 * lm["lam_max"]
    eps = 0.99 * lm["lam_next"] / lam_max
    return lam_max, eps


@pytest.mark.parametrize("inner", [0, 1, 2])
@pytest.mark.parametrize("left_only", [False, True])
def test_sign_and_dn_vs_oracle(nd, cfg1, inner, left_only):
    """Configuration of the plain method: 4^4 Haar, 16 poles, tol 1e-12, 8 deflated modes (the
    oracle's, injected), lambda_max / eps passed explicitly to both sides."""
    import torch
    dims, U, eta, lm = cfg1
    lam_max, eps = _oracle_params(lm)
    tol = 1e-12
    ref_sign, _ = overlap.sign_apply(U, dims, M, eta, lam_max, eps, 16, tol, lm["u"], lm["nu"], two_sided=not left_only)
    ref_dn, _ = overlap.dn_apply(U, dims, M, S, eta, lam_max, eps, 16, tol, lm["u"], lm["nu"], two_sided=not left_only)
    ctx = _ctx(nd, dims, U)
    try:
        nd.nd_set_lowmodes(ctx, dev(lm["u"]), list(lm["nu"]), lm["lam_next"])
        p = nd.dn_params(16, eps, lam_max, tol, 20000, inner, 0.0, left_only)
        out = torch.empty_like(dev(eta))
        info = nd.nd_apply_sign(ctx, out, dev(eta), p)
        assert rel(host(out), ref_sign) <= 1e-10
        info = nd.nd_apply_DN(ctx, out, dev(eta), p)
        assert rel(host(out), ref_dn) <= 1e-10
        assert info.n_low == 8
    finally:
        nd.nd_destroy(ctx)


def test_dn_own_lowmodes_vs_exact(nd, cfg1):
    """GPU low modes + GPU D_N against the exact D_N from the dense eigendecomposition: the
    difference stays within the error bound of Sec. 2.3 plus the rational part's delta."""
    import torch
    dims, U, eta, lm = cfg1
    w, v = lm["spectrum"], lm["eigvecs"]
    S_ex = (v * np.sign(w)) @ v.conj().T
    b = eta.reshape(-1)
    g5 = np.tile(np.repeat([1, 1, -1, -1], 3), len(b) // 12)
    exact = (1 + S) * (b + g5 * (S_ex @ b))
    ctx = _ctx(nd, dims, U)
    try:
        nu, rho, ev, li = nd.nd_lowmodes(ctx, 8, 1e-12, 20000)
        p = nd.dn_params(16, 0.0, 0.0, 1e-12, 20000, 1, 0.0, False)
        out = torch.empty_like(dev(eta))
        info = nd.nd_apply_DN(ctx, out, dev(eta), p)
        err = np.linalg.norm(host(out).reshape(-1) - exact) / np.linalg.norm(b)
        bound = 2 * (1 + S) * (li.kappa_plus + li.kappa_minus) + (1 + S) * (info.delta + 5e-12)
        assert err <= bound
        assert err <= 1e-10
    finally:
        nd.nd_destroy(ctx)


def test_dn_no_deflation_needs_eps(nd, cfg1):
    import torch
    dims, U, eta, lm = cfg1
    ctx = _ctx(nd, dims, U)
    try:
        p = nd.dn_params(16, 0.0, 0.0, 1e-12, 20000, 0, 0.0, False)
        with pytest.raises(nd.NdError) as e:
            nd.nd_apply_DN(ctx, torch.empty_like(dev(eta)), dev(eta), p)
        assert e.value.status == nd.ND_ERR_INVALID_ARG
    finally:
        nd.nd_destroy(ctx)


def test_massive_dn_vs_oracle(nd, cfg1):
    import torch
    dims, U, eta, lm = cfg1
    lam_max, eps = _oracle_params(lm)
    ref, _ = overlap.dn_apply(U, dims, M, S, eta, lam_max, eps, 20, 1e-12, lm["u"], lm["nu"], m_q=0.07)
    ctx = _ctx(nd, dims, U)
    try:
        nd.nd_set_lowmodes(ctx, dev(lm["u"]), list(lm["nu"]), lm["lam_next"])
        out = torch.empty_like(dev(eta))
        nd.nd_apply_DN(ctx, out, dev(eta), nd.dn_params(20, eps, lam_max, 1e-12, 20000, 1, 0.07, False))
        assert rel(host(out), ref) <= 1e-10
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("inner", [0, 1])
def test_force_vs_oracle(nd, inner):
    import torch
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, "near_identity", seed=0, eps=0.3)
    phi = synth.spinor(dims, seed=1)
    ref = oforce.force(U, dims, M, phi, tol=1e-13)
    ctx = _ctx(nd, dims, U, antiperiodic=False)
    try:
        F = torch.empty((4, int(np.prod(dims)), 8), dtype=torch.float64, device="cuda")
        info = nd.nd_force(ctx, F, dev(phi), 1e-13, 20000, inner)
        assert info.max_resid <= 1e-13
        assert rel(host(F), ref) <= 1e-10
    finally:
        nd.nd_destroy(ctx)


def test_force_finite_differences_gpu(nd):
    """dS/dh along random su(3) directions, S = phi^dag (Q^2)^-1 phi evaluated by GPU solves."""
    import torch
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, "haar", seed=2)
    phi = synth.spinor(dims, seed=3)

    def action(Ul):
        ctx = _ctx(nd, dims, Ul)
        try:
            x = [torch.empty_like(dev(phi))]
            nd.nd_solve(ctx, x, dev(phi), [0.0], 1e-14, 20000, 0)
            return float(np.vdot(phi, host(x[0])).real)
        finally:
            nd.nd_destroy(ctx)

    ctx = _ctx(nd, dims, U)
    try:
        F = torch.empty((4, int(np.prod(dims)), 8), dtype=torch.float64, device="cuda")
        nd.nd_force(ctx, F, dev(phi), 1e-14, 20000, 0)
        F = host(F)
    finally:
        nd.nd_destroy(ctx)
    h = 1e-5
    for seed in range(2):
        om = synth.su3_directions(dims, seed=10 + seed)
        fd = (action(oforce.rotate_links(U, om, h)) - action(oforce.rotate_links(U, om, -h))) / (2 * h)
        an = float(np.sum(om * F))
        assert abs(fd - an) <= 1e-7 * abs(an)
