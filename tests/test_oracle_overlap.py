"""Pins of the oracle's deflated sign(Q) and D_N against dense diagonalisation (LAPACK eigh
of the assembled Q) and the identities the paper relies on (Sec. 2.2, 2.3): the uniform
error bound delta, sign(Q)^2 = 1, the Ginsparg-Wilson relation, the projector-deviation
bound and the D_N error bound."""
import numpy as np
import pytest

import synth
from oracle import lowmodes, overlap, wilson

M, S = -1.4, 0.4
TOL = 1e-12


def _setup(dims, l, seed=0):
    U = synth.gauge_field(dims, "haar", seed=seed)
    lm = lowmodes.lowmodes_dense(U, dims, M, l)
    w, v = lm["spectrum"], lm["eigvecs"]
    S_ex = (v * np.sign(w)) @ v.conj().T
    lam_max = 1.01 * lm["lam_max"]
    eps = 0.99 * lm["lam_next"] / lam_max
    return U, lm, S_ex, lam_max, eps


@pytest.fixture(scope="module")
def lat2():
    return ((2, 2, 2, 2),) + _setup((2, 2, 2, 2), 8)


@pytest.fixture(scope="module")
def lat4():
    return ((4, 4, 4, 4),) + _setup((4, 4, 4, 4), 8)


@pytest.mark.parametrize("which", ["lat2", "lat4"])
@pytest.mark.parametrize("npoles", [8, 16])
def test_sign_vs_exact(which, npoles, request):
    dims, U, lm, S_ex, lam_max, eps = request.getfixturevalue(which)
    eta = synth.spinor(dims, seed=1)
    sg, info = overlap.sign_apply(U, dims, M, eta, lam_max, eps, npoles, TOL, lm["u"], lm["nu"])
    err = np.linalg.norm(sg.reshape(-1) - S_ex @ eta.reshape(-1)) / np.linalg.norm(eta)
    assert err <= info["delta"] + 20 * TOL


def test_sign_undeflated_2x4(lat2):
    dims, U, lm, S_ex, lam_max, _ = lat2
    eps = 0.99 * float(np.min(lm["spectrum"] ** 2)) / lam_max
    eta = synth.spinor(dims, seed=2)
    sg, info = overlap.sign_apply(U, dims, M, eta, lam_max, eps, 20, TOL)
    err = np.linalg.norm(sg.reshape(-1) - S_ex @ eta.reshape(-1)) / np.linalg.norm(eta)
    assert err <= info["delta"] + 1e-9


def test_sign_squared_and_gw(lat4):
    dims, U, lm, _, lam_max, eps = lat4
    eta = synth.spinor(dims, seed=3)
    args = (U, dims, M, S)
    kw = dict(u=lm["u"], nu=lm["nu"])
    s1, info = overlap.sign_apply(U, dims, M, eta, lam_max, eps, 16, TOL, **kw)
    s2, _ = overlap.sign_apply(U, dims, M, s1, lam_max, eps, 16, TOL, **kw)
    bound = 3 * info["delta"] + 50 * TOL
    assert np.linalg.norm(s2 - eta) <= bound * np.linalg.norm(eta)
    # Ginsparg-Wilson: gamma5 D + D gamma5 = abar D gamma5 D
    abar = 1 / (1 + S)
    D = lambda v: overlap.dn_apply(*args, v, lam_max, eps, 16, TOL, **kw)[0]
    g5 = overlap.gamma5
    Deta = D(eta)
    lhs = g5(Deta) + D(g5(eta))
    rhs = abar * D(g5(Deta))
    assert np.linalg.norm(lhs - rhs) <= 10 * bound * np.linalg.norm(eta)


def test_two_sided_equals_left_only_for_exact_modes(lat2):
    dims, U, lm, _, lam_max, eps = lat2
    eta = synth.spinor(dims, seed=4)
    a, info = overlap.sign_apply(U, dims, M, eta, lam_max, eps, 16, TOL, lm["u"], lm["nu"], two_sided=True)
    b, _ = overlap.sign_apply(U, dims, M, eta, lam_max, eps, 16, TOL, lm["u"], lm["nu"], two_sided=False)
    assert np.linalg.norm(a - b) <= (2 * info["delta"] + 1e-9) * np.linalg.norm(eta)


def _perturbed_modes(dims, U, lm, l, noise, seed):
    """Rayleigh-Ritz on V = span(exact low modes + noise): approximate eigenvectors."""
    r = synth.rng(seed)
    basis = lm["u"] + noise * synth.complex_gaussian(r, lm["u"].shape)
    Q = lambda x: wilson.apply_Q(U, np.ascontiguousarray(x), dims, M)
    return lowmodes.rayleigh_ritz(Q, basis)


@pytest.mark.parametrize("noise", [3e-5, 1e-4])
def test_projector_bound(lat2, noise):
    """||P_+- - (P_+-)_exact|| <= kappa (1 + 2 kappa) / (1 - 2 kappa (1 + 2 kappa))  (Sec. 2.3)."""
    dims, U, lm, _, _, _ = lat2
    l = 8
    nu, u, rho = _perturbed_modes(dims, U, lm, l, noise, seed=11)
    d = lowmodes.spectral_distances(nu, lm["lam_next"])
    kp, km = lowmodes.kappas(nu, rho, d)
    uf = u.reshape(l, -1)
    ue = lm["u"].reshape(l, -1)
    for sgn, kap in ((1, kp), (-1, km)):
        P = sum(np.outer(uf[k], uf[k].conj()) for k in range(l) if np.sign(nu[k]) == sgn)
        Pe = sum(np.outer(ue[k], ue[k].conj()) for k in range(l) if np.sign(lm["nu"][k]) == sgn)
        dev = np.linalg.norm(P - Pe, 2)
        assert dev <= lowmodes.projector_bound(kap)
        assert 1e-3 * kap < dev and kap < 0.25  # the bound is tested where it is informative


def test_ritz_residual_identity(lat2):
    """For a Ritz pair of a Hermitian Q on V, (Q - nu) u is orthogonal to V, so
    rho^2 = ||Q u||^2 - nu^2; with exact eigenvectors rho vanishes."""
    dims, U, lm, _, _, _ = lat2
    nu, u, rho = _perturbed_modes(dims, U, lm, 8, 1e-3, seed=13)
    for k in range(8):
        qu = wilson.apply_Q(U, np.ascontiguousarray(u[k]), dims, M)
        assert abs(rho[k] ** 2 - (np.vdot(qu, qu).real - nu[k] ** 2)) <= 1e-10
        assert abs(np.vdot(u[k], u[k]) - 1) < 1e-13
    nu0, _, rho0 = _perturbed_modes(dims, U, lm, 8, 0.0, seed=13)
    assert np.max(rho0) < 1e-12 and np.allclose(np.sort(nu0), np.sort(lm["nu"]), atol=1e-12)


def test_spectral_distance_reading_matches_exact(lat2):
    """With exact modes the estimator equals the exact distance to the complementary spectrum."""
    dims, U, lm, _, _, _ = lat2
    nu = lm["nu"]
    d = lowmodes.spectral_distances(nu, lm["lam_next"])
    w = lm["spectrum"]
    for k, v in enumerate(nu):
        same_in_V = [x for x in nu if np.sign(x) == np.sign(v)]
        rest = [x for x in w if not (np.sign(x) == np.sign(v) and np.any(np.isclose(x, same_in_V, rtol=0, atol=1e-12)))]
        exact = min(abs(v - x) for x in rest)
        # the estimator uses |lambda_{l+1}|^(1/2) as the nearest same-sign magnitude outside V
        assert d[k] <= exact + 1e-12


@pytest.mark.parametrize("noise", [1e-4, 1e-3])
def test_dn_error_bound(lat2, noise):
    """||D~_N^m - D_N^m|| <= (2/a)(1 + s - a m_q/2)(kappa_+ + kappa_-)  (Sec. 2.3), for the
    paper's left-only form; the rational part's own error (delta, solver) is added."""
    dims, U, lm, S_ex, lam_max, eps = lat2
    l = 8
    nu, u, rho = _perturbed_modes(dims, U, lm, l, noise, seed=12)
    d = lowmodes.spectral_distances(nu, lm["lam_next"])
    kp, km = lowmodes.kappas(nu, rho, d)
    mq = 0.05
    abar = 1 / (1 + S)
    eps_p = 0.5 * eps
    bound = 2 * (1 + S - mq / 2) * (kp + km)
    n = 12 * int(np.prod(dims))
    D_exact = (1 - abar * mq / 2) * (np.eye(n) + np.kron(np.eye(n // 12), np.kron(np.diag([1, 1, -1, -1]), np.eye(3))) @ S_ex) / abar + mq * np.eye(n)
    worst = 0.0
    for seed in range(4):
        v = synth.spinor(dims, seed=20 + seed)
        got, info = overlap.dn_apply(U, dims, M, S, v, lam_max, eps_p, 20, TOL, u, nu, m_q=mq, two_sided=False)
        err = np.linalg.norm(got.reshape(-1) - D_exact @ v.reshape(-1)) / np.linalg.norm(v)
        worst = max(worst, err)
    extra = (1 + S) * (1 - abar * mq / 2) * (info["delta"] + 1e-9)
    assert worst <= bound + extra


@pytest.mark.parametrize("m_q", [0.2, 0.05])
def test_propagator_vs_dense(lat2, m_q):
    """(D_N^m)^{-1} b by the oracle's CG against LAPACK solve of the dense D_N^m built from the
    exact sign(Q); the difference is bounded by the approximation error of sign(Q) (delta), the
    CG tolerance and ||(D_N^m)^{-1}|| <= 1/m_q (the massive overlap spectrum lies on a circle
    shifted away from 0 by m_q)."""
    dims, U, lm, S_ex, lam_max, eps = lat2
    b = synth.spinor(dims, seed=9)
    x, info = overlap.propagator(U, dims, M, S, b, lam_max, eps, 16, 1e-13, lm["u"], lm["nu"], m_q=m_q, tol=1e-11)
    assert b.dtype == np.complex128
    n = b.size
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), n // 12)
    abar = 1.0 / (1.0 + S)
    D_ex = (1.0 - abar * m_q / 2.0) * (1.0 + S) * (np.eye(n) + g5[:, None] * S_ex) + m_q * np.eye(n)
    x_ex = np.linalg.solve(D_ex, b.reshape(-1))
    assert info["resid"] <= 2e-11
    # ||x - x_ex|| <= ||D_ex^{-1}|| (||b - D x|| + ||(D - D_ex) x||), ||D - D_ex|| <= (1 + s)(delta + CG error)
    delta = overlap.zolo(16, eps)["delta"]
    bound = (info["resid"] * np.linalg.norm(b) + (1 + S) * (delta + 1e-12) * np.linalg.norm(x)) / m_q
    assert np.linalg.norm(x.reshape(-1) - x_ex) <= bound


def test_massive_dn_spectrum_on_circle(lat2):
    """With sign(Q)^2 = 1, D_N = (1 + gamma5 sign Q)/abar has its spectrum on the circle |z - 1/abar| =
    1/abar, so D_N^m = (1 - abar m/2) D_N + m has it on |z - c| = r with r = (1 - abar m/2)/abar and
    c = r + m.  The oracle's D_N^m, assembled column by column on 2^4, must put every eigenvalue
    there to within the approximation's error."""
    dims, U, lm, S_ex, lam_max, eps = lat2
    m_q = 0.3
    n = int(np.prod(dims)) * 12
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        d, info = overlap.dn_apply(U, dims, M, S, e.reshape(-1, 4, 3), lam_max, eps, 16, 1e-13, lm["u"], lm["nu"],
                                   m_q=m_q)
        cols.append(d.reshape(-1))
    D = np.array(cols).T
    abar = 1.0 / (1.0 + S)
    r = (1.0 - abar * m_q / 2.0) / abar
    ev = np.linalg.eigvals(D)
    assert np.max(np.abs(np.abs(ev - (r + m_q)) - r)) <= 1e-9
    # the massless limit sits on the circle through 0, and the mass shifts its centre
    assert np.min(ev.real) >= m_q - 1e-9
