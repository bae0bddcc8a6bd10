"""Pins of the oracle's minmax polynomial sign approximation and its Clenshaw evaluation
(Sec. 2.2: sign(Q) ~ X P_n(X^2), delta = max |1 - sqrt(y) P(y)| on [eps, 1]).

Independent checks: the n = 0 closed form; a linear-programming solution of the discretised
minimax problem (a different algorithm from the Remez exchange); convexity of the error
functional (no perturbation improves on the Remez coefficients); the alternation property; the
Clenshaw recurrence against numpy's Chebyshev series on the eigenvalues of a dense Hermitian
matrix; and the uniform bound delta against the dense sign(Q) of small lattices."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy.optimize import linprog

import synth
from oracle import chebyshev, lowmodes, overlap

M = -1.4


@pytest.mark.parametrize("eps", [0.5, 0.1, 1e-2, 1e-4])
def test_degree_zero_closed_form(eps):
    # 1 - c sqrt(y) on [eps, 1] is levelled by c = 2 / (1 + sqrt(eps)), error (1 - sqrt(eps)) / (1 + sqrt(eps))
    r = chebyshev.minmax(0, eps)
    se = np.sqrt(eps)
    assert r["c"][0] == pytest.approx(2.0 / (1.0 + se), rel=1e-13)
    assert r["delta"] == pytest.approx((1.0 - se) / (1.0 + se), rel=1e-13)


def _lp_minimax(n, eps, npts=3000):
    """min t subject to |1 - sqrt(y_j) P(y_j)| <= t on a grid (HiGHS linear program)."""
    # grid dense in the Chebyshev angle, where the extrema of the error accumulate
    y = 0.5 * (1 + eps) - 0.5 * (1 - eps) * np.cos(np.linspace(0, np.pi, npts))
    A = np.sqrt(y)[:, None] * npcheb.chebvander(chebyshev.z_of(y, eps), n)
    ones = np.ones((npts, 1))
    # variables (c_0 .. c_n, t):  1 - A c <= t  and  A c - 1 <= t
    A_ub = np.vstack([np.hstack([-A, -ones]), np.hstack([A, -ones])])
    b_ub = np.concatenate([-np.ones(npts), np.ones(npts)])
    cost = np.zeros(n + 2)
    cost[-1] = 1.0
    res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * (n + 2), method="highs")
    assert res.status == 0
    return res.x[:-1], res.x[-1]


@pytest.mark.parametrize("n,eps", [(1, 0.1), (3, 0.05), (6, 1e-2), (10, 1e-2)])
def test_matches_linear_program(n, eps):
    r = chebyshev.minmax(n, eps)
    c_lp, t_lp = _lp_minimax(n, eps)
    # the grid is a subset of [eps, 1], so the LP optimum lies at or just below delta
    assert t_lp <= r["delta"] * (1 + 1e-9)
    assert t_lp == pytest.approx(r["delta"], rel=2e-5)
    assert np.max(np.abs(c_lp - r["c"])) <= 1e-3 * np.max(np.abs(r["c"]))


@pytest.mark.parametrize("n,eps", [(4, 0.1), (20, 1e-2), (60, 1e-3)])
def test_no_perturbation_improves(n, eps):
    # max_y |h(y; c)| is convex in c: a point no direction improves is the global minimum
    r = chebyshev.minmax(n, eps)
    y = 0.5 * (1 + eps) - 0.5 * (1 - eps) * np.cos(np.linspace(0, np.pi, 20001))
    f = lambda c: np.max(np.abs(chebyshev.h_eval(c, y, eps)))
    f0 = f(r["c"])
    assert f0 == pytest.approx(r["delta"], rel=1e-6)
    rng = np.random.default_rng(5)
    for step in (1e-3, 1e-5):
        for _ in range(40):
            d = rng.standard_normal(n + 1)
            d *= step * r["delta"] / np.linalg.norm(d)
            assert f(r["c"] + d) >= f0 * (1 - 1e-9)


@pytest.mark.parametrize("n,eps", [(8, 0.05), (40, 1e-2), (150, 2e-3)])
def test_alternation(n, eps):
    r = chebyshev.minmax(n, eps)
    h = chebyshev.h_eval(r["c"], r["ref"], eps)
    assert len(h) == n + 2
    assert np.all(np.sign(h[1:]) == -np.sign(h[:-1]))
    assert np.max(np.abs(h)) - np.min(np.abs(h)) <= max(1e-8 * r["delta"], 5e-14)
    y = np.linspace(eps, 1.0, 200001)
    assert np.max(np.abs(chebyshev.h_eval(r["c"], y, eps))) <= r["delta"] * (1 + 1e-7) + 5e-14
    # both ends of the interval are extrema
    assert r["ref"][0] == pytest.approx(eps, rel=1e-9)
    assert r["ref"][-1] == pytest.approx(1.0, rel=1e-12)


def test_delta_decreases_and_degree_for():
    eps = 1e-2
    d = [chebyshev.minmax(n, eps)["delta"] for n in range(0, 30)]
    assert all(b < a for a, b in zip(d, d[1:]))
    n = chebyshev.degree_for(eps, 1e-6)
    assert chebyshev.minmax(n, eps)["delta"] <= 1e-6 < chebyshev.minmax(n - 1, eps)["delta"]


def test_clenshaw_matches_series_on_eigenvalues():
    rng = np.random.default_rng(7)
    N = 60
    Z = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Qm, _ = np.linalg.qr(Z)
    lam = rng.uniform(-1, 1, N)
    A = (Qm * lam) @ Qm.conj().T
    c = rng.standard_normal(25)
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    got = chebyshev.clenshaw(lambda w: A @ w, c, v)
    ref = (Qm * npcheb.chebval(lam, c)) @ (Qm.conj().T @ v)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_poly_apply_maps_interval():
    # P(X^2) on eigenvalues y of X^2 equals the scalar series at z(y)
    rng = np.random.default_rng(8)
    eps = 0.02
    y = rng.uniform(eps, 1, 30)
    c = chebyshev.minmax(12, eps)["c"]
    v = rng.standard_normal(30)
    got = chebyshev.poly_apply(lambda w: y * w, c, eps, v)
    assert np.allclose(got, chebyshev.p_eval(c, y, eps) * v, rtol=1e-13, atol=1e-14)


@pytest.fixture(scope="module")
def lat2():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=0)
    lm = lowmodes.lowmodes_dense(U, dims, M, 8)
    w, v = lm["spectrum"], lm["eigvecs"]
    return dims, U, lm, (v * np.sign(w)) @ v.conj().T


def test_poly_sign_uniform_bound_undeflated(lat2):
    dims, U, lm, S_ex = lat2
    lam_max = 1.01 * lm["lam_max"]
    eps = 0.99 * float(np.min(lm["spectrum"] ** 2)) / lam_max
    eta = synth.spinor(dims, seed=2)
    for degree in (20, 60):
        sg, info = overlap.sign_apply_poly(U, dims, M, eta, lam_max, eps, degree)
        err = np.linalg.norm(sg.reshape(-1) - S_ex @ eta.reshape(-1)) / np.linalg.norm(eta)
        assert err <= info["delta"] + 1e-12


def test_poly_sign_deflated_and_dn(lat2):
    dims, U, lm, S_ex = lat2
    lam_max = 1.01 * lm["lam_max"]
    eps = 0.99 * lm["lam_next"] / lam_max
    eta = synth.spinor(dims, seed=3)
    sg, info = overlap.sign_apply_poly(U, dims, M, eta, lam_max, eps, 40, lm["u"], lm["nu"])
    err = np.linalg.norm(sg.reshape(-1) - S_ex @ eta.reshape(-1)) / np.linalg.norm(eta)
    assert err <= info["delta"] + 1e-12
    # the rational and the polynomial D_N agree to the sum of their uniform errors
    dz, iz = overlap.dn_apply(U, dims, M, 0.4, eta, lam_max, eps, 16, 1e-12, lm["u"], lm["nu"])
    dp, ip = overlap.dn_apply(U, dims, M, 0.4, eta, lam_max, eps, 16, 1e-12, lm["u"], lm["nu"], degree=40)
    assert np.linalg.norm(dz - dp) <= 1.4 * (iz["delta"] + ip["delta"] + 1e-10) * np.linalg.norm(eta)


def test_rounding_level_delta_is_flagged():
    # at this degree the minmax error (~1e-16) is below what FP64 resolves: flagged, bounded
    r = chebyshev.minmax(256, 5.34e-3)
    assert r["resolved"] is False
    assert r["delta"] <= 1e-13
    assert chebyshev.minmax(40, 1e-2)["resolved"] is True
