"""Pins of the oracle's Wilson-Dirac operator (Sec. 2.1) against facts other than itself:
the Clifford algebra, the free-field plane-wave closed form, gamma5-hermiticity, gauge
covariance and dense hermiticity."""
import itertools

import numpy as np
import pytest

import synth
from oracle import wilson

M = -1.4


def test_gamma_algebra():
    g = [wilson.gamma(mu) for mu in range(4)]
    g5 = wilson.gamma(4)
    eye = np.eye(4)
    for mu, nu in itertools.product(range(4), repeat=2):
        anti = g[mu] @ g[nu] + g[nu] @ g[mu]
        assert np.allclose(anti, 2 * eye * (mu == nu), atol=1e-15)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        assert np.allclose(g5 @ g[mu] + g[mu] @ g5, 0)
    assert np.allclose(g[0] @ g[1] @ g[2] @ g[3], g5)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def _plane_wave(dims, p, chi):
    V = int(np.prod(dims))
    x = np.array(list(itertools.product(*[range(n) for n in dims])))
    phase = np.exp(1j * (x @ np.asarray(p)))
    return np.ascontiguousarray(phase[:, None, None] * chi[None, :, :]), phase


@pytest.mark.parametrize("antiperiodic", [False, True])
def test_free_field_plane_waves(antiperiodic):
    """U = 1: D_W e^{ipx} chi = [m + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu] e^{ipx} chi,
    derived from the definition of D_W; p_mu = 2 pi n_mu / L_mu (time: (2n+1) pi / T if antiperiodic)."""
    dims = (4, 6, 2, 4)
    U = synth.gauge_field(dims, "unit")
    g = [wilson.gamma(mu) for mu in range(4)]
    g5 = wilson.gamma(4)
    r = synth.rng(7)
    for trial in range(6):
        n = [int(r.integers(0, d)) for d in dims]
        p = [2 * np.pi * n[mu] / dims[mu] for mu in range(4)]
        if antiperiodic:
            p[0] = (2 * n[0] + 1) * np.pi / dims[0]
        chi = synth.complex_gaussian(r, (4, 3))
        psi, phase = _plane_wave(dims, p, chi)
        D = (M + sum(1 - np.cos(pm) for pm in p)) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[:, None, None] * (g5 @ D @ chi)[None]
        got = wilson.apply_Q(U, psi, dims, M, antiperiodic)
        assert np.max(np.abs(got - expect)) < 1e-13


def test_free_field_Q2_spectrum():
    """Free-field Q^2 eigenvalues: (m + sum(1 - cos p))^2 + sum sin^2 p, each 12-fold."""
    dims = (4, 4, 2, 4)
    U = synth.gauge_field(dims, "unit")
    Qm = wilson.dense_Q(U, dims, M)
    ev = np.sort(np.linalg.eigvalsh(Qm @ Qm))
    ex = []
    for n in itertools.product(*[range(d) for d in dims]):
        p = [2 * np.pi * n[mu] / dims[mu] for mu in range(4)]
        val = (M + sum(1 - np.cos(q) for q in p)) ** 2 + sum(np.sin(q) ** 2 for q in p)
        ex += [val] * 12
    assert np.allclose(ev, np.sort(ex), atol=1e-12)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8)])
def test_gamma5_hermiticity(dims):
    U = synth.gauge_field(dims, "haar", seed=0)
    a = synth.spinor(dims, seed=1)
    b = synth.spinor(dims, seed=2)
    lhs = np.vdot(a, wilson.apply_Q(U, b, dims, M))
    rhs = np.vdot(wilson.apply_Q(U, a, dims, M), b)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # D_W itself is gamma5-hermitian: gamma5 D_W gamma5 = D_W^dagger, but not hermitian
    dw_ab = np.vdot(a, wilson.apply_DW(U, b, dims, M))
    dw_ba = np.vdot(wilson.apply_DW(U, a, dims, M), b)
    assert abs(dw_ab - dw_ba) > 1e-3 * abs(dw_ab)


@pytest.mark.parametrize("antiperiodic", [False, True])
def test_gauge_covariance(antiperiodic):
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger, psi -> g psi  =>  Q' (g psi) = g (Q psi)."""
    dims = (4, 4, 2, 6)
    V = int(np.prod(dims))
    U = synth.gauge_field(dims, "haar", seed=3)
    psi = synth.spinor(dims, seed=4)
    g = synth.gauge_transform(dims, seed=5)
    x = np.array(list(itertools.product(*[range(n) for n in dims])))
    Ug = np.empty_like(U)
    for mu in range(4):
        y = x.copy()
        y[:, mu] = (y[:, mu] + 1) % dims[mu]
        fw = y[:, 3] + dims[3] * (y[:, 2] + dims[2] * (y[:, 1] + dims[1] * y[:, 0]))
        Ug[mu] = np.einsum("sij,sjk,slk->sil", g, U[mu], g[fw].conj())
    gpsi = np.ascontiguousarray(np.einsum("sij,saj->sai", g, psi))
    lhs = wilson.apply_Q(Ug, gpsi, dims, M, antiperiodic)
    rhs = np.einsum("sij,saj->sai", g, wilson.apply_Q(U, psi, dims, M, antiperiodic))
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_dense_hermitian_2x4():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=0)
    Qm = wilson.dense_Q(U, dims, M)
    assert np.max(np.abs(Qm - Qm.conj().T)) < 1e-14


def test_antiperiodic_differs_only_at_boundary():
    """Antiperiodic time flips the sign of exactly the hops across t = T-1 -> 0."""
    dims = (4, 2, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=1)
    psi = np.zeros((16 * 2, 4, 3), dtype=np.complex128)
    psi[5, 0, 0] = 1.0  # x0 = 0 site: its t-1 neighbour crosses the boundary
    psi = np.ascontiguousarray(psi)
    a = wilson.apply_Q(U, psi, dims, M, False)
    b = wilson.apply_Q(U, psi, dims, M, True)
    diff_sites = np.nonzero(np.abs(a - b).reshape(len(psi), -1).max(axis=1) > 0)[0]
    # only the site at x0 = T-1 (same spatial position) receives a boundary-crossing hop
    assert list(diff_sites) == [5 + 8 * 3]
