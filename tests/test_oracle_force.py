"""Pins of the oracle's force of S = phi^dagger (Q^2)^{-1} phi by central finite differences
along random su(3) directions, and of its S against a dense solve."""
import numpy as np
import pytest

import synth
from oracle import force, wilson

M = -1.4


@pytest.mark.parametrize("kind,dims", [("haar", (2, 2, 2, 4)), ("near_identity", (4, 2, 2, 2))])
def test_force_finite_differences(kind, dims):
    U = synth.gauge_field(dims, kind, seed=0, eps=0.3)
    phi = synth.spinor(dims, seed=1)
    F = force.force(U, dims, M, phi, tol=1e-14)
    h = 1e-5
    for seed in range(3):
        om = synth.su3_directions(dims, seed=3 + seed)
        sp = force.action(force.rotate_links(U, om, h), dims, M, phi, tol=1e-14)
        sm = force.action(force.rotate_links(U, om, -h), dims, M, phi, tol=1e-14)
        fd = (sp - sm) / (2 * h)
        an = float(np.sum(om * F))
        assert abs(fd - an) <= 1e-7 * abs(an) + 1e-9


def test_action_vs_dense():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=5)
    phi = synth.spinor(dims, seed=6)
    Qm = wilson.dense_Q(U, dims, M)
    ex = np.vdot(phi.reshape(-1), np.linalg.solve(Qm @ Qm, phi.reshape(-1))).real
    assert abs(force.action(U, dims, M, phi, tol=1e-14) - ex) <= 1e-11 * abs(ex)


def test_exp_is_su3():
    om = synth.rng(1).normal(size=(10, 8))
    E = force.exp_i_omega_T(om)
    assert np.allclose(np.einsum("nij,nkj->nik", E, E.conj()), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(E), 1.0, atol=1e-13)
