"""Pins of the oracle's ARPACK low-mode path against dense LAPACK diagonalisation."""
import numpy as np
import pytest

import synth
from oracle import lowmodes

M = -1.4


def test_arpack_matches_dense():
    dims = (4, 4, 2, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    l = 6
    de = lowmodes.lowmodes_dense(U, dims, M, l)
    ar = lowmodes.lowmodes_arpack(U, dims, M, l)
    assert np.allclose(ar["eval_Q2"], de["eval_Q2"], rtol=1e-10, atol=0)
    assert abs(ar["lam_max"] - de["lam_max"]) <= 1e-6 * de["lam_max"]
    assert np.allclose(np.sort(ar["nu"]), np.sort(de["nu"]), rtol=1e-9)
    Pa = np.einsum("kx,ky->xy", ar["u"].reshape(l, -1), ar["u"].reshape(l, -1).conj())
    Pd = np.einsum("kx,ky->xy", de["u"].reshape(l, -1), de["u"].reshape(l, -1).conj())
    assert np.linalg.norm(Pa - Pd, 2) < 1e-8
    assert np.max(ar["rho"]) < 1e-8


def test_lambda_max_arpack_matches_dense():
    dims = (4, 4, 2, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    de = lowmodes.lowmodes_dense(U, dims, M, 1)
    lm = lowmodes.lambda_max_arpack(U, dims, M, tol=1e-10)
    assert abs(lm - de["lam_max"]) <= 1e-8 * de["lam_max"]
    # free field: the largest Q^2 eigenvalue is the closed form max_p (m + sum(1 - cos p))^2 + sum sin^2 p,
    # reached at p = (pi, pi, pi, pi): (m + 8)^2
    Uf = synth.gauge_field(dims, "unit")
    assert abs(lowmodes.lambda_max_arpack(Uf, dims, M, tol=1e-10) - (M + 8.0) ** 2) <= 1e-8 * (M + 8.0) ** 2


def test_choose_l_rule():
    # eigenvalues of Q^2 with one clear relative gap after the 5th mode
    ev = np.array([0.01, 0.011, 0.0112, 0.0113, 0.0115, 0.05, 0.051, 0.052, 0.06, 0.061])
    assert lowmodes.choose_l(ev, 2, 8) == 5
    assert lowmodes.choose_l(ev * 37.0, 2, 8) == 5  # scale invariant
    assert lowmodes.choose_l(ev, 6, 8) == 8  # 0.052 -> 0.06 is the largest gap in that window
    assert lowmodes.choose_l(ev, 3, 3) == 3
    # ties go to the smaller l
    assert lowmodes.choose_l(np.array([1.0, 4.0, 16.0, 64.0]), 1, 3) == 1
    with pytest.raises(ValueError):
        lowmodes.choose_l(ev, 0, 3)
    with pytest.raises(ValueError):
        lowmodes.choose_l(ev, 2, 10)
