"""Pins of the oracle's ARPACK low-mode path against dense LAPACK diagonalisation."""
import numpy as np

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
