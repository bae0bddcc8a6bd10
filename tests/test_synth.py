"""The seeded input generators shared by the oracle and the GPU tests: Haar and near-identity SU(3)
links (unitarity, determinant one, Haar moments), complex-Gaussian spinors, point sources, and the
reproducibility of every draw from its seed."""
import numpy as np
import pytest

import synth


def _su3_checks(U):
    eye = np.eye(3)
    dev_unit = np.max(np.abs(np.einsum("...ji,...jk->...ik", U.conj(), U) - eye))
    dev_det = np.max(np.abs(np.linalg.det(U) - 1.0))
    return dev_unit, dev_det


def test_haar_unitary_det_one_and_moments():
    U = synth.haar_su3(40000, seed=3)
    du, dd = _su3_checks(U)
    assert du < 1e-14 and dd < 1e-13
    tr = np.trace(U, axis1=-2, axis2=-1)
    # Haar measure on SU(3): E tr U = 0, E |tr U|^2 = 1, E |tr U|^4 = 2 (so the sample mean of |tr U|^2
    # has standard deviation 1/sqrt(n))
    n = len(tr)
    assert abs(tr.mean()) < 5 / np.sqrt(n)
    assert abs(np.mean(np.abs(tr) ** 2) - 1.0) < 5 / np.sqrt(n)
    assert abs(np.mean(np.abs(tr) ** 4) - 2.0) < 0.15


def test_near_identity_links():
    eps = 0.3
    U = synth.near_identity_su3(20000, eps, seed=4)
    du, dd = _su3_checks(U)
    assert du < 1e-14 and dd < 1e-13
    # U = exp(i eps H), H = sum_a h_a lambda_a / 2 with h_a ~ N(0, 1): Re tr U = 3 - eps^2 tr(H^2)/2 + ...,
    # E tr(H^2) = sum_a E h_a^2 tr(lambda_a^2) / 4 = 8 * 2 / 4 = 4
    re_tr = np.trace(U, axis1=-2, axis2=-1).real
    assert abs(np.mean(3.0 - re_tr) - eps ** 2 * 4 / 2) < 0.02
    assert np.max(np.abs(U - np.eye(3))) < 3.0


@pytest.mark.parametrize("kind", ["haar", "near_identity"])
def test_gauge_field_layout_and_seed(kind):
    dims = (4, 2, 2, 4)
    V = int(np.prod(dims))
    a = synth.gauge_field(dims, kind, seed=5)
    b = synth.gauge_field(dims, kind, seed=5)
    c = synth.gauge_field(dims, kind, seed=6)
    assert a.shape == (4, V, 3, 3) and a.dtype == np.complex128
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    du, dd = _su3_checks(a.reshape(-1, 3, 3))
    assert du < 1e-14 and dd < 1e-13


def test_spinor_distribution_and_point_source():
    dims = (8, 8, 8, 8)
    psi = synth.spinor(dims, seed=1)
    assert psi.shape == (int(np.prod(dims)), 4, 3) and psi.dtype == np.complex128
    assert np.array_equal(psi, synth.spinor(dims, seed=1))
    # re, im ~ N(0, 1/2): E |psi|^2 = 1 per component
    assert abs(np.mean(np.abs(psi) ** 2) - 1.0) < 0.02
    assert abs(np.mean(psi.real)) < 0.01 and abs(np.mean(psi.imag)) < 0.01
    p = synth.point_source(dims, 2, 1, site=17)
    assert np.count_nonzero(p) == 1 and p[17, 2, 1] == 1.0
