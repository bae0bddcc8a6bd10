"""Pins of the oracle's multi-shift CG against dense linear solves (LAPACK) and the
collinear-residual property."""
import numpy as np
import pytest

import synth
from oracle import mscg, wilson


def _spd(n, seed, cond=1e3):
    r = synth.rng(seed)
    q, _ = np.linalg.qr(synth.complex_gaussian(r, (n, n)))
    ev = np.geomspace(1.0 / cond, 1.0, n)
    return (q * ev) @ q.conj().T


def test_single_shift_is_cg():
    A = _spd(60, 1)
    b = synth.complex_gaussian(synth.rng(2), 60)
    x, info = mscg.multishift_cg(lambda v: A @ v, b, [0.0], 1e-12)
    assert np.linalg.norm(A @ x[0] - b) <= 1e-12 * np.linalg.norm(b) * 1.0001
    assert np.allclose(x[0], np.linalg.solve(A, b), rtol=0, atol=1e-8)


def test_many_shifts_dense():
    A = _spd(80, 3, cond=1e4)
    b = synth.complex_gaussian(synth.rng(4), 80)
    sig = [1e-5, 1e-3, 0.1, 2.0, 50.0]
    x, info = mscg.multishift_cg(lambda v: A @ v, b, sig, 1e-12)
    for l, s in enumerate(sig):
        res = np.linalg.norm(b - (A + s * np.eye(80)) @ x[l]) / np.linalg.norm(b)
        assert res <= 1.5e-12
        ex = np.linalg.solve(A + s * np.eye(80), b)
        assert np.linalg.norm(x[l] - ex) <= 1e-12 * np.linalg.norm(b) / (1e-4 + s) * 2


def test_unsorted_shifts_and_reported_residuals():
    A = _spd(50, 5)
    b = synth.complex_gaussian(synth.rng(6), 50)
    sig = [3.0, 0.01, 0.5]
    x, info = mscg.multishift_cg(lambda v: A @ v, b, sig, 1e-10)
    for l, s in enumerate(sig):
        true = np.linalg.norm(b - (A + s * np.eye(50)) @ x[l]) / np.linalg.norm(b)
        assert true <= 1e-10 * 1.01
        # the recurrence residual zeta_l r is the true residual up to rounding
        assert abs(true - info["res"][l]) <= 1e-13


def test_on_Q2_2x4():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=0)
    Qm = wilson.dense_Q(U, dims, -1.4)
    b = synth.spinor(dims, seed=1)
    sig = [0.0, 0.3]
    x, _ = mscg.multishift_cg(lambda v: wilson.apply_Q2(U, v, dims, -1.4), b, sig, 1e-12)
    for l, s in enumerate(sig):
        ex = np.linalg.solve(Qm @ Qm + s * np.eye(len(Qm)), b.reshape(-1))
        assert np.linalg.norm(x[l].reshape(-1) - ex) <= 1e-9 * np.linalg.norm(ex)


def test_not_converged_raises():
    A = _spd(40, 7, cond=1e6)
    b = synth.complex_gaussian(synth.rng(8), 40)
    with pytest.raises(mscg.NotConverged):
        mscg.multishift_cg(lambda v: A @ v, b, [0.0], 1e-14, maxit=3)


def test_rational_tolerance_bounds_sum():
    A = _spd(70, 9, cond=1e3)
    b = synth.complex_gaussian(synth.rng(10), 70)
    lam_min = float(np.linalg.eigvalsh(A).min())
    sig, wts = [1e-4, 1e-2, 1.0], [0.01, 0.5, 2.0]
    tol = 1e-8
    x, _ = mscg.multishift_cg(lambda v: A @ v, b, sig, mscg.rational_tolerances(wts, sig, lam_min, tol))
    y = sum(w * xx for w, xx in zip(wts, x))
    ex = sum(w * np.linalg.solve(A + s * np.eye(70), b) for w, s in zip(wts, sig))
    assert np.linalg.norm(y - ex) <= tol * np.linalg.norm(b)
