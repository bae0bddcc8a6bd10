"""Pins of the oracle's even-odd Schur-complement operator (oracle/schur.py): hermiticity of
Qhat, the block-LDU determinant identity det D_W = (4 + m)^{12 V/2} det Dhat, the support of
the hopping blocks, and dense LAPACK solves of D_W and Q^2 against the Schur-complement route."""
import numpy as np
import pytest

import synth
from oracle import schur, wilson

M = -1.4


def _g5(v):
    out = v.copy()
    out[..., 2:, :] *= -1.0
    return out


def _g5rows(V):
    """gamma5 acting on the rows of a dense (12 V x 12 V) matrix: D_W = gamma5 Q."""
    return np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)[:, None]


@pytest.mark.parametrize("kind", ["haar", "near_identity"])
def test_hermitian_and_blocks(kind):
    dims = (4, 4, 2, 4)
    U = synth.gauge_field(dims, kind, seed=0, eps=0.3) if kind == "near_identity" else synth.gauge_field(dims, kind, seed=0)
    even = schur.parity_mask(dims)
    a = even * synth.spinor(dims, seed=1)
    b = even * synth.spinor(dims, seed=2)
    qa = schur.qhat_apply(U, dims, M, a)
    qb = schur.qhat_apply(U, dims, M, b)
    assert abs(np.vdot(a, qb) - np.vdot(qa, b)) <= 1e-13 * np.linalg.norm(a) * np.linalg.norm(qb)
    assert np.all((1 - even) * qa == 0)
    D_eo, D_oe, _, odd = schur.blocks(U, dims, M)
    assert np.all(even * D_oe(a) == 0) and np.linalg.norm(D_oe(a)) > 0
    c = odd * synth.spinor(dims, seed=3)
    assert np.all(odd * D_eo(c) == 0)


def test_determinant_identity():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=4)
    V = 16
    DW = _g5rows(V) * wilson.dense_Q(U, dims, M)
    even = schur.parity_mask(dims).reshape(V)
    cols = []
    for s in np.flatnonzero(even):
        for k in range(12):
            e = np.zeros((V, 4, 3), dtype=np.complex128)
            e[s, k // 3, k % 3] = 1.0
            cols.append(_g5(schur.qhat_apply(U, dims, M, e)).reshape(-1))  # Dhat = gamma5 Qhat
    idx = np.concatenate([np.arange(12) + 12 * s for s in np.flatnonzero(even)])
    Dhat = np.array(cols).T[idx]
    s1, ld1 = np.linalg.slogdet(DW)
    s2, ld2 = np.linalg.slogdet(Dhat)
    assert ld1 == pytest.approx(12 * (V // 2) * np.log(abs(4 + M)) + ld2, rel=1e-12, abs=1e-9)
    assert s1 == pytest.approx(s2 * np.sign(4 + M) ** (12 * V // 2), abs=1e-9)


def test_solves_match_dense():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    Q = wilson.dense_Q(U, dims, M)
    b = synth.spinor(dims, seed=5)
    DW = _g5rows(256) * Q
    x, _ = schur.dw_solve(U, dims, M, b, tol=1e-13)
    ex = np.linalg.solve(DW, b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - ex) <= 1e-10 * np.linalg.norm(ex)
    y, _ = schur.q2_solve(U, dims, M, b, tol=1e-13)
    ey = np.linalg.solve(Q @ Q, b.reshape(-1))
    assert np.linalg.norm(y.reshape(-1) - ey) <= 1e-9 * np.linalg.norm(ey)
