"""Properties of sign(Q), D_N and the propagator at the size the bench measures (16^3 x 32 Haar
links, 20 deflated low modes, 20 poles, rational part to 1e-10), where the oracle cannot follow
in seconds: hermiticity of the two-sided approximation of sign(Q) and the gamma5-hermiticity of D_N
(exact for the construction, so only the solver tolerance enters), agreement of the FP64 and
mixed-precision paths, and the residual the propagator reports against one recomputed here."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
DIMS = (32, 16, 16, 16)
M, S = -1.4, 0.4


@pytest.fixture(scope="module")
def setup():
    import torch

    import paper_1010_5636_gb300 as nd
    nd.lib()
    U = synth.gauge_field(DIMS, "haar", seed=0)
    ctx = nd.nd_create(DIMS, m=M, s=S)
    nd.nd_set_links(ctx, dev(U), (18, 12, 12))
    nd.nd_lowmodes(ctx, 20, 1e-6, 2000000)
    yield nd, ctx, torch
    nd.nd_destroy(ctx)


def _vdot(a, b):
    return complex(np.vdot(host(a).reshape(-1), host(b).reshape(-1)))


@pytest.mark.parametrize("inner", [0, 1])
def test_sign_hermitian_and_dn_gamma5_hermitian(setup, inner):
    nd, ctx, torch = setup
    a = dev(synth.spinor(DIMS, seed=21))
    b = dev(synth.spinor(DIMS, seed=22))
    p = nd.dn_params(20, 0.0, 0.0, 1e-10, 200000, inner)
    sa, sb = torch.empty_like(a), torch.empty_like(b)
    nd.nd_apply_sign(ctx, sa, a, p)
    nd.nd_apply_sign(ctx, sb, b, p)
    na, nb = float(torch.linalg.vector_norm(a)), float(torch.linalg.vector_norm(b))
    # (a, sign b) = (sign a, b) up to the rational part's error bound on each side
    assert abs(_vdot(a, sb) - _vdot(sa, b)) <= 4e-10 * na * nb
    # D_N^dagger = gamma5 D_N gamma5: (a, D_N b) = (gamma5 D_N gamma5 a, b)
    g5 = torch.ones(4, 3, dtype=torch.complex128, device="cuda")
    g5[2:] = -1
    da, db = torch.empty_like(a), torch.empty_like(b)
    nd.nd_apply_DN(ctx, db, b, p)
    nd.nd_apply_DN(ctx, da, (a.view(-1, 4, 3) * g5).reshape(a.shape), p)
    lhs = _vdot(a, db)
    rhs = _vdot((da.view(-1, 4, 3) * g5).reshape(a.shape), b)
    assert abs(lhs - rhs) <= 4e-10 * (1 + S) * na * nb


def test_mixed_matches_fp64_and_polynomial(setup):
    nd, ctx, torch = setup
    eta = dev(synth.spinor(DIMS, seed=1))
    outs = {}
    for name, p in (("fp64", nd.dn_params(20, 0.0, 0.0, 1e-10, 200000, 0)),
                    ("fp32", nd.dn_params(20, 0.0, 0.0, 1e-10, 200000, 1)),
                    ("fp16", nd.dn_params(20, 0.0, 0.0, 1e-10, 200000, 2)),
                    ("poly", nd.dn_params(0, 0.0, 0.0, 1e-10, 1, 0, approx=nd.ND_SIGN_CHEBYSHEV))):
        o = torch.empty_like(eta)
        nd.nd_apply_DN(ctx, o, eta, p)
        outs[name] = o
    ref = outs["fp64"]
    nref = float(torch.linalg.vector_norm(ref))
    for name in ("fp32", "fp16"):
        assert float(torch.linalg.vector_norm(outs[name] - ref)) <= 1e-9 * nref
    # rational and polynomial approximations of the same deflated operator: each within 1e-10
    # (relative to the source, times 1 + s) of sign(Q) on the approximation interval
    assert float(torch.linalg.vector_norm(outs["poly"] - ref)) <= 5e-9 * nref


def test_propagator_residual(setup):
    nd, ctx, torch = setup
    b = torch.zeros(int(np.prod(DIMS)), 4, 3, dtype=torch.complex128, device="cuda")
    b[0, 0, 0] = 1.0
    p = nd.dn_params(20, 0.0, 0.0, 1e-12, 200000, 1, 0.1)
    x = torch.empty_like(b)
    info = nd.nd_propagator(ctx, x, b, p, tol=1e-10, maxit=2000)
    assert info.resid <= 1e-10
    # recompute D_N^m x with an FP64 sign(Q)
    dx = torch.empty_like(x)
    nd.nd_apply_DN(ctx, dx, x, nd.dn_params(20, 0.0, 0.0, 1e-12, 200000, 0, 0.1))
    assert float(torch.linalg.vector_norm(dx - b)) <= 1e-9
