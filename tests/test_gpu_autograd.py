"""Differentiation through the C-ABI: the link gradient of S = phi^dagger (Q^2)^{-1} phi against
central finite differences of the oracle's S along random complex (non-unitary) directions,
the su(3) force obtained by torch autograd through U = exp(i omega.T) U0 against the oracle's
force, the source gradient, and the D_N vector-Jacobian product against the oracle's
gamma5 D_N gamma5."""
import numpy as np
import pytest

import synth
from oracle import force as oforce
from oracle import lowmodes, overlap
from tests.gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu
M, S = -1.4, 0.4


@pytest.fixture(scope="module")
def nd():
    import paper_1010_5636_gb300 as nd
    nd.lib()
    return nd


def test_link_gradient_finite_differences(nd):
    import torch

    from paper_1010_5636_gb300 import autograd as ag
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, "haar", seed=2)
    phi = synth.spinor(dims, seed=3)
    lat = nd.Lattice(dims, m=M, s=S)
    Ut = dev(U).requires_grad_(True)
    Sv = ag.pseudofermion_action(lat, Ut, dev(phi), tol=1e-14)
    Sv.backward()
    G = host(Ut.grad)
    assert abs(float(Sv.detach()) - oforce.action(U, dims, M, phi, tol=1e-14)) <= 1e-11 * abs(float(Sv.detach()))
    h = 1e-5
    for seed in range(3):
        D = synth.complex_gaussian(synth.rng(30 + seed), U.shape)
        sp = oforce.action(np.ascontiguousarray(U + h * D), dims, M, phi, tol=1e-14)
        sm = oforce.action(np.ascontiguousarray(U - h * D), dims, M, phi, tol=1e-14)
        fd = (sp - sm) / (2 * h)
        an = float(np.sum((G.conj() * D).real))  # torch convention: dS = Re sum conj(grad) dU
        assert abs(fd - an) <= 1e-7 * abs(an)


def test_force_through_autograd(nd):
    """d S(exp(i omega.T) U0) / d omega at omega = 0, by torch autograd over the library's
    gradient, equals the su(3) force of the oracle and of nd_force."""
    import torch

    from paper_1010_5636_gb300 import autograd as ag
    dims = (4, 4, 2, 4)
    V = int(np.prod(dims))
    U0 = synth.gauge_field(dims, "near_identity", seed=0, eps=0.3)
    phi = synth.spinor(dims, seed=1)
    ref = oforce.force(U0, dims, M, phi, tol=1e-14)
    lat = nd.Lattice(dims, m=M, s=S)
    lam = torch.from_numpy(synth.gellmann()).cuda()
    omega = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    H = torch.einsum("mva,aij->mvij", omega.to(torch.complex128), lam) / 2
    U = torch.matrix_exp(1j * H) @ dev(U0)
    Sv = ag.pseudofermion_action(lat, U, dev(phi), tol=1e-14)
    Sv.backward()
    assert rel(host(omega.grad), ref) <= 1e-10
    F = torch.empty((4, V, 8), dtype=torch.float64, device="cuda")
    nd.nd_set_links(lat.ctx, dev(U0), (18, 12, 12))
    nd.nd_force(lat.ctx, F, dev(phi), 1e-14, 100000, 0)
    assert rel(host(F), ref) <= 1e-10


@pytest.mark.parametrize("inner", [0, 1])
def test_source_gradient(nd, inner):
    import torch

    from paper_1010_5636_gb300 import autograd as ag
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, "haar", seed=5)
    phi = synth.spinor(dims, seed=6)
    X, _ = oforce.solve_Q2(U, dims, M, phi, tol=1e-14)
    lat = nd.Lattice(dims, m=M, s=S)
    ph = dev(phi).requires_grad_(True)
    Sv = ag.pseudofermion_action(lat, dev(U), ph, tol=1e-13, inner=inner)
    (2.5 * Sv).backward()
    # dS/dphi^* = X; torch's gradient of a real loss is twice that
    assert rel(host(ph.grad), 2 * 2.5 * X) <= 1e-11


def test_overlap_vjp(nd):
    """VJP of eta -> D_N eta equals gamma5 D_N gamma5 g (oracle), with the oracle's modes."""
    import torch

    from paper_1010_5636_gb300 import autograd as ag
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=0)
    lm = lowmodes.lowmodes_dense(U, dims, M, 6)
    lam_max = 1.01 * lm["lam_max"]
    eps = 0.99 * lm["lam_next"] / lam_max
    eta = synth.spinor(dims, seed=1)
    w = synth.spinor(dims, seed=2)
    expect, _ = overlap.dn_apply(U, dims, M, S, overlap.gamma5(w), lam_max, eps, 16, 1e-12, lm["u"], lm["nu"])
    expect = overlap.gamma5(expect)
    lat = nd.Lattice(dims, U=dev(U), m=M, s=S, recon=(18, 12, 12))
    nd.nd_set_lowmodes(lat.ctx, dev(lm["u"]), list(lm["nu"]), lm["lam_next"])
    p = nd.dn_params(16, eps, lam_max, 1e-12, 100000, 1, 0.0, False)
    e = dev(eta).requires_grad_(True)
    out = ag.dirac_overlap(lat, e, p)
    loss = (torch.conj(dev(w)) * out).real.sum()
    loss.backward()
    # torch's gradient of the real loss Re <w, A eta> with respect to eta is A^H w
    assert rel(host(e.grad), expect) <= 1e-10


def test_dn_dagger_massive(nd):
    """nd_apply_DN_dagger: (D_N^m)^dagger w = gamma5 D_N^m gamma5 w (oracle) for m_q > 0, and the
    left-only form (not hermitian) is refused."""
    import torch
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=0)
    lm = lowmodes.lowmodes_dense(U, dims, M, 6)
    lam_max = 1.01 * lm["lam_max"]
    eps = 0.99 * lm["lam_next"] / lam_max
    w = synth.spinor(dims, seed=2)
    expect, _ = overlap.dn_apply(U, dims, M, S, overlap.gamma5(w), lam_max, eps, 16, 1e-12, lm["u"], lm["nu"],
                                 m_q=0.1)
    expect = overlap.gamma5(expect)
    lat = nd.Lattice(dims, U=dev(U), m=M, s=S, recon=(18, 12, 12))
    nd.nd_set_lowmodes(lat.ctx, dev(lm["u"]), list(lm["nu"]), lm["lam_next"])
    out = torch.empty_like(dev(w))
    for inner in (0, 1):
        nd.nd_apply_DN_dagger(lat.ctx, out, dev(w), nd.dn_params(16, eps, lam_max, 1e-12, 100000, inner, 0.1))
        assert rel(host(out), expect) <= 1e-10
    with pytest.raises(nd.NdError) as e:
        nd.nd_apply_DN_dagger(lat.ctx, out, dev(w), nd.dn_params(16, eps, lam_max, 1e-12, 100000, 0, 0.1, True))
    assert e.value.status == nd.ND_ERR_INVALID_ARG
    lat.close()
