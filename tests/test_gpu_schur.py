"""GPU parity of the even-odd Schur-complement operator Qhat (nd_apply_Qhat) and of the
Schur-complement (Q^2)^{-1} solve (nd_solve_Q2_eo) against the oracle (oracle/schur.py), the
dense LAPACK solve at 4^4, and the whole-lattice multi-shift solver at a larger lattice."""
import numpy as np
import pytest

import synth
from oracle import schur, wilson
from tests.gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu
M = -1.4
# Qhat is two stencil passes: FP64 to rounding, FP32 / FP16 storage to their precision
TOL = {0: 1e-12, 1: 2e-6, 2: 5e-3}


@pytest.fixture(scope="module")
def nd():
    import paper_1010_5636_gb300 as nd
    nd.lib()
    return nd


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("dims,kind", [((4, 4, 4, 4), "haar"), ((6, 4, 2, 8), "near_identity")])
def test_qhat_vs_oracle(nd, prec, recon, dims, kind):
    import torch
    V = int(np.prod(dims))
    U = synth.gauge_field(dims, kind, seed=0, eps=0.3) if kind == "near_identity" else synth.gauge_field(dims, kind, seed=0)
    even = schur.parity_mask(dims)
    psi = even * synth.spinor(dims, seed=3)
    expect = schur.qhat_apply(U, dims, M, psi)
    ctx = nd.nd_create(dims, m=M)
    try:
        links = [0, 0, 0]
        links[prec] = recon
        nd.nd_set_links(ctx, dev(U), tuple(links))
        inb = torch.empty(nd.nd_spinor_bytes(ctx, prec), dtype=torch.uint8, device="cuda")
        outb = torch.zeros_like(inb)
        nd.nd_pack_spinor(ctx, inb, dev(psi), prec)
        nd.nd_apply_Qhat(ctx, outb, inb, prec)
        got = torch.empty((V, 4, 3), dtype=torch.complex128, device="cuda")
        nd.nd_unpack_spinor(ctx, got, outb, prec)
        torch.cuda.synchronize()
        g = host(got)
        assert np.all(g[even[:, 0, 0] == 0] == 0)  # odd half of out untouched (zero)
        assert rel(g, expect) <= TOL[prec]
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_q2_solve_vs_dense(nd, inner):
    import torch
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    b = synth.spinor(dims, seed=5)
    Q = wilson.dense_Q(U, dims, M)
    Q2 = Q @ Q
    ex = np.linalg.solve(Q2, b.reshape(-1))
    w = np.linalg.eigvalsh(Q2)
    tol = 1e-10
    ctx = nd.nd_create(dims, m=M)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 12, 12))
        x = torch.empty_like(dev(b))
        info = nd.nd_solve_Q2_eo(ctx, x, dev(b), tol, 5000, inner)
        print(f"inner {inner}: CG iterations {info.iters}, sweeps {info.outer}, resid {info.max_resid:.2e}")
        assert info.max_resid <= tol
        # ||x - x*|| <= ||(Q^2)^{-1}|| ||b - Q^2 x||
        assert np.linalg.norm(host(x).reshape(-1) - ex) <= 1.01 * tol * np.linalg.norm(b) / w.min()
        # the oracle's Schur route gives the same solution
        y, _ = schur.q2_solve(U, dims, M, b, tol=1e-12)
        assert np.linalg.norm(host(x).reshape(-1) - y.reshape(-1)) <= 2 * tol * np.linalg.norm(b) / w.min()
    finally:
        nd.nd_destroy(ctx)


def test_q2_solve_matches_full_lattice_solver(nd):
    """8^3x16 near-identity links: the Schur route and the whole-lattice CG (nd_solve, one shift 0)
    agree within the two solvers' residual bounds."""
    import torch
    dims = (16, 8, 8, 8)
    U = synth.gauge_field(dims, "near_identity", seed=0, eps=0.3)
    b = synth.spinor(dims, seed=6)
    tol = 1e-10
    ctx = nd.nd_create(dims, m=M)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 12, 12))
        x1 = torch.empty_like(dev(b))
        i1 = nd.nd_solve_Q2_eo(ctx, x1, dev(b), tol, 20000, 1)
        x2 = torch.empty_like(dev(b))
        i2 = nd.nd_solve(ctx, [x2], dev(b), [0.0], tol, 20000, 0)
        assert i1.max_resid <= tol and i2.max_resid <= tol
        # both residuals are <= tol ||b||, so ||x1 - x2|| <= 2 tol ||b|| / lambda_min(Q^2); lambda_min is
        # O(1) for these links (free-field value m^2 = 1.96), hence the bound below
        d = rel(host(x1), host(x2))
        print(f"Schur: {i1.iters} Qhat^2 iterations in {i1.outer} sweeps; full: {i2.iters} Q^2 iterations; rel diff {d:.2e}")
        assert d <= 1e-7
    finally:
        nd.nd_destroy(ctx)


def test_failures_keep_context_usable(nd):
    import torch
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    b = synth.spinor(dims, seed=7)
    ctx = nd.nd_create(dims, m=M)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 12, 0))
        x = torch.empty_like(dev(b))
        with pytest.raises(nd.NdError) as e:
            nd.nd_solve_Q2_eo(ctx, x, dev(b), 1e-10, 1, 0)
        assert e.value.status == nd.ND_ERR_NOT_CONVERGED
        with pytest.raises(nd.NdError) as e:
            nd.nd_solve_Q2_eo(ctx, x, dev(b), 1e-10, 100, 2)  # FP16 links not set
        assert e.value.status == nd.ND_ERR_STATE
        info = nd.nd_solve_Q2_eo(ctx, x, dev(b), 1e-10, 5000, 1)
        assert info.max_resid <= 1e-10
    finally:
        nd.nd_destroy(ctx)
