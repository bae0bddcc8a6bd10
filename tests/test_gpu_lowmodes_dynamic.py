"""GPU parity of the dynamic choice of l with kappa-driven stopping (nd_lowmodes_dynamic with the
filtered subspace iteration, nd_lowmodes_ritz with the paper's Ritz-functional minimiser; Sec. 2.3)
against the oracle's rule (oracle/lowmodes.choose_l) on the exact spectrum of the dense Q, and the
paper's projector-deviation bound ||P_+- - (P_+-)_exact|| <= kappa (1 + 2 kappa) / (1 - 2 kappa (1 + 2 kappa))
checked against the exact eigenvectors."""
import numpy as np
import pytest

import synth
from oracle import lowmodes
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
M, S = -1.4, 0.4


@pytest.fixture(scope="module")
def nd():
    import paper_1010_5636_gb300 as nd
    nd.lib()
    return nd


def _projector_deviation(A, B):
    """||P_A - P_B|| (spectral norm) for orthonormal column bases of equal dimension."""
    if A.shape[1] != B.shape[1]:
        return 1.0
    if A.shape[1] == 0:
        return 0.0
    s = np.linalg.svd(A.conj().T @ B, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - np.min(s) ** 2)))


# the sequential Ritz-functional minimiser is far slower than the block filter: a shorter window and
# a looser kappa target keep its case to seconds
@pytest.mark.parametrize("l_min,l_max,method,kappa", [(4, 12, "filter", 1e-6), (2, 6, "filter", 1e-6),
                                                      (9, 9, "filter", 1e-6), (2, 6, "ritz", 1e-4)])
def test_dynamic_l_vs_exact(nd, l_min, l_max, method, kappa):
    import torch
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    lm = lowmodes.lowmodes_dense(U, dims, M, l_max + 1)
    w, v = lm["spectrum"], lm["eigvecs"]  # all eigenpairs of Q
    order = np.argsort(np.abs(w))
    ev_q2 = w[order] ** 2
    l_exp = lowmodes.choose_l(ev_q2, l_min, l_max)
    ctx = nd.nd_create(dims, m=M, s=S)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 12, 12))
        l, nu, rho, ev, info = nd.nd_lowmodes_dynamic(ctx, l_min, l_max, kappa, 200000, method)
        print(f"{method} l_min {l_min} l_max {l_max}: l {l} (oracle {l_exp}) kappa +{info.kappa_plus:.2e} -{info.kappa_minus:.2e}"
              f" Q^2 applications {info.iters}")
        assert l == l_exp
        assert info.kappa_plus <= kappa and info.kappa_minus <= kappa
        # Ritz values are accurate to ~ (residual)^2: kappa 1e-6 gives 1e-8, 1e-4 still 1e-6
        assert np.allclose(ev, ev_q2[: l + 1], rtol=1e-8 if kappa <= 1e-6 else 1e-6)
        assert np.allclose(np.sort(nu), np.sort(w[order[:l]]), rtol=1e-9 if kappa <= 1e-6 else 1e-6, atol=1e-12)
        u_dev = torch.empty((l,) + (int(np.prod(dims)), 4, 3), dtype=torch.complex128, device="cuda")
        nd.nd_get_lowmodes(ctx, u_dev, l)
        u = host(u_dev).reshape(l, -1).T  # columns
        nu = np.asarray(nu)
        ex = v[:, order[:l]]
        wl = w[order[:l]]
        for sign, kappa in ((1, info.kappa_plus), (-1, info.kappa_minus)):
            dev_pm = _projector_deviation(u[:, sign * nu > 0], ex[:, sign * wl > 0])
            assert dev_pm <= lowmodes.projector_bound(kappa) + 1e-12
    finally:
        nd.nd_destroy(ctx)


def test_dynamic_l_feeds_dn(nd):
    """D_N after the dynamic low modes (eps from the chosen lambda_{l+1}) matches the exact D_N."""
    import torch
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    eta = synth.spinor(dims, seed=1)
    lm = lowmodes.lowmodes_dense(U, dims, M, 8)
    w, v = lm["spectrum"], lm["eigvecs"]
    S_ex = (v * np.sign(w)) @ v.conj().T
    b = eta.reshape(-1)
    g5 = np.tile(np.repeat([1, 1, -1, -1], 3), len(b) // 12)
    exact = (1 + S) * (b + g5 * (S_ex @ b))
    ctx = nd.nd_create(dims, m=M, s=S)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 12, 12))
        nd.nd_lowmodes_dynamic(ctx, 4, 12, 1e-8, 400000)
        out = torch.empty_like(dev(eta))
        info = nd.nd_apply_DN(ctx, out, dev(eta), nd.dn_params(16, 0.0, 0.0, 1e-12, 20000, 0))
        assert np.linalg.norm(host(out).reshape(-1) - exact) <= (1 + S) * (info.delta + 1e-9) * np.linalg.norm(b) + \
            1e-9 * np.linalg.norm(b)
    finally:
        nd.nd_destroy(ctx)


def test_bad_arguments_and_limit(nd):
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    ctx = nd.nd_create(dims, m=M, s=S)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 12, 12))
        for args in [(0, 4), (5, 4), (4, 65)]:
            with pytest.raises(nd.NdError) as e:
                nd.nd_lowmodes_dynamic(ctx, *args, 1e-6, 1000)
            assert e.value.status == nd.ND_ERR_INVALID_ARG
        with pytest.raises(nd.NdError) as e:
            nd.nd_lowmodes_dynamic(ctx, 4, 12, 1e-12, 50)
        assert e.value.status == nd.ND_ERR_NOT_CONVERGED
    finally:
        nd.nd_destroy(ctx)
