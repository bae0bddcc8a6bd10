"""Low-mode checkpoint: the modes, nu and lambda_{l+1} saved from one context (nd_get_lowmodes,
nd_lowmode_state) and restored into a fresh one (nd_set_lowmodes) give the same D_N."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu
M, S = -1.4, 0.4


def test_save_and_restore_lowmodes(tmp_path):
    import torch

    import paper_1010_5636_gb300 as nd
    dims = (4, 4, 4, 4)
    U = dev(synth.gauge_field(dims, "haar", seed=0))
    eta = dev(synth.spinor(dims, seed=1))
    p = nd.dn_params(16, 0.0, 0.0, 1e-12, 20000, 0)
    a = nd.nd_create(dims, m=M, s=S)
    b = nd.nd_create(dims, m=M, s=S)
    try:
        nd.nd_set_links(a, U, (18, 12, 12))
        nd.nd_set_links(b, U, (18, 12, 12))
        nd.nd_lowmodes(a, 8, 1e-12, 20000)
        l, lam_next, lam_max = nd.nd_lowmode_state(a)
        assert l == 8 and lam_next > 0 and lam_max > 0
        path = str(tmp_path / "modes.npz")
        nd.save_lowmodes(a, path)
        info = nd.load_lowmodes(b, path)
        assert nd.nd_lowmode_state(b)[:2] == (l, lam_next)
        assert info.kappa_plus < 1e-6 and info.kappa_minus < 1e-6
        ya, yb = torch.empty_like(eta), torch.empty_like(eta)
        nd.nd_apply_DN(a, ya, eta, p)
        nd.nd_apply_DN(b, yb, eta, p)
        assert rel(host(yb), host(ya)) <= 1e-12
    finally:
        nd.nd_destroy(a)
        nd.nd_destroy(b)
