"""The Lattice convenience class: each method is argument marshalling over one C-ABI call, so one
call per method against the direct entry point (or the oracle) on the 4^4 Haar lattice."""
import numpy as np
import pytest

import synth
from oracle import wilson
from tests.gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu
M, S = -1.4, 0.4


def test_lattice_methods():
    import paper_1010_5636_gb300 as nd
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=0)
    eta = synth.spinor(dims, seed=1)
    lat = nd.Lattice(dims, dev(U), m=M, s=S, recon=(18, 12, 12))
    try:
        assert rel(host(lat.Q(dev(eta))), wilson.apply_Q(U, eta, dims, M)) <= 1e-13
        l, nu, rho, ev, info = lat.lowmodes(l_range=(4, 12), kappa=1e-6)
        assert 4 <= l <= 12 and info.kappa_plus <= 1e-6
        sg, si = lat.sign(dev(eta), n_poles=16, tol=1e-12)
        dn, di = lat.DN(dev(eta), n_poles=16, tol=1e-12)
        g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), eta.size // 12).reshape(eta.shape)
        assert rel(host(dn), (1 + S) * (eta + g5 * host(sg))) <= 1e-10
        x, pi = lat.propagator(dev(eta), 1e-10, 5000, sign_tol=1e-12, n_poles=16, m_q=0.1)
        assert pi.resid <= 1e-10
        x1, i1 = lat.solve_Q2(dev(eta), 1e-10)
        x2, i2 = lat.solve_Q2(dev(eta), 1e-10, even_odd=True)
        assert i1.max_resid <= 1e-10 and i2.max_resid <= 1e-10
        assert rel(host(x1), host(x2)) <= 1e-8
    finally:
        lat.close()
