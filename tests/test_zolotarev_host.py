"""The library's host Zolotarev generator (nd_zolotarev, long-double AGM) against the
oracle's 40-digit mpmath table, without a GPU."""
import numpy as np
import pytest

from oracle import zolotarev


@pytest.mark.parametrize("n,eps", [(4, 1e-2), (8, 1e-3), (16, 1e-4), (20, 1e-4), (20, 3e-6), (32, 1e-7)])
def test_table_matches_oracle(n, eps):
    import paper_1010_5636_gb300 as nd
    sig, b, delta = nd.nd_zolotarev(n, eps)
    ref = zolotarev.zolotarev(n, eps)
    assert np.allclose(sig, ref["sigma"], rtol=1e-13, atol=0)
    assert np.allclose(b, ref["b"], rtol=1e-12, atol=0)
    # below ~1e-15 the error is set by rounding the coefficients to FP64, not by the generator
    assert abs(delta - ref["delta"]) <= 1e-6 * ref["delta"] + 1e-15


def test_bad_arguments():
    import paper_1010_5636_gb300 as nd
    with pytest.raises(nd.NdError):
        nd.nd_zolotarev(0, 1e-3)
    with pytest.raises(nd.NdError):
        nd.nd_zolotarev(8, 1.5)


@pytest.mark.parametrize("eps", [0.5, 1e-2, 1e-4])
def test_one_pole_closed_form(eps):
    """The host generator at n = 1 against sigma = sqrt(eps), b = 2 / (1/(1 + k) + 1/(2 k^(1/2)))."""
    import paper_1010_5636_gb300 as nd
    sig, b, delta = nd.nd_zolotarev(1, eps)
    k = np.sqrt(eps)
    bb = 2.0 / (1.0 / (1.0 + k) + 1.0 / (2.0 * eps ** 0.25))
    assert sig[0] == pytest.approx(k, rel=1e-13)
    assert b[0] == pytest.approx(bb, rel=1e-13)
    assert delta == pytest.approx(1.0 - bb / (1.0 + k), rel=1e-9)
