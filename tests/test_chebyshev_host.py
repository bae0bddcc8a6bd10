"""The library's host minmax-polynomial generator (nd_chebyshev, Remez exchange in C++) and its
degree search against the oracle's numpy Remez, without a GPU."""
import numpy as np
import pytest

from oracle import chebyshev


@pytest.mark.parametrize("n,eps", [(0, 0.3), (1, 0.1), (8, 0.05), (40, 1e-2), (150, 2e-3), (300, 1e-3)])
def test_table_matches_oracle(n, eps):
    import paper_1010_5636_gb300 as nd
    c, delta = nd.nd_chebyshev(n, eps)
    ref = chebyshev.minmax(n, eps)
    assert len(c) == n + 1
    assert np.max(np.abs(np.array(c) - ref["c"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["c"])))
    # the levelled error is known to a few 1e-15 absolute in FP64
    assert abs(delta - ref["delta"]) <= 1e-6 * ref["delta"] + 5e-14


@pytest.mark.parametrize("eps,target", [(0.1, 1e-3), (1e-2, 1e-8), (5e-3, 1e-6)])
def test_degree_matches_oracle(eps, target):
    import paper_1010_5636_gb300 as nd
    n = nd.nd_chebyshev_degree(eps, target)
    assert n == chebyshev.degree_for(eps, target)
    assert nd.nd_chebyshev(n, eps)[1] <= target


def test_bad_arguments():
    import paper_1010_5636_gb300 as nd
    for args in [(-1, 0.1), (2049, 0.1), (4, 0.0), (4, 1.0)]:
        with pytest.raises(nd.NdError) as e:
            nd.nd_chebyshev(*args)
        assert e.value.status == nd.ND_ERR_INVALID_ARG
    with pytest.raises(nd.NdError):
        nd.nd_chebyshev_degree(1e-2, 0.0)
