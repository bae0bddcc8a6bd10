"""Pins of the oracle's site tables by brute force: bijection, parity blocks, neighbour
relations checked against coordinates."""
import numpy as np
import pytest

from oracle import geometry


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (8, 2, 4, 6)])
def test_eo_tables(dims):
    V = int(np.prod(dims))
    x = geometry.coords(dims)
    l2e = geometry.lex_to_eo(dims)
    assert sorted(l2e.tolist()) == list(range(V))
    par = x.sum(axis=1) % 2
    assert np.all((l2e >= V // 2) == (par == 1))
    # within a parity, eo order follows lex order
    for p in (0, 1):
        sel = np.nonzero(par == p)[0]
        assert np.all(np.diff(l2e[sel]) == 1)
    nbr = geometry.neighbour_eo(dims)
    e2l = np.empty(V, dtype=np.int64)
    e2l[l2e] = np.arange(V)
    for mu in range(4):
        f, b = nbr[2 * mu], nbr[2 * mu + 1]
        assert np.all(b[f] == np.arange(V)) and np.all(f[b] == np.arange(V))
        # opposite parity, and the coordinate step is exactly +-1 along mu (mod extent)
        assert np.all((f >= V // 2) != (np.arange(V) >= V // 2))
        xs, xf = x[e2l], x[e2l[f]]
        d = (xf - xs) % np.asarray(dims)
        expect = np.zeros(4, dtype=np.int64)
        expect[mu] = 1 % dims[mu]
        assert np.all(d == expect)


def test_odd_extent_rejected():
    with pytest.raises(ValueError):
        geometry.lex_to_eo((4, 4, 4, 3))
