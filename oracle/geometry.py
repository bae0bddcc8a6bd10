"""Site tables of the oracle: lexicographic coordinates, even-odd index and neighbours.

Test infrastructure only.  The paper assigns one thread per lattice site (Sec. 2.1) and
leaves the ordering open; the reading used throughout is:
  lex(x) = x3 + L3*(x2 + L2*(x1 + L1*x0)),  parity p(x) = (x0+x1+x2+x3) mod 2,
  eo(x)  = p(x) * V/2 + floor(lex(x) / 2),   all four extents even.
Direction d = 2*mu + s names the neighbour x + mu (s = 0) or x - mu (s = 1), periodic.
"""
import numpy as np


def coords(dims):
    """x[lex, 4] by explicit nested loops over (x0, x1, x2, x3) in lex order."""
    T, L1, L2, L3 = dims
    out = np.zeros((T * L1 * L2 * L3, 4), dtype=np.int64)
    k = 0
    for x0 in range(T):
        for x1 in range(L1):
            for x2 in range(L2):
                for x3 in range(L3):
                    out[k] = (x0, x1, x2, x3)
                    k += 1
    return out


def lex_of(dims, x):
    T, L1, L2, L3 = dims
    return x[..., 3] + L3 * (x[..., 2] + L2 * (x[..., 1] + L1 * x[..., 0]))


def lex_to_eo(dims):
    if any(int(n) % 2 for n in dims):
        raise ValueError("all lattice extents must be even for even-odd ordering")
    V = int(np.prod(dims))
    x = coords(dims)
    lex = np.arange(V)
    par = x.sum(axis=1) % 2
    return par * (V // 2) + lex // 2


def neighbour_eo(dims):
    """nbr[d, e] = eo index of the neighbour in direction d of the site with eo index e."""
    V = int(np.prod(dims))
    x = coords(dims)
    l2e = lex_to_eo(dims)
    e2l = np.empty(V, dtype=np.int64)
    e2l[l2e] = np.arange(V)
    nbr = np.zeros((8, V), dtype=np.int64)
    dims_a = np.asarray(dims)
    for mu in range(4):
        for s, step in ((0, +1), (1, -1)):
            y = x.copy()
            y[:, mu] = (y[:, mu] + step) % dims_a[mu]
            nb_lex = lex_of(dims, y)
            nbr[2 * mu + s, l2e] = l2e[nb_lex]
    return nbr
