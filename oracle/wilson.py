"""ctypes front end of the oracle's C part (oracle/wilson.c): Q = gamma5 D_W and the force.

Test infrastructure only.  Operator definition: Sec. 2.1 (D_W, Q = gamma5 D_W, U_{-mu}, gamma_{-mu}).
Arrays are canonical complex128 (see ``synth``): U[4, V, 3, 3], psi[V, 4, 3].
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        d = ctypes.c_double
        p = ctypes.c_void_p
        i = ctypes.c_int
        for name in ("oracle_apply_Q", "oracle_apply_DW"):
            f = getattr(_lib, name)
            f.argtypes = [p, i, d, p, p, p]
            f.restype = None
        _lib.oracle_force.argtypes = [p, i, p, p, p, p]
        _lib.oracle_gamma.argtypes = [i, p]
        _lib.oracle_gellmann.argtypes = [i, p]
        _lib.oracle_set_threads.argtypes = [i]
        _lib.oracle_get_threads.restype = i
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _check(U, psi, dims):
    V = int(np.prod(dims))
    assert U.dtype == np.complex128 and U.shape == (4, V, 3, 3) and U.flags.c_contiguous
    assert psi.dtype == np.complex128 and psi.shape[-3:] == (V, 4, 3) and psi.flags.c_contiguous


def set_threads(n):
    lib().oracle_set_threads(int(n))


def get_threads():
    return int(lib().oracle_get_threads())


def apply_Q(U, psi, dims, m, antiperiodic_t=False):
    """Q psi = gamma5 D_W psi (Sec. 2.1).  psi may carry leading batch axes."""
    _check(U, psi, dims)
    psi = np.ascontiguousarray(psi)
    out = np.empty_like(psi)
    d = _dims(dims)
    V = int(np.prod(dims))
    flat_in = psi.reshape(-1, V, 4, 3)
    flat_out = out.reshape(-1, V, 4, 3)
    for k in range(flat_in.shape[0]):
        lib().oracle_apply_Q(_ptr(d), int(antiperiodic_t), float(m), _ptr(U), _ptr(flat_in[k]), _ptr(flat_out[k]))
    return out


def apply_DW(U, psi, dims, m, antiperiodic_t=False):
    """D_W psi (Sec. 2.1), without the gamma5."""
    _check(U, psi, dims)
    psi = np.ascontiguousarray(psi)
    out = np.empty_like(psi)
    d = _dims(dims)
    lib().oracle_apply_DW(_ptr(d), int(antiperiodic_t), float(m), _ptr(U), _ptr(psi), _ptr(out))
    return out


def apply_Q2(U, psi, dims, m, antiperiodic_t=False):
    return apply_Q(U, apply_Q(U, psi, dims, m, antiperiodic_t), dims, m, antiperiodic_t)


def gamma(mu):
    """The oracle's gamma matrix (mu = 0..3) or gamma5 (mu = 4) as a 4x4 complex array."""
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().oracle_gamma(int(mu), _ptr(out))
    return out


def gellmann(a):
    """The oracle's Gell-Mann matrix lambda^a, a = 1..8."""
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().oracle_gellmann(int(a), _ptr(out))
    return out


def force(U, X, Y, dims, antiperiodic_t=False):
    """F[mu, lex, a] = -Im tr[T^a (A1 - A2)] for given X = (Q^2)^{-1} phi and Y = Q X
    (see oracle/wilson.c for A1, A2 and the derivation from the definition of D_W)."""
    _check(U, X, dims)
    _check(U, Y, dims)
    V = int(np.prod(dims))
    F = np.zeros((4, V, 8), dtype=np.float64)
    d = _dims(dims)
    lib().oracle_force(_ptr(d), int(antiperiodic_t), _ptr(U), _ptr(np.ascontiguousarray(X)),
                       _ptr(np.ascontiguousarray(Y)), _ptr(F))
    return F


def dense_Q(U, dims, m, antiperiodic_t=False):
    """The (12V x 12V) matrix of Q, assembled column by column from unit vectors (small lattices only)."""
    V = int(np.prod(dims))
    n = 12 * V
    cols = np.zeros((n, V, 4, 3), dtype=np.complex128)
    cols.reshape(n, n)[np.arange(n), np.arange(n)] = 1.0
    out = apply_Q(U, cols, dims, m, antiperiodic_t)
    return np.ascontiguousarray(out.reshape(n, n).T)
