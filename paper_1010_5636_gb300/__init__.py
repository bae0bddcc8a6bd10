"""Python binding of libnd: the Neuberger-Dirac operator on one GB300 (sm_103a).

Argument marshalling only: every function below forwards to the C-ABI entry point of the
same name declared in include/nd.h; all arithmetic runs in the library's CUDA kernels.
PyTorch supplies device memory (tensor.data_ptr()) and the current CUDA stream.

If libnd.so is missing or no CUDA device is present the calls raise: there is no CPU
fallback.

Canonical tensors (see include/nd.h): spinors complex128 [V, 4, 3] (or float64 [V, 4, 3, 2]),
links complex128 [4, V, 3, 3], force float64 [4, V, 8], all on cuda and contiguous.
"""
import ctypes
import os

from . import build as _build

ND_OK, ND_ERR_INVALID_ARG, ND_ERR_CUDA, ND_ERR_OOM = 0, -1, -2, -3
ND_ERR_NOT_CONVERGED, ND_ERR_BREAKDOWN, ND_ERR_NAN, ND_ERR_STATE = -4, -5, -6, -7
ND_FP64, ND_FP32, ND_FP16 = 0, 1, 2
PRECS = {"fp64": ND_FP64, "fp32": ND_FP32, "fp16": ND_FP16}


class NdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class nd_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("sloppy_iters", ctypes.c_int),
                ("max_resid", ctypes.c_double), ("time_ms", ctypes.c_double)]


class nd_lowmode_info(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int), ("iters", ctypes.c_int), ("lambda_max", ctypes.c_double),
                ("lambda_next", ctypes.c_double), ("kappa_plus", ctypes.c_double),
                ("kappa_minus", ctypes.c_double), ("max_rho", ctypes.c_double), ("time_ms", ctypes.c_double)]


class nd_dn_params(ctypes.Structure):
    _fields_ = [("n_poles", ctypes.c_int), ("eps", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("inner_prec", ctypes.c_int),
                ("m_q", ctypes.c_double), ("left_only", ctypes.c_int), ("approx", ctypes.c_int),
                ("degree", ctypes.c_int)]


class nd_dn_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("sloppy_iters", ctypes.c_int), ("outer", ctypes.c_int),
                ("n_low", ctypes.c_int), ("delta", ctypes.c_double), ("eps", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("max_resid", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("degree", ctypes.c_int), ("krylov_ms", ctypes.c_double), ("krylov_live_shifts", ctypes.c_int),
                ("krylov_active_shifts", ctypes.c_int), ("residuals64", ctypes.c_int),
                ("correction_iters", ctypes.c_int), ("refine_ms", ctypes.c_double)]


class nd_prop_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("sign_iters", ctypes.c_int),
                ("resid", ctypes.c_double), ("time_ms", ctypes.c_double)]


_P, _I, _D, _L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
_SIGS = {
    "nd_create": ([ctypes.POINTER(_P), _P, _I, _D, _D, _P], _I),
    "nd_destroy": ([_P], None),
    "nd_set_stream": ([_P, _P], _I),
    "nd_status_string": ([_I], ctypes.c_char_p),
    "nd_last_error": ([_P], ctypes.c_char_p),
    "nd_volume": ([_P], _L),
    "nd_spinor_bytes": ([_P, _I], ctypes.c_size_t),
    "nd_set_links": ([_P, _P, _P], _I),
    "nd_pack_spinor": ([_P, _P, _P, _I, _I], _I),
    "nd_unpack_spinor": ([_P, _P, _P, _I, _I], _I),
    "nd_pack_spinor_f32": ([_P, _P, _P, _I, _I], _I),
    "nd_unpack_spinor_f32": ([_P, _P, _P, _I, _I], _I),
    "nd_eo_tables": ([_P, _P, _P], _I),
    "nd_apply_Q": ([_P, _P, _P, _I, _I], _I),
    "nd_apply_Q_parity": ([_P, _P, _P, _I, _I, _D], _I),
    "nd_apply_Q_canonical": ([_P, _P, _P], _I),
    "nd_apply_Q_batched": ([_P, _I, _P, _P, _P, _I, _P], _I),
    "nd_apply_Q_norms_static": ([_P, _P, _P, _I, _P], _I),
    "nd_solve": ([_P, _P, _P, _P, _I, _D, _I, _I, ctypes.POINTER(nd_solve_info)], _I),
    "nd_lowmodes": ([_P, _I, _D, _I, _P, _P, _P, ctypes.POINTER(nd_lowmode_info)], _I),
    "nd_set_lowmodes": ([_P, _I, _P, _P, _D, ctypes.POINTER(nd_lowmode_info)], _I),
    "nd_get_lowmodes": ([_P, _P, _P], _I),
    "nd_lambda_max": ([_P, _I, ctypes.POINTER(_D)], _I),
    "nd_zolotarev": ([_I, _D, _P, _P, ctypes.POINTER(_D)], _I),
    "nd_chebyshev": ([_I, _D, _P, ctypes.POINTER(_D)], _I),
    "nd_apply_Qhat": ([_P, _P, _P, _I], _I),
    "nd_lowmodes_dynamic": ([_P, _I, _I, _D, _I, ctypes.POINTER(_I), _P, _P, _P, ctypes.POINTER(nd_lowmode_info)], _I),
    "nd_lowmodes_ritz": ([_P, _I, _I, _D, _I, ctypes.POINTER(_I), _P, _P, _P, ctypes.POINTER(nd_lowmode_info)], _I),
    "nd_lowmode_state": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "nd_solve_Q2_eo": ([_P, _P, _P, _D, _I, _I, ctypes.POINTER(nd_solve_info)], _I),
    "nd_propagator": ([_P, _P, _P, ctypes.POINTER(nd_dn_params), _D, _I, ctypes.POINTER(nd_prop_info)], _I),
    "nd_chebyshev_degree": ([_D, _D, ctypes.POINTER(_I)], _I),
    "nd_apply_sign": ([_P, _P, _P, ctypes.POINTER(nd_dn_params), ctypes.POINTER(nd_dn_info)], _I),
    "nd_apply_DN": ([_P, _P, _P, ctypes.POINTER(nd_dn_params), ctypes.POINTER(nd_dn_info)], _I),
    "nd_apply_DN_dagger": ([_P, _P, _P, ctypes.POINTER(nd_dn_params), ctypes.POINTER(nd_dn_info)], _I),
    "nd_force": ([_P, _P, _P, _D, _I, _I, ctypes.POINTER(nd_solve_info)], _I),
    "nd_link_gradient": ([_P, _P, _P, ctypes.POINTER(_D), _P, _D, _I, _I, ctypes.POINTER(nd_solve_info)], _I),
}

_lib = None


def lib_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libnd.so (building it first if it is missing and nvcc is available)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise NdError(ND_ERR_STATE, "libnd.so is not built (run __graft_entry__.build())")
            _build.build()
        L = ctypes.CDLL(_build.LIB)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def declared_symbols():
    return sorted(_SIGS)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(ctx, st, what):
    if st != ND_OK:
        msg = lib().nd_last_error(ctx).decode() if ctx else lib().nd_status_string(st).decode()
        raise NdError(st, f"{what}: {msg}")


def _f64(t):
    """Canonical tensors may be complex128; the C-ABI sees interleaved float64."""
    import torch
    assert t.is_cuda and t.is_contiguous(), "canonical tensors must be contiguous CUDA tensors"
    assert t.dtype in (torch.complex128, torch.float64)
    return t


# ------------------------------------------------------------------ C-ABI wrappers (same names)

def nd_create(dims, antiperiodic_t=False, m=-1.4, s=0.4, stream=None):
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    st = lib().nd_create(ctypes.byref(h), ctypes.cast(d, ctypes.c_void_p), int(antiperiodic_t), float(m), float(s),
                         stream if stream is not None else _stream())
    _check(None, st, "nd_create")
    return h


def nd_destroy(ctx):
    lib().nd_destroy(ctx)


def nd_set_stream(ctx, stream=None):
    _check(ctx, lib().nd_set_stream(ctx, stream if stream is not None else _stream()), "nd_set_stream")


def nd_volume(ctx):
    return int(lib().nd_volume(ctx))


def nd_spinor_bytes(ctx, prec):
    return int(lib().nd_spinor_bytes(ctx, int(prec)))


def nd_set_links(ctx, U, recon=(18, 18, 12)):
    r = (ctypes.c_int * 3)(*[int(x) for x in recon])
    _check(ctx, lib().nd_set_links(ctx, _ptr(_f64(U)), ctypes.cast(r, ctypes.c_void_p)), "nd_set_links")


def nd_pack_spinor(ctx, internal, canon, prec, nrhs=1):
    _check(ctx, lib().nd_pack_spinor(ctx, _ptr(internal), _ptr(_f64(canon)), int(prec), int(nrhs)), "nd_pack_spinor")


def nd_unpack_spinor(ctx, canon, internal, prec, nrhs=1):
    _check(ctx, lib().nd_unpack_spinor(ctx, _ptr(_f64(canon)), _ptr(internal), int(prec), int(nrhs)),
           "nd_unpack_spinor")


def _f32(t):
    """Canonical single-precision tensors may be complex64; the C-ABI sees interleaved float32."""
    import torch
    assert t.is_cuda and t.is_contiguous(), "canonical tensors must be contiguous CUDA tensors"
    assert t.dtype in (torch.complex64, torch.float32)
    return t


def nd_pack_spinor_f32(ctx, internal, canon, prec, nrhs=1):
    _check(ctx, lib().nd_pack_spinor_f32(ctx, _ptr(internal), _ptr(_f32(canon)), int(prec), int(nrhs)),
           "nd_pack_spinor_f32")


def nd_unpack_spinor_f32(ctx, canon, internal, prec, nrhs=1):
    _check(ctx, lib().nd_unpack_spinor_f32(ctx, _ptr(_f32(canon)), _ptr(internal), int(prec), int(nrhs)),
           "nd_unpack_spinor_f32")


def nd_eo_tables(ctx, lex2eo, nbr):
    _check(ctx, lib().nd_eo_tables(ctx, _ptr(lex2eo), _ptr(nbr)), "nd_eo_tables")


def nd_apply_Q(ctx, out, inp, prec, nrhs=1):
    _check(ctx, lib().nd_apply_Q(ctx, _ptr(out), _ptr(inp), int(prec), int(nrhs)), "nd_apply_Q")


def nd_apply_Q_parity(ctx, out, inp, prec, parity, diag_coef):
    _check(ctx, lib().nd_apply_Q_parity(ctx, _ptr(out), _ptr(inp), int(prec), int(parity), float(diag_coef)),
           "nd_apply_Q_parity")


def nd_apply_Q_batched(ctxs, outs, ins, nrhs, prec, stream=None):
    """Q on several lattices (contexts) in one persistent launch; outs/ins: internal-layout tensors."""
    n = len(ctxs)
    cs = (ctypes.c_void_p * n)(*[c.value for c in ctxs])
    op = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
    ip = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ins])
    nr = (ctypes.c_int * n)(*[int(x) for x in nrhs])
    st = lib().nd_apply_Q_batched(ctypes.cast(cs, _P), n, ctypes.cast(op, _P), ctypes.cast(ip, _P),
                                  ctypes.cast(nr, _P), int(prec), stream if stream is not None else _stream())
    _check(ctxs[0], st, "nd_apply_Q_batched")


def nd_apply_Q_canonical(ctx, out, inp):
    _check(ctx, lib().nd_apply_Q_canonical(ctx, _ptr(_f64(out)), _ptr(_f64(inp))), "nd_apply_Q_canonical")


def nd_apply_Q_norms_static(ctx, out, inp, prec):
    """Q with fused norms and no device allocation (static scratch); returns (||out||^2, ||in||^2)."""
    norms = (ctypes.c_double * 2)()
    _check(ctx, lib().nd_apply_Q_norms_static(ctx, _ptr(out), _ptr(inp), int(prec), ctypes.cast(norms, _P)),
           "nd_apply_Q_norms_static")
    return norms[0], norms[1]


def nd_solve(ctx, xs, b, shifts, tol, maxit=100000, inner=ND_FP64):
    n = len(shifts)
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    sh = (ctypes.c_double * n)(*[float(s) for s in shifts])
    info = nd_solve_info()
    st = lib().nd_solve(ctx, ctypes.cast(xp, ctypes.c_void_p), _ptr(_f64(b)), ctypes.cast(sh, ctypes.c_void_p), n,
                        float(tol), int(maxit), int(inner), ctypes.byref(info))
    _check(ctx, st, "nd_solve")
    return info


def nd_lowmodes_dynamic(ctx, l_min, l_max, kappa_target=1e-6, maxit=1000000, method="filter"):
    """Low modes with l chosen in [l_min, l_max] by the largest relative gap, stopped at kappa_+- <=
    kappa_target; method "filter" (block Chebyshev-filtered subspace iteration) or "ritz" (the
    paper's Ritz-functional minimiser).  Returns (l, nu, rho, eval_Q2, info)."""
    fn = {"filter": lib().nd_lowmodes_dynamic, "ritz": lib().nd_lowmodes_ritz}[method]
    nu = (ctypes.c_double * l_max)()
    rho = (ctypes.c_double * l_max)()
    ev = (ctypes.c_double * (l_max + 1))()
    lo = ctypes.c_int()
    info = nd_lowmode_info()
    st = fn(ctx, int(l_min), int(l_max), float(kappa_target), int(maxit), ctypes.byref(lo), ctypes.cast(nu, _P),
            ctypes.cast(rho, _P), ctypes.cast(ev, _P), ctypes.byref(info))
    _check(ctx, st, "nd_lowmodes_" + ("dynamic" if method == "filter" else "ritz"))
    n = lo.value
    return n, list(nu)[:n], list(rho)[:n], list(ev)[:n + 1], info


def nd_lowmodes(ctx, l, tol=1e-12, maxit=100000):
    nu = (ctypes.c_double * l)()
    rho = (ctypes.c_double * l)()
    ev = (ctypes.c_double * (l + 1))()
    info = nd_lowmode_info()
    st = lib().nd_lowmodes(ctx, int(l), float(tol), int(maxit), ctypes.cast(nu, _P), ctypes.cast(rho, _P),
                           ctypes.cast(ev, _P), ctypes.byref(info))
    _check(ctx, st, "nd_lowmodes")
    return list(nu), list(rho), list(ev), info


def nd_set_lowmodes(ctx, evecs, nu, lambda_next):
    l = len(nu)
    nuc = (ctypes.c_double * l)(*[float(x) for x in nu])
    info = nd_lowmode_info()
    st = lib().nd_set_lowmodes(ctx, l, _ptr(_f64(evecs)), ctypes.cast(nuc, _P), float(lambda_next), ctypes.byref(info))
    _check(ctx, st, "nd_set_lowmodes")
    return info


def nd_get_lowmodes(ctx, evecs, l):
    nu = (ctypes.c_double * l)()
    _check(ctx, lib().nd_get_lowmodes(ctx, _ptr(_f64(evecs)), ctypes.cast(nu, _P)), "nd_get_lowmodes")
    return list(nu)


def nd_lowmode_state(ctx):
    """(l, lambda_next, lambda_max) of the context's low modes."""
    l, ln, lm = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().nd_lowmode_state(ctx, ctypes.byref(l), ctypes.byref(ln), ctypes.byref(lm)), "nd_lowmode_state")
    return l.value, ln.value, lm.value


def save_lowmodes(ctx, path):
    """Checkpoint the context's low modes (vectors, nu, lambda_next) to a .npz file."""
    import numpy as np
    import torch
    l, lam_next, lam_max = nd_lowmode_state(ctx)
    V = nd_volume(ctx)
    ev = torch.empty((max(l, 1), V, 4, 3), dtype=torch.complex128, device="cuda")
    nu = nd_get_lowmodes(ctx, ev, l) if l else []
    np.savez(path, evecs=ev[:l].cpu().numpy(), nu=np.asarray(nu, dtype=np.float64), lambda_next=lam_next,
             lambda_max=lam_max)


def load_lowmodes(ctx, path):
    """Restore low modes saved by save_lowmodes (rho and kappa are recomputed on the GPU)."""
    import numpy as np
    import torch
    d = np.load(path)
    return nd_set_lowmodes(ctx, torch.from_numpy(np.ascontiguousarray(d["evecs"])).cuda(), list(d["nu"]),
                           float(d["lambda_next"]))


def nd_lambda_max(ctx, iters=50):
    v = ctypes.c_double()
    _check(ctx, lib().nd_lambda_max(ctx, int(iters), ctypes.byref(v)), "nd_lambda_max")
    return v.value


def nd_zolotarev(n, eps):
    sig = (ctypes.c_double * n)()
    b = (ctypes.c_double * n)()
    d = ctypes.c_double()
    st = lib().nd_zolotarev(int(n), float(eps), ctypes.cast(sig, _P), ctypes.cast(b, _P), ctypes.byref(d))
    _check(None, st, "nd_zolotarev")
    return list(sig), list(b), d.value


def nd_chebyshev(degree, eps):
    """Minmax coefficients c[0..degree] of P_n on [eps, 1] and the uniform error delta."""
    c = (ctypes.c_double * (int(degree) + 1))()
    d = ctypes.c_double()
    _check(None, lib().nd_chebyshev(int(degree), float(eps), ctypes.cast(c, _P), ctypes.byref(d)), "nd_chebyshev")
    return list(c), d.value


def nd_chebyshev_degree(eps, delta_target):
    n = ctypes.c_int()
    _check(None, lib().nd_chebyshev_degree(float(eps), float(delta_target), ctypes.byref(n)), "nd_chebyshev_degree")
    return n.value


ND_SIGN_ZOLOTAREV, ND_SIGN_CHEBYSHEV = 0, 1


def dn_params(n_poles=16, eps=0.0, lambda_max=0.0, tol=1e-12, maxit=100000, inner_prec=ND_FP64, m_q=0.0,
              left_only=False, approx=ND_SIGN_ZOLOTAREV, degree=0):
    return nd_dn_params(int(n_poles), float(eps), float(lambda_max), float(tol), int(maxit), int(inner_prec),
                        float(m_q), int(left_only), int(approx), int(degree))


def nd_apply_sign(ctx, out, inp, params):
    info = nd_dn_info()
    _check(ctx, lib().nd_apply_sign(ctx, _ptr(_f64(out)), _ptr(_f64(inp)), ctypes.byref(params), ctypes.byref(info)),
           "nd_apply_sign")
    return info


def nd_apply_DN(ctx, out, inp, params):
    info = nd_dn_info()
    _check(ctx, lib().nd_apply_DN(ctx, _ptr(_f64(out)), _ptr(_f64(inp)), ctypes.byref(params), ctypes.byref(info)),
           "nd_apply_DN")
    return info


def nd_apply_DN_dagger(ctx, out, inp, params):
    """out = (D_N^m)^dagger inp = gamma5 D_N^m gamma5 inp (two-sided sign(Q) only)."""
    info = nd_dn_info()
    _check(ctx, lib().nd_apply_DN_dagger(ctx, _ptr(_f64(out)), _ptr(_f64(inp)), ctypes.byref(params),
                                         ctypes.byref(info)), "nd_apply_DN_dagger")
    return info


def nd_apply_Qhat(ctx, out, inp, prec):
    """out_e = Qhat in_e on internal fields of precision prec (even halves only)."""
    _check(ctx, lib().nd_apply_Qhat(ctx, _ptr(out), _ptr(inp), int(prec)), "nd_apply_Qhat")


def nd_solve_Q2_eo(ctx, x, b, tol=1e-10, maxit=100000, inner=ND_FP64):
    """x = (Q^2)^{-1} b via the even-odd Schur complement (canonical FP64 device tensors)."""
    info = nd_solve_info()
    _check(ctx, lib().nd_solve_Q2_eo(ctx, _ptr(_f64(x)), _ptr(_f64(b)), float(tol), int(maxit), int(inner),
                                     ctypes.byref(info)), "nd_solve_Q2_eo")
    return info


def nd_propagator(ctx, x, b, params, tol=1e-10, maxit=10000):
    """x = (D_N^m)^{-1} b (canonical FP64 device tensors); returns nd_prop_info."""
    info = nd_prop_info()
    _check(ctx, lib().nd_propagator(ctx, _ptr(_f64(x)), _ptr(_f64(b)), ctypes.byref(params), float(tol), int(maxit),
                                    ctypes.byref(info)), "nd_propagator")
    return info


def nd_force(ctx, F, phi, tol=1e-12, maxit=100000, inner=ND_FP64):
    info = nd_solve_info()
    _check(ctx, lib().nd_force(ctx, _ptr(F), _ptr(_f64(phi)), float(tol), int(maxit), int(inner), ctypes.byref(info)),
           "nd_force")
    return info


def nd_link_gradient(ctx, G, phi, tol=1e-12, maxit=100000, inner=ND_FP64, X=None):
    """Returns (S, info); G (complex128 [4, V, 3, 3] on cuda) receives dS/dU*, X (optional) receives
    (Q^2)^{-1} phi (see include/nd.h)."""
    info = nd_solve_info()
    S = ctypes.c_double()
    _check(ctx, lib().nd_link_gradient(ctx, _ptr(_f64(G)), _ptr(X if X is None else _f64(X)), ctypes.byref(S),
                                       _ptr(_f64(phi)), float(tol), int(maxit), int(inner), ctypes.byref(info)),
           "nd_link_gradient")
    return S.value, info


# ------------------------------------------------------------------ convenience object

class Lattice:
    """Owns one nd_ctx; holds links and hands out internal spinor buffers as torch tensors."""

    def __init__(self, dims, U=None, m=-1.4, s=0.4, antiperiodic_t=False, recon=(18, 18, 12)):
        import torch
        self.dims = tuple(int(d) for d in dims)
        self.m, self.s = m, s
        self.ctx = nd_create(self.dims, antiperiodic_t, m, s)
        self.V = nd_volume(self.ctx)
        if U is not None:
            self.set_links(U, recon)

    def set_links(self, U, recon=(18, 18, 12)):
        nd_set_links(self.ctx, U, recon)

    def field(self, prec, nrhs=1):
        import torch
        nbytes = nd_spinor_bytes(self.ctx, prec) * nrhs
        return torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def pack(self, canon, prec, nrhs=1):
        f = self.field(prec, nrhs)
        nd_pack_spinor(self.ctx, f, canon, prec, nrhs)
        return f

    def unpack(self, internal, prec, nrhs=1):
        import torch
        out = torch.empty((nrhs, self.V, 4, 3) if nrhs > 1 else (self.V, 4, 3), dtype=torch.complex128, device="cuda")
        nd_unpack_spinor(self.ctx, out, internal, prec, nrhs)
        return out

    # canonical FP64 [V][4][3] complex128 tensors in and out

    def Q(self, canon):
        import torch
        out = torch.empty_like(canon)
        nd_apply_Q_canonical(self.ctx, out, canon)
        return out

    def sign(self, eta, **params):
        """sign(Q) eta; params as dn_params (n_poles, eps, lambda_max, tol, maxit, inner_prec, ...)."""
        import torch
        out = torch.empty_like(eta)
        info = nd_apply_sign(self.ctx, out, eta, dn_params(**params))
        return out, info

    def DN(self, eta, **params):
        import torch
        out = torch.empty_like(eta)
        info = nd_apply_DN(self.ctx, out, eta, dn_params(**params))
        return out, info

    def propagator(self, b, tol=1e-10, maxit=10000, sign_tol=1e-12, **params):
        """(D_N^m)^{-1} b to relative residual tol; sign(Q) to sign_tol, other params as dn_params."""
        import torch
        x = torch.empty_like(b)
        info = nd_propagator(self.ctx, x, b, dn_params(tol=sign_tol, **params), tol, maxit)
        return x, info

    def lowmodes(self, l=None, tol=1e-12, maxit=100000, l_range=None, kappa=1e-6, method="filter"):
        """Fixed l (nd_lowmodes), or l chosen in l_range = (l_min, l_max) under a kappa target."""
        if l_range is None:
            return nd_lowmodes(self.ctx, l, tol, maxit)
        return nd_lowmodes_dynamic(self.ctx, l_range[0], l_range[1], kappa, maxit, method)

    def solve_Q2(self, b, tol=1e-10, maxit=100000, inner=ND_FP64, even_odd=False):
        """x = (Q^2)^{-1} b, whole lattice (nd_solve) or through the Schur complement."""
        import torch
        x = torch.empty_like(b)
        if even_odd:
            info = nd_solve_Q2_eo(self.ctx, x, b, tol, maxit, inner)
        else:
            info = nd_solve(self.ctx, [x], b, [0.0], tol, maxit, inner)
        return x, info

    def close(self):
        if getattr(self, "ctx", None):
            nd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
