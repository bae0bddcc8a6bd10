"""Low modes of the oracle: lowest eigenpairs of Q^2, Rayleigh-Ritz of Q, residues, kappa_+-.

Test infrastructure only.  Follows Sec. 2.3 (low-mode projection):
  V = span of l approximate eigenvectors, P its orthonormal projector;
  u_k in V with P Q u_k = nu_k u_k (Rayleigh-Ritz of Q on V);
  P_+ = sum_{nu_k > 0} u_k u_k^dagger,  P_- = sum_{nu_k < 0} u_k u_k^dagger;
  rho_k = ||(Q - nu_k) u_k||;
  kappa_+-^2 = sum_{+-nu_k > 0} rho_k^2 / d_k^2,
  ||P_+- - (P_+-)_exact|| <= kappa (1 + 2 kappa) / (1 - 2 kappa (1 + 2 kappa)).
The paper finds V by minimising the Ritz functional of Q^2; the oracle takes V from a
dense eigendecomposition (small lattices) or from ARPACK (scipy eigsh) on Q^2.

Reading of d_k (the paper defines it as the distance of nu_k from the exact spectrum of Q
on the complement of the exact projector of nu_k's sign, and gives no estimator): the
nearest point of that spectrum is either a mode of the opposite sign, whose smallest
magnitude is estimated by the opposite-sign nu_j in V (or by sqrt(lambda_{l+1}) if there
is none), or the first same-sign mode outside V, whose magnitude is at least
sqrt(lambda_{l+1}(Q^2)).  So d_k = min(|nu_k| + m_opp, sqrt(lambda_{l+1}) - |nu_k|).
"""
import numpy as np

from . import wilson


def rayleigh_ritz(apply_Q, basis):
    """Orthonormalise the basis [l, ...] (QR), then diagonalise M_ij = u_i^dagger Q u_j.

    Returns (nu ascending by |nu|, u [l, ...], rho)."""
    l = basis.shape[0]
    shape = basis.shape[1:]
    B = basis.reshape(l, -1).T
    q, _ = np.linalg.qr(B)
    QB = np.stack([apply_Q(q[:, k].reshape(shape)).reshape(-1) for k in range(l)], axis=1)
    M = q.conj().T @ QB
    M = 0.5 * (M + M.conj().T)
    nu, W = np.linalg.eigh(M)
    order = np.argsort(np.abs(nu), kind="stable")
    nu, W = nu[order], W[:, order]
    u = (q @ W).T
    QU = (QB @ W).T
    rho = np.linalg.norm(QU - nu[:, None] * u, axis=1)
    return nu, u.reshape((l,) + shape), rho


def spectral_distances(nu, lam_next):
    """d_k per the reading in the module docstring."""
    nu = np.asarray(nu, dtype=np.float64)
    top = np.sqrt(lam_next)
    d = np.empty_like(nu)
    for k, v in enumerate(nu):
        opp = np.abs(nu[np.sign(nu) != np.sign(v)])
        m_opp = opp.min() if opp.size else top
        d[k] = min(abs(v) + m_opp, top - abs(v))
    return d


def kappas(nu, rho, d):
    nu, rho, d = map(np.asarray, (nu, rho, d))
    kp = np.sqrt(np.sum((rho[nu > 0] / d[nu > 0]) ** 2))
    km = np.sqrt(np.sum((rho[nu < 0] / d[nu < 0]) ** 2))
    return float(kp), float(km)


def projector_bound(kappa):
    """Right-hand side of the projector-deviation inequality of Sec. 2.3."""
    k = kappa * (1 + 2 * kappa)
    return k / (1 - 2 * k) if 2 * k < 1 else np.inf


def lowmodes_dense(U, dims, m, l, antiperiodic_t=False):
    """Exact low modes from the dense matrix of Q (small lattices): the l eigenpairs of Q with
    the smallest |nu| (the l lowest modes of Q^2), plus lambda_{l+1}(Q^2) and lambda_max(Q^2)."""
    Qm = wilson.dense_Q(U, dims, m, antiperiodic_t)
    w, v = np.linalg.eigh(Qm)
    order = np.argsort(np.abs(w), kind="stable")
    V = int(np.prod(dims))
    nu = w[order[:l]]
    u = v[:, order[:l]].T.reshape(l, V, 4, 3)
    return {
        "nu": nu,
        "u": np.ascontiguousarray(u),
        "rho": np.zeros(l),
        "eval_Q2": w[order[: l + 1]] ** 2,
        "lam_next": float(w[order[l]] ** 2),
        "lam_max": float(np.max(w ** 2)),
        "spectrum": w,
        "eigvecs": v,
    }


def lowmodes_arpack(U, dims, m, l, antiperiodic_t=False, tol=1e-12):
    """Low modes by ARPACK (scipy eigsh, which='SA') on Q^2, then Rayleigh-Ritz of Q."""
    import scipy.sparse.linalg as sla
    V = int(np.prod(dims))
    n = 12 * V
    shape = (V, 4, 3)

    def q2(v):
        return wilson.apply_Q2(U, np.ascontiguousarray(v.reshape(shape)), dims, m, antiperiodic_t).reshape(-1)

    op = sla.LinearOperator((n, n), matvec=q2, dtype=np.complex128)
    w, vec = sla.eigsh(op, k=l + 1, which="SA", tol=tol)
    order = np.argsort(w)
    w, vec = w[order], vec[:, order]
    lam_max = sla.eigsh(op, k=1, which="LA", tol=1e-8, return_eigenvectors=False)[0]
    basis = vec[:, :l].T.reshape((l,) + shape)
    nu, u, rho = rayleigh_ritz(lambda x: wilson.apply_Q(U, np.ascontiguousarray(x), dims, m, antiperiodic_t), basis)
    return {"nu": nu, "u": u, "rho": rho, "eval_Q2": w, "lam_next": float(w[l]), "lam_max": float(lam_max)}


def lambda_max_arpack(U, dims, m, antiperiodic_t=False, tol=1e-8):
    """Largest eigenvalue of Q^2 by ARPACK (scipy eigsh, which='LA') on the oracle's Q^2; the
    upper end of the interval that X = Q / sqrt(lambda_max) is scaled to (Sec. 2.2)."""
    import scipy.sparse.linalg as sla
    V = int(np.prod(dims))
    n = 12 * V
    shape = (V, 4, 3)

    def q2(v):
        return wilson.apply_Q2(U, np.ascontiguousarray(v.reshape(shape)), dims, m, antiperiodic_t).reshape(-1)

    op = sla.LinearOperator((n, n), matvec=q2, dtype=np.complex128)
    return float(sla.eigsh(op, k=1, which="LA", tol=tol, return_eigenvectors=False)[0])


def choose_l(evals_q2, l_min, l_max):
    """Number of low modes to deflate (Sec. 2.3: l is chosen at run time so that the kept modes are
    well separated from the rest of the spectrum).  Reading: among l_min <= l <= l_max take the
    l with the largest relative gap between the last kept and the first remaining mode of Q,
        g_l = (sqrt(lambda_{l+1}) - sqrt(lambda_l)) / sqrt(lambda_{l+1}),
    lambda_1 <= lambda_2 <= ... the eigenvalues of Q^2; the smallest such l on ties."""
    e = np.sqrt(np.asarray(evals_q2, dtype=np.float64))
    if not (1 <= l_min <= l_max < len(e)):
        raise ValueError("need 1 <= l_min <= l_max < len(evals)")
    best, best_g = l_min, -1.0
    for l in range(l_min, l_max + 1):
        g = (e[l] - e[l - 1]) / e[l]
        if g > best_g:
            best, best_g = l, g
    return best
