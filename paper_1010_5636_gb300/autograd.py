"""torch.autograd.Function wrappers of the library's differentiable operations.

Argument marshalling only: the forward and backward passes call the C-ABI (nd_link_gradient,
nd_apply_DN), all arithmetic runs in the library's kernels.

* ``pseudofermion_action(lat, U, phi)`` -> S = phi^dagger (Q^2)^{-1} phi as a real 0-d tensor,
  differentiable in the links U (complex [4, V, 3, 3], treated as general complex matrices) and
  in phi.  One solve in the forward pass yields S, dS/dU* and dS/dphi* = (Q^2)^{-1} phi; the
  backward pass only scales them (by 2 grad_output: torch's gradient of a real function of a
  complex tensor is twice the conjugate Wirtinger derivative).  Any parametrisation of U written in torch (for example
  U = matrix_exp(i omega.T) @ U0) is differentiated through by torch, so dS/domega at omega = 0
  is the su(3) force of nd_force.
* ``dirac_overlap(lat, eta, params)`` -> D_N eta (Sec. 2.2), differentiable in the source: the
  vector-Jacobian product is D_N^dagger g = gamma5 D_N gamma5 g (nd_apply_DN_dagger), exact for the
  two-sided deflated sign (hermitian); the multi-shift solves are recomputed rather than stored.
"""
import torch

from . import ND_FP64, dn_params, nd_apply_DN, nd_apply_DN_dagger, nd_link_gradient, nd_set_links

__all__ = ["pseudofermion_action", "dirac_overlap", "PseudofermionAction", "DiracOverlap"]


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, lat, tol, inner, recon):
        U = U.detach().contiguous()
        phi = phi.detach().contiguous()
        nd_set_links(lat.ctx, U, recon)
        G = torch.empty_like(U)
        X = torch.empty_like(phi)
        S, _ = nd_link_gradient(lat.ctx, G, phi, tol, 1000000, inner, X=X)
        ctx.save_for_backward(G, X)
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gS):
        # torch's gradient of a real function of a complex tensor is twice the conjugate
        # Wirtinger derivative (dS = Re sum conj(grad) dz); the library returns the derivative itself
        G, X = ctx.saved_tensors
        gU = 2.0 * G * gS if ctx.needs_input_grad[0] else None
        gphi = 2.0 * X * gS if ctx.needs_input_grad[1] else None
        return gU, gphi, None, None, None, None


def pseudofermion_action(lat, U, phi, tol=1e-12, inner=ND_FP64, recon=(18, 12, 12)):
    return PseudofermionAction.apply(U, phi, lat, float(tol), int(inner), tuple(recon))


class DiracOverlap(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eta, lat, params):
        eta = eta.detach().contiguous()
        out = torch.empty_like(eta)
        nd_apply_DN(lat.ctx, out, eta, params)
        ctx.lat, ctx.params = lat, params
        return out

    @staticmethod
    def backward(ctx, g):
        out = torch.empty_like(g)
        nd_apply_DN_dagger(ctx.lat.ctx, out, g.contiguous(), ctx.params)
        return out, None, None


def dirac_overlap(lat, eta, params=None):
    return DiracOverlap.apply(eta, lat, params if params is not None else dn_params())
