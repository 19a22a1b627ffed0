"""The fermion action and its gauge-link gradient as a torch.autograd.Function.

    S(U) = phi^dag (D(mu)^dag D(mu))^-1 phi

The gradient comes from the library's own adjoint computation (overlap_force: every
Zolotarev pole's shifted solutions and the link outer products of the Wilson hop, on the
GPU); this module only moves tensors. PyTorch's convention for a real loss L of a
complex tensor z is dL = Re(sum conj(z.grad) dz); the library returns G with
dS = 2 Re(sum conj(G) dU), so z.grad = 2 G.

The library copies the links when the context is created, so the action and its
gradient are those of that gauge field: forward() compares U with it (a digest of the
canonical complex128 bytes) and raises ValueError when they differ, rather than return
the action of other links. phi is treated as a constant (no gradient).
"""
import numpy as np
import torch

from .binding import links_digest


class OverlapAction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, U, phi, ovl, mu, tol):
        if links_digest(U.detach().contiguous().cpu().numpy()) != ovl.links_digest:
            raise ValueError("U differs from the gauge field the overlap context was created from; "
                             "create a context from these links to differentiate at them")
        ph = phi.detach()
        if ph.is_cuda:
            ph = ph.contiguous()
        else:
            ph = np.ascontiguousarray(ph.numpy())
        G, S = ovl.force(ph, mu=mu, tol=tol)
        fctx.save_for_backward(torch.from_numpy(np.ascontiguousarray(G)).to(U.device))
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, gS):
        (G,) = fctx.saved_tensors
        return 2.0 * gS * G, None, None, None, None


def overlap_action(U, phi, ovl, mu=None, tol=1e-10):
    """S = phi^dag (D^dag D)^-1 phi at mass mu (default: the context's), differentiable
    in the gauge links U (complex128, canonical [t][z][y][x][mu][row][col] layout)."""
    if U.dtype != torch.complex128:
        raise TypeError("U must be complex128")
    return OverlapAction.apply(U, phi, ovl, ovl.mu if mu is None else mu, tol)
