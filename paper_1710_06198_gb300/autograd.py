"""torch.autograd.Function for the pseudofermion action of the twisted-mass HMC.

S(omega) = phi^dag (D D^dag)^-1 phi = ||D[U(omega)]^-1 phi||^2, with the links rotated by
U_mu(x; omega) = exp(i sum_a omega_a(x, mu) lambda_a / 2) U0_mu(x)  (lambda_a: Gell-Mann matrices).

forward  runs the two multigrid solves and the force kernel of libtmg (``tmg_force``);
backward returns dS/domega_a(x, mu) = tr(lambda_a / 2 F_mu(x)) times grad_output, i.e. the HMC
force on the links.  The force is the left-invariant derivative at U(omega); it equals the partial
derivative with respect to omega exactly at omega = 0, where HMC evaluates it.  The force is not
stored from an earlier trajectory: it is recomputed from the solutions of this forward pass.

Only argument marshalling happens here; the solves and the force run in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Context, PREC_F32, PREC_F64  # noqa: F401


def _gell_mann_halves():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return 0.5 * l


_T = _gell_mann_halves()


def rotate_links(U0, omega):
    """exp(i omega . lambda / 2) U0 (host numpy, input preparation)."""
    H = np.einsum("...a,aij->...ij", omega, _T)
    w, v = np.linalg.eigh(H)
    E = np.einsum("...ab,...b,...cb->...ac", v, np.exp(1j * w), np.conj(v))
    return np.einsum("...ab,...bc->...ac", E, U0)


class PseudofermionAction(torch.autograd.Function):
    """S = PseudofermionAction.apply(omega, phi, ctx, U0, setup, tol).

    omega: float64 tensor [T, Z, Y, X, 4, 8]; phi: complex128 numpy array or CUDA tensor
    [T, Z, Y, X, 4, 3]; ctx: a Context with operator parameters set; U0: complex128 numpy links;
    setup: (v0, MGParams) used to (re)build the multigrid for the rotated field; tol: solve
    tolerance.  Returns a 0-dim float64 tensor on omega's device.
    """

    @staticmethod
    def forward(fctx, omega, phi, ctx, U0, setup, tol):
        om = omega.detach().cpu().numpy()
        U = U0 if not np.any(om) else rotate_links(U0, om)
        ctx.load_gauge(np.ascontiguousarray(U), -1)
        ctx.setup(setup[0], setup[1])
        S, F, _ = ctx.force(phi, tol=tol)
        if hasattr(F, "cpu"):
            F = F.cpu().numpy()
        f = np.real(np.einsum("aij,...ji->...a", _T, F))
        fctx.save_for_backward(torch.from_numpy(np.ascontiguousarray(f)).to(omega.device))
        return torch.tensor(S, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(fctx, grad_out):
        (f,) = fctx.saved_tensors
        return grad_out * f, None, None, None, None, None
