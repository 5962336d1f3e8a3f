"""torch.autograd.Function for the pseudofermion action of the twisted-mass HMC.

S(omega) = phi^dag (D D^dag)^-1 phi = ||D[U(omega)]^-1 phi||^2, with the links rotated by
U_mu(x; omega) = exp(i sum_a omega_a(x, mu) lambda_a / 2) U0_mu(x)  (lambda_a: Gell-Mann matrices).

forward  loads U0, rotates it by omega (``tmg_rotate_gauge``, a kernel), brings the multigrid to the
         rotated field (a new setup, or the one-iteration setup update of Sec. 2) and runs ONE solve,
         Y = D^-1 phi, with S = ||Y||^2 (``tmg_pf_action``).  Only Y is kept for backward.
backward runs the adjoint solve X = D^-dag Y and the force kernels (``tmg_pf_force``): the HMC force
         f_a(x, mu) = tr(lambda_a / 2 F_mu(x)) is recomputed from the solution, never stored from the
         forward pass, and under ``torch.no_grad`` no adjoint solve runs at all.

The force is the left-invariant derivative at U(omega); it equals the partial derivative with
respect to omega exactly at omega = 0, where HMC evaluates it.  Backward uses the context's current
gauge field and multigrid, so it must run before the next forward on the same context (checked).

Only argument marshalling happens here: the rotation, the solves, the norm and the force all run in
the library's kernels.
"""
from __future__ import annotations

import torch

from . import Context  # noqa: F401


class PseudofermionAction(torch.autograd.Function):
    """S = PseudofermionAction.apply(omega, phi, ctx, U0, setup, tol).

    omega: float64 tensor [T, Z, Y, X, 4, 8] (CPU or CUDA); phi: complex128 numpy array or CUDA
    tensor [T, Z, Y, X, 4, 3]; ctx: a Context with operator parameters set; U0: complex128 links
    (numpy or CUDA tensor); setup: (v0, MGParams) for a new setup on the rotated field, or
    ("update", n_iter) to refine the context's existing setup by n_iter iterations; tol: solve
    tolerance.  Returns a 0-dim float64 tensor on omega's device.
    """

    @staticmethod
    def forward(fctx, omega, phi, ctx, U0, setup, tol):
        ctx.load_gauge(U0, -1)
        om = omega.detach()
        if om.is_cuda:
            ctx.rotate_gauge(om.contiguous())
        else:
            ctx.rotate_gauge(om.contiguous().numpy())
        if isinstance(setup[0], str) and setup[0] == "update":
            ctx.setup_update(int(setup[1]))
        else:
            ctx.setup(setup[0], setup[1])
        S, Y, _ = ctx.pf_action(phi, tol=tol)
        fctx.ctx, fctx.tol, fctx.version = ctx, tol, ctx.gauge_version
        fctx.Y = Y
        return torch.tensor(S, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(fctx, grad_out):
        ctx = fctx.ctx
        if ctx.gauge_version != fctx.version:
            raise RuntimeError("PseudofermionAction.backward: the context's gauge field changed after forward")
        f, _ = ctx.pf_force(fctx.Y, tol=fctx.tol)
        if not torch.is_tensor(f):
            f = torch.from_numpy(f)
        return grad_out * f.to(grad_out.device), None, None, None, None, None
