"""T(E) as a differentiable function of the local potential.

``transmission(ctx, v_loc, energies, cols, opts)`` returns T(E) (Eq.
T-realspace, coupling 2*CAP) as a torch tensor whose gradient with respect to
``v_loc`` is

    dT(E)/dV_loc(r) = 8 sum_j Gamma_R,j Re( lambda_j(r) x_j(r) ),
    lambda_j = G(E) (Gamma_L o conj(x_j)),

one adjoint solve per column with the same operator (G^T = G, Eq.
complex-sym).  The forward pass keeps the forward columns x_j on the device
(``rsn_transmission_keep``) when they fit in ``keep_bytes`` (default: a
quarter of the free device memory), and the backward pass then solves only the
adjoints from them (``rsn_transmission_vjp_reuse``): two solves per column in
all.  Columns that do not fit are not kept; the backward pass then calls
``rsn_transmission_vjp``, which solves the forward columns again with their
adjoints (memory O(slots * N) instead of O(columns * N)).

The autograd machinery only marshals arguments: every solve, reduction and
gradient accumulation runs in the CUDA library.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch

from . import binding as B


class TransmissionFn(torch.autograd.Function):
    """T(E) for a 1-D tensor of N potential values (any device, float64)."""

    @staticmethod
    def forward(ctx, v_loc: torch.Tensor, energies: Sequence[float], cols: np.ndarray, context: "B.Context",
                opts: Optional[B.SolverOpts], keep_bytes: Optional[int]):
        v = v_loc.detach().to("cpu", torch.float64).contiguous().numpy()
        context.set_potential(v)
        E = np.asarray(energies, dtype=np.float64)
        need = E.size * cols.size * context.N * 16
        if keep_bytes is None:
            free, _ = torch.cuda.mem_get_info(context.device)
            keep_bytes = free // 4
        if need <= keep_bytes:
            T, x = context.transmission_keep(E, cols, opts)
        else:
            T, x = context.transmission(E, cols, opts), None
        ctx.context = context
        ctx.energies = E
        ctx.cols = cols
        ctx.opts = opts
        ctx.v = v
        ctx.x = x
        ctx.dev = v_loc.device
        return torch.tensor(T, dtype=torch.float64, device=v_loc.device)

    @staticmethod
    def backward(ctx, grad_T: torch.Tensor):
        context = ctx.context
        context.set_potential(ctx.v)  # the potential of this forward pass
        T_bar = grad_T.detach().to("cpu", torch.float64).numpy()
        on_dev = ctx.dev.type == "cuda"
        dV = torch.empty(ctx.v.size, dtype=torch.float64, device=ctx.dev) if on_dev else None
        if ctx.x is not None:
            dv = context.transmission_vjp_reuse(ctx.energies, T_bar, ctx.cols, ctx.x, ctx.opts, dV_out=dV)
            ctx.x = None
        else:
            _, dv = context.transmission_vjp(ctx.energies, T_bar, ctx.cols, ctx.opts, dV_out=dV)
        if not on_dev:
            dV = torch.from_numpy(dv)
        return dV, None, None, None, None, None


def transmission(context: "B.Context", v_loc: torch.Tensor, energies: Sequence[float],
                 cols: Optional[Sequence[int]] = None, opts: Optional[B.SolverOpts] = None,
                 keep_bytes: Optional[int] = None) -> torch.Tensor:
    """Differentiable T(E); ``context`` must hold the junction (``set_junction``).

    ``keep_bytes``: device memory the forward columns may occupy between the
    forward and the backward pass (0: never keep them)."""
    if cols is None:
        cols = context.junction.right_columns()
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    return TransmissionFn.apply(v_loc, list(energies), cols, context, opts, keep_bytes)
