"""torch.autograd interface of the adjoint kernels.

``replica_averaged_run(params, ...)`` runs replica-averaged Brownian dynamics
on the GPU and returns the replica-averaged spring force (RSF) of every
completed window and the Bell log-survival of each chain under the RSF
criterion, as differentiable functions of each chain's (strain rate, FENE b,
spring constant H). Its backward pass is ``bd_adjoint``: pathwise derivatives
with the noise held fixed, parent checkpoints every K steps. Everything here
is argument marshalling; the forward and backward work runs in the library's
kernels, on torch's current CUDA stream.

Device memory. The run's context (state, histories, parent checkpoints and,
after the first backward, the adjoint's replay buffers: about 24 GB for 256
chains of 200 beads) is held by the autograd graph only until its backward
pass, which releases it, the way autograd frees saved tensors. A second
backward through the same graph then raises; set ``RunSpec.retain_run`` to
keep the context for repeated backward passes (it is then released with the
graph). ``release_run(output)`` frees it early without a backward pass.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import bdra
from .inputs import CRIT_RSF

EVENT_BYTES = 24          # sizeof(bd_event)


@dataclasses.dataclass
class RunSpec:
    """The non-differentiable arguments of a run."""

    chains: Sequence            # chain records (inputs.Chain); rate, b, H come from params
    dt: float
    window_steps: int
    n_steps: int
    seed: int
    init_pos: np.ndarray        # [sum N][3] float64
    checkpoint_steps: int
    precision: int = bdra.BD_PREC_FP32
    s_min: float = 1e-3
    flags: int = 0
    retain_run: bool = False    # keep the device context after backward (repeated backward passes)


class _ReplicaAveragedRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, spec: RunSpec):
        p = params.detach().to("cpu", torch.float64).numpy()
        chains = [dataclasses.replace(c, rate=float(p[i, 0]), b=float(p[i, 1]), H=float(p[i, 2]))
                  for i, c in enumerate(spec.chains)]
        dev = torch.device("cuda", torch.cuda.current_device())
        stream = torch.cuda.current_stream(dev).cuda_stream
        W = spec.n_steps // spec.window_steps
        run = bdra.Context(chains, spec.dt, spec.window_steps, spec.seed, spec.init_pos,
                           precision=spec.precision, max_windows=max(W, 1),
                           bell_mask=CRIT_RSF, flags=spec.flags, s_min=spec.s_min,
                           stream=stream, checkpoint_steps=spec.checkpoint_steps)
        run.step(spec.n_steps)
        rsf = torch.empty((W, run.M), dtype=torch.float64, device=dev)
        for w in range(W):
            bdra.bd_replica_average(run.ptr, w, rsf[w])
        ev = torch.empty(6 * run.M * EVENT_BYTES, dtype=torch.uint8, device=dev)
        ls = torch.empty((len(chains), 3), dtype=torch.float64, device=dev)
        bdra.bd_detect_events(run.ptr, ev, 6 * run.M, ls)
        ctx.run = run
        ctx.retain_run = spec.retain_run
        ctx.n_windows = W
        ctx.param_device, ctx.param_dtype = params.device, params.dtype
        return rsf, ls[:, 2].contiguous()

    @staticmethod
    def backward(ctx, g_rsf: Optional[torch.Tensor], g_ls: Optional[torch.Tensor]):
        run = ctx.run
        if run is None or not run.ptr:
            raise RuntimeError("the run's device context was released after its first backward pass "
                               "(or by release_run); set RunSpec.retain_run for repeated backward passes")
        dev = torch.device("cuda", torch.cuda.current_device())
        C = len(run.chains)
        gr = None if g_rsf is None else g_rsf.to(dev, torch.float64).contiguous()
        gl = None if g_ls is None else g_ls.to(dev, torch.float64).contiguous()
        out = torch.empty((C, 3), dtype=torch.float64, device=dev)
        bdra.bd_adjoint(run.ptr, C, run.M, ctx.n_windows, gr, gl, out)
        grad = out.to(ctx.param_device, ctx.param_dtype)
        if not ctx.retain_run:
            # bd_destroy synchronises the context's stream before it frees
            run.close()
            ctx.run = None
        return grad, None


def replica_averaged_run(params: torch.Tensor, spec: RunSpec):
    """(rsf [windows][M], log_survival [n_chains]) of a run whose chains take
    (rate, b, H) = params[c] (a [n_chains][3] tensor); differentiable in
    params through the adjoint kernels."""
    if params.shape != (len(spec.chains), 3):
        raise ValueError(f"params must be [{len(spec.chains)}][3]")
    if spec.checkpoint_steps <= 0:
        raise ValueError("checkpoint_steps must be > 0 for the backward pass")
    return _ReplicaAveragedRun.apply(params, spec)


def release_run(output: torch.Tensor) -> None:
    """Free the device context behind an output of replica_averaged_run now
    (for outputs that will not be differentiated)."""
    node = output.grad_fn
    run = getattr(node, "run", None) if node is not None else None
    if run is not None:
        run.close()
        node.run = None


def chain_params(chains: Sequence) -> torch.Tensor:
    """[n_chains][3] float64 tensor of (rate, b, H)."""
    return torch.tensor([[c.rate, c.b, c.H] for c in chains], dtype=torch.float64)
