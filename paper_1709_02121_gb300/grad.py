"""dT/dtheta of the transmission as a torch.autograd.Function.

``transmission(H, w, wl, steps)`` returns the transmission estimates T(H_i,
w_i) of a batch of 2D Gaussian-barrier problems (one instance per parameter
point, workload ``wl`` for everything else) after ``steps`` intervals, and
is differentiable in H and w.  The forward pass runs the batch without
tangents.  The backward pass replays the same run in tangent mode: the
counter-based random streams make the replay's signed particles, counts and
T identical to the forward's (checked), while every particle also carries
its likelihood-ratio tangent weight, so the replay yields dT/dH and dT/dw
(wbrw_transmission_gradients).  The forward state is thus "checkpointed" as
the seed and the parameters, and recomputed; every resampling of the replay
is a checkpoint of the histogram the forward pass produced.

All the work runs in the library's CUDA kernels; torch holds the buffers.
"""
from __future__ import annotations

import numpy as np

from .wbrw import Batch


def _instances(wl, H, w):
    return [dict(H=float(h), w=float(v), xc=wl.get("xc", 0.0), x0=wl["x0"],
                 sigma_x=wl["sigma_x"], k0=wl["k0"], n_init=int(wl["n_alpha"]),
                 n_alpha=int(wl["n_alpha"]), gamma0=wl.get("gamma0", 0.0))
            for h, v in zip(H, w)]


def run_batch(wl, H, w, steps, tangent, capacity, stream=None):
    """Run the batch; returns (T per instance, gradients or None, counters)."""
    spec = dict(wl, tangent=bool(tangent))
    b = Batch(spec, _instances(spec, H, w), capacity, stream=stream)
    try:
        b.run(steps)
        T = b.transmissions()
        g = b.transmission_gradients() if tangent else None
        if g is not None and g.ndim == 1:
            g = g[None, :]
        return T, g, b.counters()
    finally:
        b.close()


def _autograd():
    import torch

    class TransmissionLR(torch.autograd.Function):
        @staticmethod
        def forward(ctx, H, w, wl, steps, capacity):
            h = H.detach().cpu().numpy().astype(np.float64)
            v = w.detach().cpu().numpy().astype(np.float64)
            T, _, _ = run_batch(wl, h, v, steps, False, capacity)
            ctx.wl, ctx.steps, ctx.capacity = wl, steps, capacity
            ctx.T = T
            ctx.save_for_backward(H, w)
            return torch.as_tensor(T, dtype=H.dtype, device=H.device)

        @staticmethod
        def backward(ctx, grad_T):
            H, w = ctx.saved_tensors
            h = H.detach().cpu().numpy().astype(np.float64)
            v = w.detach().cpu().numpy().astype(np.float64)
            T, g, _ = run_batch(ctx.wl, h, v, ctx.steps, True, ctx.capacity)
            if not np.array_equal(T, ctx.T):
                raise RuntimeError("the tangent replay did not reproduce the forward run")
            gT = grad_T.detach().to("cpu", torch.float64).numpy()
            dH = torch.as_tensor(gT * g[:, 0], dtype=H.dtype, device=H.device)
            dw = torch.as_tensor(gT * g[:, 1], dtype=w.dtype, device=w.device)
            return dH, dw, None, None, None

    return TransmissionLR


_FN = None


def transmission(H, w, wl: dict, steps: int, capacity: int):
    """Differentiable T(H, w) (torch tensors of shape (n,)); see the module."""
    global _FN
    if _FN is None:
        _FN = _autograd()
    return _FN.apply(H, w, wl, steps, capacity)
