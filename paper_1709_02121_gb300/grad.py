"""dT/dtheta of the transmission as a torch.autograd.Function.

``transmission(H, w, wl, steps)`` returns the transmission estimates T(H_i,
w_i) of a batch of 2D Gaussian-barrier problems (one instance per parameter
point, workload ``wl`` for everything else) after ``steps`` intervals, and
is differentiable in H and w.

The tangent mode carries every particle's likelihood-ratio tangent weight
alongside its sign and yields dT/dH and dT/dw with T
(wbrw_transmission_gradients); its signed particles, counts and T are those
of the run without tangents (the counter-based random streams do not depend
on the tangents).  Two schedules:
  - one pass (default): when H or w requires a gradient, the forward pass
    runs in tangent mode and keeps the gradients; backward scales them.
    Value and gradient cost one tangent run.
  - replay (``replay=True``): the forward pass runs without tangents and the
    backward pass replays the same run in tangent mode (checked to give the
    same T).  The forward state is "checkpointed" as the seed and the
    parameters and recomputed, every resampling of the replay being a
    checkpoint of the histogram the forward pass produced: nothing is kept
    between the passes but T, at the cost of a second run.

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
        def forward(ctx, H, w, wl, steps, capacity, one_pass):
            h = H.detach().cpu().numpy().astype(np.float64)
            v = w.detach().cpu().numpy().astype(np.float64)
            T, g, _ = run_batch(wl, h, v, steps, one_pass, capacity)
            ctx.wl, ctx.steps, ctx.capacity = wl, steps, capacity
            ctx.T, ctx.g = T, g
            ctx.save_for_backward(H, w)
            return torch.as_tensor(T, dtype=H.dtype, device=H.device)

        @staticmethod
        def backward(ctx, grad_T):
            H, w = ctx.saved_tensors
            g = ctx.g
            if g is None:  # replay the forward run in tangent mode
                h = H.detach().cpu().numpy().astype(np.float64)
                v = w.detach().cpu().numpy().astype(np.float64)
                T, g, _ = run_batch(ctx.wl, h, v, ctx.steps, True, ctx.capacity)
                if not np.array_equal(T, ctx.T):
                    raise RuntimeError("the tangent replay did not reproduce the forward run")
            gT = grad_T.detach().to("cpu", torch.float64).numpy()
            dH = torch.as_tensor(gT * g[:, 0], dtype=H.dtype, device=H.device)
            dw = torch.as_tensor(gT * g[:, 1], dtype=w.dtype, device=w.device)
            return dH, dw, None, None, None, None

    return TransmissionLR


_FN = None


def transmission(H, w, wl: dict, steps: int, capacity: int, replay: bool = False):
    """Differentiable T(H, w) (torch tensors of shape (n,)); see the module
    for the one-pass and the replay schedules."""
    import torch
    global _FN
    if _FN is None:
        _FN = _autograd()
    one_pass = (not replay and torch.is_grad_enabled()
                and (H.requires_grad or w.requires_grad))
    return _FN.apply(H, w, wl, steps, capacity, one_pass)
