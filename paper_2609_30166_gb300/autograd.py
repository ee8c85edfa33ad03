"""Differentiable projector: torch.autograd around the CUDA projector.

forward  = the motion-aware ray-driven projector (Sec. 4.1 with the Sec. 2.2.2
           pose and Sec. 3.1 warp), ``ctrex_fwd_project``;
backward = the matched adjoint (exact transpose, FP32 atomics) for the
           volume and the chain rule through the warp for the motion
           parameters, ``ctrex_adjoint_project`` / ``ctrex_motion_grad``.
The deformation is recomputed in the backward kernels, never stored.  The
paper motivates geometry refinement / self-calibration (Sec. 5); it prints no
gradient, so these are the exact derivatives of its projector.
"""

from __future__ import annotations

import torch

from . import ctrex


class Projector:
    """A projector with fixed geometry and a differentiable volume, pose and
    deformation.  ``s_view`` (time scale of the deformation per view) and the
    clip-box ``margin`` (mm) are fixed; theta [V, 15] and coef [8, 8, 8, 3]
    are arguments of each call."""

    def __init__(self, cfg, P=None, s_view=None, margin=None, device=None):
        self.cfg = cfg
        self.ctx = ctrex.context_for(cfg, P=P, device=device)
        dev = self.ctx.device
        if s_view is None:
            s_view = torch.arange(cfg.n_views, dtype=torch.float32, device=dev) / max(cfg.n_views - 1, 1)
        self.s_view = torch.as_tensor(s_view, dtype=torch.float32, device=dev).contiguous()
        self.margin = float(cfg.margin if margin is None else margin)

    def _set(self, theta, coef):
        self.ctx.set_motion(theta.detach().float().contiguous(), coef.detach().float().contiguous(), self.s_view,
                            self.margin)

    def __call__(self, vol, theta, coef):
        return _Project.apply(vol, theta, coef, self)


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(actx, vol, theta, coef, proj):
        proj._set(theta, coef)
        out = proj.ctx.fwd_project(vol.detach().float().contiguous())
        actx.save_for_backward(vol, theta, coef)
        actx.proj = proj
        return out

    @staticmethod
    def backward(actx, g):
        vol, theta, coef = actx.saved_tensors
        proj = actx.proj
        proj._set(theta, coef)  # recompute the warp of these parameters
        g = g.detach().float().contiguous()
        gvol = gth = gco = None
        if actx.needs_input_grad[0]:
            gvol = proj.ctx.adjoint_project(g).to(vol.dtype)
        if actx.needs_input_grad[1] or actx.needs_input_grad[2]:
            gth, gco = proj.ctx.motion_grad(vol.detach().float().contiguous(), g,
                                            want_theta=actx.needs_input_grad[1],
                                            want_coef=actx.needs_input_grad[2])
        return gvol, gth, gco, None
