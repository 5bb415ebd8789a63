"""torch.autograd wrappers over the hand-written forward and adjoint kernels.

``render(params, cam, twist)`` rasterises the Gaussians (Eq. 1-7) from the
pose exp(twist^) T_cw and returns (rgb, depth, opacity); its backward calls
``gl_rasterize_backward``, which recomputes per-pixel transmittance from the
stored final value and returns gradients for every Gaussian attribute and
dL/dtwist, the derivative w.r.t. the twist itself (the library applies the
SE(3) left Jacobian at the twist), so a caller may keep optimising the twist
without resetting it to zero.

``photometric_loss(rgb, target, E)`` is Eq. 9 (L1 + D-SSIM after the 3x4
exposure E) with its analytic adjoint for rgb and E.

Both only marshal tensors to the C ABI; all arithmetic, the pose's included,
runs in the library.
"""
from __future__ import annotations

import torch

from . import binding

PARAM_NAMES = ("means", "log_scales", "quats", "logits", "sh")


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cam, tile, glctx, twist, means, log_scales, quats, logits, sh):
        params = dict(means=means.contiguous(), log_scales=log_scales.contiguous(), quats=quats.contiguous(),
                      logits=logits.contiguous(), sh=sh.contiguous())
        rgb, depth, opac = glctx.forward(params, cam, tile, twist=twist.detach().cpu().tolist())
        ctx.glctx = glctx
        ctx.params = params
        ctx.shape = rgb.shape
        return rgb, depth, opac

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_opac):
        p = ctx.params
        dC = g_rgb.contiguous() if g_rgb is not None else p["means"].new_zeros(ctx.shape)
        dD = g_depth.contiguous() if g_depth is not None else None
        dO = g_opac.contiguous() if g_opac is not None else None
        grads, pose = ctx.glctx.backward(p, dC, dD, dO, pose_grad=True)
        return (None, None, None, pose) + tuple(grads[k] for k in PARAM_NAMES)


def render(params: dict, cam: dict, twist: torch.Tensor | None = None, tile: int = 16,
           glctx: binding.Ctx | None = None):
    """Differentiable render: returns (rgb H x W x 3, depth H x W, opacity H x W)."""
    glctx = glctx if glctx is not None else binding.Ctx()
    if twist is None:
        twist = torch.zeros(6, device=params["means"].device, requires_grad=False)
    return _Rasterize.apply(cam, tile, glctx, twist, *(params[k] for k in PARAM_NAMES))


class _PhotometricLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, glctx, lam, rgb, target, E):
        loss, dC, dE = glctx.loss(rgb.contiguous(), target.contiguous(), E.reshape(12).contiguous(), lam)
        ctx.save_for_backward(dC, dE)
        return loss.reshape(())

    @staticmethod
    def backward(ctx, g):
        dC, dE = ctx.saved_tensors
        return None, None, dC * g, None, (dE * g).reshape(3, 4)


def photometric_loss(rgb, target, E, lam: float = 0.2, glctx: binding.Ctx | None = None):
    """Eq. 9 with exposure E (3 x 4); differentiable in rgb and E."""
    glctx = glctx if glctx is not None else binding.Ctx()
    return _PhotometricLoss.apply(glctx, lam, rgb, target, E)
