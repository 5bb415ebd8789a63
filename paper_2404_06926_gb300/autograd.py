"""torch.autograd wrappers over the hand-written forward and adjoint kernels.

``render(params, twist, cam)`` rasterises the Gaussians (Eq. 1-7) and returns
(rgb, depth, opacity); its backward calls ``gl_rasterize_backward``, which
recomputes per-pixel transmittance from the stored final value and returns
gradients for every Gaussian attribute and for a left twist xi = (rho, phi)
of the camera pose, T_cw <- exp(xi^) T_cw.  The forward applies exp(xi^) to
the pose given in ``cam``; the returned pose gradient is the derivative at the
current (perturbed) pose, the usual convention for optimising a pose on SE(3)
by left perturbations.

``photometric_loss(rgb, target, E)`` is Eq. 9 (L1 + D-SSIM after the 3x4
exposure E) with its analytic adjoint for rgb and E.

Both only marshal tensors to the C ABI; all arithmetic runs in the library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding

PARAM_NAMES = ("means", "log_scales", "quats", "logits", "sh")


def se3_exp(xi: np.ndarray):
    """exp of a twist (rho, phi) as (R, t) (Rodrigues + left Jacobian)."""
    rho, phi = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-10:
        R = np.eye(3) + K
        V = np.eye(3) + 0.5 * K
    else:
        R = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * K + (th - np.sin(th)) / th ** 3 * K @ K
    return R, V @ rho


def apply_twist(cam: dict, xi) -> dict:
    """Camera with pose exp(xi^) T_cw."""
    xi = np.asarray(xi, np.float64).reshape(6)
    if not np.any(xi):
        return cam
    Rd, td = se3_exp(xi)
    R0, t0 = np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64)
    return dict(cam, R=Rd @ R0, t=Rd @ t0 + td)


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cam, tile, glctx, twist, means, log_scales, quats, logits, sh):
        params = dict(means=means.contiguous(), log_scales=log_scales.contiguous(), quats=quats.contiguous(),
                      logits=logits.contiguous(), sh=sh.contiguous())
        c = apply_twist(cam, twist.detach().cpu().numpy())
        rgb, depth, opac = glctx.forward(params, c, tile)
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
