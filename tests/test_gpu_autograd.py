"""Form (3): the hand-written adjoint behind torch.autograd.Function, with
gradients to every Gaussian attribute, the camera pose twist and the exposure,
against the oracle's analytic gradient (itself pinned by finite differences)
and, for the twist, against central differences of the oracle's loss over the
twist itself.

The pose rendered is exp(xi^) T_cw; the library evaluates the exponential and
returns dL/dxi.  The tests form exp(xi^) independently, as the matrix
exponential of the 4 x 4 twist matrix (scipy.linalg.expm)."""
import numpy as np
import pytest

import oracle
from paper_2404_06926_gb300 import scenes

torch = pytest.importorskip("torch")
scipy_linalg = pytest.importorskip("scipy.linalg")
pytestmark = pytest.mark.gpu


def rel_stats(gpu, ref, floor_frac=1e-4):
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    floor = floor_frac * max(np.abs(ref).max(), 1e-30)
    r = np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)
    return float(np.median(r)), float(np.percentile(r, 99))


def twisted(cam, xi):
    """Camera at exp(xi^) T_cw, xi = (rho, phi), by the matrix exponential."""
    xi = np.asarray(xi, np.float64)
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -xi[5], xi[4]], [xi[5], 0, -xi[3]], [-xi[4], xi[3], 0]]
    M[:3, 3] = xi[:3]
    E = scipy_linalg.expm(M)
    R0, t0 = np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64)
    return dict(cam, R=E[:3, :3] @ R0, t=E[:3, :3] @ t0 + E[:3, 3])


def as_float32_pose(cam):
    """The pose as the kernels receive it (rounded to float32)."""
    return dict(cam, R=np.asarray(cam["R"], np.float32).astype(np.float64),
                t=np.asarray(cam["t"], np.float32).astype(np.float64))


@pytest.mark.parametrize("twist_scale", [0.0, 0.01])
def test_autograd_loss_gradients_match_oracle(twist_scale):
    from paper_2404_06926_gb300 import autograd as ag
    sc = scenes.diff_check()
    cam0 = sc["cam"]
    xi = np.random.default_rng(4).normal(0, twist_scale, 6)
    cam = as_float32_pose(twisted(cam0, xi))
    r = oracle.loss_and_grads(sc["params"], cam, sc["target"], sc["E"], 16)
    p = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda().requires_grad_(True) for k, v in sc["params"].items()}
    twist = torch.tensor(xi, dtype=torch.float32, device="cuda", requires_grad=True)
    E = torch.from_numpy(np.ascontiguousarray(sc["E"])).cuda().requires_grad_(True)
    tgt = torch.from_numpy(sc["target"]).cuda()
    rgb, depth, opac = ag.render(p, cam0, twist)
    L = ag.photometric_loss(rgb, tgt, E)
    L.backward()
    assert abs(L.item() - r["loss"]["loss"]) <= 2e-5 * r["loss"]["loss"]
    vis = r["pre"]["radius"] > 0
    for name in ("means", "log_scales", "quats", "logits", "sh"):
        med, p99 = rel_stats(p[name].grad.cpu().numpy()[vis], r["grads"][name][vis])
        assert med < 1e-3 and p99 < 1e-2, (name, med, p99)
    if twist_scale == 0.0:
        # at xi = 0 the twist gradient is the left-perturbation gradient itself
        gp = twist.grad.cpu().numpy().astype(np.float64)
        ref = r["grads"]["pose"]
        rel = np.abs(gp - ref) / np.maximum(np.abs(ref), 1e-4 * np.abs(ref).max())
        assert np.median(rel) < 1e-3 and rel.max() < 1e-2, (gp, ref, rel)
    assert np.allclose(E.grad.cpu().numpy(), r["loss"]["dL_dE"], rtol=2e-3,
                       atol=2e-4 * np.abs(r["loss"]["dL_dE"]).max())


def _fd_scene():
    """300 Gaussians in front of a 64 x 48 camera (the oracle's FD scene)."""
    rng = np.random.default_rng(7)
    W, H = 64, 48
    base = scenes.camera(W, H, 60.0, 60.0, W / 2, H / 2)
    p = scenes.random_gaussians(rng, 300, base, 3, 0.3, z_range=(1.0, 6.0), log_scale_mean=-2.3,
                                log_scale_std=0.4)
    cam = scenes.camera(W, H, 60.0, 60.0, W / 2 + 0.3, H / 2 - 0.2, R=scenes._rodrigues(rng.normal(0, 0.03, 3)),
                        t=rng.normal(0, 0.05, 3))
    target = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    E = np.hstack([np.eye(3) + rng.normal(0, 0.05, (3, 3)), rng.normal(0, 0.02, (3, 1))]).astype(np.float32)
    return p, cam, target, E


def _oracle_loss(p, cam, target, E):
    pre, bins, img = oracle.forward(p, cam, 16)
    L = oracle.loss(img["color"], target, E)["loss"]
    sig = (pre["radius"].tobytes(), pre["rect"].tobytes(), pre["flags"].tobytes(),
           img["n_contrib"].tobytes(), img["signature"].tobytes())
    return L, sig


@pytest.mark.parametrize("seed", [0, 1])
def test_twist_gradient_off_zero_matches_central_differences(seed):
    """dL/dxi at xi != 0 (a twist of 0.05 rad / 0.05 m scale) against central
    differences of the oracle's fp64 loss over xi.  A difference counts only
    where the per-pixel decisions (contributor sets, clamps, culls) are the
    same at xi +- h as at xi (h = 1e-4, else the first of 1e-5 .. 1e-8 that
    keeps them: a pose moves every Gaussian, so over a few thousand pixels
    some decision sits close to its threshold; fp64 round-off at h = 1e-8 is
    still ~1e-8 of the gradient)."""
    from paper_2404_06926_gb300 import autograd as ag
    p, cam0, target, E = _fd_scene()
    xi0 = np.random.default_rng(100 + seed).normal(0, 0.05, 6)
    xi0 = xi0.astype(np.float32).astype(np.float64)
    pd = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in p.items()}
    twist = torch.tensor(xi0, dtype=torch.float32, device="cuda", requires_grad=True)
    rgb, _, _ = ag.render(pd, cam0, twist)
    L = ag.photometric_loss(rgb, torch.from_numpy(target).cuda(), torch.from_numpy(E).cuda())
    L.backward()
    g_gpu = twist.grad.cpu().numpy().astype(np.float64)
    p64 = {k: v.astype(np.float64) for k, v in p.items()}
    L0, sig0 = _oracle_loss(p64, twisted(cam0, xi0), target, E)
    assert abs(L.item() - L0) <= 2e-5 * L0
    fd = np.full(6, np.nan)
    for k in range(6):
        for h in (1e-4, 1e-5, 1e-6, 1e-7, 1e-8):
            e = np.zeros(6)
            e[k] = h
            Lp, sp = _oracle_loss(p64, twisted(cam0, xi0 + e), target, E)
            Lm, sm = _oracle_loss(p64, twisted(cam0, xi0 - e), target, E)
            if sp == sig0 and sm == sig0:
                fd[k] = (Lp - Lm) / (2 * h)
                break
    ok = np.isfinite(fd)
    assert ok.sum() >= 5, fd
    floor = 1e-4 * np.abs(fd[ok]).max()
    rel = np.abs(g_gpu[ok] - fd[ok]) / np.maximum(np.abs(fd[ok]), floor)
    assert np.median(rel) < 1e-3 and rel.max() < 1e-2, (g_gpu, fd, rel)


def test_autograd_depth_and_opacity_outputs():
    """Gradients flow from the depth and opacity maps too (Eq. 6-7)."""
    from paper_2404_06926_gb300 import autograd as ag
    sc = scenes.small_frustum()
    cam = sc["cam"]
    rng = np.random.default_rng(3)
    H, W = cam["height"], cam["width"]
    wD = rng.normal(size=(H, W)).astype(np.float32)
    wO = rng.normal(size=(H, W)).astype(np.float32)
    pre, bins, img = oracle.forward(sc["params"], cam, 16)
    g = oracle.backward(sc["params"], cam, pre, bins, np.zeros((H, W, 3)), wD.astype(np.float64),
                        wO.astype(np.float64))
    p = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda().requires_grad_(True) for k, v in sc["params"].items()}
    rgb, depth, opac = ag.render(p, cam)
    ((depth * torch.from_numpy(wD).cuda()).sum() + (opac * torch.from_numpy(wO).cuda()).sum()).backward()
    vis = pre["radius"] > 0
    for name in ("means", "log_scales", "logits"):
        med, p99 = rel_stats(p[name].grad.cpu().numpy()[vis], g[name][vis])
        assert med < 1e-3 and p99 < 1e-2, (name, med, p99)
