"""Form (3): the hand-written adjoint behind torch.autograd.Function, with
gradients to every Gaussian attribute, the camera pose twist and the exposure,
against the oracle's analytic gradient (itself pinned by finite differences)."""
import numpy as np
import pytest

import oracle
from paper_2404_06926_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel_stats(gpu, ref, floor_frac=1e-4):
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    floor = floor_frac * max(np.abs(ref).max(), 1e-30)
    r = np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)
    return float(np.median(r)), float(np.percentile(r, 99))


@pytest.mark.parametrize("twist_scale", [0.0, 0.01])
def test_autograd_loss_gradients_match_oracle(twist_scale):
    from paper_2404_06926_gb300 import autograd as ag
    sc = scenes.diff_check()
    cam0 = sc["cam"]
    xi = np.random.default_rng(4).normal(0, twist_scale, 6)
    cam = ag.apply_twist(cam0, xi)
    # the oracle works on float32-rounded poses, as the GPU receives them
    cam = dict(cam, R=np.asarray(cam["R"], np.float32).astype(np.float64),
               t=np.asarray(cam["t"], np.float32).astype(np.float64))
    r = oracle.loss_and_grads(sc["params"], cam, sc["target"], sc["E"], 16)
    p = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda().requires_grad_(True) for k, v in sc["params"].items()}
    twist = torch.zeros(6, device="cuda", requires_grad=True)
    E = torch.from_numpy(np.ascontiguousarray(sc["E"])).cuda().requires_grad_(True)
    tgt = torch.from_numpy(sc["target"]).cuda()
    rgb, depth, opac = ag.render(p, cam, twist)
    L = ag.photometric_loss(rgb, tgt, E)
    L.backward()
    assert abs(L.item() - r["loss"]["loss"]) <= 2e-5 * r["loss"]["loss"]
    vis = r["pre"]["radius"] > 0
    for name in ("means", "log_scales", "quats", "logits", "sh"):
        med, p99 = rel_stats(p[name].grad.cpu().numpy()[vis], r["grads"][name][vis])
        assert med < 1e-3 and p99 < 1e-2, (name, med, p99)
    gp = twist.grad.cpu().numpy()
    assert np.linalg.norm(gp - r["grads"]["pose"]) <= 2e-3 * np.linalg.norm(r["grads"]["pose"])
    assert np.allclose(E.grad.cpu().numpy(), r["loss"]["dL_dE"], rtol=2e-3,
                       atol=2e-4 * np.abs(r["loss"]["dL_dE"]).max())


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
