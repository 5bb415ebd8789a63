"""Host side of the full-size keyframe-window parity test.

The benchmark's batched workload and the oracle's work on it, per view, in a
module without torch or CUDA so that spawned worker processes can import it.

Workload: the street scene of seed 4 (Sec. IV-A stand-in): 1,800,000 LiDAR
and visual points with a quarter of the LiDAR rays kept, initialised as new
Gaussians by the oracle (Sec. III-C 1: scale d/f with d the depth in the
capture pose), plus 200,000 sky Gaussians uniform by area on the 1e4 m
hemisphere with a fixed 28 m scale (the mean nearest-neighbour spacing of 2e5
points there); then seeded perturbations of scales, rotations, opacities and
SH as a map under optimisation has them.  SH degree 3.  The window: 12
keyframes along the trajectory, 4 each of 1280x1024, 1024x768 and 640x512
(fx = 0.78125 W), each with its ray-cast target under its own affine exposure.
"""
import os

import numpy as np

import oracle
from paper_2404_06926_gb300 import scenes

SEED = 4
N_POINTS, N_SKY = 1_800_000, 200_000
VIEWS = [(1280, 1024), (1024, 768), (640, 512)] * 4
TILE = 16
SAMPLE_STRIDE = 37          # every 37th Gaussian has its gradient compared
KEYS = ("means", "log_scales", "quats", "logits", "sh")


def scene():
    return scenes.Outdoor(seed=SEED, width=1280, img_height=1024, f=1000.0)


def camera(sc, k):
    pos = np.linspace(sc.traj_x[2], sc.traj_x[-12], len(VIEWS))
    kw, kh = VIEWS[k]
    return sc.camera_at(float(pos[k]), width=kw, height=kh, f=0.78125 * kw)


def sample_rows(n):
    return np.arange(0, n, SAMPLE_STRIDE)


def make_params():
    sc = scene()
    xyz, rgb, idx = sc.point_cloud(N_POINTS, keep=0.25)
    depth = np.zeros(len(xyz), np.float64)
    for i, s in enumerate(sc.traj_x):
        sel = idx == i
        if sel.any():
            cam = sc.camera_at(s)
            R, t = np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64)
            depth[sel] = (xyz[sel].astype(np.float64) @ R.T + t)[:, 2]
    keep = depth > 0.2
    pts = oracle.init_gaussians(xyz[keep], rgb[keep], depth[keep], 1000.0)
    rng = np.random.default_rng(8)
    u, v = rng.uniform(0, 1, N_SKY), rng.uniform(0, 1, N_SKY)
    r = np.sqrt(np.maximum(0.0, 1.0 - u * u))
    sky = 1e4 * np.stack([r * np.cos(2 * np.pi * v), r * np.sin(2 * np.pi * v), u], 1)
    skyp = oracle.init_gaussians(sky, np.ones((N_SKY, 3)), np.ones(N_SKY), 1.0, opacity=0.7,
                                 scale=np.full(N_SKY, 28.0))
    p = {k: np.ascontiguousarray(np.concatenate([pts[k], skyp[k]])) for k in pts}
    n = p["means"].shape[0]
    p["log_scales"] = (p["log_scales"] + rng.normal(0, 0.3, (n, 3))).astype(np.float32)
    q = p["quats"] + rng.normal(0, 0.3, (n, 4))
    p["quats"] = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    p["logits"] = (p["logits"] + rng.normal(0, 1.0, n)).astype(np.float32)
    sh = p["sh"].astype(np.float64)
    sh[:, 1:, :] += rng.normal(0, 0.05, sh[:, 1:, :].shape)
    p["sh"] = sh.astype(np.float32)
    return p


def save_params(p, d):
    for k in KEYS:
        np.save(os.path.join(d, k + ".npy"), np.ascontiguousarray(p[k], np.float32))


def load_params(d):
    return {k: np.load(os.path.join(d, k + ".npy")) for k in KEYS}


def target_path(d, k):
    return os.path.join(d, "target%d.npy" % k)


def write_target(args):
    """Worker: the ray-cast target of view k (independent of any renderer)."""
    d, k = args
    sc = scene()
    img = sc.target_image(camera(sc, k), rng=np.random.default_rng(400 + k))[0]
    np.save(target_path(d, k), img)
    return k


def oracle_view(args):
    """Worker: view k's Eq. 9 loss (identity exposure) and its gradient to
    every Gaussian attribute by the oracle; returns the loss, the visibility
    mask (radius > 0) of every Gaussian and the gradients of the sampled rows."""
    d, k = args
    p = load_params(d)
    sc = scene()
    cam = camera(sc, k)
    tgt = np.load(target_path(d, k))
    E = np.hstack([np.eye(3), np.zeros((3, 1))])
    r = oracle.loss_and_grads(p, cam, tgt, E, TILE)
    rows = sample_rows(p["means"].shape[0])
    return dict(k=k, loss=float(r["loss"]["loss"]), vis=r["pre"]["radius"] > 0,
                grads={name: np.ascontiguousarray(r["grads"][name][rows]) for name in KEYS},
                ambiguous=float(r["img"]["ambiguous"].mean()), instances=int(r["bins"]["I"]))
