"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws numbers: it holds none of the map optimiser's arithmetic
(no projection, compositing, loss or initialisation rule).  Every generator is
deterministic in its seed (numpy PCG64).

Workloads (shapes and value distributions follow the paper's setting, Sec. IV-A,
scaled to the benchmark resolutions):
  small_frustum   -- 2,000 random Gaussians in a 128x96 view, SH degree 0.
  diff_check      -- 5,000 random Gaussians in a 256x192 view, SH degree 3, with a
                     small camera twist and a near-identity exposure.
  outdoor         -- a LiDAR-camera street scene: ground plane plus box facades,
                     a spinning-LiDAR sweep per pose (1/10 kept, FoV-cropped,
                     coloured), visual points on facades, analytic ray-cast target
                     images with per-image exposure, sky in the upper rows.
"""
from __future__ import annotations

import numpy as np


def camera(width, height, fx, fy=None, cx=None, cy=None, R=None, t=None) -> dict:
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    t = np.zeros(3) if t is None else np.asarray(t, np.float64)
    return dict(width=int(width), height=int(height), fx=float(np.float32(fx)), fy=float(np.float32(fy)),
                cx=float(np.float32(cx)), cy=float(np.float32(cy)),
                R=R.astype(np.float32).astype(np.float64), t=t.astype(np.float32).astype(np.float64))


def _rodrigues(w):
    th = np.linalg.norm(w)
    if th < 1e-12:
        return np.eye(3)
    k = w / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def random_gaussians(rng, n, cam, sh_deg, sh_std, z_range=(0.5, 10.0),
                     log_scale_mean=-2.0, log_scale_std=0.5) -> dict:
    """Means uniform in the camera frustum (pixel uniform, depth uniform), then
    mapped to world by the camera pose; random unit-direction quaternions."""
    W, H = cam["width"], cam["height"]
    u = rng.uniform(0, W, n)
    v = rng.uniform(0, H, n)
    z = rng.uniform(z_range[0], z_range[1], n)
    xc = np.stack([(u - cam["cx"]) * z / cam["fx"], (v - cam["cy"]) * z / cam["fy"], z], 1)
    R, t = cam["R"], cam["t"]
    xw = (xc - t) @ R          # R^T (x_c - t)
    ls = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    q = rng.normal(0, 1, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    lg = rng.normal(0, 1, n)
    K = (sh_deg + 1) ** 2
    sh = rng.normal(0, sh_std, (n, K, 3))
    f = np.float32
    return dict(means=xw.astype(f), log_scales=ls.astype(f), quats=q.astype(f), logits=lg.astype(f),
                sh=sh.astype(f))


def small_frustum(seed=1, n=2000, width=128, height=96, f=100.0) -> dict:
    """Plain single-view step: N=2000, 128x96, fx=fy=100, identity pose, deg 0."""
    rng = np.random.default_rng(seed)
    cam = camera(width, height, f, f, width / 2, height / 2)
    params = random_gaussians(rng, n, cam, 0, 0.5)
    target = rng.uniform(0, 1, (height, width, 3)).astype(np.float32)
    E = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
    return dict(params=params, cam=cam, target=target, E=E)


def diff_check(seed=3, n=5000, width=256, height=192, f=200.0) -> dict:
    """Differentiation check: N=5000, 256x192, deg 3, small twist, near-identity E."""
    rng = np.random.default_rng(seed)
    base = camera(width, height, f, f, width / 2, height / 2)
    params = random_gaussians(rng, n, base, 3, 0.2)
    w = rng.normal(0, 0.02, 3)
    rho = rng.normal(0, 0.05, 3)
    R = _rodrigues(w)
    cam = camera(width, height, f, f, width / 2, height / 2, R=R, t=rho)
    target = rng.uniform(0, 1, (height, width, 3)).astype(np.float32)
    A = np.eye(3) + rng.normal(0, 0.05, (3, 3))
    b = rng.normal(0, 0.02, (3, 1))
    E = np.hstack([A, b]).astype(np.float32)
    return dict(params=params, cam=cam, target=target, E=E)


# ----------------------------------------------------------------------------
# Outdoor LiDAR-camera street scene
# ----------------------------------------------------------------------------
class Outdoor:
    """Procedural street: ground z=0 over a 400 x 60 m strip, box facades beside
    a smooth S-shaped road, and a sky gradient.  World frame: x along the road,
    y left, z up.  Cameras look forward (+x along the trajectory tangent)."""

    def __init__(self, seed=2, n_boxes=40, n_poses=100, spacing=1.0, height=1.5,
                 width=1280, img_height=1024, f=1000.0):
        self.rng = np.random.default_rng(seed)
        rng = self.rng
        self.seed = seed
        self.W, self.H, self.f = width, img_height, f
        # trajectory: a smooth S-curve y(x) = A sin(2 pi x / L)
        self.amp, self.period = 4.0, 120.0
        xs = np.arange(n_poses) * spacing + 5.0
        self.traj_x = xs
        self.cam_h = height
        # box facades along both sides of the road
        bx = rng.uniform(0, 400, n_boxes)
        side = rng.choice([-1.0, 1.0], n_boxes)
        dist = rng.uniform(8, 30, n_boxes)
        wdt = rng.uniform(5, 20, n_boxes)
        dep = rng.uniform(4, 12, n_boxes)
        hgt = rng.uniform(5, 30, n_boxes)
        cy = self._road_y(bx) + side * (dist + dep / 2)
        self.box_lo = np.stack([bx - wdt / 2, cy - dep / 2, np.zeros(n_boxes)], 1)
        self.box_hi = np.stack([bx + wdt / 2, cy + dep / 2, hgt], 1)
        self.box_col = rng.uniform(0.2, 0.9, (n_boxes, 3))
        self.box_freq = rng.uniform(0.5, 2.0, n_boxes)
        self.ground_col = np.array([0.35, 0.33, 0.30])

    def _road_y(self, x):
        return self.amp * np.sin(2 * np.pi * x / self.period)

    def pose(self, s):
        """World->camera (R, t) at arc parameter s (metres along x)."""
        x = s
        y = self._road_y(x)
        dy = self.amp * 2 * np.pi / self.period * np.cos(2 * np.pi * x / self.period)
        fwd = np.array([1.0, dy, 0.0])
        fwd /= np.linalg.norm(fwd)
        up = np.array([0.0, 0.0, 1.0])
        right = np.cross(fwd, up)
        right /= np.linalg.norm(right)
        down = np.cross(fwd, right)
        Rwc = np.stack([right, down, fwd], 1)      # camera axes in world (x right, y down, z fwd)
        c = np.array([x, y, self.cam_h])
        R = Rwc.T
        t = -R @ c
        return R, t

    def camera_at(self, s, width=None, height=None, f=None):
        W = self.W if width is None else width
        H = self.H if height is None else height
        f = self.f if f is None else f
        R, t = self.pose(s)
        return camera(W, H, f, f, W / 2, H / 2, R=R, t=t)

    # -- ray casting against the plane and the boxes ---------------------------
    def cast(self, o, d):
        """Nearest hit of rays o + s d (s > 0): returns (s, colour, hit mask)."""
        with np.errstate(divide="ignore", invalid="ignore"):
            return self._cast(o, d)

    def _cast(self, o, d):
        n = d.shape[0]
        best = np.full(n, np.inf)
        col = np.zeros((n, 3))
        # ground plane z = 0 within the strip
        with np.errstate(divide="ignore", invalid="ignore"):
            s = -o[..., 2] / d[:, 2] if o.ndim == 1 else -o[:, 2] / d[:, 2]
        op = o if o.ndim == 2 else np.broadcast_to(o, d.shape)
        ok = (s > 0) & np.isfinite(s)
        hx = op[:, 0] + s * d[:, 0]
        hy = op[:, 1] + s * d[:, 1]
        ok &= (hx > -20) & (hx < 420) & (np.abs(hy) < 60)
        best = np.where(ok, s, best)
        tex = 0.75 + 0.25 * ((np.floor(hx / 2.0) + np.floor(hy / 2.0)) % 2)
        lane = (np.abs(hy - self._road_y(hx)) < 0.15) * 0.4
        gcol = self.ground_col[None] * tex[:, None] + lane[:, None]
        col = np.where(ok[:, None], gcol, col)
        # boxes (slab test)
        inv = 1.0 / np.where(np.abs(d) < 1e-12, 1e-12, d)
        for b in range(self.box_lo.shape[0]):
            t0 = (self.box_lo[b] - op) * inv
            t1 = (self.box_hi[b] - op) * inv
            tmin = np.minimum(t0, t1).max(1)
            tmax = np.maximum(t0, t1).min(1)
            hit = (tmax >= tmin) & (tmin > 0) & (tmin < best)
            if not hit.any():
                continue
            p = op[hit] + tmin[hit, None] * d[hit]
            fr = self.box_freq[b]
            pat = 0.7 + 0.3 * ((np.floor(p[:, 0] * fr) + np.floor(p[:, 1] * fr)
                                + np.floor(p[:, 2] * fr * 0.7)) % 2)
            best[hit] = tmin[hit]
            col[hit] = self.box_col[b][None] * pat[:, None]
        return best, col, np.isfinite(best)

    def target_image_torch(self, cam, device="cuda", rng=None, exposure=True):
        """The same analytic ray cast as target_image, evaluated with torch on
        `device` (float32) for large images; returns a device tensor."""
        import torch
        W, H = cam["width"], cam["height"]
        f32 = dict(dtype=torch.float32, device=device)
        v, u = torch.meshgrid(torch.arange(H, **f32), torch.arange(W, **f32), indexing="ij")
        dc = torch.stack([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], torch.ones_like(u)], -1)
        R = torch.tensor(np.asarray(cam["R"]), **f32)
        t = torch.tensor(np.asarray(cam["t"]), **f32)
        d = dc.reshape(-1, 3) @ R
        d = d / d.norm(dim=1, keepdim=True)
        o = -(R.T @ t)
        best = torch.full((d.shape[0],), float("inf"), **f32)
        col = torch.zeros((d.shape[0], 3), **f32)
        s = -o[2] / d[:, 2]
        hx = o[0] + s * d[:, 0]
        hy = o[1] + s * d[:, 1]
        ok = (s > 0) & torch.isfinite(s) & (hx > -20) & (hx < 420) & (hy.abs() < 60)
        best = torch.where(ok, s, best)
        tex = 0.75 + 0.25 * torch.remainder(torch.floor(hx / 2.0) + torch.floor(hy / 2.0), 2)
        road = self.amp * torch.sin(2 * np.pi * hx / self.period)
        lane = ((hy - road).abs() < 0.15).float() * 0.4
        gcol = torch.tensor(self.ground_col, **f32)[None] * tex[:, None] + lane[:, None]
        col = torch.where(ok[:, None], gcol, col)
        dd = torch.where(d.abs() < 1e-12, torch.full_like(d, 1e-12), d)
        inv = 1.0 / dd
        lo = torch.tensor(self.box_lo, **f32)
        hi = torch.tensor(self.box_hi, **f32)
        for b in range(lo.shape[0]):
            t0 = (lo[b] - o) * inv
            t1 = (hi[b] - o) * inv
            tmin = torch.minimum(t0, t1).max(1).values
            tmax = torch.maximum(t0, t1).min(1).values
            hit = (tmax >= tmin) & (tmin > 0) & (tmin < best)
            p = o + tmin[:, None] * d
            fr = float(self.box_freq[b])
            pat = 0.7 + 0.3 * torch.remainder(torch.floor(p[:, 0] * fr) + torch.floor(p[:, 1] * fr)
                                              + torch.floor(p[:, 2] * fr * 0.7), 2)
            best = torch.where(hit, tmin, best)
            bc = torch.tensor(self.box_col[b], **f32)
            col = torch.where(hit[:, None], bc[None] * pat[:, None], col)
        e = d[:, 2].clamp(0, 1)[:, None]
        sky = (1 - e) * torch.tensor([0.75, 0.85, 0.95], **f32) + e * torch.tensor([0.35, 0.55, 0.9], **f32)
        hitm = torch.isfinite(best)
        img = torch.where(hitm[:, None], col, sky)
        if exposure:
            rng = self.rng if rng is None else rng
            a, b = rng.uniform(0.7, 1.3), rng.uniform(-0.05, 0.05)
            img = (a * img + b).clamp(0, 1)
        return img.reshape(H, W, 3).contiguous()

    def sky_colour(self, d):
        e = np.clip(d[:, 2], 0, 1)[:, None]
        return (1 - e) * np.array([0.75, 0.85, 0.95]) + e * np.array([0.35, 0.55, 0.9])

    def target_image(self, cam, rng=None, exposure=True):
        """Analytic ray cast of the procedural scene (independent of any
        splatting renderer); sky where no surface is hit; then a per-image
        affine exposure a*C + b, clamped to [0,1].  Returns (image, sky mask, (a, b))."""
        W, H = cam["width"], cam["height"]
        u, v = np.meshgrid(np.arange(W), np.arange(H))
        dc = np.stack([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], np.ones_like(u, float)], -1)
        dc = dc.reshape(-1, 3)
        R, t = cam["R"], cam["t"]
        dw = dc @ R                       # R^T d_c
        dw /= np.linalg.norm(dw, axis=1, keepdims=True)
        o = -R.T @ t
        s, col, hit = self.cast(np.broadcast_to(o, dw.shape).copy(), dw)
        img = np.where(hit[:, None], col, self.sky_colour(dw))
        a, b = 1.0, 0.0
        if exposure:
            rng = self.rng if rng is None else rng
            a = rng.uniform(0.7, 1.3)
            b = rng.uniform(-0.05, 0.05)
            img = np.clip(a * img + b, 0, 1)
        return img.reshape(H, W, 3).astype(np.float32), (~hit).reshape(H, W), (a, b)

    def lidar_sweep(self, s, keep=0.1, beams=32, fov_deg=15.0, n_az=17600, noise=0.02, rng=None,
                    hfov=None):
        """One spinning-LiDAR sweep at pose s, kept 1/`keep`, cropped to the camera
        FoV, coloured by the surface albedo.  Rays are drawn at random so the
        random 1-in-N keep happens before casting."""
        rng = self.rng if rng is None else rng
        R, t = self.pose(s)
        o = -R.T @ t
        hfov = np.arctan(self.W / 2 / self.f) if hfov is None else hfov
        n_total = beams * n_az
        frac = (2 * hfov) / (2 * np.pi)
        m = rng.binomial(n_total, keep * frac)
        el = np.deg2rad(rng.integers(0, beams, m) * (2 * fov_deg / (beams - 1)) - fov_deg)
        az = rng.uniform(-hfov, hfov, m)
        dcam = np.stack([np.sin(az) * np.cos(el), -np.sin(el), np.cos(az) * np.cos(el)], 1)
        dw = dcam @ R
        s_hit, col, hit = self.cast(np.broadcast_to(o, dw.shape).copy(), dw)
        s_hit = s_hit[hit] + rng.normal(0, noise, hit.sum())
        pts = o[None] + s_hit[:, None] * dw[hit]
        # keep only returns inside the camera image
        pc = pts @ R.T + t
        uu = self.f * pc[:, 0] / pc[:, 2] + self.W / 2
        vv = self.f * pc[:, 1] / pc[:, 2] + self.H / 2
        inside = (pc[:, 2] > 0.5) & (uu >= 0) & (uu < self.W) & (vv >= 0) & (vv < self.H)
        return pts[inside].astype(np.float32), col[hit][inside].astype(np.float32)

    def visual_points(self, s, n, rng=None):
        """Points on facades above the LiDAR's top beam, visible from pose s."""
        rng = self.rng if rng is None else rng
        R, t = self.pose(s)
        o = -R.T @ t
        u = rng.uniform(0, self.W, n * 3)
        v = rng.uniform(0, self.H * 0.45, n * 3)
        dc = np.stack([(u - self.W / 2) / self.f, (v - self.H / 2) / self.f, np.ones(n * 3)], 1)
        dw = dc @ R
        dw /= np.linalg.norm(dw, axis=1, keepdims=True)
        s_hit, col, hit = self.cast(np.broadcast_to(o, dw.shape).copy(), dw)
        pts = o[None] + s_hit[hit, None] * dw[hit]
        upper = pts[:, 2] > self.cam_h + 1.0
        pts, col = pts[upper][:n], col[hit][upper][:n]
        return pts.astype(np.float32), col.astype(np.float32)

    def point_cloud(self, n_total, poses=None, visual_frac=0.05, keep=0.1):
        """LiDAR + visual points along the trajectory, truncated to n_total
        (`keep`: fraction of LiDAR rays kept per sweep, 1/10 in the paper).
        Returns (xyz, rgb, pose index of capture)."""
        poses = self.traj_x if poses is None else poses
        xs, cs, ks = [], [], []
        per_pose = int(np.ceil(1.03 * n_total / len(poses)))
        for i, s in enumerate(poses):
            p, c = self.lidar_sweep(s, keep=keep)
            nv = int(per_pose * visual_frac)
            vp, vc = self.visual_points(s, nv)
            p = np.concatenate([p[: per_pose - len(vp)], vp])
            c = np.concatenate([c[: per_pose - len(vc)], vc])
            xs.append(p)
            cs.append(c)
            ks.append(np.full(len(p), i, np.int32))
        xyz = np.concatenate(xs)[:n_total]
        rgb = np.concatenate(cs)[:n_total]
        idx = np.concatenate(ks)[:n_total]
        return xyz, rgb, idx
