"""Per-tile load of rendered views: how long each tile's (Gaussian, tile)
list is and how far each 8x4 pixel block walks it (the last contributor of
its pixels), which is the serial work of one raster warp.

    python -m paper_2404_06926_gb300.tilestats [--small] [--views 0,5,10,15]

builds the street workload (the benchmark's 1M-Gaussian map, or the 250k
one with --small), renders the given keyframe views through the stateless
API and prints one JSON object per view.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def view_load(ctx, params: dict, cam: dict, tile: int = 16) -> dict:
    """Load statistics of one forward render (params: device tensors)."""
    ctx.forward(params, cam, tile)
    H, W = int(cam["height"]), int(cam["width"])
    TX, TY = (W + tile - 1) // tile, (H + tile - 1) // tile
    _, _, ranges = ctx.instances(TX * TY, params["means"].device)
    L = (ranges[:, 1] - ranges[:, 0]).cpu().numpy().astype(np.int64)
    _, ncon = ctx.pixel_state(H, W, params["means"].device)
    nc = ncon.cpu().numpy().astype(np.int64)
    Hp, Wp = (H + 3) // 4 * 4, (W + 7) // 8 * 8
    pad = np.zeros((Hp, Wp), np.int64)
    pad[:H, :W] = nc
    block = pad.reshape(Hp // 4, 4, Wp // 8, 8).max(axis=(1, 3))
    top = np.argsort(-L)[:5]
    return dict(instances=int(L.sum()), tiles=int(L.size), list_mean=float(L.mean()),
                list_p99=float(np.percentile(L, 99)), list_max=int(L.max()),
                heaviest_tiles=[dict(tile=int(t), x=int(t % TX) * tile, y=int(t // TX) * tile, length=int(L[t]))
                                for t in top],
                block_walk_mean=float(block.mean()), block_walk_p99=float(np.percentile(block, 99)),
                block_walk_max=int(block.max()), blocks=int(block.size))


def _street_map(binding, small: bool):
    from . import scenes
    W, H, f, n_pts, n_sky = (640, 512, 500.0, 225_000, 25_000) if small else (1280, 1024, 1000.0, 900_000, 100_000)
    sc = scenes.Outdoor(seed=2, width=W, img_height=H, f=f)
    xyz, rgb, idx = sc.point_cloud(n_pts)
    m = binding.Map(binding.default_config(n_sky=n_sky, sh_degree=3, tile_size=16, capacity_hint=n_pts + n_sky))
    for i, s in enumerate(sc.traj_x):
        sel = np.nonzero(idx == i)[0]
        if len(sel):
            m.add_points(np.ascontiguousarray(xyz[sel]), np.ascontiguousarray(rgb[sel]), sc.camera_at(s),
                         use_mask=False, kind=0)
    pos = np.linspace(sc.traj_x[2], sc.traj_x[-12], 16)
    return m, [sc.camera_at(float(s)) for s in pos]


def main():
    import torch
    from . import binding
    ap = argparse.ArgumentParser()
    ap.add_argument("--small", action="store_true")
    ap.add_argument("--views", default="0,5,10,15")
    args = ap.parse_args()
    m, cams = _street_map(binding, args.small)
    p = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in m.get_params().items()}
    ctx = binding.Ctx()
    out = {int(k): view_load(ctx, p, cams[int(k)]) for k in args.views.split(",")}
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
