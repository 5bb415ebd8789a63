"""How optimisation steps execute: records staged per warp batch (32/64),
pixels per lane (1/2/4), persistent raster grids, the binning tile size and
CUDA-graph replay of whole steps.

Batch depth, pixels per lane and persistence change no rendered pixel
(bit-exact) and no step result beyond the atomic-order tolerance; the tile
size changes the 3-sigma tile rectangles, and each size matches the oracle
run at that size; a replayed step equals an eager one, including the step
that overflows its instance buffers and is re-run."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2404_06926_gb300 import scenes

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import _parity as PT  # noqa: E402

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EXECS = [dict(batch_depth=bd, pixels_per_lane=pp, persistent=pe)
         for bd in (32, 64) for pp in (1, 2, 4) for pe in (0, 1)] + \
        [dict(batch_depth=bd, pixels_per_lane=1, persistent=pe) for bd in (128, 256) for pe in (0, 1)]


def _map(params, tile=16):
    from paper_2404_06926_gb300 import binding
    m = binding.Map(binding.default_config(n_sky=0, sh_degree=3, tile_size=tile, capacity_hint=8192))
    m.set_params(params)
    return m


def _window_scene():
    sc = scenes.diff_check()
    base = sc["cam"]
    rng = np.random.default_rng(31)
    cams, targets = [], []
    for (W, H, f) in ((256, 192, 200.0), (192, 128, 150.0), (160, 160, 170.0)):
        w = rng.normal(0, 0.02, 3)
        R = scenes._rodrigues(w) @ np.asarray(base["R"])
        t = np.asarray(base["t"]) + rng.normal(0, 0.05, 3)
        cams.append(scenes.camera(W, H, f, f, W / 2, H / 2, R=R, t=t))
        targets.append(rng.uniform(0, 1, (H, W, 3)).astype(np.float32))
    return sc["params"], cams, targets


def _agree(a, b, p0, lr, frac=0.99):
    """Fraction of entries whose moves from p0 agree within 1e-3 lr."""
    out = {}
    for name in ("means", "log_scales", "quats", "logits", "sh"):
        da = a[name].astype(np.float64) - p0[name]
        db = b[name].astype(np.float64) - p0[name]
        moved = (da != 0) | (db != 0)
        if not moved.any():
            out[name] = 1.0
            continue
        out[name] = float((np.abs(da - db)[moved] <= 1e-3 * lr[name if name != "sh" else "sh_dc"] + 1e-7).mean())
    return out


@pytest.mark.parametrize("ex", EXECS, ids=lambda e: f"b{e['batch_depth']}p{e['pixels_per_lane']}s{e['persistent']}")
def test_render_bit_identical_across_exec(ex):
    sc = scenes.diff_check()
    cam = sc["cam"]
    m = _map(sc["params"])
    H, W = cam["height"], cam["width"]
    ref = [np.empty((H, W, 3), np.float32), np.empty((H, W), np.float32), np.empty((H, W), np.float32)]
    m.render(cam, out_rgb=ref[0], out_depth=ref[1], out_opacity=ref[2])
    m.set_exec(**ex)
    got = [np.empty_like(x) for x in ref]
    m.render(cam, out_rgb=got[0], out_depth=got[1], out_opacity=got[2])
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("tile,ex", [(8, dict(batch_depth=32, pixels_per_lane=2, persistent=1)),
                                     (16, dict(batch_depth=64, pixels_per_lane=4, persistent=1)),
                                     (16, dict(batch_depth=32, pixels_per_lane=1, persistent=0)),
                                     (32, dict(batch_depth=64, pixels_per_lane=2, persistent=0)),
                                     (32, dict(batch_depth=32, pixels_per_lane=4, persistent=1)),
                                     (16, dict(batch_depth=32, pixels_per_lane=1, persistent=1, per_gaussian=1)),
                                     (8, dict(batch_depth=64, pixels_per_lane=2, persistent=0, per_gaussian=1)),
                                     (16, dict(batch_depth=128, pixels_per_lane=1, persistent=1)),
                                     (32, dict(batch_depth=256, pixels_per_lane=1, persistent=0))])
def test_window_step_parity_under_exec(tile, ex):
    """The mixed-resolution window step equals the oracle at the same tile
    size for every execution."""
    params, cams, targets = _window_scene()
    m = _map(params)
    m.set_exec(tile_size=tile, **ex)
    views = [(10 + i, cams[i], targets[i]) for i in range(3)]
    loss = m.optimize_step(views, want_loss=True)
    st = oracle.new_window_state(params, 3)
    r = oracle.optimize_window(params, st, cams, targets, step=1, Ts=tile)
    assert abs(loss - r["loss"]) <= 2e-5 * r["loss"]
    got = m.get_params()
    PT.assert_step_matches(got, params, st["p"], r["grads"], r["visible"], PT.learning_rates(oracle.DEFAULT_LR))
    for i in range(3):
        assert np.allclose(m.exposure(10 + i), st["p"]["E"][i], atol=1e-6)


@pytest.mark.parametrize("tile,ppl,persistent,pg", [(16, 1, 0, 0), (16, 2, 1, 0), (8, 1, 1, 0), (16, 1, 1, 1)])
def test_deterministic_steps_are_bit_identical(tile, ppl, persistent, pg):
    """With the deterministic backward, eager and graph-replayed maps taking
    the same steps end bit-identical, and the first step equals the oracle."""
    params, cams, targets = _window_scene()
    maps = [_map(params), _map(params)]
    for m, graphs in zip(maps, (0, 1)):
        m.set_exec(deterministic=1, use_graphs=graphs, tile_size=tile, pixels_per_lane=ppl, persistent=persistent,
                   per_gaussian=pg)
    views = [(10 + i, cams[i], targets[i]) for i in range(3)]
    losses = [[m.optimize_step(views, want_loss=True) for _ in range(4)] for m in maps]
    assert losses[0] == losses[1]
    pa, pb = maps[0].get_params(), maps[1].get_params()
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    for i in range(3):
        assert np.array_equal(maps[0].exposure(10 + i), maps[1].exposure(10 + i))
    assert maps[1].stats()["graph_replays"] == 3
    # one deterministic step against the oracle
    m = _map(params)
    m.set_exec(deterministic=1, tile_size=tile, pixels_per_lane=ppl, persistent=persistent, per_gaussian=pg)
    m.optimize_step(views)
    st = oracle.new_window_state(params, 3)
    r = oracle.optimize_window(params, st, cams, targets, step=1, Ts=tile)
    got = m.get_params()
    PT.assert_step_matches(got, params, st["p"], r["grads"], r["visible"], PT.learning_rates(oracle.DEFAULT_LR))


def test_host_and_device_targets_give_identical_steps():
    """Targets in host memory (pageable or pinned) are copied on a side
    stream while the step's first kernels run, and the loss waits for that
    copy (in captured steps through an external event node): with the
    deterministic backward, steps with host targets are bit-identical to
    steps with the same targets in device memory, eager and replayed."""
    params, cams, targets = _window_scene()
    dev = [torch.from_numpy(t).cuda() for t in targets]
    pinned = [torch.from_numpy(t).pin_memory() for t in targets]
    maps = [_map(params) for _ in range(3)]
    for m in maps:
        m.set_exec(deterministic=1, use_graphs=1)
    losses = [[], [], []]
    for _ in range(5):
        for j, imgs in enumerate((dev, targets, pinned)):
            views = [(10 + i, cams[i], imgs[i]) for i in range(3)]
            losses[j].append(maps[j].optimize_step(views, want_loss=True))
    assert losses[0] == losses[1] == losses[2]
    ref = maps[0].get_params()
    for m in maps[1:]:
        got = m.get_params()
        for k in ref:
            assert np.array_equal(ref[k], got[k]), k
        for i in range(3):
            assert np.array_equal(maps[0].exposure(10 + i), m.exposure(10 + i))
        assert m.stats()["graph_replays"] == 4


def test_graph_replay_equals_eager_over_steps():
    """With atomic gradient accumulation (the default) the order of the
    float additions depends on the warps' timing, so after several Adam steps
    the entries whose gradient is at noise level (sums of many cancelling
    pixel terms on this random-target scene) may have moved either way: the
    moves of a graph-replayed and an eager map agree for most entries (two
    eager maps usually agree on all of them, and the fraction is reported).
    Bit-identity of the two paths is checked with the deterministic backward
    in test_deterministic_steps_are_bit_identical."""
    params, cams, targets = _window_scene()
    a, a2, b = _map(params), _map(params), _map(params)
    b.set_exec(use_graphs=1)
    views = [(10 + i, cams[i], targets[i]) for i in range(3)]
    la, lb = [], []
    for _ in range(6):
        la.append(a.optimize_step(views, want_loss=True))
        a2.optimize_step(views)
        lb.append(b.optimize_step(views, want_loss=True))
    assert np.allclose(la, lb, rtol=1e-4)
    s = b.stats()
    assert s["graph_captures"] == 1 and s["graph_replays"] == 5
    frac = _agree(a.get_params(), b.get_params(), params, oracle.DEFAULT_LR)
    base = _agree(a.get_params(), a2.get_params(), params, oracle.DEFAULT_LR)
    for name, f in frac.items():
        assert f > 0.9, (name, f, base[name])
    for i in range(3):
        assert np.allclose(a.exposure(10 + i), b.exposure(10 + i), atol=1e-5)


def test_graph_overflow_is_rerun_once():
    """A replay whose view needs more instances than the captured step left
    room for updates nothing and is re-run eagerly: the results equal an
    eager map taking the same steps."""
    sc = scenes.diff_check()
    cam = sc["cam"]
    far = dict(cam, t=np.asarray(cam["t"]) + np.array([2.2, 0.0, 0.0]))   # sees a sliver of the scene
    tgt = np.ascontiguousarray(sc["target"])
    a, b = _map(sc["params"]), _map(sc["params"])
    b.set_exec(use_graphs=1)
    for m in (a, b):
        m.optimize_step([(1, far, tgt)])
    n_far = b.stats()["n_instances"]
    for m in (a, b):
        m.optimize_step([(2, cam, tgt)])
    s = b.stats()
    assert s["n_instances"] > 1.25 * n_far + 1024, (s["n_instances"], n_far)
    assert s["graph_captures"] >= 1 and s["graph_replays"] == 1 and s["graph_reruns"] == 1
    frac = _agree(a.get_params(), b.get_params(), sc["params"], oracle.DEFAULT_LR)
    for name, f in frac.items():
        assert f > 0.98, (name, f)
    assert np.allclose(a.exposure(2), b.exposure(2), atol=1e-5)
    assert np.allclose(a.exposure(1), b.exposure(1), atol=1e-5)


def test_autotune_picks_a_valid_config_and_restores_the_map():
    params, cams, targets = _window_scene()
    m = _map(params)
    views = [(10 + i, cams[i], targets[i]) for i in range(3)]
    m.optimize_step(views)
    before = m.get_params()
    mom = [m.get_moments(1), m.get_moments(2)]
    E = [m.exposure(10 + i) for i in range(3)]
    steps = m.stats()["steps"]
    best, ms = m.autotune(views, reps=2)
    assert ms > 0
    assert best["use_graphs"] == 1 and best["tile_size"] in (8, 16, 32)
    assert best["batch_depth"] in (32, 64, 128, 256) and best["pixels_per_lane"] in (1, 2, 4)
    assert best["batch_depth"] <= 64 or best["pixels_per_lane"] == 1
    assert 4 * best["pixels_per_lane"] <= best["tile_size"]
    assert m.get_exec() == best
    after = m.get_params()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    for w in (1, 2):
        got = m.get_moments(w)
        for k in got:
            assert np.array_equal(got[k], mom[w - 1][k]), (w, k)
    for i in range(3):
        assert np.array_equal(m.exposure(10 + i), E[i])
    assert m.stats()["steps"] == steps
    # and the map keeps optimising with the chosen execution
    m.optimize_step(views)


def test_window_learning_rate_scaling():
    """lr_window_exp = 0.5 scales the Gaussians' learning rates of a 3-view
    window by sqrt(3) (the exposures keep theirs): equal to the oracle step
    with those rates."""
    params, cams, targets = _window_scene()
    m = _map(params)
    m.set_config(lr_window_exp=0.5)
    m.optimize_step([(10 + i, cams[i], targets[i]) for i in range(3)])
    f = np.sqrt(3.0)
    lr = {k: (v * f if k != "exposure" else v) for k, v in oracle.DEFAULT_LR.items()}
    st = oracle.new_window_state(params, 3)
    r = oracle.optimize_window(params, st, cams, targets, step=1, Ts=16, lr=lr)
    got = m.get_params()
    vis = r["visible"]
    PT.assert_step_matches(got, params, st["p"], r["grads"], vis, PT.learning_rates(lr))
    base = PT.learning_rates(oracle.DEFAULT_LR)
    for name in PT.GROUPS:
        # the moves are sqrt(3) times those at the paper's rates
        d_gpu = PT.group(got, name)[vis].astype(np.float64) - PT.group(params, name)[vis]
        gref = PT.group(r["grads"], name)[vis]
        clear = np.abs(gref) > 1e-3 * np.sqrt(np.mean(gref ** 2))
        assert np.median(np.abs(d_gpu)[clear]) > 1.5 * base[name], name
    for i in range(3):
        assert np.allclose(m.exposure(10 + i), st["p"]["E"][i], atol=1e-6)


def test_set_config_rejects_bad_values_and_keeps_the_map():
    from paper_2404_06926_gb300 import binding
    params, cams, targets = _window_scene()
    m = _map(params)
    before = m.get_exec()
    for bad in (dict(lr_pos=-1.0), dict(tile_size=12), dict(sh_degree=0), dict(lambda_dssim=2.0)):
        with pytest.raises(binding.GLError):
            m.set_config(**bad)
    m2 = binding.Config()
    binding.lib().gl_map_get_config(m._h, binding.C.byref(m2))
    assert abs(m2.lr_pos - 1.6e-4) < 1e-10 and m2.tile_size == 16
    assert m.get_exec() == before


def test_autotune_over_several_single_view_windows_restores_the_map():
    params, cams, targets = _window_scene()
    m = _map(params)
    views = [(10 + i, cams[i], targets[i]) for i in range(3)]
    for v in views:
        m.optimize_step([v])
    before = m.get_params()
    E = [m.exposure(10 + i) for i in range(3)]
    best, ms = m.autotune(views, reps=2, keep_tile_size=True, window=1)
    assert ms > 0 and best["tile_size"] == 0
    after = m.get_params()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    for i in range(3):
        assert np.array_equal(m.exposure(10 + i), E[i])
