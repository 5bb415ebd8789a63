"""Map checkpoint: save -> load reproduces the whole optimisation state
(Gaussians, kinds, Adam moments and step, keyframes with exposure state and
images) exactly, so the loaded map renders bit-identically and continues
optimising like the original; malformed buffers are rejected without
touching the map."""
import numpy as np
import pytest

from paper_2404_06926_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _map(params=None, deg=3):
    from paper_2404_06926_gb300 import binding
    m = binding.Map(binding.default_config(n_sky=0, sh_degree=deg, tile_size=16, capacity_hint=4096))
    if params is not None:
        m.set_params(params)
    return m


def _state(m, ids):
    return (m.get_params(), m.get_moments(1), m.get_moments(2), [m.exposure(i) for i in ids], m.stats()["steps"])


def _equal(a, b):
    pa, m1a, m2a, Ea, sa = a
    pb, m1b, m2b, Eb, sb = b
    for x, y in ((pa, pb), (m1a, m1b), (m2a, m2b)):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
    for x, y in zip(Ea, Eb):
        assert np.array_equal(x, y)
    assert sa == sb


def test_save_load_round_trip_and_continue():
    sc = scenes.diff_check()
    cam, tgt = sc["cam"], np.ascontiguousarray(sc["target"])
    cam2 = dict(cam, t=np.asarray(cam["t"]) + np.array([0.05, -0.02, 0.0]))
    a = _map(sc["params"])
    a.add_keyframe(4, cam, tgt)
    a.add_keyframe(9, cam2, np.ascontiguousarray(tgt[::-1]))
    for k in (4, 9, 4):
        a.optimize_step([(k, cam if k == 4 else cam2, None)])
    buf = a.save(with_images=True)
    b = _map()
    b.load(buf)
    assert len(b) == len(a)
    _equal(_state(a, (4, 9)), _state(b, (4, 9)))
    ra, rb = a.render(cam2), b.render(cam2)
    assert np.array_equal(ra, rb)
    # the stored images came along: both maps step on keyframe 9 alone
    la = a.optimize_step([(9, cam2, None)], want_loss=True)
    lb = b.optimize_step([(9, cam2, None)], want_loss=True)
    assert abs(la - lb) <= 1e-6 * abs(la)
    assert np.allclose(a.exposure(9), b.exposure(9), atol=1e-6)
    # a checkpoint without images still restores everything else
    c = _map()
    c.load(a.save(with_images=False))
    _equal(_state(a, (4, 9)), _state(c, (4, 9)))
    with pytest.raises(Exception):
        c.optimize_step([(9, cam2, None)])   # no stored image in c


def test_malformed_checkpoints_are_rejected():
    from paper_2404_06926_gb300 import binding
    sc = scenes.diff_check()
    a = _map(sc["params"])
    buf = a.save()
    victim = _map(scenes.small_frustum()["params"], deg=0)
    before = victim.get_params()
    bad = buf.copy()
    bad[0] = ord("X")
    with pytest.raises(binding.GLError):
        victim.load(bad)
    with pytest.raises(binding.GLError):
        victim.load(buf[:100])
    with pytest.raises(binding.GLError):   # SH degree 3 into a degree-0 map
        victim.load(buf)
    after = victim.get_params()
    for k in before:
        assert np.array_equal(before[k], after[k])
