"""Bounded device waits: a radix-sort pass whose look-back can never complete
(the tile it waits for is never published) gives up after its poll limit,
raises its flag and returns; the context stays usable.  No fault, no hang:
the wait is made to run out, as a flag that nothing sets."""
import time

import numpy as np
import pytest

from paper_2404_06926_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sort_wait_gives_up_and_reports():
    from paper_2404_06926_gb300 import binding
    t0 = time.perf_counter()
    assert binding.selftest_bounded_wait() is True
    assert time.perf_counter() - t0 < 30.0
    # the context is still usable: a render through the whole pipeline
    sc = scenes.diff_check()
    m = binding.Map(binding.default_config(n_sky=0, sh_degree=3, tile_size=16, capacity_hint=8192))
    m.set_params(sc["params"])
    img = m.render(sc["cam"])
    assert np.isfinite(img).all() and img.max() > 0
