"""Comparison of an optimisation step taken by the CUDA path with the oracle's.

A first Adam step from a zero state moves every entry by about lr * sign(g)
(Sec. III-C 3; Adam as in vanilla 3DGS, Sec. IV-A), so a step is compared by
its parameter moves: where the oracle's gradient is clearly non-zero (at least
1e-3 of the group's RMS) the two moves must agree within 1e-3 of the group's
learning rate (plus 1e-7 for the float32 rounding of the stored parameter) for
at least 99% of the entries.  Entries with a gradient at noise level can move
by +-lr either way and are not compared.  The SH coefficients are two groups
with their own learning rates: the DC band (coefficient 0, three channels) and
the higher bands.
"""
import numpy as np

GROUPS = ("means", "log_scales", "quats", "logits", "sh_dc", "sh_rest")


def group(d, name):
    """The entries of parameter group `name` of a parameter dict, row per Gaussian."""
    n = len(d["logits"])
    if name == "sh_dc":
        return np.asarray(d["sh"]).reshape(n, -1, 3)[:, :1].reshape(n, -1)
    if name == "sh_rest":
        return np.asarray(d["sh"]).reshape(n, -1, 3)[:, 1:].reshape(n, -1)
    return np.asarray(d[name]).reshape(n, -1)


def step_agreement(got, p0, ref, grads, moved_rows, lr, groups=GROUPS):
    """Per group, the fraction of clearly-driven entries of `moved_rows` whose
    moves from p0 agree (got: the GPU's parameters, ref: the oracle's)."""
    out = {}
    for name in groups:
        a = group(got, name).astype(np.float64) - group(p0, name).astype(np.float64)
        b = group(ref, name).astype(np.float64) - group(p0, name).astype(np.float64)
        if a.shape[1] == 0:
            continue
        g = group(grads, name)[moved_rows]
        clear = np.abs(g) > 1e-3 * np.sqrt(np.mean(g ** 2))
        if not clear.any():
            out[name] = 1.0
            continue
        d = np.abs(a[moved_rows] - b[moved_rows])[clear]
        out[name] = float((d <= 1e-3 * lr[name] + 1e-7).mean())
    return out


def assert_step_matches(got, p0, ref, grads, vis, lr, frozen=None, frac=0.99):
    """Rows outside `vis` are unchanged if `frozen` (default: every row outside
    vis); the driven entries of the rows in vis agree in every group."""
    frozen = ~vis if frozen is None else frozen
    for name in GROUPS:
        a = group(got, name).astype(np.float64) - group(p0, name).astype(np.float64)
        if a.shape[1]:
            assert np.all(a[frozen] == 0), name
    agree = step_agreement(got, p0, ref, grads, vis, lr)
    for name, f in agree.items():
        assert f > frac, (name, f)
    return agree


def learning_rates(lr):
    """The oracle's learning-rate dict keyed by group."""
    return dict(means=lr["means"], log_scales=lr["log_scales"], quats=lr["quats"], logits=lr["logits"],
                sh_dc=lr["sh_dc"], sh_rest=lr["sh_rest"])
