"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: closed
forms, brute-force enumeration, library routines (numpy's stable sort, scipy's
KD-tree, torch.optim.Adam), quadrature identities, published generator
outputs and finite differences.  None of these tests needs a GPU.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2404_06926_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- SH basis
def _fibonacci_sphere(n):
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    r = np.sqrt(1 - z * z)
    phi = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


def test_sh_orthonormal_by_quadrature():
    """Real SH to degree 3: int Y_i Y_j dOmega = delta_ij (Fibonacci rule, 20k nodes)."""
    pts = _fibonacci_sphere(20000)
    Y = np.array([oracle.sh_basis(3, p)[0] for p in pts])
    G = (Y.T @ Y) * (4 * np.pi / len(pts))
    assert np.abs(G - np.eye(16)).max() < 1e-3


def test_sh_degree0_is_constant_and_gradient_matches_fd():
    Y0, _ = oracle.sh_basis(0, [0.3, -0.2, 0.93])
    assert Y0.shape == (1,) and abs(Y0[0] - 0.5 / np.sqrt(np.pi)) < 1e-15
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.normal(size=3)
        Y, dY = oracle.sh_basis(3, d)
        h = 1e-6
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            fd = (oracle.sh_basis(3, d + e)[0] - oracle.sh_basis(3, d - e)[0]) / (2 * h)
            assert np.allclose(fd, dY[:, j], atol=1e-7, rtol=1e-7)


def test_sh_band_rotation_invariance():
    """sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every band (addition theorem)."""
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, _ = oracle.sh_basis(3, d)
        for l in range(4):
            band = Y[l * l:(l + 1) * (l + 1)]
            assert abs((band ** 2).sum() - (2 * l + 1) / (4 * np.pi)) < 1e-12


# --------------------------------------------------------------------------- RNG
def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    for i, v in enumerate(vals):
        assert oracle.uniform(0, i) == (v >> 40) / 2.0 ** 24


# --------------------------------------------------------------------------- projection
def _one(means, ls, q=(1, 0, 0, 0), logit=2.0, deg=0, dc=(0.0, 0.0, 0.0)):
    K = (deg + 1) ** 2
    sh = np.zeros((1, K, 3), np.float32)
    sh[0, 0] = np.asarray(dc, np.float32)
    return dict(means=np.array([means], np.float32), log_scales=np.array([ls], np.float32),
                quats=np.array([q], np.float32), logits=np.array([logit], np.float32), sh=sh)


def test_on_axis_isotropic_closed_form():
    """A Gaussian of scale s at (0,0,z) projects to (cx,cy) with
    Sigma' = ((f s / z)^2 + 0.3) I; radius = ceil(3 sqrt(v + sqrt(0.1)))."""
    cam = scenes.camera(128, 96, 100.0, 100.0, 64.0, 48.0)
    for z, s in ((2.0, 0.05), (5.0, 0.2), (1.0, 0.01)):
        p = _one([0.0, 0.0, z], [np.log(s)] * 3)
        pre = oracle.preprocess(p, cam, 16)
        s32 = float(np.float32(np.exp(np.float32(np.log(s)))))
        v = (100.0 * s32 / z) ** 2 + 0.3
        assert np.allclose(pre["mean2d"][0], [64.0, 48.0], atol=1e-12)
        assert np.allclose(pre["conic"][0], [1 / v, 0.0, 1 / v], rtol=1e-6)
        assert pre["radius"][0] == int(np.ceil(3 * np.sqrt(v + np.sqrt(0.1)) - 1e-9))
        assert abs(pre["depth"][0] - z) < 1e-12


def test_rotated_anisotropic_covariance():
    """q = 90 deg about the optical axis swaps the x and y scales."""
    cam = scenes.camera(128, 96, 100.0, 100.0, 64.0, 48.0)
    c, s = np.cos(np.pi / 4), np.sin(np.pi / 4)
    z = 4.0
    ls = [np.log(0.3), np.log(0.05), np.log(0.1)]
    p = _one([0.0, 0.0, z], ls, q=(c, 0, 0, s))
    pre = oracle.preprocess(p, cam, 16)
    sx, sy = np.exp(np.float32(ls[0])), np.exp(np.float32(ls[1]))
    a = (100 * float(sy) / z) ** 2 + 0.3
    cc = (100 * float(sx) / z) ** 2 + 0.3
    q32 = np.array([c, 0, 0, s], np.float32).astype(np.float64)
    assert np.allclose(pre["conic"][0], [1 / a, 0, 1 / cc], rtol=1e-6, atol=1e-9) or \
        np.linalg.norm(q32) != 1.0


def test_pinhole_projection_and_cull():
    cam = scenes.camera(128, 96, 90.0, 110.0, 60.0, 50.0)
    p = _one([0.7, -0.4, 3.0], [np.log(0.05)] * 3)
    pre = oracle.preprocess(p, cam, 16)
    assert np.allclose(pre["mean2d"][0], [90 * 0.7 / 3 + 60, 110 * -0.4 / 3 + 50], atol=1e-6)
    behind = _one([0.0, 0.0, 0.1], [np.log(0.05)] * 3)
    assert oracle.preprocess(behind, cam, 16)["radius"][0] == 0
    assert oracle.preprocess(behind, cam, 16)["touched"][0] == 0


def test_rect_by_hand():
    """Tile rectangle [floor((u-r)/T), floor((u+r+T-1)/T)) clamped to the grid."""
    cam = scenes.camera(64, 48, 100.0, 100.0, 32.0, 24.0)
    p = _one([0.0, 0.0, 4.0], [np.log(0.08)] * 3)   # v = 4.3, r = ceil(3 sqrt(4.3+0.316)) = 7
    pre = oracle.preprocess(p, cam, 16, cull=False)
    r = pre["radius"][0]
    assert r == 7
    u = 32.0
    assert list(pre["rect"][0]) == [int(np.floor((u - r) / 16)), int(np.floor((24 - r) / 16)),
                                    int(np.floor((u + r + 15) / 16)), int(np.floor((24 + r + 15) / 16))]
    assert pre["touched"][0] == 2     # x: tiles 1,2 (px 25..39); y: tile 1 (px 17..31)


# --------------------------------------------------------------------------- binning
def test_binning_equals_bruteforce_and_stable_sort():
    sc = scenes.small_frustum()
    pre = oracle.preprocess(sc["params"], sc["cam"], 16, cull=False)
    bins = oracle.bin_instances(pre, sc["cam"])
    TX, TY = bins["TX"], bins["TY"]
    keys, vals = [], []
    for g in range(len(pre["touched"])):
        if pre["touched"][g] == 0:
            continue
        x0, y0, x1, y1 = pre["rect"][g]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                keys.append((np.uint64(ty * TX + tx) << np.uint64(32)) | np.uint64(pre["depth_bits"][g]))
                vals.append(g)
    keys = np.array(keys, np.uint64)
    vals = np.array(vals, np.uint32)
    order = np.argsort(keys, kind="stable")
    assert bins["I"] == len(keys) > 1000
    assert np.array_equal(bins["keys"], keys[order])
    assert np.array_equal(bins["vals"], vals[order])
    tiles = (keys[order] >> np.uint64(32)).astype(np.int64)
    for t in range(TX * TY):
        idx = np.nonzero(tiles == t)[0]
        if len(idx):
            assert tuple(bins["ranges"][t]) == (idx[0], idx[-1] + 1)
        else:
            assert tuple(bins["ranges"][t]) == (0, 0)
    # depth bits of positive floats order like the floats
    z = pre["depth"][pre["touched"] > 0].astype(np.float32)
    b = pre["depth_bits"][pre["touched"] > 0]
    assert np.array_equal(np.argsort(z, kind="stable"), np.argsort(b, kind="stable"))


# --------------------------------------------------------------------------- compositing
def test_single_gaussian_closed_form():
    """C(rho) = rgb * min(0.99, o exp(-|rho-mu'|^2 / (2v))) inside the rect and
    above 1/255, else 0; D = z O; O + T_final = 1."""
    cam = scenes.camera(64, 48, 100.0, 100.0, 32.0, 24.0)
    dc = (np.array([0.8, 0.3, 0.1]) - 0.5) / oracle.SH_C0
    p = _one([0.0, 0.0, 4.0], [np.log(0.08)] * 3, logit=1.5, dc=dc)
    pre, bins, img = oracle.forward(p, cam, 16)
    v = (100 * float(np.exp(np.float32(np.log(0.08)))) / 4) ** 2 + 0.3
    o = 1 / (1 + np.exp(-float(np.float32(1.5))))
    rgb = np.float32(dc).astype(np.float64) * oracle.SH_C0 + 0.5
    x0, y0, x1, y1 = pre["rect"][0]
    yy, xx = np.mgrid[0:48, 0:64]
    inside = (xx // 16 >= x0) & (xx // 16 < x1) & (yy // 16 >= y0) & (yy // 16 < y1)
    a = np.minimum(0.99, o * np.exp(-((xx - 32.0) ** 2 + (yy - 24.0) ** 2) / (2 * v)))
    a = np.where(inside & (a >= 1 / 255), a, 0.0)
    assert np.allclose(img["color"], a[..., None] * rgb, atol=1e-12)
    assert np.allclose(img["depth"], 4.0 * img["opacity"], atol=1e-12)
    assert np.allclose(img["opacity"] + img["T_final"], 1.0, atol=1e-15)


def test_partition_of_unity_and_bruteforce():
    sc = scenes.small_frustum()
    pre, bins, img = oracle.forward(sc["params"], sc["cam"], 16)
    assert np.abs(img["opacity"] + img["T_final"] - 1).max() < 1e-12
    assert (img["T_final"] >= 1e-4 * (1 - 1e-12)).all()
    bf = oracle.render_bruteforce(pre, sc["cam"], use_rect=True)
    for k in ("color", "depth", "opacity", "T_final", "n_contrib"):
        if k == "n_contrib":
            continue   # positions differ between a per-tile and a per-pixel list
        assert np.array_equal(img[k], bf[k]), k
    assert np.array_equal(img["n_contrib"] > 0, bf["n_contrib"] > 0)


def test_order_invariance():
    sc = scenes.small_frustum()
    p = sc["params"]
    perm = np.random.default_rng(5).permutation(len(p["logits"]))
    q = {k: v[perm] for k, v in p.items()}
    a = oracle.forward(p, sc["cam"], 16)[2]
    b = oracle.forward(q, sc["cam"], 16)[2]
    pre = oracle.preprocess(p, sc["cam"], 16)
    z = pre["depth_bits"][pre["touched"] > 0]
    assert len(np.unique(z)) == len(z)
    for k in ("color", "depth", "opacity", "T_final", "n_contrib"):
        assert np.array_equal(a[k], b[k]), k


def test_tile_size_invariance_of_image():
    """Tiling is an acceleration: with the same contributor sets, the image does
    not depend on the tile side (checked away from rect-truncation effects)."""
    sc = scenes.small_frustum()
    imgs = [oracle.forward(sc["params"], sc["cam"], ts)[2]["color"] for ts in (8, 16, 32)]
    # Rect truncation can differ per tile size; most pixels agree exactly.
    for im in imgs[1:]:
        same = np.all(np.abs(im - imgs[0]) < 1e-12, axis=-1)
        assert same.mean() > 0.9


# --------------------------------------------------------------------------- loss
def _window():
    d = np.arange(11) - 5
    w = np.exp(-d * d / (2 * 1.5 ** 2))
    return w / w.sum()


def test_loss_identity_and_constant_images():
    H, W = 40, 48
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 1, (H, W, 3))
    E = np.hstack([np.eye(3), np.zeros((3, 1))])
    L = oracle.loss(img, img.astype(np.float32).astype(np.float64), E)
    # same image (to float32 rounding) -> SSIM = 1, D-SSIM = 0, L1 ~ 0
    L = oracle.loss(img.astype(np.float32).astype(np.float64), img.astype(np.float32), E)
    assert abs(L["ssim"] - 1) < 1e-12 and abs(L["loss"]) < 1e-12
    # constant images: closed-form SSIM map including the zero padding
    p, q = 0.6, 0.3
    x = np.full((H, W, 3), p)
    y = np.full((H, W, 3), q, np.float32)
    L = oracle.loss(x, y, E)
    w = _window()
    sx = np.array([w[max(0, 5 - i):min(11, W - i + 5)].sum() for i in range(W)])
    sy = np.array([w[max(0, 5 - i):min(11, H - i + 5)].sum() for i in range(H)])
    s = sy[:, None] * sx[None, :]
    qq = float(np.float32(q))
    C1, C2 = 1e-4, 9e-4
    S = ((2 * p * qq * s * s + C1) * (2 * p * qq * s * (1 - s) + C2)) / \
        ((p * p * s * s + qq * qq * s * s + C1) * ((p * p + qq * qq) * s * (1 - s) + C2))
    assert abs(L["ssim"] - S.mean()) < 1e-12
    assert abs(L["l1"] - abs(p - qq)) < 1e-12
    assert abs(L["loss"] - (0.8 * abs(p - qq) + 0.2 * (1 - S.mean()))) < 1e-12
    # interior pixels: SSIM = (2pq + C1) / (p^2 + q^2 + C1)
    interior = S[5:-5, 5:-5]
    assert np.allclose(interior, (2 * p * qq + C1) / (p * p + qq * qq + C1), atol=1e-12)


def test_loss_matches_separable_library_filtering():
    """On random images the oracle's Eq. 9 equals the same statistics taken with
    scipy's separable correlation (zero padding, the 11-tap Gaussian window of
    sigma 1.5): a wrong window, padding, axis or SSIM term would differ."""
    from scipy.ndimage import correlate1d
    rng = np.random.default_rng(13)
    H, W = 37, 29
    C = rng.uniform(0, 1, (H, W, 3))
    T = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    E = np.hstack([np.eye(3), np.zeros((3, 1))])
    w = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    w /= w.sum()

    def blur(a):
        return correlate1d(correlate1d(a, w, axis=0, mode="constant"), w, axis=1, mode="constant")

    x, y = C, T.astype(np.float64)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ssim = []
    for c in range(3):
        xc, yc = x[..., c], y[..., c]
        mx, my = blur(xc), blur(yc)
        sxx, syy, sxy = blur(xc * xc) - mx * mx, blur(yc * yc) - my * my, blur(xc * yc) - mx * my
        ssim.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2)))
    S = float(np.mean(ssim))
    l1 = float(np.mean(np.abs(x - y)))
    L = oracle.loss(C, T, E)
    assert abs(L["ssim"] - S) < 1e-12
    assert abs(L["l1"] - l1) < 1e-12
    assert abs(L["loss"] - (0.8 * l1 + 0.2 * (1 - S))) < 1e-12


def test_loss_exposure_reduces_to_affine():
    """E = [aI | b 1] on C equals the plain loss of a C + b."""
    rng = np.random.default_rng(3)
    C = rng.uniform(0, 1, (24, 20, 3))
    t = rng.uniform(0, 1, (24, 20, 3)).astype(np.float32)
    a, b = 0.75, 0.0625
    E = np.hstack([a * np.eye(3), np.full((3, 1), b)])
    I = np.hstack([np.eye(3), np.zeros((3, 1))])
    assert abs(oracle.loss(C, t, E)["loss"] - oracle.loss(a * C + b, t, I)["loss"]) < 1e-14


def test_loss_gradient_fd():
    rng = np.random.default_rng(4)
    H, W = 22, 26
    C = rng.uniform(0, 1, (H, W, 3))
    t = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    E = np.hstack([np.eye(3) + rng.normal(0, 0.1, (3, 3)), rng.normal(0, 0.05, (3, 1))])
    E = E.astype(np.float32).astype(np.float64)
    L = oracle.loss(C, t, E)
    h = 1e-6
    for _ in range(40):
        i, j, c = rng.integers(H), rng.integers(W), rng.integers(3)
        Cp, Cm = C.copy(), C.copy()
        Cp[i, j, c] += h
        Cm[i, j, c] -= h
        fd = (oracle.loss(Cp, t, E)["loss"] - oracle.loss(Cm, t, E)["loss"]) / (2 * h)
        assert abs(fd - L["dL_dC"][i, j, c]) <= 1e-6 * abs(L["dL_dC"][i, j, c]) + 1e-10
    # exposure: E is float32 inside the oracle, so perturb at float32-exact steps
    for r in range(3):
        for k in range(4):
            Ep, Em = E.copy(), E.copy()
            hh = 2.0 ** -18      # small enough that no L1 residual changes sign
            Ep[r, k] += hh
            Em[r, k] -= hh
            fd = (oracle.loss(C, t, Ep)["loss"] - oracle.loss(C, t, Em)["loss"]) / (2 * hh)
            assert abs(fd - L["dL_dE"][r, k]) <= 1e-4 * abs(L["dL_dE"][r, k]) + 1e-8


# --------------------------------------------------------------------------- backward (FD)
def _small_scene(seed=7, n=300, W=64, H=48, deg=3):
    rng = np.random.default_rng(seed)
    base = scenes.camera(W, H, 60.0, 60.0, W / 2, H / 2)
    p = scenes.random_gaussians(rng, n, base, deg, 0.3, z_range=(1.0, 6.0), log_scale_mean=-2.3,
                                log_scale_std=0.4)
    w = rng.normal(0, 0.03, 3)
    cam = scenes.camera(W, H, 60.0, 60.0, W / 2 + 0.3, H / 2 - 0.2, R=scenes._rodrigues(w),
                        t=rng.normal(0, 0.05, 3))
    target = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    E = np.hstack([np.eye(3) + rng.normal(0, 0.05, (3, 3)), rng.normal(0, 0.02, (3, 1))])
    p64 = {k: v.astype(np.float64) for k, v in p.items()}
    return p64, cam, target, E.astype(np.float32)


def _eval(p, cam, target, E):
    pre, bins, img = oracle.forward(p, cam, 16)
    L = oracle.loss(img["color"], target, E)["loss"]
    sig = (pre["radius"].tobytes(), pre["rect"].tobytes(), pre["flags"].tobytes(),
           img["n_contrib"].tobytes(), img["signature"].tobytes())
    return L, sig


def _fd_check(fn_pm, analytic, h, sig0):
    (Lp, sp), (Lm, sm) = fn_pm(+h), fn_pm(-h)
    if sp != sig0 or sm != sig0:
        return None
    fd = (Lp - Lm) / (2 * h)
    return fd, analytic


@pytest.mark.slow
def test_backward_matches_central_fd_every_parameter_class():
    p, cam, target, E = _small_scene()
    r = oracle.loss_and_grads(p, cam, target, E, 16)
    g = r["grads"]
    L0, sig0 = _eval(p, cam, target, E)
    assert abs(L0 - r["loss"]["loss"]) < 1e-15
    vis = np.nonzero(r["pre"]["radius"] > 0)[0]
    rng = np.random.default_rng(11)
    results = {}
    for name, comps in (("means", 3), ("log_scales", 3), ("quats", 4), ("logits", 1), ("sh", 48)):
        errs, skipped = [], 0
        for _ in range(14):
            gi = int(rng.choice(vis))
            c = int(rng.integers(comps))

            def fn(h, gi=gi, c=c, name=name):
                q = {k: v.copy() for k, v in p.items()}
                arr = q[name].reshape(len(q["logits"]), -1)
                arr[gi, c] += h
                q[name] = arr.reshape(p[name].shape)
                return _eval(q, cam, target, E)
            an = g[name].reshape(len(p["logits"]), -1)[gi, c]
            out = _fd_check(fn, an, 1e-5, sig0)
            if out is None:
                skipped += 1
                continue
            fd, an = out
            errs.append(abs(fd - an) / max(abs(an), 1e-9))
        assert len(errs) >= 7, (name, skipped)
        results[name] = np.median(errs)
        assert np.median(errs) < 1e-5 and max(errs) < 1e-3, (name, errs)
    # pose: left perturbation exp(h xi^) T_cw
    R0, t0 = np.asarray(cam["R"]), np.asarray(cam["t"])
    for k in range(6):
        def fn(h, k=k):
            xi = np.zeros(6)
            xi[k] = h
            Rd = scenes._rodrigues(xi[3:])
            c2 = dict(cam, R=Rd @ R0, t=Rd @ t0 + xi[:3])
            return _eval(p, c2, target, E)
        out = _fd_check(fn, g["pose"][k], 1e-6, sig0)
        assert out is not None
        fd, an = out
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-9, (k, fd, an)


def test_backward_2d_depth_and_opacity_outputs_fd():
    """dL/dD and dL/dO paths: L = <wD, D> + <wO, O> checked by FD on the means."""
    p, cam, target, E = _small_scene(seed=9, n=120)
    rng = np.random.default_rng(12)
    W, H = cam["width"], cam["height"]
    wD = rng.normal(size=(H, W))
    wO = rng.normal(size=(H, W))
    pre, bins, img = oracle.forward(p, cam, 16)
    g = oracle.backward(p, cam, pre, bins, np.zeros((H, W, 3)), wD, wO)
    sig0 = (pre["radius"].tobytes(), pre["flags"].tobytes(), img["signature"].tobytes())
    vis = np.nonzero(pre["radius"] > 0)[0]
    ok = 0
    for gi in vis[:12]:
        for c in range(3):
            vals = []
            for h in (1e-5, -1e-5):
                q = {k: v.copy() for k, v in p.items()}
                q["means"][gi, c] += h
                pr, bi, im = oracle.forward(q, cam, 16)
                s = (pr["radius"].tobytes(), pr["flags"].tobytes(), im["signature"].tobytes())
                vals.append(((wD * im["depth"]).sum() + (wO * im["opacity"]).sum(), s))
            if vals[0][1] != sig0 or vals[1][1] != sig0:
                continue
            fd = (vals[0][0] - vals[1][0]) / 2e-5
            an = g["means"][gi, c]
            assert abs(fd - an) <= 1e-5 * abs(an) + 1e-8
            ok += 1
    assert ok >= 20


# --------------------------------------------------------------------------- Adam
def test_adam_first_step_closed_form_and_mask():
    rng = np.random.default_rng(6)
    p = rng.normal(size=(50, 3))
    g = rng.normal(size=(50, 3))
    m, v = np.zeros_like(p), np.zeros_like(p)
    mask = (rng.uniform(size=50) < 0.5).astype(np.uint8)
    p0 = p.copy()
    oracle.adam_update(p, m, v, g, 1e-3, 1, mask)
    upd = p0 - 1e-3 * g / (np.abs(g) + 1e-15)
    assert np.allclose(p[mask == 1], upd[mask == 1], rtol=0, atol=1e-15)
    assert np.array_equal(p[mask == 0], p0[mask == 0])
    assert np.all(m[mask == 0] == 0) and np.all(v[mask == 0] == 0)


def test_first_step_moves_each_group_by_its_learning_rate():
    """Sec. III-C 3 / IV-A: one step from zero moments is Adam's first step on
    the step's gradient, so every parameter the view sees moves by its group's
    rate against the sign of its gradient (3DGS's rates, not decayed: means
    1.6e-4, SH DC 2.5e-3 and higher bands 1/20 of it, opacity 0.05, scale 5e-3,
    rotation 1e-3; exposure 1e-3), and a Gaussian the view does not see stays
    put (sparse Adam, Sec. III-D 2).  A swapped rate between groups, or between
    the SH DC and higher bands, fails here."""
    sc = scenes.diff_check(n=600, width=96, height=72, f=80.0)
    params, cam, target, E = sc["params"], sc["cam"], sc["target"], sc["E"]
    params = {k: np.array(v) for k, v in params.items()}
    params["means"][:60] = -params["means"][:60]   # behind the camera: culled
    st = oracle.new_state(params, E)
    r = oracle.optimize_step(params, st, cam, target, E, step=1)
    g = r["grads"]
    vis = r["pre"]["radius"] > 0
    assert 0 < vis.sum() < len(vis)
    rates = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "logits": 0.05}
    for name, lr in rates.items():
        d = st["p"][name] - np.asarray(params[name], np.float64)
        gg = np.asarray(g[name], np.float64)
        on = vis.reshape((-1,) + (1,) * (gg.ndim - 1)) & (np.abs(gg) > 1e-8)
        on = np.broadcast_to(on, gg.shape)
        assert on.sum() > 0, name
        assert np.allclose(d[on], -lr * np.sign(gg[on]), rtol=1e-6, atol=0), name
        assert np.all(d[~vis] == 0), name
    d = st["p"]["sh"] - np.asarray(params["sh"], np.float64)
    gs = np.asarray(g["sh"], np.float64)
    for sl, lr in ((slice(0, 1), 2.5e-3), (slice(1, None), 2.5e-3 / 20)):
        dd, gg = d[:, sl], gs[:, sl]
        on = vis[:, None, None] & (np.abs(gg) > 1e-8)
        assert on.sum() > 0
        assert np.allclose(dd[on], -lr * np.sign(gg[on]), rtol=1e-6, atol=0)
        assert np.all(dd[~vis] == 0)
    dE = st["p"]["E"] - np.asarray(E, np.float64).reshape(3, 4)
    gE = r["loss"]["dL_dE"]
    assert np.allclose(dE, -1e-3 * np.sign(gE), rtol=1e-6, atol=0)


def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    p = rng.normal(size=(40,))
    m, v = np.zeros_like(p), np.zeros_like(p)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=5e-3, betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 6):
        g = rng.normal(size=(40,))
        oracle.adam_update(p, m, v, g, 5e-3, step)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    assert np.allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------- step composition
_GAUSS_KEYS = ("means", "log_scales", "quats", "logits", "sh")


def _two_sided_scene():
    """Gaussians in front of a camera A (identity pose, looking down +z), a
    mirrored copy in front of a camera B turned 180 degrees about y (looking
    down -z), and a few far off to the side that neither camera sees."""
    sc = scenes.small_frustum(seed=11, n=300, width=64, height=48, f=50.0)
    p = sc["params"]
    back = {k: v.copy() for k, v in p.items()}
    back["means"] = back["means"] * np.array([-1, 1, -1], np.float32)
    side = {k: v[:20].copy() for k, v in p.items()}
    side["means"] = side["means"] + np.array([500.0, 0, 0], np.float32)
    params = {k: np.ascontiguousarray(np.concatenate([p[k], back[k], side[k]])) for k in p}
    camA = sc["cam"]
    camB = scenes.camera(64, 48, 50.0, R=np.diag([-1.0, 1.0, -1.0]))
    return params, camA, camB, sc["target"], sc["E"].astype(np.float64)


def _as_params(state):
    return {k: state["p"][k].astype(np.float32) for k in _GAUSS_KEYS}


def test_window_of_one_view_is_the_plain_step():
    """Sec. III-C 3 optimises one keyframe per iteration; a window of one view
    must reduce to exactly that step (mean over one view, union of one mask)."""
    params, camA, _, tgt, E = _two_sided_scene()
    st = oracle.new_state(params, E)
    r = oracle.optimize_step(params, st, camA, tgt, E, 1)
    sw = oracle.new_window_state(params, 1)
    sw["p"]["E"][0] = E.copy()
    rw = oracle.optimize_window(params, sw, [camA], [tgt], 1)
    assert rw["loss"] == r["loss"]["loss"]
    for k in _GAUSS_KEYS:
        for d in ("p", "m", "v"):
            assert np.array_equal(st[d][k], sw[d][k]), (k, d)
    for d in ("p", "m", "v"):
        assert np.array_equal(st[d]["E"], sw[d]["E"][0]), d


def test_window_of_a_repeated_view_moves_the_map_like_one_view():
    """Two copies of one view: the mean gradient is the view's own (g/2 + g/2
    = g exactly), so the Gaussians take the plain step bit for bit; each copy's
    exposure takes a first Adam step on half the gradient, which is the same
    -lr sign(g) move up to eps."""
    params, camA, _, tgt, E = _two_sided_scene()
    st = oracle.new_state(params, E)
    r = oracle.optimize_step(params, st, camA, tgt, E, 1)
    sw = oracle.new_window_state(params, 2)
    sw["p"]["E"] = [E.copy(), E.copy()]
    rw = oracle.optimize_window(params, sw, [camA, camA], [tgt, tgt], 1)
    assert rw["loss"] == r["loss"]["loss"]
    for k in _GAUSS_KEYS:
        assert np.array_equal(st["p"][k], sw["p"][k]), k
    for v in range(2):
        assert np.allclose(sw["p"]["E"][v], st["p"]["E"], rtol=0, atol=1e-15)


def test_sparse_adam_mask_is_the_union_of_the_window_views():
    """Sparse Adam (Sec. III-D 2) updates exactly the Gaussians with a non-zero
    radius in some view of the step: those seen only by B move in an A+B
    window and stay bitwise put (moments too) in a step on A alone; those that
    no camera sees never change."""
    params, camA, camB, tgt, E = _two_sided_scene()
    n = params["means"].shape[0]
    visA = oracle.preprocess(params, camA)["radius"] > 0
    visB = oracle.preprocess(params, camB)["radius"] > 0
    onlyB = visB & ~visA
    assert onlyB.sum() > 50 and not (visA | visB)[-20:].any()
    sw = oracle.new_window_state(params, 2)
    rw = oracle.optimize_window(params, sw, [camA, camB], [tgt, tgt], 1)
    assert np.array_equal(rw["visible"], visA | visB)
    moved = np.zeros(n, bool)
    for k in _GAUSS_KEYS:
        d = (sw["p"][k] != params[k].astype(np.float64)).reshape(n, -1).any(1)
        moved |= d
        assert np.all(sw["m"][k].reshape(n, -1)[~(visA | visB)] == 0), k
    assert moved[onlyB].all() and not moved[~(visA | visB)].any()
    st = oracle.new_state(params, E)
    oracle.optimize_step(params, st, camA, tgt, E, 1)
    for k in _GAUSS_KEYS:
        rows = st["p"][k].reshape(n, -1)[~visA]
        assert np.array_equal(rows, params[k].astype(np.float64).reshape(n, -1)[~visA]), k
        assert np.all(st["v"][k].reshape(n, -1)[~visA] == 0), k


def test_dense_adam_keeps_moving_gaussians_out_of_view():
    """The dense mode (the "w/o acc" row of Table II) applies Adam to every Gaussian:
    one seen by A in step 1 but not by B in step 2 keeps moving on its first
    moment in step 2, while sparse Adam leaves it exactly where step 1 put it."""
    params, camA, camB, tgt, E = _two_sided_scene()
    n = params["means"].shape[0]
    visA = oracle.preprocess(params, camA)["radius"] > 0
    visB = oracle.preprocess(params, camB)["radius"] > 0
    onlyA = visA & ~visB
    assert onlyA.sum() > 50
    out = {}
    for sparse in (True, False):
        st = oracle.new_state(params, E)
        oracle.optimize_step(params, st, camA, tgt, E, 1, sparse=sparse)
        after1 = {(d, k): st[d][k].copy() for d in ("p", "m", "v") for k in _GAUSS_KEYS}
        oracle.optimize_step(_as_params(st), st, camB, tgt, st["p"]["E"].copy(), 2, sparse=sparse)
        out[sparse] = (after1, st)
    after1, st = out[True]
    for k in _GAUSS_KEYS:
        for d in ("p", "m", "v"):
            assert np.array_equal(st[d][k].reshape(n, -1)[onlyA], after1[d, k].reshape(n, -1)[onlyA]), (d, k)
    after1, st = out[False]
    m1 = after1["m", "means"].reshape(n, -1)[onlyA]
    v1 = after1["v", "means"].reshape(n, -1)[onlyA]
    assert (m1 != 0).any(1).mean() > 0.9
    # no gradient in step 2: m2 = b1 m1, v2 = b2 v1, and the bias-corrected move
    # of Adam (Kingma and Ba 2015, Algorithm 1) is lr m2/(1-b1^2) / (sqrt(v2/(1-b2^2)) + eps)
    assert np.array_equal(st["m"]["means"].reshape(n, -1)[onlyA], 0.9 * m1)
    expect = 1.6e-4 * (0.9 * m1 / (1 - 0.9 ** 2)) / (np.sqrt(0.999 * v1 / (1 - 0.999 ** 2)) + 1e-15)
    moved = after1["p", "means"].reshape(n, -1)[onlyA] - st["p"]["means"].reshape(n, -1)[onlyA]
    assert np.allclose(moved, expect, rtol=1e-9, atol=1e-18)
    assert (np.abs(moved).max(1)[(m1 != 0).any(1)] > 0).all()


# --------------------------------------------------------------------------- sky / expansion
def test_sky_points_hemisphere_and_nearest_neighbour():
    from scipy.spatial import cKDTree
    from scipy.stats import kstest
    xyz, nn = oracle.sky_points(1000, 1e4, seed=5)
    r = np.linalg.norm(xyz.astype(np.float64), axis=1)
    assert np.allclose(r, 1e4, rtol=1e-6)
    assert (xyz[:, 2] >= 0).all()
    d, _ = cKDTree(xyz.astype(np.float64)).query(xyz.astype(np.float64), k=2)
    assert np.allclose(nn, d[:, 1], rtol=1e-12)
    # area-uniform on the hemisphere <=> height uniform on [0, R]
    assert kstest(xyz[:, 2] / 1e4, "uniform").pvalue > 1e-3


def test_expand_mask_special_cases():
    cam = scenes.camera(64, 48, 60.0)
    rng = np.random.default_rng(9)
    pts = np.stack([rng.uniform(-2, 2, 400), rng.uniform(-2, 2, 400), rng.uniform(-1, 6, 400)], 1)
    pts = pts.astype(np.float32)
    keep_all, depth, k = oracle.expand_mask(pts, cam, None)
    assert k == (pts[:, 2] > 0.2).sum() and np.array_equal(keep_all, pts[:, 2] > np.float32(0.2))
    zero = np.zeros((48, 64))
    keep0, _, k0 = oracle.expand_mask(pts, cam, zero)
    u = 60 * pts[:, 0] / pts[:, 2] + 32
    v = 60 * pts[:, 1] / pts[:, 2] + 24
    inside = (pts[:, 2] > 0.2) & (np.floor(u + 0.5) >= 0) & (np.floor(u + 0.5) < 64) & \
        (np.floor(v + 0.5) >= 0) & (np.floor(v + 0.5) < 48)
    assert abs(k0 - inside.sum()) <= 2    # float32 rounding at the border
    keep1, _, k1 = oracle.expand_mask(pts, cam, np.ones((48, 64)))
    assert k1 == 0


def test_init_gaussians_follows_paper():
    xyz = np.array([[1.0, 2.0, 3.0]], np.float32)
    rgb = np.array([[0.2, 0.5, 0.9]], np.float32)
    g = oracle.init_gaussians(xyz, rgb, np.array([8.0]), 400.0)
    assert np.allclose(g["log_scales"], np.log(8.0 / 400.0))
    assert np.allclose(g["quats"], [[1, 0, 0, 0]])
    assert np.allclose(1 / (1 + np.exp(-g["logits"].astype(np.float64))), 0.1, atol=1e-7)
    assert np.allclose(g["sh"][0, 0] * oracle.SH_C0 + 0.5, rgb[0], atol=1e-6)
    assert np.all(g["sh"][0, 1:] == 0)


def test_decision_exp_within_two_ulp_of_exp():
    """The float32 exp of the decision path is within 2 ulp of the exact
    exponential (evaluated in double) over the range log-scales take."""
    xs = np.concatenate([np.linspace(-30, 30, 4001), np.random.default_rng(0).uniform(-12, 8, 4000)])
    xs = xs.astype(np.float32)
    for x in xs:
        y = oracle.expf_decision(x)
        ref = np.exp(np.float64(x))
        ulp = np.spacing(np.float32(ref))
        assert abs(y - ref) <= 2 * ulp, (x, y, ref)
    assert oracle.expf_decision(0.0) == 1.0
    assert oracle.expf_decision(np.float32(np.log(2.0))) == np.float32(2.0) or \
        abs(oracle.expf_decision(np.float32(np.log(2.0))) - 2.0) <= 2 * np.spacing(np.float32(2.0))


def test_decision_log_within_two_ulp_of_log():
    """The float32 log of the decision path is within 4 ulp of the exact
    logarithm (double) from subnormals to 1e30 (a wrong coefficient or
    reduction step would be off by far more), and exact at 1."""
    rng = np.random.default_rng(1)
    xs = np.concatenate([10.0 ** rng.uniform(-44, 30, 6000), rng.uniform(0.5, 2.0, 4000),
                         np.linspace(0.01, 300.0, 3000)]).astype(np.float32)
    for x in xs:
        if x <= 0:
            continue
        y = oracle.logf_decision(x)
        ref = np.log(np.float64(x))
        ulp = np.spacing(np.float32(abs(ref))) if ref != 0 else np.float32(1e-45)
        assert abs(y - ref) <= 4 * ulp + 1e-12, (x, y, ref)
    assert oracle.logf_decision(1.0) == 0.0
    for k in (-20, -1, 1, 7, 30):
        assert abs(oracle.logf_decision(np.float32(2.0 ** k)) - k * np.log(2.0)) <= 4 * np.spacing(np.float32(abs(k) * 0.7))
    assert oracle.logf_decision(0.0) == -np.inf


def _tile_pairs(bins):
    TX = bins["TX"]
    tiles = (bins["keys"] >> np.uint64(32)).astype(np.int64)
    return set(zip(bins["vals"].astype(np.int64).tolist(), tiles.tolist())), TX


@pytest.mark.parametrize("scene", ["small_frustum", "diff_check"])
@pytest.mark.parametrize("tile", [8, 16])
def test_exact_tile_culling_drops_only_invisible_tiles(scene, tile):
    """Every (Gaussian, tile) pair the exact culling drops has alpha < 1/255
    at each pixel centre of the tile, evaluated independently in double from
    the double path's mean, conic and opacity; and culling drops some pairs."""
    sc = getattr(scenes, scene)()
    cam = sc["cam"]
    pre_c = oracle.preprocess(sc["params"], cam, tile, cull=True)
    pre_f = oracle.preprocess(sc["params"], cam, tile, cull=False)
    assert np.array_equal(pre_c["radius"], pre_f["radius"])
    assert (pre_c["touched"] <= pre_f["touched"]).all()
    kept, TX = _tile_pairs(oracle.bin_instances(pre_c, cam))
    full, _ = _tile_pairs(oracle.bin_instances(pre_f, cam))
    assert kept <= full
    dropped = full - kept
    assert len(dropped) > 0.05 * len(full), (len(dropped), len(full))
    W, H = cam["width"], cam["height"]
    ys, xs = np.mgrid[0:tile, 0:tile]
    for g, t in dropped:
        px = (t % TX) * tile + xs
        py = (t // TX) * tile + ys
        dx = pre_f["mean2d"][g, 0] - px
        dy = pre_f["mean2d"][g, 1] - py
        A, B, C = pre_f["conic"][g]
        q = A * dx * dx + 2 * B * dx * dy + C * dy * dy
        amax = (pre_f["opacity"][g] * np.exp(-0.5 * q)).max()
        assert amax < 1.0 / 255.0, (g, t, amax)


@pytest.mark.parametrize("scene", ["small_frustum", "diff_check"])
def test_exact_tile_culling_keeps_the_image(scene):
    """Culling only removes pairs that every pixel would skip: colour, depth,
    opacity and final transmittance are bit-identical with and without it."""
    sc = getattr(scenes, scene)()
    a = oracle.forward(sc["params"], sc["cam"], 16, cull=True)[2]
    b = oracle.forward(sc["params"], sc["cam"], 16, cull=False)[2]
    for k in ("color", "depth", "opacity", "T_final"):
        assert np.array_equal(a[k], b[k]), k
