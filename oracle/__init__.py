"""CPU oracle for the Gaussian-LIC map optimisation step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product path (the CUDA library and its
Python binding) never does: it shares no code, header, table or constant with
this file or with ``gl_oracle.c``.

The arithmetic lives in ``gl_oracle.c`` (plain C, double precision, with the
integer-deciding projection in float32 without contraction); this module
compiles it with gcc and wraps it for numpy.  Each function cites the passage
of arXiv 2404.06926 it restates.

Parameter dictionaries (any float dtype; converted to double.  The float32
decision path rounds them to float32 itself, so parity inputs should be
float32-representable, as the map stores them):
  means (N,3), log_scales (N,3), quats (N,4) as (w,x,y,z), logits (N,),
  sh (N,K,3) with K = (deg+1)^2.
Camera dictionaries: fx, fy, cx, cy, width, height, R (3,3) world->camera,
  t (3,), so that x_c = R x_w + t (Eq. 2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gl_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Readings of the paper's silent constants, as the oracle states them.
Z_NEAR = 0.2
DILATION = 0.3
ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4
LAMBDA_DSSIM = 0.2          # Sec. IV-A
TAU = 0.99                  # Sec. IV-A
OPACITY_FG = 0.1            # o_a, Sec. IV-A
OPACITY_SKY = 0.7           # o_b, Sec. IV-A
SKY_RADIUS = 1.0e4          # R, Sec. IV-A
SH_C0 = 0.5 / np.sqrt(np.pi)


def build(force: bool = False) -> str:
    """Compile gl_oracle.c into a shared object (gcc, no FP contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-Wno-unknown-pragmas",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


class _Cam(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32),
                ("R", C.c_double * 9), ("t", C.c_double * 3)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        lib.orc_sh_basis.argtypes = [i32, dbl, dbl, dbl, P, P]
        lib.orc_preprocess.argtypes = [i64, i32, P, P, P, P, P, P, i32, i32] + [P] * 11
        lib.orc_num_instances.argtypes = [i64, P]
        lib.orc_num_instances.restype = i64
        lib.orc_bin.argtypes = [i64, P, P, P, P, i32, i32, i32, i32, P, P, P]
        lib.orc_bin.restype = i64
        lib.orc_render.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, dbl, dbl, P, P, P, P, P, P, P]
        lib.orc_render_bruteforce.argtypes = [i32, i32, i32, i64, P, P, P, P, P, P, P, P, i32,
                                              P, P, P, P, P]
        lib.orc_loss.argtypes = [i32, i32, P, P, P, dbl, P, P, P, P]
        lib.orc_loss.restype = dbl
        lib.orc_backward_2d.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, P, P, P, i64, P]
        lib.orc_backward_params.argtypes = [i64, i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_adam.argtypes = [i64, i32, P, P, P, P, P, dbl, dbl, dbl, dbl, i64]
        lib.orc_expf_decision.argtypes = [C.c_float]
        lib.orc_expf_decision.restype = C.c_float
        lib.orc_logf_decision.argtypes = [C.c_float]
        lib.orc_logf_decision.restype = C.c_float
        lib.orc_uniform.argtypes = [C.c_uint64, C.c_uint64]
        lib.orc_uniform.restype = dbl
        lib.orc_sky.argtypes = [i64, dbl, C.c_uint64, P, P]
        lib.orc_expand_mask.argtypes = [i64, P, P, P, dbl, P, P]
        lib.orc_expand_mask.restype = i64
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def make_cam(cam: dict) -> _Cam:
    c = _Cam()
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    R = np.asarray(cam["R"], np.float64).reshape(9)
    t = np.asarray(cam["t"], np.float64).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    return c


def sh_degree(params: dict) -> int:
    K = params["sh"].shape[1]
    deg = int(round(np.sqrt(K))) - 1
    assert (deg + 1) ** 2 == K and 0 <= deg <= 3
    return deg


def sh_basis(deg: int, d):
    """Real SH basis to degree 3 at a unit direction, and its gradient."""
    lib = _load()
    Y = np.zeros(16)
    dY = np.zeros(48)
    lib.orc_sh_basis(deg, float(d[0]), float(d[1]), float(d[2]), _p(Y), _p(dY))
    nb = (deg + 1) ** 2
    return Y[:nb].copy(), dY.reshape(16, 3)[:nb].copy()


def _prm(params):
    return (_c(params["means"], np.float64), _c(params["log_scales"], np.float64),
            _c(params["quats"], np.float64), _c(params["logits"], np.float64),
            _c(params["sh"], np.float64))


def tiles(cam: dict, Ts: int):
    return (int(cam["width"]) + Ts - 1) // Ts, (int(cam["height"]) + Ts - 1) // Ts


def preprocess(params: dict, cam: dict, Ts: int = 16, cull: bool = True) -> dict:
    """Eq. 1-3 and the SH colour for every Gaussian (Sec. III-A).  With cull,
    a tile of the 3-sigma rectangle counts only if the Gaussian can reach
    alpha >= 1/255 at one of its pixel centres (exact tile culling)."""
    lib = _load()
    m, ls, q, lg, sh = _prm(params)
    n = m.shape[0]
    deg = sh_degree(params)
    out = dict(radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
               touched=np.zeros(n, np.uint32), depth_bits=np.zeros(n, np.uint32),
               mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
               rgb=np.zeros((n, 3)), depth=np.zeros(n), flags=np.zeros(n, np.uint8),
               cullp=np.zeros((n, 8), np.float32))
    c = make_cam(cam)
    lib.orc_preprocess(n, deg, _p(m), _p(ls), _p(q), _p(lg), _p(sh), C.byref(c), Ts, int(bool(cull)),
                       _p(out["radius"]), _p(out["rect"]), _p(out["touched"]), _p(out["depth_bits"]),
                       _p(out["mean2d"]), _p(out["conic"]), _p(out["opacity"]), _p(out["rgb"]),
                       _p(out["depth"]), _p(out["flags"]), _p(out["cullp"]))
    out["Ts"] = Ts
    out["cull"] = bool(cull)
    return out


def bin_instances(pre: dict, cam: dict) -> dict:
    """(tile | depth) key duplication, stable sort and per-tile ranges (Sec. III-A)."""
    lib = _load()
    n = pre["touched"].shape[0]
    TX, TY = tiles(cam, pre["Ts"])
    I = int(lib.orc_num_instances(n, _p(pre["touched"])))
    keys = np.zeros(max(I, 1), np.uint64)
    vals = np.zeros(max(I, 1), np.uint32)
    ranges = np.zeros((TX * TY, 2), np.uint32)
    lib.orc_bin(n, _p(pre["rect"]), _p(pre["touched"]), _p(pre["depth_bits"]),
                _p(pre["cullp"]) if pre.get("cull", False) else None, pre["Ts"], TX, TY, 1,
                _p(keys), _p(vals), _p(ranges))
    return dict(keys=keys[:I], vals=vals[:I], ranges=ranges, I=I, TX=TX, TY=TY)


def render(pre: dict, bins: dict, cam: dict, amb_alpha_rel: float = 2e-5,
           amb_T_rel: float = 1e-4) -> dict:
    """Front-to-back compositing, Eq. 4-7, per tile in sorted order."""
    lib = _load()
    W, H = int(cam["width"]), int(cam["height"])
    P = W * H
    out = dict(color=np.zeros((H, W, 3)), depth=np.zeros((H, W)), opacity=np.zeros((H, W)),
               T_final=np.zeros((H, W)), n_contrib=np.zeros((H, W), np.int32),
               ambiguous=np.zeros((H, W), np.uint8), signature=np.zeros((H, W), np.uint64))
    vals = bins["vals"] if bins["I"] > 0 else np.zeros(1, np.uint32)
    lib.orc_render(W, H, pre["Ts"], 1, _p(vals), _p(bins["ranges"]), _p(pre["mean2d"]),
                   _p(pre["conic"]), _p(pre["opacity"]), _p(pre["rgb"]), _p(pre["depth"]),
                   amb_alpha_rel, amb_T_rel, _p(out["color"]), _p(out["depth"]),
                   _p(out["opacity"]), _p(out["T_final"]), _p(out["n_contrib"]),
                   _p(out["ambiguous"]), _p(out["signature"]))
    assert P == out["T_final"].size
    return out


def render_bruteforce(pre: dict, cam: dict, use_rect: bool = True) -> dict:
    """Per-pixel global depth sort and direct compositing (a pin, not a path)."""
    lib = _load()
    W, H = int(cam["width"]), int(cam["height"])
    n = pre["touched"].shape[0]
    out = dict(color=np.zeros((H, W, 3)), depth=np.zeros((H, W)), opacity=np.zeros((H, W)),
               T_final=np.zeros((H, W)), n_contrib=np.zeros((H, W), np.int32))
    lib.orc_render_bruteforce(W, H, pre["Ts"], n, _p(pre["rect"]), _p(pre["touched"]),
                              _p(pre["depth_bits"]), _p(pre["mean2d"]), _p(pre["conic"]),
                              _p(pre["opacity"]), _p(pre["rgb"]), _p(pre["depth"]), int(use_rect),
                              _p(out["color"]), _p(out["depth"]), _p(out["opacity"]),
                              _p(out["T_final"]), _p(out["n_contrib"]))
    return out


def loss(color, target, E, lam: float = LAMBDA_DSSIM) -> dict:
    """Eq. 9 with the 3x4 exposure affine E applied to the rendered colour."""
    lib = _load()
    color = _c(color, np.float64)
    H, W = color.shape[:2]
    target = _c(target, np.float32)
    E = _c(np.asarray(E).reshape(12), np.float32)
    dC = np.zeros_like(color)
    dE = np.zeros(12)
    ss = C.c_double()
    l1 = C.c_double()
    L = lib.orc_loss(W, H, _p(color), _p(target), _p(E), lam, _p(dC), _p(dE), C.byref(ss),
                     C.byref(l1))
    return dict(loss=L, dL_dC=dC, dL_dE=dE.reshape(3, 4), ssim=ss.value, l1=l1.value)


def backward(params: dict, cam: dict, pre: dict, bins: dict, dL_dC, dL_dD=None, dL_dO=None) -> dict:
    """Analytic backward of Eq. 1-7 and the SH colour to every parameter and the pose."""
    lib = _load()
    m, ls, q, lg, sh = _prm(params)
    n = m.shape[0]
    deg = sh_degree(params)
    W, H = int(cam["width"]), int(cam["height"])
    g2d = np.zeros((n, 10))
    vals = bins["vals"] if bins["I"] > 0 else np.zeros(1, np.uint32)
    dC = _c(dL_dC, np.float64)
    dD = None if dL_dD is None else _c(dL_dD, np.float64)
    dO = None if dL_dO is None else _c(dL_dO, np.float64)
    lib.orc_backward_2d(W, H, pre["Ts"], 1, _p(vals), _p(bins["ranges"]), _p(pre["mean2d"]),
                        _p(pre["conic"]), _p(pre["opacity"]), _p(pre["rgb"]), _p(pre["depth"]),
                        _p(dC), _p(dD), _p(dO), n, _p(g2d))
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               logits=np.zeros(n), sh=np.zeros(sh.shape, np.float64), pose=np.zeros(6), g2d=g2d)
    c = make_cam(cam)
    lib.orc_backward_params(n, deg, _p(m), _p(ls), _p(q), _p(lg), _p(sh), C.byref(c),
                            _p(pre["radius"]), _p(g2d), _p(out["means"]), _p(out["log_scales"]),
                            _p(out["quats"]), _p(out["logits"]), _p(out["sh"]), _p(out["pose"]))
    return out


def adam_update(p, m, v, g, lr, step, mask=None, b1=0.9, b2=0.999, eps=1e-15):
    """In-place Adam on double arrays; rows with mask == 0 are left untouched."""
    lib = _load()
    assert p.dtype == np.float64 and m.dtype == np.float64 and v.dtype == np.float64
    g = _c(g, np.float64)
    stride = int(np.prod(p.shape[1:])) if p.ndim > 1 else 1
    mk = None if mask is None else _c(mask, np.uint8)
    lib.orc_adam(p.size, stride, _p(mk), _p(p), _p(m), _p(v), _p(g), lr, b1, b2, eps, int(step))


# ---------------------------------------------------------------------------
# Timing build: the float instantiation of gl_oracle.c with OpenMP, timed as
# the CPU baseline of the benchmark (never used as a checker).
# ---------------------------------------------------------------------------
_TIMING_PATH = os.path.join(_OUT_DIR, "liboracle_f32_omp.so")
_tlib = None


def build_timing(force: bool = False) -> str:
    """Compile gl_oracle.c with -DORC_REAL=float -O3 -fopenmp (no FP contraction)."""
    with _lock:
        if (not force and os.path.exists(_TIMING_PATH)
                and os.path.getmtime(_TIMING_PATH) >= os.path.getmtime(_SRC)):
            return _TIMING_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _TIMING_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-DORC_REAL=float",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _TIMING_PATH)
        return _TIMING_PATH


def _load_timing():
    global _tlib
    if _tlib is None:
        lib = C.CDLL(build_timing())
        P = C.c_void_p
        i64, i32, f32 = C.c_int64, C.c_int, C.c_float
        lib.orc_num_threads.restype = i32
        lib.orc_set_num_threads.argtypes = [i32]
        lib.orc_sky.argtypes = [i64, C.c_double, C.c_uint64, P, P]
        lib.orc_preprocess.argtypes = [i64, i32, P, P, P, P, P, P, i32, i32] + [P] * 11
        lib.orc_num_instances.argtypes = [i64, P]
        lib.orc_num_instances.restype = i64
        lib.orc_bin.argtypes = [i64, P, P, P, P, i32, i32, i32, i32, P, P, P]
        lib.orc_bin.restype = i64
        lib.orc_render.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, f32, f32, P, P, P, P, P, P, P]
        lib.orc_loss.argtypes = [i32, i32, P, P, P, f32, P, P, P, P]
        lib.orc_loss.restype = f32
        lib.orc_backward_2d.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, P, P, P, i64, P]
        lib.orc_backward_params.argtypes = [i64, i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_adam.argtypes = [i64, i32, P, P, P, P, P, f32, f32, f32, f32, i64]
        _tlib = lib
    return _tlib


def sky_points_parallel(n: int, radius: float = SKY_RADIUS, seed: int = 0):
    """sky_points by the timing build: the same double arithmetic per point
    (identical results), its brute-force nearest-neighbour loop parallel."""
    lib = _load_timing()
    xyz = np.zeros((n, 3), np.float32)
    nn = np.zeros(n)
    lib.orc_sky(n, radius, C.c_uint64(seed), _p(xyz), _p(nn))
    return xyz, nn


def timing_threads(n: int | None = None) -> int:
    """Threads the timing build uses (OMP_NUM_THREADS, else every host core);
    with n, set them first."""
    lib = _load_timing()
    if n is not None:
        lib.orc_set_num_threads(int(n))
    return int(lib.orc_num_threads())


class TimedStep:
    """One optimisation step of the float32 oracle (timing build): preprocess,
    binning, compositing, loss (Eq. 9), backward to the parameters and sparse
    Adam, on the parameters given (held fixed: the step is re-timed, not
    applied).  `sample(k)` times a bounded sample of the step -- every k-th
    tile for binning, compositing and the 2-D backward, every k-th Gaussian
    for the preprocess, the parameter backward and Adam, the loss in full --
    and extrapolates each sampled phase by k; k = 1 is the whole step."""

    def __init__(self, params: dict, cam: dict, target, E, Ts: int = 16):
        self.lib = _load_timing()
        self.cam, self.Ts = cam, Ts
        self.p = {k: np.ascontiguousarray(v, np.float32) for k, v in params.items()}
        self.n = self.p["means"].shape[0]
        self.deg = sh_degree(self.p)
        self.target = np.ascontiguousarray(target, np.float32)
        self.E = np.ascontiguousarray(np.asarray(E, np.float32).reshape(12))
        self.c = make_cam(cam)
        self.full = None

    def _pre(self, p, n):
        out = dict(radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
                   touched=np.zeros(n, np.uint32), depth_bits=np.zeros(n, np.uint32),
                   mean2d=np.zeros((n, 2), np.float32), conic=np.zeros((n, 3), np.float32),
                   opacity=np.zeros(n, np.float32), rgb=np.zeros((n, 3), np.float32),
                   depth=np.zeros(n, np.float32), flags=np.zeros(n, np.uint8), cullp=np.zeros((n, 8), np.float32))
        self.lib.orc_preprocess(n, self.deg, _p(p["means"]), _p(p["log_scales"]), _p(p["quats"]), _p(p["logits"]),
                                _p(p["sh"]), C.byref(self.c), self.Ts, 1, _p(out["radius"]), _p(out["rect"]),
                                _p(out["touched"]), _p(out["depth_bits"]), _p(out["mean2d"]), _p(out["conic"]),
                                _p(out["opacity"]), _p(out["rgb"]), _p(out["depth"]), _p(out["flags"]),
                                _p(out["cullp"]))
        return out

    def sample(self, k: int = 1) -> dict:
        """Phase times (s) of one (sampled) step and the extrapolated step time."""
        import time
        lib, n, Ts = self.lib, self.n, self.Ts
        W, H = int(self.cam["width"]), int(self.cam["height"])
        TX, TY = tiles(self.cam, Ts)
        k = max(1, int(k))
        sub = self.p if k == 1 else {key: np.ascontiguousarray(v[::k]) for key, v in self.p.items()}
        ns = sub["means"].shape[0]
        t = {}
        t0 = time.perf_counter()
        pre_s = self._pre(sub, ns)
        t["preprocess"] = time.perf_counter() - t0
        if k == 1:
            pre = pre_s
        else:
            if self.full is None:
                self.full = self._pre(self.p, n)
            pre = self.full
        I = int(lib.orc_num_instances(n, _p(pre["touched"])))
        keys = np.zeros(max(I, 1), np.uint64)
        vals = np.zeros(max(I, 1), np.uint32)
        ranges = np.zeros((TX * TY, 2), np.uint32)
        t0 = time.perf_counter()
        lib.orc_bin(n, _p(pre["rect"]), _p(pre["touched"]), _p(pre["depth_bits"]), _p(pre["cullp"]), Ts, TX, TY,
                    k, _p(keys), _p(vals), _p(ranges))
        t["bin"] = time.perf_counter() - t0
        img = {key: np.zeros(sh, dt) for key, sh, dt in
               (("C", (H, W, 3), np.float32), ("D", (H, W), np.float32), ("O", (H, W), np.float32),
                ("T", (H, W), np.float32), ("nc", (H, W), np.int32), ("amb", (H, W), np.uint8))}
        t0 = time.perf_counter()
        lib.orc_render(W, H, Ts, k, _p(vals), _p(ranges), _p(pre["mean2d"]), _p(pre["conic"]), _p(pre["opacity"]),
                       _p(pre["rgb"]), _p(pre["depth"]), 0.0, 0.0, _p(img["C"]), _p(img["D"]), _p(img["O"]),
                       _p(img["T"]), _p(img["nc"]), _p(img["amb"]), None)
        t["render"] = time.perf_counter() - t0
        dC = np.zeros((H, W, 3), np.float32)
        dE = np.zeros(12, np.float32)
        ss, l1 = C.c_float(), C.c_float()
        t0 = time.perf_counter()
        lib.orc_loss(W, H, _p(img["C"]), _p(self.target), _p(self.E), 0.2, _p(dC), _p(dE), C.byref(ss),
                     C.byref(l1))
        t["loss"] = time.perf_counter() - t0
        g2d = np.zeros((n, 10), np.float32)
        t0 = time.perf_counter()
        lib.orc_backward_2d(W, H, Ts, k, _p(vals), _p(ranges), _p(pre["mean2d"]), _p(pre["conic"]),
                            _p(pre["opacity"]), _p(pre["rgb"]), _p(pre["depth"]), _p(dC), None, None, n, _p(g2d))
        t["backward_2d"] = time.perf_counter() - t0
        g2s = g2d if k == 1 else np.ascontiguousarray(g2d[::k])
        grads = {key: np.zeros_like(v) for key, v in sub.items()}
        pose = np.zeros(6, np.float32)
        t0 = time.perf_counter()
        lib.orc_backward_params(ns, self.deg, _p(sub["means"]), _p(sub["log_scales"]), _p(sub["quats"]),
                                _p(sub["logits"]), _p(sub["sh"]), C.byref(self.c), _p(pre_s["radius"]), _p(g2s),
                                _p(grads["means"]), _p(grads["log_scales"]), _p(grads["quats"]),
                                _p(grads["logits"]), _p(grads["sh"]), _p(pose))
        t["backward_params"] = time.perf_counter() - t0
        mask = (pre_s["radius"] > 0).astype(np.uint8)
        work = {key: v.copy() for key, v in sub.items()}
        mom = {key: (np.zeros_like(v), np.zeros_like(v)) for key, v in sub.items()}
        t0 = time.perf_counter()
        for key, lr in (("means", 1.6e-4), ("log_scales", 5e-3), ("quats", 1e-3), ("logits", 0.05),
                        ("sh", 2.5e-3)):
            v = work[key]
            stride = int(np.prod(v.shape[1:])) if v.ndim > 1 else 1
            lib.orc_adam(v.size, stride, _p(mask), _p(v), _p(mom[key][0]), _p(mom[key][1]), _p(grads[key]), lr,
                         0.9, 0.999, 1e-15, 1)
        t["adam"] = time.perf_counter() - t0
        step = t["loss"] + k * sum(v for key, v in t.items() if key != "loss")
        return dict(phases=t, k=k, step_s=step, wall_s=sum(t.values()), instances=I)


def expf_decision(x: float) -> float:
    """exp as the float32 decision path evaluates it (see gl_oracle.c)."""
    return float(_load().orc_expf_decision(float(x)))


def logf_decision(x: float) -> float:
    """log as the float32 decision path evaluates it (see gl_oracle.c)."""
    return float(_load().orc_logf_decision(float(x)))


def uniform(seed: int, i: int) -> float:
    return _load().orc_uniform(C.c_uint64(seed), C.c_uint64(i))


def sky_points(n: int, radius: float = SKY_RADIUS, seed: int = 0):
    """Sky hemisphere sampling and nearest-neighbour scale (Sec. III-C 1)."""
    lib = _load()
    xyz = np.zeros((n, 3), np.float32)
    nn = np.zeros(n)
    lib.orc_sky(n, radius, C.c_uint64(seed), _p(xyz), _p(nn))
    return xyz, nn


def expand_mask(xyz, cam: dict, opacity=None, tau: float = TAU):
    """Eq. 8: keep points that land on pixels with rendered opacity below tau."""
    lib = _load()
    xyz = _c(xyz, np.float32)
    n = xyz.shape[0]
    keep = np.zeros(n, np.uint8)
    depth = np.zeros(n, np.float32)
    op = None if opacity is None else _c(opacity, np.float64)
    c = make_cam(cam)
    k = lib.orc_expand_mask(n, _p(xyz), C.byref(c), _p(op), tau, _p(keep), _p(depth))
    return keep.astype(bool), depth, int(k)


def init_gaussians(xyz, rgb, depth, fx, opacity=OPACITY_FG, scale=None, sh_deg=3) -> dict:
    """New Gaussians from points (Sec. III-C 1): centre, SH DC from colour,
    identity rotation, opacity o_a, isotropic scale d / f (or `scale`)."""
    n = xyz.shape[0]
    K = (sh_deg + 1) ** 2
    sh = np.zeros((n, K, 3), np.float64)
    sh[:, 0, :] = (np.asarray(rgb, np.float64) - 0.5) / SH_C0
    s = np.asarray(depth, np.float64) / float(fx) if scale is None else np.asarray(scale, np.float64)
    ls = np.repeat(np.log(s)[:, None], 3, axis=1)
    q = np.zeros((n, 4))
    q[:, 0] = 1.0
    lg = np.full(n, np.log(opacity / (1.0 - opacity)))
    return dict(means=np.asarray(xyz, np.float32), log_scales=ls.astype(np.float32),
                quats=q.astype(np.float32), logits=lg.astype(np.float32), sh=sh.astype(np.float32))


def forward(params: dict, cam: dict, Ts: int = 16, cull: bool = True):
    """Preprocess, bin and render: returns (pre, bins, image dict)."""
    pre = preprocess(params, cam, Ts, cull)
    bins = bin_instances(pre, cam)
    img = render(pre, bins, cam)
    return pre, bins, img


def loss_and_grads(params: dict, cam: dict, target, E, Ts: int = 16, lam: float = LAMBDA_DSSIM):
    """One forward + loss + backward (no parameter update)."""
    pre, bins, img = forward(params, cam, Ts)
    L = loss(img["color"], target, E, lam)
    g = backward(params, cam, pre, bins, L["dL_dC"])
    return dict(pre=pre, bins=bins, img=img, loss=L, grads=g)


# Learning rates: "same as vanilla 3DGS, not decayed" (Sec. IV-A); values are readings.
DEFAULT_LR = dict(means=1.6e-4, sh_dc=2.5e-3, sh_rest=2.5e-3 / 20.0, logits=0.05,
                  log_scales=5e-3, quats=1e-3, exposure=1e-3)


def optimize_step(params: dict, state: dict, cam: dict, target, E, step: int,
                  Ts: int = 16, lr: dict | None = None, sparse: bool = True,
                  lam: float = LAMBDA_DSSIM) -> dict:
    """One single-view optimisation step (Sec. III-C 3): loss, backward, Adam.
    `state` holds double copies of params/moments and the exposure moments;
    it is updated in place.  Sparse Adam (Sec. III-D 2) skips Gaussians
    with zero screen radius in this view."""
    lr = dict(DEFAULT_LR, **(lr or {}))
    r = loss_and_grads(params, cam, target, E, Ts, lam)
    g = r["grads"]
    mask = (r["pre"]["radius"] > 0).astype(np.uint8) if sparse else None
    for name in ("means", "log_scales", "quats", "logits"):
        adam_update(state["p"][name], state["m"][name], state["v"][name], g[name], lr[name], step, mask)
    # SH: DC and higher bands take different learning rates.
    sh_p, sh_m, sh_v = state["p"]["sh"], state["m"]["sh"], state["v"]["sh"]
    for sl, key in ((slice(0, 1), "sh_dc"), (slice(1, None), "sh_rest")):
        if sh_p[:, sl].size == 0:
            continue
        pp, mm, vv = (np.ascontiguousarray(a[:, sl]) for a in (sh_p, sh_m, sh_v))
        adam_update(pp, mm, vv, np.ascontiguousarray(g["sh"][:, sl]), lr[key], step, mask)
        sh_p[:, sl], sh_m[:, sl], sh_v[:, sl] = pp, mm, vv
    adam_update(state["p"]["E"], state["m"]["E"], state["v"]["E"], r["loss"]["dL_dE"].reshape(3, 4),
                lr["exposure"], step)
    return r


def new_state(params: dict, E=None) -> dict:
    p = {k: np.asarray(v, np.float64).copy() for k, v in params.items()}
    p["E"] = np.asarray(E if E is not None else np.hstack([np.eye(3), np.zeros((3, 1))]),
                        np.float64).reshape(3, 4).copy()
    return dict(p=p, m={k: np.zeros_like(v) for k, v in p.items()},
                v={k: np.zeros_like(v) for k, v in p.items()})


def optimize_window(params: dict, state: dict, cams, targets, step: int, Ts: int = 16,
                    lr: dict | None = None, sparse: bool = True, lam: float = LAMBDA_DSSIM,
                    exposure_steps=None) -> dict:
    """One window step over several keyframe views: the loss is the mean of the
    per-view losses (Eq. 9 with each view's exposure), the Gaussians take one
    Adam step on the mean gradient (sparse: Gaussians visible in any view), and
    each view's exposure takes one Adam step on its own (1/n-weighted) gradient.
    `state["p"]["E"]` is a list of the views' 3x4 exposures (moments alike)."""
    lr = dict(DEFAULT_LR, **(lr or {}))
    n = len(cams)
    exposure_steps = exposure_steps or [1] * n
    acc, vis, losses, dEs = None, None, [], []
    for v in range(n):
        r = loss_and_grads(params, cams[v], targets[v], state["p"]["E"][v], Ts, lam)
        g = r["grads"]
        if acc is None:
            acc = {k: g[k] / n for k in ("means", "log_scales", "quats", "logits", "sh")}
            vis = r["pre"]["radius"] > 0
        else:
            for k in acc:
                acc[k] = acc[k] + g[k] / n
            vis = vis | (r["pre"]["radius"] > 0)
        losses.append(r["loss"]["loss"])
        dEs.append(r["loss"]["dL_dE"] / n)
    mask = vis.astype(np.uint8) if sparse else None
    for name in ("means", "log_scales", "quats", "logits"):
        adam_update(state["p"][name], state["m"][name], state["v"][name], acc[name], lr[name], step, mask)
    sh_p, sh_m, sh_v = state["p"]["sh"], state["m"]["sh"], state["v"]["sh"]
    for sl, key in ((slice(0, 1), "sh_dc"), (slice(1, None), "sh_rest")):
        if sh_p[:, sl].size == 0:
            continue
        pp, mm, vv = (np.ascontiguousarray(a[:, sl]) for a in (sh_p, sh_m, sh_v))
        adam_update(pp, mm, vv, np.ascontiguousarray(acc["sh"][:, sl]), lr[key], step, mask)
        sh_p[:, sl], sh_m[:, sl], sh_v[:, sl] = pp, mm, vv
    for v in range(n):
        adam_update(state["p"]["E"][v], state["m"]["E"][v], state["v"]["E"][v], dEs[v], lr["exposure"],
                    exposure_steps[v])
    return dict(loss=float(np.mean(losses)), losses=losses, visible=vis, grads=acc)


def new_window_state(params: dict, n_views: int) -> dict:
    p = {k: np.asarray(v, np.float64).copy() for k, v in params.items()}
    I34 = np.hstack([np.eye(3), np.zeros((3, 1))])
    st = dict(p=p, m={k: np.zeros_like(v) for k, v in p.items()}, v={k: np.zeros_like(v) for k, v in p.items()})
    for d in ("p", "m", "v"):
        st[d]["E"] = [(I34.copy() if d == "p" else np.zeros((3, 4))) for _ in range(n_views)]
    return st
