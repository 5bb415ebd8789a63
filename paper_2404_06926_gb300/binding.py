"""Thin ctypes binding of the C ABI in include/gl_map.h (argument marshalling only).

Every step of the optimisation runs in the CUDA library; this module converts
torch tensors and numpy arrays to the plain pointers and structs the ABI takes,
raises ``GLError`` on a non-zero status, and loads nothing until first use.
There is no CPU fallback: if the library has not been built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libglmap.so")
_lib = None

STATUS = {0: "GL_OK", 1: "GL_ERR_INVALID", 2: "GL_ERR_OOM", 3: "GL_ERR_CUDA", 4: "GL_ERR_CAPACITY",
          5: "GL_ERR_TIMEOUT", 6: "GL_ERR_BUSY", 7: "GL_ERR_NOT_FOUND"}


class GLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class Pose(C.Structure):
    _fields_ = [("R_cw", C.c_float * 9), ("t_cw", C.c_float * 3)]


class Keyframe(C.Structure):
    _fields_ = [("id", C.c_int64), ("pose", Pose), ("K", Intrinsics), ("image", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("sh_degree", C.c_int32), ("tile_size", C.c_int32), ("sparse_adam", C.c_int32),
                ("reserved0", C.c_int32), ("seed", C.c_uint64),
                ("lambda_dssim", C.c_float), ("tau", C.c_float), ("opacity_fg", C.c_float),
                ("opacity_sky", C.c_float), ("sky_radius", C.c_float), ("reserved1", C.c_int32),
                ("n_sky", C.c_int64),
                ("lr_pos", C.c_float), ("lr_sh_dc", C.c_float), ("lr_sh_rest", C.c_float),
                ("lr_opacity", C.c_float), ("lr_scale", C.c_float), ("lr_rot", C.c_float),
                ("lr_exposure", C.c_float), ("adam_b1", C.c_float), ("adam_b2", C.c_float),
                ("adam_eps", C.c_float), ("capacity_hint", C.c_int64), ("lr_window_exp", C.c_float),
                ("reserved2", C.c_int32)]


NUM_PHASES = 10


class Stats(C.Structure):
    _fields_ = [("n_gaussians", C.c_int64), ("n_visible", C.c_int64), ("n_instances", C.c_int64),
                ("sum_contrib", C.c_int64), ("pixels", C.c_int64), ("steps", C.c_int64),
                ("phase_ms", C.c_double * NUM_PHASES), ("phase_calls", C.c_int64 * NUM_PHASES),
                ("graph_captures", C.c_int64), ("graph_replays", C.c_int64), ("graph_reruns", C.c_int64),
                ("timed_steps", C.c_int64), ("timed_views", C.c_int64), ("timed_visible", C.c_int64),
                ("timed_instances", C.c_int64), ("timed_contrib", C.c_int64), ("timed_pixels", C.c_int64)]


class ExecConfig(C.Structure):
    _fields_ = [("use_graphs", C.c_int32), ("persistent", C.c_int32), ("batch_depth", C.c_int32),
                ("pixels_per_lane", C.c_int32), ("tile_size", C.c_int32), ("deterministic", C.c_int32),
                ("segment", C.c_int32), ("exact_cull", C.c_int32), ("per_gaussian", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("reserved", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("logits", C.c_void_p), ("sh", C.c_void_p)]


def lib():
    """Load the CUDA library; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        P, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
        sigs = {
            "gl_last_error": ([], C.c_char_p),
            "gl_version": ([], i32),
            "gl_config_default": ([P], i32),
            "gl_map_create": ([P, P, P], i32),
            "gl_map_destroy": ([P], i32),
            "gl_map_size": ([P, P], i32),
            "gl_map_add_points": ([P, P, P, i64, i32, P, P, i32, P], i32),
            "gl_map_add_keyframe": ([P, P], i32),
            "gl_render": ([P, P, P, P, P, P, P], i32),
            "gl_optimize_step": ([P, P, i32, P], i32),
            "gl_map_get_params": ([P, P, P], i32),
            "gl_map_set_params": ([P, P], i32),
            "gl_map_get_moments": ([P, i32, P], i32),
            "gl_map_get_exposure": ([P, i64, P], i32),
            "gl_ctx_create": ([P, P], i32),
            "gl_ctx_destroy": ([P], i32),
            "gl_rasterize_forward": ([P, P, P, P, P, i32, P, P, P], i32),
            "gl_rasterize_backward": ([P, P, P, P, P, P, P], i32),
            "gl_photometric_loss": ([P, P, P, P, i32, i32, f32, P, P, P], i32),
            "gl_ctx_get_preprocess": ([P, P, P, P, P, P, P, P], i32),
            "gl_ctx_num_instances": ([P, P], i32),
            "gl_ctx_get_instances": ([P, P, P, P], i32),
            "gl_ctx_get_pixel_state": ([P, P, P], i32),
            "gl_map_set_timing": ([P, i32], i32),
            "gl_map_get_stats": ([P, P], i32),
            "gl_phase_name": ([i32], C.c_char_p),
            "gl_kernel_launch_count": ([], i64),
            "gl_photometric_loss_noalloc": ([P, P, P, i32, i32, f32, P, P, P, P], i32),
            "gl_map_set_exec": ([P, P], i32),
            "gl_ctx_set_exec": ([P, P], i32),
            "gl_map_get_exec": ([P, P], i32),
            "gl_map_autotune": ([P, P, i32, i32, i32, i32, P, P], i32),
            "gl_map_checkpoint_size": ([P, i32, P], i32),
            "gl_map_set_config": ([P, P], i32),
            "gl_server_config_default": ([P], i32),
            "gl_server_create": ([P, P, P], i32),
            "gl_server_submit": ([P, P, P], i32),
            "gl_server_wait": ([P, C.c_uint64, C.c_double, P], i32),
            "gl_server_drain": ([P], i32),
            "gl_server_get_stats": ([P, P], i32),
            "gl_server_get_version": ([P, i64, P, i64, P], i32),
            "gl_server_destroy": ([P], i32),
            "gl_map_get_config": ([P, P], i32),
            "gl_map_save": ([P, i32, P, i64], i32),
            "gl_map_load": ([P, P, i64], i32),
            "gl_selftest_bounded_wait": ([P], i32),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(status):
    if status != 0:
        raise GLError(status, lib().gl_last_error().decode())


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (contiguous), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    assert x.is_contiguous(), "tensor must be contiguous"
    return x.data_ptr()


def intrinsics(cam: dict) -> Intrinsics:
    return Intrinsics(float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"]),
                      int(cam["width"]), int(cam["height"]))


def pose(cam: dict) -> Pose:
    p = Pose()
    R = np.asarray(cam["R"], np.float32).reshape(9)
    t = np.asarray(cam["t"], np.float32).reshape(3)
    for i in range(9):
        p.R_cw[i] = float(R[i])
    for i in range(3):
        p.t_cw[i] = float(t[i])
    return p


def gaussians(params: dict, n=None) -> Gaussians:
    """Struct of pointers over a dict of tensors/arrays: means, log_scales,
    quats, logits, sh (shapes n*3, n*3, n*4, n, n*K*3)."""
    sh = params["sh"]
    K = sh.shape[1]
    deg = int(round(K ** 0.5)) - 1
    g = Gaussians()
    g.n = int(params["means"].shape[0] if n is None else n)
    g.sh_degree = deg
    g.means = _ptr(params["means"])
    g.log_scales = _ptr(params["log_scales"])
    g.quats = _ptr(params["quats"])
    g.logits = _ptr(params["logits"])
    g.sh = _ptr(params["sh"])
    return g


def default_config(**over) -> Config:
    c = Config()
    check(lib().gl_config_default(C.byref(c)))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Ctx:
    """Owner of the per-view scratch of the differentiable single-view API."""

    def __init__(self, stream=None):
        self._h = C.c_void_p()
        self.stream = stream
        check(lib().gl_ctx_create(_stream_ptr(stream), C.byref(self._h)))

    def close(self):
        if self._h:
            check(lib().gl_ctx_destroy(self._h))
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, params: dict, cam: dict, tile: int = 16, depth: bool = True, opacity: bool = True,
                twist=None):
        """Render from the pose exp(twist^) T_cw (twist: 6 numbers (rho, phi)
        or None for T_cw itself)."""
        import torch
        H, W = int(cam["height"]), int(cam["width"])
        dev = params["means"].device
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        dep = torch.empty((H, W), dtype=torch.float32, device=dev) if depth else None
        opa = torch.empty((H, W), dtype=torch.float32, device=dev) if opacity else None
        g = gaussians(params)
        K, P = intrinsics(cam), pose(cam)
        tw = None
        if twist is not None:
            tw = (C.c_float * 6)(*[float(x) for x in twist])
        check(lib().gl_rasterize_forward(self._h, C.byref(g), C.byref(P), tw, C.byref(K), int(tile),
                                         _ptr(rgb), _ptr(dep), _ptr(opa)))
        return rgb, dep, opa

    def backward(self, params: dict, dL_drgb, dL_ddepth=None, dL_dopacity=None, pose_grad=True):
        import torch
        grads = {k: torch.empty_like(v) for k, v in params.items()}
        g = gaussians(params)
        gg = gaussians(grads)
        pg = torch.empty(6, dtype=torch.float32, device=dL_drgb.device) if pose_grad else None
        check(lib().gl_rasterize_backward(self._h, C.byref(g), _ptr(dL_drgb), _ptr(dL_ddepth),
                                          _ptr(dL_dopacity), C.byref(gg), _ptr(pg)))
        return grads, pg

    def loss(self, rgb, target, E, lam: float = 0.2):
        import torch
        H, W = rgb.shape[:2]
        loss = torch.empty(1, dtype=torch.float32, device=rgb.device)
        dC = torch.empty_like(rgb)
        dE = torch.empty(12, dtype=torch.float32, device=rgb.device)
        check(lib().gl_photometric_loss(self._h, _ptr(rgb), _ptr(target), _ptr(E), int(W), int(H),
                                        float(lam), _ptr(loss), _ptr(dC), _ptr(dE)))
        return loss, dC, dE.view(3, 4)

    # introspection of the last forward
    def set_exec(self, batch_depth=32, pixels_per_lane=1, persistent=0, deterministic=0, segment=0, exact_cull=1,
                 per_gaussian=0):
        """Raster execution of this context's calls (see gl_ctx_set_exec)."""
        e = ExecConfig(0, int(persistent), int(batch_depth), int(pixels_per_lane), 0, int(deterministic),
                       int(segment), int(exact_cull), int(per_gaussian))
        check(lib().gl_ctx_set_exec(self._h, C.byref(e)))

    def preprocess(self, n: int, device):
        import torch
        out = dict(radius=torch.empty(n, dtype=torch.int32, device=device),
                   rect=torch.empty((n, 4), dtype=torch.int32, device=device),
                   mean2d=torch.empty((n, 2), device=device), conic=torch.empty((n, 3), device=device),
                   opacity=torch.empty(n, device=device), rgb=torch.empty((n, 3), device=device),
                   depth=torch.empty(n, device=device))
        check(lib().gl_ctx_get_preprocess(self._h, *[_ptr(out[k]) for k in
                                                      ("radius", "rect", "mean2d", "conic", "opacity",
                                                       "rgb", "depth")]))
        return out

    def num_instances(self) -> int:
        I = C.c_int64()
        check(lib().gl_ctx_num_instances(self._h, C.byref(I)))
        return I.value

    def instances(self, num_tiles: int, device):
        import torch
        I = self.num_instances()
        keys = torch.empty(max(I, 1), dtype=torch.int64, device=device)
        vals = torch.empty(max(I, 1), dtype=torch.int32, device=device)
        ranges = torch.empty((num_tiles, 2), dtype=torch.int32, device=device)
        check(lib().gl_ctx_get_instances(self._h, _ptr(keys), _ptr(vals), _ptr(ranges)))
        return keys[:I], vals[:I], ranges

    def pixel_state(self, H: int, W: int, device):
        import torch
        T = torch.empty((H, W), device=device)
        n = torch.empty((H, W), dtype=torch.int32, device=device)
        check(lib().gl_ctx_get_pixel_state(self._h, _ptr(T), _ptr(n)))
        return T, n


def photometric_loss_noalloc(rgb, target, E, lam: float = 0.2, stream=None):
    """Eq. 9 loss through the entry point that allocates no device memory
    (its scratch is a fixed array inside the library)."""
    import torch
    H, W = rgb.shape[:2]
    loss = torch.empty(1, dtype=torch.float32, device=rgb.device)
    dC = torch.empty_like(rgb)
    dE = torch.empty(12, dtype=torch.float32, device=rgb.device)
    check(lib().gl_photometric_loss_noalloc(_ptr(rgb), _ptr(target), _ptr(E), int(W), int(H), float(lam),
                                            _ptr(loss), _ptr(dC), _ptr(dE), _stream_ptr(stream)))
    return loss, dC, dE.view(3, 4)


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().gl_kernel_launch_count())


def selftest_bounded_wait() -> bool:
    """Run the device self-test of the bounded waits (a radix-sort pass whose
    look-back can never complete); True if the wait gave up and raised its
    flag.  Takes about a second."""
    expired = C.c_int32(0)
    check(lib().gl_selftest_bounded_wait(C.byref(expired)))
    return bool(expired.value)


def keyframe(kid: int, cam: dict, image=None) -> Keyframe:
    k = Keyframe()
    k.id = int(kid)
    k.pose = pose(cam)
    k.K = intrinsics(cam)
    k.image = _ptr(image) if image is not None else None
    return k


class Map:
    """Owner of a device-resident Gaussian map (gl_map)."""

    def __init__(self, config: Config | None = None, stream=None, **over):
        self.config = config if config is not None else default_config(**over)
        self._h = C.c_void_p()
        self.stream = stream
        check(lib().gl_map_create(C.byref(self.config), _stream_ptr(stream), C.byref(self._h)))
        self.deg = self.config.sh_degree

    def close(self):
        if self._h:
            check(lib().gl_map_destroy(self._h))
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        n = C.c_int64()
        check(lib().gl_map_size(self._h, C.byref(n)))
        return n.value

    def add_points(self, xyz, rgb, cam: dict, use_mask: bool = True, kind: int = 0) -> int:
        n_added = C.c_int64()
        K, P = intrinsics(cam), pose(cam)
        check(lib().gl_map_add_points(self._h, _ptr(xyz), _ptr(rgb), int(xyz.shape[0]), int(kind),
                                      C.byref(P), C.byref(K), int(bool(use_mask)), C.byref(n_added)))
        return n_added.value

    def add_keyframe(self, kid: int, cam: dict, image):
        k = keyframe(kid, cam, image)
        check(lib().gl_map_add_keyframe(self._h, C.byref(k)))

    def render(self, cam: dict, E=None, out_rgb=None, out_depth=None, out_opacity=None):
        H, W = int(cam["height"]), int(cam["width"])
        if out_rgb is None:
            out_rgb = np.empty((H, W, 3), np.float32)
        Ep = None
        if E is not None:
            E = np.ascontiguousarray(np.asarray(E, np.float32).reshape(12))
            Ep = E.ctypes.data
        K, P = intrinsics(cam), pose(cam)
        check(lib().gl_render(self._h, C.byref(P), C.byref(K), Ep, _ptr(out_rgb), _ptr(out_depth),
                              _ptr(out_opacity)))
        return out_rgb

    def optimize_step(self, views, want_loss: bool = False):
        """views: list of (id, cam, image-or-None)."""
        arr = (Keyframe * len(views))()
        for i, (kid, cam, img) in enumerate(views):
            arr[i] = keyframe(kid, cam, img)
        loss = C.c_float()
        check(lib().gl_optimize_step(self._h, arr, len(views), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def _alloc(self, n):
        K = (self.deg + 1) ** 2
        return dict(means=np.zeros((n, 3), np.float32), log_scales=np.zeros((n, 3), np.float32),
                    quats=np.zeros((n, 4), np.float32), logits=np.zeros(n, np.float32),
                    sh=np.zeros((n, K, 3), np.float32))

    def get_params(self) -> dict:
        n = len(self)
        out = self._alloc(n)
        g = gaussians(out, n)
        check(lib().gl_map_get_params(self._h, C.byref(g), None))
        return out

    def set_params(self, params: dict):
        g = gaussians(params)
        check(lib().gl_map_set_params(self._h, C.byref(g)))

    def get_moments(self, which: int) -> dict:
        n = len(self)
        out = self._alloc(n)
        g = gaussians(out, n)
        check(lib().gl_map_get_moments(self._h, int(which), C.byref(g)))
        return out

    def set_timing(self, on: bool):
        check(lib().gl_map_set_timing(self._h, int(bool(on))))

    def set_exec(self, use_graphs=None, persistent=None, batch_depth=None, pixels_per_lane=None,
                 tile_size=None, deterministic=None, segment=None, exact_cull=None, per_gaussian=None):
        """Change how steps execute (fields left as None keep their value)."""
        e = ExecConfig()
        check(lib().gl_map_get_exec(self._h, C.byref(e)))
        for k, v in dict(use_graphs=use_graphs, persistent=persistent, batch_depth=batch_depth,
                         pixels_per_lane=pixels_per_lane, tile_size=tile_size, deterministic=deterministic,
                         segment=segment, exact_cull=exact_cull, per_gaussian=per_gaussian).items():
            if v is not None:
                setattr(e, k, int(v))
        check(lib().gl_map_set_exec(self._h, C.byref(e)))
        return e.as_dict()

    def set_config(self, **over):
        """Change run-time fields of the map's configuration (see gl_map_set_config)."""
        cfg = Config()
        check(lib().gl_map_get_config(self._h, C.byref(cfg)))
        for k, v in over.items():
            setattr(cfg, k, v)
        check(lib().gl_map_set_config(self._h, C.byref(cfg)))
        self.config = cfg

    def save(self, with_images: bool = False) -> np.ndarray:
        """The map's whole optimisation state as a host byte array."""
        n = C.c_int64()
        check(lib().gl_map_checkpoint_size(self._h, int(bool(with_images)), C.byref(n)))
        buf = np.empty(n.value, np.uint8)
        check(lib().gl_map_save(self._h, int(bool(with_images)), buf.ctypes.data, n.value))
        return buf

    def load(self, buf) -> None:
        """Replace the map's state with a buffer written by save()."""
        buf = np.ascontiguousarray(np.frombuffer(buf, np.uint8) if isinstance(buf, (bytes, bytearray)) else buf,
                                   dtype=np.uint8)
        check(lib().gl_map_load(self._h, buf.ctypes.data, buf.nbytes))

    def get_exec(self) -> dict:
        e = ExecConfig()
        check(lib().gl_map_get_exec(self._h, C.byref(e)))
        return e.as_dict()

    def autotune(self, views, reps: int = 3, keep_tile_size: bool = False, window: int | None = None):
        """Time every execution candidate on `views` (list of (id, cam,
        image-or-None)) taken as consecutive windows of `window` views (default:
        one window of all), install the fastest; returns (config, ms per step)."""
        window = len(views) if window is None else int(window)
        arr = (Keyframe * len(views))()
        for i, (kid, cam, img) in enumerate(views):
            arr[i] = keyframe(kid, cam, img)
        e = ExecConfig()
        ms = C.c_float()
        check(lib().gl_map_autotune(self._h, arr, len(views), window, int(reps), int(bool(keep_tile_size)),
                                    C.byref(e), C.byref(ms)))
        return e.as_dict(), ms.value

    def stats(self) -> dict:
        st = Stats()
        check(lib().gl_map_get_stats(self._h, C.byref(st)))
        out = {k: getattr(st, k) for k in ("n_gaussians", "n_visible", "n_instances", "sum_contrib",
                                           "pixels", "steps", "graph_captures", "graph_replays",
                                           "graph_reruns", "timed_steps", "timed_views", "timed_visible",
                                           "timed_instances", "timed_contrib", "timed_pixels")}
        out["phases"] = {lib().gl_phase_name(i).decode(): (st.phase_ms[i], st.phase_calls[i])
                         for i in range(NUM_PHASES)}
        return out

    def exposure(self, kid: int):
        E = np.zeros(12, np.float32)
        check(lib().gl_map_get_exposure(self._h, int(kid), E.ctypes.data))
        return E.reshape(3, 4)


# ---------------------------------------------------------------------------
# Serving loop
# ---------------------------------------------------------------------------
REQ_KEYFRAME_UPDATE, REQ_OPTIMIZE, REQ_RENDER = 1, 2, 3
REQ_NAMES = {1: "keyframe_update", 2: "optimize", 3: "render"}


class ServerConfig(C.Structure):
    _fields_ = [("queue_capacity", C.c_int32), ("render_batch", C.c_int32), ("reserve_bytes", C.c_int64),
                ("record_versions", C.c_int32), ("max_gaussians", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_steps", C.c_int32), ("window", C.c_int32), ("point_kind", C.c_int32),
                ("seed", C.c_uint64), ("xyz", C.c_void_p), ("rgb", C.c_void_p), ("n_points", C.c_int64),
                ("keyframe", Keyframe), ("out_rgb", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_int32), ("version", C.c_int64), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("loss", C.c_float), ("batch", C.c_int32),
                ("n_added", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64 * 4), ("completed", C.c_int64 * 4), ("failed", C.c_int64 * 4),
                ("p50_ms", C.c_double * 4), ("p99_ms", C.c_double * 4), ("mean_ms", C.c_double * 4),
                ("steps", C.c_int64), ("steps_per_s", C.c_double), ("renders_per_s", C.c_double),
                ("mean_render_batch", C.c_double), ("memory_waits", C.c_int64), ("busy_rejects", C.c_int64),
                ("version", C.c_int64), ("map_size", C.c_int64), ("points_capped", C.c_int64)]


class Server:
    """Request loop over a Map (see gl_server_create).  Host inputs are copied
    at submission; a render's output array must stay alive until wait()."""

    def __init__(self, m: Map, queue_capacity=256, render_batch=8, reserve_bytes=1 << 30, record_versions=False,
                 max_gaussians=0):
        cfg = ServerConfig()
        check(lib().gl_server_config_default(C.byref(cfg)))
        cfg.queue_capacity, cfg.render_batch = int(queue_capacity), int(render_batch)
        cfg.reserve_bytes, cfg.record_versions = int(reserve_bytes), int(bool(record_versions))
        cfg.max_gaussians = int(max_gaussians)
        self.map = m
        self._h = C.c_void_p()
        self._keep = {}   # ticket -> output arrays kept alive
        check(lib().gl_server_create(m._h, C.byref(cfg), C.byref(self._h)))

    def close(self):
        if self._h:
            check(lib().gl_server_destroy(self._h))
            self._h = C.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _submit(self, r: Request, keep=None) -> int:
        t = C.c_uint64()
        check(lib().gl_server_submit(self._h, C.byref(r), C.byref(t)))
        if keep is not None:
            self._keep[t.value] = keep
        return t.value

    def keyframe_update(self, kid, cam, image, xyz, rgb, n_steps=0, window=1, seed=0, point_kind=0) -> int:
        xyz = np.ascontiguousarray(xyz, np.float32)
        rgb = np.ascontiguousarray(rgb, np.float32)
        r = Request(kind=REQ_KEYFRAME_UPDATE, n_steps=int(n_steps), window=int(window), point_kind=int(point_kind),
                    seed=int(seed), xyz=_ptr(xyz), rgb=_ptr(rgb), n_points=len(xyz))
        r.keyframe = keyframe(kid, cam, image)
        return self._submit(r)

    def optimize(self, n_steps, window=1, seed=0) -> int:
        return self._submit(Request(kind=REQ_OPTIMIZE, n_steps=int(n_steps), window=int(window), seed=int(seed)))

    def render(self, cam, out=None) -> int:
        if out is None:
            out = np.empty((int(cam["height"]), int(cam["width"]), 3), np.float32)
        r = Request(kind=REQ_RENDER)
        r.keyframe = keyframe(-1, cam, None)
        r.out_rgb = _ptr(out)
        return self._submit(r, keep=out)

    def wait(self, ticket: int, timeout: float = -1.0):
        """(result dict, render output or None)."""
        res = Result()
        check(lib().gl_server_wait(self._h, int(ticket), float(timeout), C.byref(res)))
        return res.as_dict(), self._keep.pop(ticket, None)

    def drain(self):
        check(lib().gl_server_drain(self._h))

    def stats(self) -> dict:
        st = ServerStats()
        check(lib().gl_server_get_stats(self._h, C.byref(st)))
        out = {"steps": st.steps, "steps_per_s": st.steps_per_s, "renders_per_s": st.renders_per_s,
               "mean_render_batch": st.mean_render_batch, "memory_waits": st.memory_waits,
               "busy_rejects": st.busy_rejects, "version": st.version, "map_size": st.map_size,
               "points_capped": st.points_capped}
        for k, name in REQ_NAMES.items():
            out[name] = {"submitted": st.submitted[k], "completed": st.completed[k], "failed": st.failed[k],
                         "p50_ms": st.p50_ms[k], "p99_ms": st.p99_ms[k], "mean_ms": st.mean_ms[k]}
        return out

    def version(self, v: int) -> np.ndarray:
        n = C.c_int64()
        check(lib().gl_server_get_version(self._h, int(v), None, 0, C.byref(n)))
        buf = np.empty(n.value, np.uint8)
        check(lib().gl_server_get_version(self._h, int(v), buf.ctypes.data, n.value, C.byref(n)))
        return buf
