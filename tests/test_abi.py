"""The C-ABI library builds, loads without a GPU, exports every declared entry
point, and its structs have the layout the Python binding marshals."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gl_map.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^GL_API\s+[\w\s\*]+?\b(gl_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2404_06926_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gl_map_create", "gl_map_add_points", "gl_render", "gl_optimize_step",
                     "gl_map_destroy", "gl_rasterize_forward", "gl_rasterize_backward",
                     "gl_photometric_loss", "gl_last_error"):
        assert required in names


def test_library_loads_and_exports_every_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # only the ABI is exported
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(_declared())


def test_calls_without_gpu_fail_cleanly(libpath):
    """No compute call: only calls that validate arguments before touching CUDA."""
    from paper_2404_06926_gb300 import binding
    L = binding.lib()
    assert L.gl_version() == 102
    cfg = binding.default_config()
    assert cfg.sh_degree == 3 and cfg.tile_size == 16 and abs(cfg.lambda_dssim - 0.2) < 1e-7
    assert abs(cfg.tau - 0.99) < 1e-7 and cfg.n_sky == 100000
    assert L.gl_map_create(None, None, None) == 1
    assert b"null" in L.gl_last_error()
    e = binding.ExecConfig(1, 0, 32, 1, 0, 0)
    assert L.gl_map_set_exec(None, ctypes.byref(e)) == 1
    assert L.gl_map_autotune(None, None, 1, 1, 1, 0, None, None) == 1
    assert L.gl_map_load(None, None, 0) == 1
    sc = binding.ServerConfig()
    assert L.gl_server_config_default(ctypes.byref(sc)) == 0 and sc.queue_capacity == 256 and sc.render_batch == 8
    assert L.gl_server_create(None, None, None) == 1
    assert L.gl_server_submit(None, None, None) == 1
    assert L.gl_map_save(None, 0, None, 0) == 1
    assert L.gl_selftest_bounded_wait(None) == 1


def test_struct_layouts_match_c(libpath, tmp_path):
    from paper_2404_06926_gb300 import binding as B
    prog = tmp_path / "layout.c"
    prog.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gl_intrinsics), sizeof(gl_pose),
         sizeof(gl_keyframe), sizeof(gl_config), sizeof(gl_gaussians), sizeof(gl_stats), sizeof(gl_exec_config),
         sizeof(gl_server_config), sizeof(gl_request), sizeof(gl_result), sizeof(gl_server_stats));
  printf("%zu %zu %zu %zu\\n", offsetof(gl_keyframe, image), offsetof(gl_config, n_sky),
         offsetof(gl_config, capacity_hint), offsetof(gl_gaussians, sh));
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(prog)], check=True)
    a, b = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n")[:2]
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [ctypes.sizeof(t) for t in (B.Intrinsics, B.Pose, B.Keyframe, B.Config, B.Gaussians, B.Stats,
                                                 B.ExecConfig, B.ServerConfig, B.Request, B.Result, B.ServerStats)]
    assert offs == [B.Keyframe.image.offset, B.Config.n_sky.offset, B.Config.capacity_hint.offset,
                    B.Gaussians.sh.offset]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2404_06926_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        binding.lib()
