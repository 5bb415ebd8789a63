"""The loss entry point that allocates no device memory gives what the
allocating one gives.

gl_photometric_loss_noalloc serves callers that cannot allocate device memory
during a call (a real-time thread that must not trigger cudaMalloc's
device-wide synchronisation, or a process whose memory belongs to another
allocator).  Its scratch is a fixed array inside the library, shared by every
call, so this checks two calls in a row against gl_photometric_loss, and that
an image beyond the array's limit is rejected.  Collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(seed, H, W):
    rng = np.random.default_rng(seed)
    C = torch.from_numpy(rng.uniform(0, 1, (H, W, 3)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.uniform(0, 1, (H, W, 3)).astype(np.float32)).cuda()
    E = np.hstack([np.eye(3) + rng.normal(0, 0.05, (3, 3)), rng.normal(0, 0.02, (3, 1))])
    return C, T, torch.from_numpy(np.ascontiguousarray(E.astype(np.float32).reshape(12))).cuda()


def test_noalloc_loss_matches_allocating_entry_point_twice():
    from paper_2404_06926_gb300 import binding
    ctx = binding.Ctx()
    for seed, (H, W) in ((1, (192, 256)), (2, (100, 77))):
        C, T, E = _inputs(seed, H, W)
        l_ref, dC_ref, dE_ref = ctx.loss(C, T, E)
        l_na, dC_na, dE_na = binding.photometric_loss_noalloc(C, T, E)
        torch.cuda.synchronize()
        assert abs(l_na.item() - l_ref.item()) <= 1e-5 * abs(l_ref.item())
        scale = dC_ref.abs().max().item()
        assert (dC_na - dC_ref).abs().max().item() <= 1e-5 * scale
        assert (dE_na - dE_ref).abs().max().item() <= 1e-5 * dE_ref.abs().max().item() + 1e-12


def test_noalloc_rejects_images_beyond_its_scratch():
    from paper_2404_06926_gb300 import binding
    C, T, E = _inputs(3, 8, 8)
    import ctypes
    lib = binding.lib()
    st = lib.gl_photometric_loss_noalloc(C.data_ptr(), T.data_ptr(), E.data_ptr(), 4128, 4096,
                                         ctypes.c_float(0.2), C.data_ptr(), C.data_ptr(), C.data_ptr(),
                                         None)
    assert st == 1 and b"too large" in lib.gl_last_error()
