"""The loss entry point that allocates no device memory gives what the
allocating one gives, gives the oracle's loss, and allocates nothing.

gl_photometric_loss_noalloc serves callers that cannot allocate device memory
during a call (a real-time thread that must not trigger cudaMalloc's
device-wide synchronisation, or a process whose memory belongs to another
allocator).  Its scratch is a fixed array inside the library, shared by every
call, so this checks two calls in a row against gl_photometric_loss and the
oracle's Eq. 9, that device memory in use is the same before and after those
calls (after one warm-up call, which may load the library's device code), and
that an image beyond the array's limit is rejected.  Collected last on
purpose.
"""
import ctypes
import gc

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(seed, H, W):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    T = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    E = np.hstack([np.eye(3) + rng.normal(0, 0.05, (3, 3)), rng.normal(0, 0.02, (3, 1))]).astype(np.float32)
    return C, T, E


def _call(lib, C, T, E, out, stream):
    loss, dC, dE = out
    H, W = C.shape[:2]
    return lib.gl_photometric_loss_noalloc(C.data_ptr(), T.data_ptr(), E.data_ptr(), int(W), int(H),
                                           ctypes.c_float(0.2), loss.data_ptr(), dC.data_ptr(), dE.data_ptr(),
                                           ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_loss_matches_allocating_entry_point_and_oracle_twice():
    from paper_2404_06926_gb300 import binding
    lib = binding.lib()
    ctx = binding.Ctx()
    stream = torch.cuda.current_stream()
    cases = []
    for seed, (H, W) in ((1, (192, 256)), (2, (100, 77))):
        C, T, E = _inputs(seed, H, W)
        dev = tuple(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (C, T, E.reshape(12)))
        out = (torch.empty(1, device="cuda"), torch.empty((H, W, 3), device="cuda"), torch.empty(12, device="cuda"))
        cases.append(((C, T, E), dev, out))
    # warm-up: the first call on a device may load the library's device code
    assert _call(lib, *cases[0][1], cases[0][2], stream) == 0
    torch.cuda.synchronize()
    # objects left by earlier tests free device memory when collected: collect
    # them now and keep the collector off while memory is measured
    gc.collect()
    gc.disable()
    try:
        torch.cuda.synchronize()
        used0 = torch.cuda.memory_allocated()
        free0 = torch.cuda.mem_get_info()[0]
        for host, dev, out in cases:      # two calls in a row, on different sizes
            assert _call(lib, *dev, out, stream) == 0, lib.gl_last_error()
        torch.cuda.synchronize()
        used1 = torch.cuda.memory_allocated()
        free1 = torch.cuda.mem_get_info()[0]
    finally:
        gc.enable()
    assert used1 == used0
    assert free1 == free0, (free0, free1)
    for (C, T, E), dev, out in cases:
        l_na, dC_na, dE_na = (x.cpu().numpy().astype(np.float64) for x in out)
        l_ref, dC_ref, dE_ref = ctx.loss(*dev)
        scale = dC_ref.abs().max().item()
        assert abs(l_na[0] - l_ref.item()) <= 1e-5 * abs(l_ref.item())
        assert np.abs(dC_na - dC_ref.cpu().numpy()).max() <= 1e-5 * scale
        assert np.abs(dE_na - dE_ref.cpu().numpy().reshape(12)).max() <= 1e-5 * dE_ref.abs().max().item() + 1e-12
        L = oracle.loss(C.astype(np.float64), T, E)
        assert abs(l_na[0] - L["loss"]) <= 1e-5 * abs(L["loss"])
        r = np.abs(dC_na - L["dL_dC"]) / np.maximum(np.abs(L["dL_dC"]), 1e-4 * np.abs(L["dL_dC"]).max())
        assert np.median(r) < 1e-3 and np.percentile(r, 99) < 1e-2
        assert np.allclose(dE_na.reshape(3, 4), L["dL_dE"], rtol=1e-3, atol=1e-6 * np.abs(L["dL_dE"]).max())


def test_noalloc_rejects_images_beyond_its_scratch():
    from paper_2404_06926_gb300 import binding
    C, T, E = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in _inputs(3, 8, 8))
    lib = binding.lib()
    st = lib.gl_photometric_loss_noalloc(C.data_ptr(), T.data_ptr(), E.data_ptr(), 4128, 4096,
                                         ctypes.c_float(0.2), C.data_ptr(), C.data_ptr(), C.data_ptr(),
                                         None)
    assert st == 1 and b"too large" in lib.gl_last_error()
