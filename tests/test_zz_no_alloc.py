"""pivbos_render_noalloc: the render for callers that cannot allocate device
memory (a host application whose own pool owns the whole device, or a loop
that cannot afford the synchronisation of cudaMalloc).  Called through the C
ABI and checked against pivbos_render on the same inputs, on two calls in a
row -- the second with fewer sources than the first, so that it runs on the
scratch array the first call left behind.  Both calls run the same kernels
on fixed-point images, so the images and the status counts must be equal bit
for bit, in a medium and without one.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1812_05902_gb300 import scenes
from gpu_helpers import gpu_handles

pytestmark = pytest.mark.gpu


def _render_both(fr, handles):
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    med, opt = handles
    mh = med.h if med is not None else None
    L = P.lib()
    W, H = fr.optics.width, fr.optics.height
    src = torch.tensor(fr.sources, dtype=torch.float64, device="cuda")
    ref = torch.zeros((H, W), dtype=torch.int64, device="cuda")
    ref_st = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.pivbos_render(mh, opt.h, ctypes.c_void_p(src.data_ptr()), len(fr.sources), 1,
                           fr.rays_per_source, fr.seed, fr.frame_index, fr.integrator, fr.step,
                           ctypes.c_void_p(ref.data_ptr()), 1, ctypes.c_void_p(ref_st.data_ptr()), stream) == P.OK
    img = torch.zeros((H, W), dtype=torch.int64, device="cuda")
    st = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device="cuda")
    rc = L.pivbos_render_noalloc(mh, opt.h, ctypes.c_void_p(src.data_ptr()), len(fr.sources),
                                 fr.rays_per_source, fr.seed, fr.frame_index, fr.integrator, fr.step,
                                 ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(st.data_ptr()), stream)
    assert rc == P.OK, P.pivbos_last_error()
    assert L.pivbos_sync(stream) == P.OK
    return ref.cpu().numpy(), ref_st.cpu().numpy(), img.cpu().numpy(), st.cpu().numpy()


def _check_two_calls(big, small, handles):
    for fr in (big, small):
        ref, ref_st, img, st = _render_both(fr, handles)
        assert np.array_equal(st, ref_st)
        assert int(ref_st[0]) > 0
        assert img.sum() == ref.sum() == int(ref_st[0]) << 32
        assert np.array_equal(img, ref)


def test_noalloc_render_matches_render_on_two_calls_in_a_row():
    big = scenes.c2(scale=0.003, grid=40)[0]      # 300 dots x 300 rays
    small = scenes.c2(scale=0.003, grid=40)[0]
    small.sources = small.sources[:77]            # fewer sources than the first call
    small.seed = 11
    _check_two_calls(big, small, gpu_handles(big))


def test_noalloc_render_without_a_medium_matches_render():
    """m == NULL: rays straight everywhere, the same two calls in a row."""
    big = scenes.c1(scale=0.01)[0]
    big.medium = None
    big.sources = big.sources[:200]
    big.rays_per_source = 500
    small = scenes.c1(scale=0.01)[0]
    small.medium = None
    small.sources = small.sources[:31]
    small.rays_per_source = 500
    small.seed = 5
    _check_two_calls(big, small, gpu_handles(big))


def test_noalloc_render_shares_the_device_status_word():
    """A device-side error latched around a render without allocation is
    what the next pivbos_sync reports: both paths use the one per-device
    status word (here latched by the bounded-wait self-test)."""
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    fr = scenes.c0(scale=0.01, rays_per_source=8)[0]
    med, opt = gpu_handles(fr)
    L = P.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    src = torch.tensor(fr.sources, dtype=torch.float64, device="cuda")
    img = torch.zeros((fr.optics.height, fr.optics.width), dtype=torch.int64, device="cuda")
    assert L.pivbos_sync(stream) == P.OK
    P.pivbos_selftest_wait_timeout(4096)
    rc = L.pivbos_render_noalloc(med.h, opt.h, ctypes.c_void_p(src.data_ptr()), len(fr.sources),
                                 fr.rays_per_source, fr.seed, fr.frame_index, fr.integrator, fr.step,
                                 ctypes.c_void_p(img.data_ptr()), None, stream)
    assert rc == P.OK, P.pivbos_last_error()
    assert L.pivbos_sync(stream) == P.ERR_DEVICE_TIMEOUT
    assert L.pivbos_sync(stream) == P.OK


def test_noalloc_rejects_too_many_sources_and_host_buffers():
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    fr = scenes.c0(scale=0.01, rays_per_source=2)[0]
    med, opt = gpu_handles(fr)
    L = P.lib()
    img = torch.zeros((256, 256), dtype=torch.int64, device="cuda")
    src = torch.zeros((P.NOALLOC_MAX_SOURCES + 1, 3), dtype=torch.float64, device="cuda")
    rc = L.pivbos_render_noalloc(med.h, opt.h, ctypes.c_void_p(src.data_ptr()), P.NOALLOC_MAX_SOURCES + 1, 1, 0,
                                 0, 0, 1e-4, ctypes.c_void_p(img.data_ptr()), None, None)
    assert rc == P.ERR_UNSUPPORTED
    assert "exceed" in P.pivbos_last_error()
    host_src = np.ascontiguousarray(fr.sources)
    rc = L.pivbos_render_noalloc(med.h, opt.h, ctypes.c_void_p(host_src.ctypes.data), len(fr.sources), 1, 0, 0,
                                 0, 1e-4, ctypes.c_void_p(img.data_ptr()), None, None)
    assert rc == P.ERR_INVALID_ARG
    assert int(img.sum()) == 0
