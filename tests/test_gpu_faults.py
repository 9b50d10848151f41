"""Failure detection without a GPU fault: the bounded mbarrier wait the
tensor-core kernels use gives up on a barrier nothing arrives at, latches a
device timeout that pivbos_sync reports once, and leaves the context usable
(a render right after it is still exact)."""
import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes
from gpu_helpers import compare_images, gpu_render

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_a_timeout_and_the_context_survives():
    from paper_1812_05902_gb300 import pivbos as P
    P.pivbos_sync()                                   # start from a clear status word
    P.pivbos_selftest_wait_timeout(4096)
    with pytest.raises(P.PivbosError) as err:
        P.pivbos_sync()
    assert err.value.status == P.ERR_DEVICE_TIMEOUT
    P.pivbos_sync()                                   # reported once, then cleared
    fr = scenes.c0(scale=0.01, rays_per_source=20)[0]
    img_g, st_g = gpu_render(fr)
    img_o, st_o = oracle.render_frame(fr)
    compare_images(img_g, img_o, st_g, st_o, fr)
