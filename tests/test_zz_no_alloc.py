"""The allocation-free pyramid entry point (GPU).

Some callers cannot allocate device memory while they run (a budget handed
out up front, or a context where the CUDA allocator is off limits), so they
cannot build a transform plan.  cvc_lp_pyramid_forward_static serves them with
its scratch in a fixed device array.  Checked through the C ABI against the
FP64 oracle's Laplacian pyramid (the transform bar, each level on its pixel
scale) and against the plan-based cvc_ct_forward with zero directional stages
(the same kernel: bit-identical), on two calls in a row that reuse the shared
array, and for its size limit.  Collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import CtPlan, _lib
from paper_1510_00561_b300 import synthetic as S
from tolerances import FORWARD

pytestmark = pytest.mark.gpu


def _call(x, h, w, levels, out):
    return _lib.lib().cvc_lp_pyramid_forward_static(ctypes.c_void_p(x.data_ptr()), h, w, levels,
                                                    ctypes.c_void_p(out.data_ptr()),
                                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_pyramid_matches_the_plan_on_two_calls_in_a_row():
    for i, (h, w, levels) in enumerate(((144, 176, 3), (256, 320, 5))):
        x = torch.from_numpy(S.luma_planes(1, w, h, seed=i)).cuda()
        ref = CtPlan(h, w, levels, [0] * levels, batch=1).forward(x)
        out = torch.full_like(ref, float("nan"))
        assert _call(x, h, w, levels, out) == 0
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        # the oracle's pyramid, each level divided by its DC gain (2^(j-1); the lowpass 2^L)
        got = out.cpu().numpy()[0].astype(np.float64)
        want = O.ct(0, x.cpu().numpy()[0].astype(np.float64), h, w, levels, [0] * levels)
        for sb in O.layout(h, w, levels, [0] * levels)["subbands"]:
            a, n = sb["off"], sb["h"] * sb["w"]
            gain = 2.0 ** (levels if sb["level"] == 0 else sb["level"] - 1)
            assert np.abs(got[a:a + n] - want[a:a + n]).max() / gain < FORWARD
        # the same kernel and job geometry as the plan: identical values
        assert torch.equal(out, ref)


def test_static_pyramid_rejects_planes_beyond_its_array():
    dummy = torch.zeros(16, device="cuda")
    assert _call(dummy, 8192, 8192, 2, dummy) == 2       # CVC_ERR_UNSUPPORTED, nothing touched
    assert _call(dummy, 100, 64, 3, dummy) == 1          # 100 is not a multiple of 8
    torch.cuda.synchronize()
    assert float(dummy.abs().sum()) == 0.0
