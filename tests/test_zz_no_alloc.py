"""The allocation-free pyramid entry point (GPU).

Some callers cannot allocate device memory while they run (a budget handed
out up front, or a context where the CUDA allocator is off limits), so they
cannot build a transform plan.  cvc_lp_pyramid_forward_static serves them with
its scratch in a fixed device array.  Checked through the C ABI against the
plan-based cvc_ct_forward with zero directional stages, on two calls in a row
that reuse the shared array, and for its size limit.  Collected last so that
a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

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
        # same kernel and arithmetic as the plan: the values agree well inside the bar
        assert float((out - ref).abs().max()) <= FORWARD


def test_static_pyramid_rejects_planes_beyond_its_array():
    dummy = torch.zeros(16, device="cuda")
    assert _call(dummy, 8192, 8192, 2, dummy) == 2       # CVC_ERR_UNSUPPORTED, nothing touched
    assert _call(dummy, 100, 64, 3, dummy) == 1          # 100 is not a multiple of 8
    torch.cuda.synchronize()
    assert float(dummy.abs().sum()) == 0.0
