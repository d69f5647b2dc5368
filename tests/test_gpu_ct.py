"""GPU parity of the contourlet transform (forward, inverse and both adjoints)
against the FP64 oracle, through the C ABI.  Tolerance: 1e-4 max abs on the
0-255 scale (the transform's parity bar)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import CtPlan
from paper_1510_00561_b300 import synthetic as S
from tolerances import FORWARD, INVERSE, ROUND_TRIP

pytestmark = pytest.mark.gpu

TOL = FORWARD

CASES = [
    (64, 64, 3, [3, 2, 2]),          # one tile per level
    (144, 176, 3, [3, 2, 2]),        # QCIF luma: ragged 64-tiles
    (200, 136, 3, [3, 2, 2]),        # several tiles plus an 8-wide tail
    (96, 160, 4, [4, 3, 3, 2]),      # VGA-style decomposition
    (64, 96, 2, [0, 1]),             # undivided detail and the quincunx split
    (128, 128, 2, [6, 5]),           # deepest directional trees
    (72, 88, 3, [3, 2, 2]),          # QCIF chroma: tiny coarse levels (9 x 11 lowpass)
]


def _coef_err(c, ref, H, W, L, k):
    """max |c - ref| on the 0-255 scale of the input.  The LP has DC gain 2 per
    level, so level-j coefficients are numbers 2^(j-1) times larger than pixels
    and the lowpass 2^L times (§3.4 normalises it by exactly that factor); each
    is divided by its level's gain before comparing.  In single precision the
    raw coarse-level values (up to 16 * 255 at level 5) carry rounding of ~2e-4
    by themselves, so the bar only makes sense on this scale."""
    lay = O.layout(H, W, L, k)
    d = np.abs(np.asarray(c, np.float64) - ref)
    for sb in lay["subbands"]:
        g = 2.0 ** -L if sb["level"] == 0 else 2.0 ** -(sb["level"] - 1)
        d[sb["off"]:sb["off"] + sb["h"] * sb["w"]] *= g
    return d.max()


def _planes(b, H, W, seed=0):
    return np.random.default_rng(seed).uniform(0, 255, (b, H, W)).astype(np.float32)


@pytest.mark.parametrize("H,W,L,k", CASES)
def test_forward_and_inverse_match_oracle(H, W, L, k):
    x = _planes(2, H, W)
    plan = CtPlan(H, W, L, k, batch=2)
    xt = torch.from_numpy(x).cuda()
    c = plan.forward(xt)
    xr = plan.inverse(c)
    torch.cuda.synchronize()
    c_np, xr_np = c.cpu().numpy(), xr.cpu().numpy()
    for b in range(2):
        ref = O.ct(0, x[b].astype(np.float64), H, W, L, k)
        assert _coef_err(c_np[b], ref, H, W, L, k) < TOL
        # inverse of the same coefficients in the oracle: the parity bar
        xin = O.ct(1, c_np[b].astype(np.float64), H, W, L, k)
        assert np.abs(xr_np[b] - xin).max() < INVERSE
        # GPU round trip: carries the forward's and the inverse's errors
        assert np.abs(xr_np[b] - x[b]).max() < ROUND_TRIP


@pytest.mark.parametrize("H,W,L,k", CASES[:4] + CASES[5:6])
def test_adjoints_match_oracle(H, W, L, k):
    plan = CtPlan(H, W, L, k, batch=1)
    r = np.random.default_rng(3)
    cb = r.standard_normal((1, plan.total)).astype(np.float32) * 50
    xb = r.standard_normal((1, H, W)).astype(np.float32) * 50
    xa = plan.forward_adjoint(torch.from_numpy(cb).cuda()).cpu().numpy()[0]
    ca = plan.inverse_adjoint(torch.from_numpy(xb).cuda()).cpu().numpy()[0]
    # adjoint outputs are gradients, not pixels: their magnitudes grow with the
    # filter-bank depth (values in the thousands for 6 DFB stages), so the bar is
    # relative to the output scale -- 2e-6 of the largest value, ~30 float32 ulps
    for got, ref in ((xa, O.ct(2, cb[0].astype(np.float64), H, W, L, k)),
                     (ca, O.ct(3, xb[0].astype(np.float64), H, W, L, k))):
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


def test_adjoint_dot_products_on_gpu():
    H, W, L, k = 144, 176, 3, [3, 2, 2]
    plan = CtPlan(H, W, L, k, batch=1)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(1, H, W, device="cuda", generator=g, dtype=torch.float32)
    y = torch.randn(1, plan.total, device="cuda", generator=g, dtype=torch.float32)
    lhs = (plan.forward(x).double() * y.double()).sum()
    rhs = (x.double() * plan.forward_adjoint(y).double()).sum()
    assert abs(float(lhs - rhs)) < 1e-4 * float(lhs.abs().clamp(min=1))
    lhs = (plan.inverse(y).double() * x.double()).sum()
    rhs = (y.double() * plan.inverse_adjoint(x).double()).sum()
    assert abs(float(lhs - rhs)) < 1e-4 * float(lhs.abs().clamp(min=1))


def test_batch_entries_are_independent():
    H, W, L, k = 64, 64, 3, [3, 2, 2]
    x = _planes(3, H, W, seed=5)
    p3 = CtPlan(H, W, L, k, batch=3)
    p1 = CtPlan(H, W, L, k, batch=1)
    c3 = p3.forward(torch.from_numpy(x).cuda())
    for b in range(3):
        c1 = p1.forward(torch.from_numpy(x[b:b + 1].copy()).cuda())
        assert torch.equal(c1[0], c3[b])   # same kernels, same arithmetic order: bit-identical


@pytest.mark.parametrize("content", ["uniform", "smooth"])
def test_full_size_1080p_luma(content):
    """The 1080p luma decomposition of the benchmark (1088 x 1920, 5 levels,
    32/16/16/8/8 directions): full forward parity and round trip, on uniform
    noise and on the differentiable workload's planes (a quarter uniform
    noise, three quarters smooth seeded field)."""
    H, W, L, k = 1088, 1920, 5, [5, 4, 4, 3, 3]
    x = _planes(1, H, W, seed=11) if content == "uniform" else S.luma_planes(1, W, H, seed=11)
    plan = CtPlan(H, W, L, k, batch=1)
    xt = torch.from_numpy(x).cuda()
    c = plan.forward(xt)
    xr = plan.inverse(c)
    ref = O.ct(0, x[0].astype(np.float64), H, W, L, k)
    assert _coef_err(c.cpu().numpy()[0], ref, H, W, L, k) < TOL
    xin = O.ct(1, c.cpu().numpy()[0].astype(np.float64), H, W, L, k)
    assert np.abs(xr.cpu().numpy()[0] - xin).max() < INVERSE
    assert float((xr - xt).abs().max()) < ROUND_TRIP


def test_constant_plane_has_zero_details():
    H, W, L, k = 128, 128, 3, [3, 2, 2]
    plan = CtPlan(H, W, L, k)
    c = plan.forward(torch.full((1, H, W), 99.0, device="cuda"))[0].cpu().numpy()
    nlow = (H >> L) * (W >> L)
    np.testing.assert_allclose(c[:nlow], 99.0 * 2 ** L, atol=1e-3)
    assert np.abs(c[nlow:]).max() < 1e-3


@pytest.mark.parametrize("H,W,L,k", [(144, 176, 3, [3, 2, 2]), (72, 88, 3, [3, 2, 2]), (1088, 1920, 5, [5, 4, 4, 3, 3])])
def test_pyramid_tail_gives_the_same_bits(H, W, L, k):
    """With its coarse levels in one block per plane (the pyramid tail, as many levels as fit in
    shared memory: QCIF luma levels 2-3, a whole QCIF chroma plane, 1080p luma level 5), the
    transform and its inverse give exactly the bits of the per-level launches."""
    x = _planes(2, H, W, seed=7)
    xt = torch.from_numpy(x).cuda()
    ref = CtPlan(H, W, L, k, batch=2)
    fused = CtPlan(H, W, L, k, batch=2)
    fused.set_fusion(6)
    c0, c1 = ref.forward(xt), fused.forward(xt)
    assert torch.equal(c0, c1)
    assert torch.equal(ref.inverse(c0), fused.inverse(c1))
