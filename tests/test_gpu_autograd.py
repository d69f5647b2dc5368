"""Differentiable contourlet transform on the GPU (autograd Functions whose
backward passes are the hand-written adjoint kernels), against the FP64
oracle:

  - soft thresholding forward / backward kernels on identical FP32 inputs;
  - the gradients of the threshold-tuning loss mean((S soft_T(A x) - x)^2)
    with respect to the 80 subband thresholds and to the pixels, against the
    oracle's adjoint-chain gradient and against FP64 central differences
    (eps = 1e-3) of the oracle's loss on 16 thresholds and 16 pixels;
  - the full differentiable workload: batch 8 of 1920x1080 luma planes
    (padded to 1088 rows), 5 levels, 32/16/16/8/8 directions.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import CtPlan, kernel_launches
from paper_1510_00561_b300 import synthetic as S
from paper_1510_00561_b300.autograd import ThresholdedReconstruction, ct_forward, ct_inverse
from tolerances import GRAD_REL, SUM_REL

pytestmark = pytest.mark.gpu

L5, K5 = 5, [5, 4, 4, 3, 3]


def _rel(a, b):
    return float(np.abs(a - b).max() / max(1e-30, np.abs(b).max()))


def test_soft_threshold_kernels_match_oracle():
    H, W, B = 256, 192, 2
    plan = CtPlan(H, W, L5, K5, batch=B)
    assert plan.subbands == 80
    g = torch.Generator().manual_seed(0)
    c = (torch.randn((B, plan.total), generator=g) * 6).float()
    T = (torch.rand(80, generator=g) * 6 + 0.5).float()
    gy = torch.randn((B, plan.total), generator=g).float()
    y = plan.soft_threshold(c.cuda(), T.cuda()).cpu().numpy()
    ref = O.soft_threshold(c.double().numpy(), H, W, L5, K5, T.double().numpy())
    assert np.abs(y - ref).max() <= 2.0 ** -23 * np.abs(c.numpy()).max()
    gc, gT = plan.soft_threshold_backward(c.cuda(), T.cuda(), gy.cuda())
    gc_ref, gT_ref = O.soft_threshold_vjp(c.double().numpy(), H, W, L5, K5, T.double().numpy(), gy.double().numpy())
    assert np.array_equal(gc.cpu().numpy().astype(np.float64), gc_ref)
    lay = O.layout(H, W, L5, K5)
    for s, sb in enumerate(lay["subbands"][1:]):
        mag = np.abs(gy.double().numpy()[:, sb["off"]:sb["off"] + sb["h"] * sb["w"]]).sum()
        assert abs(float(gT[s]) - gT_ref[s]) <= SUM_REL * mag
    # repeatable bit for bit
    gc2, gT2 = plan.soft_threshold_backward(c.cuda(), T.cuda(), gy.cuda())
    assert torch.equal(gT, gT2) and torch.equal(gc, gc2)


def _model_grads(x_np, T_np):
    B, H, W = x_np.shape
    model = ThresholdedReconstruction(H, W, L5, K5, B)
    with torch.no_grad():
        model.T.copy_(torch.from_numpy(T_np).float())
    x = torch.from_numpy(x_np).float().cuda().requires_grad_(True)
    n0 = kernel_launches()
    loss = torch.mean((model(x) - x) ** 2)
    loss.backward()
    torch.cuda.synchronize()
    assert kernel_launches() > n0            # forward and backward ran in the library's kernels
    return float(loss.detach()), model.T.grad.cpu().numpy().astype(np.float64), x.grad.cpu().numpy().astype(np.float64)


def test_loss_gradients_match_oracle_and_finite_differences():
    B, H, W = 2, 128, 128
    x = S.luma_planes(B, W, H, seed=3).astype(np.float64)
    rng = np.random.default_rng(7)
    T = rng.uniform(2, 6, 80)
    lay = O.layout(H, W, L5, K5)
    c = np.stack([O.ct(0, x[b], H, W, L5, K5) for b in range(B)])
    eps = 1e-3
    for s in range(80):     # keep every magnitude 2 eps away from its threshold
        sb = lay["subbands"][s + 1]
        while np.min(np.abs(np.abs(c[:, sb["off"]:sb["off"] + sb["h"] * sb["w"]]) - T[s])) <= 2 * eps:
            T[s] += 7 * eps
    loss, gT, gx = _model_grads(x, T)
    loss_ref, gT_ref, gx_ref = O.threshold_loss(x, L5, K5, T)
    assert abs(loss - loss_ref) <= GRAD_REL * loss_ref
    assert _rel(gT, gT_ref) <= GRAD_REL
    assert _rel(gx, gx_ref) <= GRAD_REL
    # FP64 central differences of the oracle's loss
    f = lambda xx, TT: O.threshold_loss(xx, L5, K5, TT, want_grad=False)
    for s in rng.choice(80, 16, replace=False):
        d = np.zeros(80)
        d[s] = eps
        fd = (f(x, T + d) - f(x, T - d)) / (2 * eps)
        assert abs(gT[s] - fd) <= GRAD_REL * np.abs(gT_ref).max()
    done = 0
    for p in rng.permutation(B * H * W)[:64]:
        b, yy, xx = np.unravel_index(p, (B, H, W))
        d = np.zeros_like(x)
        d[b, yy, xx] = eps
        ok = True
        for sgn in (1, -1):
            cc = O.ct(0, (x + sgn * d)[b], H, W, L5, K5)
            ok &= np.array_equal(np.abs(O.soft_threshold(cc, H, W, L5, K5, T)) > 0,
                                 np.abs(O.soft_threshold(c[b], H, W, L5, K5, T)) > 0)
        if not ok:
            continue
        fd = (f(x + d, T) - f(x - d, T)) / (2 * eps)
        assert abs(gx[b, yy, xx] - fd) <= GRAD_REL * np.abs(gx_ref).max()
        done += 1
        if done == 16:
            break
    assert done == 16


def test_adjoint_functions_are_transposes():
    B, H, W = 2, 128, 192
    plan = CtPlan(H, W, L5, K5, batch=B)
    g = torch.Generator().manual_seed(1)
    x = torch.randn((B, H, W), generator=g).cuda().requires_grad_(True)
    c = torch.randn((B, plan.total), generator=g).cuda().requires_grad_(True)
    u = torch.randn((B, plan.total), generator=g).cuda()
    v = torch.randn((B, H, W), generator=g).cuda()
    (ct_forward(x, plan) * u).sum().backward()       # x.grad = A^T u
    (ct_inverse(c, plan) * v).sum().backward()       # c.grad = S^T v
    with torch.no_grad():
        lhs1 = float((plan.forward(x.detach()).double() * u.double()).sum())
        rhs1 = float((x.detach().double() * x.grad.double()).sum())
        lhs2 = float((plan.inverse(c.detach()).double() * v.double()).sum())
        rhs2 = float((c.detach().double() * c.grad.double()).sum())
    assert abs(lhs1 - rhs1) <= 1e-5 * abs(lhs1) + 1e-3
    assert abs(lhs2 - rhs2) <= 1e-5 * abs(lhs2) + 1e-3


def test_full_size_differentiable_workload():
    """Batch 8 of 1920x1080 planes padded to 1088 rows, thresholds 4.0: the
    80 threshold gradients and 16 pixel gradients against the oracle."""
    B, H, W = 8, 1088, 1920
    x = S.luma_planes(B, W, H, seed=0).astype(np.float64)
    T = np.full(80, 4.0)
    loss, gT, gx = _model_grads(x, T)
    loss_ref, gT_ref, gx_ref = O.threshold_loss(x, L5, K5, T)
    assert abs(loss - loss_ref) <= GRAD_REL * loss_ref
    assert _rel(gT, gT_ref) <= GRAD_REL
    idx = np.random.default_rng(0).choice(B * H * W, 16, replace=False)
    assert np.abs(gx.ravel()[idx] - gx_ref.ravel()[idx]).max() <= GRAD_REL * np.abs(gx_ref).max()
