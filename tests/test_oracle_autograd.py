"""Pins of the oracle's soft thresholding and of the threshold-tuning loss
gradient (FP64, CPU).  Every check ties the oracle to something other than
its own formulas:

  - the soft threshold is the proximal map of T|z|: brute-force minimisation
    of (z - c)^2 / 2 + T |z| over a fine grid picks the same value;
  - its vector-Jacobian product matches central finite differences of the
    soft threshold itself;
  - the loss gradients (through the adjoint transforms) match central finite
    differences of the loss in FP64 with eps = 1e-3, on 16 threshold entries
    and 16 pixels, at points where no coefficient crosses its threshold
    within eps (the loss is then exactly quadratic, so the central difference
    has no truncation error);
  - T = 0 reconstructs exactly (perfect reconstruction) with zero gradients;
    thresholds above every magnitude zero the subbands and their gradients.
"""
import numpy as np
import pytest

import oracle as O

CFG = (64, 64, 5, [5, 4, 4, 3, 3])     # the differentiable workload's decomposition on a small plane
SMALL = (32, 32, 2, [3, 2])


def _nsub(H, W, L, k):
    return len(O.layout(H, W, L, k)["subbands"]) - 1


def test_soft_threshold_is_the_proximal_map():
    H, W, L, k = SMALL
    rng = np.random.default_rng(0)
    n = O.layout(H, W, L, k)["total"]
    c = rng.normal(0, 6, n)
    T = rng.uniform(0.5, 8, _nsub(H, W, L, k))
    y = O.soft_threshold(c, H, W, L, k, T)
    lay = O.layout(H, W, L, k)
    z = np.linspace(-40, 40, 160001)          # grid step 5e-4
    for s, sb in enumerate(lay["subbands"]):
        idx = sb["off"] + rng.integers(0, sb["h"] * sb["w"], 4)
        for i in idx:
            if s == 0:
                assert y[i] == c[i]
                continue
            obj = 0.5 * (z - c[i]) ** 2 + T[s - 1] * np.abs(z)
            assert abs(z[np.argmin(obj)] - y[i]) <= 5e-4


def test_soft_threshold_vjp_matches_finite_differences():
    H, W, L, k = SMALL
    rng = np.random.default_rng(1)
    n = O.layout(H, W, L, k)["total"]
    c = rng.normal(0, 6, (2, n))
    T = rng.uniform(0.5, 8, _nsub(H, W, L, k))
    g = rng.normal(0, 1, (2, n))
    eps = 1e-4
    lay = O.layout(H, W, L, k)
    for s in range(len(T)):          # no magnitude within 2 eps of its threshold: f is linear there
        while not _kink_free(c, lay, T, s, eps):
            T[s] += 7 * eps
    gc, gT = O.soft_threshold_vjp(c, H, W, L, k, T, g)
    f = lambda cc, TT: float(np.sum(g * O.soft_threshold(cc, H, W, L, k, TT)))
    for s in range(len(T)):
        d = np.zeros_like(T)
        d[s] = eps
        fd = (f(c, T + d) - f(c, T - d)) / (2 * eps)
        assert abs(fd - gT[s]) <= 1e-6 * max(1.0, abs(gT[s]))
    T_of = np.zeros(n, dtype=int) - 1
    for si, sb in enumerate(lay["subbands"][1:]):
        T_of[sb["off"]:sb["off"] + sb["h"] * sb["w"]] = si
    for i in rng.integers(0, n, 20):
        if T_of[i] >= 0 and abs(abs(c[1, i]) - T[T_of[i]]) <= 2 * eps:
            continue
        d = np.zeros_like(c)
        d[1, i] = eps
        fd = (f(c + d, T) - f(c - d, T)) / (2 * eps)
        assert abs(fd - gc[1, i]) <= 1e-6


def _kink_free(c, lay, T, s, eps):
    sb = lay["subbands"][s + 1]
    v = np.abs(c[:, sb["off"]:sb["off"] + sb["h"] * sb["w"]])
    return np.min(np.abs(v - T[s])) > 2 * eps


def test_loss_gradient_matches_finite_differences():
    H, W, L, k = CFG
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 255, (2, H, W)) * 0.25 + 100.0
    lay = O.layout(H, W, L, k)
    nT = _nsub(H, W, L, k)
    assert nT == 80
    T = rng.uniform(2, 6, nT)
    c = np.stack([O.ct(0, x[b], H, W, L, k) for b in range(2)])
    eps = 1e-3
    # move thresholds off the coefficient magnitudes so that +-eps crosses no kink
    for s in range(nT):
        while not _kink_free(c, lay, T, s, eps):
            T[s] += 7 * eps
    loss, gT, gx = O.threshold_loss(x, L, k, T)
    for s in rng.choice(nT, 16, replace=False):
        d = np.zeros(nT)
        d[s] = eps
        fd = (O.threshold_loss(x, L, k, T + d, want_grad=False) - O.threshold_loss(x, L, k, T - d, want_grad=False)) / (2 * eps)
        assert abs(fd - gT[s]) <= 1e-7 * max(1e-3, np.abs(gT).max()), (s, fd, gT[s])
    checked = 0
    for p in rng.permutation(H * W):
        b, yy, xx = p % 2, (p // 2) % H, (p // (2 * H)) % W
        d = np.zeros_like(x)
        d[b, yy, xx] = eps
        cp = np.stack([O.ct(0, (x + d)[i], H, W, L, k) for i in range(2)])
        cm = np.stack([O.ct(0, (x - d)[i], H, W, L, k) for i in range(2)])
        mask = lambda cc: np.abs(O.soft_threshold(cc, H, W, L, k, T)) > 0
        if not (np.array_equal(mask(cp), mask(c)) and np.array_equal(mask(cm), mask(c))):
            continue      # a coefficient crosses its threshold within eps: not a quadratic piece
        fd = (O.threshold_loss(x + d, L, k, T, want_grad=False) - O.threshold_loss(x - d, L, k, T, want_grad=False)) / (2 * eps)
        assert abs(fd - gx[b, yy, xx]) <= 1e-7 * max(1e-3, np.abs(gx).max()), (b, yy, xx, fd, gx[b, yy, xx])
        checked += 1
        if checked == 16:
            break
    assert checked == 16


def test_zero_thresholds_reconstruct_exactly():
    H, W, L, k = CFG
    x = np.random.default_rng(3).uniform(0, 255, (1, H, W))
    loss, gT, gx = O.threshold_loss(x, L, k, np.zeros(_nsub(H, W, L, k)))
    assert loss < 1e-20 and np.abs(gx).max() < 1e-11 and np.abs(gT).max() < 1e-9


def test_huge_thresholds_keep_only_the_lowpass():
    H, W, L, k = CFG
    x = np.random.default_rng(4).uniform(0, 255, (1, H, W))
    c = O.ct(0, x[0], H, W, L, k)
    T = np.full(_nsub(H, W, L, k), np.abs(c).max() + 1)
    y = O.soft_threshold(c, H, W, L, k, T)
    low = O.layout(H, W, L, k)["subbands"][0]
    n_low = low["h"] * low["w"]
    assert np.array_equal(y[:n_low], c[:n_low]) and not y[n_low:].any()
    loss, gT, gx = O.threshold_loss(x, L, k, T)
    assert not gT.any()
    # only the lowpass survives: the reconstruction is the pyramid's coarse approximation
    xr = O.ct(1, y, H, W, L, k)
    assert loss == pytest.approx(np.mean((xr - x[0]) ** 2), rel=1e-12)
