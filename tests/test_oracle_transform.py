"""Pins of the oracle's transform (CPU only): CDF 9/7 taps, Laplacian pyramid,
directional filter bank, full contourlet transform and their adjoints.

Each check compares the oracle with something other than itself: published
filter taps, a brute-force direct 2-D convolution, an FFT model of the filter
bank, perfect reconstruction, closed-form sizes, dot-product identities.
"""
import os

import numpy as np
import pytest

import oracle as O
import dfb_model

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------- CDF 9/7 (§2.1, [18])
def _golden_taps():
    h = np.zeros(5)
    g = np.zeros(4)
    for line in open(os.path.join(GOLD, "cdf97_taps.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f, n, v = line.split()
        (h if f == "h" else g)[int(n)] = float(v)
    return h, g


def test_cdf97_matches_published_table():
    h, g = O.cdf97()
    hp, gp = _golden_taps()
    np.testing.assert_allclose(h[4:], hp, atol=1e-9)
    np.testing.assert_allclose(g[3:], gp, atol=1e-9)


def test_cdf97_structure():
    h, g = O.cdf97()
    np.testing.assert_allclose(h, h[::-1], atol=0)
    np.testing.assert_allclose(g, g[::-1], atol=0)
    assert abs(h.sum() - np.sqrt(2)) < 1e-14 and abs(g.sum() - np.sqrt(2)) < 1e-14
    # biorthogonality: sum_k h[k] g[k - 2n] = delta[n]
    for n in range(-3, 4):
        s = sum(h[kk + 4] * g[kk - 2 * n + 3] for kk in range(-4, 5) if -3 <= kk - 2 * n <= 3)
        assert abs(s - (1.0 if n == 0 else 0.0)) < 1e-14
    # four zeros at w = pi for both filters: alternating moments vanish up to order 3
    for f, R in ((h, 4), (g, 3)):
        t = np.arange(-R, R + 1)
        for p in range(4):
            assert abs(np.sum(f * (-1.0) ** t * t ** p)) < 1e-12


# ----------------------------------------------------------------- LP (§2.1, Fig. 1)
def _direct_lowpass(x, h):
    """c[m,n] = sum_{a,b} h[a] h[b] x[2m-a, 2n-b], computed with the explicit 9x9 kernel."""
    H, W = x.shape
    K = np.outer(h, h)
    c = np.zeros((H // 2, W // 2))
    for m in range(H // 2):
        for n in range(W // 2):
            rows = (2 * m - np.arange(-4, 5)) % H
            cols = (2 * n - np.arange(-4, 5)) % W
            c[m, n] = np.sum(K * x[np.ix_(rows, cols)])
    return c


def _direct_expand(c, g, H, W):
    """Zero-insertion upsampling followed by periodic 2-D convolution with the 7x7 g g^T."""
    up = np.zeros((H, W))
    up[::2, ::2] = c
    K = np.outer(g, g)
    out = np.zeros((H, W))
    for a in range(-3, 4):
        for b in range(-3, 4):
            out += K[a + 3, b + 3] * np.roll(up, (a, b), axis=(0, 1))
    return out


@pytest.mark.parametrize("shape", [(8, 8), (16, 8), (24, 16), (10, 6)])
def test_lp_analysis_brute_force(shape):
    x = _rng(1).uniform(0, 255, shape)
    h, g = O.cdf97()
    c, d = O.lp_analysis(x)
    c_ref = _direct_lowpass(x, h)
    np.testing.assert_allclose(c, c_ref, atol=1e-10)
    np.testing.assert_allclose(d, x - _direct_expand(c_ref, g, *shape), atol=1e-10)


@pytest.mark.parametrize("shape", [(8, 8), (32, 48), (18, 22), (64, 32)])
def test_lp_perfect_reconstruction(shape):
    x = _rng(2).uniform(0, 255, shape)
    c, d = O.lp_analysis(x)
    np.testing.assert_allclose(O.lp_synthesis(c, d), x, atol=1e-10)


def test_lp_constant_image():
    x = np.full((16, 24), 137.0)
    c, d = O.lp_analysis(x)
    assert np.abs(d).max() < 1e-12
    np.testing.assert_allclose(c, 2 * 137.0, atol=1e-12)  # DC gain (sqrt 2)^2 per level


def test_lp_biorthogonal_2d():
    # down(up(c, g), h) = c  -> synthesis of (c, 0) re-analysed gives back c, zero detail
    c = _rng(3).standard_normal((8, 12))
    x = O.lp_synthesis(c, np.zeros((16, 24)))
    c2, d2 = O.lp_analysis(x)
    np.testing.assert_allclose(c2, c, atol=1e-12)
    assert np.abs(d2).max() < 1e-12


def test_lp_adjoints():
    r = _rng(4)
    H, W = 16, 24
    x = r.standard_normal((H, W))
    cb, db = r.standard_normal((H // 2, W // 2)), r.standard_normal((H, W))
    c, d = O.lp_analysis(x)
    lhs = np.sum(c * cb) + np.sum(d * db)
    rhs = np.sum(x * O.lp_analysis_adjoint(cb, db))
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))
    xb = r.standard_normal((H, W))
    cs, ds = O.lp_synthesis_adjoint(xb)
    lhs = np.sum(O.lp_synthesis(cb, db) * xb)
    rhs = np.sum(cb * cs) + np.sum(db * ds)
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


# ----------------------------------------------------------------- DFB (§2.1)
@pytest.mark.parametrize("k,shape", [(1, (8, 8)), (2, (16, 16)), (3, (16, 24)), (4, (32, 16)),
                                     (5, (32, 32)), (3, (8, 8))])
def test_dfb_matches_frequency_model(k, shape):
    x = _rng(5).standard_normal(shape)
    y = O.dfb(0, x, *shape, k)
    np.testing.assert_allclose(y, dfb_model.analysis(x, k), atol=1e-11)


@pytest.mark.parametrize("k,shape", [(1, (8, 8)), (2, (12, 20)), (3, (16, 24)), (4, (32, 48)),
                                     (5, (64, 32)), (6, (64, 64))])
def test_dfb_perfect_reconstruction(k, shape):
    x = _rng(6).uniform(-100, 100, shape)
    y = O.dfb(0, x, *shape, k)
    np.testing.assert_allclose(O.dfb(1, y, *shape, k), x, atol=1e-10)


def test_dfb_zero_and_linearity():
    r = _rng(7)
    a, b = r.standard_normal((16, 16)), r.standard_normal((16, 16))
    assert np.all(O.dfb(0, np.zeros((16, 16)), 16, 16, 3) == 0)
    np.testing.assert_allclose(O.dfb(0, 2 * a - 3 * b, 16, 16, 3),
                               2 * O.dfb(0, a, 16, 16, 3) - 3 * O.dfb(0, b, 16, 16, 3), atol=1e-12)


@pytest.mark.parametrize("k,floor,mean_floor", [(2, 0.50, 0.62), (3, 0.30, 0.50), (4, 0.15, 0.40)])
def test_dfb_wedges(k, floor, mean_floor):
    """Each subband keeps most of its energy in its own wedge (chance level is 2^-k)."""
    fr = dfb_model.wedge_fractions(k)
    assert min(fr) > floor and np.mean(fr) > mean_floor, fr


def test_dfb_plane_wave_direction():
    """A plane wave well inside a wedge lands mostly in that wedge's subband (k = 3)."""
    H = W = 64
    r, c = np.mgrid[0:H, 0:W]
    chans, _, _ = dfb_model.leaves(H, W, 3)
    sizes = [(H // 4, W // 2)] * 4 + [(H // 2, W // 4)] * 4
    hits = 0
    for idx, ch in enumerate(chans):
        # wedge centre direction
        m = 1
        s_mid = (ch["i"] + 0.5) / 2 ** m
        f = 0.75 * np.pi
        if ch["T"] == "c":
            wc, wr = f / np.hypot(1, s_mid), f * s_mid / np.hypot(1, s_mid)
        else:
            wr, wc = f / np.hypot(1, s_mid), f * s_mid / np.hypot(1, s_mid)
        x = np.cos(wr * r + wc * c)
        y = O.dfb(0, x, H, W, 3)
        e, off = [], 0
        for (h, w) in sizes:
            e.append(np.sum(y[off:off + h * w] ** 2))
            off += h * w
        hits += int(np.argmax(e) == idx)
    assert hits >= 6, hits


# ---------------------------------------------- longer PKVA prototypes
def test_lagrange_taps_of_the_model():
    """the interpolation formula gives the known prototypes: (-1, 9, 9, -1)/16 for
    4 taps (the table the oracle and the model use) and sums of 1"""
    t4 = dfb_model.lagrange_fan_taps(4)
    assert t4 == pytest.approx(dfb_model.BETA_T, abs=1e-15)
    for n in (6, 8):
        t = dfb_model.lagrange_fan_taps(n)
        beta = [(-1.0) ** (((a - 1) // 2) % 2) * v for a, v in sorted(t.items())]
        assert sum(beta) == pytest.approx(1.0, abs=1e-14) and beta == pytest.approx(beta[::-1])
    assert [round(v * 256) for _, v in sorted(dfb_model.lagrange_fan_taps(6).items())] == [-3, -25, -150, 150, 25, 3]


@pytest.mark.parametrize("taps", [6, 8])
@pytest.mark.parametrize("k,shape", [(1, (8, 8)), (2, (16, 16)), (3, (16, 24)), (4, (32, 16)), (5, (32, 32))])
def test_longer_prototype_dfb_matches_frequency_model(taps, k, shape):
    x = _rng(15).standard_normal(shape)
    y = O.dfb(0, x, *shape, k, taps=taps)
    np.testing.assert_allclose(y, dfb_model.analysis(x, k, dfb_model.lagrange_fan_taps(taps)), atol=1e-11)
    np.testing.assert_allclose(O.dfb(1, y, *shape, k, taps=taps), x, atol=1e-10)


@pytest.mark.parametrize("taps", [6, 8])
def test_longer_prototype_adjoints_and_ct(taps):
    r = _rng(16)
    H, W, k = 32, 32, 4
    x, yb = r.standard_normal((H, W)), r.standard_normal(H * W)
    lhs, rhs = np.sum(O.dfb(0, x, H, W, k, taps) * yb), np.sum(x * O.dfb(2, yb, H, W, k, taps))
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))
    lhs, rhs = np.sum(O.dfb(1, yb, H, W, k, taps) * x), np.sum(yb * O.dfb(3, x, H, W, k, taps))
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))
    x = r.uniform(0, 255, (64, 96))
    c = O.ct(0, x, 64, 96, 3, [3, 2, 2], taps)
    np.testing.assert_allclose(O.ct(1, c, 64, 96, 3, [3, 2, 2], taps), x, atol=1e-9)
    assert not np.allclose(c, O.ct(0, x, 64, 96, 3, [3, 2, 2]))     # a different transform


@pytest.mark.parametrize("k", [2, 3, 4])
def test_longer_prototypes_are_more_directional(k):
    """the point of a longer beta: a sharper fan, so more of every subband's energy
    stays in its own wedge"""
    f4 = dfb_model.wedge_fractions(k)
    f6 = dfb_model.wedge_fractions(k, taps=dfb_model.lagrange_fan_taps(6))
    f8 = dfb_model.wedge_fractions(k, taps=dfb_model.lagrange_fan_taps(8))
    assert np.mean(f4) < np.mean(f6) < np.mean(f8)
    assert min(f4) < min(f6) <= min(f8) + 1e-12


def test_dfb_adjoints():
    r = _rng(8)
    for k, (H, W) in ((1, (8, 8)), (3, (16, 24)), (4, (32, 32))):
        x = r.standard_normal((H, W))
        yb = r.standard_normal(H * W)
        lhs = np.sum(O.dfb(0, x, H, W, k) * yb)
        rhs = np.sum(x * O.dfb(2, yb, H, W, k))
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))
        lhs = np.sum(O.dfb(1, yb, H, W, k) * x)
        rhs = np.sum(yb * O.dfb(3, x, H, W, k))
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


# ----------------------------------------------------------------- CT (§2.1, §3.3)
def _closed_form_total(H, W, L):
    # P * (4/3 - 4^-L / 3) for an H x W plane
    return (H * W * (4 ** (L + 1) - 1)) // (3 * 4 ** L)


@pytest.mark.parametrize("H,W,L,k", [(144, 176, 3, [3, 2, 2]), (72, 88, 3, [3, 2, 2]),
                                     (480, 640, 4, [4, 3, 3, 2]), (240, 320, 4, [4, 3, 3, 2]),
                                     (1088, 1920, 5, [5, 4, 4, 3, 3]), (576, 960, 5, [5, 4, 4, 3, 3])])
def test_layout_totals(H, W, L, k):
    lay = O.layout(H, W, L, k)
    assert lay["total"] == _closed_form_total(H, W, L)
    assert len(lay["subbands"]) == 1 + sum(2 ** kk for kk in k)
    offs = [s["off"] for s in lay["subbands"]]
    assert offs == sorted(offs)


def test_layout_frame_totals_match_published_sizes():
    # coefficient counts per frame (Y + two 4:2:0 chroma planes, padded)
    def frame(H, W, Hc, Wc, L, k):
        return O.layout(H, W, L, k)["total"] + 2 * O.layout(Hc, Wc, L, k)["total"]
    assert frame(144, 176, 72, 88, 3, [3, 2, 2]) == 50490
    assert frame(480, 640, 240, 320, 4, [4, 3, 3, 2]) == 613800
    assert frame(1088, 1920, 576, 960, 5, [5, 4, 4, 3, 3]) == 4258800


def test_modulus():
    assert O.modulus(3, [3, 2, 2]) == 8
    assert O.modulus(4, [4, 3, 3, 2]) == 16
    assert O.modulus(5, [5, 4, 4, 3, 3]) == 64


@pytest.mark.parametrize("H,W,L,k", [(64, 64, 3, [3, 2, 2]), (144, 176, 3, [3, 2, 2]),
                                     (64, 128, 4, [4, 3, 3, 2]), (128, 64, 2, [5, 1]), (32, 32, 2, [0, 2])])
def test_ct_perfect_reconstruction(H, W, L, k):
    x = _rng(9).uniform(0, 255, (H, W))
    co = O.ct(0, x, H, W, L, k)
    np.testing.assert_allclose(O.ct(1, co, H, W, L, k), x, atol=1e-10)


def test_ct_constant_image_has_zero_details():
    H, W, L, k = 64, 64, 3, [3, 2, 2]
    co = O.ct(0, np.full((H, W), 77.0), H, W, L, k)
    lay = O.layout(H, W, L, k)
    low = lay["subbands"][0]
    np.testing.assert_allclose(co[:low["h"] * low["w"]], 77.0 * 2 ** L, atol=1e-10)
    assert np.abs(co[low["h"] * low["w"]:]).max() < 1e-11


def test_ct_adjoints():
    r = _rng(10)
    H, W, L, k = 64, 64, 3, [3, 2, 2]
    n = O.layout(H, W, L, k)["total"]
    x, yb = r.standard_normal((H, W)), r.standard_normal(n)
    lhs = np.sum(O.ct(0, x, H, W, L, k) * yb)
    rhs = np.sum(x * O.ct(2, yb, H, W, L, k))
    assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(lhs))
    lhs = np.sum(O.ct(1, yb, H, W, L, k) * x)
    rhs = np.sum(yb * O.ct(3, x, H, W, L, k))
    assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(lhs))


def test_ct_rejects_unaligned_sizes():
    with pytest.raises(ValueError):
        O.ct(0, np.zeros((60, 64)), 60, 64, 3, [3, 2, 2])
