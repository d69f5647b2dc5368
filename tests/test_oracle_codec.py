"""Pins of the oracle's integer and codec stages (CPU only): YCoCg-R colour,
4:2:0 chroma, mirror padding, quantiser, run-length coding, K/P frame
differencing and the bitstream.

The expected values are the paper's equations (Table 1), exhaustive
enumeration, hand-worked examples written out below (each with the rule it
exercises), and whole-codec invariants (constant frames decode exactly,
encoder and decoder states agree after every frame).
"""
import numpy as np
import pytest

import oracle as O
from paper_1510_00561_b300 import synthetic as S


# ---------------------------------------------------------- colour (Table 1, Eq. 1-6)
def test_ycocgr_exhaustive_round_trip():
    v = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=-1).astype(np.uint8)
    y, co, cg = O.ycocgr_forward(rgb)
    assert y.min() >= 0 and y.max() <= 255
    assert co.min() >= -255 and co.max() <= 255 and cg.min() >= -255 and cg.max() <= 255
    assert np.array_equal(O.ycocgr_inverse(y, co, cg), rgb)


def test_ycocgr_relates_to_table1():
    """YCoCg-R is Table 1 with the chroma doubled: Co_R = 2 Co exactly (Eq. 2),
    Y_R and Cg_R / 2 within one integer step of Eq. 1 and Eq. 3."""
    rgb = np.random.default_rng(0).integers(0, 256, (100000, 3), dtype=np.uint8)
    y, co, cg = O.ycocgr_forward(rgb)
    R, G, B = (rgb[:, i].astype(np.float64) for i in range(3))
    Yf = R / 4 + G / 2 + B / 4
    Cof = R / 2 - B / 2
    Cgf = -R / 4 + G / 2 - B / 4
    assert np.array_equal(co, 2 * Cof)
    assert np.abs(y - Yf).max() <= 0.75
    assert np.abs(cg - 2 * Cgf).max() <= 1.0
    # and Eq. 4-6 invert Eq. 1-3 in exact arithmetic
    assert np.abs(Yf + Cof - Cgf - R).max() < 1e-12
    assert np.abs(Yf + Cgf - G).max() < 1e-12
    assert np.abs(Yf - Cof - Cgf - B).max() < 1e-12


def test_ycocgr_worked_examples():
    # hand evaluation of Co = R-B, t = B + floor(Co/2), Cg = G - t, Y = t + floor(Cg/2):
    #   (255,0,0): Co=255,  t=0+127=127,     Cg=-127, Y=127+floor(-63.5)=63
    #   (0,0,255): Co=-255, t=255-128=127,   Cg=-127, Y=63
    #   (10,20,30): Co=-20, t=30-10=20,      Cg=0,    Y=20
    cases = {(255, 0, 0): (63, 255, -127), (0, 0, 255): (63, -255, -127), (10, 20, 30): (20, -20, 0)}
    for rgb, exp in cases.items():
        y, co, cg = O.ycocgr_forward(np.array([rgb], np.uint8))
        assert (int(y[0]), int(co[0]), int(cg[0])) == exp


def test_ycocgr_inverse_clamps():
    # out-of-gamut decoded triples clamp to [0, 255]
    rgb = O.ycocgr_inverse(np.array([255], np.int16), np.array([255], np.int16), np.array([255], np.int16))
    # t = 255 - 127 = 128, G = 383 -> 255, B = 128 - 127 = 1, R = 256 -> 255
    assert rgb.tolist() == [[255, 255, 1]]


# ---------------------------------------------------------- chroma (§3.1)
def test_chroma_down_worked_examples():
    # rounded 2x2 mean floor((s+2)/4): s=1 -> 0, s=2 -> 1, s=-2 -> 0, s=-3 -> -1, s=6 -> 2
    blocks = {(0, 0, 0, 1): 0, (1, 1, 0, 0): 1, (-1, -1, 0, 0): 0, (-1, -1, -1, 0): -1, (3, 3, 0, 0): 2}
    for b, exp in blocks.items():
        p = np.array([[b[0], b[1]], [b[2], b[3]]], np.int16)
        assert int(O.chroma_down(p)[0, 0]) == exp


def test_chroma_down_odd_sizes_replicate():
    p = np.array([[4, 8, 12]], np.int16)        # 1 x 3 -> 1 x 2; last column / row replicated
    # block 0: (4 + 8 + 4 + 8) = 24 -> 6 ; block 1: (12 + 12 + 12 + 12) = 48 -> 12
    assert O.chroma_down(p).tolist() == [[6, 12]]


def test_chroma_up_constant_and_ramp():
    c = np.full((5, 7), -37, np.int16)
    assert np.all(O.chroma_up(c, 10, 14) == -37)
    # bilinear interpolation reproduces a linear ramp away from the clamped border:
    # chroma c[i] = 4i sampled at (y - 1/2)/2  ->  value 2y - 1
    c = (4 * np.arange(8, dtype=np.int16))[None, :].repeat(3, 0)
    up = O.chroma_up(c, 6, 16)
    assert np.array_equal(up[:, 1:15], np.broadcast_to(2 * np.arange(1, 15) - 1, (6, 14)))
    assert np.all(up[:, 0] == 0) and np.all(up[:, 15] == 28)   # clamped ends


def test_chroma_up_weights():
    # full-res (1,1) of a 2x2 chroma grid: nearest (0,0) weight 9, (1,0) 3, (0,1) 3, (1,1) 1
    c = np.array([[16, 0], [0, 0]], np.int16)
    up = O.chroma_up(c, 4, 4)
    assert up[1, 1] == (9 * 16 + 8) // 16 and up[2, 2] == (1 * 16 + 8) // 16
    assert up[0, 0] == 16 and up[1, 2] == (3 * 16 + 8) // 16


def test_pad_mirror():
    p = np.arange(6, dtype=np.float64).reshape(2, 3)
    out = O.pad_mirror(p, 4, 5)
    assert out.tolist() == [[0, 1, 2, 2, 1], [3, 4, 5, 5, 4], [3, 4, 5, 5, 4], [0, 1, 2, 2, 1]]


# ---------------------------------------------------------- quantiser (§3.4-§3.6)
def test_quantize_rounding_and_ties():
    assert O.quantize(2.5 * 8, 8, 0.0, False, 3) == 3          # tie rounds away from zero
    assert O.quantize(-2.5 * 8, 8, 0.0, False, 3) == -3
    assert O.quantize(2.49 * 8, 8, 0.0, False, 3) == 2
    assert O.quantize(7.4, 1, 0.0, False, 3) == 7               # QP = 1: plain rounding (§3.5)
    assert O.quantize(0.5, 1, 0.0, False, 3) == 1
    assert O.quantize(-0.5, 1, 0.0, False, 3) == -1


def test_quantize_threshold_subbands_only():
    assert O.quantize(3.9, 1, 4.0, False, 3) == 0               # |c| < T -> zero
    assert O.quantize(-4.0, 1, 4.0, False, 3) == -4             # |c| >= T kept
    assert O.quantize(3.0 * 8, 1, 100.0, True, 3) == 3          # lowpass is not thresholded


def test_quantize_lowpass_normalisation():
    # lowpass scaled by 2^-L before dividing by QPL: c = 8 * 100.5 * 2 -> 201/2 = 100.5 -> 101
    assert O.quantize(8 * 100.5 * 2, 2, 0.0, True, 3) == 101
    assert O.quantize(32 * 255.0, 1, 0.0, True, 5) == 255


def test_quantize_overflow():
    with pytest.raises(OverflowError):
        O.quantize(32767.6, 1, 0.0, False, 3)
    assert O.quantize(32767.4, 1, 0.0, False, 3) == 32767


def test_quantize_power_of_two_is_exact_division():
    # for QP a power of two, float and double division agree, so the decision is unambiguous
    c = np.random.default_rng(1).standard_normal(20000).astype(np.float32) * 300
    for qp in (1, 2, 4, 8, 16):
        q = np.array([O.quantize(float(v), qp, 0.0, False, 3) for v in c[:2000]])
        t = c[:2000].astype(np.float64) / qp
        ref = np.sign(t) * np.floor(np.abs(t) + 0.5)
        assert np.array_equal(q, ref)


# ---------------------------------------------------------- RLE (§3.8)
@pytest.mark.parametrize("row,tokens", [
    ([0, 0, 3, 0, -1], [0, 2, 3, 0, 1, -1]),
    ([0, 0, 0, 0, 0], [0, 5]),
    ([5, -6, 7], [5, -6, 7]),
    ([1, 0, 1, 0, 1, 0], [1, 0, 1, 1, 0, 1, 1, 0, 1]),
    ([0], [0, 1]),
    ([9], [9]),
    ([-32767, 0, 0, 32767], [-32767, 0, 2, 32767]),
])
def test_rle_worked_examples(row, tokens):
    assert O.rle_row(np.array(row, np.int16)).tolist() == tokens
    assert O.rle_expand(np.array(tokens, np.int16), len(row)).tolist() == row


def test_rle_round_trip_random():
    r = np.random.default_rng(2)
    for _ in range(50):
        w = int(r.integers(1, 200))
        row = (r.integers(-3, 4, w) * (r.random(w) < 0.3)).astype(np.int16)
        tok = O.rle_row(row)
        assert np.array_equal(O.rle_expand(tok, w), row)
        assert tok.size == np.count_nonzero(row) + 2 * np.count_nonzero(np.diff(np.r_[1, row != 0].astype(int)) == -1)


@pytest.mark.parametrize("tokens,n", [([0], 1), ([0, 0], 1), ([0, 3], 2), ([1, 2], 1), ([0, -1], 1), ([], 1)])
def test_rle_rejects_corrupt(tokens, n):
    with pytest.raises(ValueError):
        O.rle_expand(np.array(tokens, np.int16), n)


# ---------------------------------------------------------- codec (§3.7-§3.9)
QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=8)


def _codec(**kw):
    p = dict(QCIF)
    p.update(kw)
    return O.Codec(**p)


def test_header_layout():
    c = _codec(width=40, height=24, levels=2, dirs_log2=[2, 1], qph=12, qpl=3, key_interval=4)
    frame = np.full((24, 40, 3), 90, np.uint8)
    s, ft = c.encode(frame)
    assert ft == 0
    hdr = bytes(s[:32])
    assert hdr[:4] == b"CVC1" and hdr[4:6] == b"\x01\x00" and hdr[6] == 0 and hdr[7] == 2
    assert hdr[8:12] == b"\x00\x00\x00\x00"
    assert int.from_bytes(hdr[12:14], "little") == 24 and int.from_bytes(hdr[14:16], "little") == 40
    assert list(hdr[16:22]) == [2, 1, 0, 0, 0, 0]
    assert int.from_bytes(hdr[22:24], "little") == 12 and int.from_bytes(hdr[24:26], "little") == 3
    ncomp = int.from_bytes(hdr[28:32], "little")
    assert ncomp == 3 * (1 + 4 + 2)


def test_constant_frame_stream_is_exact():
    """A flat frame has zero details: every subband row codes as (0, width), the
    K-frame lowpass is raw with a first-difference column filter (first row = value,
    the rest 0), and the frame decodes exactly."""
    c = _codec()
    frame = np.zeros((144, 176, 3), np.uint8)
    frame[...] = (100, 150, 50)
    s, ft = c.encode(frame)
    y, co, cg = O.ycocgr_forward(frame[:1, :1])
    ncomp = c.ncomp
    counts = np.frombuffer(bytes(s[32:32 + 4 * ncomp]), "<u4")
    tok = np.frombuffer(bytes(s[32 + 4 * ncomp:]), "<i2")
    lays = [O.layout(144, 176, 3, [3, 2, 2])] + [O.layout(72, 88, 3, [3, 2, 2])] * 2
    pos, j = 0, 0
    for p, lay in enumerate(lays):
        val = [int(y[0, 0]), int(co[0, 0]), int(cg[0, 0])][p]
        for sb in lay["subbands"]:
            t = tok[pos:pos + counts[j]]
            if sb["kind"] == 0:
                exp = np.zeros((sb["h"], sb["w"]), np.int16)
                exp[0, :] = val                       # QPL = 1, lowpass = value exactly
                assert np.array_equal(t, exp.ravel())
            else:
                assert np.array_equal(t, np.tile([0, sb["w"]], sb["h"]))
            pos += counts[j]
            j += 1
    assert np.array_equal(c.decode(s), frame)
    # the next (P) frame of the same content: every component is one zero run per row
    s2, ft2 = c.encode(frame)
    assert ft2 == 1
    assert s2.size == 32 + 4 * ncomp + 2 * 2 * sum(sb["h"] for lay in lays for sb in lay["subbands"])
    assert np.array_equal(c.decode(s2), frame)


def test_frame_types_and_state_agreement():
    v = S.SyntheticVideo(S.spec_for(176, 144, seed=3))
    c = _codec()
    dec = _codec()
    types = []
    for t in range(10):
        f = v.frame(t)
        s, ft = c.encode(f)
        types.append(ft)
        r1 = c.decode(s)          # the encoder object's own decoder
        r2 = dec.decode(s)        # an independent decoder instance
        assert np.array_equal(r1, r2)
        psnr = 10 * np.log10(255.0 ** 2 / np.mean((r1.astype(float) - f) ** 2))
        assert psnr > 28.0
    assert types == [0, 1, 1, 1, 1, 1, 1, 1, 0, 1]


def test_near_lossless_at_unit_steps():
    """QPH = QPL = 1: only coefficient rounding (§3.6) and the 4:2:0 chroma path lose
    information; luma stays above 45 dB (the paper reports 58.93 dB for rounding
    alone on natural images, §3.6 -- context, not a bound)."""
    v = S.SyntheticVideo(S.spec_for(176, 144, seed=1))
    c = _codec(qph=1, qpl=1)
    f = v.frame(0)
    s, _ = c.encode(f)
    r = c.decode(s)
    yf = O.ycocgr_forward(f)[0].astype(float)
    yr = O.ycocgr_forward(r)[0].astype(float)
    assert 10 * np.log10(255.0 ** 2 / np.mean((yf - yr) ** 2)) > 45.0


def test_decoder_requires_key_frame_first():
    v = S.SyntheticVideo(S.spec_for(176, 144))
    c = _codec()
    c.encode(v.frame(0))
    s1, ft = c.encode(v.frame(1))
    assert ft == 1
    fresh = _codec()
    assert fresh.decode_status(s1) == O.ESTATE


def test_decoder_rejects_corruption():
    v = S.SyntheticVideo(S.spec_for(176, 144))
    c = _codec()
    s, _ = c.encode(v.frame(0))
    d = _codec()
    bad = s.copy()
    bad[0] = ord("X")
    assert d.decode_status(bad) == O.ECORRUPT
    assert d.decode_status(s[:-2]) == O.ECORRUPT
    bad = s.copy()
    bad[32:36] = 0   # first component claims zero tokens
    assert d.decode_status(bad) == O.ECORRUPT


def test_wrapping_differences_are_lossless():
    """K/P differences wrap in 16 bits (§3.7 reading): an extreme code change between
    two frames is still carried exactly by the P-frame residual tokens."""
    c = _codec(width=16, height=16, levels=1, dirs_log2=[1], qph=1, qpl=1, key_interval=100)
    n = c.ncoef
    rng = np.random.default_rng(4)
    a = rng.integers(-16000, 16000, n).astype(np.float32)
    b = -a
    c.encode_from_coeffs(a)
    s1, ft = c.encode_from_coeffs(b)
    assert ft == 1
    lays = [O.layout(16, 16, 1, [1])] + [O.layout(8, 8, 1, [1])] * 2
    counts = np.frombuffer(bytes(s1[32:32 + 4 * c.ncomp]), "<u4")
    tok = np.frombuffer(bytes(s1[32 + 4 * c.ncomp:]), "<i2")
    pos, j, base = 0, 0, 0
    for lay in lays:
        for sb in lay["subbands"]:
            m = sb["h"] * sb["w"]
            low = sb["kind"] == 0
            qa = np.array([O.quantize(float(v), 1, 0.0, low, 1) for v in a[base + sb["off"]:base + sb["off"] + m]])
            qb = np.array([O.quantize(float(v), 1, 0.0, low, 1) for v in b[base + sb["off"]:base + sb["off"] + m]])
            exp = ((qb - qa) & 0xFFFF).astype(np.uint16).view(np.int16)
            got = O.rle_expand(tok[pos:pos + counts[j]], m)
            assert np.array_equal(got, exp)
            pos += counts[j]
            j += 1
        base += lay["total"]
