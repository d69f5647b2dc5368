"""Pins of the oracle's 8-bit storage variant (§3.1 Table 1, §3.5, §3.6):

  - Table 1 in its real-valued form, each component rounded to a byte, chroma
    offset by +127: the values of the primaries and greys worked out by hand;
  - the round trip of every one of the 2^24 RGB colours is within 1 of the
    colour (each of the three roundings errs by at most 1/2 and the inverse
    has unit coefficients, so the error is at most 3/2, an integer);
  - the quantiser: hand-worked cases of one rounding of the quotient and of
    the byte clamp of the code;
  - a grey frame decodes exactly; at QPH = 181 the synthetic K-frame's
    subband codes are -1, 1 or zero runs, almost all zero; header byte 5
    records the storage, and a decoder of the other storage refuses the
    stream.
"""
import numpy as np
import pytest

import oracle as O
from paper_1510_00561_b300 import synthetic as S


def test_table1_values_of_primaries_and_greys():
    rgb = np.array([[0, 0, 0], [255, 255, 255], [255, 0, 0], [0, 255, 0], [0, 0, 255], [10, 20, 30],
                    [1, 0, 0], [0, 0, 1], [0, 1, 0], [128, 128, 128]], np.uint8)
    y, co, cg = O.ycocg8_forward(rgb)
    # red: Y = 63.75 -> 64, Co = 127.5 -> 128 (+127 = 255), Cg = -63.75 -> -64 (+127 = 63)
    # green: Y = 127.5 -> 128, Cg = 127.5 -> 128 -> 255; blue: Co = -127.5 -> -128 -> -1 -> 0
    # (1,0,0): Y 0.25 -> 0, Co 0.5 -> 1; (0,0,1): Co -0.5 -> -1; (0,1,0): Y 0.5 -> 1, Cg 0.5 -> 1
    assert y.tolist() == [0, 255, 64, 128, 64, 20, 0, 0, 1, 128]
    assert co.tolist() == [127, 127, 255, 127, 0, 117, 128, 126, 127, 127]
    assert cg.tolist() == [127, 127, 63, 255, 63, 127, 127, 127, 128, 127]
    back = O.ycocg8_inverse(y, co, cg)
    # blue: Y 64, Co -127 (the clamp), Cg -64 gives R = 64 - 127 + 64 = 1: within the bound below
    assert back[:5].tolist() == [[0, 0, 0], [255, 255, 255], [255, 0, 0], [0, 255, 0], [1, 0, 255]]


def test_every_colour_round_trips_within_one():
    v = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8)
    y, co, cg = O.ycocg8_forward(rgb)
    for p in (y, co, cg):
        assert p.min() >= 0 and p.max() <= 255
    back = O.ycocg8_inverse(y, co, cg)
    err = np.abs(back.astype(np.int16) - rgb.astype(np.int16))
    assert err.max() == 1
    grey = (rgb[:, 0] == rgb[:, 1]) & (rgb[:, 1] == rgb[:, 2])
    assert err[grey].max() == 0
    # reported, not pinned: the share of colours that come back exactly, and the PSNR
    exact = (err.max(axis=1) == 0).mean()
    psnr = 10 * np.log10(255.0 ** 2 / (err.astype(np.float64) ** 2).mean())
    assert 0.2 < exact < 1.0 and psnr > 50


def test_quantiser_keeps_codes_in_a_byte():
    q = O.quantize8
    assert [q(c, 1, 0.0, False, 3) for c in (200.4, -300.0, 12.5, -12.5, 12.4, 127.4, -128.4)] == \
        [127, -128, 13, -13, 12, 127, -128]
    # one rounding, of the quotient (§3.5 then §3.6): 0.6 / 2 = 0.3 -> 0, 1.4 / 2 -> 1
    assert q(0.6, 2, 0.0, False, 3) == 0 and q(1.4, 2, 0.0, False, 3) == 1 and q(-3.0, 2, 0.0, False, 3) == -2
    # QPH = 181: 0 exactly when |c| < 90.5; the byte bounds the code, not the coefficient
    assert q(90.4, 181, 0.0, False, 3) == 0 and q(90.6, 181, 0.0, False, 3) == 1
    assert q(-90.6, 181, 0.0, False, 3) == -1 and q(271.4, 181, 0.0, False, 3) == 1
    assert q(271.6, 181, 0.0, False, 3) == 2 and q(1e6, 181, 0.0, False, 3) == 127
    rng = np.random.default_rng(0)
    codes = [q(float(c), 7, 0.0, False, 3) for c in rng.normal(0, 2000, 2000)]
    assert min(codes) == -128 and max(codes) == 127
    # lowpass (3 levels): normalised by 1/8, divided, rounded, clamped to [0, 255]
    assert q(8 * 100.5, 1, 0.0, True, 3) == 101 and q(8 * 300.0, 1, 0.0, True, 3) == 255
    assert q(-8.0, 1, 0.0, True, 3) == 0 and q(8 * 255.0, 71, 0.0, True, 3) == 4
    # the subband threshold acts first
    assert q(5.0, 1, 6.0, False, 3) == 0 and q(-6.0, 1, 6.0, False, 3) == -6


QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4)


@pytest.mark.parametrize("v", [0, 77, 255])
def test_grey_frames_decode_exactly(v):
    c = O.Codec(**QCIF, storage8=True)
    d = O.Codec(**QCIF, storage8=True)
    f = np.full((144, 176, 3), v, np.uint8)
    for _ in range(3):                               # a K-frame, then P-frames
        s, _ = c.encode(f)
        assert s[5] == 1
        assert np.array_equal(d.decode(s), f)


def _directional_tokens(stream, c):
    """per component: (is_lowpass, tokens) of a frame"""
    hdr = 32 + 4 * c.ncomp
    counts = np.frombuffer(stream[32:hdr].tobytes(), "<u4")
    toks = np.frombuffer(stream[hdr:hdr + 2 * int(counts.sum())].tobytes(), "<i2")
    out, pos = [], 0
    nlow = 1 + sum(1 << k for k in c.dirs)         # components of one plane
    for j, n in enumerate(counts):
        out.append((j % nlow == 0, toks[pos:pos + n]))
        pos += n
    return out


def test_qph_181_leaves_only_unit_codes():
    """§3.5: the paper says QPH = 181 zeroes every subband element, which holds
    exactly when every coefficient is below 90.5 in magnitude.  On the synthetic
    frame the codes are -1, 0 or 1 and almost all zero (measured)."""
    kw = dict(QCIF, qph=181, qpl=12)
    c = O.Codec(**kw, storage8=True)
    nz = total = 0
    for f in S.SyntheticVideo(S.spec_for(176, 144, seed=3)).frames(1):
        s, ft = c.encode(f)
        assert ft == 0
        for low, t in _directional_tokens(s, c):
            if low:
                continue
            i = 0
            while i < len(t):
                if t[i] == 0:                          # a zero run: (0, n)
                    total += int(t[i + 1])
                    i += 2
                else:
                    assert t[i] in (-1, 1)
                    nz += 1
                    total += 1
                    i += 1
    assert total > 0 and nz / total < 0.05


def test_header_records_the_storage():
    f = S.SyntheticVideo(S.spec_for(176, 144, seed=4)).frame(0)
    s8, _ = O.Codec(**QCIF, storage8=True).encode(f)
    s16, _ = O.Codec(**QCIF).encode(f)
    assert s8[5] == 1 and s16[5] == 0
    with pytest.raises(RuntimeError, match="status 5"):
        O.Codec(**QCIF).decode(s8)
    with pytest.raises(RuntimeError, match="status 5"):
        O.Codec(**QCIF, storage8=True).decode(s16)
    # at QPH = QPL = 1 the bytes cost little next to the 4:2:0 chroma, which
    # dominates the RGB error of both storages on these coloured edges
    kw = dict(QCIF, qph=1, qpl=1)

    def psnr(st8):
        c, d = O.Codec(**kw, storage8=st8), O.Codec(**kw, storage8=st8)
        rgb = d.decode(c.encode(f)[0])
        return 10 * np.log10(255.0 ** 2 / ((rgb.astype(np.float64) - f) ** 2).mean())

    assert abs(psnr(True) - psnr(False)) < 0.5
