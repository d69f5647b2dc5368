"""Pins of the oracle's scaled decode (§3.3: every LP scale of a stream can be
decoded on its own).  Scale s reconstructs the level-s approximation from
the lowpass and levels s+1..L, normalised by 2^-s, at ceil(H/2^s) x
ceil(W/2^s).  Checked against things other than the decode path itself:

  - a constant frame decodes to the same constant at every scale;
  - with unit quantisation steps the scale-s planes equal the level-s lowpass
    of the encoder's own planes, computed directly by the oracle's forward
    pyramid, within the quantisation error;
  - output sizes for odd frames, and scale 0 equal to the plain decode;
  - decoding some frames at a coarse scale keeps the decoder state of every
    component, so a later full-resolution decode is unchanged.
"""
import numpy as np
import pytest

import oracle as O
from paper_1510_00561_b300 import synthetic as S


def _codec(w, h, L, k, qph=8, qpl=1, kint=8):
    return O.Codec(w, h, L, k, qph, qpl, 0.0, kint)


@pytest.mark.parametrize("w,h,L,k", [(176, 144, 3, [3, 2, 2]), (99, 77, 2, [2, 2])])
def test_constant_frame_at_every_scale(w, h, L, k):
    frame = np.empty((h, w, 3), np.uint8)
    frame[..., 0], frame[..., 1], frame[..., 2] = 120, 64, 200
    enc = _codec(w, h, L, k)
    s, _ = enc.encode(frame)
    full = _codec(w, h, L, k).decode(s)
    for sc in range(L + 1):
        dec = _codec(w, h, L, k)
        rgb = dec.decode(s, scale=sc)
        f = 1 << sc
        assert rgb.shape == ((h + f - 1) // f, (w + f - 1) // f, 3)
        assert np.array_equal(rgb, np.broadcast_to(full[0, 0], rgb.shape)), sc


def _lowpass(plane, s):
    for _ in range(s):
        plane, _ = O.lp_analysis(plane)
    return plane * 2.0 ** -s


@pytest.mark.parametrize("sc", [1, 2, 3])
def test_scaled_planes_are_the_pyramid_lowpass(sc):
    w, h, L, k = 176, 144, 3, [3, 2, 2]
    frame = S.SyntheticVideo(S.spec_for(w, h, seed=3)).frame(0)
    enc = _codec(w, h, L, k, qph=1, qpl=1)
    s, _ = enc.encode(frame)
    yp, cop, cgp = enc.planes(frame)
    _, planes = _codec(w, h, L, k, qph=1, qpl=1).decode(s, want_planes=True, scale=sc)
    for got, src in zip(planes, (yp, cop, cgp)):
        ref = _lowpass(src, sc)
        assert got.shape == ref.shape
        err = np.abs(got - ref)
        # unit steps: every coefficient is off by at most 1/2 (the lowpass by 2^L/2 before
        # its 2^-L normalisation); the coarse synthesis spreads that over a few samples
        assert err.max() < 3.0 and err.mean() < 0.5, (sc, err.max(), err.mean())


def test_scale_zero_is_the_plain_decode_and_state_carries_over():
    w, h, L, k = 99, 77, 2, [2, 2]
    frames = S.SyntheticVideo(S.spec_for(w, h, seed=5)).frames(4)
    enc = _codec(w, h, L, k, kint=8)
    streams = [enc.encode(f)[0] for f in frames]
    ref = _codec(w, h, L, k, kint=8)
    mixed = _codec(w, h, L, k, kint=8)
    outs_ref = [ref.decode(s) for s in streams]
    assert np.array_equal(_codec(w, h, L, k).decode(streams[0], scale=0), outs_ref[0])
    # frames 0-2 at coarse scales, frame 3 at full resolution
    mixed.decode(streams[0], scale=2)
    mixed.decode(streams[1], scale=1)
    r2 = mixed.decode(streams[2], scale=1)
    assert r2.shape == (39, 50, 3)
    assert np.array_equal(mixed.decode(streams[3]), outs_ref[3])


def test_invalid_scale_is_refused():
    w, h, L, k = 99, 77, 2, [2, 2]
    frame = S.SyntheticVideo(S.spec_for(w, h, seed=6)).frame(0)
    s, _ = _codec(w, h, L, k).encode(frame)
    with pytest.raises(Exception):
        _codec(w, h, L, k).decode(s, scale=3)
