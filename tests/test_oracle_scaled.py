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


def _sequence(w, h, L, k, n, seed, kint=3):
    frames = S.SyntheticVideo(S.spec_for(w, h, seed=seed)).frames(n)
    enc = _codec(w, h, L, k, kint=kint)
    return [enc.encode(f)[0] for f in frames]


def _dropped_token_bytes(stream, w, h, L, k, drop):
    """bytes of the tokens of components of levels 1..drop (from the count table)"""
    c = _codec(w, h, L, k)
    lays = [O.layout(c.Hp, c.Wp, L, k)] + [O.layout(c.Hcp, c.Wcp, L, k)] * 2
    counts = np.frombuffer(bytes(stream[32:32 + 4 * c.ncomp]), "<u4")
    j = n = 0
    for lay in lays:
        for sb in lay["subbands"]:
            if sb["kind"] != 0 and sb["level"] <= drop:
                n += 2 * int(counts[j])
            j += 1
    return n


@pytest.mark.parametrize("w,h,L,k", [(176, 144, 3, [3, 2, 2]), (99, 77, 2, [2, 0])])
def test_dropping_fine_levels_leaves_every_coarser_scale_unchanged(w, h, L, k):
    """§3.3: a receiver at scale s can be sent the stream without levels 1..s.
    Decoding a K/P sequence with levels 1..d dropped gives, at every scale
    s >= d, exactly the frames of the complete sequence at that scale; the
    dropped stream is shorter by exactly the dropped components' tokens."""
    seq = _sequence(w, h, L, k, 5, seed=11)
    for d in range(L + 1):
        dropped = [_codec(w, h, L, k).drop_levels(s, d) for s in seq]
        for s, t in zip(seq, dropped):
            assert t.size == s.size - _dropped_token_bytes(s, w, h, L, k, d)
            assert t[26] | (t[27] << 8) == d
            if d == 0:
                assert np.array_equal(s, t)
        for sc in range(d, L + 1):
            full, part = _codec(w, h, L, k), _codec(w, h, L, k)
            for s, t in zip(seq, dropped):
                assert np.array_equal(full.decode(s, scale=sc), part.decode(t, scale=sc)), (d, sc)


def test_dropped_levels_bound_the_decodable_scales():
    w, h, L, k = 176, 144, 3, [3, 2, 2]
    seq = _sequence(w, h, L, k, 5, seed=12)          # K P P K P
    c = _codec(w, h, L, k)
    d2 = [c.drop_levels(s, 2) for s in seq]
    dec = _codec(w, h, L, k)
    with pytest.raises(RuntimeError, match="status 9"):
        dec.decode(d2[0], scale=1)                   # the stream lacks level 2
    dec.decode(d2[0], scale=2)                       # K-frame without levels 1-2
    with pytest.raises(RuntimeError, match="status 9"):
        dec.decode(seq[1], scale=0)                  # complete P-frame, but no state for levels 1-2
    dec.decode(seq[1], scale=2)
    dec.decode(seq[2], scale=3)
    ref = _codec(w, h, L, k)
    for s in seq:
        r = ref.decode(s)
    # a complete K-frame restores every level: full-scale decoding resumes
    assert np.array_equal(dec.decode(seq[3]), _codec(w, h, L, k).decode(seq[3]))
    assert np.array_equal(dec.decode(seq[4]), r)


def test_stream_drop_only_removes():
    w, h, L, k = 99, 77, 2, [2, 2]
    s = _sequence(w, h, L, k, 1, seed=13)[0]
    c = _codec(w, h, L, k)
    d1 = c.drop_levels(s, 1)
    assert np.array_equal(c.drop_levels(d1, 2), c.drop_levels(s, 2))
    assert np.array_equal(c.drop_levels(d1, 1), d1)
    with pytest.raises(RuntimeError, match="status 1"):
        c.drop_levels(d1, 0)
    with pytest.raises(RuntimeError, match="status 1"):
        c.drop_levels(s, 3)
    # the lowpass components always stay; everything of level 1 is gone
    counts = np.frombuffer(bytes(d1[32:32 + 4 * c.ncomp]), "<u4")
    lay = O.layout(c.Hp, c.Wp, L, k)
    for j, sb in enumerate(lay["subbands"]):
        assert (counts[j] == 0) == (sb["level"] == 1)
