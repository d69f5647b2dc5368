"""cvc_stream_drop_levels (host code of the library, no GPU): the frame
without its finest levels (§3.3: a receiver's resolution is served by
dropping what refers to higher resolutions, without re-encoding) must be
byte-identical to the oracle's on the oracle's own streams, work in place,
and refuse what it cannot do."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1510_00561_b300 import _lib as L
from paper_1510_00561_b300 import synthetic as S

CASES = [(176, 144, 3, [3, 2, 2]), (99, 77, 2, [2, 0]), (64, 48, 2, [1, 0]), (640, 480, 4, [4, 3, 3, 2])]


def _drop(prm, src, drop, cap=None, inplace=False):
    src = np.ascontiguousarray(src, dtype=np.uint8).copy()
    out = src if inplace else np.zeros(cap if cap is not None else max(1, src.size), np.uint8)
    n = ctypes.c_size_t(0)
    st = L.lib().cvc_stream_drop_levels(ctypes.byref(prm), src.ctypes.data, src.size, drop, out.ctypes.data,
                                        out.size, ctypes.byref(n))
    return st, out[:n.value].copy(), n.value


@pytest.mark.parametrize("w,h,Lv,k", CASES)
def test_drop_matches_the_oracle(w, h, Lv, k):
    prm = L.params(w, h, Lv, k, 8, 1, 0.0, 3)
    enc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 3)
    for f in S.SyntheticVideo(S.spec_for(w, h, seed=7)).frames(2):      # a K- and a P-frame
        s, _ = enc.encode(f)
        for d in range(Lv + 1):
            ref = enc.drop_levels(s, d)
            st, got, _ = _drop(prm, s, d)
            assert st == 0 and np.array_equal(got, ref), d
            st, got2, _ = _drop(prm, s, d, inplace=True)
            assert st == 0 and np.array_equal(got2, ref), d
            # dropping more from a dropped frame equals dropping it all at once
            for d2 in range(d, Lv + 1):
                st, got3, _ = _drop(prm, ref, d2)
                assert st == 0 and np.array_equal(got3, enc.drop_levels(s, d2))


def test_drop_refusals():
    w, h, Lv, k = 99, 77, 2, [2, 2]
    prm = L.params(w, h, Lv, k, 8, 1, 0.0, 3)
    enc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 3)
    s, _ = enc.encode(S.SyntheticVideo(S.spec_for(w, h, seed=8)).frame(0))
    d1 = enc.drop_levels(s, 1)
    assert _drop(prm, d1, 0)[0] == 1          # cannot put levels back
    assert _drop(prm, s, 3)[0] == 1           # beyond the pyramid
    st, _, need = _drop(prm, s, 1, cap=10)
    assert st == 3 and need == d1.size        # capacity: the size needed comes back
    bad = s.copy()
    bad[0] = ord("X")
    assert _drop(prm, bad, 1)[0] == 5
    assert _drop(prm, s[:40], 1)[0] == 5      # truncated count table
    other = L.params(w, h, 2, [2, 1], 8, 1, 0.0, 3)
    assert _drop(other, s, 1)[0] == 5         # another decomposition: component count differs


def test_drop_keeps_the_motion_vectors():
    w, h, Lv, k = 176, 144, 3, [3, 2, 2]
    prm = L.params(w, h, Lv, k, 8, 1, 0.0, 4, motion_range=8)
    enc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 4, motion_range=8)
    frames = S.SyntheticVideo(S.spec_for(w, h, seed=9)).frames(2)
    enc.encode(frames[0])
    s, t = enc.encode(frames[1])
    assert t == 2
    for d in range(Lv + 1):
        st, got, _ = _drop(prm, s, d)
        assert st == 0 and np.array_equal(got, enc.drop_levels(s, d))
        assert np.array_equal(got[-2 * 99:], s[-2 * 99:])     # 9 x 11 blocks of (dy, dx)
    # the vectors of a frame are no use to a stream without motion
    assert _drop(L.params(w, h, Lv, k, 8, 1, 0.0, 4), s, 1)[0] == 5


def _deflate_like_the_container(frame, ncomp):
    """a deflated frame of the container layout with zlib streams (the dropper only moves bytes)"""
    import zlib
    hdr = 32 + 4 * ncomp
    counts = np.frombuffer(bytes(frame[32:hdr]), "<u4")
    streams, segs, pos = [], [], hdr
    for n in counts:
        tok = bytes(frame[pos:pos + 2 * int(n)])
        pos += 2 * int(n)
        streams.append(zlib.compress(tok, 6)[2:-4] if n else b"")
        segs += [(len(tok[k:k + 256]) * 7) & 0xFFFF for k in range(0, len(tok), 256)]
    head = bytearray(frame[:hdr])
    head[4] = 2
    seg = np.array(segs, "<u2").tobytes()
    seg += bytes(((len(seg) + 3) // 4) * 4 - len(seg))
    lens = np.array([len(x) for x in streams], "<u4").tobytes()
    return np.frombuffer(bytes(head) + lens + seg + b"".join(streams) + bytes(frame[pos:]), np.uint8)


@pytest.mark.parametrize("motion", [0, 8])
def test_drop_of_deflated_frames_equals_deflating_the_dropped_frame(motion):
    w, h, Lv, k = 176, 144, 3, [3, 2, 2]
    prm = L.params(w, h, Lv, k, 8, 1, 0.0, 4, motion_range=motion)
    enc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 4, motion_range=motion)
    for f in S.SyntheticVideo(S.spec_for(w, h, seed=10)).frames(2):
        s, _ = enc.encode(f)
        box = _deflate_like_the_container(s, enc.ncomp)
        for d in range(Lv + 1):
            st, got, _ = _drop(prm, box, d)
            assert st == 0
            assert np.array_equal(got, _deflate_like_the_container(enc.drop_levels(s, d), enc.ncomp)), d
            st, got2, _ = _drop(prm, box, d, inplace=True)
            assert st == 0 and np.array_equal(got2, got)
            # and the oracle inflates what remains to the dropped frame
            assert np.array_equal(enc.inflate_container(got), enc.drop_levels(s, d))


def test_cvc_nts_frames_cannot_lose_levels():
    """§3.9: a CVC-NTS frame is one DEFLATE stream, so transmission scalability is gone"""
    w, h, Lv, k = 176, 144, 3, [3, 2, 2]
    prm = L.params(w, h, Lv, k, 8, 1, 0.0, 4)
    enc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 4)
    s, _ = enc.encode(S.SyntheticVideo(S.spec_for(w, h, seed=11)).frame(0))
    box = _deflate_like_the_container(s, enc.ncomp).copy()
    box[4] = 3
    assert _drop(prm, box, 1)[0] == 2


def test_drop_of_8bit_storage_frames():
    """header byte 5 (the 8-bit storage of §3.6) passes through the dropper"""
    w, h, Lv, k = 176, 144, 3, [3, 2, 2]
    prm = L.params(w, h, Lv, k, 8, 1, 0.0, 3, storage8=True)
    enc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 3, storage8=True)
    for f in S.SyntheticVideo(S.spec_for(w, h, seed=12)).frames(2):
        s, _ = enc.encode(f)
        for d in range(Lv + 1):
            st, got, _ = _drop(prm, s, d)
            assert st == 0 and got[5] == 1 and np.array_equal(got, enc.drop_levels(s, d))
