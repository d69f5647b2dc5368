"""The DEFLATE stage on the GPU (§3.9, scalable and CVC-NTS modes),
cvc_deflate_frame / cvc_inflate_frame.

What is unique is checked exactly, the rest for validity:
  - every component stream is a raw DEFLATE stream that zlib inflates to
    exactly that component's token bytes (an independent inflater);
  - the oracle's zlib-based container inflater rebuilds the exact frame;
  - the GPU inflate rebuilds the exact frame (and the codec decodes it);
  - each stream's code is an optimal prefix code of its bytes plus the
    end-of-block code (cost equal to the oracle's Huffman cost) whenever that
    optimum needs no code longer than 15 bits, and within 1% of it otherwise;
  - corrupt containers and short buffers are refused;
  - CVC-NTS: the frame's token bytes are one such stream (version byte 3),
    and the same checks hold for it.
"""
import zlib

import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import Codec, CvcError, Deflater
from paper_1510_00561_b300 import synthetic as S

pytestmark = pytest.mark.gpu

QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4)
VGA = dict(width=640, height=480, levels=4, dirs_log2=[4, 3, 3, 2], qph=4, qpl=1, key_interval=10, motion_range=8)
HD = dict(width=1920, height=1080, levels=5, dirs_log2=[5, 4, 4, 3, 3], qph=8, qpl=1, key_interval=10)


def _codec(kw):
    return Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"], 0.0,
                 kw["key_interval"], kw.get("motion_range", 0))


def _oracle(kw):
    return O.Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"], 0.0,
                   kw["key_interval"], kw.get("motion_range", 0))


def _parts(frame, packed, ncomp):
    """per component: (token bytes, stream bytes, segment bit lengths)"""
    hdr = 32 + 4 * ncomp
    counts = np.frombuffer(bytes(frame[32:hdr]), "<u4").astype(np.int64)
    lens = np.frombuffer(bytes(packed[hdr:hdr + 4 * ncomp]), "<u4").astype(np.int64)
    nseg = [(2 * n + 255) // 256 for n in counts]
    segs = np.frombuffer(bytes(packed[hdr + 4 * ncomp:hdr + 4 * ncomp + 2 * sum(nseg)]), "<u2").astype(np.int64)
    pos = hdr + 4 * ncomp + ((2 * sum(nseg) + 3) // 4) * 4
    tp, sp, out = hdr, 0, []
    for n, nb, k in zip(counts, lens, nseg):
        out.append((bytes(frame[tp:tp + 2 * n]), bytes(packed[pos:pos + nb]), segs[sp:sp + k]))
        tp += 2 * n
        pos += nb
        sp += k
    return out


def _check(kw, frame_dev, dfl, oc):
    frame = frame_dev.cpu().numpy()
    packed = dfl.deflate(frame_dev).clone()
    pk = packed.cpu().numpy()
    assert pk[4] == 2 and np.array_equal(pk[:4], frame[:4]) and np.array_equal(pk[5:32 + 4 * oc.ncomp],
                                                                                  frame[5:32 + 4 * oc.ncomp])
    total_tok = total_stream = 0
    for tok, stream, segs in _parts(frame, pk, oc.ncomp):
        if not tok:
            assert not stream and segs.size == 0
            continue
        assert zlib.decompress(stream, wbits=-15) == tok
        hist = np.bincount(np.frombuffer(tok, np.uint8), minlength=256).astype(np.uint64)
        cost, depth = O.huffman_cost(np.append(hist, 1))
        lit_bits = int(segs.sum())
        # the literals take lit_bits, the end-of-block code 1..15 more
        if depth <= 15:
            assert cost - 15 <= lit_bits <= cost - 1, (cost, lit_bits)
        else:
            assert lit_bits <= 1.01 * cost
        total_tok += len(tok)
        total_stream += len(stream)
    assert np.array_equal(oc.inflate_container(pk), frame)
    back = dfl.inflate(packed)
    assert torch.equal(back, frame_dev)
    return total_tok, total_stream, packed.numel()


@pytest.mark.parametrize("kw,n", [(QCIF, 5), (VGA, 3), (HD, 2)], ids=["qcif", "vga_motion", "1080p"])
def test_deflate_round_trip(kw, n):
    g = _codec(kw)
    dfl = Deflater(**kw)
    oc = _oracle(kw)
    frames = S.SyntheticVideo(S.spec_for(kw["width"], kw["height"], seed=70)).frames(n)
    ratios = []
    for f in frames:
        s, _ = g.encode(torch.from_numpy(f).cuda())
        s = s.clone()
        tok, stream, packed = _check(kw, s, dfl, oc)
        ratios.append(stream / tok)
    assert max(ratios) < 0.6


def test_inflated_frames_decode_like_the_originals():
    kw = QCIF
    g, d1, d2 = _codec(kw), _codec(kw), _codec(kw)
    dfl = Deflater(**kw)
    for f in S.SyntheticVideo(S.spec_for(176, 144, seed=71)).frames(4):
        s, _ = g.encode(torch.from_numpy(f).cuda())
        s = s.clone()
        back = dfl.inflate(dfl.deflate(s).clone()).clone()
        assert torch.equal(back, s)
        assert torch.equal(d1.decode(s.clone()), d2.decode(back))


def test_deflate_of_dropped_levels_and_sizes_against_zlib():
    kw = QCIF
    g = _codec(kw)
    dfl = Deflater(**kw)
    oc = _oracle(kw)
    frames = S.SyntheticVideo(S.spec_for(176, 144, seed=72)).frames(2)
    for f in frames:
        s, _ = g.encode(torch.from_numpy(f).cuda())
        for dlev in (1, 3):
            x = torch.from_numpy(g.drop_levels(s.cpu(), dlev)).cuda()
            _check(kw, x, dfl, oc)
        # the Huffman-only streams are as small as zlib's Huffman-only streams of the same bytes
        frame = s.cpu().numpy()
        packed = dfl.deflate(s.clone()).cpu().numpy()
        for tok, stream, _ in _parts(frame, packed, oc.ncomp):
            if len(tok) < 64:
                continue
            z = zlib.compressobj(9, zlib.DEFLATED, -15, 9, zlib.Z_HUFFMAN_ONLY)
            ref = len(z.compress(tok) + z.flush())
            assert len(stream) <= ref * 1.02 + 8, (len(stream), ref)


def test_corrupt_and_short_buffers_are_refused():
    kw = QCIF
    g = _codec(kw)
    dfl = Deflater(**kw)
    f = S.SyntheticVideo(S.spec_for(176, 144, seed=73)).frame(0)
    s, _ = g.encode(torch.from_numpy(f).cuda())
    s = s.clone()
    packed = dfl.deflate(s).clone()
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(CvcError) as e:
        dfl.deflate(s, out=small)
    assert e.value.status == 3
    with pytest.raises(CvcError) as e:
        dfl.inflate(packed, out=small)
    assert e.value.status == 3
    bad = packed.clone()
    bad[4] = 1                                        # not a deflated frame
    with pytest.raises(CvcError) as e:
        dfl.inflate(bad)
    assert e.value.status == 5
    ncomp = _oracle(kw).ncomp
    first = int(np.frombuffer(bytes(packed[32 + 4 * ncomp:36 + 4 * ncomp].cpu().numpy()), "<u4")[0])
    assert first > 0
    bad = packed.clone()
    counts = np.frombuffer(bytes(packed[32:32 + 4 * ncomp].cpu().numpy()), "<u4")
    nseg = sum((2 * int(n) + 255) // 256 for n in counts)
    start = 32 + 8 * ncomp + ((2 * nseg + 3) // 4) * 4
    bad[start] ^= 0x06                                # BTYPE of the first stream: no longer dynamic
    with pytest.raises(CvcError) as e:
        dfl.inflate(bad)
    assert e.value.status == 5
    with pytest.raises(CvcError) as e:
        dfl.inflate(packed[:-5].clone())
    assert e.value.status == 5
    with pytest.raises(CvcError) as e:
        dfl.deflate(packed)                           # already deflated
    assert e.value.status == 5


def test_dropping_levels_of_deflated_frames():
    """§3.3 + §3.9: a deflated frame loses whole component streams; that equals
    deflating the frame without those levels, and decodes at the coarser scales."""
    kw = dict(QCIF, motion_range=8)
    g = _codec(kw)
    dfl = Deflater(**kw)
    frames = S.SyntheticVideo(S.spec_for(176, 144, seed=74)).frames(3)
    streams = [g.encode(torch.from_numpy(f).cuda())[0].clone() for f in frames]
    for d in range(kw["levels"] + 1):
        full, part = _codec(kw), _codec(kw)
        for s in streams:
            packed = dfl.deflate(s).clone()
            thin = g.drop_levels(packed.cpu(), d)
            ref = dfl.deflate(torch.from_numpy(g.drop_levels(s.cpu(), d)).cuda()).cpu().numpy()
            assert np.array_equal(thin, ref)
            back = dfl.inflate(torch.from_numpy(thin).cuda()).clone()
            assert torch.equal(part.decode(back, scale=d), full.decode(s.clone(), scale=d))


def test_batched_calls_equal_single_frame_calls():
    """cvc_deflate_frames / cvc_inflate_frames over 8 frames (a K-frame period with
    dropped levels mixed in) give exactly the single-frame results."""
    kw = dict(QCIF, key_interval=3, motion_range=8)
    g = _codec(kw)
    one = Deflater(**kw)
    many = Deflater(max_frames=8, **kw)
    frames = S.SyntheticVideo(S.spec_for(176, 144, seed=75)).frames(8)
    streams = [g.encode(torch.from_numpy(f).cuda())[0].clone() for f in frames]
    streams[3] = torch.from_numpy(g.drop_levels(streams[3].cpu(), 2)).cuda()
    outs = [torch.zeros(s.numel() + 65536, dtype=torch.uint8, device="cuda") for s in streams]
    packed, sts = many.deflate_many(streams, outs)
    assert sts == [0] * 8
    for s, p in zip(streams, packed):
        assert torch.equal(p, one.deflate(s))
    backs = [torch.zeros(s.numel() + 16, dtype=torch.uint8, device="cuda") for s in streams]
    back, sts = many.inflate_many([p.clone() for p in packed], backs)
    assert sts == [0] * 8
    for s, b in zip(streams, back):
        assert torch.equal(b, s)
    # a short buffer fails its own frame only
    outs[5] = torch.zeros(64, dtype=torch.uint8, device="cuda")
    packed, sts = many.deflate_many(streams, outs)
    assert sts[5] == 3 and all(v == 0 for i, v in enumerate(sts) if i != 5)
    assert torch.equal(packed[4], one.deflate(streams[4]))


def _check_nts(frame_dev, dfl, oc):
    frame = frame_dev.cpu().numpy()
    packed = dfl.deflate(frame_dev).clone()
    pk = packed.cpu().numpy()
    hdr = 32 + 4 * oc.ncomp
    assert pk[4] == 3 and np.array_equal(pk[:4], frame[:4]) and np.array_equal(pk[5:hdr], frame[5:hdr])
    counts = np.frombuffer(bytes(frame[32:hdr]), "<u4").astype(np.int64)
    tok = bytes(frame[hdr:hdr + 2 * int(counts.sum())])
    nb = int(np.frombuffer(bytes(pk[hdr:hdr + 4]), "<u4")[0])
    nseg = (len(tok) + 255) // 256
    segs = np.frombuffer(bytes(pk[hdr + 4:hdr + 4 + 2 * nseg]), "<u2").astype(np.int64)
    pos = hdr + 4 + ((2 * nseg + 3) // 4) * 4
    stream = bytes(pk[pos:pos + nb])
    assert zlib.decompress(stream, wbits=-15) == tok
    # segment k covers token bytes [256 k, 256 k + 256) of the frame
    hist = np.bincount(np.frombuffer(tok, np.uint8), minlength=256).astype(np.uint64)
    cost, depth = O.huffman_cost(np.append(hist, 1))
    if depth <= 15:
        assert cost - 15 <= int(segs.sum()) <= cost - 1
    else:
        assert int(segs.sum()) <= 1.01 * cost
    assert np.array_equal(pk[pos + nb:], frame[hdr + len(tok):])     # the motion vectors
    assert np.array_equal(oc.inflate_container(pk), frame)
    assert torch.equal(dfl.inflate(packed), frame_dev)
    return packed


@pytest.mark.parametrize("kw,n", [(QCIF, 5), (VGA, 3), (HD, 2)], ids=["qcif", "vga_motion", "1080p"])
def test_cvc_nts_round_trip(kw, n):
    """§3.9 CVC-NTS: one stream over all the components of a frame; a frame of
    1080p spans many segment groups"""
    g = _codec(kw)
    nts, sc = Deflater(nts=True, **kw), Deflater(**kw)
    oc = _oracle(kw)
    dec_a, dec_b = _codec(kw), _codec(kw)
    for f in S.SyntheticVideo(S.spec_for(kw["width"], kw["height"], seed=76)).frames(n):
        s, _ = g.encode(torch.from_numpy(f).cuda())
        s = s.clone()
        packed = _check_nts(s, nts, oc)
        # the scalable inflater reads both forms
        back = sc.inflate(packed).clone()
        assert torch.equal(back, s)
        # decoding at every scale is unaffected (scalability at the decoder stays)
        assert torch.equal(dec_a.decode(back), dec_b.decode(s.clone()))


def test_cvc_nts_refusals_and_batches():
    kw = dict(QCIF, key_interval=3, motion_range=8)
    g = _codec(kw)
    frames = S.SyntheticVideo(S.spec_for(176, 144, seed=77)).frames(6)
    streams = [g.encode(torch.from_numpy(f).cuda())[0].clone() for f in frames]
    one, many = Deflater(nts=True, **kw), Deflater(max_frames=6, nts=True, **kw)
    scal = Deflater(max_frames=6, **kw)
    outs = [torch.zeros(s.numel() + 65536, dtype=torch.uint8, device="cuda") for s in streams]
    packed, sts = many.deflate_many(streams, outs)
    assert sts == [0] * 6
    for s, p in zip(streams, packed):
        assert torch.equal(p, one.deflate(s))
    # an inflate call mixing both container forms
    mixed = [p.clone() if i % 2 else scal.deflate(streams[i]).clone() for i, p in enumerate(packed)]
    backs = [torch.zeros(s.numel() + 16, dtype=torch.uint8, device="cuda") for s in streams]
    back, sts = many.inflate_many(mixed, backs)
    assert sts == [0] * 6
    for s, b in zip(streams, back):
        assert torch.equal(b, s)
    p = packed[0].clone()
    with pytest.raises(CvcError) as e:
        g.drop_levels(p.cpu(), 1)                     # one stream: nothing to drop in transit
    assert e.value.status == 2
    bad = p.clone()
    bad[4] = 2                                        # read as a per-component container
    with pytest.raises(CvcError) as e:
        one.inflate(bad)
    assert e.value.status == 5
    with pytest.raises(CvcError) as e:
        one.inflate(p[:-3].clone())
    assert e.value.status == 5
