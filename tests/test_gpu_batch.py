"""Batched multi-stream coding through cvc_batch_step: one graph-replayed
launch sequence covers every stream of the batch, and each stream's
bitstream, reconstruction and coder state must be bit-identical to a plain
cvc_codec of the same parameters fed the same frames.

The mixed workload is the streaming one: 16 streams each of QCIF, CIF, VGA
and 720p with 3/3/4/5 pyramid levels, key frame every 10, step 8.  Stream j
of a resolution class starts j frames into that class's synthetic sequence,
so every stream sees different content.
"""
import pytest
import torch

from paper_1510_00561_b300 import Batch, Codec, CvcError
from paper_1510_00561_b300 import synthetic as S

pytestmark = pytest.mark.gpu

CLASSES = [dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2]),
           dict(width=352, height=288, levels=3, dirs_log2=[3, 2, 2]),
           dict(width=640, height=480, levels=4, dirs_log2=[4, 3, 3, 2]),
           dict(width=1280, height=720, levels=5, dirs_log2=[5, 4, 4, 3, 3])]
COMMON = dict(qph=8, qpl=1, key_interval=10)

_cache = {}


def _streams(per_class):
    return [dict(c, **COMMON) for c in CLASSES for _ in range(per_class)]


def _class_frames(ci, n):
    key = (ci, n)
    if key not in _cache:
        c = CLASSES[ci]
        v = S.SyntheticVideo(S.spec_for(c["width"], c["height"], seed=40 + ci))
        _cache[key] = [torch.from_numpy(f).cuda() for f in v.frames(n)]
    return _cache[key]


def _inputs(per_class, T):
    out = []
    for ci in range(len(CLASSES)):
        fr = _class_frames(ci, T + per_class)
        for j in range(per_class):
            out.append(fr[j:j + T])
    return out


def _rgb_buffers(streams, fill=0):
    return [torch.full((s["height"], s["width"], 3), fill, dtype=torch.uint8, device="cuda") for s in streams]


def test_mixed_batch_is_bit_identical_to_plain_codecs():
    """The whole mixed workload: 64 streams x 30 frames (three K-frame periods)."""
    per, T = 16, 30
    streams = _streams(per)
    frames = _inputs(per, T)
    b = Batch(streams)
    plain = [Codec(**s) for s in streams]
    outs = _rgb_buffers(streams)
    for t in range(T):
        res = b.step(3, rgb=[f[t] for f in frames], rgb_out=outs)
        for i, c in enumerate(plain):
            r = res[i]
            ref, ft = c.encode(frames[i][t])
            assert r["enc_status"] == 0 and r["dec_status"] == 0
            assert r["frame_type"] == ft == (0 if t % 10 == 0 else 1)
            assert r["dec_frame_type"] == ft and r["dec_frame_index"] == t
            assert torch.equal(r["bytes"], ref), "stream %d frame %d: bitstream differs" % (i, t)
            rgb = c.decode(ref.clone())
            assert torch.equal(outs[i], rgb), "stream %d frame %d: reconstruction differs" % (i, t)


def test_encode_and_decode_steps_with_idle_streams():
    per, T = 2, 7
    streams = _streams(per)
    n = len(streams)
    frames = _inputs(per, T)
    b = Batch(streams)
    enc_plain = [Codec(**s) for s in streams]
    dec_plain = [Codec(**s) for s in streams]
    outs = _rgb_buffers(streams)

    def active(i, t):
        return (i + t) % 3 != 0

    for t in range(T):
        rgb = [frames[i][t] if active(i, t) else None for i in range(n)]
        res = b.step(1, rgb=rgb)
        ins = []
        for i in range(n):
            if not active(i, t):
                assert res[i]["frame_type"] == -1 and res[i]["out_len"] == 0
                ins.append(None)
                continue
            ref, ft = enc_plain[i].encode(frames[i][t])
            assert res[i]["frame_type"] == ft
            assert torch.equal(res[i]["bytes"], ref)
            ins.append(ref.clone())
        res = b.step(2, streams_in=ins, rgb_out=[outs[i] if ins[i] is not None else None for i in range(n)])
        for i in range(n):
            if ins[i] is None:
                assert res[i]["dec_frame_type"] == -1
                continue
            assert res[i]["dec_status"] == 0
            assert torch.equal(outs[i], dec_plain[i].decode(ins[i]))


def test_launch_shapes_fusion_depths_and_graph_replay_change_nothing():
    """Launch shapes, graph replay, the pyramid tail's fusion depth (0: every level its own
    launches, the default; 1, 2: tails of at most that many levels; 6: as many levels as fit)
    and the row-split DFB block width (0: by launch size; 128; 256) give bit-identical
    bitstreams and reconstructions: every variant runs the same tile computations."""
    streams = _streams(1)
    frames = _inputs(1, 3)
    ref = None
    for graphs, rows, tok, fuse, bt in [(True, 8, 1184, 0, 0), (False, 8, 1184, 0, 0), (True, 1, 1, 0, 0),
                                        (True, 32, 65535, 0, 0), (True, 3, 7, 0, 0), (True, 8, 1184, 6, 0),
                                        (False, 8, 1184, 6, 0), (True, 8, 1184, 1, 0), (True, 8, 1184, 2, 0),
                                        (True, 8, 1184, 0, 128), (True, 8, 1184, 0, 256), (False, 8, 1184, 2, 256)]:
        b = Batch(streams)
        b.set_graphs(graphs)
        b.set_shape(rows, tok)
        b.set_fusion(fuse)
        b.set_dfb_threads(bt)
        outs = _rgb_buffers(streams)
        got = []
        for t in range(3):
            res = b.step(3, rgb=[f[t] for f in frames], rgb_out=outs)
            got.append([r["bytes"].clone() for r in res] + [o.clone() for o in outs])
        if ref is None:
            ref = got
            continue
        for a, c in zip(ref, got):
            for x, y in zip(a, c):
                assert torch.equal(x, y), (graphs, rows, tok, fuse, bt)
    # block widths other than 0, 128 and 256 are refused
    for bad in (-1, 64, 192, 512):
        with pytest.raises(CvcError):
            b.set_dfb_threads(bad)


def test_autotune_keeps_state_and_output():
    streams = _streams(1)
    frames = _inputs(1, 3)
    b = Batch(streams)
    plain = [Codec(**s) for s in streams]
    outs = _rgb_buffers(streams)
    rows, tok, fuse, bt = b.autotune(3, rgb=[f[0] for f in frames], rgb_out=outs, reps=2)
    assert 1 <= rows <= 32 and 1 <= tok <= 65535 and fuse in (0, 1, 2, 6) and bt in (0, 128, 256)
    for t in range(3):
        res = b.step(3, rgb=[f[t] for f in frames], rgb_out=outs)
        for i, c in enumerate(plain):
            ref, ft = c.encode(frames[i][t])
            assert res[i]["frame_type"] == ft == (0 if t == 0 else 1)
            assert torch.equal(res[i]["bytes"], ref)
            assert torch.equal(outs[i], c.decode(ref.clone()))


def test_per_stream_errors_stay_with_their_stream():
    streams = _streams(1)
    n = len(streams)
    frames = _inputs(1, 2)
    b = Batch(streams)
    plain = [Codec(**s) for s in streams]
    # a too-small output buffer fails only stream 1, whose state stays unchanged
    tiny = torch.empty(64, dtype=torch.uint8, device="cuda")
    outs = [None] * n
    outs[1] = tiny
    res = b.step(1, rgb=[f[0] for f in frames], outs=outs, check=False)
    assert res[1]["enc_status"] == 3 and res[1]["out_len"] > 64
    assert all(res[i]["enc_status"] == 0 for i in range(n) if i != 1)
    s0 = [res[i]["bytes"].clone() if i != 1 else None for i in range(n)]
    refs0 = [c.encode(frames[i][0])[0] for i, c in enumerate(plain)]
    res = b.step(1, rgb=[frames[i][1] if i != 1 else frames[i][0] for i in range(n)])
    assert res[1]["frame_type"] == 0 and torch.equal(res[1]["bytes"], refs0[1])
    s0[1] = res[1]["bytes"].clone()
    for i in range(n):
        if i != 1:
            assert res[i]["frame_type"] == 1
    # decoding: a corrupt stream and a P-frame without its reference fail alone
    d = Batch(streams)
    bad = s0[2].clone()
    bad[0] = ord("X")
    ins = list(s0)
    ins[2] = bad
    ins[3] = res[3]["bytes"].clone()       # a P-frame first
    outs_rgb = _rgb_buffers(streams, fill=77)
    r = d.step(2, streams_in=ins, rgb_out=outs_rgb, check=False)
    assert r[2]["dec_status"] == 5 and r[3]["dec_status"] == 9
    assert r[0]["dec_status"] == 0 and r[1]["dec_status"] == 0
    assert bool((outs_rgb[2] == 77).all()) and bool((outs_rgb[3] == 77).all())
    ref_dec = Codec(**streams[0])
    assert torch.equal(outs_rgb[0], ref_dec.decode(s0[0]))
    with pytest.raises(CvcError) as e:
        d.step(2, streams_in=ins, rgb_out=outs_rgb)
    assert e.value.status in (5, 9)


def test_invalid_calls_do_nothing():
    streams = _streams(1)
    b = Batch(streams)
    frames = _inputs(1, 1)
    rgb = [f[0] for f in frames]
    rgb[2] = torch.zeros((480, 100, 3), dtype=torch.uint8, device="cuda")   # rows shorter than the frame's
    with pytest.raises(CvcError) as e:
        b.step(1, rgb=rgb)
    assert e.value.status == 1
    with pytest.raises(CvcError) as e:
        b.step(0, rgb=[f[0] for f in frames])
    assert e.value.status == 1
    res = b.step(1, rgb=[f[0] for f in frames])
    assert all(r["frame_type"] == 0 for r in res)


def test_device_bytes_estimate_matches_allocation():
    streams = _streams(2)
    est = Batch.device_bytes(streams)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    b = Batch(streams)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    assert b.n == len(streams)
    slack = 64 << 20
    assert est - slack <= used <= est + est // 20 + slack, (est, used)


def test_1080p_batch_matches_plain():
    """The benchmark's configuration: concurrent 1080p streams, 5 levels, 32/16/16/8/8."""
    cfg = dict(width=1920, height=1080, levels=5, dirs_log2=[5, 4, 4, 3, 3], qph=8, qpl=1, key_interval=10)
    v = S.SyntheticVideo(S.spec_for(1920, 1080, seed=7))
    frames = [torch.from_numpy(f).cuda() for f in v.frames(6)]
    b = Batch([cfg] * 4)
    plain = [Codec(**cfg) for _ in range(4)]
    outs = _rgb_buffers([cfg] * 4)
    for t in range(3):
        inp = [frames[t + j] for j in range(4)]          # stream j is the sequence shifted by j frames
        res = b.step(3, rgb=inp, rgb_out=outs)
        for j, c in enumerate(plain):
            ref, ft = c.encode(inp[j])
            assert res[j]["frame_type"] == ft and torch.equal(res[j]["bytes"], ref)
            assert torch.equal(outs[j], c.decode(ref.clone()))
