"""Asynchronous calls (cvc_encode_frame_async, cvc_decode_frame_async,
cvc_batch_step_async, cvc_get_error) through the C ABI.

The coder state lives on the device and advances there, so calls queue back
to back on one stream with one synchronisation at the end, and must give
exactly the bytes, lengths, frame types and pixels of the synchronous calls
made in the same order.  Failures are reported in device memory and in the
codec's device status word, and leave the coder state as it was.
"""
import pytest
import torch

from paper_1510_00561_b300 import Batch, Codec
from paper_1510_00561_b300 import synthetic as S

pytestmark = pytest.mark.gpu

QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=3)
OK, CAPACITY, CORRUPT, STATE = 0, 3, 5, 9


def _codec(kw):
    return Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"], 0.0,
                 kw["key_interval"], motion_range=kw.get("motion_range", 0))


def _frames(kw, n, seed):
    v = S.SyntheticVideo(S.spec_for(kw["width"], kw["height"], seed=seed))
    return [torch.from_numpy(f).cuda() for f in v.frames(n)]


@pytest.mark.parametrize("motion", [0, 8], ids=["zero_motion", "motion"])
def test_eight_queued_encode_decode_pairs_equal_the_synchronous_calls(motion):
    kw = dict(QCIF, motion_range=motion)
    T = 8
    frames = _frames(kw, T, seed=60)
    # synchronous reference
    se, sd = _codec(kw), _codec(kw)
    ref = []
    for f in frames:
        s, ft = se.encode(f)
        s = s.clone()
        ref.append((s, ft, sd.decode(s).clone()))
    # the same calls queued on one stream, one synchronisation at the end
    ae, ad = _codec(kw), _codec(kw)
    outs = [torch.empty(ae.max_stream, dtype=torch.uint8, device="cuda") for _ in range(T)]
    rgbs = [torch.zeros((kw["height"], kw["width"], 3), dtype=torch.uint8, device="cuda") for _ in range(T)]
    lens = torch.full((T,), -1, dtype=torch.int64, device="cuda")
    types = torch.full((T,), -7, dtype=torch.int32, device="cuda")
    est = torch.full((T,), -7, dtype=torch.int32, device="cuda")
    dst = torch.full((T,), -7, dtype=torch.int32, device="cuda")
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        for t in range(T):
            ae.encode_async(frames[t], outs[t], lens[t:t + 1], types[t:t + 1], est[t:t + 1], stream=st)
            ad.decode_async(outs[t], rgbs[t], in_len=lens[t:t + 1], status=dst[t:t + 1], stream=st)
    st.synchronize()
    assert (est == OK).all() and (dst == OK).all()
    for t, (s, ft, rgb) in enumerate(ref):
        n = int(lens[t])
        assert n == s.numel() and int(types[t]) == ft, t
        assert torch.equal(outs[t][:n], s), "frame %d: bitstream differs from the synchronous call" % t
        assert torch.equal(rgbs[t], rgb), "frame %d: reconstruction differs" % t
    assert ae.get_error(st) == OK and ad.get_error(st) == OK
    # the device state advanced exactly as the synchronous codecs' did: the next calls agree too
    f = _frames(kw, T + 1, seed=60)[T]
    s_sync, ft_sync = se.encode(f)
    s_async, ft_async = ae.encode(f)
    assert ft_sync == ft_async and torch.equal(s_sync, s_async)


def test_async_failures_go_to_device_memory_and_leave_the_state():
    kw = QCIF
    f0, f1 = _frames(kw, 2, seed=61)
    enc = _codec(kw)
    big = torch.empty(enc.max_stream, dtype=torch.uint8, device="cuda")
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(2, dtype=torch.int64, device="cuda")
    ty = torch.zeros(2, dtype=torch.int32, device="cuda")
    es = torch.zeros(2, dtype=torch.int32, device="cuda")
    enc.encode_async(f0, small, ln[0:1], ty[0:1], es[0:1])      # too small: CAPACITY, state unchanged
    enc.encode_async(f0, big, ln[1:2], ty[1:2], es[1:2])        # the same frame again: still the K-frame
    torch.cuda.synchronize()
    assert int(es[0]) == CAPACITY and int(ln[0]) == int(ln[1]) > 64
    assert int(es[1]) == OK and int(ty[1]) == 0
    assert enc.get_error() == CAPACITY and enc.get_error() == OK   # read and cleared
    ref, _ = _codec(kw).encode(f0)
    assert torch.equal(big[:int(ln[1])], ref)
    # a P-frame first: STATE on the device, the decoder still waits for a K-frame
    s1, _ = enc.encode(f1)
    s1 = s1.clone()
    dec = _codec(kw)
    rgb = torch.zeros((kw["height"], kw["width"], 3), dtype=torch.uint8, device="cuda")
    ds = torch.zeros(3, dtype=torch.int32, device="cuda")
    k0 = big[:int(ln[1])].clone()
    dec.decode_async(s1, rgb, status=ds[0:1])
    bad = k0.clone()
    bad[0] = ord("X")
    dec.decode_async(bad, rgb, status=ds[1:2])                   # corrupt: CORRUPT, nothing changes
    dec.decode_async(k0, rgb, status=ds[2:3])
    torch.cuda.synchronize()
    assert ds.tolist() == [STATE, CORRUPT, OK]
    assert dec.get_error() == STATE and dec.get_error() == OK    # the first failure is kept
    ref_dec = _codec(kw)
    assert torch.equal(rgb, ref_dec.decode(k0.clone()))
    assert torch.equal(dec.decode(s1.clone()), ref_dec.decode(s1.clone()))


def test_reset_is_stream_ordered():
    kw = QCIF
    frames = _frames(kw, 3, seed=62)
    enc = _codec(kw)
    out = [torch.empty(enc.max_stream, dtype=torch.uint8, device="cuda") for _ in range(3)]
    ty = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    enc.encode_async(frames[0], out[0], frame_type=ty[0:1])
    enc.encode_async(frames[1], out[1], frame_type=ty[1:2])
    enc.reset()                                                  # after the two queued calls
    enc.encode_async(frames[2], out[2], frame_type=ty[2:3])
    torch.cuda.synchronize()
    assert ty.tolist() == [0, 1, 0]


def test_queued_batch_steps_equal_plain_codecs():
    streams = [dict(QCIF), dict(QCIF, key_interval=2),
               dict(width=99, height=77, levels=2, dirs_log2=[2, 2], qph=6, qpl=2, key_interval=4),
               dict(width=352, height=288, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=10)]
    T = 6
    frames = [_frames(s, T, seed=63 + i) for i, s in enumerate(streams)]
    b = Batch(streams)
    outs = [[torch.empty(b.info[i].max_stream_bytes, dtype=torch.uint8, device="cuda") for i in range(len(streams))]
            for _ in range(T)]
    rgbs = [[torch.zeros((s["height"], s["width"], 3), dtype=torch.uint8, device="cuda") for s in streams]
            for _ in range(T)]
    results = [b.results_buffer() for _ in range(T)]
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        for t in range(T):
            b.step_async(3, rgb=[fr[t] for fr in frames], rgb_out=rgbs[t], outs=outs[t], results=results[t],
                         stream=st)
    st.synchronize()
    plain_e = [_codec(s) for s in streams]
    plain_d = [_codec(s) for s in streams]
    for t in range(T):
        res = b.results_of(results[t])
        for i, s in enumerate(streams):
            ref, ft = plain_e[i].encode(frames[i][t])
            r = res[i]
            assert r["enc_status"] == OK and r["dec_status"] == OK
            assert r["frame_type"] == ft and r["dec_frame_type"] == ft and r["dec_frame_index"] == t
            assert r["out_len"] == ref.numel() and torch.equal(outs[t][i][:r["out_len"]], ref), (t, i)
            assert torch.equal(rgbs[t][i], plain_d[i].decode(ref.clone())), (t, i)
    for i in range(len(streams)):
        assert b.get_error(i, st) == OK
