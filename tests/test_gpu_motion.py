"""Motion-compensated P-frames on the GPU (§3.2, §3.7) against the oracle.

Bar (as for the zero-motion codec):
  - the motion vectors are bit-identical to the oracle's full search on the
    GPU's own padded luma planes (integer sums, the same tie rules);
  - the bitstream is bit-identical to the oracle's entropy side fed the
    GPU's single-precision coefficients and luma (prediction, residuals,
    RLE, vector field);
  - the decoder's reconstruction is within the synthesis bound of the
    oracle's decode of the same stream, RGB identical except near rounding
    ties;
  - batches mixing streams with and without motion are bit-identical to
    plain codecs; scaled decoding and dropped levels work on them.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import Batch, Codec, CvcError
from paper_1510_00561_b300 import synthetic as S
from decode_check import check_decode, check_scaled_decode
from tolerances import INVERSE

pytestmark = pytest.mark.gpu

QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4, motion_range=8)
ODD = dict(width=99, height=77, levels=2, dirs_log2=[2, 2], qph=6, qpl=2, key_interval=3, motion_range=5,
           threshold=3.0)
VGA = dict(width=640, height=480, levels=4, dirs_log2=[4, 3, 3, 2], qph=8, qpl=1, key_interval=10, motion_range=16)


def _gpu(kw):
    return Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"],
                 kw.get("threshold", 0.0), kw["key_interval"], kw.get("motion_range", 0))


def _oracle(kw):
    return O.Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"],
                   kw.get("threshold", 0.0), kw["key_interval"], kw.get("motion_range", 0))


def _frames(kw, n, seed):
    return S.SyntheticVideo(S.spec_for(kw["width"], kw["height"], seed=seed)).frames(n)


def _nblocks(g):
    return ((g.Hp + 15) // 16) * ((g.Wp + 15) // 16)


def _run(kw, frames):
    g, o, od = _gpu(kw), _oracle(kw), _oracle(kw)
    prev_luma = None
    for t, f in enumerate(frames):
        s, ft = g.encode(torch.from_numpy(f).cuda())
        assert ft == (0 if t % kw["key_interval"] == 0 else 2)
        s_np = s.cpu().numpy()
        planes = g.inspect(0).cpu().numpy()
        luma = planes[:g.Hp * g.Wp].reshape(g.Hp, g.Wp)
        assert (luma == np.round(luma)).all() and luma.min() >= 0 and luma.max() <= 255
        luma = luma.astype(np.uint8)
        if ft == 2:
            mv = np.frombuffer(bytes(s_np[-2 * _nblocks(g):]), np.int8).reshape(-1, 2)
            ref = O.motion_search(luma, prev_luma, kw["motion_range"]).reshape(-1, 2)
            assert np.array_equal(mv, ref), "motion vectors differ at frame %d" % t
        prev_luma = luma
        ref_stream, rft = o.encode_from_coeffs(g.inspect(1).cpu().numpy(), luma=luma)
        assert rft == ft and np.array_equal(s_np, ref_stream), "bitstream mismatch at frame %d" % t
        rgb = g.decode(s.clone()).cpu().numpy()
        recon = g.inspect(2).cpu().numpy().astype(np.float64)
        rgb_ref, planes_ref = od.decode(s_np, want_planes=True)
        pref = np.concatenate([p.ravel() for p in planes_ref])
        assert np.abs(recon - pref).max() < INVERSE
        check_decode(rgb, recon, planes_ref, kw["height"], kw["width"], g.Hc, g.Wc)
    return g


@pytest.mark.parametrize("kw,n", [(QCIF, 6), (ODD, 4), (VGA, 3)], ids=["qcif", "odd", "vga"])
def test_motion_codec_matches_the_oracle(kw, n):
    _run(kw, _frames(kw, n, seed=50))


def test_motion_1080p():
    kw = dict(width=1920, height=1080, levels=5, dirs_log2=[5, 4, 4, 3, 3], qph=8, qpl=1, key_interval=10,
              motion_range=8)
    _run(kw, _frames(kw, 2, seed=51))


def test_mixed_batch_with_and_without_motion_is_bit_identical_to_plain_codecs():
    zero = dict(QCIF, motion_range=0)
    cfgs = [QCIF, zero, ODD, VGA, QCIF, dict(ODD, motion_range=0)]
    T = 5
    frames = [[torch.from_numpy(f).cuda() for f in _frames(kw, T, seed=60 + i)] for i, kw in enumerate(cfgs)]
    b = Batch(cfgs)
    enc = [_gpu(kw) for kw in cfgs]
    dec = [_gpu(kw) for kw in cfgs]
    outs = [torch.zeros((kw["height"], kw["width"], 3), dtype=torch.uint8, device="cuda") for kw in cfgs]
    for t in range(T):
        res = b.step(3, rgb=[fr[t] for fr in frames], rgb_out=outs)
        for i in range(len(cfgs)):
            s, ft = enc[i].encode(frames[i][t])
            assert res[i]["frame_type"] == ft and torch.equal(res[i]["bytes"], s)
            assert res[i]["dec_frame_type"] == ft
            assert torch.equal(outs[i], dec[i].decode(s.clone())), (t, i)


def test_scaled_and_dropped_decoding_of_motion_streams():
    kw = dict(QCIF, key_interval=3)
    frames = _frames(kw, 5, seed=52)
    g = _gpu(kw)
    streams = [g.encode(torch.from_numpy(f).cuda())[0].clone() for f in frames]
    for d in range(kw["levels"] + 1):
        dropped = [torch.from_numpy(g.drop_levels(s.cpu(), d)).cuda() for s in streams]
        for sc in range(d, kw["levels"] + 1):
            full, part, og = _gpu(kw), _gpu(kw), _oracle(kw)
            for s, x in zip(streams, dropped):
                a = full.decode(s.clone(), scale=sc)
                b = part.decode(x, scale=sc)
                assert torch.equal(a, b), (d, sc)
                check_scaled_decode(part, b.cpu().numpy(), og, x.cpu().numpy(), sc)


def test_motion_stream_errors():
    kw = ODD
    frames = _frames(kw, 2, seed=53)
    g = _gpu(kw)
    s0 = g.encode(torch.from_numpy(frames[0]).cuda())[0].clone()
    s1, t1 = g.encode(torch.from_numpy(frames[1]).cuda())
    s1 = s1.clone()
    assert t1 == 2
    z = _gpu(dict(kw, motion_range=0))
    z.decode(s0.clone())
    with pytest.raises(CvcError) as e:
        z.decode(s1.clone())                          # vectors for a decoder without motion
    assert e.value.status == 5
    d = _gpu(kw)
    d.decode(s0.clone())
    bad = s1.clone()
    bad[-1] = 6                                       # beyond the range of 5
    with pytest.raises(CvcError) as e:
        d.decode(bad)
    assert e.value.status == 5
    with pytest.raises(CvcError) as e:
        d.decode(s1[:-1].clone())                     # truncated vector field
    assert e.value.status == 5
    d.decode(s1.clone())                              # rejected frames left the state as it was
    with pytest.raises(CvcError):
        Codec(99, 77, 2, [2, 2], 6, 2, 0.0, 3, 65)
