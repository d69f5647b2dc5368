"""The 8-bit storage variant on the GPU (§3.1 Table 1, §3.6) against the oracle.

Bar (as for the int16 codec):
  - the padded planes (Table 1, bytes, chroma + 127, 4:2:0) are identical to
    the oracle's (integers);
  - the bitstream is bit-identical to the oracle's entropy side fed the GPU's
    single-precision coefficients (byte clamp, quantiser, K/P, motion, RLE);
  - the decoder's reconstruction is within the synthesis bound of the
    oracle's decode of the same stream, RGB identical except near rounding
    ties, at every scale;
  - at QPH = 181 the subband codes of a 1080p K-frame fit a byte and are
    almost all zero (the paper says all; 0.02% of its coefficients reach the
    90.5 that a non-zero code needs);
  - batches mixing both storages are bit-identical to plain codecs; each
    decoder refuses the other storage's streams; DEFLATE carries the frames.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import Batch, Codec, CvcError, Deflater
from paper_1510_00561_b300 import synthetic as S
from decode_check import check_decode, check_scaled_decode
from tolerances import INVERSE

pytestmark = pytest.mark.gpu

QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4, motion_range=8,
            storage8=True)
ODD = dict(width=99, height=77, levels=2, dirs_log2=[2, 2], qph=6, qpl=2, key_interval=3, threshold=3.0,
           storage8=True)
HD181 = dict(width=1920, height=1080, levels=5, dirs_log2=[5, 4, 4, 3, 3], qph=181, qpl=12, key_interval=10,
             storage8=True)


def _args(kw):
    return (kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"], kw.get("threshold", 0.0),
            kw["key_interval"], kw.get("motion_range", 0))


def _gpu(kw):
    return Codec(*_args(kw), storage8=kw.get("storage8", False))


def _oracle(kw):
    return O.Codec(*_args(kw), storage8=kw.get("storage8", False))


def _frames(kw, n, seed):
    return S.SyntheticVideo(S.spec_for(kw["width"], kw["height"], seed=seed)).frames(n)


def _run(kw, frames):
    g, o, od = _gpu(kw), _oracle(kw), _oracle(kw)
    streams = []
    for t, f in enumerate(frames):
        s, ft = g.encode(torch.from_numpy(f).cuda())
        s_np = s.cpu().numpy()
        assert s_np[5] == 1
        planes = g.inspect(0).cpu().numpy()
        ref = np.concatenate([p.ravel() for p in o.planes(f)])
        assert np.array_equal(planes, ref), "planes differ at frame %d" % t
        luma = planes[:g.Hp * g.Wp].reshape(g.Hp, g.Wp).astype(np.uint8)
        ref_stream, rft = o.encode_from_coeffs(g.inspect(1).cpu().numpy(),
                                               luma=luma if kw.get("motion_range") else None)
        assert rft == ft and np.array_equal(s_np, ref_stream), "bitstream mismatch at frame %d" % t
        rgb = g.decode(s.clone()).cpu().numpy()
        recon = g.inspect(2).cpu().numpy().astype(np.float64)
        rgb_ref, planes_ref = od.decode(s_np, want_planes=True)
        pref = np.concatenate([p.ravel() for p in planes_ref])
        assert np.abs(recon - pref).max() < INVERSE
        check_decode(rgb, recon, planes_ref, kw["height"], kw["width"], g.Hc, g.Wc, storage8=True)
        streams.append(s_np)
    return g, streams


@pytest.mark.parametrize("kw,n", [(QCIF, 6), (ODD, 4)], ids=["qcif_motion", "odd"])
def test_storage8_codec_matches_the_oracle(kw, n):
    _run(kw, _frames(kw, n, seed=80))


def test_storage8_1080p_at_qph_181_leaves_few_codes():
    g, streams = _run(HD181, _frames(HD181, 2, seed=81))
    s = streams[0]                                   # the K-frame
    ncomp = g.ncomp
    hdr = 32 + 4 * ncomp
    counts = np.frombuffer(s[32:hdr].tobytes(), "<u4")
    toks = np.frombuffer(s[hdr:hdr + 2 * int(counts.sum())].tobytes(), "<i2")
    nsub = 1 + sum(1 << k for k in HD181["dirs_log2"])
    pos, nz, total = 0, 0, 0
    for j, n in enumerate(counts):
        t = toks[pos:pos + n]
        pos += n
        if j % nsub == 0:
            continue                                 # a lowpass band
        i = 0
        while i < len(t):
            if t[i] == 0:
                total += int(t[i + 1])
                i += 2
            else:
                assert -128 <= t[i] <= 127
                nz += 1
                total += 1
                i += 1
    L = HD181["levels"]
    nlow = (g.Hp >> L) * (g.Wp >> L) + 2 * (g.Hcp >> L) * (g.Wcp >> L)
    assert total == g.ncoef - nlow                   # every subband element accounted for
    assert nz / total < 1e-3


def test_scaled_decoding_of_storage8_streams():
    kw = dict(QCIF, key_interval=3)
    frames = _frames(kw, 4, seed=82)
    g = _gpu(kw)
    streams = [g.encode(torch.from_numpy(f).cuda())[0].clone() for f in frames]
    for sc in range(kw["levels"] + 1):
        d, og = _gpu(kw), _oracle(kw)
        for s in streams:
            a = d.decode(s.clone(), scale=sc).cpu().numpy()
            check_scaled_decode(d, a, og, s.cpu().numpy(), sc, storage8=True)


def test_each_decoder_refuses_the_other_storage():
    kw = ODD
    f = _frames(kw, 1, seed=83)[0]
    s8 = _gpu(kw).encode(torch.from_numpy(f).cuda())[0].clone()
    s16 = _gpu(dict(kw, storage8=False)).encode(torch.from_numpy(f).cuda())[0].clone()
    assert int(s8[5]) == 1 and int(s16[5]) == 0
    with pytest.raises(CvcError) as e:
        _gpu(dict(kw, storage8=False)).decode(s8.clone())
    assert e.value.status == 5
    with pytest.raises(CvcError) as e:
        _gpu(kw).decode(s16.clone())
    assert e.value.status == 5
    _gpu(kw).decode(s8.clone())


def test_mixed_batch_of_both_storages_is_bit_identical_to_plain_codecs():
    cfgs = [QCIF, dict(QCIF, storage8=False), ODD, dict(ODD, storage8=False)]
    T = 4
    frames = [[torch.from_numpy(f).cuda() for f in _frames(kw, T, seed=84 + i)] for i, kw in enumerate(cfgs)]
    b = Batch(cfgs)
    enc = [_gpu(kw) for kw in cfgs]
    dec = [_gpu(kw) for kw in cfgs]
    outs = [torch.zeros((kw["height"], kw["width"], 3), dtype=torch.uint8, device="cuda") for kw in cfgs]
    for t in range(T):
        res = b.step(3, rgb=[fr[t] for fr in frames], rgb_out=outs)
        for i in range(len(cfgs)):
            s, ft = enc[i].encode(frames[i][t])
            assert res[i]["frame_type"] == ft and torch.equal(res[i]["bytes"], s)
            assert torch.equal(outs[i], dec[i].decode(s.clone())), (t, i)


@pytest.mark.parametrize("nts", [False, True], ids=["scalable", "nts"])
def test_deflate_of_storage8_frames(nts):
    kw = QCIF
    g, oc = _gpu(kw), _oracle(kw)
    dfl = Deflater(nts=nts, **kw)
    for f in _frames(kw, 3, seed=85):
        s = g.encode(torch.from_numpy(f).cuda())[0].clone()
        packed = dfl.deflate(s).clone()
        assert int(packed[5]) == 1
        assert np.array_equal(oc.inflate_container(packed.cpu().numpy()), s.cpu().numpy())
        assert torch.equal(dfl.inflate(packed), s)
