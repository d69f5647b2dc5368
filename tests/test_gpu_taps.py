"""Longer PKVA prototypes on the GPU (6- and 8-tap Lagrange half-band DFB,
the tile kernels instantiated for their length) against the oracle, through
the C ABI.

Bar (as for the 4-tap tile kernels):
  - the transform within 1e-4 per level on the 0-255 scale, the inverse of
    the same coefficients within the synthesis bound, adjoints within 2e-6
    of their scale;
  - codec bitstreams bit-identical to the oracle's entropy side fed the GPU's
    coefficients; decoding within the synthesis bound of the oracle's decode,
    at every scale;
  - batches mixing 4-, 6- and 8-tap streams bit-identical to plain codecs;
    a decoder refuses a stream of another prototype.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import Batch, Codec, CtPlan, CvcError
from paper_1510_00561_b300 import synthetic as S
from decode_check import check_decode, check_scaled_decode
from tolerances import FORWARD, INVERSE, ROUND_TRIP

pytestmark = pytest.mark.gpu

CASES = [(144, 176, 3, [3, 2, 2]), (96, 160, 4, [4, 3, 3, 2]), (64, 96, 2, [0, 1]), (128, 128, 2, [6, 5])]


def _coef_err(c, ref, H, W, L, k):
    """max |c - ref| with every level divided by its DC gain (2^(j-1), lowpass 2^L)"""
    lay = O.layout(H, W, L, k)
    d = np.abs(np.asarray(c, np.float64) - ref)
    for sb in lay["subbands"]:
        g = 2.0 ** -L if sb["level"] == 0 else 2.0 ** -(sb["level"] - 1)
        d[sb["off"]:sb["off"] + sb["h"] * sb["w"]] *= g
    return d.max()


@pytest.mark.parametrize("taps", [6, 8])
@pytest.mark.parametrize("H,W,L,k", CASES)
def test_transform_matches_oracle(taps, H, W, L, k):
    x = np.random.default_rng(taps).uniform(0, 255, (2, H, W)).astype(np.float32)
    plan = CtPlan(H, W, L, k, batch=2, dfb_taps=taps)
    c = plan.forward(torch.from_numpy(x).cuda())
    xr = plan.inverse(c)
    c_np, xr_np = c.cpu().numpy(), xr.cpu().numpy()
    for b in range(2):
        ref = O.ct(0, x[b].astype(np.float64), H, W, L, k, taps)
        assert _coef_err(c_np[b], ref, H, W, L, k) < FORWARD
        xin = O.ct(1, c_np[b].astype(np.float64), H, W, L, k, taps)
        assert np.abs(xr_np[b] - xin).max() < INVERSE
        assert np.abs(xr_np[b] - x[b]).max() < ROUND_TRIP
    # a different transform from the 4-tap one
    c4 = CtPlan(H, W, L, k, batch=2).forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.abs(c4 - c_np).max() > 1.0


@pytest.mark.parametrize("taps", [6, 8])
def test_adjoints_match_oracle(taps):
    H, W, L, k = 96, 160, 4, [4, 3, 3, 2]
    plan = CtPlan(H, W, L, k, batch=1, dfb_taps=taps)
    r = np.random.default_rng(3)
    cb = r.standard_normal((1, plan.total)).astype(np.float32) * 50
    xb = r.standard_normal((1, H, W)).astype(np.float32) * 50
    xa = plan.forward_adjoint(torch.from_numpy(cb).cuda()).cpu().numpy()[0]
    ca = plan.inverse_adjoint(torch.from_numpy(xb).cuda()).cpu().numpy()[0]
    for got, ref in ((xa, O.ct(2, cb[0].astype(np.float64), H, W, L, k, taps)),
                     (ca, O.ct(3, xb[0].astype(np.float64), H, W, L, k, taps))):
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4, motion_range=8)
ODD = dict(width=99, height=77, levels=2, dirs_log2=[2, 2], qph=6, qpl=2, key_interval=3)


def _args(kw):
    return (kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"], 0.0, kw["key_interval"],
            kw.get("motion_range", 0))


def _gpu(kw, taps):
    return Codec(*_args(kw), dfb_taps=taps)


def _oracle(kw, taps):
    return O.Codec(*_args(kw), dfb_taps=taps)


@pytest.mark.parametrize("taps", [6, 8])
@pytest.mark.parametrize("kw,n", [(QCIF, 5), (ODD, 3)], ids=["qcif_motion", "odd"])
def test_codec_matches_the_oracle(kw, n, taps):
    g, o, od = _gpu(kw, taps), _oracle(kw, taps), _oracle(kw, taps)
    for t, f in enumerate(S.SyntheticVideo(S.spec_for(kw["width"], kw["height"], seed=90)).frames(n)):
        s, ft = g.encode(torch.from_numpy(f).cuda())
        s_np = s.cpu().numpy()
        assert s_np[5] == (taps // 2 - 2) << 1
        planes = g.inspect(0).cpu().numpy()
        luma = planes[:g.Hp * g.Wp].reshape(g.Hp, g.Wp).astype(np.uint8)
        ref, rft = o.encode_from_coeffs(g.inspect(1).cpu().numpy(), luma=luma if kw.get("motion_range") else None)
        assert rft == ft and np.array_equal(s_np, ref), "bitstream mismatch at frame %d" % t
        rgb = g.decode(s.clone()).cpu().numpy()
        recon = g.inspect(2).cpu().numpy().astype(np.float64)
        rgb_ref, planes_ref = od.decode(s_np, want_planes=True)
        pref = np.concatenate([p.ravel() for p in planes_ref])
        assert np.abs(recon - pref).max() < INVERSE
        check_decode(rgb, recon, planes_ref, kw["height"], kw["width"], g.Hc, g.Wc)


def test_scaled_decoding_with_a_longer_prototype():
    kw = dict(QCIF, key_interval=3)
    g = _gpu(kw, 6)
    streams = [g.encode(torch.from_numpy(f).cuda())[0].clone()
               for f in S.SyntheticVideo(S.spec_for(176, 144, seed=91)).frames(4)]
    for sc in range(kw["levels"] + 1):
        d, og = _gpu(kw, 6), _oracle(kw, 6)
        for s in streams:
            a = d.decode(s.clone(), scale=sc).cpu().numpy()
            check_scaled_decode(d, a, og, s.cpu().numpy(), sc)


def test_mixed_prototypes_in_one_batch_and_refusals():
    cfgs = [dict(QCIF, dfb_taps=6), dict(QCIF), dict(ODD, dfb_taps=8), dict(ODD, dfb_taps=6)]
    T = 4
    frames = [[torch.from_numpy(f).cuda() for f in S.SyntheticVideo(S.spec_for(kw["width"], kw["height"],
                                                                                 seed=92 + i)).frames(T)]
              for i, kw in enumerate(cfgs)]
    b = Batch(cfgs)
    enc = [_gpu(kw, kw.get("dfb_taps", 4)) for kw in cfgs]
    dec = [_gpu(kw, kw.get("dfb_taps", 4)) for kw in cfgs]
    outs = [torch.zeros((kw["height"], kw["width"], 3), dtype=torch.uint8, device="cuda") for kw in cfgs]
    for t in range(T):
        res = b.step(3, rgb=[fr[t] for fr in frames], rgb_out=outs)
        for i in range(len(cfgs)):
            s, ft = enc[i].encode(frames[i][t])
            assert res[i]["frame_type"] == ft and torch.equal(res[i]["bytes"], s)
            assert torch.equal(outs[i], dec[i].decode(s.clone())), (t, i)
    s6 = _gpu(ODD, 6).encode(frames[3][0])[0].clone()
    with pytest.raises(CvcError) as e:
        _gpu(ODD, 4).decode(s6.clone())
    assert e.value.status == 5
    with pytest.raises(CvcError) as e:
        _gpu(ODD, 8).decode(s6.clone())
    assert e.value.status == 5
    _gpu(ODD, 6).decode(s6.clone())
    with pytest.raises(CvcError):
        Codec(*_args(ODD), dfb_taps=5)


def test_1080p_codec_with_a_longer_prototype():
    """the bench's size: one 1080p K-frame with the 6-tap prototype; every coefficient
    against the oracle's transform of the GPU's own planes, and the bitstream bit for bit"""
    kw = dict(width=1920, height=1080, levels=5, dirs_log2=[5, 4, 4, 3, 3], qph=8, qpl=1, key_interval=10)
    g, o = _gpu(kw, 6), _oracle(kw, 6)
    f = S.SyntheticVideo(S.spec_for(1920, 1080, seed=93)).frames(1)[0]
    s, ft = g.encode(torch.from_numpy(f).cuda())
    planes = g.inspect(0).cpu().numpy().astype(np.float64)
    coef = g.inspect(1).cpu().numpy()
    dims = [(g.Hp, g.Wp), (g.Hcp, g.Wcp), (g.Hcp, g.Wcp)]
    po = co = 0
    for H, W in dims:
        n = O.layout(H, W, 5, kw["dirs_log2"])["total"]
        ref = O.ct(0, planes[po:po + H * W].reshape(H, W), H, W, 5, kw["dirs_log2"], 6)
        assert _coef_err(coef[co:co + n], ref, H, W, 5, kw["dirs_log2"]) < FORWARD
        po += H * W
        co += n
    ref_stream, rft = o.encode_from_coeffs(coef)
    assert rft == ft == 0 and np.array_equal(s.cpu().numpy(), ref_stream)
