"""Scalable decoding on the GPU (§3.3: every pyramid scale of a frame can be
decoded on its own), through cvc_decode_frame_scaled and
cvc_batch_step_scaled, against the oracle's scaled decode.

Bar:
  - scale L (the lowpass band itself): RGB bit-identical to the oracle (both
    sides hold the same exact dequantised values);
  - 0 < scale < L: the reconstructed level-s planes within the synthesis
    bar (tolerances.INVERSE) of the oracle's; the output stage bit-exact on
    the GPU's own planes, a rounded sample different from the oracle's only
    within that bar of a rounding tie (decode_check.py);
  - the decoder state is updated in full at every scale, so a later
    full-scale decode is bit-identical to that of a decoder that decoded
    every frame at full scale;
  - batched steps at a scale are bit-identical to plain codecs at that scale.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import Batch, Codec, CvcError
from paper_1510_00561_b300 import synthetic as S
from decode_check import check_decode
from tolerances import INVERSE

pytestmark = pytest.mark.gpu

QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4)
ODD = dict(width=99, height=77, levels=2, dirs_log2=[2, 2], qph=6, qpl=2, key_interval=3, threshold=3.0)
VGA = dict(width=640, height=480, levels=4, dirs_log2=[4, 3, 3, 2], qph=8, qpl=1, key_interval=10)


def _gpu(kw):
    return Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"],
                 kw.get("threshold", 0.0), kw["key_interval"])


def _oracle(kw):
    return O.Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"],
                   kw.get("threshold", 0.0), kw["key_interval"])


def _frames(kw, n, seed):
    v = S.SyntheticVideo(S.spec_for(kw["width"], kw["height"], seed=seed))
    return v.frames(n)


def _encode_all(kw, frames):
    g = _gpu(kw)
    return [g.encode(torch.from_numpy(f).cuda())[0].clone() for f in frames]


def _check_frame(g, rgb, scale, og, s_np, kw):
    rgb_ref, planes_ref = og.decode(s_np, want_planes=True, scale=scale)
    assert rgb.shape == rgb_ref.shape
    L = kw["levels"]
    if scale < L:
        # level-s planes of the GPU (before normalisation) sit where the full planes would
        recon = g.inspect(2).cpu().numpy().astype(np.float64)
        pos = 0
        for p in planes_ref:
            n = p.size
            got = recon[pos:pos + n] * 2.0 ** -scale
            assert np.abs(got - p.ravel()).max() < INVERSE
            pos += n
        f = 1 << scale
        check_decode(rgb, recon, planes_ref, rgb.shape[0], rgb.shape[1], (g.Hc + f - 1) // f, (g.Wc + f - 1) // f,
                     norm=2.0 ** -scale)
    else:
        assert np.array_equal(rgb, rgb_ref)


@pytest.mark.parametrize("kw", [QCIF, ODD, VGA], ids=["qcif", "odd", "vga"])
def test_every_scale_matches_the_oracle(kw):
    """A K-frame and P-frames, each decoded at every scale by fresh decoders
    that decoded the earlier frames at full scale."""
    frames = _frames(kw, 3, seed=21)
    streams = _encode_all(kw, frames)
    L = kw["levels"]
    for scale in range(L + 1):
        g, og = _gpu(kw), _oracle(kw)
        for t, st in enumerate(streams):
            s_np = st.cpu().numpy()
            if t == 1:               # the middle frame at full scale
                g.decode(st.clone())
                og.decode(s_np)
                continue
            rgb = g.decode(st.clone(), scale=scale).cpu().numpy()
            h, w = g.scaled_size(scale)
            assert rgb.shape == (h, w, 3)
            _check_frame(g, rgb, scale, og, s_np, kw)


def test_scale_changes_keep_the_decoder_state():
    """Frames at coarse scales, then full scale: identical to a decoder that
    decoded every frame at full scale."""
    kw = QCIF
    frames = _frames(kw, 6, seed=22)
    streams = _encode_all(kw, frames)
    ref, mixed = _gpu(kw), _gpu(kw)
    og = _oracle(kw)
    for t, s in enumerate(streams):
        full = ref.decode(s.clone()).clone()
        sc = [3, 1, 2, 0, 2, 0][t]
        got = mixed.decode(s.clone(), scale=sc)
        if sc == 0:
            assert torch.equal(got, full)
        _check_frame(mixed, got.cpu().numpy(), sc, og, s.cpu().numpy(), kw)


def test_graph_and_direct_launches_agree_at_every_scale():
    kw = ODD
    frames = _frames(kw, 2, seed=23)
    streams = _encode_all(kw, frames)
    for scale in range(kw["levels"] + 1):
        outs = []
        for graphs in (True, False):
            b = Batch([kw])
            b.set_graphs(graphs)
            h, w = b.scaled_size(0, scale)
            res = []
            for s in streams:
                o = torch.full((h, w, 3), 7, dtype=torch.uint8, device="cuda")
                r = b.step(2, streams_in=[s], rgb_out=[o], scale=scale)
                assert r[0]["dec_status"] == 0
                res.append(o)
            outs.append(res)
        for a, c in zip(*outs):
            assert torch.equal(a, c)


def test_batched_scaled_steps_match_plain_codecs():
    """A mixed batch (levels 2..4) decoding and encoding + decoding at each
    scale up to the smallest level count: bit-identical to plain codecs at
    that scale; a stream without enough levels may join when it does not
    decode."""
    cfgs = [QCIF, ODD, VGA, QCIF]
    T = 3
    frames = [_frames(kw, T, seed=30 + i) for i, kw in enumerate(cfgs)]
    streams = [_encode_all(kw, fr) for kw, fr in zip(cfgs, frames)]
    for scale in range(3):
        b = Batch(cfgs)
        plain = [_gpu(kw) for kw in cfgs]
        for t in range(T):
            outs = []
            for i, kw in enumerate(cfgs):
                h, w = b.scaled_size(i, scale)
                outs.append(torch.zeros((h, w, 3), dtype=torch.uint8, device="cuda"))
            res = b.step(2, streams_in=[s[t] for s in streams], rgb_out=outs, scale=scale)
            for i in range(len(cfgs)):
                assert res[i]["dec_status"] == 0
                ref = plain[i].decode(streams[i][t].clone(), scale=scale)
                assert torch.equal(outs[i], ref), (scale, t, i)
    # encode + decode of the step's own output at scale 2: the encoder is unchanged
    b = Batch(cfgs)
    enc = [_gpu(kw) for kw in cfgs]
    dec = [_gpu(kw) for kw in cfgs]
    for t in range(T):
        outs = [torch.zeros(b.scaled_size(i, 2) + (3,), dtype=torch.uint8, device="cuda") for i in range(len(cfgs))]
        res = b.step(3, rgb=[torch.from_numpy(fr[t]).cuda() for fr in frames], rgb_out=outs, scale=2)
        for i in range(len(cfgs)):
            s_ref, _ = enc[i].encode(torch.from_numpy(frames[i][t]).cuda())
            assert torch.equal(res[i]["bytes"], s_ref)
            assert torch.equal(outs[i], dec[i].decode(s_ref.clone(), scale=2))
    # scale 3: only streams with 3 or more levels may decode
    b = Batch(cfgs)
    outs = [None, None, torch.zeros(b.scaled_size(2, 3) + (3,), dtype=torch.uint8, device="cuda"), None]
    ins = [None, None, streams[2][0], None]
    res = b.step(2, streams_in=ins, rgb_out=outs, scale=3)
    assert res[2]["dec_status"] == 0
    assert torch.equal(outs[2], _gpu(VGA).decode(streams[2][0].clone(), scale=3))
    # ... and a step in which the 2-level stream would decode at scale 3 is refused whole
    sized = [torch.zeros(b.scaled_size(i, 3) + (3,), dtype=torch.uint8, device="cuda") for i in range(len(cfgs))]
    with pytest.raises(CvcError) as e:
        b.step(2, streams_in=[s[0] for s in streams], rgb_out=sized, scale=3)
    assert e.value.status == 1
    assert all(float(o.float().sum()) == 0.0 for o in sized)


def test_full_size_1080p_scales():
    """The benchmark configuration at scales 2 and 5 (the 60 x 34 lowpass band)."""
    kw = dict(width=1920, height=1080, levels=5, dirs_log2=[5, 4, 4, 3, 3], qph=8, qpl=1, key_interval=10)
    frames = _frames(kw, 1, seed=0)
    s = _encode_all(kw, frames)[0]
    for scale in (2, 5):
        g, og = _gpu(kw), _oracle(kw)
        rgb = g.decode(s.clone(), scale=scale).cpu().numpy()
        assert rgb.shape == ((1080 + (1 << scale) - 1) >> scale, 1920 >> scale, 3)
        _check_frame(g, rgb, scale, og, s.cpu().numpy(), kw)


def test_invalid_scales_are_refused():
    kw = ODD
    s = _encode_all(kw, _frames(kw, 1, seed=24))[0]
    g = _gpu(kw)
    for scale in (-1, 3):
        with pytest.raises(CvcError) as e:
            g.decode(s.clone(), out=torch.zeros((77, 99, 3), dtype=torch.uint8, device="cuda"), scale=scale)
        assert e.value.status == 1
    # an output row shorter than the scale's width
    with pytest.raises(CvcError) as e:
        g.decode(s.clone(), out=torch.zeros((39, 49, 3), dtype=torch.uint8, device="cuda"), scale=1)
    assert e.value.status == 1
    # nothing was decoded: the stream still needs its K-frame and decodes normally
    out = g.decode(s.clone(), scale=1)
    assert out.shape == (39, 50, 3)


def _host(s):
    return s.cpu().numpy()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("kw", [QCIF, VGA], ids=["qcif", "vga"])
def test_dropped_levels_decode_like_complete_frames(kw):
    """§3.3: frames without their finest d levels (cvc_stream_drop_levels)
    decode at every scale s >= d exactly as the complete frames do, and
    match the oracle's decode of the same dropped frames."""
    frames = _frames(kw, 5, seed=25)
    kw = dict(kw, key_interval=3)                     # K P P K P
    streams = _encode_all(kw, frames)
    L = kw["levels"]
    g = _gpu(kw)
    for d in range(1, L + 1):
        dropped = [g.drop_levels(_host(s), d) for s in streams]
        for s, t in zip(streams, dropped):
            assert t.size < s.numel()
        for sc in range(d, L + 1):
            full, part, og = _gpu(kw), _gpu(kw), _oracle(kw)
            for t, (s, x) in enumerate(zip(streams, dropped)):
                a = full.decode(s.clone(), scale=sc)
                b = part.decode(_dev(x), scale=sc)
                assert torch.equal(a, b), (d, sc, t)
                if sc == d:
                    _check_frame(part, b.cpu().numpy(), sc, og, x, kw)
                else:
                    og.decode(x, scale=sc)


def test_dropped_levels_bound_the_decodable_scales():
    kw = dict(QCIF, key_interval=3)
    streams = _encode_all(kw, _frames(kw, 5, seed=26))      # K P P K P
    g = _gpu(kw)
    d2 = [_dev(g.drop_levels(_host(s), 2)) for s in streams]
    dec = _gpu(kw)
    with pytest.raises(CvcError) as e:
        dec.decode(d2[0], scale=1)                           # the frame lacks level 2
    assert e.value.status == 9
    dec.decode(d2[0], scale=2)
    with pytest.raises(CvcError) as e:
        dec.decode(streams[1].clone(), scale=0)              # no state for levels 1-2
    assert e.value.status == 9
    dec.decode(streams[1].clone(), scale=2)
    dec.decode(streams[2].clone(), scale=3)
    ref = _gpu(kw)
    for s in streams:
        last = ref.decode(s.clone()).clone()
    # a complete K-frame restores every level
    assert torch.equal(dec.decode(streams[3].clone()), _gpu(kw).decode(streams[3].clone()))
    assert torch.equal(dec.decode(streams[4].clone()), last)
    # a corrupt drop count is refused
    bad = streams[0].clone()
    bad[26] = 7
    with pytest.raises(CvcError) as e:
        _gpu(kw).decode(bad, scale=3)
    assert e.value.status == 5


def test_batch_with_different_drops_per_stream():
    cfgs = [QCIF, VGA, QCIF, VGA]
    drops = [0, 1, 2, 2]
    T = 3
    frames = [_frames(kw, T, seed=40 + i) for i, kw in enumerate(cfgs)]
    streams = [_encode_all(kw, fr) for kw, fr in zip(cfgs, frames)]
    g = [_gpu(kw) for kw in cfgs]
    for scale in (2, 3):
        b = Batch(cfgs)
        plain = [_gpu(kw) for kw in cfgs]
        for t in range(T):
            ins = [_dev(g[i].drop_levels(_host(streams[i][t]), drops[i])) for i in range(len(cfgs))]
            outs = [torch.zeros(b.scaled_size(i, scale) + (3,), dtype=torch.uint8, device="cuda")
                    for i in range(len(cfgs))]
            res = b.step(2, streams_in=ins, rgb_out=outs, scale=scale)
            for i in range(len(cfgs)):
                assert res[i]["dec_status"] == 0
                assert torch.equal(outs[i], plain[i].decode(streams[i][t].clone(), scale=scale)), (scale, t, i)
