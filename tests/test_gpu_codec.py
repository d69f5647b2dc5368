"""GPU parity of the codec path against the oracle, through the C ABI.

Bar (per stage):
  - colour + 4:2:0 + padding: bit-exact planes;
  - transform: 1e-4 on the 0-255 scale (see tolerances.py);
  - quantiser, K/P differencing, RLE, bitstream: bit-exact when the oracle is
    fed the GPU's own single-precision coefficients;
  - decoder: reconstructed planes within the inverse bar (tolerances.INVERSE,
    1e-4) of the oracle's decode of the same stream; the output stage bit-exact
    on the GPU's own planes, and a rounded plane sample different from the
    oracle's only where the oracle's value lies within that bar of a rounding
    tie (decode_check.py); PSNR within 0.01 dB.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import Codec, CvcError
from paper_1510_00561_b300 import synthetic as S
from decode_check import check_decode
from tolerances import FORWARD, INVERSE

pytestmark = pytest.mark.gpu

QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=8)


def _pair(**kw):
    g = Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"],
              kw.get("threshold", 0.0), kw["key_interval"])
    o = O.Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"],
                kw.get("threshold", 0.0), kw["key_interval"])
    return g, o


def _coef_err(c, ref, cod):
    """per-level gain-normalised max error over the three planes (see test_gpu_ct)."""
    err = 0.0
    off = 0
    for H, W in ((cod.Hp, cod.Wp), (cod.Hcp, cod.Wcp), (cod.Hcp, cod.Wcp)):
        lay = O.layout(H, W, cod.levels, cod.dirs)
        for sb in lay["subbands"]:
            g = 2.0 ** -cod.levels if sb["level"] == 0 else 2.0 ** -(sb["level"] - 1)
            a = off + sb["off"]
            n = sb["h"] * sb["w"]
            err = max(err, float(np.abs(c[a:a + n].astype(np.float64) - ref[a:a + n]).max()) * g)
        off += lay["total"]
    return err


def _psnr(a, b):
    mse = np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2)
    return 10 * np.log10(255.0 ** 2 / max(mse, 1e-12))


def _run_sequence(kw, frames, check_coeffs_every=1):
    g, o = _pair(**kw)
    og = O.Codec(kw["width"], kw["height"], kw["levels"], kw["dirs_log2"], kw["qph"], kw["qpl"],
                 kw.get("threshold", 0.0), kw["key_interval"])   # independent decoder of the GPU stream
    for t, f in enumerate(frames):
        ft_expect = 0 if t % kw["key_interval"] == 0 else 1
        s, ft = g.encode(torch.from_numpy(f).cuda())
        assert ft == ft_expect
        s_np = s.cpu().numpy()
        # colour, chroma and padding are bit-exact
        yp, cop, cgp = o.planes(f)
        planes = g.inspect(0).cpu().numpy()
        ny, nc = g.Hp * g.Wp, g.Hcp * g.Wcp
        assert np.array_equal(planes[:ny], yp.ravel().astype(np.float32))
        assert np.array_equal(planes[ny:ny + nc], cop.ravel().astype(np.float32))
        assert np.array_equal(planes[ny + nc:], cgp.ravel().astype(np.float32))
        # the transform matches the FP64 oracle on those planes
        coef = g.inspect(1).cpu().numpy()
        if t % check_coeffs_every == 0:
            ref = np.concatenate([O.ct(0, p, p.shape[0], p.shape[1], kw["levels"], kw["dirs_log2"])
                                  for p in (yp, cop, cgp)])
            assert _coef_err(coef, ref, g) < FORWARD
        # quantiser, K/P and RLE are bit-exact from the GPU's own coefficients
        ref_stream, rft = o.encode_from_coeffs(coef)
        assert rft == ft
        assert np.array_equal(s_np, ref_stream), "bitstream mismatch at frame %d" % t
        # decode on the GPU and in the oracle
        rgb = g.decode(s.clone()).cpu().numpy()
        recon = g.inspect(2).cpu().numpy()
        rgb_ref, planes_ref = og.decode(s_np, want_planes=True)
        pref = np.concatenate([p.ravel() for p in planes_ref])
        assert np.abs(recon.astype(np.float64) - pref).max() < INVERSE
        check_decode(rgb, recon, planes_ref, kw["height"], kw["width"], g.Hc, g.Wc)
        assert abs(_psnr(rgb, f) - _psnr(rgb_ref, f)) <= 0.01
    return g


def test_qcif_sequence_matches_oracle():
    """Plain pipeline, QCIF: 16 frames, 3-level 9/7 LP + 8/4/4 directions, K every 8, step 8."""
    v = S.SyntheticVideo(S.spec_for(176, 144, seed=0))
    _run_sequence(QCIF, v.frames(16))


@pytest.mark.parametrize("qph", [4, 8, 16])
def test_vga_frames_match_oracle(qph):
    """VGA decomposition (4 levels, 16/8/8/4 directions, K every 10) over 12 frames: a whole
    K-frame period (a K-frame and its chain of nine P-frames) and the next K-frame and P-frame."""
    kw = dict(width=640, height=480, levels=4, dirs_log2=[4, 3, 3, 2], qph=qph, qpl=1, key_interval=10)
    v = S.SyntheticVideo(S.spec_for(640, 480, seed=qph))
    _run_sequence(kw, v.frames(12), check_coeffs_every=4)


def test_odd_frame_size_padding_paths():
    kw = dict(width=99, height=77, levels=2, dirs_log2=[2, 2], qph=6, qpl=2, key_interval=3, threshold=3.0)
    v = S.SyntheticVideo(S.spec_for(99, 77, seed=2))
    _run_sequence(kw, v.frames(4))


def test_threshold_and_k1_decomposition():
    kw = dict(width=64, height=48, levels=2, dirs_log2=[1, 0], qph=3, qpl=1, key_interval=2, threshold=10.0)
    v = S.SyntheticVideo(S.spec_for(64, 48, seed=4))
    _run_sequence(kw, v.frames(3))


def test_full_size_1080p_frame():
    """The benchmark configuration: 1920x1080, 5 levels, 32/16/16/8/8, step 8."""
    kw = dict(width=1920, height=1080, levels=5, dirs_log2=[5, 4, 4, 3, 3], qph=8, qpl=1, key_interval=10)
    v = S.SyntheticVideo(S.spec_for(1920, 1080, seed=0))
    _run_sequence(kw, v.frames(2), check_coeffs_every=1)


def _codes(stream, lays, prev):
    """The quantised codes a frame carries: its tokens expanded per component (§3.8), the K-frame
    lowpass column differences summed back and P-frame residuals added to the previous codes
    (§3.7), with 16-bit wrap-around; the oracle's RLE expander does the expansion."""
    ncomp = sum(len(lay["subbands"]) for lay in lays)
    ftype = int(stream[6])
    cnt = np.frombuffer(bytes(stream[32:32 + 4 * ncomp]), "<u4")
    tok = np.frombuffer(bytes(stream[32 + 4 * ncomp:]), "<i2")
    parts, pos, j = [], 0, 0
    for lay in lays:
        for sb in lay["subbands"]:
            h, w = sb["h"], sb["w"]
            t = tok[pos:pos + cnt[j]]
            if ftype == 0 and sb["kind"] == 0:
                r = np.cumsum(t.astype(np.int64).reshape(h, w), axis=0).ravel()
            else:
                r = O.rle_expand(t, h * w).astype(np.int64)
            parts.append(r)
            pos += cnt[j]
            j += 1
    q = np.concatenate(parts)
    if ftype == 1:
        q = q + prev
    return ((q + 32768) % 65536) - 32768


def test_fp64_oracle_symbols_1080p_key_and_p_frame():
    """The quantised symbols of the GPU's FP32 coefficients against those of the oracle's FP64
    coefficients (both through the oracle's own quantiser, §3.5-3.6), on a 1080p K-frame and the
    P-frame after it: they agree except at rounding ties, at most 1e-5 of the symbols, each off by
    one."""
    kw = dict(width=1920, height=1080, levels=5, dirs_log2=[5, 4, 4, 3, 3], qph=8, qpl=1, key_interval=10)
    g, o32 = _pair(**kw)
    o64 = O.Codec(1920, 1080, 5, kw["dirs_log2"], 8, 1, 0.0, 10)
    ofp = O.Codec(1920, 1080, 5, kw["dirs_log2"], 8, 1, 0.0, 10)
    lays = [O.layout(g.Hp, g.Wp, 5, kw["dirs_log2"])] + [O.layout(g.Hcp, g.Wcp, 5, kw["dirs_log2"])] * 2
    q32 = q64 = None
    for t, f in enumerate(S.SyntheticVideo(S.spec_for(1920, 1080, seed=9)).frames(2)):
        s, ft = g.encode(torch.from_numpy(f).cuda())
        assert ft == t
        s32, _ = o32.encode_from_coeffs(g.inspect(1).cpu().numpy())
        assert np.array_equal(s.cpu().numpy(), s32)
        _, _, c64 = ofp.encode(f, want_coeffs=True)
        s64, _ = o64.encode_from_coeffs(c64.astype(np.float32))
        q32 = _codes(s32, lays, q32)
        q64 = _codes(s64, lays, q64)
        d = q32 != q64
        assert np.abs(q32 - q64)[d].max(initial=0) <= 1
        assert d.sum() <= 1e-5 * d.size, (t, int(d.sum()), d.size)


def test_capacity_error_leaves_state_unchanged():
    g, _ = _pair(**QCIF)
    v = S.SyntheticVideo(S.spec_for(176, 144, seed=1))
    f0, f1 = (torch.from_numpy(x).cuda() for x in v.frames(2))
    s0, _ = g.encode(f0)
    small = torch.empty(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(CvcError) as e:
        g.encode(f1, out=small)
    assert e.value.status == 3 and e.value.needed > 100
    s1, ft = g.encode(f1)
    assert ft == 1 and s1.numel() == e.value.needed
    g2, _ = _pair(**QCIF)
    g2.encode(f0)
    s1b, _ = g2.encode(f1)
    assert torch.equal(s1, s1b)


def test_decoder_errors():
    g, _ = _pair(**QCIF)
    v = S.SyntheticVideo(S.spec_for(176, 144, seed=1))
    s0, _ = g.encode(torch.from_numpy(v.frame(0)).cuda())
    s0 = s0.clone()
    s1, _ = g.encode(torch.from_numpy(v.frame(1)).cuda())
    s1 = s1.clone()
    d, _ = _pair(**QCIF)
    with pytest.raises(CvcError) as e:            # P-frame first
        d.decode(s1)
    assert e.value.status == 9
    bad = s0.clone()
    bad[0] = ord("X")
    with pytest.raises(CvcError) as e:
        d.decode(bad)
    assert e.value.status == 5
    with pytest.raises(CvcError) as e:            # truncated
        d.decode(s0[:-2].clone())
    assert e.value.status == 5
    other = Codec(176, 144, 3, [3, 2, 2], 9, 1, 0.0, 8)
    with pytest.raises(CvcError) as e:            # parameter mismatch
        other.decode(s0)
    assert e.value.status == 5
    # after the failures the decoder still accepts the valid sequence
    r0 = d.decode(s0)
    r1 = d.decode(s1)
    assert r0.shape == r1.shape == (144, 176, 3)
