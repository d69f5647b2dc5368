"""GPU parity of the codec path against the oracle, through the C ABI.

Bar (per stage):
  - colour + 4:2:0 + padding: bit-exact planes;
  - transform: 1e-4 on the 0-255 scale (see tolerances.py);
  - quantiser, K/P differencing, RLE, bitstream: bit-exact when the oracle is
    fed the GPU's own single-precision coefficients;
  - decoder: reconstructed planes within the single-precision storage bound of
    the synthesis path (tolerances.inverse_bound) of the oracle's decode of the
    same stream; final RGB identical except where a plane value sits within
    that bound of a rounding tie; PSNR within 0.01 dB.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import Codec, CvcError
from paper_1510_00561_b300 import synthetic as S
from tolerances import FORWARD, inverse_bound

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
        assert np.abs(recon.astype(np.float64) - pref).max() < inverse_bound(kw["levels"], kw["dirs_log2"])
        diff = np.abs(rgb.astype(int) - rgb_ref.astype(int))
        assert (diff > 0).mean() <= 1e-3
        assert abs(_psnr(rgb, f) - _psnr(rgb_ref, f)) <= 0.01
    return g


def test_qcif_sequence_matches_oracle():
    """Plain pipeline, QCIF: 16 frames, 3-level 9/7 LP + 8/4/4 directions, K every 8, step 8."""
    v = S.SyntheticVideo(S.spec_for(176, 144, seed=0))
    _run_sequence(QCIF, v.frames(16))


@pytest.mark.parametrize("qph", [4, 8, 16])
def test_vga_frames_match_oracle(qph):
    """VGA decomposition (4 levels, 16/8/8/4 directions, K every 10) over a K and two P frames."""
    kw = dict(width=640, height=480, levels=4, dirs_log2=[4, 3, 3, 2], qph=qph, qpl=1, key_interval=10)
    v = S.SyntheticVideo(S.spec_for(640, 480, seed=qph))
    _run_sequence(kw, v.frames(3), check_coeffs_every=3)


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


def test_end_to_end_against_fp64_oracle_symbols():
    """Oracle coefficients in FP64 vs the GPU's FP32: quantised symbols agree except
    for rare rounding ties, each off by one."""
    g, o = _pair(**QCIF)
    f = S.SyntheticVideo(S.spec_for(176, 144, seed=9)).frame(0)
    s, _ = g.encode(torch.from_numpy(f).cuda())
    so, _ = o.encode(f)
    n = g.ncomp
    tg = np.frombuffer(bytes(s.cpu().numpy()[32 + 4 * n:]), "<i2")
    to = np.frombuffer(bytes(so[32 + 4 * n:]), "<i2")
    if tg.size == to.size and np.array_equal(tg, to):
        return
    # expand both to codes and compare
    cg = np.frombuffer(bytes(s.cpu().numpy()[32:32 + 4 * n]), "<u4")
    co = np.frombuffer(bytes(so[32:32 + 4 * n]), "<u4")
    lays = [O.layout(g.Hp, g.Wp, 3, [3, 2, 2])] + [O.layout(g.Hcp, g.Wcp, 3, [3, 2, 2])] * 2
    pg = po = 0
    mism = total = 0
    j = 0
    for lay in lays:
        for sb in lay["subbands"]:
            m = sb["h"] * sb["w"]
            if sb["kind"] == 0:
                a, b = tg[pg:pg + cg[j]], to[po:po + co[j]]
            else:
                a, b = O.rle_expand(tg[pg:pg + cg[j]], m), O.rle_expand(to[po:po + co[j]], m)
            mism += int(np.count_nonzero(a != b))
            assert np.abs(a.astype(int) - b.astype(int)).max() <= 1
            total += m
            pg += cg[j]
            po += co[j]
            j += 1
    assert mism / total <= 1e-4


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
