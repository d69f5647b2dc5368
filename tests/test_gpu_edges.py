"""Edge cases of the codec on the GPU against the oracle.

  - tiny frames (1 x 1 up to 17 x 3), where every plane is smaller than one
    LP or DFB tile: padded planes identical, coefficients within the
    transform bar, bitstreams bit-identical to the oracle's entropy side,
    reconstruction within the synthesis bound;
  - the deepest pyramid (6 levels, 64 down to 2 directions) on 256 x 256;
  - a frame size whose mirror padding would reach past the frame is refused
    by both;
  - the largest motion range (64: the search window is the whole QCIF
    frame): vectors and bitstreams bit-identical;
  - zero-length and truncated buffers are refused and leave the decoder as
    it was.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1510_00561_b300 import Codec, CvcError, Deflater, drop_levels
from paper_1510_00561_b300 import synthetic as S
from tolerances import FORWARD, INVERSE, ROUND_TRIP

pytestmark = pytest.mark.gpu


def _coef_err(c, ref, H, W, L, k):
    lay = O.layout(H, W, L, k)
    d = np.abs(np.asarray(c, np.float64) - ref)
    for sb in lay["subbands"]:
        g = 2.0 ** -L if sb["level"] == 0 else 2.0 ** -(sb["level"] - 1)
        d[sb["off"]:sb["off"] + sb["h"] * sb["w"]] *= g
    return d.max()


def _check_sequence(w, h, L, k, frames, motion=0, qph=4):
    g = Codec(w, h, L, k, qph, 1, 0.0, 3, motion)
    o, od = O.Codec(w, h, L, k, qph, 1, 0.0, 3, motion), O.Codec(w, h, L, k, qph, 1, 0.0, 3, motion)
    for t, f in enumerate(frames):
        s, ft = g.encode(torch.from_numpy(f).cuda())
        s_np = s.cpu().numpy()
        planes = g.inspect(0).cpu().numpy()
        ref_planes = o.planes(f)
        assert np.array_equal(planes, np.concatenate([p.ravel() for p in ref_planes])), t
        coef = g.inspect(1).cpu().numpy()
        co = 0
        for p in ref_planes:
            H, W = p.shape
            n = O.layout(H, W, L, k)["total"]
            assert _coef_err(coef[co:co + n], O.ct(0, p, H, W, L, k), H, W, L, k) < FORWARD, t
            co += n
        luma = planes[:g.Hp * g.Wp].reshape(g.Hp, g.Wp).astype(np.uint8)
        ref, rft = o.encode_from_coeffs(coef, luma=luma if motion else None)
        assert rft == ft and np.array_equal(s_np, ref), t
        rgb = g.decode(s.clone()).cpu().numpy()
        recon = g.inspect(2).cpu().numpy().astype(np.float64)
        rgb_ref, pr = od.decode(s_np, want_planes=True)
        assert np.abs(recon - np.concatenate([p.ravel() for p in pr])).max() < INVERSE
        assert np.abs(rgb.astype(int) - rgb_ref.astype(int)).max() <= 1
    return g


TINY = [(1, 1, 1, [0]), (2, 3, 1, [1]), (5, 7, 1, [0]), (7, 5, 2, [1, 0]), (17, 3, 1, [1]), (3, 17, 2, [1, 1])]


@pytest.mark.parametrize("w,h,L,k", TINY)
def test_tiny_frames_match_the_oracle(w, h, L, k):
    rng = np.random.default_rng(w * 31 + h)
    frames = [rng.integers(0, 256, (h, w, 3), dtype=np.uint8) for _ in range(4)]
    _check_sequence(w, h, L, k, frames)
    _check_sequence(w, h, L, k, frames, motion=2)


def test_deepest_pyramid():
    frames = S.SyntheticVideo(S.spec_for(256, 256, seed=95)).frames(3)
    _check_sequence(256, 256, 6, [6, 5, 4, 3, 2, 1], frames)


def test_padding_past_the_frame_is_refused():
    # 1 x 1 with two levels pads to 4 x 4: the mirror would reach past the frame
    with pytest.raises(CvcError):
        Codec(1, 1, 2, [0, 0], 4, 1, 0.0, 3)
    with pytest.raises(ValueError):
        O.Codec(1, 1, 2, [0, 0], 4, 1, 0.0, 3)


def test_largest_motion_range():
    frames = S.SyntheticVideo(S.spec_for(176, 144, seed=96)).frames(3)
    g = _check_sequence(176, 144, 3, [3, 2, 2], frames, motion=64, qph=8)
    assert g.motion_range == 64


def test_zero_length_and_truncated_buffers_are_refused():
    kw = dict(width=99, height=77, levels=2, dirs_log2=[2, 2], qph=6, qpl=2, key_interval=3)
    g = Codec(99, 77, 2, [2, 2], 6, 2, 0.0, 3)
    d, ref = Codec(99, 77, 2, [2, 2], 6, 2, 0.0, 3), Codec(99, 77, 2, [2, 2], 6, 2, 0.0, 3)
    frames = S.SyntheticVideo(S.spec_for(99, 77, seed=97)).frames(2)
    s0 = g.encode(torch.from_numpy(frames[0]).cuda())[0].clone()
    s1 = g.encode(torch.from_numpy(frames[1]).cuda())[0].clone()
    d.decode(s0.clone())
    ref.decode(s0.clone())
    empty = torch.empty(0, dtype=torch.uint8, device="cuda")
    for bad in (empty, s1[:31].clone(), s1[:-1].clone()):
        with pytest.raises(CvcError) as e:
            d.decode(bad)
        assert e.value.status in (1, 5)
    assert torch.equal(d.decode(s1.clone()), ref.decode(s1.clone()))   # the state was left as it was
    dfl = Deflater(**kw)
    for bad in (empty, dfl.deflate(s1.clone())[:40].clone()):
        with pytest.raises(CvcError) as e:
            dfl.inflate(bad)
        assert e.value.status in (1, 5)
    with pytest.raises(CvcError) as e:
        drop_levels(kw, np.zeros(0, np.uint8), 1)
    assert e.value.status in (1, 5)
