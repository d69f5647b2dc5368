"""The decoder's output stage checked exactly (test helper, no GPU needed).

A decoded frame is its reconstructed planes (single precision on the GPU,
double in the oracle) rounded half away from zero in single precision,
clamped, the chroma upsampled and the colour transform inverted (§3.1, §3.9).
Given the GPU's planes and RGB and the oracle's planes of the same stream,
`check_decode` asserts:

  1. the GPU's RGB is exactly what the oracle's own chroma upsampler and
     colour inverse make of the GPU's rounded planes: the integer output
     stage is bit-exact;
  2. the GPU's rounded planes differ from the oracle's only at samples whose
     oracle value lies within the inverse bar of a rounding tie (k + 1/2),
     and then by one: every differing RGB byte traces back to such a tie.

It returns the number of tie-adjacent samples that rounded differently.
"""
import numpy as np

import oracle as O
from tolerances import INVERSE


def _roundf(v):
    """round half away from zero of single-precision values (exact: in double, |v| + 0.5 does not round)"""
    v = np.asarray(v, np.float32).astype(np.float64)
    return (np.sign(v) * np.floor(np.abs(v) + 0.5)).astype(np.int64)


def _tie_distance(v):
    """distance of each single-precision value to the nearest k + 1/2"""
    a = np.abs(np.asarray(v, np.float32).astype(np.float64))
    return np.abs(a - np.floor(a) - 0.5)


def check_decode(rgb, recon, planes_ref, height, width, chroma_height, chroma_width, storage8=False, norm=1.0,
                 bar=INVERSE):
    """rgb: the GPU's output (h, w, 3) uint8; recon: the GPU's reconstructed planes, flat, Y then Co then Cg
    with the shapes of planes_ref (before multiplying by norm, a power of two); planes_ref: the oracle's
    (normalised) planes; height x width and chroma_height x chroma_width: the output sizes."""
    clo = 0 if storage8 else -255
    recon = np.asarray(recon, np.float32).ravel()
    sizes = ((height, width, 0), (chroma_height, chroma_width, clo), (chroma_height, chroma_width, clo))
    ints, pos, flips = [], 0, 0
    for p, (h, w, lo) in zip(planes_ref, sizes):
        n = p.size
        g = (recon[pos:pos + n] * np.float32(norm)).reshape(p.shape)[:h, :w]
        pos += n
        o = np.asarray(p, np.float64)[:h, :w].astype(np.float32)
        qg = np.clip(_roundf(g), lo, 255)
        qo = np.clip(_roundf(o), lo, 255)
        d = qg != qo
        if d.any():
            assert np.abs(qg - qo)[d].max() == 1, "a plane sample rounded to a code two apart"
            far = _tie_distance(o)[d].max()
            assert far < bar, "a plane sample %.3g from a rounding tie rounded differently" % far
            flips += int(d.sum())
        ints.append(qg.astype(np.int16))
    y, co, cg = ints
    co_up = O.chroma_up(co, height, width)
    cg_up = O.chroma_up(cg, height, width)
    want = O.ycocg8_inverse(y, co_up, cg_up) if storage8 else O.ycocgr_inverse(y, co_up, cg_up)
    assert rgb.shape == want.shape, (rgb.shape, want.shape)
    assert np.array_equal(rgb, want), "RGB differs from the output stage applied to the GPU's own planes"
    return flips


def check_scaled_decode(codec, rgb, oracle_codec, stream, scale, storage8=False):
    """Decode `stream` in the oracle at `scale` (advancing its decoder) and check the GPU codec's output
    `rgb` of the same frame against it: the lowpass band itself (scale = levels) is exact on both sides;
    other scales go through check_decode with the GPU codec's reconstructed planes."""
    want, planes_ref = oracle_codec.decode(np.asarray(stream), want_planes=True, scale=scale)
    rgb = np.asarray(rgb)
    if scale == codec.levels:
        assert np.array_equal(rgb, want)
        return 0
    f = 1 << scale
    return check_decode(rgb, codec.inspect(2).cpu().numpy(), planes_ref, rgb.shape[0], rgb.shape[1],
                        (codec.Hc + f - 1) // f, (codec.Wc + f - 1) // f, storage8=storage8, norm=2.0 ** -scale)
