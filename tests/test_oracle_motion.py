"""Pins of the oracle's motion estimation and motion-compensated P-frames
(§3.2, §3.7), against things other than the oracle's own code:

  - the search is the full-search argmin by definition (numpy enumeration of
    every candidate on small planes, including the tie rules);
  - a translated texture gives back its translation;
  - static content gives zero vectors and the tokens of zero-motion coding;
  - a global translation by a multiple of 2^L makes every LP component's
    prediction exact away from the borders (the vector mapping to each
    component's scale);
  - the element size (ey, ex) of every component kind, both directional
    families included, and the rounding of the scaled vectors, against a
    hand-worked table (a swapped (ey, ex) for the transposed family or a
    truncating shift fails it);
  - a periodic translation by a multiple of the pyramid modulus makes the
    residual of every component exactly zero wherever its block found the
    translation, directional subbands included (8/4/4 and 32/16/16/8/8);
  - streams with motion survive level dropping and scaled decoding.
"""
import numpy as np
import pytest

import oracle as O
from paper_1510_00561_b300 import synthetic as S


def _brute(cur, prev, R):
    H, W = cur.shape
    out = np.zeros(((H + 15) // 16, (W + 15) // 16, 2), np.int8)
    c64, p64 = cur.astype(np.int64), prev.astype(np.int64)
    for by in range(out.shape[0]):
        for bx in range(out.shape[1]):
            y0, x0 = 16 * by, 16 * bx
            bh, bw = min(16, H - y0), min(16, W - x0)
            best = None
            for dy in range(-R, R + 1):
                for dx in range(-R, R + 1):
                    if y0 + dy < 0 or y0 + dy + bh > H or x0 + dx < 0 or x0 + dx + bw > W:
                        continue
                    d = c64[y0:y0 + bh, x0:x0 + bw] - p64[y0 + dy:y0 + dy + bh, x0 + dx:x0 + dx + bw]
                    key = (int((d * d).sum()), abs(dy) + abs(dx))      # raster order breaks the rest
                    if best is None or key < best[0]:
                        best = (key, dy, dx)
            out[by, bx] = best[1], best[2]
    return out


def test_search_is_the_full_search_argmin():
    rng = np.random.default_rng(0)
    for H, W, R in ((40, 36, 3), (32, 48, 2), (17, 21, 4)):
        cur = rng.integers(0, 256, (H, W), dtype=np.uint8)
        prev = np.clip(cur.astype(int) + rng.integers(-20, 21, (H, W)), 0, 255).astype(np.uint8)
        prev = np.roll(prev, (1, -2), axis=(0, 1))
        assert np.array_equal(O.motion_search(cur, prev, R), _brute(cur, prev, R))
        # coarse values give many equal sums: the tie rules decide
        cur4, prev4 = cur // 64, prev // 64
        assert np.array_equal(O.motion_search(cur4, prev4, R), _brute(cur4, prev4, R))


def test_tie_rules():
    H, W = 48, 48
    # constant planes: every candidate ties, the zero vector wins
    assert not O.motion_search(np.full((H, W), 9, np.uint8), np.full((H, W), 9, np.uint8), 4).any()
    # rows alternating a / b, the current frame shifted by one row: every odd dy matches
    # exactly; of the two with |dy| + |dx| = 1 the first in raster order (dy = -1) wins
    prev = np.where(np.arange(H)[:, None] % 2 == 0, 40, 200).astype(np.uint8).repeat(W, axis=1)
    cur = np.roll(prev, -1, axis=0)
    mv = O.motion_search(cur, prev, 3)
    assert (mv[1:-1, :, 0] == -1).all() and (mv[..., 1] == 0).all()


def test_translated_texture_gives_back_its_translation():
    rng = np.random.default_rng(1)
    big = rng.integers(0, 256, (120, 140), dtype=np.uint8)
    H, W, dy, dx = 64, 80, 3, -2
    cur = big[20:20 + H, 30:30 + W]
    prev = big[20 + dy:20 + dy + H, 30 + dx:30 + dx + W]
    mv = O.motion_search(cur, prev, 4)
    # cur(y, x) = prev(y - dy, x - dx): every block whose displaced block fits finds (-dy, -dx)
    for by in range(mv.shape[0]):
        for bx in range(mv.shape[1]):
            y0, x0 = 16 * by, 16 * bx
            if 0 <= y0 - dy and y0 - dy + 16 <= H and 0 <= x0 - dx and x0 - dx + 16 <= W:
                assert tuple(mv[by, bx]) == (-dy, -dx)


def _frame_of(bigs, y, x, h, w):
    return np.stack([b[y:y + h, x:x + w] for b in bigs], axis=2).astype(np.uint8)


def _components(stream, c, lays):
    """(plane, layout subband, residual codes) of every component of a P-frame"""
    counts = np.frombuffer(bytes(stream[32:32 + 4 * c.ncomp]), "<u4")
    tok = np.frombuffer(bytes(stream[32 + 4 * c.ncomp:32 + 4 * c.ncomp + 2 * int(counts.sum())]), "<i2")
    out, t, j = [], 0, 0
    for p, lay in enumerate(lays):
        for sb in lay["subbands"]:
            n = int(counts[j])
            out.append((p, sb, O.rle_expand(tok[t:t + n], sb["h"] * sb["w"]).reshape(sb["h"], sb["w"])))
            t += n
            j += 1
    return out


def test_global_translation_is_predicted_exactly_away_from_the_borders():
    """An LP-only pyramid (no directional stages), L = 3: a texture moved by
    (-16, +16) pixels, so that cur(y, x) = prev(y + 16, x - 16), a whole number
    of elements in every component.  Each component's element covers
    2^ey x 2^ex luma samples (chroma one level more), the vector (16, -16)
    scales to (16 / 2^ey, -16 / 2^ex) elements, and the residual of
    every component is exactly zero wherever the element and its source lie
    away from the frame borders (by the pyramid's reach) and the block's
    search found the translation (not the left block column or the bottom
    block row, whose displaced blocks would leave the plane)."""
    rng = np.random.default_rng(2)
    bigs = []
    for _ in range(3):
        b = rng.integers(0, 256, (400, 460))
        bigs.append(((b + np.roll(b, 1, 0) + np.roll(b, 1, 1)) // 3).astype(np.uint8))
    H, W = 288, 352
    kw = dict(width=W, height=H, levels=3, dirs_log2=[0, 0, 0], qph=4, qpl=1, key_interval=8)
    c = O.Codec(**kw, motion_range=16)
    c.encode(_frame_of(bigs, 40, 40, H, W))
    s, ft = c.encode(_frame_of(bigs, 56, 24, H, W))
    assert ft == 2 and (c.Hp, c.Wp) == (H, W)
    nby, nbx = H // 16, W // 16
    mv = np.frombuffer(bytes(s[-2 * nby * nbx:]), np.int8).reshape(nby, nbx, 2)
    assert (mv[:-2, 1:] == (16, -16)).all()
    lays = [O.layout(c.Hp, c.Wp, 3, [0, 0, 0])] + [O.layout(c.Hcp, c.Wcp, 3, [0, 0, 0])] * 2
    for p, sb, r in _components(s, c, lays):
        reach = 40 * (1 + (p > 0))               # the 3-level 9/7 pyramid's footprint, in luma samples
        y0, y1, x0, x1 = reach, H - 32 - reach, 16 + reach, W - reach
        ey = int(np.log2((c.Hp if p == 0 else c.Hcp) / sb["h"])) + (p > 0)
        ex = int(np.log2((c.Wp if p == 0 else c.Wcp) / sb["w"])) + (p > 0)
        inner = r[-(-y0 >> ey):y1 >> ey, -(-x0 >> ex):x1 >> ex]
        assert inner.size > 0 and not inner.any(), (p, sb["level"], sb["kind"])
    zero = O.Codec(**kw)
    zero.encode(_frame_of(bigs, 40, 40, H, W))
    s0, _ = zero.encode(_frame_of(bigs, 56, 24, H, W))
    assert s.size < s0.size / 2


def test_static_video_gives_zero_vectors_and_the_zero_motion_tokens():
    w, h = 176, 144
    f = S.SyntheticVideo(S.spec_for(w, h, seed=3)).frame(0)
    kw = dict(width=w, height=h, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=8)
    m, z = O.Codec(**kw, motion_range=8), O.Codec(**kw)
    for t in range(3):
        sm, ftm = m.encode(f)
        sz, ftz = z.encode(f)
        if t == 0:
            assert ftm == ftz == 0 and np.array_equal(sm, sz)
            continue
        assert ftm == 2 and ftz == 1
        nmv = ((m.Hp + 15) // 16) * ((m.Wp + 15) // 16)
        assert sm.size == sz.size + 2 * nmv and not sm[sz.size:].any()
        assert np.array_equal(sm[7:sz.size], sz[7:]) and np.array_equal(sm[:6], sz[:6])


@pytest.mark.parametrize("w,h,L,k", [(176, 144, 3, [3, 2, 2]), (99, 77, 2, [2, 0])])
def test_motion_streams_decode_drop_and_scale(w, h, L, k):
    frames = S.SyntheticVideo(S.spec_for(w, h, seed=4)).frames(5)
    kw = dict(width=w, height=h, levels=L, dirs_log2=k, qph=8, qpl=1, key_interval=4)
    enc, zero = O.Codec(**kw, motion_range=8), O.Codec(**kw)
    seq = [enc.encode(f) for f in frames]
    assert [t for _, t in seq] == [0, 2, 2, 2, 0]
    seq = [s for s, _ in seq]
    zseq = [zero.encode(f)[0] for f in frames]
    dec, zdec = O.Codec(**kw, motion_range=8), O.Codec(**kw)
    for f, s, zs in zip(frames, seq, zseq):
        a, b = dec.decode(s), zdec.decode(zs)
        # same quantisers, a different predictor: the reconstructions are equally close
        pa = np.mean((a.astype(float) - f) ** 2)
        pb = np.mean((b.astype(float) - f) ** 2)
        assert abs(10 * np.log10(pa / pb)) < 0.5
    # dropped levels keep the vectors; every scale at or above the drop is unchanged
    for d in range(1, L + 1):
        dropped = [enc.drop_levels(s, d) for s in seq]
        for sc in range(d, L + 1):
            full, part = O.Codec(**kw, motion_range=8), O.Codec(**kw, motion_range=8)
            for s, x in zip(seq, dropped):
                assert np.array_equal(full.decode(s, scale=sc), part.decode(x, scale=sc))


def test_motion_stream_refusals():
    w, h = 99, 77
    kw = dict(width=w, height=h, levels=2, dirs_log2=[2, 2], qph=8, qpl=1, key_interval=4)
    frames = S.SyntheticVideo(S.spec_for(w, h, seed=5)).frames(2)
    enc = O.Codec(**kw, motion_range=4)
    s0, _ = enc.encode(frames[0])
    s1, t1 = enc.encode(frames[1])
    assert t1 == 2
    z = O.Codec(**kw)
    z.decode(s0)
    with pytest.raises(RuntimeError, match="status 5"):
        z.decode(s1)                                   # a decoder without motion
    d = O.Codec(**kw, motion_range=4)
    d.decode(s0)
    bad = s1.copy()
    bad[-1] = 5                                       # a vector beyond the range
    with pytest.raises(RuntimeError, match="status 5"):
        d.decode(bad)
    with pytest.raises(RuntimeError, match="status 5"):
        d.decode(s1[:-1])                              # truncated vector field
    d.decode(s1)
    with pytest.raises(ValueError):
        O.Codec(**kw, motion_range=65)


# Element size of every component of a 176 x 144 frame with 3 levels and 8/4/4
# directions, worked out by hand from the layout (§2.1: level j of a plane is
# (H >> (j-1)) x (W >> (j-1)); with k stages, directions d < 2^(k-1) are
# (h >> (k-1)) x (w / 2) and the others (h / 2) x (w >> (k-1)); chroma planes
# are half size): (luma rows, luma columns) per element, as powers of two.
QCIF_ELEMENT = {
    # plane 0 (luma 144 x 176)
    (0, 0, "low"): (3, 3),        # 18 x 22
    (0, 1, "c"): (2, 1),          # 36 x 88
    (0, 1, "r"): (1, 2),          # 72 x 44
    (0, 2, "c"): (2, 2),          # 36 x 44
    (0, 2, "r"): (2, 2),          # 36 x 44
    (0, 3, "c"): (3, 3),          # 18 x 22
    (0, 3, "r"): (3, 3),          # 18 x 22
    # planes 1, 2 (chroma 72 x 88): one element of a 72 x 88 plane is 2 x 2 luma samples
    (1, 0, "low"): (4, 4),        # 9 x 11
    (1, 1, "c"): (3, 2),          # 18 x 44
    (1, 1, "r"): (2, 3),          # 36 x 22
    (1, 2, "c"): (3, 3),          # 18 x 22
    (1, 2, "r"): (3, 3),
    (1, 3, "c"): (4, 4),          # 9 x 11
    (1, 3, "r"): (4, 4),
}

# v / 2^e rounded half away from zero, written out for v = -8 .. 8
ROUNDED = {
    0: list(range(-8, 9)),
    1: [-4, -4, -3, -3, -2, -2, -1, -1, 0, 1, 1, 2, 2, 3, 3, 4, 4],
    2: [-2, -2, -2, -1, -1, -1, -1, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2],
    3: [-1, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1],
    4: [-1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1],
}


def test_prediction_of_every_component_kind_against_a_hand_worked_table():
    """§3.7 maps the block vectors "to the corresponding scale and range" of each
    component.  A K-frame whose codes are distinct within each component, then a
    P-frame of zero coefficients whose luma moves every 16 x 16 block by its own
    vector (odd and even values in -8..8, so that halving rounds): the P-frame's
    residual is minus the prediction, which must read, for element (i, k), the
    previous code at (i + rnd(dy / 2^ey), k + rnd(dx / 2^ex)) clamped, with (ey, ex)
    from the table above (transposed between the two directional families) and the
    rounding of the table ROUNDED; (dy, dx) is the vector of the block holding the
    element's first luma sample."""
    H, W, L, k = 144, 176, 3, [3, 2, 2]
    c = O.Codec(W, H, L, k, 1, 1, 0.0, 100, motion_range=8)
    lays = [O.layout(H, W, L, k)] + [O.layout(H // 2, W // 2, L, k)] * 2
    # K-frame: codes 1 + (index within the component); the lowpass carries the 2^-L normalisation
    coef = np.zeros(c.ncoef, np.float32)
    prev_codes, pos = [], 0
    for lay in lays:
        for sb in lay["subbands"]:
            n = sb["h"] * sb["w"]
            q = (1 + np.arange(n)).reshape(sb["h"], sb["w"])
            coef[pos:pos + n] = (q * (2 ** L if sb["kind"] == 0 else 1)).ravel()
            prev_codes.append(q)
            pos += n
    rng = np.random.default_rng(7)
    tex = rng.integers(0, 256, (H, W), dtype=np.uint8)
    s0, ft0 = c.encode_from_coeffs(coef, luma=tex)
    assert ft0 == 0
    # P-frame luma: block (by, bx) shows the texture displaced by its vector
    nby, nbx = H // 16, W // 16
    vec = np.zeros((nby, nbx, 2), np.int64)
    cur = np.zeros_like(tex)
    for by in range(nby):
        for bx in range(nbx):
            y0, x0 = 16 * by, 16 * bx
            dy, dx = (3 * by + 5 * bx) % 17 - 8, (7 * by + 2 * bx + 4) % 17 - 8
            if not 0 <= y0 + dy <= H - 16:
                dy = -dy
            if not 0 <= x0 + dx <= W - 16:
                dx = -dx
            vec[by, bx] = dy, dx
            cur[y0:y0 + 16, x0:x0 + 16] = tex[y0 + dy:y0 + dy + 16, x0 + dx:x0 + dx + 16]
    assert len(set(vec[..., 0].ravel())) == 17 and len(set(vec[..., 1].ravel())) == 17
    s1, ft1 = c.encode_from_coeffs(np.zeros(c.ncoef, np.float32), luma=cur)
    assert ft1 == 2
    mv = np.frombuffer(bytes(s1[-2 * nby * nbx:]), np.int8).reshape(nby, nbx, 2)
    assert np.array_equal(mv, vec)                      # the search finds the designed vectors
    for (p, sb, r), q in zip(_components(s1, c, lays), prev_codes):
        kind = "low" if sb["kind"] == 0 else ("c" if sb["kind"] == 1 or sb["dir"] < (1 << k[sb["level"] - 1]) // 2
                                              else "r")
        ey, ex = QCIF_ELEMENT[(min(p, 1), sb["level"], kind)]
        h, w = sb["h"], sb["w"]
        want = np.zeros((h, w), np.int64)
        for i in range(h):
            for kk in range(w):
                by, bx = min((i << ey) >> 4, nby - 1), min((kk << ex) >> 4, nbx - 1)
                dy, dx = vec[by, bx]
                si = min(max(i + ROUNDED[ey][dy + 8], 0), h - 1)
                sk = min(max(kk + ROUNDED[ex][dx + 8], 0), w - 1)
                want[i, kk] = q[si, sk]
        assert np.array_equal(-r.astype(np.int64), want), (p, sb["level"], kind)


@pytest.mark.parametrize("W,H,L,k,shift", [(176, 144, 3, [3, 2, 2], 16), (256, 256, 5, [5, 4, 4, 3, 3], 64)],
                         ids=["qcif_8-4-4", "256_32-16-16-8-8"])
def test_periodic_translation_is_predicted_exactly_in_every_directional_subband(W, H, L, k, shift):
    """A frame and its periodic translation by a multiple of the pyramid modulus (8 for
    8/4/4, 64 for 32/16/16/8/8): with periodic extension every stage of the LP and the
    DFB commutes with that translation, so every component whose element spans a divisor
    of the shift in luma samples (all of them at 8/4/4; at 32/16/16/8/8 all but the
    coarsest chroma subbands, whose elements span 128) is the previous one moved by
    (shift / 2^ey, -shift / 2^ex) elements, directional subbands of both families
    included.  The P-frame residual must then be exactly zero wherever the element's
    block found the translation and its source lies inside the component."""
    rng = np.random.default_rng(11)
    prev = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    cur = np.roll(prev, (-shift, shift), axis=(0, 1))           # cur(y, x) = prev(y + shift, x - shift)
    c = O.Codec(W, H, L, k, 4, 1, 0.0, 100, motion_range=shift)
    assert (c.Hp, c.Wp) == (H, W)
    c.encode(prev)
    s, ft = c.encode(cur)
    assert ft == 2
    nby, nbx = H // 16, W // 16
    mv = np.frombuffer(bytes(s[-2 * nby * nbx:]), np.int8).reshape(nby, nbx, 2)
    good = (mv[..., 0] == shift) & (mv[..., 1] == -shift)
    assert good[:nby - shift // 16 - 1, shift // 16:].all()
    lays = [O.layout(H, W, L, k)] + [O.layout(H // 2, W // 2, L, k)] * 2
    checked = set()
    for p, sb, r in _components(s, c, lays):
        ph, pw = (H, W) if p == 0 else (H // 2, W // 2)
        ey = int(np.log2(ph / sb["h"])) + (p > 0)               # luma samples per element, as powers of two
        ex = int(np.log2(pw / sb["w"])) + (p > 0)
        if shift % (1 << ey) or shift % (1 << ex):
            assert p > 0 and sb["level"] == L                   # only the coarsest chroma subbands
            continue
        sy, sx = shift >> ey, -(shift >> ex)
        i = np.arange(sb["h"])[:, None]
        kk = np.arange(sb["w"])[None, :]
        blk = good[np.minimum((i << ey) >> 4, nby - 1), np.minimum((kk << ex) >> 4, nbx - 1)]
        inside = (i + sy < sb["h"]) & (kk + sx >= 0)
        region = blk & inside
        assert region.any(), (p, sb["level"], sb["dir"])
        assert not r[region].any(), (p, sb["level"], sb["dir"], int(np.count_nonzero(r[region])))
        checked.add((p > 0, sb["kind"]))
    assert {(False, 0), (False, 1), (False, 2), (True, 1), (True, 2)} <= checked
