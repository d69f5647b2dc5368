"""CPU checks of the index arithmetic of the tiled row-split DFB stage, the
tiled RLE and the single-precision LP level tile (tests/tile_models.py
restates their indexing): in bounds, every output once, and equal to the plain
definitions -- the row-split stencil of the plan emulator (§2.1), a row-by-row
run-length coder (§3.8) and the periodic down / up filtering of one pyramid
level (§2.1, Fig. 1)."""
import itertools

import numpy as np
import pytest

from plan_emulator import _down, _rowsplit_stencil, _up
from tile_models import geometry, lp_level_tile, passes, rle_tile, row_split_stage

# (R2, C, slope index i): ragged and periodic-wrapping arrays, arrays narrower than one
# staged window, negative slopes (the tree's first channels), long shears
STAGES = [(17, 30, 0), (20, 125, 3), (33, 250, 5), (3, 7, 2), (18, 44, -1), (20, 130, -3)]


def _plain(E, O, i, NT, fo, alphas):
    a1, g1, a2, g2 = alphas
    E, O = E.copy(), O.copy()
    if fo:
        O = a1 * O + g1 * _rowsplit_stencil(E, i, True, NT)
        E = a2 * E + g2 * _rowsplit_stencil(O, i, False, NT)
    else:
        E = a1 * E + g1 * _rowsplit_stencil(O, i, False, NT)
        O = a2 * O + g2 * _rowsplit_stencil(E, i, True, NT)
    return E, O


@pytest.mark.parametrize("NT", [4, 6, 8])
def test_row_split_frame_and_quads(NT):
    """the straightened frame, quads and both staging / store paths compute the stage; first target
    coset odd (forward) and even (inverse), four and eight working warps"""
    g = geometry(NT)
    assert g["COLS"] % 4 == 0 and g["COLS"] + 2 * g["R"] <= g["CB"]
    rng = np.random.default_rng(NT)
    for k, ((R2, C, i), fo) in enumerate(itertools.product(STAGES, (0, 1))):
        P = passes(NT, fo)
        assert max(P["NQ1"], P["NQ2"]) <= 32
        E, O = rng.standard_normal((R2, C)), rng.standard_normal((R2, C))
        alphas = (0.5, -0.5, 1.0, 1.0) if fo else (1.0, -1.0, 2.0, 1.0)
        tin, tout, nw = k % 2, (k // 2) % 2, (4, 8)[(k // 3) % 2]
        Eg, Og = row_split_stage(E, O, i, NT, fo, alphas, tin, tout, nw)
        Er, Or = _plain(E, O, i, NT, fo, alphas)
        assert np.isfinite(Eg).all() and np.isfinite(Og).all()
        assert max(np.abs(Eg - Er).max(), np.abs(Og - Or).max()) < 1e-12, (R2, C, i, fo, tin, tout, nw)


def _rle_rows(codes, w):
    out = []
    for r0 in range(0, len(codes), w):
        row, x = codes[r0:r0 + w], 0
        while x < len(row):
            if row[x] != 0:
                out.append(int(row[x]))
                x += 1
            else:
                n = 0
                while x < len(row) and row[x] == 0:
                    n, x = n + 1, x + 1
                out += [0, n]
    return out


def test_rle_tiles():
    """tiles of every row width class (narrower than a chunk, chunk-sized, longer than a block's
    pass), unaligned starts, sparse and dense codes, all-zero tiles"""
    rng = np.random.default_rng(0)
    for trial in range(60):
        w = int(rng.choice([1, 3, 7, 8, 9, 30, 60, 120, 960, 3000]))
        rows = int(rng.integers(1, max(2, 4096 // w + 1)))
        pre = int(rng.integers(0, 16))
        res = np.zeros(pre + w * rows + 16, np.int16)
        dens = rng.choice([0.02, 0.3, 0.9])
        if trial % 6:
            live = rng.random(res.size) < dens
            res[live] = rng.integers(-50, 50, int(live.sum()))
        assert rle_tile(res, pre, w * rows, w) == _rle_rows(res[pre:pre + w * rows], w), (w, rows, pre)


def _dc_taps(rng, n, phases):
    """random asymmetric taps (a mirrored index fails the check) with the 9/7 pair's DC gains, which
    the tile's centring relies on: sum sqrt(2) for the decimating filter, 1/sqrt(2) per phase for the
    expanding one"""
    f = rng.uniform(0.2, 1.0, n)
    for p in range(phases):
        f[p::phases] *= (np.sqrt(2) / phases) / f[p::phases].sum()
    return f


@pytest.mark.parametrize("RA, RS, syn", [(4, 3, False), (4, 3, True), (3, 4, False)])
def test_lp_level_tile(RA, RS, syn):
    """the forward level's geometry (9 analysis taps, 7 synthesis taps), its synthesis and the
    adjoint's (7, 9) on corner and interior tiles of a 192 x 128 periodic image with pixel-scale
    values, against the whole-image definitions c = down(x), d = x - up(c) and
    x = d + up(c - down(d))"""
    rng = np.random.default_rng(RA * 10 + syn)
    fa, fs = _dc_taps(rng, 2 * RA + 1, 1), _dc_taps(rng, 2 * RS + 1, 2)
    H, W = 192, 128
    main = rng.integers(0, 256, (H, W)).astype(np.float64) if not syn else rng.standard_normal((H, W))
    cin = 500 * rng.random((H // 2, W // 2)) if syn else None
    lo = 1e-6 * rng.standard_normal((H // 2, W // 2)) if syn else None
    if syn:
        want_out = main + _up(cin + lo - _down(main, fa), fs)
    else:
        want_c = _down(main, fa)
        want_out = main - _up(want_c, fs)
    for ty, tx in ((0, 0), (1, 1), (2, 1)):
        out, cout = lp_level_tile(RA, RS, syn, fa, fs, main, ty, tx, cin, lo)
        ys, xs = slice(64 * ty, 64 * ty + 64), slice(64 * tx, 64 * tx + 64)
        assert np.abs(out - want_out[ys, xs]).max() < 1e-9, (ty, tx)
        if not syn:
            cs, cx = slice(32 * ty, 32 * ty + 32), slice(32 * tx, 32 * tx + 32)
            assert np.abs(cout - want_c[cs, cx]).max() < 1e-9, (ty, tx)
