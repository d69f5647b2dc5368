"""CPU checks of the index arithmetic of the tiled row-split DFB stage and the
tiled RLE (tests/tile_models.py restates their indexing): in bounds, every
output once, and equal to the plain definitions -- the row-split stencil of
the plan emulator (§2.1) and a row-by-row run-length coder (§3.8)."""
import itertools

import numpy as np
import pytest

from plan_emulator import _rowsplit_stencil
from tile_models import geometry, passes, rle_tile, row_split_stage

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
