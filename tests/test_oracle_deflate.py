"""Pins of the oracle's DEFLATE side (§3.9):
  - the optimal prefix-code cost equals a brute-force minimum over every
    set of code lengths that satisfies Kraft's inequality (small alphabets),
    and known small cases;
  - the container inflater rebuilds a frame from per-component streams that
    zlib wrote (any DEFLATE strategy), and from the one stream of a CVC-NTS
    container, and refuses broken ones.
"""
import itertools
import zlib

import numpy as np
import pytest

import oracle as O
from paper_1510_00561_b300 import synthetic as S


def _brute(freq):
    f = [x for x in freq if x]
    if len(f) == 1:
        return f[0]
    best = None
    for lens in itertools.product(range(1, len(f)), repeat=len(f)):
        if sum(2.0 ** -l for l in lens) <= 1.0:
            c = sum(a * b for a, b in zip(f, lens))
            best = c if best is None else min(best, c)
    return best


def test_huffman_cost_is_the_optimal_prefix_code():
    rng = np.random.default_rng(0)
    assert O.huffman_cost([1, 1, 2, 4])[0] == 14          # lengths 3, 3, 2, 1
    assert O.huffman_cost([5, 0, 0])[0] == 5
    assert O.huffman_cost([3, 3, 3, 3])[0] == 24
    for n in (2, 3, 4, 5, 6):
        for _ in range(8):
            f = rng.integers(0, 20, n)
            if (f > 0).sum() == 0:
                continue
            assert O.huffman_cost(f)[0] == _brute(list(f)), f
    # Fibonacci weights give the deepest tree: n - 1 levels
    fib = [1, 1, 2, 3, 5, 8, 13, 21, 34, 55]
    assert O.huffman_cost(fib)[1] == len(fib) - 1


def _container(frame, ncomp, strategy, nts=False):
    hdr = 32 + 4 * ncomp
    counts = np.frombuffer(bytes(frame[32:hdr]), "<u4")
    toks, pos = [], hdr
    for n in counts:
        toks.append(bytes(frame[pos:pos + 2 * int(n)]))
        pos += 2 * int(n)
    if nts:                                             # CVC-NTS: one stream over all token bytes
        toks = [b"".join(toks)]
    streams, nseg = [], 0
    for tok in toks:
        nseg += (len(tok) + 255) // 256
        if tok:
            z = zlib.compressobj(6, zlib.DEFLATED, -15, 8, strategy)
            streams.append(z.compress(tok) + z.flush())
        else:
            streams.append(b"")
    tail = bytes(frame[pos:])
    head = bytearray(frame[:hdr])
    head[4] = 3 if nts else 2
    lens = np.array([len(s) for s in streams], "<u4").tobytes()
    seg = bytes(((2 * nseg + 3) // 4) * 4)
    return np.frombuffer(bytes(head) + lens + seg + b"".join(streams) + tail, np.uint8)


@pytest.mark.parametrize("nts", [False, True], ids=["scalable", "nts"])
@pytest.mark.parametrize("strategy", [zlib.Z_DEFAULT_STRATEGY, zlib.Z_HUFFMAN_ONLY, zlib.Z_FIXED])
def test_container_inflate_rebuilds_the_frame(strategy, nts):
    w, h = 176, 144
    kw = dict(width=w, height=h, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4, motion_range=8)
    c = O.Codec(**kw)
    frames = S.SyntheticVideo(S.spec_for(w, h, seed=1)).frames(2)
    for f in frames:                                     # a K-frame, then a P-frame with vectors
        s, _ = c.encode(f)
        for d in (0, 2):
            x = c.drop_levels(s, d)
            box = _container(x, c.ncomp, strategy, nts)
            assert np.array_equal(c.inflate_container(box), x)
    other = box.copy()
    other[4] = 2 if nts else 3                           # the other container form: the tables disagree
    with pytest.raises(RuntimeError, match="status 5"):
        c.inflate_container(other)
    bad = box.copy()
    bad[32 + 4 * c.ncomp] += 1                           # the first stream's length
    with pytest.raises(RuntimeError, match="status 5"):
        c.inflate_container(bad)
    with pytest.raises(RuntimeError, match="status 5"):
        c.inflate_container(box[:-3])
