"""Host-side reading of libcvc's launch plans (test helper, no GPU).

``cvc_debug_plan_tables`` dumps the job tables the CUDA kernels execute.  This
module parses them, checks that every element a job reads or writes lies
inside its buffer and that no job of a launch writes what another job of the
same launch touches, and executes the tables in double precision with the
semantics of the two kernels:

  LP level job (analysis):   cout = down(main, fa);       out = main - up(cout, fs)
  LP level job (synthesis):  v = cin - down(main, fa);    out = main + up(v, fs)
  DFB lifting job:           out(u,v) = alpha tin(u,v) + gamma sum_t w_t src_sel(u+dr, v+dc)  (periodic)

  DFB stages 1+2 job:        the fan filter bank stages 1 (and 2) on the
                             whole periodic detail image, whose polyphase
                             classes are the stage-2 channels (comp[q])
  DFB row-split job:         one stage s >= 3 of a channel: even / odd rows
                             E, O of its array, stencil row offset (a +- 1)/2,
                             column offset -i*a + (b-a)/2 (periodic)
  plain DFB pass (longer     one lifting pass of stage s over a whole detail
  prototypes), two launches: image: the samples of the target parity in their
                             stage-s channel, the n x n stencil of the n-tap
                             fan taps (from the Lagrange formula) in the
                             channel's lattice basis (periodic), split as the
                             kernels split it: the first launch leaves the
                             diagonal sums S[p] = sum_u bt[2u-1] x[p + u (B1 -
                             B2)] at the other parity in the spare buffer T,
                             the second sums bt[a] S[t + ((a-1)/2) B1 +
                             ((a+1)/2) B2] at the targets
  plain DFB copy:            the detail image to / from the level's subbands

so that a test can compare the planned computation with the oracle before
any kernel runs on a GPU.  Each pass sets target = alpha*target + gamma*sum.
"""
import ctypes

import numpy as np

import oracle as O
from paper_1510_00561_b300 import _lib as L

VIEW = np.dtype([("off", "<i8"), ("b", "<i4"), ("rs", "<i4"), ("cs", "<i4"), ("pad", "<i4")])
LPJOB = np.dtype([("main", VIEW), ("cin", VIEW), ("cout", VIEW), ("out", VIEW), ("H", "<i4"), ("W", "<i4"),
                  ("tiles_x", "<i4"), ("first_block", "<i4")])
AJOB = np.dtype([("D", VIEW), ("comp", VIEW, (4,)), ("H", "<i4"), ("W", "<i4"), ("nst", "<i4"),
                 ("tiles_x", "<i4"), ("first_block", "<i4"), ("pad", "<i4")])
BJOB = np.dtype([("pe", VIEW), ("po", VIEW), ("c0", VIEW), ("c1", VIEW), ("R2", "<i4"), ("C", "<i4"),
                 ("i", "<i4"), ("tiles_x", "<i4"), ("first_block", "<i4"), ("pad", "<i4")])
GJOB = np.dtype([("D", VIEW), ("T", VIEW), ("slot0", "<i8"), ("H", "<i4"), ("W", "<i4"), ("k", "<i4"), ("ntaps", "<i4"),
                 ("first_block", "<i4"), ("pad", "<i4")])
BT = np.array([-1.0, -9.0, 9.0, 1.0]) / 16
A4 = [-3, -1, 1, 3]
# (first target is the odd coset, alpha1, gamma1, alpha2, gamma2) per mode
PASSES = {0: (1, 0.5, -0.5, 1.0, 1.0), 3: (0, 1.0, 1.0, 2.0, -1.0),
          1: (0, 1.0, -1.0, 2.0, 1.0), 2: (1, 0.5, 0.5, 1.0, -1.0)}


# decoder output stage of one stream at one pyramid scale
SCALEDESC = np.dtype([("H", "<i4"), ("W", "<i4"), ("Hc", "<i4"), ("Wc", "<i4"), ("rs_y", "<i4"), ("rs_c", "<i4"),
                      ("src", "<i4"), ("blk0", "<i4"), ("off", "<i8", (3,)), ("norm", "<f4"), ("pad", "<i4")])


def _dump(call):
    used = ctypes.c_size_t(0)
    st = call(None, 0, ctypes.byref(used))
    assert st == 3, st
    buf = (ctypes.c_uint8 * used.value)()
    st = call(buf, used.value, ctypes.byref(used))
    assert st == 0, st
    return bytes(buf)


def tables(mode, params=None, h=0, w=0, levels=0, dirs=(), batch=1):
    lib = L.lib()
    pp = ctypes.byref(params) if params is not None else None
    raw = _dump(lambda buf, cap, used: lib.cvc_debug_plan_tables(pp, h, w, levels, L.ints(dirs), batch, mode,
                                                                 buf, cap, used))
    elems, launches, tail = _parse(raw)
    assert len(tail) == 0
    return elems, launches


def scale_tables(params, n, scale):
    """(elems, inverse launches, output records) of the decoder at pyramid scale `scale`."""
    lib = L.lib()
    raw = _dump(lambda buf, cap, used: lib.cvc_debug_scale_tables(params, n, scale, buf, cap, used))
    elems, launches, tail = _parse(raw)
    return elems, launches, np.frombuffer(tail, SCALEDESC)


def _parse(raw):
    magic, nl, lpb, ab, bb, tail_sz, gb = np.frombuffer(raw[:28], "<u4")
    assert tail_sz in (0, SCALEDESC.itemsize)
    assert magic == 0x43564350 and lpb == LPJOB.itemsize and ab == AJOB.itemsize and bb == BJOB.itemsize
    assert gb == GJOB.itemsize
    elems = np.frombuffer(raw[28:60], "<u8").astype(np.int64)
    pos = 60
    launches = []
    for _ in range(nl):
        kind, nj = np.frombuffer(raw[pos:pos + 8], "<u4")
        pos += 8
        extra = None
        if kind >= 3:
            st, tgt = np.frombuffer(raw[pos:pos + 8], "<u4")
            al, ga = np.frombuffer(raw[pos + 8:pos + 16], "<f4")
            extra = (int(st), int(tgt), float(al), float(ga))
            pos += 16
        dt = (LPJOB, AJOB, BJOB, GJOB, GJOB, GJOB)[kind]
        jobs = np.frombuffer(raw[pos:pos + nj * dt.itemsize], dt)
        pos += nj * dt.itemsize
        launches.append((int(kind), jobs, extra))
    return elems, launches, raw[pos:]


def _fan_taps(n):
    """fan taps of the n-tap Lagrange half-band prototype: weight of the sample at odd a
    when interpolating at 0, times (-1)^((a - 1) / 2)"""
    pts = list(range(-(n - 1), n, 2))
    out = []
    for a in pts:
        w = np.prod([b / (b - a) for b in pts if b != a])
        out.append((a, (-1.0) ** (((a - 1) // 2) % 2) * w))
    return out


def _g_basis(s, T, i):
    if s == 1:
        return np.ones_like(i), np.zeros_like(i), np.zeros_like(i), np.ones_like(i)
    if s == 2:
        one = np.ones_like(i)
        return one, one, np.where(T == 0, 1, -1), np.where(T == 0, -1, 1)
    q = 2 ** (s - 2)
    c = T == 0
    return (np.where(c, q, -2 * i), np.where(c, -2 * i, q), np.where(c, q, -2 * i - 2),
            np.where(c, -2 * i - 2, q))


def _g_walk(H, W, s, descend):
    """per sample of an H x W image: stage-s parity, basis, and (descend) the child's
    origin, family and tree index after stage s"""
    r, c = np.mgrid[0:H, 0:W]
    o_r, o_c = np.zeros_like(r), np.zeros_like(r)
    T, i, cid = np.zeros_like(r), np.zeros_like(r), np.zeros_like(r)
    for st in range(1, s + 1):
        b0, b1, b2, b3 = _g_basis(st, T, i)
        det = b0 * b3 - b1 * b2
        dr, dc = r - o_r, c - o_c
        n1, n2 = b3 * dr - b2 * dc, b0 * dc - b1 * dr
        assert np.all(n1 % det == 0) and np.all(n2 % det == 0), "sample off its channel's lattice"
        par = (n1 // det + n2 // det) & 1
        if st == s and not descend:
            return par, (b0, b1, b2, b3)
        cid = 2 * cid + par
        o_r, o_c = o_r + par * b0, o_c + par * b1
        if st == 1:
            T, i = par, np.zeros_like(par)
        elif st == 2:
            i = np.where(par == 1, 0, -1)
        else:
            i = 2 * i + par
    return cid, o_r, o_c, T


def _g_sums(img, T, s, target, n):
    """first launch of a pass: diagonal sums at the samples of the other parity"""
    H, W = img.shape
    par, (b0, b1, b2, b3) = _g_walk(H, W, s, False)
    r, c = np.mgrid[0:H, 0:W]
    S = np.zeros_like(img)
    for b, wb in _fan_taps(n):
        u = (b + 1) // 2
        S += wb * img[(r + u * (b0 - b2)) % H, (c + u * (b1 - b3)) % W]
    m = par != target
    T[m] = S[m]


def _g_pass(img, T, s, target, alpha, gamma, n):
    """second launch: the targets from the sums"""
    H, W = img.shape
    par, (b0, b1, b2, b3) = _g_walk(H, W, s, False)
    r, c = np.mgrid[0:H, 0:W]
    acc = np.zeros_like(img)
    for a, wa in _fan_taps(n):
        d1, d2 = (a - 1) // 2, (a + 1) // 2
        acc += wa * T[(r + d1 * b0 + d2 * b2) % H, (c + d1 * b1 + d2 * b3) % W]
    m = par == target
    img[m] = alpha * img[m] + gamma * acc[m]


def _g_leaf_index(J):
    """coefficient offset (from slot0) of every sample of the job's detail image"""
    H, W, k = int(J["H"]), int(J["W"]), int(J["k"])
    cid, o_r, o_c, T = _g_walk(H, W, k, True)
    r, c = np.mgrid[0:H, 0:W]
    if k == 1:
        a, b, w = r, c >> 1, W // 2
    else:
        R = np.where(T == 0, 2 ** (k - 1), 2)
        C = np.where(T == 0, 2, 2 ** (k - 1))
        a, b, w = (r - o_r % R) // R, (c - o_c % C) // C, W // C
    idx = cid * ((H * W) >> k) + a * w + b
    assert np.array_equal(np.sort(idx.ravel()), np.arange(H * W)), "the copy is not a bijection"
    return idx


def _stage_a_pass(img, stage, odd, alpha, gamma):
    """One pass of DFB stage 1 or 2 over the whole periodic image, in place."""
    H, W = img.shape
    r, c = np.mgrid[0:H, 0:W]
    if stage == 1:
        mask = ((r + c) & 1) == odd
        offs = [((a + b) // 2, (a - b) // 2) for a in A4 for b in A4]
        acc = sum(BT[t // 4] * BT[t % 4] * np.roll(img, (-dy, -dx), axis=(0, 1)) for t, (dy, dx) in enumerate(offs))
    else:
        mask = (c & 1) == odd
        fam_c = (r & 1) == (c & 1)
        acc_c = sum(BT[ia] * BT[ib] * np.roll(img, (-a, -b), axis=(0, 1))
                    for ia, a in enumerate(A4) for ib, b in enumerate(A4))
        acc_r = sum(BT[ia] * BT[ib] * np.roll(img, (-b, -a), axis=(0, 1))
                    for ia, a in enumerate(A4) for ib, b in enumerate(A4))
        acc = np.where(fam_c, acc_c, acc_r)
    img[mask] = alpha * img[mask] + gamma * acc[mask]


def _rowsplit_stencil(S, i, odd_target):
    acc = np.zeros_like(S)
    for ia, a in enumerate(A4):
        for ib, b in enumerate(A4):
            dr = (a + 1) // 2 if odd_target else (a - 1) // 2
            dc = -i * a + (b - a) // 2
            acc += BT[ia] * BT[ib] * np.roll(S, (-dr, -dc), axis=(0, 1))
    return acc


def _index(v, rows, cols):
    u = np.arange(rows, dtype=np.int64)[:, None]
    c = np.arange(cols, dtype=np.int64)[None, :]
    return int(v["b"]), v["off"] + u * v["rs"] + c * v["cs"]


def _check(b, idx, elems, what):
    assert idx.min() >= 0 and idx.max() < elems[b], "%s: index range [%d, %d] outside buffer %d of %d" % (
        what, idx.min(), idx.max(), b, elems[b])


def _down(x, f):
    R = (len(f) - 1) // 2
    t = sum(f[a + R] * np.roll(x, a, axis=1) for a in range(-R, R + 1))[:, ::2]
    return sum(f[a + R] * np.roll(t, a, axis=0) for a in range(-R, R + 1))[::2, :]


def _up(v, f):
    H, W = 2 * v.shape[0], 2 * v.shape[1]
    R = (len(f) - 1) // 2
    z = np.zeros((v.shape[0], W))
    z[:, ::2] = v
    t = sum(f[a + R] * np.roll(z, a, axis=1) for a in range(-R, R + 1))
    z = np.zeros((H, W))
    z[::2, :] = t
    return sum(f[a + R] * np.roll(z, a, axis=0) for a in range(-R, R + 1))


def _views_of(kind, J, synth, extra=None):
    """(reads, writes): lists of (name, view, rows, cols) a job touches."""
    if kind == 3:
        H, W = int(J["H"]), int(J["W"])
        return [("D", J["D"], H, W), ("T", J["T"], H, W)], [("T", J["T"], H, W)]
    if kind == 5:
        H, W = int(J["H"]), int(J["W"])
        D = [("D", J["D"], H, W)]
        return D + [("T", J["T"], H, W)], D
    if kind == 4:
        H, W = int(J["H"]), int(J["W"])
        lay = np.zeros(1, VIEW)[0]
        lay["off"], lay["b"], lay["rs"], lay["cs"] = int(J["slot0"]), 1, W, 1
        D, L = [("D", J["D"], H, W)], [("layout", lay, H, W)]     # the level's 2^k subbands, H*W elements
        return (D, L) if extra[1] == 1 else (L, D)
    if kind == 0:
        H, W = int(J["H"]), int(J["W"])
        if not synth:
            return [("main", J["main"], H, W)], [("cout", J["cout"], H // 2, W // 2), ("out", J["out"], H, W)]
        return [("main", J["main"], H, W), ("cin", J["cin"], H // 2, W // 2)], [("out", J["out"], H, W)]
    if kind == 1:
        H, W = int(J["H"]), int(J["W"])
        comps = [("comp%d" % q, J["comp"][q], H // 2, W // 2) for q in range(4)]
        D = [("D", J["D"], H, W)]
        return (D, comps) if not synth else (comps, D)
    R2, C = int(J["R2"]), int(J["C"])
    par = [("pe", J["pe"], R2, C), ("po", J["po"], R2, C)]
    chi = [("c0", J["c0"], R2, C), ("c1", J["c1"], R2, C)]
    return (par, chi) if not synth else (chi, par)


def run(mode, elems, launches, bufs):
    """Execute the launches on bufs (dict base id -> float64 array); checks bounds and hazards."""
    h, g = O.cdf97()
    fa, fs = (h, g) if mode in (0, 1) else (g, h)
    synth = mode in (1, 2)
    fo, a1, g1, a2, g2 = PASSES[mode]
    for kind, jobs, extra in launches:
        results, wjob, rjob = [], [], []
        for ji, J in enumerate(jobs):
            reads, writes = _views_of(kind, J, synth, extra)
            rd = {}
            for name, v, rr, cc in reads:
                b, idx = _index(v, rr, cc)
                _check(b, idx, elems, "read " + name)
                rd[name] = bufs[b][idx]
                rjob.append((ji, (b, idx)))
            out = {}
            if kind == 3:
                T = rd["T"].copy()
                _g_sums(rd["D"], T, extra[0], extra[1], int(J["ntaps"]))
                out["T"] = T
            elif kind == 5:
                img = rd["D"].copy()
                _g_pass(img, rd["T"], extra[0], extra[1], extra[2], extra[3], int(J["ntaps"]))
                out["D"] = img
            elif kind == 4:
                idx = _g_leaf_index(J)
                if extra[1] == 1:
                    lay = np.zeros(rd["D"].size)
                    lay[idx.ravel()] = rd["D"].ravel()
                    out["layout"] = lay.reshape(rd["D"].shape)
                else:
                    out["D"] = rd["layout"].ravel()[idx]
            elif kind == 0:
                X = rd["main"]
                if not synth:
                    out["cout"] = _down(X, fa)
                    out["out"] = X - _up(out["cout"], fs)
                else:
                    out["out"] = X + _up(rd["cin"] - _down(X, fa), fs)
            elif kind == 1:
                H, W = int(J["H"]), int(J["W"])
                nst = int(J["nst"])
                img = np.zeros((H, W))
                if not synth:
                    img[:] = rd["D"]
                else:
                    for q in range(4):
                        img[q >> 1::2, q & 1::2] = rd["comp%d" % q]
                stages = list(range(1, nst + 1)) if not synth else list(range(nst, 0, -1))
                for stg in stages:
                    _stage_a_pass(img, stg, fo, a1, g1)
                    _stage_a_pass(img, stg, 1 - fo, a2, g2)
                if not synth:
                    for q in range(4):
                        out["comp%d" % q] = img[q >> 1::2, q & 1::2].copy()
                else:
                    out["D"] = img
            else:
                i = int(J["i"])
                E, Od = (rd["pe"], rd["po"]) if not synth else (rd["c0"], rd["c1"])
                E, Od = E.copy(), Od.copy()
                if fo:
                    Od = a1 * Od + g1 * _rowsplit_stencil(E, i, True)
                    E = a2 * E + g2 * _rowsplit_stencil(Od, i, False)
                else:
                    E = a1 * E + g1 * _rowsplit_stencil(Od, i, False)
                    Od = a2 * Od + g2 * _rowsplit_stencil(E, i, True)
                if not synth:
                    out["c0"], out["c1"] = E, Od
                else:
                    out["pe"], out["po"] = E, Od
            for name, v, rr, cc in writes:
                b, idx = _index(v, rr, cc)
                _check(b, idx, elems, "write " + name)
                results.append((b, idx, out[name]))
                wjob.append((ji, b, idx))
        # no job writes an element that another job of the same launch reads or writes
        # (a plain DFB pass reads and writes its own image: in place, by parity)
        for b in set(x[1] for x in wjob):
            w_idx = [(ji, ix.ravel()) for ji, wb, ix in wjob if wb == b]
            allw = np.concatenate([ix for _, ix in w_idx])
            owner = np.concatenate([np.full(ix.size, i) for i, ix in w_idx])
            order = np.argsort(allw, kind="stable")
            allw, owner = allw[order], owner[order]
            assert np.all(np.diff(allw) > 0), "two jobs of one launch write the same element"
            for i, (rb, ridx) in rjob:
                if rb != b:
                    continue
                r = ridx.ravel()
                pos = np.clip(np.searchsorted(allw, r), 0, allw.size - 1)
                hit = allw[pos] == r
                assert np.all(owner[pos][hit] == i), "a job reads what another job of its launch writes"
        for b, idx, val in results:
            bufs[b][idx] = val
    return bufs


def check_only(elems, launches, mode):
    """Bounds of every job of every launch, without executing (for full-size plans)."""
    synth = mode in (1, 2)
    for kind, jobs, extra in launches:
        for J in jobs:
            reads, writes = _views_of(kind, J, synth, extra)
            for name, v, rr, cc in reads + writes:
                b, idx = _index(v, rr, cc)
                _check(b, idx, elems, name)
