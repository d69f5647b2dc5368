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

DFB jobs carry their prototype length n; their stencils use the n fan taps
computed here from the Lagrange interpolation formula, not from the library.

so that a test can compare the planned computation with the oracle before
any kernel runs on a GPU.  Each pass sets target = alpha*target + gamma*sum.
"""
import ctypes

import numpy as np

import oracle as O
from paper_1510_00561_b300 import _lib as L

VIEW = np.dtype([("off", "<i8"), ("b", "<i4"), ("rs", "<i4"), ("cs", "<i4"), ("pad", "<i4")])
LPJOB = np.dtype([("main", VIEW), ("cin", VIEW), ("cout", VIEW), ("out", VIEW), ("cin_lo", VIEW), ("out_lo", VIEW),
                  ("H", "<i4"), ("W", "<i4"),
                  ("tiles_x", "<i4"), ("first_block", "<i4"), ("stream", "<i4"), ("pad2", "<i4")])
AJOB = np.dtype([("D", VIEW), ("comp", VIEW, (4,)), ("H", "<i4"), ("W", "<i4"), ("nst", "<i4"),
                 ("tiles_x", "<i4"), ("first_block", "<i4"), ("ntaps", "<i4"), ("stream", "<i4"),
                 ("pad2", "<i4")])
BJOB = np.dtype([("pe", VIEW), ("po", VIEW), ("c0", VIEW), ("c1", VIEW), ("R2", "<i4"), ("C", "<i4"),
                 ("i", "<i4"), ("tiles_x", "<i4"), ("first_block", "<i4"), ("ntaps", "<i4"), ("stream", "<i4"),
                 ("pad2", "<i4")])
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
    magic, nl, lpb, ab, bb, tail_sz = np.frombuffer(raw[:24], "<u4")
    assert tail_sz in (0, SCALEDESC.itemsize)
    assert magic == 0x43564350 and lpb == LPJOB.itemsize and ab == AJOB.itemsize and bb == BJOB.itemsize
    elems = np.frombuffer(raw[24:56], "<u8").astype(np.int64)
    pos = 56
    launches = []
    for _ in range(nl):
        kind, nj = np.frombuffer(raw[pos:pos + 8], "<u4")
        pos += 8
        extra = None
        if kind == 3:
            launches.append((3, _parse_tail(raw[pos:pos + nj]), None))
            pos += nj
            continue
        dt = (LPJOB, AJOB, BJOB)[kind]
        jobs = np.frombuffer(raw[pos:pos + nj * dt.itemsize], dt)
        pos += nj * dt.itemsize
        launches.append((int(kind), jobs, extra))
    return elems, launches, raw[pos:]


def _parse_tail(blob):
    """a pyramid-tail launch: [(resident floats, stream, [(kind, job record), ...]) per plane]"""
    nplanes, _ntaps = np.frombuffer(blob[:8], "<u4")
    pos, planes = 8, []
    for _ in range(nplanes):
        ws, stream, nsteps, _ = np.frombuffer(blob[pos:pos + 16], "<i4")
        pos += 16
        steps = []
        for _ in range(nsteps):
            kind = int(np.frombuffer(blob[pos:pos + 4], "<u4")[0])
            pos += 8
            dt = (LPJOB, AJOB, BJOB)[kind]
            steps.append((kind, np.frombuffer(blob[pos:pos + dt.itemsize], dt)))
            pos += dt.itemsize
        planes.append((int(ws), int(stream), steps))
    assert pos == len(blob)
    return planes


def _flatten(elems, launches):
    """the launches with every tail expanded into one-job launches, each with the bounds it runs
    under: (kind, jobs, extra, elems), where base 4 (B_SMEM) is the plane's resident workspace,
    and a fresh workspace marker before each tail plane"""
    base = list(elems) + [0]
    for kind, jobs, extra in launches:
        if kind != 3:
            yield kind, jobs, extra, base
            continue
        for ws, _stream, steps in jobs:
            e = list(elems) + [ws]
            yield "smem", ws, None, e
            for k, J in steps:
                yield k, J, None, e


def _fan_taps(n):
    """fan taps of the n-tap Lagrange half-band prototype: weight of the sample at odd a
    when interpolating at 0, times (-1)^((a - 1) / 2)"""
    pts = list(range(-(n - 1), n, 2))
    out = []
    for a in pts:
        w = np.prod([b / (b - a) for b in pts if b != a])
        out.append((a, (-1.0) ** (((a - 1) // 2) % 2) * w))
    return out


def _stage_a_pass(img, stage, odd, alpha, gamma, n=4):
    """One pass of DFB stage 1 or 2 over the whole periodic image, in place (n-tap prototype)."""
    H, W = img.shape
    r, c = np.mgrid[0:H, 0:W]
    taps = _fan_taps(n)
    if stage == 1:
        mask = ((r + c) & 1) == odd
        acc = sum(wa * wb * np.roll(img, (-((a + b) // 2), -((a - b) // 2)), axis=(0, 1))
                  for a, wa in taps for b, wb in taps)
    else:
        mask = (c & 1) == odd
        fam_c = (r & 1) == (c & 1)
        acc_c = sum(wa * wb * np.roll(img, (-a, -b), axis=(0, 1)) for a, wa in taps for b, wb in taps)
        acc_r = sum(wa * wb * np.roll(img, (-b, -a), axis=(0, 1)) for a, wa in taps for b, wb in taps)
        acc = np.where(fam_c, acc_c, acc_r)
    img[mask] = alpha * img[mask] + gamma * acc[mask]


def _rowsplit_stencil(S, i, odd_target, n=4):
    acc = np.zeros_like(S)
    for a, wa in _fan_taps(n):
        for b, wb in _fan_taps(n):
            dr = (a + 1) // 2 if odd_target else (a - 1) // 2
            dc = -i * a + (b - a) // 2
            acc += wa * wb * np.roll(S, (-dr, -dc), axis=(0, 1))
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
    if kind == 0:
        H, W = int(J["H"]), int(J["W"])
        if not synth:
            return [("main", J["main"], H, W)], [("cout", J["cout"], H // 2, W // 2), ("out", J["out"], H, W)]
        # float-float lowpass images between synthesis levels: optional low-order halves
        reads = [("main", J["main"], H, W), ("cin", J["cin"], H // 2, W // 2)]
        writes = [("out", J["out"], H, W)]
        if int(J["cin_lo"]["b"]) >= 0:
            reads.append(("cin_lo", J["cin_lo"], H // 2, W // 2))
        if int(J["out_lo"]["b"]) >= 0:
            writes.append(("out_lo", J["out_lo"], H, W))
        return reads, writes
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
    for kind, jobs, extra, elems in _flatten(elems, launches):
        if kind == "smem":
            bufs[4] = np.full(jobs, np.nan)     # a tail plane's resident workspace, never read before written
            continue
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
            if kind == 0:
                X = rd["main"]
                if not synth:
                    out["cout"] = _down(X, fa)
                    out["out"] = X - _up(out["cout"], fs)
                else:
                    # in double precision the whole value sits in the high part
                    out["out"] = X + _up(rd["cin"] + rd.get("cin_lo", 0.0) - _down(X, fa), fs)
                    if int(J["out_lo"]["b"]) >= 0:
                        out["out_lo"] = np.zeros_like(out["out"])
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
                n = int(J["ntaps"])
                for stg in stages:
                    _stage_a_pass(img, stg, fo, a1, g1, n)
                    _stage_a_pass(img, stg, 1 - fo, a2, g2, n)
                if not synth:
                    for q in range(4):
                        out["comp%d" % q] = img[q >> 1::2, q & 1::2].copy()
                else:
                    out["D"] = img
            else:
                i = int(J["i"])
                E, Od = (rd["pe"], rd["po"]) if not synth else (rd["c0"], rd["c1"])
                E, Od = E.copy(), Od.copy()
                n = int(J["ntaps"])
                if fo:
                    Od = a1 * Od + g1 * _rowsplit_stencil(E, i, True, n)
                    E = a2 * E + g2 * _rowsplit_stencil(Od, i, False, n)
                else:
                    E = a1 * E + g1 * _rowsplit_stencil(Od, i, False, n)
                    Od = a2 * Od + g2 * _rowsplit_stencil(E, i, True, n)
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
    for kind, jobs, extra, elems in _flatten(elems, launches):
        if kind == "smem":
            continue
        for J in jobs:
            reads, writes = _views_of(kind, J, synth, extra)
            for name, v, rr, cc in reads + writes:
                b, idx = _index(v, rr, cc)
                _check(b, idx, elems, name)
