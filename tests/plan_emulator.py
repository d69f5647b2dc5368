"""Host-side reading of libcvc's launch plans (test helper, no GPU).

``cvc_debug_plan_tables`` dumps the job tables the CUDA kernels execute.  This
module parses them, checks that every element a job reads or writes lies
inside its buffer and that no job of a launch writes what another job of the
same launch touches, and executes the tables in double precision with the
semantics of the two kernels:

  LP level job (analysis):   cout = down(main, fa);       out = main - up(cout, fs)
  LP level job (synthesis):  v = cin - down(main, fa);    out = main + up(v, fs)
  DFB lifting job:           out(u,v) = alpha tin(u,v) + gamma sum_t w_t src_sel(u+dr, v+dc)  (periodic)

so that a test can compare the planned computation with the oracle before
any kernel runs on a GPU.
"""
import ctypes

import numpy as np

import oracle as O
from paper_1510_00561_b300 import _lib as L

VIEW = np.dtype([("off", "<i8"), ("b", "<i4"), ("rs", "<i4"), ("cs", "<i4"), ("pad", "<i4")])
LPJOB = np.dtype([("main", VIEW), ("cin", VIEW), ("cout", VIEW), ("out", VIEW), ("H", "<i4"), ("W", "<i4"),
                  ("tiles_x", "<i4"), ("first_block", "<i4")])
LIFTJOB = np.dtype([("out", VIEW), ("tin", VIEW), ("src", VIEW, (2,)), ("rows", "<i4"), ("cols", "<i4"),
                    ("alpha", "<f4"), ("gamma", "<f4"), ("w", "<f4", (16,)), ("sel", "i1", (16,)),
                    ("dr", "<i2", (16,)), ("dc", "<i2", (16,)), ("first_block", "<i4"), ("pad", "<i4")])


def tables(mode, params=None, h=0, w=0, levels=0, dirs=(), batch=1):
    lib = L.lib()
    used = ctypes.c_size_t(0)
    pp = ctypes.byref(params) if params is not None else None
    st = lib.cvc_debug_plan_tables(pp, h, w, levels, L.ints(dirs), batch, mode, None, 0, ctypes.byref(used))
    assert st == 3, st
    buf = (ctypes.c_uint8 * used.value)()
    st = lib.cvc_debug_plan_tables(pp, h, w, levels, L.ints(dirs), batch, mode, buf, used.value, ctypes.byref(used))
    assert st == 0, st
    raw = bytes(buf)
    magic, nl, lpb, lfb = np.frombuffer(raw[:16], "<u4")
    assert magic == 0x43564350 and lpb == LPJOB.itemsize and lfb == LIFTJOB.itemsize
    elems = np.frombuffer(raw[16:48], "<u8").astype(np.int64)
    pos = 48
    launches = []
    for _ in range(nl):
        kind, nj = np.frombuffer(raw[pos:pos + 8], "<u4")
        pos += 8
        dt = LPJOB if kind == 0 else LIFTJOB
        jobs = np.frombuffer(raw[pos:pos + nj * dt.itemsize], dt)
        pos += nj * dt.itemsize
        launches.append((int(kind), jobs))
    assert pos == len(raw)
    return elems, launches


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


def run(mode, elems, launches, bufs):
    """Execute the launches on bufs (dict base id -> float64 array); checks bounds and hazards."""
    h, g = O.cdf97()
    fa, fs = (h, g) if mode in (0, 1) else (g, h)
    synth = mode in (1, 2)
    for kind, jobs in launches:
        writes, results = [], []
        wjob, rjob = [], []
        for ji, J in enumerate(jobs):
            if kind == 0:
                H, W = int(J["H"]), int(J["W"])
                bm, im = _index(J["main"], H, W)
                _check(bm, im, elems, "lp main")
                X = bufs[bm][im]
                rjob.append((ji, (bm, im)))
                if not synth:
                    bc, ic = _index(J["cout"], H // 2, W // 2)
                    _check(bc, ic, elems, "lp cout")
                    c = _down(X, fa)
                    results.append((bc, ic, c))
                    writes.append((bc, ic))
                    wjob.append((ji, bc, ic))
                    out = X - _up(c, fs)
                else:
                    bc, ic = _index(J["cin"], H // 2, W // 2)
                    _check(bc, ic, elems, "lp cin")
                    rjob.append((ji, (bc, ic)))
                    out = X + _up(bufs[bc][ic] - _down(X, fa), fs)
                bo, io = _index(J["out"], H, W)
                _check(bo, io, elems, "lp out")
                results.append((bo, io, out))
                writes.append((bo, io))
                wjob.append((ji, bo, io))
            else:
                R, C = int(J["rows"]), int(J["cols"])
                bo, io = _index(J["out"], R, C)
                bt, it = _index(J["tin"], R, C)
                _check(bo, io, elems, "lift out")
                _check(bt, it, elems, "lift tin")
                srcs = []
                for s in range(2):
                    bs, is_ = _index(J["src"][s], R, C)
                    _check(bs, is_, elems, "lift src")
                    srcs.append((bs, is_))
                acc = np.zeros((R, C))
                used = set()
                for t in range(16):
                    bs, is_ = srcs[int(J["sel"][t])]
                    used.add(int(J["sel"][t]))
                    sh = np.roll(is_, (-int(J["dr"][t]), -int(J["dc"][t])), axis=(0, 1))
                    acc += float(J["w"][t]) * bufs[bs][sh]
                out = float(J["alpha"]) * bufs[bt][it] + float(J["gamma"]) * acc
                results.append((bo, io, out))
                writes.append((bo, io))
                wjob.append((ji, bo, io))
                rjob.append((ji, (bt, it)))
                for s in used:
                    rjob.append((ji, srcs[s]))
        # no job writes an element that another job of the same launch reads or writes
        for b in set(x[0] for x in writes):
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
                pos = np.searchsorted(allw, r)
                pos = np.clip(pos, 0, allw.size - 1)
                hit = allw[pos] == r
                assert np.all(owner[pos][hit] == i), "a job reads what another job of its launch writes"
        for b, idx, val in results:
            bufs[b][idx] = val
    return bufs


def check_only(elems, launches, mode):
    """Bounds of every job of every launch, without executing (for full-size plans)."""
    synth = mode in (1, 2)
    for kind, jobs in launches:
        for J in jobs:
            if kind == 0:
                H, W = int(J["H"]), int(J["W"])
                for name, (r, c) in (("main", (H, W)), ("out", (H, W)),
                                     ("cin" if synth else "cout", (H // 2, W // 2))):
                    b, idx = _index(J[name], r, c)
                    _check(b, idx, elems, "lp " + name)
            else:
                R, C = int(J["rows"]), int(J["cols"])
                for name in ("out", "tin"):
                    b, idx = _index(J[name], R, C)
                    _check(b, idx, elems, "lift " + name)
                for s in set(int(x) for x in J["sel"]):
                    b, idx = _index(J["src"][s], R, C)
                    _check(b, idx, elems, "lift src")
