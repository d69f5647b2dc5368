"""The launch plans of libcvc (CPU only, no GPU): every job stays inside its
buffers, no launch has a cross-job read/write hazard, and executing the job
tables with the kernels' semantics in double precision reproduces the
oracle's transform.  This checks the host planner (views, strides, stencil
offsets, pass order) independently of the GPU."""
import numpy as np
import pytest

import oracle as O
import plan_emulator as E
from paper_1510_00561_b300 import _lib as L

PLANS = [(64, 64, 3, [3, 2, 2], 2), (144, 176, 3, [3, 2, 2], 1), (96, 160, 4, [4, 3, 3, 2], 1),
         (64, 96, 2, [0, 1], 1), (128, 128, 2, [6, 5], 1), (72, 88, 3, [3, 2, 2], 1), (128, 256, 5, [5, 4, 4, 3, 3], 1)]


def _buffers(elems):
    return {b: np.zeros(int(elems[b])) for b in range(4)}


@pytest.mark.parametrize("H,W,Lv,k,batch", PLANS)
@pytest.mark.parametrize("mode,fuse", [(0, 0), (1, 0), (2, 0), (3, 0), (0, 6), (1, 6), (0, 1), (1, 2)])
def test_plan_tables_compute_the_transform(H, W, Lv, k, batch, mode, fuse):
    """fuse: the pyramid tail's fusion depth (the forward and inverse run their coarse levels
    in one block per plane, the images resident in a per-plane scratch buffer)"""
    elems, launches = E.tables(mode | (fuse << 8), h=H, w=W, levels=Lv, dirs=k, batch=batch)
    assert (fuse > 0) == any(kind == 3 for kind, _, _ in launches)
    n = O.layout(H, W, Lv, k)["total"]
    assert elems[0] == batch * H * W and elems[1] == batch * n and elems[3] == batch * H * W
    rng = np.random.default_rng(mode)
    bufs = _buffers(elems)
    in_base, out_base = {0: (0, 1), 1: (1, 3), 2: (1, 3), 3: (0, 1)}[mode]
    x = rng.uniform(-50, 255, elems[in_base])
    bufs[in_base][:] = x
    E.run(mode, elems, launches, bufs)
    for b in range(batch):
        if mode in (0, 3):
            xin = x[b * H * W:(b + 1) * H * W].reshape(H, W)
            ref = O.ct(mode, xin, H, W, Lv, k)
            got = bufs[1][b * n:(b + 1) * n]
        else:
            cin = x[b * n:(b + 1) * n]
            ref = O.ct(mode, cin, H, W, Lv, k).ravel()
            got = bufs[3][b * H * W:(b + 1) * H * W]
        assert np.abs(got - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("fuse", [0, 6])
@pytest.mark.parametrize("w,h,Lv,k", [(176, 144, 3, [3, 2, 2]), (99, 77, 2, [2, 2]), (64, 48, 2, [1, 0])])
def test_codec_plan_tables(w, h, Lv, k, fuse):
    prm = L.Params(w, h, Lv, L.ints(k), 8, 1, 0.0, 8, 1)
    elems, launches = E.tables(0 | (fuse << 8), params=prm)
    oc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 8)
    rng = np.random.default_rng(1)
    frame = rng.integers(0, 256, (h, w, 3), dtype=np.uint8)
    yp, cop, cgp = oc.planes(frame)
    bufs = _buffers(elems)
    bufs[0][:] = np.concatenate([yp.ravel(), cop.ravel(), cgp.ravel()])
    E.run(0, elems, launches, bufs)
    ref = np.concatenate([O.ct(0, p, p.shape[0], p.shape[1], Lv, k) for p in (yp, cop, cgp)])
    assert np.abs(bufs[1] - ref).max() < 1e-7
    # and the inverse tables invert it
    elems, launches = E.tables(1 | (fuse << 8), params=prm)
    E.run(1, elems, launches, bufs)
    assert np.abs(bufs[3] - bufs[0]).max() < 1e-8


def test_benchmark_codec_plan_is_in_bounds():
    """The 1080p configuration: bounds and hazards of every forward and inverse job."""
    prm = L.Params(1920, 1080, 5, L.ints([5, 4, 4, 3, 3]), 8, 1, 0.0, 10, 1)
    for mode in (0, 1, 0 | 6 << 8, 1 | 6 << 8):
        elems, launches = E.tables(mode, params=prm)
        E.check_only(elems, launches, mode & 255)


MIXED = [(99, 77, 2, [2, 2]), (64, 48, 3, [3, 2, 2]), (40, 30, 1, [0]), (96, 64, 2, [1, 0])]


def test_batch_plan_tables_of_mixed_streams():
    """A batch of streams with different sizes and decompositions shares one
    launch sequence; its tables must compute every stream's transform (and
    its inverse) exactly as a codec of that stream alone would."""
    prms = (L.Params * len(MIXED))(*[L.Params(w, h, Lv, L.ints(k), 8, 1, 0.0, 8, 1) for w, h, Lv, k in MIXED])
    elems, launches = _mixed_tables(prms, 0)
    rng = np.random.default_rng(5)
    planes, refs = [], []
    for w, h, Lv, k in MIXED:
        oc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 8)
        yp, cop, cgp = oc.planes(rng.integers(0, 256, (h, w, 3), dtype=np.uint8))
        planes += [yp.ravel(), cop.ravel(), cgp.ravel()]
        refs += [O.ct(0, p, p.shape[0], p.shape[1], Lv, k) for p in (yp, cop, cgp)]
    bufs = _buffers(elems)
    bufs[0][:] = np.concatenate(planes)
    E.run(0, elems, launches, bufs)
    assert np.abs(bufs[1] - np.concatenate(refs)).max() < 1e-7
    elems, launches = _mixed_tables(prms, 1)
    E.run(1, elems, launches, bufs)
    assert np.abs(bufs[3] - bufs[0]).max() < 1e-8


def _mixed_tables(prms, mode):
    import ctypes
    return E.tables(mode, params=ctypes.cast(prms, ctypes.POINTER(L.Params)).contents, batch=len(MIXED))


def test_mixed_stream_batch_of_the_streaming_workload_is_in_bounds():
    """64 streams, 16 each of QCIF, CIF, VGA and 720p: bounds and hazards of every job."""
    cfg = [(176, 144, 3, [3, 2, 2]), (352, 288, 3, [3, 2, 2]), (640, 480, 4, [4, 3, 3, 2]),
           (1280, 720, 5, [5, 4, 4, 3, 3])]
    prms = (L.Params * 64)(*[L.Params(w, h, Lv, L.ints(k), 8, 1, 0.0, 10, 1)
                             for w, h, Lv, k in cfg for _ in range(16)])
    import ctypes
    first = ctypes.cast(prms, ctypes.POINTER(L.Params)).contents
    for mode in (0, 1):
        elems, launches = E.tables(mode, params=first, batch=64)
        E.check_only(elems, launches, mode)


SCALED = [(99, 77, 2, [2, 2]), (64, 48, 3, [3, 2, 2]), (40, 30, 1, [0]), (176, 144, 3, [3, 0, 2]),
          (96, 64, 2, [1, 0])]


@pytest.mark.parametrize("scale", [0, 1, 2, 3])
def test_scaled_decoder_tables(scale):
    """The decoder back end at pyramid scale s (§3.3) over a batch of mixed
    streams: the inverse-transform tables of the sub-pyramids stay in bounds
    and, executed on random coefficients, give every stream's level-s lowpass
    planes (the oracle's inverse of the lowpass and levels s+1..L, over 2^s);
    the output records address those planes (or, at s = L, the lowpass band
    itself) with the right sizes and block offsets."""
    import ctypes
    prms = (L.Params * len(SCALED))(*[L.Params(w, h, Lv, L.ints(k), 8, 1, 0.0, 8, 1) for w, h, Lv, k in SCALED])
    elems, launches, desc = E.scale_tables(ctypes.cast(prms, ctypes.POINTER(L.Params)), len(SCALED), scale)
    assert len(desc) == len(SCALED)
    rng = np.random.default_rng(scale)
    bufs = _buffers(elems)
    bufs[1][:] = rng.uniform(-60, 60, elems[1])
    E.run(1, elems, launches, bufs)
    coef_off = plane_off = blk = 0
    for i, (w, h, Lv, k) in enumerate(SCALED):
        oc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 8)
        dims = [(oc.Hp, oc.Wp), (oc.Hcp, oc.Wcp), (oc.Hcp, oc.Wcp)]
        lays = [O.layout(H, W, Lv, k) for H, W in dims]
        if Lv >= scale:
            Q = desc[i]
            f = 1 << scale
            hc, wc = (h + 1) // 2, (w + 1) // 2
            assert (Q["H"], Q["W"], Q["Hc"], Q["Wc"]) == ((h + f - 1) // f, (w + f - 1) // f,
                                                          (hc + f - 1) // f, (wc + f - 1) // f)
            assert Q["blk0"] == blk and Q["norm"] == 2.0 ** -scale
            blk += Q["H"]
            src = bufs[1] if Q["src"] else bufs[3]
            assert Q["src"] == (scale == Lv)
            poff = coef_off
            for p, ((H, W), lay) in enumerate(zip(dims, lays)):
                cp = bufs[1][poff:poff + lay["total"]]
                sb = lay["subbands"]
                nlow = sb[0]["h"] * sb[0]["w"]
                if scale == Lv:
                    ref = cp[:nlow].reshape(sb[0]["h"], sb[0]["w"])
                else:
                    first = 1 + sum(1 << k[j] for j in range(scale))
                    sub = np.concatenate([cp[:nlow], cp[sb[first]["off"]:]])
                    ref = O.ct(1, sub, H >> scale, W >> scale, Lv - scale, k[scale:]).reshape(H >> scale, W >> scale)
                ref = ref * 2.0 ** -scale
                rows, cols = (Q["H"], Q["W"]) if p == 0 else (Q["Hc"], Q["Wc"])
                rs = Q["rs_y"] if p == 0 else Q["rs_c"]
                assert rs == ref.shape[1] and rows <= ref.shape[0] and cols <= ref.shape[1]
                idx = Q["off"][p] + np.arange(ref.shape[0])[:, None] * rs + np.arange(ref.shape[1])[None, :]
                assert idx.min() >= 0 and idx.max() < len(src)
                got = src[idx] * float(Q["norm"])
                assert np.abs(got - ref).max() < 1e-8 * max(1.0, np.abs(ref).max()), (i, p)
                poff += lay["total"]
        coef_off += sum(l["total"] for l in lays)
        plane_off += sum(H * W for H, W in dims)
    assert elems[1] == coef_off and elems[3] == plane_off


def test_scale_tables_refuse_a_scale_beyond_every_stream():
    import ctypes
    prms = (L.Params * 2)(L.Params(99, 77, 2, L.ints([2, 2]), 8, 1, 0.0, 8, 1),
                          L.Params(40, 30, 1, L.ints([0]), 8, 1, 0.0, 8, 1))
    used = ctypes.c_size_t(0)
    lib = L.lib()
    assert lib.cvc_debug_scale_tables(prms, 2, 3, None, 0, ctypes.byref(used)) == 1
    assert lib.cvc_debug_scale_tables(prms, 2, -1, None, 0, ctypes.byref(used)) == 1
    assert lib.cvc_debug_scale_tables(prms, 2, 2, None, 0, ctypes.byref(used)) == 3


# ------------------------------------------------- longer DFB prototypes
@pytest.mark.parametrize("taps", [6, 8])
@pytest.mark.parametrize("w,h,Lv,k", [(176, 144, 3, [3, 2, 2]), (64, 48, 2, [1, 0]), (128, 96, 3, [4, 3, 1])])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_longer_prototype_plan_tables_compute_the_transform(taps, w, h, Lv, k, mode):
    """the tile launches of a longer prototype, executed with their semantics (the
    prototype's taps), reproduce the oracle's transform with that prototype"""
    prm = L.params(w, h, Lv, k, 8, 1, 0.0, 8, dfb_taps=taps)
    elems, launches = E.tables(mode, params=prm)
    assert all(int(J["ntaps"]) == taps for kd, jobs, _ in launches if kd in (1, 2) for J in jobs)
    oc = O.Codec(w, h, Lv, k, 8, 1, 0.0, 8)
    dims = [(oc.Hp, oc.Wp), (oc.Hcp, oc.Wcp), (oc.Hcp, oc.Wcp)]
    ns = [O.layout(a, b, Lv, k)["total"] for a, b in dims]
    rng = np.random.default_rng(mode + taps)
    bufs = _buffers(elems)
    in_base, out_base = {0: (0, 1), 1: (1, 3), 2: (1, 3), 3: (0, 1)}[mode]
    x = rng.uniform(-50, 255, elems[in_base])
    bufs[in_base][:] = x
    E.run(mode, elems, launches, bufs)
    po, co = 0, 0
    for (H, W), n in zip(dims, ns):
        if mode in (0, 3):
            ref = O.ct(mode, x[po:po + H * W].reshape(H, W), H, W, Lv, k, taps)
            got = bufs[1][co:co + n]
        else:
            ref = O.ct(mode, x[co:co + n], H, W, Lv, k, taps).ravel()
            got = bufs[3][po:po + H * W]
        assert np.abs(got - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())
        po += H * W
        co += n


def test_mixed_prototype_codec_plans_in_bounds():
    """a batch mixing prototypes: launches of each length side by side, in bounds, at 1080p"""
    prms = (L.Params * 3)(L.params(1920, 1080, 5, [5, 4, 4, 3, 3], 8, 1, 0.0, 10, dfb_taps=6),
                          L.params(1920, 1080, 5, [5, 4, 4, 3, 3], 8, 1, 0.0, 10),
                          L.params(640, 480, 4, [4, 3, 3, 2], 8, 1, 0.0, 10, dfb_taps=8))
    import ctypes
    for mode in (0, 1):
        elems, launches = E.tables(mode, params=ctypes.cast(prms, ctypes.POINTER(L.Params)).contents, batch=3)
        assert {int(J["ntaps"]) for kd, jobs, _ in launches if kd in (1, 2) for J in jobs} == {4, 6, 8}
        E.check_only(elems, launches, mode)
