"""FP64 CPU oracle of the CVC contourlet codec hot path -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package never imports the product: the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, double precision); this module
only marshals numpy arrays through ctypes.  Section numbers in the C source
refer to Katsigiannis, Papaioannou, Maroulis, arXiv:1510.00561.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, published filter taps,
brute-force direct convolution, an independent frequency-domain model of the
filter bank, invariants, hand-worked examples).  One claim of the paper stays
unpinned: §3.5's "QPH = 181 zeroes every directional coefficient" (it depends
on an 8-bit normalisation the paper never defines).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_F = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_I16 = np.ctypeslib.ndpointer(dtype=np.int16, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_IP = ctypes.POINTER(ctypes.c_int)

OK, EINVAL, ECAPACITY, EOVERFLOW, ECORRUPT, ESTATE = 0, 1, 3, 4, 5, 9
MODE_FORWARD, MODE_INVERSE, MODE_FORWARD_ADJOINT, MODE_INVERSE_ADJOINT = 0, 1, 2, 3


class _Subband(ctypes.Structure):
    _fields_ = [("off", ctypes.c_long), ("h", ctypes.c_int), ("w", ctypes.c_int),
                ("level", ctypes.c_int), ("dir", ctypes.c_int), ("kind", ctypes.c_int)]


class _Layout(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("L", ctypes.c_int),
                ("k", ctypes.c_int * 6), ("nsub", ctypes.c_int),
                ("sb", _Subband * (1 + 6 * 64)), ("total", ctypes.c_long)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_modulus.argtypes = [ctypes.c_int, _IP]
        L.or_layout_make.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP, ctypes.POINTER(_Layout)]
        L.or_cdf97.argtypes = [_D, _D]
        L.or_lp_analysis.argtypes = [_D, ctypes.c_int, ctypes.c_int, _D, _D]
        L.or_lp_synthesis.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, _D]
        L.or_lp_analysis_adjoint.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, _D]
        L.or_lp_synthesis_adjoint.argtypes = [_D, ctypes.c_int, ctypes.c_int, _D, _D]
        L.or_dfb.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.or_dfb_taps.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.or_ct_taps.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP, ctypes.c_int, _D]
        L.or_codec_set_taps.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_soft_threshold.argtypes = [_D, ctypes.POINTER(_Layout), ctypes.c_int, _D, _D]
        L.or_soft_threshold_vjp.argtypes = [_D, ctypes.POINTER(_Layout), ctypes.c_int, _D, _D, _D, _D]
        L.or_ct.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP, _D]
        L.or_ycocgr_forward.argtypes = [_U8, ctypes.c_long, _I16, _I16, _I16]
        L.or_ycocgr_inverse.argtypes = [_I16, _I16, _I16, ctypes.c_long, _U8]
        L.or_chroma_down.argtypes = [_I16, ctypes.c_int, ctypes.c_int, _I16]
        L.or_chroma_up.argtypes = [_I16, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I16]
        L.or_pad_mirror.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.or_quantize.argtypes = [ctypes.c_float, ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int, _IP]
        L.or_quantize8.argtypes = [ctypes.c_float, ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int]
        L.or_ycocg8_forward.argtypes = [_U8, ctypes.c_long, _I16, _I16, _I16]
        L.or_ycocg8_inverse.argtypes = [_I16, _I16, _I16, ctypes.c_long, _U8]
        L.or_codec_set_storage8.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_rle_row.argtypes = [_I16, ctypes.c_int, _I16]
        L.or_rle_row.restype = ctypes.c_long
        L.or_rle_expand.argtypes = [_I16, ctypes.c_long, _I16, ctypes.c_long]
        L.or_codec_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_float, ctypes.c_int]
        L.or_codec_create.restype = ctypes.c_void_p
        L.or_codec_destroy.argtypes = [ctypes.c_void_p]
        L.or_codec_reset.argtypes = [ctypes.c_void_p]
        L.or_codec_coeff_count.argtypes = [ctypes.c_void_p]
        L.or_codec_coeff_count.restype = ctypes.c_long
        L.or_codec_max_stream.argtypes = [ctypes.c_void_p]
        L.or_codec_max_stream.restype = ctypes.c_long
        L.or_codec_ncomp.argtypes = [ctypes.c_void_p]
        L.or_codec_dims.argtypes = [ctypes.c_void_p, _IP]
        L.or_codec_planes.argtypes = [ctypes.c_void_p, _U8, _D, _D, _D]
        L.or_encode_from_coeffs.argtypes = [ctypes.c_void_p, _F, _U8, ctypes.c_long,
                                            ctypes.POINTER(ctypes.c_long), _IP]
        L.or_encode.argtypes = [ctypes.c_void_p, _U8, _U8, ctypes.c_long, ctypes.POINTER(ctypes.c_long),
                                _IP, ctypes.c_void_p]
        L.or_decode.argtypes = [ctypes.c_void_p, _U8, ctypes.c_long, _U8, ctypes.c_void_p]
        L.or_decode_scaled.argtypes = [ctypes.c_void_p, _U8, ctypes.c_long, ctypes.c_int, _U8, ctypes.c_void_p]
        L.or_codec_set_motion.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_motion_search.argtypes = [_U8, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")]
        L.or_encode_from_coeffs_luma.argtypes = [ctypes.c_void_p, _F, _U8, _U8, ctypes.c_long,
                                                 ctypes.POINTER(ctypes.c_long), _IP]
        L.or_huffman_cost.argtypes = [np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS"), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]
        L.or_huffman_cost.restype = ctypes.c_ulonglong
        L.or_inflate_container.argtypes = [ctypes.c_void_p, _U8, ctypes.c_long, _U8, ctypes.c_long,
                                           ctypes.POINTER(ctypes.c_long)]
        L.or_stream_drop.argtypes = [ctypes.c_void_p, _U8, ctypes.c_long, ctypes.c_int, _U8, ctypes.c_long,
                                     ctypes.POINTER(ctypes.c_long)]
        _lib = L
    return _lib


def _ints(seq):
    arr = (ctypes.c_int * max(6, len(seq)))(*seq)
    return arr


def motion_search(cur, prev, range_):
    """§3.2 full-search block matching of two luma planes (uint8, same shape); returns
    the (nby, nbx, 2) int8 field of (dy, dx)."""
    cur = np.ascontiguousarray(cur, dtype=np.uint8)
    prev = np.ascontiguousarray(prev, dtype=np.uint8)
    H, W = cur.shape
    nby, nbx = (H + 15) // 16, (W + 15) // 16
    mv = np.zeros(nby * nbx * 2, np.int8)
    lib().or_motion_search(cur.ravel(), prev.ravel(), H, W, range_, mv)
    return mv.reshape(nby, nbx, 2)


def huffman_cost(freq):
    """(cost, longest code) of an optimal prefix code for the frequencies (§3.9)."""
    f = np.ascontiguousarray(freq, dtype=np.uint64)
    d = ctypes.c_int(0)
    cost = lib().or_huffman_cost(f, f.size, ctypes.byref(d))
    return int(cost), d.value


def cdf97():
    h = np.zeros(9)
    g = np.zeros(7)
    lib().or_cdf97(h, g)
    return h, g


def modulus(L, k):
    return lib().or_modulus(L, _ints(k))


def layout(H, W, L, k):
    lay = _Layout()
    st = lib().or_layout_make(H, W, L, _ints(k), ctypes.byref(lay))
    if st:
        raise ValueError("layout: invalid arguments (status %d)" % st)
    subs = [dict(off=lay.sb[i].off, h=lay.sb[i].h, w=lay.sb[i].w, level=lay.sb[i].level,
                 dir=lay.sb[i].dir, kind=lay.sb[i].kind) for i in range(lay.nsub)]
    return dict(H=H, W=W, L=L, k=list(k), subbands=subs, total=lay.total)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def lp_analysis(x):
    x = _f64(x)
    H, W = x.shape
    c = np.zeros((H // 2, W // 2))
    d = np.zeros((H, W))
    lib().or_lp_analysis(x, H, W, c, d)
    return c, d


def lp_synthesis(c, d):
    c, d = _f64(c), _f64(d)
    H, W = d.shape
    x = np.zeros((H, W))
    lib().or_lp_synthesis(c, d, H, W, x)
    return x


def lp_analysis_adjoint(cbar, dbar):
    cbar, dbar = _f64(cbar), _f64(dbar)
    H, W = dbar.shape
    x = np.zeros((H, W))
    lib().or_lp_analysis_adjoint(cbar, dbar, H, W, x)
    return x


def lp_synthesis_adjoint(xbar):
    xbar = _f64(xbar)
    H, W = xbar.shape
    c = np.zeros((H // 2, W // 2))
    d = np.zeros((H, W))
    lib().or_lp_synthesis_adjoint(xbar, H, W, c, d)
    return c, d


def dfb(mode, x, H, W, k, taps=4):
    """mode 0/3: x is an H x W plane, returns concatenated subbands (1-D);
    mode 1/2: x is the concatenated subbands, returns the H x W plane.
    taps: the prototype's length (4, 6 or 8)."""
    x = _f64(x).ravel()
    out = np.zeros(H * W)
    st = lib().or_dfb_taps(mode, x, H, W, k, taps, out)
    if st:
        raise ValueError("dfb: invalid arguments")
    return out if mode in (0, 3) else out.reshape(H, W)


def ct(mode, x, H, W, L, k, taps=4):
    """mode 0/3: plane -> coefficient vector; mode 1/2: coefficient vector -> plane."""
    lay = layout(H, W, L, k)
    x = _f64(x).ravel()
    n_out = lay["total"] if mode in (0, 3) else H * W
    out = np.zeros(n_out)
    st = lib().or_ct_taps(mode, x, H, W, L, _ints(k), taps, out)
    if st:
        raise ValueError("ct: invalid arguments")
    return out if mode in (0, 3) else out.reshape(H, W)


def _layout_struct(H, W, L, k):
    lay = _Layout()
    if lib().or_layout_make(H, W, L, _ints(k), ctypes.byref(lay)):
        raise ValueError("layout: invalid arguments")
    return lay


def soft_threshold(c, H, W, L, k, T):
    """Per-subband soft threshold of coefficient vectors c (batch, total) or (total,)."""
    lay = _layout_struct(H, W, L, k)
    c = _f64(c)
    batch = c.size // lay.total
    y = np.zeros(c.size)
    lib().or_soft_threshold(c.ravel(), ctypes.byref(lay), batch, _f64(T).ravel(), y)
    return y.reshape(c.shape)


def soft_threshold_vjp(c, H, W, L, k, T, g):
    """(dL/dc, dL/dT) of the soft threshold for upstream gradient g = dL/dy."""
    lay = _layout_struct(H, W, L, k)
    c = _f64(c)
    batch = c.size // lay.total
    gc = np.zeros(c.size)
    gT = np.zeros(lay.nsub - 1)
    lib().or_soft_threshold_vjp(c.ravel(), ctypes.byref(lay), batch, _f64(T).ravel(), _f64(g).ravel(), gc, gT)
    return gc.reshape(c.shape), gT


def threshold_loss(x, L, k, T, want_grad=True):
    """Loss of thresholded reconstruction, mean over all pixels of
    (S(soft_T(A x)) - x)^2 for planes x (batch, H, W), and its gradients
    (dL/dT, dL/dx) by the chain rule through the adjoint transforms:
    r = S y - x;  dL/dy = S^T (2 r / N);  (dL/dc, dL/dT) = vjp;  dL/dx = A^T dL/dc - 2 r / N."""
    x = _f64(x)
    B, H, W = x.shape
    N = x.size
    c = np.stack([ct(MODE_FORWARD, x[b], H, W, L, k) for b in range(B)])
    y = soft_threshold(c, H, W, L, k, T)
    r = np.stack([ct(MODE_INVERSE, y[b], H, W, L, k) for b in range(B)]) - x
    loss = float(np.sum(r * r) / N)
    if not want_grad:
        return loss
    gxh = 2.0 * r / N
    gy = np.stack([ct(MODE_INVERSE_ADJOINT, gxh[b], H, W, L, k) for b in range(B)])
    gc, gT = soft_threshold_vjp(c, H, W, L, k, T, gy)
    gx = np.stack([ct(MODE_FORWARD_ADJOINT, gc[b], H, W, L, k) for b in range(B)]) - gxh
    return loss, gT, gx


def ycocgr_forward(rgb):
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    n = rgb.size // 3
    y, co, cg = (np.zeros(n, np.int16) for _ in range(3))
    lib().or_ycocgr_forward(rgb.reshape(-1), n, y, co, cg)
    shp = rgb.shape[:-1]
    return y.reshape(shp), co.reshape(shp), cg.reshape(shp)


def ycocgr_inverse(y, co, cg):
    y, co, cg = (np.ascontiguousarray(a, dtype=np.int16) for a in (y, co, cg))
    n = y.size
    rgb = np.zeros(n * 3, np.uint8)
    lib().or_ycocgr_inverse(y.reshape(-1), co.reshape(-1), cg.reshape(-1), n, rgb)
    return rgb.reshape(y.shape + (3,))


def ycocg8_forward(rgb):
    """Table 1, real-valued, 8-bit storage: (Y, Co + 127, Cg + 127) as bytes in int16 arrays"""
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    n = rgb.size // 3
    y, co, cg = (np.zeros(n, np.int16) for _ in range(3))
    lib().or_ycocg8_forward(rgb.reshape(-1), n, y, co, cg)
    shp = rgb.shape[:-1]
    return y.reshape(shp), co.reshape(shp), cg.reshape(shp)


def ycocg8_inverse(y, co, cg):
    y, co, cg = (np.ascontiguousarray(a, dtype=np.int16) for a in (y, co, cg))
    n = y.size
    rgb = np.zeros(n * 3, np.uint8)
    lib().or_ycocg8_inverse(y.reshape(-1), co.reshape(-1), cg.reshape(-1), n, rgb)
    return rgb.reshape(y.shape + (3,))


def chroma_down(p):
    p = np.ascontiguousarray(p, dtype=np.int16)
    H, W = p.shape
    out = np.zeros(((H + 1) // 2, (W + 1) // 2), np.int16)
    lib().or_chroma_down(p, H, W, out)
    return out


def chroma_up(p, H, W):
    p = np.ascontiguousarray(p, dtype=np.int16)
    Hc, Wc = p.shape
    out = np.zeros((H, W), np.int16)
    lib().or_chroma_up(p, Hc, Wc, H, W, out)
    return out


def pad_mirror(p, Hp, Wp):
    p = _f64(p)
    H, W = p.shape
    out = np.zeros((Hp, Wp))
    lib().or_pad_mirror(p, H, W, Hp, Wp, out)
    return out


def quantize(c, qp, threshold, is_lowpass, levels):
    ovf = ctypes.c_int(0)
    q = lib().or_quantize(ctypes.c_float(c), qp, ctypes.c_float(threshold), int(is_lowpass), levels,
                          ctypes.byref(ovf))
    if ovf.value:
        raise OverflowError("quantised code outside int16")
    return q


def quantize8(c, qp, threshold, is_lowpass, levels):
    """the quantiser under 8-bit storage (the coefficient rounded and clamped to a byte first)"""
    return lib().or_quantize8(ctypes.c_float(c), qp, ctypes.c_float(threshold), int(is_lowpass), levels)


def rle_row(row):
    row = np.ascontiguousarray(row, dtype=np.int16)
    tok = np.zeros(2 * row.size + 2, np.int16)
    n = lib().or_rle_row(row, row.size, tok)
    return tok[:n].copy()


def rle_expand(tokens, n):
    tokens = np.ascontiguousarray(tokens, dtype=np.int16)
    out = np.zeros(n, np.int16)
    st = lib().or_rle_expand(tokens, tokens.size, out, n)
    if st:
        raise ValueError("corrupt token stream")
    return out


class Codec:
    """The oracle codec: one video stream, encoder and decoder state."""

    def __init__(self, width, height, levels, dirs_log2, qph, qpl=None, threshold=0.0, key_interval=10,
                 motion_range=0, storage8=False, dfb_taps=4):
        if qpl is None:
            qpl = max(1, qph // 14)
        self.width, self.height, self.levels = width, height, levels
        self.dirs = list(dirs_log2)
        self.qph, self.qpl, self.threshold, self.key_interval = qph, qpl, threshold, key_interval
        self.motion_range = motion_range
        self._h = lib().or_codec_create(width, height, levels, _ints(self.dirs), qph, qpl,
                                        ctypes.c_float(threshold), key_interval)
        if not self._h:
            raise ValueError("oracle codec: invalid parameters")
        if lib().or_codec_set_motion(self._h, motion_range):
            raise ValueError("oracle codec: invalid motion range")
        self.storage8 = bool(storage8)
        lib().or_codec_set_storage8(self._h, int(self.storage8))
        self.dfb_taps = dfb_taps
        if lib().or_codec_set_taps(self._h, dfb_taps):
            raise ValueError("oracle codec: invalid DFB prototype length")
        self.ncoef = lib().or_codec_coeff_count(self._h)
        self.ncomp = lib().or_codec_ncomp(self._h)
        self.max_stream = lib().or_codec_max_stream(self._h)
        d = (ctypes.c_int * 4)()
        lib().or_codec_dims(self._h, d)
        self.Hp, self.Wp, self.Hcp, self.Wcp = list(d)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_codec_destroy(h)
            self._h = None

    def reset(self):
        lib().or_codec_reset(self._h)

    def planes(self, rgb):
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        y = np.zeros((self.Hp, self.Wp))
        co = np.zeros((self.Hcp, self.Wcp))
        cg = np.zeros((self.Hcp, self.Wcp))
        lib().or_codec_planes(self._h, rgb.reshape(-1), y, co, cg)
        return y, co, cg

    def encode(self, rgb, want_coeffs=False):
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        out = np.zeros(self.max_stream, np.uint8)
        n = ctypes.c_long(0)
        ft = ctypes.c_int(0)
        co = np.zeros(self.ncoef) if want_coeffs else None
        st = lib().or_encode(self._h, rgb.reshape(-1), out, out.size, ctypes.byref(n), ctypes.byref(ft),
                             co.ctypes.data if co is not None else None)
        if st:
            raise RuntimeError("oracle encode failed: status %d" % st)
        res = (out[:n.value].copy(), ft.value)
        return res + (co,) if want_coeffs else res

    def encode_from_coeffs(self, coeffs_f32, luma=None):
        """The entropy side from given coefficients; `luma` (the frame's padded luma plane,
        Hp x Wp, values 0..255) is needed by a codec with a motion range."""
        cf = np.ascontiguousarray(coeffs_f32, dtype=np.float32).ravel()
        assert cf.size == self.ncoef
        out = np.zeros(self.max_stream, np.uint8)
        n = ctypes.c_long(0)
        ft = ctypes.c_int(0)
        if luma is not None:
            lu = np.ascontiguousarray(luma, dtype=np.uint8).ravel()
            assert lu.size == self.Hp * self.Wp
            st = lib().or_encode_from_coeffs_luma(self._h, cf, lu, out, out.size, ctypes.byref(n), ctypes.byref(ft))
        else:
            st = lib().or_encode_from_coeffs(self._h, cf, out, out.size, ctypes.byref(n), ctypes.byref(ft))
        if st:
            raise RuntimeError("oracle encode failed: status %d" % st)
        return out[:n.value].copy(), ft.value

    def decode(self, stream, want_planes=False, scale=0):
        """Decode one frame; scale s > 0 reconstructs the level-s approximation (§3.3) as
        ceil(H/2^s) x ceil(W/2^s) RGB from the lowpass and levels s+1..L."""
        s = np.ascontiguousarray(stream, dtype=np.uint8)
        f = 1 << scale
        h, w = (self.height + f - 1) // f, (self.width + f - 1) // f
        Hp, Wp, Hcp, Wcp = self.Hp >> scale, self.Wp >> scale, self.Hcp >> scale, self.Wcp >> scale
        rgb = np.zeros((h, w, 3), np.uint8)
        pl = np.zeros(Hp * Wp + 2 * Hcp * Wcp) if want_planes else None
        st = lib().or_decode_scaled(self._h, s, s.size, scale, rgb.reshape(-1),
                                    pl.ctypes.data if pl is not None else None)
        if st:
            raise RuntimeError("oracle decode failed: status %d" % st)
        if want_planes:
            ny, nc = Hp * Wp, Hcp * Wcp
            return rgb, (pl[:ny].reshape(Hp, Wp), pl[ny:ny + nc].reshape(Hcp, Wcp), pl[ny + nc:].reshape(Hcp, Wcp))
        return rgb

    def drop_levels(self, stream, drop):
        """The frame without its finest `drop` levels (§3.3); raises on a bad stream or drop."""
        s = np.ascontiguousarray(stream, dtype=np.uint8)
        out = np.zeros(max(1, s.size), np.uint8)
        n = ctypes.c_long(0)
        st = lib().or_stream_drop(self._h, s, s.size, drop, out, out.size, ctypes.byref(n))
        if st:
            raise RuntimeError("oracle stream drop failed: status %d" % st)
        return out[:n.value].copy()

    def inflate_container(self, packed):
        """The frame inside a deflated frame, inflated stream by stream with zlib."""
        s = np.ascontiguousarray(packed, dtype=np.uint8)
        cap = max(1, self.max_stream)
        out = np.zeros(cap, np.uint8)
        n = ctypes.c_long(0)
        st = lib().or_inflate_container(self._h, s, s.size, out, cap, ctypes.byref(n))
        if st:
            raise RuntimeError("oracle inflate failed: status %d" % st)
        return out[:n.value].copy()

    def decode_status(self, stream):
        s = np.ascontiguousarray(stream, dtype=np.uint8)
        rgb = np.zeros((self.height, self.width, 3), np.uint8)
        return lib().or_decode(self._h, s, s.size, rgb.reshape(-1), None)
