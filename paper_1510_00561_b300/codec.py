"""Python front end of libcvc: the contourlet transform plan and the video codec.

PyTorch provides device memory and streams; every step of the transform and
of the codec runs in the library's CUDA kernels (see include/cvc.h).
"""
import ctypes

import torch

from . import _lib as _L


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def kernel_launches():
    """Kernels libcvc has launched in this process."""
    return int(_L.lib().cvc_kernel_launches())


def modulus(levels, dirs_log2):
    return _L.lib().cvc_modulus(levels, _L.ints(dirs_log2))


def ct_layout(h, w, levels, dirs_log2):
    """Coefficient layout of one h x w plane: dict(total, modulus, subbands=[...])."""
    lay = _L.CtLayout()
    _L.check(_L.lib().cvc_ct_layout(h, w, levels, _L.ints(dirs_log2), ctypes.byref(lay)), "cvc_ct_layout")
    subs = [dict(off=lay.sub[i].off, h=lay.sub[i].h, w=lay.sub[i].w, level=lay.sub[i].level,
                 dir=lay.sub[i].dir, kind=lay.sub[i].kind) for i in range(lay.nsub)]
    return dict(total=lay.total, modulus=lay.modulus, subbands=subs)


class CtPlan:
    """Contourlet transform of `batch` dense h x w float32 planes (§2.1).

    forward: x (batch, h, w) -> coefficients (batch, total)
    inverse: coefficients -> x;  forward_adjoint / inverse_adjoint: the transposes.
    """

    def __init__(self, h, w, levels, dirs_log2, batch=1):
        self.h, self.w, self.levels, self.dirs = h, w, levels, list(dirs_log2)
        self.batch = batch
        p = ctypes.c_void_p()
        _L.check(_L.lib().cvc_ct_plan_create(h, w, levels, _L.ints(dirs_log2), batch, ctypes.byref(p)),
                 "cvc_ct_plan_create")
        self._h = p
        self.total = _L.lib().cvc_ct_plan_coeffs(p)
        self.layout = ct_layout(h, w, levels, dirs_log2)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _L._lib is not None:
            _L.lib().cvc_ct_plan_destroy(h)
            self._h = None

    def _run(self, fn, src, shape_in, shape_out, out):
        if not (src.is_cuda and src.dtype == torch.float32 and src.is_contiguous()):
            raise ValueError("expected a contiguous float32 CUDA tensor")
        if tuple(src.shape) != shape_in:
            raise ValueError("expected shape %s, got %s" % (shape_in, tuple(src.shape)))
        if out is None:
            out = torch.empty(shape_out, dtype=torch.float32, device=src.device)
        _L.check(getattr(_L.lib(), fn)(self._h, _ptr(src), _ptr(out), _stream()), fn)
        return out

    def forward(self, x, out=None):
        return self._run("cvc_ct_forward", x, (self.batch, self.h, self.w), (self.batch, self.total), out)

    def inverse(self, c, out=None):
        return self._run("cvc_ct_inverse", c, (self.batch, self.total), (self.batch, self.h, self.w), out)

    def forward_adjoint(self, cbar, out=None):
        return self._run("cvc_ct_forward_adjoint", cbar, (self.batch, self.total), (self.batch, self.h, self.w), out)

    def inverse_adjoint(self, xbar, out=None):
        return self._run("cvc_ct_inverse_adjoint", xbar, (self.batch, self.h, self.w), (self.batch, self.total), out)


class Codec:
    """One CVC video stream on the GPU (encoder and decoder state resident in HBM)."""

    def __init__(self, width, height, levels, dirs_log2, qph, qpl=None, threshold=0.0, key_interval=10):
        if qpl is None:
            qpl = max(1, qph // 14)
        self.width, self.height, self.levels, self.dirs = width, height, levels, list(dirs_log2)
        self.qph, self.qpl, self.threshold, self.key_interval = qph, qpl, threshold, key_interval
        prm = _L.Params(width, height, levels, _L.ints(dirs_log2), qph, qpl, threshold, key_interval, 1)
        p = ctypes.c_void_p()
        _L.check(_L.lib().cvc_create(ctypes.byref(prm), ctypes.byref(p)), "cvc_create")
        self._h = p
        info = _L.CodecInfo()
        _L.check(_L.lib().cvc_codec_info(p, ctypes.byref(info)), "cvc_codec_info")
        self.Hp, self.Wp = info.padded_height, info.padded_width
        self.Hc, self.Wc = info.chroma_height, info.chroma_width
        self.Hcp, self.Wcp = info.padded_chroma_height, info.padded_chroma_width
        self.ncoef, self.ncomp, self.max_stream = info.coeffs, info.components, info.max_stream_bytes
        self.nplane = self.Hp * self.Wp + 2 * self.Hcp * self.Wcp

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _L._lib is not None:
            _L.lib().cvc_destroy(h)
            self._h = None

    def reset(self):
        _L.check(_L.lib().cvc_reset(self._h), "cvc_reset")

    def encode(self, rgb, out=None, stream=None):
        """rgb: (H, W, 3) uint8 CUDA tensor (rows may be strided).  Returns (bytes view, frame_type)."""
        if not (rgb.is_cuda and rgb.dtype == torch.uint8 and rgb.dim() == 3 and rgb.shape[2] == 3
                and rgb.stride(2) == 1 and rgb.stride(1) == 3):
            raise ValueError("expected an (H, W, 3) uint8 CUDA tensor with interleaved channels")
        if out is None:
            out = torch.empty(self.max_stream, dtype=torch.uint8, device=rgb.device)
        n = ctypes.c_size_t(0)
        ft = ctypes.c_int(0)
        st = _L.lib().cvc_encode_frame(self._h, _ptr(rgb), rgb.stride(0), _ptr(out), out.numel(), ctypes.byref(n),
                                       ctypes.byref(ft), _stream(stream))
        if st != 0:
            err = _L.CvcError(st, "cvc_encode_frame")
            err.needed = n.value
            raise err
        return out[:n.value], ft.value

    def decode(self, stream_bytes, out=None, stream=None):
        """stream_bytes: uint8 CUDA tensor holding one encoded frame.  Returns (H, W, 3) uint8."""
        if not (stream_bytes.is_cuda and stream_bytes.dtype == torch.uint8 and stream_bytes.is_contiguous()):
            raise ValueError("expected a contiguous uint8 CUDA tensor")
        if out is None:
            out = torch.empty((self.height, self.width, 3), dtype=torch.uint8, device=stream_bytes.device)
        _L.check(_L.lib().cvc_decode_frame(self._h, _ptr(stream_bytes), stream_bytes.numel(), _ptr(out),
                                           out.stride(0), _stream(stream)), "cvc_decode_frame")
        return out

    def inspect(self, which):
        """0: encoder padded planes, 1: encoder coefficients, 2: decoder reconstructed planes (float32)."""
        n = self.ncoef if which == 1 else self.nplane
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        _L.check(_L.lib().cvc_codec_inspect(self._h, which, _ptr(out), n, _stream()), "cvc_codec_inspect")
        return out

    def set_timing(self, on=True):
        """Per-stage CUDA-event timing of encode / decode (see cvc_codec_set_timing)."""
        _L.check(_L.lib().cvc_codec_set_timing(self._h, int(bool(on))), "cvc_codec_set_timing")

    def timing(self):
        """dict stage -> (milliseconds, kernel launches) accumulated since set_timing(True)."""
        ms = (ctypes.c_double * _L.NUM_STAGES)()
        n = (ctypes.c_longlong * _L.NUM_STAGES)()
        _L.check(_L.lib().cvc_codec_timing(self._h, ms, n), "cvc_codec_timing")
        return {name: (ms[i], n[i]) for i, name in enumerate(_L.STAGE_NAMES)}

    def split_planes(self, flat):
        ny, nc = self.Hp * self.Wp, self.Hcp * self.Wcp
        return (flat[:ny].view(self.Hp, self.Wp), flat[ny:ny + nc].view(self.Hcp, self.Wcp),
                flat[ny + nc:].view(self.Hcp, self.Wcp))
