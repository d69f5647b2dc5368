"""Python front end of libcvc: the contourlet transform plan and the video codec.

PyTorch provides device memory and streams; every step of the transform and
of the codec runs in the library's CUDA kernels (see include/cvc.h).
"""
import ctypes

import numpy as np
import torch

from . import _lib as _L


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _opt(t, dtype):
    """device pointer of an optional one-element CUDA tensor of `dtype`"""
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.numel() >= 1):
        raise ValueError("expected a CUDA tensor of %s" % dtype)
    return t.data_ptr()


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

    def __init__(self, h, w, levels, dirs_log2, batch=1, dfb_taps=4):
        self.h, self.w, self.levels, self.dirs = h, w, levels, list(dirs_log2)
        self.batch, self.dfb_taps = batch, dfb_taps
        p = ctypes.c_void_p()
        _L.check(_L.lib().cvc_ct_plan_create_taps(h, w, levels, _L.ints(dirs_log2), batch, dfb_taps,
                                                  ctypes.byref(p)), "cvc_ct_plan_create_taps")
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

    def set_fusion(self, levels):
        """cvc_ct_plan_set_fusion: the most coarse levels of each plane in one block (0: none)"""
        _L.check(_L.lib().cvc_ct_plan_set_fusion(self._h, int(levels)), "cvc_ct_plan_set_fusion")

    @property
    def subbands(self):
        """Number of directional subbands (one soft threshold each)."""
        return _L.lib().cvc_ct_plan_subbands(self._h)

    def _check_coeffs(self, t):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and tuple(t.shape) == (self.batch, self.total)):
            raise ValueError("expected contiguous float32 CUDA coefficients of shape %s" % ((self.batch, self.total),))

    def _check_thresholds(self, T):
        if not (T.is_cuda and T.dtype == torch.float32 and T.is_contiguous() and T.numel() == self.subbands):
            raise ValueError("expected %d contiguous float32 CUDA thresholds" % self.subbands)

    def soft_threshold(self, c, T, out=None):
        """sign(c) max(|c| - T[s], 0) per directional subband s; lowpass unchanged."""
        self._check_coeffs(c)
        self._check_thresholds(T)
        if out is None:
            out = torch.empty_like(c)
        _L.check(_L.lib().cvc_ct_soft_threshold(self._h, _ptr(c), _ptr(T), _ptr(out), _stream()),
                 "cvc_ct_soft_threshold")
        return out

    def soft_threshold_backward(self, c, T, grad_out):
        """(dL/dc, dL/dT) of soft_threshold for the upstream gradient dL/dy."""
        self._check_coeffs(c)
        self._check_coeffs(grad_out)
        self._check_thresholds(T)
        gc = torch.empty_like(c)
        gT = torch.empty_like(T)
        _L.check(_L.lib().cvc_ct_soft_threshold_backward(self._h, _ptr(c), _ptr(T), _ptr(grad_out), _ptr(gc),
                                                         _ptr(gT), _stream()), "cvc_ct_soft_threshold_backward")
        return gc, gT


class Codec:
    """One CVC video stream on the GPU (encoder and decoder state resident in HBM)."""

    def __init__(self, width, height, levels, dirs_log2, qph, qpl=None, threshold=0.0, key_interval=10,
                 motion_range=0, storage8=False, dfb_taps=4):
        prm = _L.params(width, height, levels, dirs_log2, qph, qpl, threshold, key_interval, motion_range, storage8,
                        dfb_taps)
        self.width, self.height, self.levels, self.dirs = width, height, levels, list(dirs_log2)
        self.qph, self.qpl, self.threshold, self.key_interval = qph, prm.qpl, threshold, key_interval
        self.motion_range, self.storage8, self.dfb_taps = motion_range, bool(storage8), dfb_taps
        self._prm = prm
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

    def encode_async(self, rgb, out, out_len=None, frame_type=None, status=None, stream=None):
        """cvc_encode_frame_async: queue the encode of rgb into out (uint8 CUDA tensor) without
        waiting; the device writes the length, frame type and status into the given CUDA tensors
        (int64 / int32 / int32 of one element each, or None)."""
        if not (rgb.is_cuda and rgb.dtype == torch.uint8 and rgb.dim() == 3 and rgb.shape[2] == 3
                and rgb.stride(2) == 1 and rgb.stride(1) == 3):
            raise ValueError("expected an (H, W, 3) uint8 CUDA tensor with interleaved channels")
        _L.check(_L.lib().cvc_encode_frame_async(self._h, _ptr(rgb), rgb.stride(0), _ptr(out), out.numel(),
                                                 _opt(out_len, torch.int64), _opt(frame_type, torch.int32),
                                                 _opt(status, torch.int32), _stream(stream)),
                 "cvc_encode_frame_async")

    def decode_async(self, stream_bytes, out, in_len=None, status=None, scale=0, stream=None):
        """cvc_decode_frame_async: queue the decode of stream_bytes (uint8 CUDA tensor, its whole
        size the capacity) into out; in_len (int64 CUDA tensor of one element, e.g. an encode's
        out_len) gives the frame's length on the device; status receives the decoder's status."""
        if not (stream_bytes.is_cuda and stream_bytes.dtype == torch.uint8 and stream_bytes.is_contiguous()):
            raise ValueError("expected a contiguous uint8 CUDA tensor")
        _L.check(_L.lib().cvc_decode_frame_async(self._h, _ptr(stream_bytes), stream_bytes.numel(),
                                                 _opt(in_len, torch.int64), int(scale), _ptr(out), out.stride(0),
                                                 _opt(status, torch.int32), _stream(stream)),
                 "cvc_decode_frame_async")

    def get_error(self, stream=None):
        """cvc_get_error: the first failure of an asynchronous call since the last read (0: none)."""
        v = ctypes.c_int(0)
        _L.check(_L.lib().cvc_get_error(self._h, _stream(stream), ctypes.byref(v)), "cvc_get_error")
        return v.value

    def scaled_size(self, scale):
        """(height, width) of the decoder's output at pyramid scale `scale`."""
        f = 1 << scale
        return (self.height + f - 1) // f, (self.width + f - 1) // f

    def decode(self, stream_bytes, out=None, stream=None, scale=0):
        """stream_bytes: uint8 CUDA tensor holding one encoded frame.  Returns (H, W, 3) uint8,
        or the frame at pyramid scale `scale` (ceil(H / 2^scale) x ceil(W / 2^scale),
        cvc_decode_frame_scaled)."""
        if not (stream_bytes.is_cuda and stream_bytes.dtype == torch.uint8 and stream_bytes.is_contiguous()):
            raise ValueError("expected a contiguous uint8 CUDA tensor")
        if out is None:
            h, w = self.scaled_size(scale) if 0 <= scale <= self.levels else (1, 1)
            out = torch.empty((h, w, 3), dtype=torch.uint8, device=stream_bytes.device)
        _L.check(_L.lib().cvc_decode_frame_scaled(self._h, _ptr(stream_bytes), stream_bytes.numel(), int(scale),
                                                  _ptr(out), out.stride(0), _stream(stream)),
                 "cvc_decode_frame_scaled")
        return out

    def drop_levels(self, stream_bytes, drop):
        """The frame without its finest `drop` levels (cvc_stream_drop_levels, host memory):
        stream_bytes is a host uint8 array or CPU tensor; returns a numpy uint8 array that
        decodes at scales >= drop."""
        return drop_levels(self._prm, stream_bytes, drop)

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


def drop_levels(params, stream_bytes, drop):
    """cvc_stream_drop_levels for a frame of a stream with `params` (a cvc_params or a dict of
    Codec keyword arguments); host bytes in, numpy uint8 out."""
    if isinstance(params, dict):
        params = _L.params(**params)
    if isinstance(stream_bytes, torch.Tensor):
        stream_bytes = stream_bytes.cpu().numpy()
    src = np.ascontiguousarray(stream_bytes, dtype=np.uint8)
    out = np.empty(max(1, src.size), np.uint8)
    n = ctypes.c_size_t(0)
    _L.check(_L.lib().cvc_stream_drop_levels(ctypes.byref(params), src.ctypes.data, src.size, int(drop),
                                             out.ctypes.data, out.size, ctypes.byref(n)),
             "cvc_stream_drop_levels")
    return out[:n.value].copy()


class Deflater:
    """The DEFLATE stage (§3.9) for frames of one parameter set: Huffman-only
    DEFLATE streams on the GPU (cvc_deflate_*), one per component (scalable
    mode) or, with nts=True, one per frame (CVC-NTS).  Inflate reads both."""

    def __init__(self, max_frames=1, nts=False, **stream):
        prm = _L.params(**stream)
        p = ctypes.c_void_p()
        _L.check(_L.lib().cvc_deflate_create_batch(ctypes.byref(prm), int(max_frames), ctypes.byref(p)),
                 "cvc_deflate_create_batch")
        self._h = p
        self.max_frames = max_frames
        self.nts = bool(nts)
        _L.check(_L.lib().cvc_deflate_set_nts(p, int(self.nts)), "cvc_deflate_set_nts")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _L._lib is not None:
            _L.lib().cvc_deflate_destroy(h)
            self._h = None

    def _run(self, fn, name, src, out, guess, stream):
        if not (src.is_cuda and src.dtype == torch.uint8 and src.is_contiguous()):
            raise ValueError("expected a contiguous uint8 CUDA tensor")
        n = ctypes.c_size_t(0)
        for _ in range(2):
            o = out if out is not None else torch.empty(max(16, guess), dtype=torch.uint8, device=src.device)
            st = fn(self._h, _ptr(src), src.numel(), _ptr(o), o.numel(), ctypes.byref(n), _stream(stream))
            if st == 3 and out is None:          # too small: once more with the size needed
                guess = n.value
                continue
            _L.check(st, name)
            return o[:n.value]
        _L.check(st, name)

    def deflate(self, frame, out=None, stream=None):
        """frame: uint8 CUDA tensor of one encoded frame; returns the deflated frame (a view of out)."""
        return self._run(_L.lib().cvc_deflate_frame, "cvc_deflate_frame", frame, out,
                         frame.numel() + frame.numel() // 4 + 65536, stream)

    def inflate(self, packed, out=None, stream=None):
        """the frame inside a deflated frame (uint8 CUDA tensors)."""
        return self._run(_L.lib().cvc_inflate_frame, "cvc_inflate_frame", packed, out, 8 * packed.numel() + 65536,
                         stream)

    def _many(self, fn, name, srcs, outs, stream):
        n = len(srcs)
        P, Z = ctypes.c_void_p * n, ctypes.c_size_t * n
        lens, sts = Z(), (ctypes.c_int * n)()
        st = fn(self._h, n, P(*[_ptr(x) for x in srcs]), Z(*[x.numel() for x in srcs]), P(*[_ptr(o) for o in outs]),
                Z(*[o.numel() for o in outs]), lens, sts, _stream(stream))
        if st in (1, 6):
            raise _L.CvcError(st, name)
        return [o[:lens[i]] if sts[i] == 0 else None for i, o in enumerate(outs)], list(sts)

    def deflate_many(self, frames, outs, stream=None):
        """deflate up to max_frames frames in one launch sequence (cvc_deflate_frames);
        returns (views of outs, per-frame statuses)."""
        return self._many(_L.lib().cvc_deflate_frames, "cvc_deflate_frames", frames, outs, stream)

    def inflate_many(self, packed, outs, stream=None):
        """inflate up to max_frames deflated frames in one launch sequence (cvc_inflate_frames)."""
        return self._many(_L.lib().cvc_inflate_frames, "cvc_inflate_frames", packed, outs, stream)


def _info(fn, h, i=None):
    info = _L.CodecInfo()
    args = (h, i, ctypes.byref(info)) if i is not None else (h, ctypes.byref(info))
    _L.check(fn(*args), fn.__name__)
    return info


class Batch:
    """Many CVC streams coded together: one graph-replayed launch sequence per step.

    streams: list of dicts with the Codec constructor's keyword arguments
    (width, height, levels, dirs_log2, qph, qpl, threshold, key_interval).
    Each stream's output is bit-identical to a Codec of the same parameters.
    """

    def __init__(self, streams):
        self.streams = [dict(s) for s in streams]
        n = len(self.streams)
        arr = (_L.Params * n)(*[_L.params(**s) for s in self.streams])
        self._params = arr
        p = ctypes.c_void_p()
        _L.check(_L.lib().cvc_batch_create(arr, n, ctypes.byref(p)), "cvc_batch_create")
        self._h = p
        self.n = n
        self.info = [_info(_L.lib().cvc_batch_info, p, i) for i in range(n)]
        self._io = (_L.BatchIo * n)()
        self._res = (_L.BatchResult * n)()
        self._out = [None] * n

    @staticmethod
    def device_bytes(streams):
        """Device bytes a batch of these streams would allocate (no device call)."""
        arr = (_L.Params * len(streams))(*[_L.params(**s) for s in streams])
        b = ctypes.c_size_t(0)
        _L.check(_L.lib().cvc_batch_device_bytes(arr, len(streams), ctypes.byref(b)), "cvc_batch_device_bytes")
        return b.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _L._lib is not None:
            _L.lib().cvc_batch_destroy(h)
            self._h = None

    def reset(self, i=-1):
        _L.check(_L.lib().cvc_batch_reset(self._h, i), "cvc_batch_reset")

    def out_buffer(self, i, device="cuda"):
        """A persistent bitstream buffer of stream i (worst-case size)."""
        if self._out[i] is None:
            self._out[i] = torch.empty(self.info[i].max_stream_bytes, dtype=torch.uint8, device=device)
        return self._out[i]

    def _fill(self, rgb, streams_in, rgb_out, outs):
        for i in range(self.n):
            io = self._io[i]
            x = rgb[i] if rgb is not None else None
            io.d_rgb = x.data_ptr() if x is not None else None
            io.pitch_bytes = x.stride(0) if x is not None else 0
            o = outs[i] if outs is not None and outs[i] is not None else (self.out_buffer(i) if x is not None
                                                                           else None)
            io.d_out = o.data_ptr() if o is not None else None
            io.out_cap = o.numel() if o is not None else 0
            b = streams_in[i] if streams_in is not None else None
            io.d_in = b.data_ptr() if b is not None else None
            io.in_len = b.numel() if b is not None else 0
            y = rgb_out[i] if rgb_out is not None else None
            io.d_rgb_out = y.data_ptr() if y is not None else None
            io.pitch_out = y.stride(0) if y is not None else 0

    def scaled_size(self, i, scale):
        """(height, width) of stream i's decoder output at pyramid scale `scale`."""
        f = 1 << scale
        s = self.streams[i]
        return (s["height"] + f - 1) // f, (s["width"] + f - 1) // f

    def step(self, what, rgb=None, streams_in=None, rgb_out=None, outs=None, stream=None, check=True, scale=0):
        """One step over every stream (entries None take no part).

        what: 1 encode, 2 decode, 3 encode + decode of the step's own output.
        scale: pyramid scale of every decoder output (cvc_batch_step_scaled).
        Returns a list of per-stream dicts (statuses, out_len, frame types,
        the encoded bytes as a view of the stream's output buffer)."""
        self._fill(rgb, streams_in, rgb_out, outs)
        st = _L.lib().cvc_batch_step_scaled(self._h, what, self._io, int(scale), self._res, _stream(stream))
        if st in (1, 6):
            raise _L.CvcError(st, "cvc_batch_step")
        res = []
        for i in range(self.n):
            r = self._res[i]
            d = dict(enc_status=r.enc_status, dec_status=r.dec_status, out_len=r.out_len,
                     frame_type=r.frame_type, dec_frame_type=r.dec_frame_type, dec_frame_index=r.dec_frame_index)
            if r.frame_type >= 0 and r.enc_status == 0:
                o = outs[i] if outs is not None and outs[i] is not None else self._out[i]
                d["bytes"] = o[:r.out_len]
            res.append(d)
        if check and st != 0:
            raise _L.CvcError(st, "cvc_batch_step")
        return res

    def step_async(self, what, rgb=None, streams_in=None, rgb_out=None, outs=None, in_len=None, results=None,
                   stream=None, scale=0):
        """cvc_batch_step_async: queue one step without waiting.  in_len: int64 CUDA tensor of n
        decoder input lengths (or None: each input's size); results: uint8 CUDA tensor of
        n * sizeof(cvc_batch_result) bytes receiving the per-stream results (see results_of)."""
        self._fill(rgb, streams_in, rgb_out, outs)
        if in_len is not None and not (in_len.is_cuda and in_len.dtype == torch.int64 and in_len.numel() >= self.n):
            raise ValueError("in_len: an int64 CUDA tensor of one length per stream")
        if results is not None and results.numel() < self.n * ctypes.sizeof(_L.BatchResult):
            raise ValueError("results: too small")
        _L.check(_L.lib().cvc_batch_step_async(self._h, what, self._io,
                                               in_len.data_ptr() if in_len is not None else None, int(scale),
                                               results.data_ptr() if results is not None else None,
                                               _stream(stream)), "cvc_batch_step_async")

    def results_buffer(self, device="cuda"):
        """a device buffer for step_async's per-stream results"""
        return torch.zeros(self.n * ctypes.sizeof(_L.BatchResult), dtype=torch.uint8, device=device)

    def results_of(self, buf):
        """the per-stream result dicts held in a results buffer (copied to the host)"""
        raw = bytes(buf.cpu().numpy())
        out = []
        for i in range(self.n):
            r = _L.BatchResult.from_buffer_copy(raw, i * ctypes.sizeof(_L.BatchResult))
            out.append(dict(enc_status=r.enc_status, dec_status=r.dec_status, out_len=r.out_len,
                            frame_type=r.frame_type, dec_frame_type=r.dec_frame_type,
                            dec_frame_index=r.dec_frame_index))
        return out

    def get_error(self, i, stream=None):
        """cvc_batch_get_error for stream i"""
        v = ctypes.c_int(0)
        _L.check(_L.lib().cvc_batch_get_error(self._h, i, _stream(stream), ctypes.byref(v)), "cvc_batch_get_error")
        return v.value

    def set_shape(self, rle_rows, tok_blocks):
        _L.check(_L.lib().cvc_batch_set_shape(self._h, rle_rows, tok_blocks), "cvc_batch_set_shape")

    def set_graphs(self, on):
        _L.check(_L.lib().cvc_batch_set_graphs(self._h, int(bool(on))), "cvc_batch_set_graphs")

    def set_timing(self, on=True):
        _L.check(_L.lib().cvc_batch_set_timing(self._h, int(bool(on))), "cvc_batch_set_timing")

    def timing(self):
        """dict stage -> (milliseconds, kernel launches) accumulated since set_timing(True)."""
        ms = (ctypes.c_double * _L.NUM_STAGES)()
        n = (ctypes.c_longlong * _L.NUM_STAGES)()
        _L.check(_L.lib().cvc_batch_timing(self._h, ms, n), "cvc_batch_timing")
        return {name: (ms[i], n[i]) for i, name in enumerate(_L.STAGE_NAMES)}

    def autotune(self, what, rgb=None, streams_in=None, rgb_out=None, reps=5, stream=None):
        """Time candidate launch shapes, fusion depths and row-split DFB block widths on these
        inputs, keep the fastest; returns (rle_rows, tok_blocks, fusion depth, block width)."""
        self._fill(rgb, streams_in, rgb_out, None)
        shape = (ctypes.c_int * 4)()
        _L.check(_L.lib().cvc_batch_autotune(self._h, what, self._io, reps, shape, _stream(stream)),
                 "cvc_batch_autotune")
        return shape[0], shape[1], shape[2], shape[3]

    def set_fusion(self, levels):
        """cvc_batch_set_fusion: the most coarse levels of each plane in its pyramid tail (0: none)"""
        _L.check(_L.lib().cvc_batch_set_fusion(self._h, int(levels)), "cvc_batch_set_fusion")

    def set_dfb_threads(self, threads):
        """cvc_batch_set_dfb_threads: threads per block of the row-split DFB launches (0: by
        launch size, 128 or 256)"""
        _L.check(_L.lib().cvc_batch_set_dfb_threads(self._h, int(threads)), "cvc_batch_set_dfb_threads")


class Server:
    """Continuous-batching request loop over many streams (cvc_server_*).

    open(**codec kwargs) -> session id (admitted now or when memory frees);
    submit(session, kind, rgb=..., out=..., stream_in=..., rgb_out=..., tag=...)
    queues a request (kind 1 encode, 2 decode, 3 encode + decode of its own
    output); poll() runs the loop and returns completions as dicts.  Request
    buffers must stay alive until their completion is returned.
    """

    def __init__(self, budget_bytes, slots_per_shard=8, steps_in_flight=1):
        cfg = _L.ServerConfig(int(budget_bytes), int(slots_per_shard), int(steps_in_flight))
        p = ctypes.c_void_p()
        _L.check(_L.lib().cvc_server_create(ctypes.byref(cfg), ctypes.byref(p)), "cvc_server_create")
        self._h = p
        self._cpl = (_L.ServerCompletion * 4096)()
        self._keep = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _L._lib is not None:
            _L.lib().cvc_server_destroy(h)
            self._h = None

    @staticmethod
    def now_ns():
        return int(_L.lib().cvc_server_now_ns())

    def open(self, **stream):
        prm = _L.params(**stream)
        sid = ctypes.c_int(-1)
        _L.check(_L.lib().cvc_server_open(self._h, ctypes.byref(prm), ctypes.byref(sid)), "cvc_server_open")
        return sid.value

    def close(self, session):
        _L.check(_L.lib().cvc_server_close(self._h, session), "cvc_server_close")

    def submit(self, session, kind, rgb=None, out=None, stream_in=None, rgb_out=None, tag=0):
        io = _L.BatchIo()
        if rgb is not None:
            io.d_rgb, io.pitch_bytes = rgb.data_ptr(), rgb.stride(0)
        if out is not None:
            io.d_out, io.out_cap = out.data_ptr(), out.numel()
        if stream_in is not None:
            io.d_in, io.in_len = stream_in.data_ptr(), stream_in.numel()
        if rgb_out is not None:
            io.d_rgb_out, io.pitch_out = rgb_out.data_ptr(), rgb_out.stride(0)
        _L.check(_L.lib().cvc_server_submit(self._h, session, kind, ctypes.byref(io), int(tag)), "cvc_server_submit")
        self._keep[int(tag)] = (rgb, out, stream_in, rgb_out)   # alive until completion

    def submit_io(self, session, kind, io, tag):
        """submit with a prepared cvc_batch_io (_lib.BatchIo); the caller keeps its buffers alive"""
        _L.check(_L.lib().cvc_server_submit(self._h, session, kind, ctypes.byref(io), int(tag)), "cvc_server_submit")

    def poll_raw(self, wait_us=0):
        """poll() as (tag, enc_status, dec_status, t_done_ns) tuples, for callers that keep their own buffers"""
        n = ctypes.c_int(0)
        _L.check(_L.lib().cvc_server_poll(self._h, int(wait_us), self._cpl, len(self._cpl), ctypes.byref(n)),
                 "cvc_server_poll")
        c = self._cpl
        return [(c[i].tag, c[i].enc_status, c[i].dec_status, c[i].t_done_ns) for i in range(n.value)]

    def poll(self, wait_us=0):
        n = ctypes.c_int(0)
        _L.check(_L.lib().cvc_server_poll(self._h, int(wait_us), self._cpl, len(self._cpl), ctypes.byref(n)),
                 "cvc_server_poll")
        res = []
        for i in range(n.value):
            c = self._cpl[i]
            self._keep.pop(int(c.tag), None)
            res.append(dict(tag=c.tag, session=c.session, kind=c.kind, enc_status=c.enc_status,
                            dec_status=c.dec_status, out_len=c.out_len, frame_type=c.frame_type,
                            dec_frame_type=c.dec_frame_type, t_submit_ns=c.t_submit_ns,
                            t_launch_ns=c.t_launch_ns, t_done_ns=c.t_done_ns))
        return res

    def stats(self):
        st = _L.ServerStats()
        _L.check(_L.lib().cvc_server_get_stats(self._h, ctypes.byref(st)), "cvc_server_get_stats")
        return {f: getattr(st, f) for f, _ in _L.ServerStats._fields_}
