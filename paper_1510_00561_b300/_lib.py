"""ctypes view of libcvc.so (include/cvc.h).  Argument marshalling only.

The library must have been built (``python -m paper_1510_00561_b300.build``
or ``__graft_entry__.build()``); loading fails loudly otherwise -- there is
no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcvc.so")

MAX_LEVELS = 6
NUM_STAGES = 10
STAGE_NAMES = ("colour_fwd", "lp_analysis", "dfb_analysis", "quantise_kp", "rle_stream",
               "parse_unrle", "unquantise_kp", "dfb_synthesis", "lp_synthesis", "colour_inv")
MAX_SUBBANDS = 1 + 6 * 64

STATUS = {0: "CVC_OK", 1: "CVC_ERR_INVALID_ARG", 2: "CVC_ERR_UNSUPPORTED", 3: "CVC_ERR_CAPACITY",
          4: "CVC_ERR_OVERFLOW", 5: "CVC_ERR_CORRUPT", 6: "CVC_ERR_CUDA", 7: "CVC_ERR_TIMEOUT",
          8: "CVC_ERR_NOMEM", 9: "CVC_ERR_STATE"}


class CvcError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        name = STATUS.get(status, str(status))
        msg = _lib.cvc_status_string(status).decode() if _lib is not None else name
        super().__init__("%s: %s (%s)" % (where, name, msg))


class Subband(ctypes.Structure):
    _fields_ = [("off", ctypes.c_longlong), ("h", ctypes.c_int), ("w", ctypes.c_int),
                ("level", ctypes.c_int), ("dir", ctypes.c_int), ("kind", ctypes.c_int)]


class CtLayout(ctypes.Structure):
    _fields_ = [("height", ctypes.c_int), ("width", ctypes.c_int), ("levels", ctypes.c_int),
                ("dirs_log2", ctypes.c_int * MAX_LEVELS), ("modulus", ctypes.c_int), ("nsub", ctypes.c_int),
                ("sub", Subband * MAX_SUBBANDS), ("total", ctypes.c_longlong)]


class Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("levels", ctypes.c_int),
                ("dirs_log2", ctypes.c_int * MAX_LEVELS), ("qph", ctypes.c_int), ("qpl", ctypes.c_int),
                ("subband_threshold", ctypes.c_float), ("key_interval", ctypes.c_int),
                ("chroma_420", ctypes.c_int), ("motion_range", ctypes.c_int), ("storage8", ctypes.c_int),
                ("dfb_taps", ctypes.c_int)]


class CodecInfo(ctypes.Structure):
    _fields_ = [("padded_height", ctypes.c_int), ("padded_width", ctypes.c_int),
                ("chroma_height", ctypes.c_int), ("chroma_width", ctypes.c_int),
                ("padded_chroma_height", ctypes.c_int), ("padded_chroma_width", ctypes.c_int),
                ("coeffs", ctypes.c_longlong), ("components", ctypes.c_int),
                ("max_stream_bytes", ctypes.c_longlong)]


class BatchIo(ctypes.Structure):
    _fields_ = [("d_rgb", ctypes.c_void_p), ("pitch_bytes", ctypes.c_size_t), ("d_out", ctypes.c_void_p),
                ("out_cap", ctypes.c_size_t), ("d_in", ctypes.c_void_p), ("in_len", ctypes.c_size_t),
                ("d_rgb_out", ctypes.c_void_p), ("pitch_out", ctypes.c_size_t)]


class BatchResult(ctypes.Structure):
    _fields_ = [("enc_status", ctypes.c_int), ("dec_status", ctypes.c_int), ("out_len", ctypes.c_size_t),
                ("frame_type", ctypes.c_int), ("dec_frame_type", ctypes.c_int),
                ("dec_frame_index", ctypes.c_uint32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("slots_per_shard", ctypes.c_int),
                ("steps_in_flight", ctypes.c_int)]


class ServerCompletion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("session", ctypes.c_int), ("kind", ctypes.c_int),
                ("enc_status", ctypes.c_int), ("dec_status", ctypes.c_int), ("out_len", ctypes.c_size_t),
                ("frame_type", ctypes.c_int), ("dec_frame_type", ctypes.c_int),
                ("t_submit_ns", ctypes.c_int64), ("t_launch_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
                ("peak_used_bytes", ctypes.c_size_t), ("shards", ctypes.c_int), ("active_sessions", ctypes.c_int),
                ("waiting_sessions", ctypes.c_int), ("steps", ctypes.c_longlong),
                ("requests_done", ctypes.c_longlong), ("requests_queued", ctypes.c_longlong)]


STEP_ENCODE, STEP_DECODE, STEP_ENCODE_DECODE = 1, 2, 3

_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t


def lib():
    """Load libcvc.so once; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcvc.so is not built (%s); run `python -m paper_1510_00561_b300.build`"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.cvc_status_string.argtypes = [_I]
        L.cvc_status_string.restype = ctypes.c_char_p
        L.cvc_modulus.argtypes = [_I, ctypes.POINTER(_I)]
        L.cvc_ct_layout.argtypes = [_I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(CtLayout)]
        L.cvc_ct_plan_create.argtypes = [_I, _I, _I, ctypes.POINTER(_I), _I, ctypes.POINTER(_P)]
        L.cvc_ct_plan_create_taps.argtypes = [_I, _I, _I, ctypes.POINTER(_I), _I, _I, ctypes.POINTER(_P)]
        L.cvc_ct_plan_destroy.argtypes = [_P]
        L.cvc_ct_plan_set_fusion.argtypes = [_P, _I]
        L.cvc_ct_plan_coeffs.argtypes = [_P]
        L.cvc_ct_plan_coeffs.restype = ctypes.c_longlong
        for name in ("cvc_ct_forward", "cvc_ct_inverse", "cvc_ct_forward_adjoint", "cvc_ct_inverse_adjoint"):
            getattr(L, name).argtypes = [_P, _P, _P, _P]
        L.cvc_ct_plan_subbands.argtypes = [_P]
        L.cvc_ct_soft_threshold.argtypes = [_P, _P, _P, _P, _P]
        L.cvc_ct_soft_threshold_backward.argtypes = [_P, _P, _P, _P, _P, _P, _P]
        L.cvc_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(_P)]
        L.cvc_destroy.argtypes = [_P]
        L.cvc_reset.argtypes = [_P]
        L.cvc_codec_info.argtypes = [_P, ctypes.POINTER(CodecInfo)]
        L.cvc_encode_frame.argtypes = [_P, _P, _SZ, _P, _SZ, ctypes.POINTER(_SZ), ctypes.POINTER(_I), _P]
        L.cvc_decode_frame.argtypes = [_P, _P, _SZ, _P, _SZ, _P]
        L.cvc_decode_frame_scaled.argtypes = [_P, _P, _SZ, _I, _P, _SZ, _P]
        L.cvc_encode_frame_async.argtypes = [_P, _P, _SZ, _P, _SZ, _P, _P, _P, _P]
        L.cvc_decode_frame_async.argtypes = [_P, _P, _SZ, _P, _I, _P, _SZ, _P, _P]
        L.cvc_get_error.argtypes = [_P, _P, ctypes.POINTER(_I)]
        L.cvc_deflate_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(_P)]
        L.cvc_deflate_create_batch.argtypes = [ctypes.POINTER(Params), _I, ctypes.POINTER(_P)]
        L.cvc_deflate_frames.argtypes = [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_SZ), ctypes.POINTER(_P),
                                         ctypes.POINTER(_SZ), ctypes.POINTER(_SZ), ctypes.POINTER(_I), _P]
        L.cvc_inflate_frames.argtypes = [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_SZ), ctypes.POINTER(_P),
                                         ctypes.POINTER(_SZ), ctypes.POINTER(_SZ), ctypes.POINTER(_I), _P]
        L.cvc_deflate_destroy.argtypes = [_P]
        L.cvc_deflate_set_nts.argtypes = [_P, _I]
        L.cvc_deflate_frame.argtypes = [_P, _P, _SZ, _P, _SZ, ctypes.POINTER(_SZ), _P]
        L.cvc_inflate_frame.argtypes = [_P, _P, _SZ, _P, _SZ, ctypes.POINTER(_SZ), _P]
        L.cvc_stream_drop_levels.argtypes = [ctypes.POINTER(Params), _P, _SZ, _I, _P, _SZ, ctypes.POINTER(_SZ)]
        L.cvc_codec_inspect.argtypes = [_P, _I, _P, _SZ, _P]
        L.cvc_codec_set_timing.argtypes = [_P, _I]
        L.cvc_codec_timing.argtypes = [_P, _P, _P]
        L.cvc_kernel_launches.argtypes = []
        L.cvc_kernel_launches.restype = ctypes.c_ulonglong
        L.cvc_lp_pyramid_forward_static.argtypes = [_P, _I, _I, _I, _P, _P]
        L.cvc_batch_create.argtypes = [ctypes.POINTER(Params), _I, ctypes.POINTER(_P)]
        L.cvc_batch_destroy.argtypes = [_P]
        L.cvc_batch_device_bytes.argtypes = [ctypes.POINTER(Params), _I, ctypes.POINTER(_SZ)]
        L.cvc_batch_info.argtypes = [_P, _I, ctypes.POINTER(CodecInfo)]
        L.cvc_batch_reset.argtypes = [_P, _I]
        L.cvc_batch_step.argtypes = [_P, _I, ctypes.POINTER(BatchIo), ctypes.POINTER(BatchResult), _P]
        L.cvc_batch_step_scaled.argtypes = [_P, _I, ctypes.POINTER(BatchIo), _I, ctypes.POINTER(BatchResult), _P]
        L.cvc_batch_step_async.argtypes = [_P, _I, ctypes.POINTER(BatchIo), _P, _I, _P, _P]
        L.cvc_batch_get_error.argtypes = [_P, _I, _P, ctypes.POINTER(_I)]
        L.cvc_batch_set_shape.argtypes = [_P, _I, _I]
        L.cvc_batch_set_fusion.argtypes = [_P, _I]
        L.cvc_batch_set_dfb_threads.argtypes = [_P, _I]
        L.cvc_batch_autotune.argtypes = [_P, _I, ctypes.POINTER(BatchIo), _I, ctypes.POINTER(_I), _P]
        L.cvc_batch_set_graphs.argtypes = [_P, _I]
        L.cvc_batch_set_timing.argtypes = [_P, _I]
        L.cvc_batch_timing.argtypes = [_P, _P, _P]
        L.cvc_server_now_ns.argtypes = []
        L.cvc_server_now_ns.restype = ctypes.c_int64
        L.cvc_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]
        L.cvc_server_destroy.argtypes = [_P]
        L.cvc_server_open.argtypes = [_P, ctypes.POINTER(Params), ctypes.POINTER(_I)]
        L.cvc_server_close.argtypes = [_P, _I]
        L.cvc_server_submit.argtypes = [_P, _I, _I, ctypes.POINTER(BatchIo), ctypes.c_uint64]
        L.cvc_server_poll.argtypes = [_P, _I, ctypes.POINTER(ServerCompletion), _I, ctypes.POINTER(_I)]
        L.cvc_server_get_stats.argtypes = [_P, ctypes.POINTER(ServerStats)]
        L.cvc_debug_plan_tables.argtypes = [ctypes.POINTER(Params), _I, _I, _I, ctypes.POINTER(_I), _I, _I, _P,
                                            _SZ, ctypes.POINTER(_SZ)]
        L.cvc_debug_scale_tables.argtypes = [ctypes.POINTER(Params), _I, _I, _P, _SZ, ctypes.POINTER(_SZ)]
        _lib = L
    return _lib


def params(width, height, levels, dirs_log2, qph, qpl=None, threshold=0.0, key_interval=10, motion_range=0,
           storage8=False, dfb_taps=4):
    """cvc_params of one stream (qpl defaults to max(1, qph // 14))."""
    if qpl is None:
        qpl = max(1, qph // 14)
    return Params(width, height, levels, ints(dirs_log2), qph, qpl, threshold, key_interval, 1, motion_range,
                  int(bool(storage8)), int(dfb_taps))


def check(status, where):
    if status != 0:
        raise CvcError(status, where)


def ints(seq, n=MAX_LEVELS):
    vals = list(seq) + [0] * (n - len(seq))
    return (_I * n)(*vals)
