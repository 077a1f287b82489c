"""Python binding of liblic (include/lic.h): argument marshalling only.

Every step of the codec chain runs in the library's CUDA kernels; this
module only converts torch tensors / numpy arrays into pointers and calls the
C ABI by the same names.  PyTorch is used for device memory and streams.
If liblic.so is missing the import of the binding fails loudly: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblic.so")

FACTORIZED = 0
HYPERPRIOR = 1
CONV_AUTO = 0
CONV_SIMT = 1
FP32 = 0
BF16 = 1
NORM_GDN = 0
NORM_1DN = 1
FORMAT_1 = 1
FORMAT_2 = 2
FP8 = 2

T_Y, T_SY, T_Z, T_SZ, T_SIGMA, T_IDX, T_XPRE, T_YHAT = range(8)

OK = 0
E_INVALID_ARG, E_UNSUPPORTED, E_OOM, E_CORRUPT_STREAM, E_TIMEOUT, E_CUDA, E_BUSY = -1, -2, -3, -4, -5, -6, -7

EXPORTED = [
    "lic_codec_create", "lic_codec_destroy", "lic_sync", "lic_encode", "lic_decode",
    "lic_bitstreams_download", "lic_decoded_shape", "lic_read_tensor", "lic_analysis",
    "lic_synthesis", "lic_hyper_analysis", "lic_hyper_synthesis", "lic_encode_latents",
    "lic_decode_latents", "lic_build_tables", "lic_scale_table", "lic_strerror",
    "lic_profile_enable", "lic_profile_report", "lic_launch_count", "lic_encode_latents_noalloc",
    "lic_test_bounded_wait", "lic_bitstreams_release", "lic_codec_device_bytes", "lic_codec_workspace_bytes",
    "lic_probe_mma_rate", "lic_strip_resume_records",
    # include/lic_student.h (learned form)
    "lic_student_create", "lic_student_destroy", "lic_student_grad", "lic_student_step", "lic_student_read",
    "lic_student_read_activation", "lic_student_read_output_grad", "lic_student_steps", "lic_student_forward", "lic_student_profile_enable", "lic_student_profile_report",
    "lic_student_launch_count", "lic_codec_set_student", "lic_codec_student_report",
    # include/lic_serve.h (serving form)
    "lic_server_create", "lic_server_destroy", "lic_server_prepare", "lic_server_submit", "lic_server_poll",
    "lic_server_drain", "lic_server_stats_get", "lic_server_clock_ms",
]

STUDENT_PARAM, STUDENT_GRAD, STUDENT_ADAM_M, STUDENT_ADAM_V = range(4)
STUDENT_MAX_BATCH = 64

NOALLOC_SCRATCH_BYTES = 32 << 20


class LicError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_lib().lic_strerror(code).decode()} ({code})")


class _Param(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("data", ctypes.POINTER(ctypes.c_float)),
                ("numel", ctypes.c_int64)]


class _Weights(ctypes.Structure):
    _fields_ = [("params", ctypes.POINTER(_Param)), ("count", ctypes.c_int)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("band_rows", ctypes.c_int),
                ("conv_impl", ctypes.c_int), ("norm", ctypes.c_int), ("format", ctypes.c_int),
                ("resume_groups", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class _StudentOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_batch", ctypes.c_int), ("crop", ctypes.c_int),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("halo", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class _ServerOptions(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int), ("lanes", ctypes.c_int), ("max_pending", ctypes.c_int),
                ("graphs", ctypes.c_int), ("max_wait_ms", ctypes.c_double), ("hbm_budget", ctypes.c_int64),
                ("reserved", ctypes.c_int * 4)]


class _ServerResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("stream_id", ctypes.c_int), ("status", ctypes.c_int),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("batch", ctypes.c_int), ("bytes", ctypes.c_int64),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("refused_busy", ctypes.c_int64),
                ("refused_budget", ctypes.c_int64), ("batches", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("buckets", ctypes.c_int)]


class _Bitstreams(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("on_device", ctypes.c_int),
                ("data", ctypes.c_void_p), ("offsets", ctypes.POINTER(ctypes.c_int64)),
                ("sizes", ctypes.POINTER(ctypes.c_int64)), ("d_offsets", ctypes.c_void_p),
                ("d_sizes", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("owner", ctypes.c_void_p)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run python paper_2208_01641_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        L.lic_codec_create.argtypes = [i, i, i, ctypes.POINTER(_Weights), ctypes.POINTER(_Options),
                                       ctypes.POINTER(vp)]
        L.lic_codec_destroy.argtypes = [vp]
        L.lic_codec_destroy.restype = None
        L.lic_sync.argtypes = [vp, vp]
        L.lic_encode.argtypes = [vp, vp, i, i, i, ctypes.POINTER(_Bitstreams), vp]
        L.lic_decode.argtypes = [vp, ctypes.POINTER(_Bitstreams), vp, vp]
        L.lic_bitstreams_release.argtypes = [vp, ctypes.POINTER(_Bitstreams)]
        L.lic_codec_device_bytes.argtypes = [vp]
        L.lic_codec_device_bytes.restype = i64
        L.lic_codec_workspace_bytes.argtypes = [vp, i, i, i]
        L.lic_codec_workspace_bytes.restype = i64
        L.lic_bitstreams_download.argtypes = [ctypes.POINTER(_Bitstreams), vp, i64, vp]
        L.lic_bitstreams_download.restype = i64
        L.lic_decoded_shape.argtypes = [vp, i64, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        L.lic_read_tensor.argtypes = [vp, i, vp, ctypes.POINTER(i64), vp]
        L.lic_analysis.argtypes = [vp, vp, i, i, i, vp, vp]
        L.lic_synthesis.argtypes = [vp, vp, i, i, i, vp, vp]
        L.lic_hyper_analysis.argtypes = [vp, vp, i, i, i, vp, vp]
        L.lic_hyper_synthesis.argtypes = [vp, vp, i, i, i, vp, vp, vp]
        L.lic_encode_latents.argtypes = [vp, vp, vp, vp, i, i, i, i, i, ctypes.POINTER(_Bitstreams), vp]
        L.lic_decode_latents.argtypes = [vp, ctypes.POINTER(_Bitstreams), vp, vp, vp]
        L.lic_encode_latents_noalloc.argtypes = [vp, vp, vp, vp, i, i, i, i, i, vp, i64, vp, vp]
        L.lic_build_tables.argtypes = [ctypes.POINTER(_Weights), i, i, i64, vp, vp, vp, vp, vp]
        L.lic_scale_table.argtypes = [vp]
        L.lic_scale_table.restype = None
        L.lic_profile_enable.argtypes = [vp, i]
        L.lic_profile_report.argtypes = [vp, ctypes.c_char_p, i]
        L.lic_launch_count.argtypes = [vp]
        L.lic_launch_count.restype = i64
        L.lic_test_bounded_wait.argtypes = [vp, i64, vp]
        L.lic_probe_mma_rate.argtypes = [i, i, ctypes.POINTER(ctypes.c_double)]
        L.lic_strip_resume_records.argtypes = [vp, i64, vp, i64, ctypes.POINTER(i64)]
        L.lic_student_create.argtypes = [ctypes.POINTER(_Weights), i, i, ctypes.POINTER(_StudentOptions),
                                         ctypes.POINTER(vp)]
        L.lic_student_destroy.argtypes = [vp]
        L.lic_student_destroy.restype = None
        L.lic_student_grad.argtypes = [vp, vp, vp, i, i, i, vp, i, ctypes.POINTER(ctypes.c_float), vp]
        L.lic_student_step.argtypes = [vp, vp, vp, i, i, i, vp, i, ctypes.POINTER(ctypes.c_float), vp]
        L.lic_student_read.argtypes = [vp, ctypes.c_char_p, i, vp, i64]
        L.lic_student_read_activation.argtypes = [vp, i, vp, i64]
        L.lic_student_read_output_grad.argtypes = [vp, i, vp, i64]
        L.lic_student_steps.argtypes = [vp]
        L.lic_student_steps.restype = i64
        L.lic_student_forward.argtypes = [vp, vp, i, i, i, vp, vp]
        L.lic_student_profile_enable.argtypes = [vp, i]
        L.lic_student_profile_report.argtypes = [vp, ctypes.c_char_p, i]
        L.lic_student_launch_count.argtypes = [vp]
        L.lic_student_launch_count.restype = i64
        L.lic_codec_set_student.argtypes = [vp, vp, ctypes.c_float, i]
        L.lic_codec_student_report.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), vp, i]
        L.lic_server_create.argtypes = [i, i, i, ctypes.POINTER(_Weights), ctypes.POINTER(_Options),
                                        ctypes.POINTER(_ServerOptions), ctypes.POINTER(vp)]
        L.lic_server_destroy.argtypes = [vp]
        L.lic_server_destroy.restype = None
        L.lic_server_prepare.argtypes = [vp, i, i]
        L.lic_server_submit.argtypes = [vp, i, vp, i, i, vp, ctypes.POINTER(ctypes.c_uint64)]
        L.lic_server_poll.argtypes = [vp, ctypes.POINTER(_ServerResult), i, ctypes.c_double]
        L.lic_server_drain.argtypes = [vp, ctypes.c_double]
        L.lic_server_stats_get.argtypes = [vp, ctypes.POINTER(_ServerStats)]
        L.lic_server_clock_ms.argtypes = [vp]
        L.lic_server_clock_ms.restype = ctypes.c_double
        L.lic_strerror.argtypes = [i]
        L.lic_strerror.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def lib():
    """The loaded liblic.so (ctypes handle)."""
    return _lib()


def _check(rc, what):
    if rc < 0:
        raise LicError(rc, what)
    return rc


def _ptr(t) -> int:
    """Data pointer of a torch tensor or numpy array (no copies)."""
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _weights_struct(weights: Dict[str, np.ndarray]):
    keep = []
    arr = (_Param * len(weights))()
    for k, (name, a) in enumerate(weights.items()):
        a = np.ascontiguousarray(a, dtype=np.float32)
        nb = name.encode()
        keep += [a, nb]
        arr[k].name = nb
        arr[k].data = a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        arr[k].numel = a.size
    w = _Weights(arr, len(weights))
    return w, (keep, arr)


def build_tables(weights: Dict[str, np.ndarray], gauss: bool):
    """Host-only table build (lic_build_tables): (medians, lo, hi, start, cdf)."""
    w, keep = _weights_struct(weights)
    C = weights["eb.H0"].shape[0]
    cap_t, cap_c = C + 64, (C + 64) * 4097
    med = np.zeros(C, np.float32)
    lo = np.zeros(cap_t, np.int32)
    hi = np.zeros(cap_t, np.int32)
    start = np.zeros(cap_t, np.int64)
    cdf = np.zeros(cap_c, np.uint32)
    n = _check(_lib().lic_build_tables(ctypes.byref(w), 1 if gauss else 0, cap_t, cap_c, _ptr(med), _ptr(lo),
                                       _ptr(hi), _ptr(start), _ptr(cdf)), "lic_build_tables")
    return med, lo[:n], hi[:n], start[:n], cdf


def scale_table():
    T = np.zeros(64, np.float32)
    _lib().lic_scale_table(_ptr(T))
    return T


class Bitstreams:
    """A batch of frame containers returned by encode: library-owned
    buffers, valid until release() (called when the object is collected).
    The codec may reuse released buffers in its next encode on any stream,
    so release a batch (or drop the last reference) only once the calls that
    read it are enqueued on the stream of that next encode."""

    def __init__(self, codec: "Codec", s: _Bitstreams, stream):
        self.codec, self.s, self.stream = codec, s, stream

    @property
    def count(self):
        return self.s.count

    @property
    def shape(self):
        """(H, W): the frame size of every frame of the batch."""
        return self.s.H, self.s.W

    def sizes(self):
        """Frame sizes in bytes (synchronizes the stream)."""
        self.codec.sync(self.stream)
        return [int(self.s.sizes[i]) for i in range(self.s.count)]

    def to_bytes(self):
        """Per-frame bytes objects (synchronizes the stream)."""
        self.codec.sync(self.stream)
        total = int(self.s.offsets[self.s.count])
        buf = np.zeros(max(total, 1), np.uint8)
        _check(_lib().lic_bitstreams_download(ctypes.byref(self.s), _ptr(buf), buf.size, self.stream),
               "lic_bitstreams_download")
        return [buf[self.s.offsets[i]:self.s.offsets[i] + self.s.sizes[i]].tobytes()
                for i in range(self.s.count)]

    def release(self):
        """Return the buffers to the codec's pool (lic_bitstreams_release)."""
        c = self.codec
        if self.s.owner and c is not None and getattr(c, "h", None):
            _check(_lib().lic_bitstreams_release(c.h, ctypes.byref(self.s)), "lic_bitstreams_release")
        self.codec = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def host_bitstreams(frames, H: int = 0, W: int = 0):
    """A lic_bitstreams view of host bytes objects (for lic_decode).  With
    H = W = 0 the library reads the frame size from frame 0's header."""
    sizes = np.array([len(f) for f in frames], np.int64)
    offs = np.zeros(len(frames) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    data = np.frombuffer(b"".join(frames) or b"\0", np.uint8).copy()
    s = _Bitstreams(len(frames), 0, data.ctypes.data, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                    sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None, None, H, W, None)
    s._keep = (data, offs, sizes)
    return s


class Codec:
    """One codec on the current CUDA device (lic_codec_create)."""

    def __init__(self, kind: int, N: int, M: int, weights: Dict[str, np.ndarray], band_rows: int = 16,
                 conv_impl: int = CONV_AUTO, precision: int = FP32, norm: int = NORM_GDN,
                 format: int = FORMAT_1, resume_groups: int = 0):
        self.kind, self.N, self.M = kind, N, M
        w, keep = _weights_struct(weights)
        opt = _Options(precision, band_rows, conv_impl, norm, format, resume_groups)
        h = ctypes.c_void_p()
        _check(_lib().lic_codec_create(kind, N, M, ctypes.byref(w), ctypes.byref(opt), ctypes.byref(h)),
               "lic_codec_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib().lic_codec_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        return _check(_lib().lic_sync(self.h, _stream(stream)), "lic_sync")

    def sync_status(self, stream=None) -> int:
        """lic_sync's return code without raising."""
        return _lib().lic_sync(self.h, _stream(stream))

    def profile(self, enable: bool):
        _check(_lib().lic_profile_enable(self.h, 1 if enable else 0), "lic_profile_enable")

    def profile_report(self):
        import json
        n = _check(_lib().lic_profile_report(self.h, None, 0), "lic_profile_report")
        buf = ctypes.create_string_buffer(n + 1)
        _check(_lib().lic_profile_report(self.h, buf, n + 1), "lic_profile_report")
        return json.loads(buf.value.decode())

    def launch_count(self) -> int:
        return int(_lib().lic_launch_count(self.h))

    def test_bounded_wait(self, limit_cycles: int, stream=None):
        """Diagnostics: a bounded wait that runs out (lic_test_bounded_wait)."""
        _check(_lib().lic_test_bounded_wait(self.h, limit_cycles, _stream(stream)), "lic_test_bounded_wait")

    def set_student(self, student: Optional["Student"], min_psnr_db: float = 35.0, checked: bool = False):
        """Decode with ``student`` in place of g_s (None restores g_s)."""
        self._student = student
        _check(_lib().lic_codec_set_student(self.h, student.h if student else None, float(min_psnr_db),
                                            1 if checked else 0), "lic_codec_set_student")

    def student_report(self, cap: int = 1024):
        """(frames checked, fallbacks, per-frame PSNR of the last checked decode)."""
        fr, fb = ctypes.c_int64(), ctypes.c_int64()
        ps = np.zeros(cap, np.float32)
        n = _check(_lib().lic_codec_student_report(self.h, ctypes.byref(fr), ctypes.byref(fb), _ptr(ps), cap),
                   "lic_codec_student_report")
        return fr.value, fb.value, ps[:min(n, cap)]

    def encode(self, frames, stream=None) -> Bitstreams:
        B, C, H, W = frames.shape
        assert C == 3
        st = _stream(stream)
        s = _Bitstreams()
        _check(_lib().lic_encode(self.h, _ptr(frames), B, H, W, ctypes.byref(s), st), "lic_encode")
        return Bitstreams(self, s, st)

    def decode(self, bs, out, stream=None):
        """Decode a batch into out (B x 3 x H x W float32, device or host);
        the frame size comes from the batch."""
        st = _stream(stream)
        s = bs.s if isinstance(bs, Bitstreams) else bs
        _check(_lib().lic_decode(self.h, ctypes.byref(s), _ptr(out), st), "lic_decode")
        return out

    def decode_status(self, bs, out, stream=None) -> int:
        st = _stream(stream)
        s = bs.s if isinstance(bs, Bitstreams) else bs
        return _lib().lic_decode(self.h, ctypes.byref(s), _ptr(out), st)

    def device_bytes(self) -> int:
        """Device memory the codec holds (lic_codec_device_bytes)."""
        return _check(_lib().lic_codec_device_bytes(self.h), "lic_codec_device_bytes")

    def workspace_bytes(self, B: int, H: int, W: int) -> int:
        """Workspace + one batch that B frames of H x W need (lic_codec_workspace_bytes)."""
        return _check(_lib().lic_codec_workspace_bytes(self.h, B, H, W), "lic_codec_workspace_bytes")

    def read_tensor(self, which: int, dst, stream=None):
        n = ctypes.c_int64()
        need = self.tensor_count(which)
        have = dst.size if isinstance(dst, np.ndarray) else dst.numel()
        if have != need:
            raise ValueError(f"read_tensor: destination holds {have} elements, tensor has {need}")
        _check(_lib().lic_read_tensor(self.h, which, _ptr(dst), ctypes.byref(n), _stream(stream)),
               "lic_read_tensor")
        return dst

    def tensor_count(self, which: int) -> int:
        n = ctypes.c_int64()
        _check(_lib().lic_read_tensor(self.h, which, None, ctypes.byref(n), None), "lic_read_tensor")
        return n.value

    def analysis(self, frames, y, stream=None):
        B, _, H, W = frames.shape
        _check(_lib().lic_analysis(self.h, _ptr(frames), B, H, W, _ptr(y), _stream(stream)), "lic_analysis")
        return y

    def synthesis(self, yhat, x, stream=None):
        B, _, Hy, Wy = yhat.shape
        _check(_lib().lic_synthesis(self.h, _ptr(yhat), B, Hy, Wy, _ptr(x), _stream(stream)), "lic_synthesis")
        return x

    def hyper_analysis(self, y, z, stream=None):
        B, _, Hy, Wy = y.shape
        _check(_lib().lic_hyper_analysis(self.h, _ptr(y), B, Hy, Wy, _ptr(z), _stream(stream)),
               "lic_hyper_analysis")
        return z

    def hyper_synthesis(self, zhat, sigma, idx=None, stream=None):
        B, _, Hz, Wz = zhat.shape
        _check(_lib().lic_hyper_synthesis(self.h, _ptr(zhat), B, Hz, Wz, _ptr(sigma),
                                          _ptr(idx) if idx is not None else None, _stream(stream)),
               "lic_hyper_synthesis")
        return sigma

    def encode_latents(self, s_y, idx, s_z, H: int, W: int, stream=None) -> Bitstreams:
        B, _, Hy, Wy = s_y.shape
        st = _stream(stream)
        s = _Bitstreams()
        _check(_lib().lic_encode_latents(self.h, _ptr(s_y), _ptr(idx) if idx is not None else None,
                                         _ptr(s_z) if s_z is not None else None, B, H, W, Hy, Wy,
                                         ctypes.byref(s), st), "lic_encode_latents")
        return Bitstreams(self, s, st)

    def encode_latents_noalloc(self, s_y, idx, s_z, H: int, W: int, data, layout, stream=None) -> int:
        """lic_encode_latents_noalloc into caller buffers (data: device
        uint8, layout: device int64[2B+1]); returns the ABI's code."""
        B, _, Hy, Wy = s_y.shape
        return _lib().lic_encode_latents_noalloc(
            self.h, _ptr(s_y), _ptr(idx) if idx is not None else None, _ptr(s_z) if s_z is not None else None,
            B, H, W, Hy, Wy, _ptr(data), data.numel(), _ptr(layout), _stream(stream))

    def decode_latents(self, bs, s_y, s_z=None, stream=None):
        s = bs.s if isinstance(bs, Bitstreams) else bs
        _check(_lib().lic_decode_latents(self.h, ctypes.byref(s), _ptr(s_y),
                                         _ptr(s_z) if s_z is not None else None, _stream(stream)),
               "lic_decode_latents")


def mma_rate(kind: int, iters: int = 20000) -> float:
    """Measured dense tensor-pipe rate in TFLOP/s (lic_probe_mma_rate):
    kind 0 tf32, 1 bf16, 2 e4m3."""
    t = ctypes.c_double()
    _check(_lib().lic_probe_mma_rate(kind, iters, ctypes.byref(t)), "lic_probe_mma_rate")
    return t.value


def strip_resume_records(frame: bytes) -> bytes:
    """A format-2 frame without its resume records (lic_strip_resume_records)."""
    buf = np.frombuffer(frame, np.uint8).copy()
    out = np.zeros(max(1, len(frame)), np.uint8)
    n = ctypes.c_int64()
    _check(_lib().lic_strip_resume_records(_ptr(buf), len(frame), _ptr(out), out.size, ctypes.byref(n)),
           "lic_strip_resume_records")
    return out[:n.value].tobytes()


def decoded_shape(frame: bytes):
    k, h, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    buf = np.frombuffer(frame, np.uint8).copy()
    _check(_lib().lic_decoded_shape(_ptr(buf), len(frame), ctypes.byref(k), ctypes.byref(h), ctypes.byref(w)),
           "lic_decoded_shape")
    return k.value, h.value, w.value


def _profile_json(fn, h):
    import json
    n = _check(fn(h, None, 0), "profile_report")
    buf = ctypes.create_string_buffer(n + 1)
    _check(fn(h, buf, n + 1), "profile_report")
    return json.loads(buf.value.decode())


class Student:
    """The learned form's student synthesis net (include/lic_student.h)."""

    def __init__(self, weights: Dict[str, np.ndarray], M: int = 192, C: int = 64, max_batch: int = 16,
                 crop: int = 256, lr: float = 1e-4, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 precision: int = FP32, halo: int = 0):
        self.M, self.C, self.crop, self.halo = M, C, crop, halo
        self.shapes = {k: tuple(np.shape(v)) for k, v in weights.items() if k.startswith("student.")}
        w, keep = _weights_struct(weights)
        opt = _StudentOptions(precision, max_batch, crop, lr, beta1, beta2, eps, halo)
        h = ctypes.c_void_p()
        _check(_lib().lic_student_create(ctypes.byref(w), M, C, ctypes.byref(opt), ctypes.byref(h)),
               "lic_student_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib().lic_student_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, fn, name, yhat_pool, xhat_pool, crops, want_loss, stream):
        P, M, Hy, Wy = yhat_pool.shape
        crops = np.ascontiguousarray(crops, dtype=np.int32)
        loss = ctypes.c_float()
        _check(fn(self.h, _ptr(yhat_pool), _ptr(xhat_pool), P, Hy, Wy, _ptr(crops), crops.shape[0],
                  ctypes.byref(loss) if want_loss else None, _stream(stream)), name)
        return loss.value if want_loss else None

    def grad(self, yhat_pool, xhat_pool, crops, want_loss=True, stream=None):
        """Loss and gradients of one batch (lic_student_grad)."""
        return self._call(_lib().lic_student_grad, "lic_student_grad", yhat_pool, xhat_pool, crops, want_loss,
                          stream)

    def step(self, yhat_pool, xhat_pool, crops, want_loss=False, stream=None):
        """Gradients and one Adam step (lic_student_step)."""
        return self._call(_lib().lic_student_step, "lic_student_step", yhat_pool, xhat_pool, crops, want_loss,
                          stream)

    def read(self, name: str, what: int = STUDENT_PARAM) -> np.ndarray:
        out = np.zeros(self.shapes[name], np.float32)
        _check(_lib().lic_student_read(self.h, name.encode(), what, _ptr(out), out.size), "lic_student_read")
        return out

    def activation(self, layer: int, B: int) -> np.ndarray:
        """Post-ReLU h_layer of the last training batch, NHWC (layer 0: the
        gathered y_hat window)."""
        side = (self.crop + 32 * self.halo) >> (4 - layer)
        out = np.zeros((B, side, side, self.M if layer == 0 else self.C), np.float32)
        _check(_lib().lic_student_read_activation(self.h, layer, _ptr(out), out.size),
               "lic_student_read_activation")
        return out

    def output_grad(self, layer: int, B: int) -> np.ndarray:
        """dz_layer of the last training batch (the loss gradient at transposed
        conv `layer`'s pre-activation output), NHWC."""
        side = (self.crop + 32 * self.halo) >> (3 - layer)
        out = np.zeros((B, side, side, 3 if layer == 3 else self.C), np.float32)
        _check(_lib().lic_student_read_output_grad(self.h, layer, _ptr(out), out.size),
               "lic_student_read_output_grad")
        return out

    def params(self) -> "Dict[str, np.ndarray]":
        return {k: self.read(k) for k in self.shapes}

    def steps(self) -> int:
        return int(_lib().lic_student_steps(self.h))

    def forward(self, yhat, x, stream=None):
        B, M, Hy, Wy = yhat.shape
        _check(_lib().lic_student_forward(self.h, _ptr(yhat), B, Hy, Wy, _ptr(x), _stream(stream)),
               "lic_student_forward")

    def profile(self, enable: bool):
        _check(_lib().lic_student_profile_enable(self.h, 1 if enable else 0), "lic_student_profile_enable")

    def profile_report(self):
        return _profile_json(_lib().lic_student_profile_report, self.h)

    def launch_count(self) -> int:
        return int(_lib().lic_student_launch_count(self.h))


class Server:
    """The serving form (include/lic_serve.h): frames of many streams and
    resolutions, batched per resolution, encoded and decoded on lanes of
    codecs running concurrently.  Keeps each submitted frame (and output
    buffer) alive until its result has been polled."""

    def __init__(self, kind: int, N: int, M: int, weights: Dict[str, np.ndarray], precision: int = FP32,
                 max_batch: int = 8, lanes: int = 2, max_pending: int = 256, graphs: bool = True,
                 max_wait_ms: float = 2.0, hbm_budget: int = 40 << 30, band_rows: int = 16):
        w, keep = _weights_struct(weights)
        copt = _Options(precision, band_rows, CONV_AUTO, NORM_GDN)
        opt = _ServerOptions(max_batch, lanes, max_pending, 1 if graphs else 0, max_wait_ms, hbm_budget)
        h = ctypes.c_void_p()
        _check(_lib().lic_server_create(kind, N, M, ctypes.byref(w), ctypes.byref(copt), ctypes.byref(opt),
                                        ctypes.byref(h)), "lic_server_create")
        self.h = h
        self._live = {}

    def close(self):
        if getattr(self, "h", None):
            _lib().lic_server_destroy(self.h)
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prepare(self, H: int, W: int):
        _check(_lib().lic_server_prepare(self.h, H, W), "lic_server_prepare")

    def submit(self, stream_id: int, frame, decoded=None) -> int:
        """Queue one 3 x H x W frame; returns its ticket.  Raises LicError
        (code E_BUSY / E_OOM) when admission refuses it."""
        H, W = frame.shape[-2], frame.shape[-1]
        t = ctypes.c_uint64()
        _check(_lib().lic_server_submit(self.h, stream_id, _ptr(frame), H, W,
                                        _ptr(decoded) if decoded is not None else None, ctypes.byref(t)),
               "lic_server_submit")
        self._live[t.value] = (frame, decoded)
        return t.value

    def poll(self, cap: int = 256, wait_ms: float = 0.0):
        buf = (_ServerResult * cap)()
        n = _check(_lib().lic_server_poll(self.h, buf, cap, wait_ms), "lic_server_poll")
        out = []
        for k in range(n):
            r = buf[k]
            self._live.pop(r.ticket, None)
            out.append({f: getattr(r, f) for f, _ in _ServerResult._fields_})
        return out

    def drain(self, timeout_ms: float = 60000.0):
        _check(_lib().lic_server_drain(self.h, timeout_ms), "lic_server_drain")

    def stats(self):
        s = _ServerStats()
        _check(_lib().lic_server_stats_get(self.h, ctypes.byref(s)), "lic_server_stats_get")
        return {f: getattr(s, f) for f, _ in _ServerStats._fields_}

    def clock_ms(self) -> float:
        return float(_lib().lic_server_clock_ms(self.h))
