"""FP64 CPU reference ("oracle") of the codec chain -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product (only the seeded input
generators, which hold no codec arithmetic).

The numerical kernels are plain C in ``oracle.c`` (double precision, loops
written as the definitions read); this module loads them with ctypes and
strings them together in the order of the paper's Fig. 1 / Sec. III:

  encoder  x -> g_a -> y -> Q -> E       (+ h_a -> z -> Q -> E, h_s -> scales)
  decoder  E^-1 -> Q^-1 -> g_s -> x_hat  (+ z first, then h_s, then y)

The learned form's distilled student synthesis net (4 transposed convs,
ReLU, MSE against the teacher's g_s output) has its forward pass, its
backward pass by the chain rule, and Adam (Kingma & Ba 2015, Algorithm 1)
here too; they are pinned by finite differences, torch float64 autograd
and the constant-gradient closed form of Adam.

The bitstream container is the project's own format (the paper integrates
CompressAI's coder and defines no format); it is written out below
byte by byte.
"""
from __future__ import annotations

import ctypes
import math
import os
import struct
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

KIND_FACTORIZED = 0
KIND_HYPERPRIOR = 1
BAND_ROWS = 16          # latent rows per y substream
LANES = 32              # interleaved rANS states per substream


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2 -ffp-contract=off, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                   os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB_PATH
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-D_GNU_SOURCE", "-o", _LIB_PATH, src, "-lm"]
    subprocess.check_call(cmd)
    return _LIB_PATH


class _Table(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int), ("hi", ctypes.c_int), ("n", ctypes.c_int),
                ("cdf", ctypes.POINTER(ctypes.c_uint32))]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        ip = ctypes.c_int
        L.orc_conv2d.argtypes = [dp, ip, ip, ip, ip, dp, dp, ip, ip, ip, dp]
        L.orc_deconv2d.argtypes = [dp, ip, ip, ip, ip, dp, dp, ip, ip, ip, dp]
        L.orc_gdn.argtypes = [dp, ip, ip, ip, ip, dp, dp, ip]
        L.orc_norm1d.argtypes = [dp, ip, ip, ip, ip, dp, dp, ip]
        L.orc_deconv2d_wgrad.argtypes = [dp, ip, ip, ip, ip, dp, ip, ip, ip, dp]
        L.orc_relu.argtypes = [dp, ctypes.c_int64]
        L.orc_abs.argtypes = [dp, ctypes.c_int64]
        L.orc_eb_logits.argtypes = [dp, ctypes.c_double]
        L.orc_eb_logits.restype = ctypes.c_double
        L.orc_eb_table.argtypes = [dp, fp, ctypes.POINTER(ip), ctypes.POINTER(ip),
                                   ctypes.POINTER(ctypes.c_uint32)]
        L.orc_eb_pmf.argtypes = [dp, fp, ctypes.POINTER(ip), ctypes.POINTER(ip), dp, ip]
        L.orc_quantize_pmf.argtypes = [dp, ip, ctypes.POINTER(ctypes.c_uint32)]
        L.orc_scale_table.argtypes = [fp]
        L.orc_gauss_table.argtypes = [ip, ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_uint32)]
        L.orc_gauss_ztau.restype = ctypes.c_double
        L.orc_quantize.argtypes = [fp, ip, ip, ip, fp, ctypes.POINTER(ctypes.c_int32)]
        L.orc_dequantize.argtypes = [ctypes.POINTER(ctypes.c_int32), ip, ip, ip, fp, fp]
        L.orc_scale_index.argtypes = [fp, ctypes.c_int64, fp, ctypes.POINTER(ctypes.c_uint8)]
        L.orc_rans_encode.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ip, ctypes.POINTER(_Table), ctypes.POINTER(ctypes.c_uint16),
                                      ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), dp]
        L.orc_rans_decode.argtypes = [ctypes.POINTER(ctypes.c_uint16), ctypes.c_int64, ip,
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_Table),
                                      ctypes.POINTER(ctypes.c_int32)]
        u16p, u32p, i64p = (ctypes.POINTER(ctypes.c_uint16), ctypes.POINTER(ctypes.c_uint32),
                            ctypes.POINTER(ctypes.c_int64))
        L.orc_rans2_encode.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ip,
                                       ctypes.POINTER(_Table), ip, u16p, ctypes.c_int64, i64p, u32p,
                                       ctypes.c_int64, i64p, i64p, dp]
        L.orc_rans2_decode_range.argtypes = [u16p, ctypes.c_int64, ip, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(_Table), u32p, ip, ip,
                                             ctypes.POINTER(ctypes.c_int32)]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# transforms
# --------------------------------------------------------------------------

def conv2d(x, w, b, stride):
    """Zero-padded conv, pad k//2 (C1).  x: B x Cin x H x W."""
    x, w = _f64(x), _f64(w)
    B, Cin, H, W = x.shape
    Cout, _, k, _ = w.shape
    p = k // 2
    Ho, Wo = (H + 2 * p - k) // stride + 1, (W + 2 * p - k) // stride + 1
    y = np.empty((B, Cout, Ho, Wo))
    bb = _f64(b) if b is not None else None
    lib().orc_conv2d(_p(x, ctypes.c_double), B, Cin, H, W, _p(w, ctypes.c_double),
                     _p(bb, ctypes.c_double) if bb is not None else None, Cout, k, stride,
                     _p(y, ctypes.c_double))
    return y


def deconv2d(x, w, b, stride):
    """Transposed conv k, stride s, pad k//2, output padding s-1 (C2).  w: Cin x Cout x k x k."""
    x, w = _f64(x), _f64(w)
    B, Cin, H, W = x.shape
    _, Cout, k, _ = w.shape
    y = np.empty((B, Cout, stride * H, stride * W))
    bb = _f64(b) if b is not None else None
    lib().orc_deconv2d(_p(x, ctypes.c_double), B, Cin, H, W, _p(w, ctypes.c_double),
                       _p(bb, ctypes.c_double) if bb is not None else None, Cout, k, stride,
                       _p(y, ctypes.c_double))
    return y


def gdn(x, beta, gamma, inverse=False):
    """GDN / IGDN; a 1-D gamma selects 1DN (per-channel, no mixing)."""
    y = _f64(x).copy()
    B, C, H, W = y.shape
    if np.ndim(gamma) == 1:
        lib().orc_norm1d(_p(y, ctypes.c_double), B, C, H, W, _p(_f64(beta), ctypes.c_double),
                         _p(_f64(gamma), ctypes.c_double), 1 if inverse else 0)
        return y
    lib().orc_gdn(_p(y, ctypes.c_double), B, C, H, W, _p(_f64(beta), ctypes.c_double),
                  _p(_f64(gamma), ctypes.c_double), 1 if inverse else 0)
    return y


def relu(x):
    return np.maximum(_f64(x), 0.0)


# --------------------------------------------------------------------------
# codec transforms (g_a, g_s, h_a, h_s)
# --------------------------------------------------------------------------

def g_a(Wt, x):
    """Analysis transform [1]: 4 x (conv5x5/2), GDN after the first three."""
    h = _f64(x)
    for i in range(4):
        h = conv2d(h, Wt[f"g_a.conv{i}.weight"], Wt[f"g_a.conv{i}.bias"], 2)
        if i < 3:
            h = gdn(h, Wt[f"g_a.gdn{i}.beta"], Wt[f"g_a.gdn{i}.gamma"])
    return h


def g_s(Wt, yhat):
    """Synthesis transform [1]: 4 x (deconv5x5/2), IGDN after the first three.
    Returns the unclamped reconstruction."""
    h = _f64(yhat)
    for i in range(4):
        h = deconv2d(h, Wt[f"g_s.deconv{i}.weight"], Wt[f"g_s.deconv{i}.bias"], 2)
        if i < 3:
            h = gdn(h, Wt[f"g_s.igdn{i}.beta"], Wt[f"g_s.igdn{i}.gamma"], inverse=True)
    return h


def h_a(Wt, y):
    """Hyper analysis [2]: on |y|: conv3x3/1, ReLU, conv5x5/2, ReLU, conv5x5/2."""
    h = np.abs(_f64(y))
    h = relu(conv2d(h, Wt["h_a.conv0.weight"], Wt["h_a.conv0.bias"], 1))
    h = relu(conv2d(h, Wt["h_a.conv1.weight"], Wt["h_a.conv1.bias"], 2))
    return conv2d(h, Wt["h_a.conv2.weight"], Wt["h_a.conv2.bias"], 2)


def h_s(Wt, zhat):
    """Hyper synthesis [2]: deconv5x5/2, ReLU, deconv5x5/2, ReLU, conv3x3/1, ReLU -> scales."""
    h = relu(deconv2d(zhat, Wt["h_s.deconv0.weight"], Wt["h_s.deconv0.bias"], 2))
    h = relu(deconv2d(h, Wt["h_s.deconv1.weight"], Wt["h_s.deconv1.bias"], 2))
    return relu(conv2d(h, Wt["h_s.conv2.weight"], Wt["h_s.conv2.bias"], 1))


# --------------------------------------------------------------------------
# entropy models
# --------------------------------------------------------------------------

def eb_pack(Wt):
    """Per-channel parameter blocks of the entropy bottleneck (C x 58 doubles)."""
    C = Wt["eb.H0"].shape[0]
    parts = [Wt[f"eb.H{k}"].reshape(C, -1) for k in range(5)]
    parts += [Wt[f"eb.b{k}"].reshape(C, -1) for k in range(5)]
    parts += [Wt[f"eb.a{k}"].reshape(C, -1) for k in range(4)]
    P = np.ascontiguousarray(np.concatenate(parts, axis=1), dtype=np.float64)
    assert P.shape[1] == 58
    return P


@dataclass
class Table:
    lo: int
    hi: int
    cdf: np.ndarray  # uint32, n+1 entries

    @property
    def n(self):
        return self.lo + self.hi + 2


def eb_tables(Wt):
    """(medians float32[C], [Table]) of the factorized entropy bottleneck."""
    P = eb_pack(Wt)
    C = P.shape[0]
    med = np.zeros(C, dtype=np.float32)
    tabs = []
    for c in range(C):
        cdf = np.zeros(4097, dtype=np.uint32)
        m = ctypes.c_float()
        lo, hi = ctypes.c_int(), ctypes.c_int()
        row = np.ascontiguousarray(P[c])
        rc = lib().orc_eb_table(_p(row, ctypes.c_double), ctypes.byref(m), ctypes.byref(lo),
                                ctypes.byref(hi), _p(cdf, ctypes.c_uint32))
        if rc != 0:
            raise ValueError(f"entropy bottleneck channel {c}: table build failed")
        med[c] = m.value
        tabs.append(Table(lo.value, hi.value, cdf[:lo.value + hi.value + 3].copy()))
    return med, tabs


def eb_pmf(Wt, c):
    """(median float32, lo, hi, pmf float64[lo+hi+2]) of channel c of the
    entropy bottleneck before frequency quantization (C7): the unit-bin
    likelihoods of s in [-lo, hi] around the median, then the escape mass."""
    row = np.ascontiguousarray(eb_pack(Wt)[c])
    pm = np.zeros(4096, dtype=np.float64)
    m = ctypes.c_float()
    lo, hi = ctypes.c_int(), ctypes.c_int()
    n = lib().orc_eb_pmf(_p(row, ctypes.c_double), ctypes.byref(m), ctypes.byref(lo),
                         ctypes.byref(hi), _p(pm, ctypes.c_double), 4096)
    if n < 0:
        raise ValueError(f"entropy bottleneck channel {c}: support above 4096 symbols")
    return np.float32(m.value), lo.value, hi.value, pm[:n].copy()


def eb_logits(Wt, c, x):
    P = eb_pack(Wt)
    row = np.ascontiguousarray(P[c])
    return lib().orc_eb_logits(_p(row, ctypes.c_double), float(x))


def scale_table():
    T = np.zeros(64, dtype=np.float32)
    lib().orc_scale_table(_p(T, ctypes.c_float))
    return T


def gauss_ztau():
    return lib().orc_gauss_ztau()


def gauss_tables():
    tabs = []
    for k in range(64):
        cdf = np.zeros(4097, dtype=np.uint32)
        c = ctypes.c_int()
        if lib().orc_gauss_table(k, ctypes.byref(c), _p(cdf, ctypes.c_uint32)) != 0:
            raise ValueError(f"gaussian table {k} failed")
        tabs.append(Table(c.value, c.value, cdf[:2 * c.value + 3].copy()))
    return tabs


def quantize_pmf(p):
    p = _f64(p)
    cdf = np.zeros(len(p) + 1, dtype=np.uint32)
    rc = lib().orc_quantize_pmf(_p(p, ctypes.c_double), len(p), _p(cdf, ctypes.c_uint32))
    if rc != 0:
        raise ValueError("pmf quantization failed")
    return cdf


# --------------------------------------------------------------------------
# quantization / index
# --------------------------------------------------------------------------

def quantize(y, mu=None):
    """s = rint(fl32(y - mu)) (C10); y is taken as float32."""
    y = np.ascontiguousarray(y, dtype=np.float32)
    B, C = y.shape[:2]
    HW = int(np.prod(y.shape[2:]))
    s = np.zeros(y.shape, dtype=np.int32)
    m = np.ascontiguousarray(mu, dtype=np.float32) if mu is not None else None
    lib().orc_quantize(_p(y, ctypes.c_float), B, C, HW,
                       _p(m, ctypes.c_float) if m is not None else None, _p(s, ctypes.c_int32))
    return s


def dequantize(s, mu=None):
    s = np.ascontiguousarray(s, dtype=np.int32)
    B, C = s.shape[:2]
    HW = int(np.prod(s.shape[2:]))
    y = np.zeros(s.shape, dtype=np.float32)
    m = np.ascontiguousarray(mu, dtype=np.float32) if mu is not None else None
    lib().orc_dequantize(_p(s, ctypes.c_int32), B, C, HW,
                         _p(m, ctypes.c_float) if m is not None else None, _p(y, ctypes.c_float))
    return y


def scale_index(sigma):
    sig = np.ascontiguousarray(sigma, dtype=np.float32)
    idx = np.zeros(sig.shape, dtype=np.uint8)
    T = scale_table()
    lib().orc_scale_index(_p(sig, ctypes.c_float), sig.size, _p(T, ctypes.c_float),
                          _p(idx, ctypes.c_uint8))
    return idx


# --------------------------------------------------------------------------
# rANS substreams
# --------------------------------------------------------------------------

def _ctables(tabs):
    arr = (_Table * len(tabs))()
    keep = []
    for i, t in enumerate(tabs):
        c = np.ascontiguousarray(t.cdf, dtype=np.uint32)
        keep.append(c)
        arr[i].lo, arr[i].hi, arr[i].n = t.lo, t.hi, t.n
        arr[i].cdf = _p(c, ctypes.c_uint32)
    return arr, keep


def rans_encode(s, tab_of, tabs, with_stats=False):
    """One substream: int32 symbols s[i] coded with tabs[tab_of[i]] (C12, C13)."""
    s = np.ascontiguousarray(s, dtype=np.int32).ravel()
    t = np.ascontiguousarray(tab_of, dtype=np.int32).ravel()
    n = len(s)
    cap = 10 * n + 64
    words = np.zeros(cap, dtype=np.uint16)
    nw = ctypes.c_int64()
    lw = np.zeros(32, dtype=np.int64)
    lb = np.zeros(32, dtype=np.float64)
    arr, keep = _ctables(tabs)
    rc = lib().orc_rans_encode(_p(s, ctypes.c_int32), _p(t, ctypes.c_int32), n, arr,
                               _p(words, ctypes.c_uint16), cap, ctypes.byref(nw),
                               _p(lw, ctypes.c_int64), _p(lb, ctypes.c_double))
    if rc != 0:
        raise ValueError("rans encode failed")
    out = words[:nw.value].copy()
    return (out, lw, lb) if with_stats else out


def rans_decode(words, n, tab_of, tabs):
    w = np.ascontiguousarray(words, dtype=np.uint16)
    t = np.ascontiguousarray(tab_of, dtype=np.int32).ravel()
    s = np.zeros(n, dtype=np.int32)
    arr, keep = _ctables(tabs)
    rc = lib().orc_rans_decode(_p(w, ctypes.c_uint16), len(w), n, _p(t, ctypes.c_int32), arr,
                               _p(s, ctypes.c_int32))
    if rc != 0:
        raise ValueError("corrupt substream")
    return s


def rans2_encode(s, tab_of, tabs, S=0, with_stats=False):
    """One format-2 substream (escape payloads outside the rANS words) and,
    with S > 0, its resume records (an array of shape (nrec, 35), uint32)."""
    s = np.ascontiguousarray(s, dtype=np.int32).ravel()
    t = np.ascontiguousarray(tab_of, dtype=np.int32).ravel()
    n = len(s)
    cap = 4 * n + 80
    out = np.zeros(cap, dtype=np.uint16)
    ng = (n + 31) // 32
    nr_max = (ng - 1) // S if (S > 0 and ng > 0) else 0
    rec = np.zeros(max(1, 35 * nr_max), dtype=np.uint32)
    ln, nrec = ctypes.c_int64(), ctypes.c_int64()
    lw = np.zeros(32, dtype=np.int64)
    lb = np.zeros(32, dtype=np.float64)
    arr, keep = _ctables(tabs)
    rc = lib().orc_rans2_encode(_p(s, ctypes.c_int32), _p(t, ctypes.c_int32), n, arr, int(S),
                                _p(out, ctypes.c_uint16), cap, ctypes.byref(ln), _p(rec, ctypes.c_uint32),
                                rec.size, ctypes.byref(nrec), _p(lw, ctypes.c_int64), _p(lb, ctypes.c_double))
    if rc != 0:
        raise ValueError("rans2 encode failed")
    words = out[:ln.value].copy()
    recs = rec[:35 * nrec.value].reshape(nrec.value, 35).copy()
    return (words, recs, lw, lb) if with_stats else (words, recs)


def rans2_decode(words, n, tab_of, tabs, rec=None, g0=0, g1=None):
    """Symbols of groups [g0, g1) of a format-2 substream (all of them by
    default), from its start or from the resume record of group g0; the
    returned array has n entries, those outside the range left 0."""
    w = np.ascontiguousarray(words, dtype=np.uint16)
    t = np.ascontiguousarray(tab_of, dtype=np.int32).ravel()
    out = np.zeros(max(n, 1), dtype=np.int32)
    g1 = (n + 31) // 32 if g1 is None else g1
    arr, keep = _ctables(tabs)
    r = None if rec is None else np.ascontiguousarray(rec, dtype=np.uint32)
    rc = lib().orc_rans2_decode_range(_p(w, ctypes.c_uint16), len(w), n, _p(t, ctypes.c_int32), arr,
                                      _p(r, ctypes.c_uint32) if r is not None else None, int(g0), int(g1),
                                      _p(out, ctypes.c_int32))
    if rc != 0:
        raise ValueError("corrupt substream")
    return out[:n]


# --------------------------------------------------------------------------
# frame container (project-defined; little endian)
#   'LIC1' | u16 version=1 | u16 kind | u16 N | u16 M | u32 H | u32 W |
#   u32 Hp | u32 Wp | u16 R | u16 0 | u32 nsub | u32 off[nsub+1] (words) |
#   u16 payload[off[nsub]]
# Substreams: hyperprior z first (one per channel, raster order), then y
# (one per channel and band of R latent rows, raster order inside a band).
# --------------------------------------------------------------------------

HEADER = struct.Struct("<4sHHHHIIIIHHI")
REC_U32 = 35   # u32 per resume record (format 2)


def pad_size(H, W):
    return (H + 63) // 64 * 64, (W + 63) // 64 * 64


def pack_frame(kind, N, M, H, W, Hp, Wp, R, subs, version=1, S=0, recs=None):
    """Format 1: header, u32 word offsets, substreams.  Format 2 adds the
    resume-record spacing S in the header's last u16 and, when S > 0, a
    trailer with every substream's records in order (35 u32 each)."""
    offs = [0]
    for s in subs:
        offs.append(offs[-1] + len(s))
    head = HEADER.pack(b"LIC1", version, kind, N, M, H, W, Hp, Wp, R, S if version == 2 else 0, len(subs))
    body = np.concatenate(subs).astype("<u2").tobytes() if subs else b""
    tail = b""
    if version == 2 and S > 0 and recs:
        tail = np.concatenate([np.asarray(r, np.uint32).ravel() for r in recs]).astype("<u4").tobytes()
    return head + np.asarray(offs, dtype="<u4").tobytes() + body + tail


def unpack_frame(buf):
    (magic, ver, kind, N, M, H, W, Hp, Wp, R, S, nsub) = HEADER.unpack_from(buf, 0)
    if magic != b"LIC1" or ver not in (1, 2) or (ver == 1 and S != 0):
        raise ValueError("bad header")
    offs = np.frombuffer(buf, dtype="<u4", count=nsub + 1, offset=HEADER.size)
    base = HEADER.size + 4 * (nsub + 1)
    if len(buf) < base + 2 * int(offs[-1]):
        raise ValueError("truncated")
    words = np.frombuffer(buf, dtype="<u2", count=int(offs[-1]), offset=base)
    subs = [words[offs[i]:offs[i + 1]] for i in range(nsub)]
    tail = np.frombuffer(buf, dtype="<u4", offset=base + 2 * int(offs[-1]))
    return dict(kind=kind, N=N, M=M, H=H, W=W, Hp=Hp, Wp=Wp, R=R, S=S, version=ver, subs=subs, trailer=tail)


def strip_records(buf):
    """A format-2 frame without its resume records: the trailer dropped and
    S set to 0 (the substreams are unchanged; a decoder then reads each
    substream from its start)."""
    h = unpack_frame(buf)
    if h["version"] != 2 or h["S"] == 0:
        return bytes(buf)
    end = HEADER.size + 4 * (len(h["subs"]) + 1) + 2 * sum(len(x) for x in h["subs"])
    out = bytearray(buf[:end])
    struct.pack_into("<H", out, 30, 0)
    return bytes(out)


def _bands(Hy, R):
    return [(r, min(r + R, Hy)) for r in range(0, Hy, R)]


@dataclass
class Codec:
    kind: int
    N: int
    M: int
    W: dict
    R: int = BAND_ROWS
    version: int = 1        # substream format: 1 escape nibbles in the rANS words, 2 outside them
    S: int = 0              # format 2: resume record every S groups of 32 symbols (0: none)
    med: np.ndarray = field(default=None)
    eb: list = field(default=None)
    gauss: list = field(default=None)

    def __post_init__(self):
        self.med, self.eb = eb_tables(self.W)
        if self.kind == KIND_HYPERPRIOR:
            self.gauss = gauss_tables()


def _substream_plan(codec: Codec, Hy, Wy, R=None):
    """(kind, channel, row0, row1) of every substream of a frame, in order:
    hyperprior z channels first, then each y channel's bands of R rows."""
    plan = []
    if codec.kind == KIND_HYPERPRIOR:
        plan += [("z", c, 0, Hy // 4) for c in range(codec.N)]
    for c in range(codec.M):
        plan += [("y", c, r0, r1) for r0, r1 in _bands(Hy, codec.R if R is None else R)]
    return plan


def encode_latents(codec: Codec, s_y, idx=None, s_z=None):
    """Substreams of one frame from its integer symbols.
    s_y: M x Hy x Wy int32; idx: M x Hy x Wy uint8 (hyper); s_z: N x Hz x Wz.
    Format 1 returns the list of substreams; format 2 returns (substreams,
    resume records per substream)."""
    subs, recs = [], []
    M, Hy, Wy = s_y.shape
    for part, c, r0, r1 in _substream_plan(codec, Hy, Wy):
        if part == "z":
            sym = s_z[c].ravel()
            tab, tabs = np.full(sym.size, c), codec.eb
        else:
            sym = s_y[c, r0:r1].ravel()
            if codec.kind == KIND_HYPERPRIOR:
                tab, tabs = idx[c, r0:r1].ravel().astype(np.int32), codec.gauss
            else:
                tab, tabs = np.full(sym.size, c), codec.eb
        if codec.version == 2:
            w, r = rans2_encode(sym, tab, tabs, codec.S)
            subs.append(w)
            recs.append(r)
        else:
            subs.append(rans_encode(sym, tab, tabs))
    return (subs, recs) if codec.version == 2 else subs


def _pack(codec: Codec, H, W, Hp, Wp, enc):
    if codec.version == 2:
        subs, recs = enc
        return pack_frame(codec.kind, codec.N, codec.M, H, W, Hp, Wp, codec.R, subs, 2, codec.S, recs)
    return pack_frame(codec.kind, codec.N, codec.M, H, W, Hp, Wp, codec.R, enc)


def encode(codec: Codec, frames):
    """Oracle encoder, FP64 transforms: frames B x 3 x H x W -> list of bytes.

    Also returns the intermediate values (dict) for stage-wise comparison."""
    frames = np.asarray(frames, dtype=np.float32)
    B, _, H, W = frames.shape
    Hp, Wp = pad_size(H, W)
    xp = np.pad(frames, ((0, 0), (0, 0), (0, Hp - H), (0, Wp - W)), mode="edge")
    y = g_a(codec.W, xp)
    inter = dict(y=y)
    out = []
    if codec.kind == KIND_HYPERPRIOR:
        z = h_a(codec.W, y)
        s_z = quantize(z.astype(np.float32), codec.med)
        zhat = dequantize(s_z, codec.med)
        sigma = h_s(codec.W, zhat)
        idx = scale_index(sigma.astype(np.float32))
        s_y = quantize(y.astype(np.float32))
        inter.update(z=z, s_z=s_z, zhat=zhat, sigma=sigma, idx=idx, s_y=s_y)
        for b in range(B):
            out.append(_pack(codec, H, W, Hp, Wp, encode_latents(codec, s_y[b], idx[b], s_z[b])))
    else:
        s_y = quantize(y.astype(np.float32), codec.med)
        inter.update(s_y=s_y)
        for b in range(B):
            out.append(_pack(codec, H, W, Hp, Wp, encode_latents(codec, s_y[b])))
    return out, inter


def _decode_sub(hdr, words, n, tab, tabs, recs):
    """One substream of either format; format 2 with records decodes each
    segment between records from its own record (as a parallel decoder
    would), and the whole substream must then also decode from its start."""
    if hdr["version"] == 1:
        return rans_decode(words, n, tab, tabs)
    whole = rans2_decode(words, n, tab, tabs)
    if len(recs):
        S, ng = hdr["S"], (n + 31) // 32
        seg = np.zeros(n, np.int32)
        bounds = [0] + [S * (r + 1) for r in range(len(recs))] + [ng]
        for r in range(len(recs) + 1):
            part = rans2_decode(words, n, tab, tabs, None if r == 0 else recs[r - 1], bounds[r], bounds[r + 1])
            seg[32 * bounds[r]:32 * bounds[r + 1]] = part[32 * bounds[r]:32 * bounds[r + 1]]
        if not np.array_equal(seg, whole):
            raise ValueError("resume records disagree with the substream")
    return whole


def decode_latents(codec: Codec, hdr):
    """Integer symbols of one frame from its parsed container (z, then h_s, then y)."""
    Hp, Wp, R = hdr["Hp"], hdr["Wp"], hdr["R"]
    Hy, Wy = Hp // 16, Wp // 16
    subs = hdr["subs"]
    S = hdr.get("S", 0) if hdr.get("version", 1) == 2 else 0
    plan = _substream_plan(codec, Hy, Wy, R)
    # resume records: per substream ((groups - 1) // S of them), in order
    trailer = hdr.get("trailer", np.zeros(0, np.uint32))
    nrec = []
    for part, c, r0, r1 in plan:
        n = (Hy // 4) * (Wy // 4) if part == "z" else (r1 - r0) * Wy
        ng = (n + 31) // 32
        nrec.append((ng - 1) // S if (S > 0 and ng > 0) else 0)
    if len(trailer) != REC_U32 * sum(nrec):
        raise ValueError("resume trailer size")
    recs, o = [], 0
    for k in nrec:
        recs.append(trailer[o:o + REC_U32 * k].reshape(k, REC_U32))
        o += REC_U32 * k
    k = 0
    res = {}
    if codec.kind == KIND_HYPERPRIOR:
        Hz, Wz = Hp // 64, Wp // 64
        s_z = np.zeros((codec.N, Hz, Wz), dtype=np.int32)
        for c in range(codec.N):
            s_z[c] = _decode_sub(hdr, subs[k], Hz * Wz, np.full(Hz * Wz, c), codec.eb, recs[k]).reshape(Hz, Wz)
            k += 1
        zhat = dequantize(s_z[None], codec.med)
        sigma = h_s(codec.W, zhat)
        idx = scale_index(sigma.astype(np.float32))[0]
        res.update(s_z=s_z, zhat=zhat[0], sigma=sigma[0], idx=idx)
    s_y = np.zeros((codec.M, Hy, Wy), dtype=np.int32)
    for c in range(codec.M):
        for r0, r1 in _bands(Hy, R):
            n = (r1 - r0) * Wy
            if codec.kind == KIND_HYPERPRIOR:
                t = idx[c, r0:r1].ravel().astype(np.int32)
                s_y[c, r0:r1] = _decode_sub(hdr, subs[k], n, t, codec.gauss, recs[k]).reshape(r1 - r0, Wy)
            else:
                s_y[c, r0:r1] = _decode_sub(hdr, subs[k], n, np.full(n, c), codec.eb, recs[k]).reshape(r1 - r0, Wy)
            k += 1
    res["s_y"] = s_y
    return res


def decode(codec: Codec, bitstreams):
    """Oracle decoder: list of frame bytes -> (B x 3 x H x W float64 clamped
    to [0, 1], intermediates)."""
    outs, inter = [], []
    for buf in bitstreams:
        hdr = unpack_frame(buf)
        lat = decode_latents(codec, hdr)
        mu = codec.med if codec.kind == KIND_FACTORIZED else None
        yhat = dequantize(lat["s_y"][None], mu)
        xr = g_s(codec.W, yhat)
        lat["x_pre"] = xr[0]
        outs.append(np.clip(xr[0], 0.0, 1.0)[:, :hdr["H"], :hdr["W"]])
        inter.append(lat)
    return np.stack(outs), inter


# --------------------------------------------------------------------------
# distilled student synthesis net (learned form): 4 x deconv5x5/2, ReLU
# after the first three, no IGDN; trained by MSE against the teacher's x_hat
# --------------------------------------------------------------------------

def deconv2d_wgrad(x, g, k=5, stride=2):
    x, g = _f64(x), _f64(g)
    B, Cin, H, W = x.shape
    Cout = g.shape[1]
    dw = np.zeros((Cin, Cout, k, k))
    lib().orc_deconv2d_wgrad(_p(x, ctypes.c_double), B, Cin, H, W, _p(g, ctypes.c_double), Cout, k, stride,
                             _p(dw, ctypes.c_double))
    return dw


def student_forward(P, yhat):
    """Activations [h0 = y_hat, h1, h2, h3] (post-ReLU) and the output."""
    hs = [_f64(yhat)]
    for l in range(4):
        z = deconv2d(hs[-1], P[f"student.deconv{l}.weight"], P[f"student.deconv{l}.bias"], 2)
        if l < 3:
            hs.append(relu(z))
        else:
            return hs, z


def student_loss_grads(P, yhat, target, masks=None):
    """MSE loss mean((out - target)^2) and its gradients with respect to every
    student parameter, by the chain rule: output gradient 2 (out - t) / n; per
    layer, the weight gradient of the transposed conv, the bias gradient
    (sum over positions), and the input gradient (the strided conv with the
    same weights -- the transposed conv's adjoint) masked by ReLU.

    masks: optional {l: boolean array shaped like h_l} for l = 1..3, the ReLU
    decisions h_l > 0 taken elsewhere (a pre-activation within rounding of 0
    may fall either way); by default h_l > 0 of this forward pass."""
    hs, out = student_forward(P, yhat)
    t = _f64(target)
    # the loss covers the central target-sized square of the output (all of
    # it when the sizes agree); the gradient is zero outside it
    o = (out.shape[-1] - t.shape[-1]) // 2
    core = out[:, :, o:o + t.shape[-2], o:o + t.shape[-1]]
    n = t.size
    loss = float(np.mean((core - t) ** 2))
    g = np.zeros_like(out)
    g[:, :, o:o + t.shape[-2], o:o + t.shape[-1]] = 2.0 * (core - t) / n
    grads = {}
    for l in range(3, -1, -1):
        w = _f64(P[f"student.deconv{l}.weight"])
        grads[f"student.deconv{l}.weight"] = deconv2d_wgrad(hs[l], g)
        grads[f"student.deconv{l}.bias"] = g.sum(axis=(0, 2, 3))
        if l > 0:
            mask = (hs[l] > 0) if masks is None else masks[l]
            g = conv2d(g, w, None, 2) * mask
    return loss, grads


def adam_step(P, G, m, v, t, lr=1e-4, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of every tensor in P,
    in place: m <- b1 m + (1 - b1) g; v <- b2 v + (1 - b2) g^2;
    m_hat = m / (1 - b1^t); v_hat = v / (1 - b2^t);
    theta <- theta - lr m_hat / (sqrt(v_hat) + eps).  t counts from 1."""
    for k in P:
        g = _f64(G[k])
        m[k] = beta1 * m[k] + (1.0 - beta1) * g
        v[k] = beta2 * v[k] + (1.0 - beta2) * g * g
        mh = m[k] / (1.0 - beta1 ** t)
        vh = v[k] / (1.0 - beta2 ** t)
        P[k] = _f64(P[k]) - lr * mh / (np.sqrt(vh) + eps)


def student_crops(yhat_pool, xhat_pool, crops, crop, halo=0):
    """A training batch: for each (frame, row, col) in latent units, the
    latent window of side crop/16 + 2 halo at (row, col) of y_hat, and the
    crop-square window of x_hat at 16 (row + halo), 16 (col + halo) -- the
    pixels the central crop of the window's output covers."""
    lc = crop // 16 + 2 * halo
    ys = np.stack([yhat_pool[f, :, r:r + lc, c:c + lc] for f, r, c in crops])
    xs = np.stack([xhat_pool[f, :, 16 * (r + halo):16 * (r + halo) + crop, 16 * (c + halo):16 * (c + halo) + crop]
                   for f, r, c in crops])
    return ys, xs


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)
