"""Seeded synthetic inputs: frames and codec parameters.

This module is the one place both the CUDA path and the FP64 oracle take
their inputs from.  It holds no arithmetic of the codec itself: it draws
random numbers (SplitMix64), shapes them into images and into initial
parameter tensors, and rounds everything to float32 so that both sides see
bit-identical inputs.

The paper (Sec. IV) evaluates CompressAI's pretrained factorized-prior [1]
and scale-hyperprior [2] models on a sample image and on Kodak; neither the
weights nor the images are available, so seeded stand-ins of the same shapes
are used (the recipe is spelled out below and in the design notes).
"""
from __future__ import annotations

import math
from collections import OrderedDict

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

KIND_FACTORIZED = 0
KIND_HYPERPRIOR = 1

WEIGHT_SEED = 1234
FRAME_SEED_BASE = 1000


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First ``n`` outputs of SplitMix64 started from state ``seed``.

    Output i is mix(seed + (i+1)*0x9E3779B97F4A7C15) with the published
    SplitMix64 finaliser (Steele, Lea, Flood 2014), all arithmetic mod 2^64.
    """
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# --------------------------------------------------------------------------
# Codec parameters
# --------------------------------------------------------------------------

def _layer_list(kind: int, N: int, M: int):
    """(name, op, Cin, Cout, k) for every conv-like layer, in the fixed order.

    g_a: 4 x conv5x5/2 (3->N->N->N->M) with GDN between (Ballé 2017 [1]);
    g_s: the mirror with transposed convs and IGDN;
    h_a: conv3x3/1 M->N, ReLU, conv5x5/2, ReLU, conv5x5/2;
    h_s: deconv5x5/2, ReLU, deconv5x5/2, ReLU, conv3x3/1 N->M, ReLU (Ballé 2018 [2]).
    """
    L = [
        ("g_a.conv0", "conv", 3, N, 5), ("g_a.conv1", "conv", N, N, 5),
        ("g_a.conv2", "conv", N, N, 5), ("g_a.conv3", "conv", N, M, 5),
        ("g_s.deconv0", "deconv", M, N, 5), ("g_s.deconv1", "deconv", N, N, 5),
        ("g_s.deconv2", "deconv", N, N, 5), ("g_s.deconv3", "deconv", N, 3, 5),
    ]
    if kind == KIND_HYPERPRIOR:
        L += [
            ("h_a.conv0", "conv", M, N, 3), ("h_a.conv1", "conv", N, N, 5),
            ("h_a.conv2", "conv", N, N, 5),
            ("h_s.deconv0", "deconv", N, N, 5), ("h_s.deconv1", "deconv", N, N, 5),
            ("h_s.conv2", "conv", N, M, 3),
        ]
    return L


# Per-layer multipliers of the Kaiming-uniform weight bound and additive bias
# offsets.  They keep an untrained, seeded codec in a codec-like regime: the
# reconstruction mostly inside [0, 1] and the hyper-synthesis scales of the
# order of the latents they describe.  Chosen once by measurement of the
# statistics of the seeded codec; they are part of the input recipe.
WEIGHT_GAIN = {
    "g_s.deconv3": 0.25,
    "h_s.conv2": 0.5,
}
BIAS_OFFSET = {
    "g_s.deconv3": 0.5,
    "h_s.conv2": 0.5,
}

EB_FILTERS = (1, 3, 3, 3, 3, 1)
EB_INIT_SCALE = 10.0


def param_names(kind: int, N: int, M: int):
    """Ordered parameter names (also the seed order)."""
    names = []
    for name, op, cin, cout, k in _layer_list(kind, N, M):
        names += [name + ".weight", name + ".bias"]
    for i in range(3):
        names += [f"g_a.gdn{i}.beta", f"g_a.gdn{i}.gamma"]
    for i in range(3):
        names += [f"g_s.igdn{i}.beta", f"g_s.igdn{i}.gamma"]
    for k in range(5):
        names += [f"eb.H{k}", f"eb.b{k}"]
        if k < 4:
            names.append(f"eb.a{k}")
    return names


def _param_seed(j: int) -> int:
    return (WEIGHT_SEED << 20) + j


NORM_GDN = 0
NORM_1DN = 1


def make_weights(kind: int, N: int = 128, M: int = 192, norm: int = NORM_GDN) -> "OrderedDict[str, np.ndarray]":
    """Seeded parameters of a factorized-prior (kind 0) or hyperprior (kind 1) codec.

    Recipe:
    * conv weight [Cout, Cin, k, k] and deconv weight [Cin, Cout, k, k]:
      U(-g*sqrt(6/fan_in), g*sqrt(6/fan_in)), fan_in = Cin*k*k with Cin the
      layer's input channels, g = WEIGHT_GAIN (default 1);
    * bias: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) + BIAS_OFFSET (default 0);
    * GDN/IGDN: beta = 1, gamma = 0.1*I + U(0, 0.01) on every entry; with
      norm = NORM_1DN the per-channel gamma [C] = 0.1 + U(0, 0.01) instead
      (same parameter names, same streams);
    * entropy bottleneck of C channels (C = M for the factorized codec, the
      latent it codes; C = N for the hyperprior, coding z), filters
      (1,3,3,3,3,1), init_scale 10 as in Ballé 2018 [2] appendix 6.1:
      H_k = log(expm1(1/(S*f_out))) with S = init_scale^(1/5), b_k ~ U(-0.5, 0.5),
      a_k = 0.
    Parameter j (in ``param_names`` order) draws from SplitMix64 stream
    ``(1234 << 20) + j``.  Every tensor is returned as float32.
    The factorized and hyperprior codecs share g_a/g_s parameters (same
    names, same stream indices).
    """
    names = param_names(kind, N, M)
    seed_of = {n: _param_seed(j) for j, n in enumerate(names)}
    out: "OrderedDict[str, np.ndarray]" = OrderedDict()
    layers = {name: (op, cin, cout, k) for name, op, cin, cout, k in _layer_list(kind, N, M)}
    C_eb = M if kind == KIND_FACTORIZED else N
    S = EB_INIT_SCALE ** (1.0 / (len(EB_FILTERS) - 1))
    for pname in names:
        seed = seed_of[pname]
        base, leaf = pname.rsplit(".", 1)
        if base in layers:
            op, cin, cout, k = layers[base]
            fan_in = cin * k * k
            if leaf == "weight":
                shape = (cout, cin, k, k) if op == "conv" else (cin, cout, k, k)
                bound = WEIGHT_GAIN.get(base, 1.0) * math.sqrt(6.0 / fan_in)
                u = uniform01(seed, int(np.prod(shape)))
                arr = ((2.0 * u - 1.0) * bound).reshape(shape)
            else:
                bound = 1.0 / math.sqrt(fan_in)
                u = uniform01(seed, cout)
                arr = (2.0 * u - 1.0) * bound + BIAS_OFFSET.get(base, 0.0)
        elif ".gdn" in base or ".igdn" in base:
            C = N
            if leaf == "beta":
                arr = np.ones(C)
            elif norm == NORM_1DN:
                arr = 0.1 + 0.01 * uniform01(seed, C)
            else:
                arr = 0.1 * np.eye(C) + 0.01 * uniform01(seed, C * C).reshape(C, C)
        else:  # entropy bottleneck
            k = int(leaf[1:])
            fin, fout = EB_FILTERS[k], EB_FILTERS[k + 1]
            if leaf[0] == "H":
                init = math.log(math.expm1(1.0 / S / fout))
                arr = np.full((C_eb, fout, fin), init)
            elif leaf[0] == "b":
                arr = uniform01(seed, C_eb * fout).reshape(C_eb, fout) - 0.5
            else:
                arr = np.zeros((C_eb, fout))
        out[pname] = np.ascontiguousarray(arr, dtype=np.float32)
    return out


# --------------------------------------------------------------------------
# Frames
# --------------------------------------------------------------------------

def _gauss_kernel(sigma: float, radius: int) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-0.5 * (t / sigma) ** 2)
    return g / g.sum()


def _lowpass_reflect(a: np.ndarray, g: np.ndarray) -> np.ndarray:
    r = (len(g) - 1) // 2
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        p = np.pad(a, pad, mode="reflect")
        acc = np.zeros_like(a)
        n = a.shape[axis]
        for t, gt in enumerate(g):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(t, t + n)
            acc += gt * p[tuple(sl)]
        a = acc
    return a


def make_frame(index: int, H: int, W: int) -> np.ndarray:
    """One seeded 3 x H x W float32 frame in [0, 1].

    Stand-in for the paper's sample image / Kodak (Sec. V): per channel a
    random linear gradient, plus 0.15 x unit-std Gaussian noise low-passed by
    a separable Gaussian (sigma 8 px, radius 24, reflect), then 8 solid
    rectangles (side U[W/16, W/4], colour U(0,1)^3) pasted over, then a clamp
    to [0, 1].  Frame ``index`` draws from SplitMix64 stream 1000 + index.
    """
    seed = FRAME_SEED_BASE + index
    # Draw order: 9 gradient coefficients, 2*H*W*3 noise uniforms
    # (Box-Muller pairs), 8*(4+3) rectangle parameters.
    n_noise = 3 * H * W
    n_pairs = (n_noise + 1) // 2
    u = uniform01(seed, 9 + 2 * n_pairs + 8 * 7)
    coef = u[:9].reshape(3, 3)
    u1 = u[9:9 + n_pairs]
    u2 = u[9 + n_pairs:9 + 2 * n_pairs]
    rect = u[9 + 2 * n_pairs:].reshape(8, 7)
    r = np.sqrt(-2.0 * np.log1p(-u1))          # 1-u1 in (0, 1]
    th = 2.0 * math.pi * u2
    gauss = np.concatenate([r * np.cos(th), r * np.sin(th)])[:n_noise].reshape(3, H, W)

    yy = np.linspace(0.0, 1.0, H)[:, None]
    xx = np.linspace(0.0, 1.0, W)[None, :]
    g = _gauss_kernel(8.0, 24)
    img = np.empty((3, H, W), dtype=np.float64)
    for c in range(3):
        a, b, cc = coef[c]
        grad = (a + b * xx + cc * yy) / (a + b + cc)
        n = gauss[c]
        if H > 48 and W > 48:
            n = _lowpass_reflect(n, g)
        sd = n.std()
        n = n / sd if sd > 0 else n
        img[c] = grad + 0.15 * n
    lo_side, hi_side = W / 16.0, W / 4.0
    for k in range(8):
        px, py, sw, sh, cr, cg, cb = rect[k]
        w = int(lo_side + sw * (hi_side - lo_side))
        h = int(lo_side + sh * (hi_side - lo_side))
        x0 = int(px * max(W - w, 1))
        y0 = int(py * max(H - h, 1))
        img[0, y0:y0 + h, x0:x0 + w] = cr
        img[1, y0:y0 + h, x0:x0 + w] = cg
        img[2, y0:y0 + h, x0:x0 + w] = cb
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def make_frames(B: int, H: int, W: int, first: int = 0) -> np.ndarray:
    """B seeded frames stacked as a B x 3 x H x W float32 array."""
    return np.stack([make_frame(first + i, H, W) for i in range(B)])


# --------------------------------------------------------------------------
# Distilled student synthesis net (learned form)
# --------------------------------------------------------------------------

STUDENT_SEED = 4321
CROP_SEED = 7777


def student_param_names():
    return [f"student.deconv{l}.{leaf}" for l in range(4) for leaf in ("weight", "bias")]


def make_student_weights(M: int = 192, C: int = 64) -> "OrderedDict[str, np.ndarray]":
    """Initial parameters of the student g_s: 4 transposed convs 5x5 / 2,
    M -> C -> C -> C -> 3, weights [Cin, Cout, 5, 5].  Same Kaiming-uniform
    recipe as the codec (fan_in = Cin*25); the last layer takes the codec's
    g_s.deconv3 gain (0.25) and bias offset (0.5) so the initial output sits
    inside [0, 1].  Parameter j draws from SplitMix64 stream (4321 << 20) + j."""
    chans = (M, C, C, C, 3)
    out: "OrderedDict[str, np.ndarray]" = OrderedDict()
    for j, pname in enumerate(student_param_names()):
        l = int(pname.split(".")[1][len("deconv"):])
        cin, cout = chans[l], chans[l + 1]
        fan_in = cin * 25
        u = uniform01((STUDENT_SEED << 20) + j, cin * cout * 25 if pname.endswith("weight") else cout)
        if pname.endswith("weight"):
            bound = (0.25 if l == 3 else 1.0) * math.sqrt(6.0 / fan_in)
            arr = ((2.0 * u - 1.0) * bound).reshape(cin, cout, 5, 5)
        else:
            arr = (2.0 * u - 1.0) / math.sqrt(fan_in) + (0.5 if l == 3 else 0.0)
        out[pname] = np.ascontiguousarray(arr, dtype=np.float32)
    return out


def draw_crops(step: int, B: int, P: int, Hy: int, Wy: int, lc: int) -> np.ndarray:
    """Crop positions of training step ``step``: B rows of (frame, row, col)
    in latent units, frame uniform over the P pool frames and the lc x lc
    latent window uniform over the Hy x Wy latent plane.  SplitMix64 stream
    (7777 << 20) + step."""
    u = uniform01((CROP_SEED << 20) + step, 3 * B).reshape(B, 3)
    f = np.minimum((u[:, 0] * P).astype(np.int64), P - 1)
    r = np.minimum((u[:, 1] * (Hy - lc + 1)).astype(np.int64), Hy - lc)
    c = np.minimum((u[:, 2] * (Wy - lc + 1)).astype(np.int64), Wy - lc)
    return np.ascontiguousarray(np.stack([f, r, c], axis=1), dtype=np.int32)


# --------------------------------------------------------------------------
# Serving workload
# --------------------------------------------------------------------------

SERVE_SEED = 7
SERVE_STREAMS = ((6, 480, 640), (6, 720, 1280), (4, 1080, 1920))   # (streams, H, W)


def poisson_arrivals(seconds: float, rate: float = 30.0, streams=SERVE_STREAMS, seed: int = SERVE_SEED):
    """Arrival times of every stream's frames over [0, seconds): each stream
    a Poisson process of ``rate`` frames/s (exponential gaps -ln(1-u)/rate,
    u from SplitMix64 stream (seed << 20) + stream index).  Returns a list of
    (t_seconds, stream_id, H, W) sorted by time."""
    out = []
    sid = 0
    for count, H, W in streams:
        for _ in range(count):
            n = int(seconds * rate * 3 + 64)
            gaps = -np.log1p(-uniform01((seed << 20) + sid, n)) / rate
            t = np.cumsum(gaps)
            out += [(float(x), sid, H, W) for x in t[t < seconds]]
            sid += 1
    out.sort()
    return out
