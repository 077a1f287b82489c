"""Pins of the FP64 oracle against facts it does not compute itself:
library routines (torch float64 conv, scipy's normal quantile, numpy rint),
closed forms, identities, invariants, brute force and hand-computed
bitstreams.  Each test names the definition it pins.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2208_01641_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(7)


# ---------------------------------------------------------------- transforms

def naive_conv(x, w, b, s):
    """7-loop brute force of the strided zero-padded convolution (C1)."""
    B, Cin, H, W = x.shape
    Cout, _, k, _ = w.shape
    p = k // 2
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1
    y = np.zeros((B, Cout, Ho, Wo))
    for n in range(B):
        for o in range(Cout):
            for i in range(Ho):
                for j in range(Wo):
                    acc = b[o]
                    for c in range(Cin):
                        for u in range(k):
                            for v in range(k):
                                r, q = s * i + u - p, s * j + v - p
                                if 0 <= r < H and 0 <= q < W:
                                    acc += w[o, c, u, v] * x[n, c, r, q]
                    y[n, o, i, j] = acc
    return y


@pytest.mark.parametrize("k,s", [(5, 2), (3, 1)])
def test_conv_brute_force(k, s):
    x = rng.standard_normal((2, 3, 6, 8))
    w = rng.standard_normal((4, 3, k, k))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(O.conv2d(x, w, b, s), naive_conv(x, w, b, s), rtol=0, atol=1e-12)


@pytest.mark.parametrize("k,s,cin,cout,hw", [(5, 2, 5, 7, 12), (3, 1, 6, 4, 9), (5, 2, 3, 8, 16)])
def test_conv_matches_torch_f64(k, s, cin, cout, hw):
    x = rng.standard_normal((2, cin, hw, hw + 2))
    w = rng.standard_normal((cout, cin, k, k))
    b = rng.standard_normal(cout)
    ref = torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b),
                                     stride=s, padding=k // 2).numpy()
    np.testing.assert_allclose(O.conv2d(x, w, b, s), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("cin,cout,h,w", [(5, 7, 4, 6), (3, 2, 7, 5)])
def test_deconv_matches_torch_f64(cin, cout, h, w):
    x = rng.standard_normal((2, cin, h, w))
    wt = rng.standard_normal((cin, cout, 5, 5))
    b = rng.standard_normal(cout)
    ref = torch.nn.functional.conv_transpose2d(torch.from_numpy(x), torch.from_numpy(wt),
                                               torch.from_numpy(b), stride=2, padding=2,
                                               output_padding=1).numpy()
    out = O.deconv2d(x, wt, b, 2)
    assert out.shape == (2, cout, 2 * h, 2 * w)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12)


def test_conv_deconv_adjoint():
    """<conv_W x, y> = <x, deconv_W y> with zero bias (C2): the transposed
    convolution is the adjoint of the strided convolution."""
    x = rng.standard_normal((1, 6, 16, 12))
    w = rng.standard_normal((5, 6, 5, 5))
    y = rng.standard_normal((1, 5, 8, 6))
    lhs = float(np.sum(O.conv2d(x, w, None, 2) * y))
    rhs = float(np.sum(x * O.deconv2d(y, w, None, 2)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_gdn_identity():
    """GDN with gamma = 0, beta = 1 is the identity, exactly (C3)."""
    x = rng.standard_normal((2, 5, 3, 4))
    out = O.gdn(x, np.ones(5), np.zeros((5, 5)))
    assert np.array_equal(out, x)
    assert np.array_equal(O.gdn(x, np.ones(5), np.zeros((5, 5)), inverse=True), x)


def test_gdn_off_diagonal_closed_form():
    """One off-diagonal gamma[0,1] = g: y0 = x0/sqrt(b0 + g x1^2), y1 = x1/sqrt(b1).
    Fails if gamma is transposed or the square is dropped."""
    x = rng.standard_normal((1, 2, 3, 3))
    beta = np.array([0.7, 1.3])
    gamma = np.array([[0.0, 0.4], [0.0, 0.0]])
    out = O.gdn(x, beta, gamma)
    np.testing.assert_allclose(out[:, 0], x[:, 0] / np.sqrt(0.7 + 0.4 * x[:, 1] ** 2), atol=1e-15)
    np.testing.assert_allclose(out[:, 1], x[:, 1] / math.sqrt(1.3), atol=1e-15)
    inv = O.gdn(x, beta, gamma, inverse=True)
    np.testing.assert_allclose(inv[:, 0], x[:, 0] * np.sqrt(0.7 + 0.4 * x[:, 1] ** 2), atol=1e-15)


def test_gdn_scale_invariance():
    """With beta = 0, GDN is invariant to positive scaling and IGDN is
    homogeneous of degree 2 (invariant of the definition)."""
    x = rng.standard_normal((1, 4, 2, 2)) + 0.1
    gamma = np.abs(rng.standard_normal((4, 4))) + 0.1
    z = np.zeros(4)
    np.testing.assert_allclose(O.gdn(3.0 * x, z, gamma), O.gdn(x, z, gamma), rtol=1e-13)
    np.testing.assert_allclose(O.gdn(3.0 * x, z, gamma, True), 9.0 * O.gdn(x, z, gamma, True), rtol=1e-13)


# ---------------------------------------------------------- entropy models

def _eb_params(C, s_vals, b=0.0, a=0.0):
    """Entropy-bottleneck parameters whose softplus(H_k) entries all equal s_vals[k]."""
    W = {}
    f = synth.EB_FILTERS
    for k in range(5):
        W[f"eb.H{k}"] = np.full((C, f[k + 1], f[k]), math.log(math.expm1(s_vals[k])))
        W[f"eb.b{k}"] = np.full((C, f[k + 1]), b)
        if k < 4:
            W[f"eb.a{k}"] = np.full((C, f[k + 1]), a)
    return W


def test_eb_linear_closed_form():
    """a = b = 0: the net is linear, logit(x) = 3^4 * prod_k softplus(H_k) * x."""
    s = [0.3, 0.2, 0.5, 0.25, 0.4]
    W = _eb_params(1, s)
    slope = 81 * np.prod(s)
    for x in (-3.0, 0.5, 7.25):
        assert abs(O.eb_logits(W, 0, x) - slope * x) < 1e-12


def test_eb_scalar_recursion_closed_form():
    """Equal entries per layer make every hidden unit equal, so the 1-3-3-3-3-1
    net reduces to a scalar recursion h <- w_k*h + b + tanh(a)*tanh(w_k*h + b)
    with w_1 = s_1 and w_k = 3 s_k afterwards."""
    s = [0.9, 0.4, 0.7, 0.5, 0.6]
    b, a = 0.3, 0.8
    W = _eb_params(1, s, b=b, a=a)
    for x in (-2.0, 0.1, 1.7):
        h = x
        for k in range(5):
            h = (s[k] if k == 0 else 3 * s[k]) * h + b
            if k < 4:
                h = h + math.tanh(a) * math.tanh(h)
        assert abs(O.eb_logits(W, 0, x) - h) < 1e-12


def test_eb_cdf_monotone_and_limits():
    W = synth.make_weights(synth.KIND_HYPERPRIOR, 8, 12)
    xs = np.linspace(-500, 500, 2001)
    for c in range(8):
        lg = np.array([O.eb_logits(W, c, x) for x in xs])
        assert np.all(np.diff(lg) > 0)
        cdf = 1 / (1 + np.exp(-lg))
        assert cdf[0] < 1e-9 and cdf[-1] > 1 - 1e-9


def test_eb_median_and_tails_linear_case():
    """Linear net of slope k: median 0, tails at logit(tau/2)/k (C7)."""
    s = [0.5, 0.5, 0.5, 0.5, 0.5]
    W = _eb_params(1, s)
    med, tabs = O.eb_tables(W)
    assert med[0] == 0.0
    slope = 81 * 0.5 ** 5
    q = -math.log((1 - 5e-10) / 5e-10) / slope
    assert tabs[0].lo == math.ceil(-q) and tabs[0].hi == math.ceil(-q)


def _check_cdf(cdf):
    cdf = np.asarray(cdf, dtype=np.int64)
    f = np.diff(cdf)
    assert cdf[0] == 0 and cdf[-1] == 65536
    assert np.all(f >= 1)


def test_eb_tables_valid():
    W = synth.make_weights(synth.KIND_HYPERPRIOR, 16, 24)
    med, tabs = O.eb_tables(W)
    assert len(tabs) == 16
    for t in tabs:
        assert len(t.cdf) == t.n + 1 and t.n <= 4096
        _check_cdf(t.cdf)


def test_scale_table_pins():
    """64 log-spaced scales 0.11 .. 256 (configs): end points and constant ratio."""
    T = O.scale_table()
    assert T[0] == np.float32(0.11) and T[63] == np.float32(256.0)
    r = T[1:].astype(np.float64) / T[:-1]
    assert np.allclose(r, (256 / 0.11) ** (1 / 63), rtol=1e-6)
    assert abs(r.mean() - 1.13095) < 1e-5


def test_ztau_matches_scipy():
    from scipy.special import ndtri
    assert abs(O.gauss_ztau() + ndtri(0.5e-9)) < 1e-9


def test_gauss_pmf_sums_to_one_and_matches_erfc():
    """The pmf of table k (plus its escape mass) sums to 1, and each entry
    equals an independent computation with scipy's normal CDF (C8)."""
    from scipy.stats import norm
    T = O.scale_table()
    z = O.gauss_ztau()
    tabs = O.gauss_tables()
    for k in (0, 17, 40, 63):
        sg = float(T[k])
        c = math.ceil(sg * z)
        s = np.arange(-c, c + 1)
        p = norm.cdf((0.5 - np.abs(s)) / sg) - norm.cdf((-0.5 - np.abs(s)) / sg)
        esc = 2 * norm.cdf((-c - 0.5) / sg)
        assert abs(p.sum() + esc - 1.0) < 1e-12
        t = tabs[k]
        assert t.lo == c
        f = np.diff(t.cdf.astype(np.int64))
        # every quantized frequency within one unit (plus the deficit/surplus fix) of 65536 p
        approx = np.maximum(1, np.floor(np.append(p, esc) * 65536 + 0.5))
        assert np.abs(f - approx).sum() == abs(65536 - approx.sum())


def test_gauss_tables_valid_and_sizes():
    tabs = O.gauss_tables()
    assert len(tabs) == 64
    for t in tabs:
        _check_cdf(t.cdf)
    assert tabs[63].n == 3132
    assert sum(t.n for t in tabs) == 27192


def test_quantize_pmf_rules():
    """Frequency quantization (C9) on pmfs worked out by hand."""
    assert list(O.quantize_pmf([0.25] * 4)) == [0, 16384, 32768, 49152, 65536]
    # deficit: 3 x floor(65536/3 + .5) = 3 x 21845 = 65535 -> +1 to the first largest
    assert list(np.diff(O.quantize_pmf([1 / 3] * 3))) == [21846, 21845, 21845]
    # surplus: two tiny symbols forced to 1 -> 2 units taken from the largest
    # surplus: two tiny symbols forced to 1 -> both units taken from the first largest
    p = [0.5, 0.5, 1e-9, 1e-9]
    assert list(np.diff(O.quantize_pmf(p))) == [32766, 32768, 1, 1]
    # surplus larger than the largest can give: 4000 x 17 = 68000, 2464 over;
    # each symbol in index order gives 16 until the surplus is gone
    p = [16.5 / 65536] * 4000
    f = np.diff(O.quantize_pmf(p))
    assert list(f) == [1] * 154 + [17] * 3846


# ------------------------------------------------------ quantization / index

def test_quantize_special_values():
    y = np.array([[[0.5, 1.5, -0.5, 2.5, -2.5, 0.49999997, np.nan, 3e9, -3e9]]], dtype=np.float32)
    s = O.quantize(y)
    assert list(s.ravel()) == [0, 2, 0, 2, -2, 0, 0, 2 ** 30, -(2 ** 30)]


def test_quantize_matches_numpy_rint_with_mean():
    y = (rng.standard_normal((2, 3, 50)) * 20).astype(np.float32)
    mu = rng.standard_normal(3).astype(np.float32)
    d = (y - mu[None, :, None]).astype(np.float32)
    assert np.array_equal(O.quantize(y, mu), np.rint(d).astype(np.int32))
    yh = O.dequantize(O.quantize(y, mu), mu)
    assert np.array_equal(yh, (np.rint(d) + mu[None, :, None]).astype(np.float32))


def test_scale_index_brute_force():
    """idx = min{k : T[k] >= max(sigma, 0.11f)} checked against numpy's
    searchsorted over every float bit pattern near each table entry and a
    dense stride over [0.1, 300] (C11)."""
    T = O.scale_table()
    bits = [np.arange(0x3DCCCCCD - 4096, 0x43960000, 13, dtype=np.uint32)]
    for t in T:
        tb = np.float32(t).view(np.uint32)
        bits.append(np.arange(tb - 64, tb + 64, dtype=np.uint32))
    vals = np.concatenate(bits).view(np.float32)
    vals = np.concatenate([vals, np.array([0.0, -1.0, 1e30, np.inf, np.nan], np.float32)])
    idx = O.scale_index(vals)
    v = np.maximum(np.nan_to_num(vals, nan=1e38), T[0])
    ref = np.minimum(np.searchsorted(T, v, side="left"), 63)
    ref[np.isnan(vals)] = 63
    assert np.array_equal(idx, ref.astype(np.uint8))
    assert O.scale_index(T).tolist() == list(range(64))


# ---------------------------------------------------------------------- rANS

def _tab(lo, hi, cdf):
    return O.Table(lo, hi, np.asarray(cdf, dtype=np.uint32))


def test_rans_hand_computed():
    g = json.load(open(os.path.join(GOLD, "rans_hand.json")))
    for key in ("uniform3", "escape1"):
        case = g[key]
        t = _tab(case["lo"], case["hi"], case["cdf"])
        sy = np.array(case["symbols"], np.int32)
        words = O.rans_encode(sy, np.zeros(len(sy)), [t])
        assert words.tolist() == case["words"], key
        assert O.rans_decode(words, len(sy), np.zeros(len(sy)), [t]).tolist() == case["symbols"]


def _random_tables():
    tabs = O.gauss_tables()
    return tabs


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1000])
def test_rans_roundtrip_gauss(n):
    tabs = _random_tables()
    idx = rng.integers(0, 64, n).astype(np.int32)
    T = O.scale_table()
    s = np.rint(rng.standard_normal(n) * T[idx] * 1.3).astype(np.int32)
    w = O.rans_encode(s, idx, tabs)
    assert O.rans_decode(w, n, idx, tabs).tolist() == s.tolist()


def test_rans_roundtrip_adversarial():
    tabs = _random_tables()
    n = 300
    idx = np.zeros(n, np.int32)
    # all escapes, with payloads of 1..8 nibbles and both signs, plus extremes
    s = np.array([(1 if i % 2 else -1) * (2 + (7 ** (i % 11))) for i in range(n)], np.int32)
    s[:4] = [2 ** 30, -(2 ** 30), 2, -2]
    w = O.rans_encode(s, idx, tabs)
    assert O.rans_decode(w, n, idx, tabs).tolist() == s.tolist()
    # f = 1 symbols: the outer ends of the widest table
    t = tabs[63]
    s = np.array([-t.lo, t.hi] * 40, np.int32)
    idx = np.full(len(s), 63, np.int32)
    w = O.rans_encode(s, idx, tabs)
    assert O.rans_decode(w, len(s), idx, tabs).tolist() == s.tolist()


def test_rans_corrupt_is_detected():
    tabs = _random_tables()
    idx = np.full(200, 20, np.int32)
    s = rng.integers(-3, 4, 200).astype(np.int32)
    w = O.rans_encode(s, idx, tabs)
    with pytest.raises(ValueError):
        O.rans_decode(w[:10], 200, idx, tabs)


def test_rans_code_length_bound():
    """Per interleaved state: emitted bits <= 1.01 * sum(-log2 p) + 64
    (each state's 32-bit flush is the +64 reading's constant).  Also a
    single-state check over a whole substream (n < 32 is a single lane each)."""
    tabs = _random_tables()
    T = O.scale_table()
    for k in (3, 12, 30, 50):
        n = 32 * 400
        idx = np.full(n, k, np.int32)
        s = np.rint(rng.standard_normal(n) * T[k]).astype(np.int32)
        w, lw, lb = O.rans_encode(s, idx, tabs, with_stats=True)
        assert len(w) == lw.sum() + 64
        bits = 16.0 * (lw + 2)
        assert np.all(bits <= 1.01 * lb + 64), (k, bits - lb)


# -------------------------------------------------------- container / chain

def test_container_roundtrip():
    subs = [np.array([1, 2, 3], np.uint16), np.array([], np.uint16), np.array([9], np.uint16)]
    buf = O.pack_frame(1, 128, 192, 720, 1280, 768, 1280, 16, subs)
    assert buf[:4] == b"LIC1" and len(buf) == 36 + 4 * 4 + 2 * 4
    h = O.unpack_frame(buf)
    assert (h["H"], h["W"], h["Hp"], h["Wp"], h["R"]) == (720, 1280, 768, 1280, 16)
    assert [x.tolist() for x in h["subs"]] == [[1, 2, 3], [], [9]]


@pytest.mark.parametrize("kind", [0, 1])
def test_oracle_chain_lossless_symbols(kind):
    """Encode then decode: the decoder recovers exactly the encoder's symbols
    (and, for the hyperprior, the same scale indices), and the frame is
    g_s of the dequantized symbols, clamped and cropped."""
    N, M = 16, 24
    W = synth.make_weights(kind, N, M)
    C = O.Codec(kind, N, M, W)
    x = synth.make_frames(1, 70, 100)
    bs, enc = O.encode(C, x)
    xr, dec = O.decode(C, bs)
    assert xr.shape == (1, 3, 70, 100)
    assert np.array_equal(dec[0]["s_y"], enc["s_y"][0])
    if kind == 1:
        assert np.array_equal(dec[0]["s_z"], enc["s_z"][0])
        assert np.array_equal(dec[0]["idx"], enc["idx"][0])
    mu = C.med if kind == 0 else None
    ref = O.g_s(W, O.dequantize(enc["s_y"], mu))
    assert np.array_equal(xr, np.clip(ref, 0, 1)[:, :, :70, :100])


def test_norm1d_is_gdn_with_diagonal_gamma():
    """1DN (no channel mixing) equals the pinned GDN with a diagonal gamma
    matrix, forward and inverse; with gamma = 0, beta = 1 it is the identity."""
    x = rng.standard_normal((2, 6, 3, 4)) * 2
    beta = 0.5 + rng.random(6)
    g = 0.05 + rng.random(6)
    for inv in (False, True):
        np.testing.assert_allclose(O.gdn(x, beta, g, inverse=inv), O.gdn(x, beta, np.diag(g), inverse=inv),
                                   rtol=1e-14, atol=0)
    assert np.array_equal(O.gdn(x, np.ones(6), np.zeros(6)), x)


def test_norm1d_codec_roundtrip():
    W = synth.make_weights(1, 16, 24, norm=synth.NORM_1DN)
    assert W["g_a.gdn0.gamma"].shape == (16,)
    C = O.Codec(1, 16, 24, W)
    x = synth.make_frames(1, 64, 64)
    bs, enc = O.encode(C, x)
    xr, dec = O.decode(C, bs)
    assert np.array_equal(dec[0]["s_y"], enc["s_y"][0])


def _tiny_student(seed=3, ch=(5, 4, 3, 4, 3)):
    r = np.random.default_rng(seed)
    P = {}
    for l in range(4):
        P[f"student.deconv{l}.weight"] = r.standard_normal((ch[l], ch[l + 1], 5, 5)) * 0.3
        P[f"student.deconv{l}.bias"] = r.standard_normal(ch[l + 1]) * 0.1
    return P


def test_student_gradients_match_finite_differences():
    """The oracle's backward pass (chain rule through 4 transposed convs and
    ReLUs, MSE) against central finite differences of the loss at sampled
    coordinates of every parameter tensor."""
    P = _tiny_student()
    r = np.random.default_rng(4)
    yhat = r.standard_normal((2, 5, 3, 4))
    target = r.standard_normal((2, 3, 48, 64))
    loss, grads = O.student_loss_grads(P, yhat, target)
    eps = 1e-6
    for name, gval in grads.items():
        for _ in range(4):
            idx = tuple(r.integers(0, s) for s in P[name].shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][idx] += eps
            Pm[name][idx] -= eps
            fd = (O.student_loss_grads(Pp, yhat, target)[0] - O.student_loss_grads(Pm, yhat, target)[0]) / (2 * eps)
            assert abs(fd - gval[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, gval[idx])


def test_deconv_wgrad_matches_torch_autograd():
    """Weight gradient of the transposed conv against torch's float64 autograd
    of conv_transpose2d (a library routine)."""
    r = np.random.default_rng(6)
    x = r.standard_normal((2, 4, 5, 6))
    g = r.standard_normal((2, 3, 10, 12))
    w = torch.zeros((4, 3, 5, 5), dtype=torch.float64, requires_grad=True)
    y = torch.nn.functional.conv_transpose2d(torch.from_numpy(x), w, stride=2, padding=2, output_padding=1)
    (y * torch.from_numpy(g)).sum().backward()
    np.testing.assert_allclose(O.deconv2d_wgrad(x, g), w.grad.numpy(), rtol=0, atol=1e-12)


def test_adam_constant_gradient_closed_form():
    """Adam with a constant gradient g has m_hat = g and v_hat = g^2 at every
    step (the bias corrections cancel the geometric sums exactly), so each
    step moves theta by -lr g / (|g| + eps); a zero gradient moves nothing."""
    r = np.random.default_rng(9)
    g = r.standard_normal(50) * 10.0 ** r.uniform(-4, 1, 50)
    g[:3] = 0.0
    P = {"w": r.standard_normal(50)}
    start = P["w"].copy()
    m = {"w": np.zeros(50)}
    v = {"w": np.zeros(50)}
    lr, eps = 1e-3, 1e-8
    for t in range(1, 6):
        O.adam_step(P, {"w": g}, m, v, t, lr=lr, eps=eps)
        want = start - t * lr * g / (np.abs(g) + eps)
        np.testing.assert_allclose(P["w"], want, rtol=0, atol=1e-12)
    assert np.array_equal(P["w"][:3], start[:3])


def test_student_training_decreases_loss():
    """A few oracle Adam steps on a fixed tiny batch lower the student's MSE
    (a consistency check of gradient sign and update direction together)."""
    P = _tiny_student(seed=11)
    r = np.random.default_rng(12)
    yhat = r.standard_normal((2, 5, 3, 4))
    target = r.standard_normal((2, 3, 48, 64)) * 0.1
    m = {k: np.zeros_like(v) for k, v in P.items()}
    v = {k: np.zeros_like(x) for k, x in P.items()}
    l0 = O.student_loss_grads(P, yhat, target)[0]
    for t in range(1, 21):
        loss, grads = O.student_loss_grads(P, yhat, target)
        O.adam_step(P, grads, m, v, t, lr=1e-2)
    assert O.student_loss_grads(P, yhat, target)[0] < 0.5 * l0


def test_student_loss_window_matches_finite_differences():
    """With a latent halo the output (80 x 80 here) is larger than the target
    (48 x 48): the loss covers the central square only, and its gradient --
    zero outside that square -- still matches central differences."""
    P = _tiny_student(seed=5)
    r = np.random.default_rng(6)
    yhat = r.standard_normal((2, 5, 5, 5))
    target = r.standard_normal((2, 3, 48, 48))
    loss, grads = O.student_loss_grads(P, yhat, target)
    _, out = O.student_forward(P, yhat)
    assert abs(loss - np.mean((out[:, :, 16:64, 16:64] - target) ** 2)) < 1e-12
    eps = 1e-6
    for name, gval in grads.items():
        for _ in range(3):
            idx = tuple(r.integers(0, s) for s in P[name].shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][idx] += eps
            Pm[name][idx] -= eps
            fd = (O.student_loss_grads(Pp, yhat, target)[0] - O.student_loss_grads(Pm, yhat, target)[0]) / (2 * eps)
            assert abs(fd - gval[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx)


# ------------------------------------------- rANS substream format 2 (escapes outside)

def test_rans2_hand_computed():
    g = json.load(open(os.path.join(GOLD, "rans2_hand.json")))
    for key in ("escape3", "resume33"):
        case = g[key]
        t = _tab(case["lo"], case["hi"], case["cdf"])
        sy = np.array(case["symbols"], np.int32)
        tab = np.zeros(len(sy), np.int32)
        words, recs = O.rans2_encode(sy, tab, [t], case["S"])
        assert words.tolist() == case["words"], key
        assert recs.tolist() == case["records"], key
        assert O.rans2_decode(words, len(sy), tab, [t]).tolist() == case["symbols"]
        for r, rec in enumerate(recs):
            G = case["S"] * (r + 1)
            got = O.rans2_decode(words, len(sy), tab, [t], rec, G, (len(sy) + 31) // 32)
            assert got[32 * G:].tolist() == case["symbols"][32 * G:]


def _v2_roundtrip(s, idx, tabs, S):
    n = len(s)
    w, recs = O.rans2_encode(s, idx, tabs, S)
    assert O.rans2_decode(w, n, idx, tabs).tolist() == s.tolist()
    ng = (n + 31) // 32
    bounds = [0] + [S * (r + 1) for r in range(len(recs))] + [ng]
    assert len(recs) == ((ng - 1) // S if S and ng else 0)
    for r in range(len(recs) + 1):
        part = O.rans2_decode(w, n, idx, tabs, None if r == 0 else recs[r - 1], bounds[r], bounds[r + 1])
        sl = slice(32 * bounds[r], 32 * bounds[r + 1])
        assert part[sl].tolist() == s[sl].tolist(), r
    return w


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1000])
@pytest.mark.parametrize("S", [0, 1, 3])
def test_rans2_roundtrip_and_resume_records(n, S):
    tabs = _random_tables()
    idx = rng.integers(0, 64, n).astype(np.int32)
    T = O.scale_table()
    s = np.rint(rng.standard_normal(n) * T[idx] * 1.3).astype(np.int32)
    s[::13] = rng.integers(-20000, 20000, len(s[::13]))
    _v2_roundtrip(s, idx, tabs, S)


def test_rans2_adversarial():
    tabs = _random_tables()
    n = 300
    idx = np.zeros(n, np.int32)
    s = np.array([(1 if i % 2 else -1) * (2 + (7 ** (i % 11))) for i in range(n)], np.int32)
    s[:4] = [2 ** 30, -(2 ** 30), 2, -2]
    _v2_roundtrip(s, idx, tabs, 2)
    t = tabs[63]
    s = np.array([-t.lo, t.hi] * 40, np.int32)
    _v2_roundtrip(s, np.full(len(s), 63, np.int32), tabs, 1)


def test_rans2_rans_words_equal_format1_without_escapes():
    """Format 2 changes only where escapes go: with none, its rANS section is
    format 1's stream word for word, and the substream is that plus nw."""
    tabs = _random_tables()
    n = 2000
    idx = rng.integers(0, 64, n).astype(np.int32)
    T = O.scale_table()
    s = np.clip(np.rint(rng.standard_normal(n) * T[idx]), -1, 1).astype(np.int32)
    w1 = O.rans_encode(s, idx, tabs)
    w2, _ = O.rans2_encode(s, idx, tabs)
    assert int(w2[0]) | (int(w2[1]) << 16) == len(w1)
    assert w2[2:].tolist() == w1.tolist()


def test_rans2_escape_bits_leave_the_word_stream():
    """With escapes, format 2's rANS section has exactly as many words as a
    format-1 stream of the same symbols with every escape payload removed
    (the escape symbol alone), and the payload and count sections hold
    4 bits per nibble: n_k + 1 nibbles per escape."""
    tabs = _random_tables()
    n = 640
    idx = np.full(n, 5, np.int32)
    t = tabs[5]
    s = rng.integers(-t.lo, t.hi + 1, n).astype(np.int32)
    esc = rng.random(n) < 0.2
    s[esc] = t.hi + 1 + rng.integers(0, 5000, int(esc.sum()))
    w2, _ = O.rans2_encode(s, idx, tabs)
    nw = int(w2[0]) | (int(w2[1]) << 16)
    s_plain = s.copy()
    s_plain[esc] = t.hi + 1          # payload v = 0: one nibble in format 1
    w1 = O.rans_encode(s_plain, idx, tabs)
    # format 1 puts two uniform nibbles per such escape in the words; format 2 none
    v = 2 * (s[esc] - t.hi - 1)
    nn = np.array([max(1, (int(x).bit_length() + 3) // 4) for x in v])
    assert len(w2) == 2 + nw + (nn.sum() + 3) // 4 + (int(esc.sum()) + 3) // 4
    assert nw <= len(w1)


def test_rans2_corrupt_is_detected():
    tabs = _random_tables()
    idx = np.full(200, 20, np.int32)
    s = rng.integers(-3, 4, 200).astype(np.int32)
    s[::7] = 9000
    w, _ = O.rans2_encode(s, idx, tabs)
    for bad in (w[:40], w[:-1], np.concatenate([w, [0]])):
        with pytest.raises(ValueError):
            O.rans2_decode(bad, 200, idx, tabs)
    w2 = w.copy()
    w2[-1] ^= 0x7          # count nibble 0 changed: the payload positions shift
    with pytest.raises(ValueError):
        O.rans2_decode(w2, 200, idx, tabs)


def test_rans2_code_length_bound():
    """As for format 1, per interleaved state (escape nibbles counted on
    their lane): bits <= 1.01 * sum(-log2 p) + 64."""
    tabs = _random_tables()
    T = O.scale_table()
    for k in (3, 30):
        n = 32 * 400
        idx = np.full(n, k, np.int32)
        s = np.rint(rng.standard_normal(n) * T[k] * 1.5).astype(np.int32)
        w, recs, lw, lb = O.rans2_encode(s, idx, tabs, with_stats=True)
        nw = int(w[0]) | (int(w[1]) << 16)
        assert nw == lw.sum() + 64
        bits = 16.0 * (lw + 2)
        extra = 16.0 * (len(w) - 2 - nw)     # the escape sections, all lanes
        assert bits.sum() + extra <= 1.01 * lb.sum() + 64 * 32 + 32


@pytest.mark.parametrize("kind", [0, 1])
def test_format2_container_chain_and_strip(kind):
    W = synth.make_weights(kind, 32, 64)
    x = synth.make_frames(1, 200, 330, first=4)
    oc1 = O.Codec(kind, 32, 64, W)
    bs1, inter = O.encode(oc1, x)
    for S in (0, 2):
        oc = O.Codec(kind, 32, 64, W, version=2, S=S)
        bs, inter2 = O.encode(oc, x)
        assert np.array_equal(inter2["s_y"], inter["s_y"])
        h = O.unpack_frame(bs[0])
        assert h["version"] == 2 and h["S"] == S and (len(h["trailer"]) > 0) == (S > 0)
        xr, di = O.decode(oc, bs)
        assert np.array_equal(di[0]["s_y"], inter["s_y"][0])
        st = O.strip_records(bs[0])
        assert O.unpack_frame(st)["S"] == 0 and len(st) <= len(bs[0])
        xr2, di2 = O.decode(oc, [st])
        assert np.array_equal(xr2, xr)
        if S == 0:
            assert st == bs[0]
