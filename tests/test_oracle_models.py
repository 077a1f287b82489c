"""Pins of the oracle's entropy-bottleneck likelihoods and of its composed
transforms -- the two parts that the primitive pins (conv brute force, GDN
identities, logit closed forms) do not reach by themselves.  CPU only.

Entropy bottleneck (Balle et al. 2018, appendix 6.1; the hyperprior paper is
the cited [2]): the table a channel codes with is built from the unit-bin
likelihoods c(m+s+1/2) - c(m+s-1/2) of the cumulative c = sigmoid(logit)
around the median m, plus one escape symbol holding both tails.  Here the
logit has a closed form (affine for a linear net, a scalar recursion when
every hidden unit of a layer is equal), which the test evaluates in 60-digit
arithmetic; median, tails, every likelihood and the escape mass must agree.
A likelihood taken without the sign flip loses ~1e-6 of its relative
accuracy in the upper tail, a swapped tail changes the escape mass, and a
bin off by one changes every entry: each fails here.

Composed transforms (g_a, g_s of [1]; h_a, h_s of [2]; the chain of the
paper's Sec. III-A/B and Fig. 1): each is recomposed from torch float64
library convolutions with GDN written as an einsum, from the layer lists of
the two codec configurations, and compared on small tensors; invariants
(h_a even in y, h_s non-negative) and planted mistakes show the comparison
is sensitive to the errors it is meant to catch."""
import math

import mpmath as mp
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O
from paper_2208_01641_b300 import synth

mp.mp.dps = 60
TAU = 1e-9   # tail mass of the entropy bottleneck's support


# ------------------------------------------------------------- entropy bottleneck

def _eb_params(s_vals, b=0.0, a=0.0):
    """One channel whose softplus(H_k) entries all equal s_vals[k], biases b, a."""
    W = {}
    f = synth.EB_FILTERS
    for k in range(5):
        W[f"eb.H{k}"] = np.full((1, f[k + 1], f[k]), math.log(math.expm1(s_vals[k])))
        W[f"eb.b{k}"] = np.full((1, f[k + 1]), b)
        if k < 4:
            W[f"eb.a{k}"] = np.full((1, f[k + 1]), a)
    return W


def _logit_equal_units(s_vals, b, a):
    """Closed form of the logit when every unit of a layer is equal: the
    1-3-3-3-3-1 net reduces to h <- w_k h + b (+ tanh(a) tanh(.) for k < 4),
    w_0 = s_0 and w_k = 3 s_k (three equal inputs) after.  mpmath, exact to
    60 digits for float inputs."""
    S = [mp.log1p(mp.expm1(mp.mpf(v))) for v in s_vals]   # softplus(log(expm1 s)) = s
    ta = mp.tanh(mp.mpf(a))

    def logit(x):
        h = mp.mpf(x)
        for k in range(5):
            h = (S[k] if k == 0 else 3 * S[k]) * h + b
            if k < 4:
                h = h + ta * mp.tanh(h)
        return h
    return logit


def _root(fn, target):
    """Solve fn(x) = target for a monotone increasing fn by bisection, 60 digits."""
    lo, hi = mp.mpf(-1e6), mp.mpf(1e6)
    for _ in range(260):
        mid = (lo + hi) / 2
        if fn(mid) < target:
            lo = mid
        else:
            hi = mid
    return hi


def _sig(x):
    return 1 / (1 + mp.exp(-x))


def _expected_table(logit):
    """Median (float32), lo, hi and the likelihoods + escape of C7, in mpmath."""
    m = np.float32(float(_root(logit, 0)))
    md = mp.mpf(float(m))
    tq = mp.log((mp.mpf(TAU) / 2) / (1 - mp.mpf(TAU) / 2))
    qlo, qhi = _root(logit, tq), _root(logit, -tq)
    lo = max(0, int(mp.ceil(md - qlo)))
    hi = max(0, int(mp.ceil(qhi - md)))
    pm = [_sig(logit(md + s + mp.mpf(0.5))) - _sig(logit(md + s - mp.mpf(0.5)))
          for s in range(-lo, hi + 1)]
    esc = _sig(logit(md - lo - mp.mpf(0.5))) + 1 - _sig(logit(md + hi + mp.mpf(0.5)))
    return m, lo, hi, pm + [esc]


def _check_pmf(W, logit, rel):
    m, lo, hi, pm = O.eb_pmf(W, 0)
    em, elo, ehi, epm = _expected_table(logit)
    assert m == em, (m, em)
    assert (lo, hi) == (elo, ehi)
    assert len(pm) == len(epm) == lo + hi + 2
    err = max(abs(mp.mpf(float(p)) - q) / q for p, q in zip(pm, epm))
    assert err < rel, f"worst relative likelihood error {float(err):.3g}"
    return lo, hi, pm, epm


def test_eb_pmf_linear_net_closed_form():
    """a = b = 0: logit(x) = k x with k = 3^4 prod s_k, median 0, symmetric
    support; each likelihood sigmoid(k(s+1/2)) - sigmoid(k(s-1/2)) and the
    escape 2 sigmoid(-k(hi+1/2)), to 1e-15 absolute and 1e-11 relative."""
    s = [0.5, 0.3, 0.4, 0.45, 0.35]
    k = 81 * np.prod(s)
    W = _eb_params(s)
    lo, hi, pm, epm = _check_pmf(W, lambda x: mp.mpf(k) * x, 1e-11)
    assert lo == hi
    assert max(abs(float(p) - float(q)) for p, q in zip(pm, epm)) < 1e-15
    assert abs(float(pm[-1]) - float(2 * _sig(-mp.mpf(k) * (hi + mp.mpf(0.5))))) < 1e-20


def test_eb_pmf_nonlinear_asymmetric_channel():
    """b, a != 0 makes the cumulative nonlinear and its tails unequal
    (lo != hi), so a swapped tail or a flip on the wrong side shows."""
    s, b, a = [0.45, 0.35, 0.4, 0.3, 0.5], 0.7, 0.8
    W = _eb_params(s, b=b, a=a)
    lo, hi, pm, epm = _check_pmf(W, _logit_equal_units(s, b, a), 1e-10)
    assert lo != hi
    # tiny upper-tail bins are where the sign flip matters: they are matched
    # to 1e-10 relative above; the naive difference would be ~1e-6 off
    assert min(float(q) for q in epm[:-1]) < 1e-9
    assert abs(sum(float(p) for p in pm) - 1.0) < 1e-13
    # the same differences taken without the flip, in double, from the
    # oracle's own logits: the tolerance above would reject them
    m = float(O.eb_pmf(W, 0)[0])
    naive = [1 / (1 + math.exp(-O.eb_logits(W, 0, m + k + 0.5))) - 1 / (1 + math.exp(-O.eb_logits(W, 0, m + k - 0.5)))
             for k in range(-lo, hi + 1)]
    assert max(abs(mp.mpf(v) - q) / q for v, q in zip(naive, epm)) > 1e-8


def test_eb_pmf_seeded_channel_sums_and_quantizes():
    """On a seeded codec channel: the likelihoods and escape sum to 1, every
    entry lies in (0, 1), and the channel's table is their frequency
    quantization (the table builder adds nothing after the likelihoods)."""
    Wt = synth.make_weights(synth.KIND_HYPERPRIOR, 8, 12)
    med, tabs = O.eb_tables(Wt)
    for c in (0, 5):
        m, lo, hi, pm = O.eb_pmf(Wt, c)
        assert m == med[c] and (lo, hi) == (tabs[c].lo, tabs[c].hi)
        assert abs(pm.sum() - 1.0) < 1e-12 and np.all(pm > 0) and np.all(pm < 1)
        assert np.array_equal(O.quantize_pmf(pm), tabs[c].cdf)


# ------------------------------------------------------------- composed transforms

def _t(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64))


def _gdn_t(x, beta, gamma, inverse=False):
    """y_i = x_i / sqrt(beta_i + sum_j gamma_ij x_j^2) (x_i * sqrt(.) inverse)."""
    n = _t(beta)[None, :, None, None] + torch.einsum("ij,bjhw->bihw", _t(gamma), x * x)
    return x * torch.sqrt(n) if inverse else x / torch.sqrt(n)


def torch_g_a(W, x):
    """conv5x5/2 3->N, GDN, conv5x5/2, GDN, conv5x5/2, GDN, conv5x5/2 N->M."""
    h = _t(x)
    for i in range(4):
        h = F.conv2d(h, _t(W[f"g_a.conv{i}.weight"]), _t(W[f"g_a.conv{i}.bias"]), stride=2, padding=2)
        if i < 3:
            h = _gdn_t(h, W[f"g_a.gdn{i}.beta"], W[f"g_a.gdn{i}.gamma"])
    return h.numpy()


def torch_g_s(W, y):
    """deconv5x5/2 M->N, IGDN, deconv, IGDN, deconv, IGDN, deconv N->3."""
    h = _t(y)
    for i in range(4):
        h = F.conv_transpose2d(h, _t(W[f"g_s.deconv{i}.weight"]), _t(W[f"g_s.deconv{i}.bias"]),
                               stride=2, padding=2, output_padding=1)
        if i < 3:
            h = _gdn_t(h, W[f"g_s.igdn{i}.beta"], W[f"g_s.igdn{i}.gamma"], inverse=True)
    return h.numpy()


def torch_h_a(W, y):
    """On |y|: conv3x3/1 M->N, ReLU, conv5x5/2, ReLU, conv5x5/2."""
    h = torch.abs(_t(y))
    h = F.relu(F.conv2d(h, _t(W["h_a.conv0.weight"]), _t(W["h_a.conv0.bias"]), stride=1, padding=1))
    h = F.relu(F.conv2d(h, _t(W["h_a.conv1.weight"]), _t(W["h_a.conv1.bias"]), stride=2, padding=2))
    return F.conv2d(h, _t(W["h_a.conv2.weight"]), _t(W["h_a.conv2.bias"]), stride=2, padding=2).numpy()


def torch_h_s(W, z):
    """deconv5x5/2, ReLU, deconv5x5/2, ReLU, conv3x3/1 N->M, ReLU."""
    h = _t(z)
    for i in range(2):
        h = F.relu(F.conv_transpose2d(h, _t(W[f"h_s.deconv{i}.weight"]), _t(W[f"h_s.deconv{i}.bias"]),
                                      stride=2, padding=2, output_padding=1))
    return F.relu(F.conv2d(h, _t(W["h_s.conv2.weight"]), _t(W["h_s.conv2.bias"]), stride=1, padding=1)).numpy()


N, M = 8, 12


@pytest.fixture(scope="module")
def weights():
    return synth.make_weights(synth.KIND_HYPERPRIOR, N, M)


@pytest.fixture(scope="module")
def frame():
    return synth.make_frames(2, 64, 128, first=11).astype(np.float64)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


def test_g_a_and_g_s_match_torch_composition(weights, frame):
    y = O.g_a(weights, frame)
    assert y.shape == (2, M, 4, 8)
    assert _rel(y, torch_g_a(weights, frame)) < 1e-12
    x = O.g_s(weights, y)
    assert x.shape == frame.shape
    assert _rel(x, torch_g_s(weights, y)) < 1e-12


def test_h_a_and_h_s_match_torch_composition(weights):
    r = np.random.default_rng(5)
    y = 3.0 * r.standard_normal((2, M, 16, 12))
    z = O.h_a(weights, y)
    assert z.shape == (2, N, 4, 3)
    assert _rel(z, torch_h_a(weights, y)) < 1e-12
    zin = 3.0 * r.standard_normal((2, N, 4, 3))
    sig = O.h_s(weights, zin)
    assert sig.shape == (2, M, 16, 12)
    assert _rel(sig, torch_h_s(weights, zin)) < 1e-12


def test_hyper_transform_invariants(weights):
    """h_a reads |y|: h_a(y) = h_a(-y) exactly.  h_s ends in a ReLU: the
    scales are >= 0, and on these inputs some pre-activations are negative,
    so the final ReLU is exercised (exact zeros appear)."""
    r = np.random.default_rng(6)
    y = 3.0 * r.standard_normal((1, M, 8, 8))
    assert np.array_equal(O.h_a(weights, y), O.h_a(weights, -y))
    sig = O.h_s(weights, 3.0 * r.standard_normal((1, N, 2, 2)))
    assert sig.min() >= 0.0 and np.count_nonzero(sig == 0.0) > 0


def test_planted_mistakes_are_caught(weights, frame, monkeypatch):
    """Each planted mistake in the oracle (on the CPU) moves the composed
    transform far beyond the 1e-12 of the comparisons above."""
    y = O.g_a(weights, frame)
    ref_ga, ref_gs = torch_g_a(weights, frame), torch_g_s(weights, y)
    real_gdn, real_relu = O.gdn, O.relu
    # a transposed gamma in every GDN / IGDN
    monkeypatch.setattr(O, "gdn", lambda x, b, g, inverse=False: real_gdn(x, b, np.ascontiguousarray(g.T), inverse))
    assert _rel(O.g_a(weights, frame), ref_ga) > 1e-6
    assert _rel(O.g_s(weights, y), ref_gs) > 1e-6
    monkeypatch.setattr(O, "gdn", real_gdn)
    # a dropped ReLU (h_s's final one included)
    r = np.random.default_rng(7)
    zin = 3.0 * r.standard_normal((1, N, 2, 2))
    ref_hs = torch_h_s(weights, zin)
    monkeypatch.setattr(O, "relu", lambda x: np.asarray(x, dtype=np.float64))
    assert _rel(O.h_s(weights, zin), ref_hs) > 1e-3
    monkeypatch.setattr(O, "relu", real_relu)
    # GDN after the last analysis conv (its parameters borrowed from GDN 2)
    real_conv = O.conv2d
    calls = []

    def conv_then_extra_gdn(x, w, b, stride):
        out = real_conv(x, w, b, stride)
        calls.append(1)
        if len(calls) == 4:
            return real_gdn(out, np.ones(M), 0.1 * np.eye(M), False)
        return out
    monkeypatch.setattr(O, "conv2d", conv_then_extra_gdn)
    assert _rel(O.g_a(weights, frame), ref_ga) > 1e-6


@pytest.mark.parametrize("kind", [synth.KIND_FACTORIZED, synth.KIND_HYPERPRIOR])
def test_chain_order_matches_torch_composition(kind):
    """The oracle's encoder and decoder, stage by stage, against the torch
    compositions and the paper's order (Sec. III-A/B): y = g_a(x);
    hyperprior: z = h_a(y), s_z = rint(z - median), z_hat = s_z + median,
    sigma = h_s(z_hat) (from z_hat, not z), idx = index(sigma), s_y = rint(y);
    factorized: s_y = rint(y - median); decoder x_hat = clamp(g_s(y_hat))."""
    Wt = synth.make_weights(kind, N, M)
    codec = O.Codec(kind, N, M, Wt)
    x = synth.make_frames(1, 64, 64, first=21)
    streams, inter = O.encode(codec, x)
    y = torch_g_a(Wt, x.astype(np.float64))
    assert _rel(inter["y"], y) < 1e-12
    y32 = inter["y"].astype(np.float32)
    if kind == synth.KIND_HYPERPRIOR:
        z = torch_h_a(Wt, inter["y"])
        assert _rel(inter["z"], z) < 1e-12
        med = codec.med[None, :, None, None]
        s_z = np.rint(inter["z"].astype(np.float32) - med).astype(np.int32)
        assert np.array_equal(inter["s_z"], s_z)
        zhat = (s_z + med).astype(np.float32)
        assert np.array_equal(inter["zhat"], zhat)
        sig = torch_h_s(Wt, zhat)
        assert _rel(inter["sigma"], sig) < 1e-12
        T = O.scale_table()
        s32 = np.maximum(inter["sigma"].astype(np.float32), T[0])
        idx = np.array([min(np.searchsorted(T, v, side="left"), 63) for v in s32.ravel()])
        assert np.array_equal(inter["idx"].ravel(), idx)
        assert np.array_equal(inter["s_y"], np.rint(y32).astype(np.int32))
        yhat = inter["s_y"].astype(np.float32)
    else:
        med = codec.med[None, :, None, None]
        assert np.array_equal(inter["s_y"], np.rint(y32 - med).astype(np.int32))
        yhat = (inter["s_y"] + med).astype(np.float32)
    xr, dinter = O.decode(codec, streams)
    assert np.array_equal(dinter[0]["s_y"], inter["s_y"][0])
    ref = np.clip(torch_g_s(Wt, yhat), 0.0, 1.0)[:, :, :64, :64]
    assert _rel(xr, ref) < 1e-12
