"""CUDA path vs the FP64 oracle, through the C ABI (marked gpu).

Rules (the paper states no numerics; these are the project's readings):
* float stages (g_a, h_a, h_s, g_s), fed identical float32 inputs: max-abs
  difference <= 1e-4 against the FP64 oracle;
* integer stages fed the GPU's own float32 values (quantized symbols, scale
  indices, bitstream bytes): identical, no tolerance;
* end to end from the frame: a symbol or index may differ from the FP64
  chain only where the oracle's value lies within 1e-4 * max(1, |v|) of a
  rounding boundary (k + 1/2) or of a scale-table entry;
* encoder and decoder scale indices: identical, always.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
N, M = 128, 192


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def weights():
    return {k: synth.make_weights(k, N, M) for k in (0, 1)}


@pytest.fixture(scope="module")
def codecs(weights):
    out = {}
    for impl in (lic.CONV_AUTO, lic.CONV_SIMT):
        for k in (0, 1):
            out[(k, impl)] = lic.Codec(k, N, M, weights[k], conv_impl=impl)
    return out


@pytest.fixture(scope="module")
def ocodecs(weights):
    return {k: O.Codec(k, N, M, weights[k]) for k in (0, 1)}


def pad(x):
    H, W = x.shape[2:]
    Hp, Wp = O.pad_size(H, W)
    return np.pad(x, ((0, 0), (0, 0), (0, Hp - H), (0, Wp - W)), mode="edge")


IMPLS = [lic.CONV_AUTO, lic.CONV_SIMT]


# ------------------------------------------------------------ float stages

@pytest.mark.parametrize("impl", IMPLS)
def test_analysis_matches_oracle(codecs, weights, impl):
    x = synth.make_frames(2, 100, 150)            # pads to 128 x 192: ragged
    c = codecs[(1, impl)]
    y = torch.empty(2, M, 8, 12, device="cuda")
    c.analysis(dev(x), y)
    torch.cuda.synchronize()
    ref = O.g_a(weights[1], pad(x))
    err = np.abs(y.cpu().numpy() - ref).max()
    assert err <= TOL, err


# 24 x 40 latents: 384 x 640 outputs, many tiles a CTA and long K walks (the
# tensor-core accumulator's truncation drift shows there first)
@pytest.mark.parametrize("impl", IMPLS)
@pytest.mark.parametrize("hw", [(6, 9), (24, 40)])
def test_synthesis_matches_oracle(codecs, weights, impl, hw):
    rng = np.random.default_rng(3)
    h, w = hw
    yhat = np.rint(rng.standard_normal((2, M, h, w)) * 2).astype(np.float32)
    c = codecs[(0, impl)]
    x = torch.empty(2, 3, 16 * h, 16 * w, device="cuda")
    c.synthesis(dev(yhat), x)
    torch.cuda.synchronize()
    ref = O.g_s(weights[0], yhat)
    err = np.abs(x.cpu().numpy() - ref).max()
    assert err <= TOL, err


@pytest.mark.parametrize("impl", IMPLS)
def test_hyper_transforms_match_oracle(codecs, weights, impl):
    rng = np.random.default_rng(4)
    y = (rng.standard_normal((2, M, 12, 20)) * 1.5).astype(np.float32)
    c = codecs[(1, impl)]
    z = torch.empty(2, N, 3, 5, device="cuda")
    c.hyper_analysis(dev(y), z)
    torch.cuda.synchronize()
    ref = O.h_a(weights[1], y)
    assert np.abs(z.cpu().numpy() - ref).max() <= TOL
    zhat = np.rint(ref).astype(np.float32)
    sig = torch.empty(2, M, 12, 20, device="cuda")
    idx = torch.empty(2, M, 12, 20, dtype=torch.uint8, device="cuda")
    c.hyper_synthesis(dev(zhat), sig, idx)
    torch.cuda.synchronize()
    sref = O.h_s(weights[1], zhat)
    s_gpu = sig.cpu().numpy()
    assert np.abs(s_gpu - sref).max() <= TOL
    # stage-wise strict: the index of the GPU's own scales
    assert np.array_equal(idx.cpu().numpy(), O.scale_index(s_gpu))


def test_batch_does_not_change_a_frames_arithmetic(codecs):
    """A frame coded in a batch of three and coded alone gives the same
    bitstream and the same reconstruction, bit for bit.  At N = 128 the
    hyper transforms' small grids are cut into K slices whose count depends
    on the layer and the frame size only; this pins that."""
    c = codecs[(1, lic.CONV_AUTO)]
    x = synth.make_frames(3, 128, 192, first=60)
    bs = c.encode(dev(x))
    out3 = torch.empty(3, 3, 128, 192, device="cuda")
    c.decode(bs, out3)
    assert c.sync_status() == lic.OK
    b3 = bs.to_bytes()
    for i in range(3):
        bi = c.encode(dev(x[i:i + 1]))
        out1 = torch.empty(1, 3, 128, 192, device="cuda")
        c.decode(bi, out1)
        assert c.sync_status() == lic.OK
        assert bi.to_bytes()[0] == b3[i], i
        assert torch.equal(out1[0], out3[i]), i


# --------------------------------------------------- integer stages, strict

def encode_and_read(c, x):
    bs = c.encode(dev(x))
    c.sync()
    B, _, H, W = x.shape
    Hp, Wp = O.pad_size(H, W)
    Hy, Wy = Hp // 16, Wp // 16
    out = dict(bytes=bs.to_bytes())
    y = np.zeros((B, M, Hy, Wy), np.float32)
    sy = np.zeros((B, M, Hy, Wy), np.int32)
    c.read_tensor(lic.T_Y, y)
    c.read_tensor(lic.T_SY, sy)
    out.update(y=y, s_y=sy)
    if c.kind == 1:
        z = np.zeros((B, N, Hy // 4, Wy // 4), np.float32)
        sz = np.zeros((B, N, Hy // 4, Wy // 4), np.int32)
        sg = np.zeros((B, M, Hy, Wy), np.float32)
        idx = np.zeros((B, M, Hy, Wy), np.uint8)
        c.read_tensor(lic.T_Z, z)
        c.read_tensor(lic.T_SZ, sz)
        c.read_tensor(lic.T_SIGMA, sg)
        c.read_tensor(lic.T_IDX, idx)
        out.update(z=z, s_z=sz, sigma=sg, idx=idx)
    return bs, out


@pytest.mark.parametrize("kind", [0, 1])
def test_symbols_indices_and_bitstreams_bit_exact(codecs, ocodecs, kind):
    x = synth.make_frames(2, 100, 150, first=5)
    c, oc = codecs[(kind, lic.CONV_AUTO)], ocodecs[kind]
    bs, g = encode_and_read(c, x)
    mu = oc.med if kind == 0 else None
    assert np.array_equal(g["s_y"], O.quantize(g["y"], mu))
    if kind == 1:
        assert np.array_equal(g["s_z"], O.quantize(g["z"], oc.med))
        assert np.array_equal(g["idx"], O.scale_index(g["sigma"]))
    Hp, Wp = O.pad_size(100, 150)
    for b in range(2):
        subs = O.encode_latents(oc, g["s_y"][b], g.get("idx", [None] * 2)[b], g.get("s_z", [None] * 2)[b])
        ref = O.pack_frame(kind, N, M, 100, 150, Hp, Wp, oc.R, subs)
        assert g["bytes"][b] == ref, f"frame {b} bitstream differs"


@pytest.mark.parametrize("kind", [0, 1])
def test_roundtrip_lossless_and_decoder_matches_oracle(codecs, ocodecs, weights, kind):
    x = synth.make_frames(2, 70, 130, first=9)
    c, oc = codecs[(kind, lic.CONV_AUTO)], ocodecs[kind]
    bs, g = encode_and_read(c, x)
    out = torch.empty(2, 3, 70, 130, device="cuda")
    c.decode(bs, out)
    assert c.sync_status() == lic.OK
    sy = np.zeros_like(g["s_y"])
    c.read_tensor(lic.T_SY, sy)
    assert np.array_equal(sy, g["s_y"])
    if kind == 1:
        idx = np.zeros_like(g["idx"])
        c.read_tensor(lic.T_IDX, idx)
        assert np.array_equal(idx, g["idx"]), "encoder and decoder indices differ"
    # the oracle decodes the GPU's bytes to the same symbols and a frame within 1e-4
    ref, inter = O.decode(oc, g["bytes"])
    for b in range(2):
        assert np.array_equal(inter[b]["s_y"], g["s_y"][b])
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL
    # host-resident input bitstreams and host output frames
    host_out = np.zeros((2, 3, 70, 130), np.float32)
    c.decode(lic.host_bitstreams(g["bytes"]), host_out)
    assert c.sync_status() == lic.OK
    assert np.array_equal(host_out, out.cpu().numpy())


def near_boundary(v, mu=None):
    d = v if mu is None else v - mu
    frac = d - np.floor(d)
    return np.abs(frac - 0.5) <= TOL * np.maximum(1.0, np.abs(d))


def test_end_to_end_from_frame(codecs, ocodecs):
    x = synth.make_frames(2, 128, 192, first=20)
    c, oc = codecs[(1, lic.CONV_AUTO)], ocodecs[1]
    _, g = encode_and_read(c, x)
    _, inter = O.encode(oc, x)
    bad = g["s_y"] != inter["s_y"]
    assert np.all(near_boundary(inter["y"][bad])), int(bad.sum())
    badz = g["s_z"] != inter["s_z"]
    muz = np.broadcast_to(oc.med[None, :, None, None], inter["z"].shape)
    assert np.all(near_boundary(inter["z"][badz], muz[badz])), int(badz.sum())
    if not badz.any():
        T = O.scale_table().astype(np.float64)
        badi = g["idx"] != inter["idx"]
        sg = inter["sigma"][badi]
        near = np.min(np.abs(sg[:, None] - T[None, :]), axis=1) <= TOL * np.maximum(1.0, sg)
        assert np.all(near), int(badi.sum())


# ------------------------------------------------------- entropy edge cases

def test_entropy_adversarial_factorized(codecs, ocodecs):
    """Escapes of every payload length, many escapes in one group of 32,
    the f = 1 ends of each table's support, ragged bands: GPU bytes equal
    the oracle's and the GPU decoder returns the symbols."""
    c, oc = codecs[(0, lic.CONV_AUTO)], ocodecs[0]
    rng = np.random.default_rng(11)
    B, Hy, Wy = 2, 20, 12        # 20 rows: a full band of 16 and a ragged band of 4
    sy = rng.integers(-3, 4, (B, M, Hy, Wy)).astype(np.int32)
    sy[0, 0] = 2 ** 30
    sy[0, 1] = -(2 ** 30)
    sy[0, 2] = rng.integers(-(2 ** 20), 2 ** 20, (Hy, Wy))
    sy[1, 5, :, ::2] = 7 ** np.arange(Wy // 2)[None, :] + 300
    for ch in range(6, 12):
        t = oc.eb[ch]
        sy[1, ch, ::2] = -t.lo
        sy[1, ch, 1::2] = t.hi
    bs = c.encode_latents(dev(sy), None, None, 320, 192)
    got = bs.to_bytes()
    for b in range(B):
        subs = O.encode_latents(oc, sy[b])
        assert got[b] == O.pack_frame(0, N, M, 320, 192, 16 * Hy, 16 * Wy, oc.R, subs)
    out_y = torch.empty(B, M, Hy, Wy, dtype=torch.int32, device="cuda")
    c.decode_latents(bs, out_y)
    assert c.sync_status() == lic.OK
    assert np.array_equal(out_y.cpu().numpy(), sy)


def test_entropy_adversarial_hyperprior(codecs, ocodecs):
    """z symbols far outside the bottleneck's support (escapes), y symbols
    coded with the indices h_s gives for those z (as any encoder must), with
    escapes forced into y: bytes equal the oracle's; the decoder returns
    both planes exactly."""
    c, oc = codecs[(1, lic.CONV_AUTO)], ocodecs[1]
    rng = np.random.default_rng(12)
    B, Hy, Wy = 2, 20, 12
    sz = rng.integers(-400, 400, (B, N, Hy // 4, Wy // 4)).astype(np.int32)
    zhat = O.dequantize(sz, oc.med)
    sig = torch.empty(B, M, Hy, Wy, device="cuda")
    idx = torch.empty(B, M, Hy, Wy, dtype=torch.uint8, device="cuda")
    c.hyper_synthesis(dev(zhat), sig, idx)
    torch.cuda.synchronize()
    idx_np = idx.cpu().numpy()
    sy = rng.integers(-3, 4, (B, M, Hy, Wy)).astype(np.int32)
    sy[0, 3] = 5000
    sy[1, 7, :, 1::2] = -123456
    bs = c.encode_latents(dev(sy), idx, dev(sz), 320, 192)
    got = bs.to_bytes()
    for b in range(B):
        subs = O.encode_latents(oc, sy[b], idx_np[b], sz[b])
        assert got[b] == O.pack_frame(1, N, M, 320, 192, 16 * Hy, 16 * Wy, oc.R, subs)
    out_y = torch.empty(B, M, Hy, Wy, dtype=torch.int32, device="cuda")
    out_z = torch.empty(B, N, Hy // 4, Wy // 4, dtype=torch.int32, device="cuda")
    c.decode_latents(bs, out_y, out_z)
    assert c.sync_status() == lic.OK
    assert np.array_equal(out_z.cpu().numpy(), sz)
    assert np.array_equal(out_y.cpu().numpy(), sy)


def test_corrupt_and_truncated_streams_are_reported(codecs):
    c = codecs[(1, lic.CONV_AUTO)]
    x = synth.make_frames(1, 64, 64, first=30)
    bs = c.encode(dev(x))
    good = bs.to_bytes()[0]
    out = torch.empty(1, 3, 64, 64, device="cuda")
    # truncated payload
    c.decode(lic.host_bitstreams([good[: len(good) // 2]]), out)
    assert c.sync_status() == lic.E_CORRUPT_STREAM
    # wrong magic: with the frame size given, the device's header check latches it ...
    c.decode(lic.host_bitstreams([b"XXXX" + good[4:]], 64, 64), out)
    assert c.sync_status() == lic.E_CORRUPT_STREAM
    # ... and with the size to be read from that header, the call refuses it at once
    assert c.decode_status(lic.host_bitstreams([b"XXXX" + good[4:]]), out) == lic.E_CORRUPT_STREAM
    assert c.sync_status() == lic.OK
    # offset table pointing past the payload
    bad = bytearray(good)
    bad[36 + 4:36 + 8] = (0xFFFFFF).to_bytes(4, "little")
    c.decode(lic.host_bitstreams([bytes(bad)]), out)
    assert c.sync_status() == lic.E_CORRUPT_STREAM
    # random payload bytes: decoding ends (either way) and the context stays usable
    rng = np.random.default_rng(0)
    noisy = bytearray(good)
    hdr = 36 + 4 * (N + M * 1 + 1)
    noisy[hdr:] = rng.integers(0, 256, len(good) - hdr, dtype=np.uint8).tobytes()
    c.decode(lic.host_bitstreams([bytes(noisy)]), out)
    assert c.sync_status() in (lic.OK, lic.E_CORRUPT_STREAM)
    c.decode(lic.host_bitstreams([good]), out)
    assert c.sync_status() == lic.OK


# ------------------------------------------- full size, sampled with the oracle

def test_full_size_720p_batch8_sampled(codecs, ocodecs, weights):
    """The bench workload (8 x 1280x720, padded to 1280x768): properties at
    full size, plus sampled y and x_hat values computed by the oracle on
    crops whose receptive fields lie inside the crop."""
    B, H, W = 8, 720, 1280
    x = synth.make_frames(B, H, W)
    c, oc = codecs[(1, lic.CONV_AUTO)], ocodecs[1]
    xd = dev(x)
    bs = c.encode(xd)
    out = torch.empty(B, 3, H, W, device="cuda")
    c.decode(bs, out)
    assert c.sync_status() == lic.OK
    Hy, Wy = 48, 80
    y = np.zeros((B, M, Hy, Wy), np.float32)
    xpre = np.zeros((B, 3, 768, 1280), np.float32)
    sy = np.zeros((B, M, Hy, Wy), np.int32)
    c.read_tensor(lic.T_SY, sy)
    c.read_tensor(lic.T_XPRE, xpre)
    # encoder side again for y / idx (the decode overwrote the shared buffers)
    bs = c.encode(xd)
    g_bytes = bs.to_bytes()
    c.read_tensor(lic.T_Y, y)
    sy_enc = np.zeros_like(sy)
    c.read_tensor(lic.T_SY, sy_enc)
    assert np.array_equal(sy, sy_enc), "decoded symbols differ from encoded"
    xp = pad(x)
    # sampled y: a 192 x 192 crop at a 16-aligned offset; y inside the crop
    # whose 61-pixel receptive field (plus the zero-padding fringe) is inside
    for (b, oy, ox) in [(0, 256, 512), (5, 320, 960), (7, 0, 0)]:
        crop = xp[b:b + 1, :, oy:oy + 192, ox:ox + 192]
        ry = O.g_a(weights[1], crop)[0]
        i0 = 0 if oy == 0 else 4
        j0 = 0 if ox == 0 else 4
        sl = (slice(None), slice(i0, 8), slice(j0, 8))
        gy = y[b, :, oy // 16:oy // 16 + 12, ox // 16:ox // 16 + 12]
        assert np.abs(gy[sl] - ry[sl]).max() <= TOL
    # sampled x_hat: the oracle's g_s on a 12 x 12 window of the decoded
    # symbols; interior outputs are exact
    yhat = sy.astype(np.float32)
    for (b, iy, ix) in [(1, 20, 30), (6, 36, 68)]:
        win = yhat[b:b + 1, :, iy:iy + 12, ix:ix + 12]
        rx = O.g_s(weights[1], win)[0]
        gx = xpre[b, :, 16 * iy:16 * iy + 192, 16 * ix:16 * ix + 192]
        assert np.abs(gx[:, 64:128, 64:128] - rx[:, 64:128, 64:128]).max() <= TOL
    # the entropy coder at full size: bytes equal the oracle's coding of the
    # GPU's symbols for two frames
    idx = np.zeros((B, M, Hy, Wy), np.uint8)
    sz = np.zeros((B, N, Hy // 4, Wy // 4), np.int32)
    c.read_tensor(lic.T_IDX, idx)
    c.read_tensor(lic.T_SZ, sz)
    for b in (0, 7):
        subs = O.encode_latents(oc, sy_enc[b], idx[b], sz[b])
        assert g_bytes[b] == O.pack_frame(1, N, M, H, W, 768, 1280, oc.R, subs)


def test_degenerate_inputs(codecs, ocodecs):
    """An empty batch is refused before any device work; the smallest and the
    thinnest frames (almost all replicate padding, a 64 x 64 or 64 x 1280 padded
    grid with one 4 x 4 latent row) code losslessly, and the decoder's output
    equals the oracle's decoding of the GPU's own bytes."""
    c, oc = codecs[(1, lic.CONV_AUTO)], ocodecs[1]
    with pytest.raises(lic.LicError) as e:
        c.encode(torch.empty(0, 3, 64, 64, device="cuda"))
    assert e.value.code == lic.E_INVALID_ARG
    for (H, Wd) in [(1, 1), (1, 1280), (65, 3)]:
        x = synth.make_frames(1, H, Wd, first=40)
        bs = c.encode(dev(x))
        out = torch.empty(1, 3, H, Wd, device="cuda")
        c.decode(bs, out)
        assert c.sync_status() == lic.OK
        got = bs.to_bytes()
        assert lic.decoded_shape(got[0])[1:] == (H, Wd)
        ref, _ = O.decode(oc, got)
        assert np.abs(out.cpu().numpy() - ref).max() <= TOL, (H, Wd)
        bs.release()


def test_4k_frame_sampled(codecs, ocodecs, weights):
    """The largest frame size exercised: one 3840x2160 frame (padded to
    3840x2176; latent grid 136 x 240): lossless symbols, encoder and decoder
    indices identical, sampled y and x_hat against the oracle as at 720p, and
    the entropy coder's bytes equal the oracle's coding of the GPU's symbols."""
    B, H, Wd = 1, 2160, 3840
    Hp, Wp = O.pad_size(H, Wd)
    Hy, Wy = Hp // 16, Wp // 16
    c, oc = codecs[(1, lic.CONV_AUTO)], ocodecs[1]
    x = synth.make_frames(B, H, Wd, first=50)
    bs = c.encode(dev(x))
    y = np.zeros((B, M, Hy, Wy), np.float32)
    sy_enc = np.zeros((B, M, Hy, Wy), np.int32)
    idx_enc = np.zeros((B, M, Hy, Wy), np.uint8)
    sz = np.zeros((B, N, Hy // 4, Wy // 4), np.int32)
    c.read_tensor(lic.T_Y, y)
    c.read_tensor(lic.T_SY, sy_enc)
    c.read_tensor(lic.T_IDX, idx_enc)
    c.read_tensor(lic.T_SZ, sz)
    got = bs.to_bytes()
    out = torch.empty(B, 3, H, Wd, device="cuda")
    c.decode(bs, out)
    assert c.sync_status() == lic.OK
    sy = np.zeros_like(sy_enc)
    idx = np.zeros_like(idx_enc)
    xpre = np.zeros((B, 3, Hp, Wp), np.float32)
    c.read_tensor(lic.T_SY, sy)
    c.read_tensor(lic.T_IDX, idx)
    c.read_tensor(lic.T_XPRE, xpre)
    assert np.array_equal(sy, sy_enc) and np.array_equal(idx, idx_enc)
    xp = pad(x)
    for (oy, ox) in [(1984, 3648), (1024, 2048)]:   # the bottom-right corner's padding, an interior
        ry = O.g_a(weights[1], xp[:, :, oy:oy + 192, ox:ox + 192])[0]
        gy = y[0, :, oy // 16:oy // 16 + 12, ox // 16:ox // 16 + 12]
        i1 = 12 if oy + 192 == Hp else 8
        j1 = 12 if ox + 192 == Wp else 8
        assert np.abs(gy[:, 4:i1, 4:j1] - ry[:, 4:i1, 4:j1]).max() <= TOL
    for (iy, ix) in [(120, 220), (60, 100)]:
        rx = O.g_s(weights[1], sy[:, :, iy:iy + 12, ix:ix + 12].astype(np.float32))[0]
        gx = xpre[0, :, 16 * iy:16 * iy + 192, 16 * ix:16 * ix + 192]
        assert np.abs(gx[:, 64:128, 64:128] - rx[:, 64:128, 64:128]).max() <= TOL
    subs = O.encode_latents(oc, sy_enc[0], idx_enc[0], sz[0])
    assert got[0] == O.pack_frame(1, N, M, H, Wd, Hp, Wp, oc.R, subs)
