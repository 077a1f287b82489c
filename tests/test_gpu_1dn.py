"""1DN (the paper's variant C activation, read as GDN without channel
mixing) through the C ABI against the FP64 oracle (marked gpu): the same
float bar (max-abs 1e-4 on identical float32 inputs) and integer bar
(symbols, indices and bitstream bytes identical) as GDN."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu
N, M = 128, 192
TOL = 1e-4


def pad(x):
    H, W = x.shape[2:]
    Hp, Wp = O.pad_size(H, W)
    return np.pad(x, ((0, 0), (0, 0), (0, Hp - H), (0, Wp - W)), mode="edge")


@pytest.fixture(scope="module")
def W1():
    return synth.make_weights(1, N, M, norm=synth.NORM_1DN)


@pytest.mark.parametrize("impl", [lic.CONV_AUTO, lic.CONV_SIMT])
def test_1dn_transforms_match_oracle(W1, impl):
    c = lic.Codec(1, N, M, W1, conv_impl=impl, norm=lic.NORM_1DN)
    x = synth.make_frames(2, 100, 150, first=70)
    y = torch.empty(2, M, 8, 12, device="cuda")
    c.analysis(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    assert np.abs(y.cpu().numpy() - O.g_a(W1, pad(x))).max() <= TOL
    yhat = np.rint(np.random.default_rng(5).standard_normal((2, M, 6, 9)) * 2).astype(np.float32)
    xr = torch.empty(2, 3, 96, 144, device="cuda")
    c.synthesis(torch.from_numpy(yhat).cuda(), xr)
    torch.cuda.synchronize()
    assert np.abs(xr.cpu().numpy() - O.g_s(W1, yhat)).max() <= TOL
    c.close()


def test_1dn_codec_bitstreams_and_roundtrip(W1):
    c = lic.Codec(1, N, M, W1, norm=lic.NORM_1DN)
    oc = O.Codec(1, N, M, W1)
    x = synth.make_frames(2, 100, 150, first=75)
    bs = c.encode(torch.from_numpy(x).cuda())
    got = bs.to_bytes()
    sy = np.zeros((2, M, 8, 12), np.int32)
    y = np.zeros((2, M, 8, 12), np.float32)
    z = np.zeros((2, N, 2, 3), np.float32)
    sz = np.zeros((2, N, 2, 3), np.int32)
    sg = np.zeros((2, M, 8, 12), np.float32)
    idx = np.zeros((2, M, 8, 12), np.uint8)
    for t, a in ((lic.T_SY, sy), (lic.T_Y, y), (lic.T_Z, z), (lic.T_SZ, sz), (lic.T_SIGMA, sg), (lic.T_IDX, idx)):
        c.read_tensor(t, a)
    assert np.array_equal(sy, O.quantize(y))
    assert np.array_equal(sz, O.quantize(z, oc.med))
    assert np.array_equal(idx, O.scale_index(sg))
    for b in range(2):
        subs = O.encode_latents(oc, sy[b], idx[b], sz[b])
        assert got[b] == O.pack_frame(1, N, M, 100, 150, 128, 192, oc.R, subs)
    out = torch.empty(2, 3, 100, 150, device="cuda")
    c.decode(bs, out)
    assert c.sync_status() == lic.OK
    ref, inter = O.decode(oc, got)
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL
    c.close()


def test_1dn_full_size_720p_sampled(W1):
    """1DN at the bench's size (2 x 1280x720, padded to 1280x768): g_a conv0's tap
    form and every persistent layer walk many tiles a CTA here.  Sampled y against
    the oracle's g_a on a crop whose receptive field lies inside it, sampled x_hat
    against the oracle's g_s on a window of the decoded symbols, encoder and
    decoder indices identical, and the decoded symbols equal the encoded ones."""
    B, H, Wd = 2, 720, 1280
    c = lic.Codec(1, N, M, W1, norm=lic.NORM_1DN)
    x = synth.make_frames(B, H, Wd, first=80)
    xd = torch.from_numpy(x).cuda()
    Hy, Wy = 48, 80
    bs = c.encode(xd)
    y = np.zeros((B, M, Hy, Wy), np.float32)
    sy_enc = np.zeros((B, M, Hy, Wy), np.int32)
    idx_enc = np.zeros((B, M, Hy, Wy), np.uint8)
    c.read_tensor(lic.T_Y, y)
    c.read_tensor(lic.T_SY, sy_enc)
    c.read_tensor(lic.T_IDX, idx_enc)
    out = torch.empty(B, 3, H, Wd, device="cuda")
    c.decode(bs, out)
    assert c.sync_status() == lic.OK
    sy = np.zeros_like(sy_enc)
    idx = np.zeros_like(idx_enc)
    xpre = np.zeros((B, 3, 768, 1280), np.float32)
    c.read_tensor(lic.T_SY, sy)
    c.read_tensor(lic.T_IDX, idx)
    c.read_tensor(lic.T_XPRE, xpre)
    assert np.array_equal(sy, sy_enc)
    assert np.array_equal(idx, idx_enc)
    xp = pad(x)
    for (b, oy, ox) in [(0, 320, 704), (1, 576, 1088)]:
        ry = O.g_a(W1, xp[b:b + 1, :, oy:oy + 192, ox:ox + 192])[0]
        gy = y[b, :, oy // 16:oy // 16 + 12, ox // 16:ox // 16 + 12]
        assert np.abs(gy[:, 4:8, 4:8] - ry[:, 4:8, 4:8]).max() <= TOL
    yhat = sy.astype(np.float32)
    for (b, iy, ix) in [(0, 10, 40), (1, 30, 60)]:
        rx = O.g_s(W1, yhat[b:b + 1, :, iy:iy + 12, ix:ix + 12])[0]
        gx = xpre[b, :, 16 * iy:16 * iy + 192, 16 * ix:16 * ix + 192]
        assert np.abs(gx[:, 64:128, 64:128] - rx[:, 64:128, 64:128]).max() <= TOL
    c.close()
