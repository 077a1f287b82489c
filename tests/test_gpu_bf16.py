"""The precision forms (lic_options.precision = LIC_BF16 / LIC_FP8) against
the FP64 oracle (marked gpu).  g_a / g_s convolutions run on bf16 (or e4m3
with per-output-channel weight scales) operands with float32 accumulation;
GDN norms, h_a, h_s and the scale index stay float32.  Both must keep the
entropy stages lossless and encoder / decoder scale indices identical; BF16
must reconstruct within 40 dB PSNR of the FP64 chain; FP8's PSNR and latent
error are reported (and held to a loose floor)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu
N, M = 128, 192


FLOOR = {lic.BF16: (40.0, 0.1), lic.FP8: (25.0, 1.0)}
NAME = {lic.BF16: "bf16", lic.FP8: "fp8"}


@pytest.fixture(scope="module")
def setup():
    out = {}
    for kind in (0, 1):
        W = synth.make_weights(kind, N, M)
        oc = O.Codec(kind, N, M, W)
        for prec in (lic.BF16, lic.FP8):
            out[(kind, prec)] = (W, lic.Codec(kind, N, M, W, precision=prec), oc)
    return out


@pytest.mark.parametrize("prec", [lic.BF16, lic.FP8])
@pytest.mark.parametrize("kind", [1, 0])
def test_precision_form_against_fp64(setup, kind, prec, capsys):
    W, c, oc = setup[(kind, prec)]
    B, H, Wd = 2, 200, 330
    x = synth.make_frames(B, H, Wd, first=60)
    bs = c.encode(torch.from_numpy(x).cuda())
    out = torch.empty(B, 3, H, Wd, device="cuda")
    c.sync()
    Hy, Wy = 16, 24
    sy = np.zeros((B, M, Hy, Wy), np.int32)
    y = np.zeros((B, M, Hy, Wy), np.float32)
    c.read_tensor(lic.T_SY, sy)
    c.read_tensor(lic.T_Y, y)
    if kind == 1:
        idx_enc = np.zeros((B, M, Hy, Wy), np.uint8)
        c.read_tensor(lic.T_IDX, idx_enc)
    c.decode(bs, out)
    assert c.sync_status() == lic.OK
    sy_dec = np.zeros_like(sy)
    c.read_tensor(lic.T_SY, sy_dec)
    assert np.array_equal(sy_dec, sy), "entropy coding must stay lossless"
    if kind == 1:
        idx_dec = np.zeros_like(idx_enc)
        c.read_tensor(lic.T_IDX, idx_dec)
        assert np.array_equal(idx_dec, idx_enc), "encoder and decoder indices differ"
    ref_bs, inter = O.encode(oc, x)
    ref, _ = O.decode(oc, ref_bs)
    p = O.psnr(out.cpu().numpy(), ref)
    yerr = float(np.abs(y - inter["y"]).max())
    flips = float(np.mean(sy != inter["s_y"]))
    with capsys.disabled():
        print(f"\n[{NAME[prec]} form kind={kind}] PSNR vs FP64 chain {p:.2f} dB, max|y - y64| {yerr:.4f}, "
              f"symbols differing {100 * flips:.3f}%")
    min_psnr, max_yerr = FLOOR[prec]
    assert p >= min_psnr, p
    assert yerr < max_yerr, yerr


@pytest.mark.parametrize("prec", [lic.BF16, lic.FP8])
def test_precision_form_full_size_720p_sampled(setup, prec, capsys):
    """The precision forms at the bench's size (2 x 1280x720, padded to 1280x768),
    where every persistent layer walks many tiles a CTA: lossless entropy stages,
    encoder and decoder indices identical, sampled y within the form's floor of the
    oracle's g_a on a crop, and x_hat on windows of the decoded symbols within the
    form's PSNR floor of the oracle's g_s."""
    W, c, oc = setup[(1, prec)]
    B, H, Wd = 2, 720, 1280
    x = synth.make_frames(B, H, Wd, first=90)
    bs = c.encode(torch.from_numpy(x).cuda())
    c.sync()
    Hy, Wy = 48, 80
    y = np.zeros((B, M, Hy, Wy), np.float32)
    sy = np.zeros((B, M, Hy, Wy), np.int32)
    idx_enc = np.zeros((B, M, Hy, Wy), np.uint8)
    c.read_tensor(lic.T_Y, y)
    c.read_tensor(lic.T_SY, sy)
    c.read_tensor(lic.T_IDX, idx_enc)
    out = torch.empty(B, 3, H, Wd, device="cuda")
    c.decode(bs, out)
    assert c.sync_status() == lic.OK
    sy_dec = np.zeros_like(sy)
    idx_dec = np.zeros_like(idx_enc)
    xpre = np.zeros((B, 3, 768, 1280), np.float32)
    c.read_tensor(lic.T_SY, sy_dec)
    c.read_tensor(lic.T_IDX, idx_dec)
    c.read_tensor(lic.T_XPRE, xpre)
    assert np.array_equal(sy_dec, sy), "entropy coding must stay lossless"
    assert np.array_equal(idx_dec, idx_enc), "encoder and decoder indices differ"
    min_psnr, max_yerr = FLOOR[prec]
    xp = np.pad(x, ((0, 0), (0, 0), (0, 48), (0, 0)), mode="edge")
    yerr = 0.0
    for (b, oy, ox) in [(0, 256, 512), (1, 576, 1024)]:
        ry = O.g_a(W, xp[b:b + 1, :, oy:oy + 192, ox:ox + 192])[0]
        gy = y[b, :, oy // 16:oy // 16 + 12, ox // 16:ox // 16 + 12]
        yerr = max(yerr, float(np.abs(gy[:, 4:8, 4:8] - ry[:, 4:8, 4:8]).max()))
    ps = []
    for (b, iy, ix) in [(0, 20, 30), (1, 34, 60)]:
        rx = O.g_s(W, sy_dec[b:b + 1, :, iy:iy + 12, ix:ix + 12].astype(np.float32))[0]
        gx = xpre[b, :, 16 * iy:16 * iy + 192, 16 * ix:16 * ix + 192]
        ps.append(O.psnr(gx[:, 64:128, 64:128], rx[:, 64:128, 64:128]))
    with capsys.disabled():
        print(f"\n[{NAME[prec]} form, 2 x 720p] window PSNR vs FP64 g_s {min(ps):.2f} dB, "
              f"max|y - y64| on crops {yerr:.4f}")
    assert min(ps) >= min_psnr, ps
    assert yerr < max_yerr, yerr
