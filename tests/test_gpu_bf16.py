"""The BF16 precision form (lic_options.precision = LIC_BF16) against the
FP64 oracle (marked gpu).  g_a / g_s convolutions run on bf16 operands with
float32 accumulation; GDN norms, h_a, h_s and the scale index stay float32.
Its bar: the entropy stages stay lossless, encoder and decoder derive
identical scale indices, and the reconstruction is within 40 dB PSNR of the
FP64 chain's; the latent error against FP64 is reported."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu
N, M = 128, 192


@pytest.fixture(scope="module")
def setup():
    out = {}
    for kind in (0, 1):
        W = synth.make_weights(kind, N, M)
        out[kind] = (W, lic.Codec(kind, N, M, W, precision=lic.BF16), O.Codec(kind, N, M, W))
    return out


@pytest.mark.parametrize("kind", [1, 0])
def test_bf16_form_against_fp64(setup, kind, capsys):
    W, c, oc = setup[kind]
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
    c.decode(bs, H, Wd, out)
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
        print(f"\n[bf16 form kind={kind}] PSNR vs FP64 chain {p:.2f} dB, max|y - y64| {yerr:.4f}, "
              f"symbols differing {100 * flips:.3f}%")
    assert p >= 40.0, p
    assert yerr < 0.1, yerr
