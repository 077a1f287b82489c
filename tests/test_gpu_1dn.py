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
