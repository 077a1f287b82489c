"""Substream format 2 -- escape payloads outside the rANS words, optional
resume records (the decoder-adaptive coder) -- through the C ABI, marked gpu.

Integer stages are held to the bit-exact bar: containers equal the oracle's
on adversarial symbols (escapes of every payload length, f = 1 table ends,
ragged bands, whole planes), with and without resume records; the decoder
returns the symbols whether it follows the records (one warp per segment),
ignores them (another spacing) or is given the stream with its records
stripped.  Format 2 codes the same symbols as format 1, so a frame's
reconstruction is identical in both.  Corrupt streams are reported, never
fault."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu
N, M = 128, 192
TOL = 1e-4


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def weights():
    return {k: synth.make_weights(k, N, M) for k in (0, 1)}


def adversarial(kind, oc, c, B, Hy, Wy, seed):
    """Symbols with escapes of 1..8 nibbles, table ends, and (hyperprior)
    the indices h_s gives for escape-heavy z."""
    rng = np.random.default_rng(seed)
    sy = rng.integers(-3, 4, (B, M, Hy, Wy)).astype(np.int32)
    sy[0, 0] = 2 ** 30
    sy[0, 1] = -(2 ** 30)
    sy[0, 2] = rng.integers(-(2 ** 20), 2 ** 20, (Hy, Wy))
    sy[-1, 5, :, ::2] = (7 ** (np.arange(Wy // 2) % 11))[None, :] + 300
    sy[-1, 9] = np.where(rng.random((Hy, Wy)) < 0.8, 5000, 0)
    if kind == 0:
        for ch in range(12, 16):
            t = oc.eb[ch]
            sy[-1, ch, ::2] = -t.lo
            sy[-1, ch, 1::2] = t.hi
        return sy, None, None
    sz = rng.integers(-400, 400, (B, N, Hy // 4, Wy // 4)).astype(np.int32)
    sig = torch.empty(B, M, Hy, Wy, device="cuda")
    idx = torch.empty(B, M, Hy, Wy, dtype=torch.uint8, device="cuda")
    c.hyper_synthesis(dev(O.dequantize(sz, oc.med)), sig, idx)
    torch.cuda.synchronize()
    return sy, idx.cpu().numpy(), sz


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("R,S", [(16, 0), (16, 1), (1000, 0), (1000, 4)])
def test_format2_bytes_equal_oracle_and_decode(weights, kind, R, S):
    W = weights[kind]
    c = lic.Codec(kind, N, M, W, band_rows=R, format=lic.FORMAT_2, resume_groups=S)
    oc = O.Codec(kind, N, M, W, R=R, version=2, S=S)
    B, Hy, Wy = 2, 20, 12          # R = 16: a full band and a ragged band of 4 rows
    sy, idx, sz = adversarial(kind, oc, c, B, Hy, Wy, 21 + kind)
    H, Wd = 16 * Hy - 5, 16 * Wy - 7
    bs = c.encode_latents(dev(sy), dev(idx) if idx is not None else None, dev(sz) if sz is not None else None, H, Wd)
    got = bs.to_bytes()
    for b in range(B):
        if kind == 1:
            enc = O.encode_latents(oc, sy[b], idx[b], sz[b])
        else:
            enc = O.encode_latents(oc, sy[b])
        ref = O.pack_frame(kind, N, M, H, Wd, 16 * Hy, 16 * Wy, R, enc[0], 2, S, enc[1])
        assert got[b] == ref, f"frame {b}: containers differ from the oracle's"
    out_y = torch.empty(B, M, Hy, Wy, dtype=torch.int32, device="cuda")
    out_z = torch.empty(B, N, Hy // 4, Wy // 4, dtype=torch.int32, device="cuda")
    c.decode_latents(bs, out_y, out_z if kind == 1 else None)
    assert c.sync_status() == lic.OK
    assert np.array_equal(out_y.cpu().numpy(), sy)
    if kind == 1:
        assert np.array_equal(out_z.cpu().numpy(), sz)
    if S:
        # the same stream with its records stripped, and the stream as it is given to a
        # decoder set up with another spacing: both decode every substream from its start
        stripped = [lic.strip_resume_records(f) for f in got]
        assert all(len(s) < len(f) for s, f in zip(stripped, got))
        assert stripped == [O.strip_records(f) for f in got]
        other = lic.Codec(kind, N, M, W, band_rows=R, format=lic.FORMAT_2, resume_groups=S + 1)
        for codec, frames in ((c, stripped), (other, got)):
            out_y.zero_()
            codec.decode_latents(lic.host_bitstreams(frames), out_y, out_z if kind == 1 else None)
            assert codec.sync_status() == lic.OK
            assert np.array_equal(out_y.cpu().numpy(), sy)
        other.close()
    c.close()


def test_format2_chain_equals_format1_and_oracle(weights):
    """Whole frames through both formats: the same symbols, so the same
    reconstruction bit for bit; the format-2 bytes decode in the oracle to
    the GPU decoder's symbols, and its g_s of them is within 1e-4."""
    W = weights[1]
    x = dev(synth.make_frames(2, 520, 200, first=17))     # 36 latent rows: 3 bands in format 1
    c1 = lic.Codec(1, N, M, W)
    c2 = lic.Codec(1, N, M, W, band_rows=1000, format=lic.FORMAT_2, resume_groups=2)
    o1, o2 = torch.empty_like(x), torch.empty_like(x)
    b1 = c1.encode(x)
    c1.decode(b1, o1)
    b2 = c2.encode(x)
    c2.decode(b2, o2)
    assert c1.sync_status() == lic.OK and c2.sync_status() == lic.OK
    assert torch.equal(o1, o2)
    # the integer stages exact: the oracle's containers of the GPU decoder's own
    # symbols and indices are the GPU's bytes; the float stage: the oracle's g_s of
    # those symbols within 1e-4 of the GPU's frames
    oc = O.Codec(1, N, M, W, R=1000, version=2, S=2)
    sy = np.zeros((2, M, 36, 16), np.int32)
    idx = np.zeros((2, M, 36, 16), np.uint8)
    sz = np.zeros((2, N, 9, 4), np.int32)
    c2.read_tensor(lic.T_SY, sy)
    c2.read_tensor(lic.T_IDX, idx)
    c2.read_tensor(lic.T_SZ, sz)
    got = b2.to_bytes()
    for b in range(2):
        subs, recs = O.encode_latents(oc, sy[b], idx[b], sz[b])
        assert got[b] == O.pack_frame(1, N, M, 520, 200, 576, 256, 1000, subs, 2, 2, recs)
    ref = np.clip(O.g_s(W, sy.astype(np.float32)), 0.0, 1.0)[:, :, :520, :200]
    err = float(np.abs(o2.cpu().numpy() - ref).max())
    assert err <= TOL, err
    # whole planes code fewer bytes than 16-row bands (one 32-state flush per plane, not three)
    s1, s2 = sum(b1.sizes()), sum(lic.strip_resume_records(f).__len__() for f in b2.to_bytes())
    assert s2 < s1
    c1.close()
    c2.close()


def test_format2_corrupt_streams_are_reported(weights):
    W = weights[1]
    c = lic.Codec(1, N, M, W, band_rows=1000, format=lic.FORMAT_2, resume_groups=1)
    x = dev(synth.make_frames(1, 128, 192, first=33))
    good = c.encode(x).to_bytes()[0]
    out = torch.empty(1, 3, 128, 192, device="cuda")
    cases = {"truncated": good[: len(good) // 2], "one byte short": good[:-1]}
    bad = bytearray(good)
    base = 36 + 4 * (N + M + 1)
    bad[base + 2 * 300] ^= 0xFF                       # a rANS or nibble word of a z substream
    cases["payload"] = bytes(bad)
    bad = bytearray(good)
    bad[len(good) - 140 + 8 + 4] ^= 0x55              # a lane state in the last resume record
    cases["record"] = bytes(bad)
    for name, blob in cases.items():
        st = c.decode_status(lic.host_bitstreams([blob], 128, 192), out)
        code = c.sync_status()
        assert st in (lic.OK, lic.E_CORRUPT_STREAM) and code in (lic.OK, lic.E_CORRUPT_STREAM), name
        if name != "payload":   # a flipped word may still decode to valid symbols
            assert lic.E_CORRUPT_STREAM in (st, code), name
    c.decode(lic.host_bitstreams([good]), out)
    assert c.sync_status() == lic.OK
    c.close()
