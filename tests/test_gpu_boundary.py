"""The C ABI's ownership rules (include/lic.h), marked gpu.

An encoded batch is library-owned and stays valid until it is released,
whatever is encoded meanwhile: two batches encoded back to back decode
correctly afterwards, and their bytes equal the oracle's container of the
same symbols (the integer stages' bit-exact bar).  Released buffers are
pooled and reused (no new device memory), releasing twice is refused, at
most 64 batches may be live, the frame size of a batch can be read from its
first header, and the workspace estimate that serving admission relies on
equals what encode + decode actually allocate."""
import ctypes

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
def W():
    return synth.make_weights(lic.HYPERPRIOR, N, M)


def oracle_containers(c, oc, B, H, Wd):
    """The oracle's containers of the symbols the GPU decoder just produced."""
    Hy, Wy = (H + 63) // 64 * 4, (Wd + 63) // 64 * 4
    sy = np.zeros((B, M, Hy, Wy), np.int32)
    idx = np.zeros((B, M, Hy, Wy), np.uint8)
    sz = np.zeros((B, N, Hy // 4, Wy // 4), np.int32)
    c.read_tensor(lic.T_SY, sy)
    c.read_tensor(lic.T_IDX, idx)
    c.read_tensor(lic.T_SZ, sz)
    Hp, Wp = O.pad_size(H, Wd)
    return [O.pack_frame(1, N, M, H, Wd, Hp, Wp, oc.R, O.encode_latents(oc, sy[b], idx[b], sz[b]))
            for b in range(B)]


def test_two_live_batches_decode_afterwards_and_match_the_oracle(W):
    c = lic.Codec(lic.HYPERPRIOR, N, M, W)
    oc = O.Codec(lic.HYPERPRIOR, N, M, W)
    xa = synth.make_frames(2, 64, 96, first=5)
    xb = synth.make_frames(3, 128, 64, first=9)
    a = c.encode(dev(xa))
    b = c.encode(dev(xb))           # a stays valid: its buffers are its own
    assert a.s.owner and b.s.owner and a.s.owner != b.s.owner
    assert a.shape == (64, 96) and b.shape == (128, 64)
    for bs, x in ((a, xa), (b, xb)):
        B, _, H, Wd = x.shape
        out = torch.empty(B, 3, H, Wd, device="cuda")
        c.decode(bs, out)
        assert c.sync_status() == lic.OK
        got = bs.to_bytes()
        assert got == oracle_containers(c, oc, B, H, Wd)
        ref, inter = O.decode(oc, got)
        err = float(np.abs(out.cpu().numpy() - ref).max())
        assert err <= TOL, err
    c.close()


def test_release_pools_buffers_and_guards_misuse(W):
    c = lic.Codec(lic.HYPERPRIOR, N, M, W)
    x = dev(synth.make_frames(1, 64, 64, first=2))
    a = c.encode(x)
    ref = a.to_bytes()
    held = c.device_bytes()
    stale = lic._Bitstreams.from_buffer_copy(a.s)
    a.release()
    assert not a.s.owner and a.s.count == 0
    # a second release of the same batch is refused; a cleared struct is a no-op
    assert lic.lib().lic_bitstreams_release(c.h, ctypes.byref(stale)) == lic.E_INVALID_ARG
    assert lic.lib().lic_bitstreams_release(c.h, ctypes.byref(a.s)) == lic.OK
    b = c.encode(x)                 # reuses the released buffers
    assert c.device_bytes() == held
    assert b.to_bytes() == ref
    # the frame size read from frame 0's header (device batch, H = W = 0)
    view = lic._Bitstreams.from_buffer_copy(b.s)
    view.H = view.W = 0
    out1 = torch.empty(1, 3, 64, 64, device="cuda")
    out2 = torch.empty(1, 3, 64, 64, device="cuda")
    c.decode(b, out1)
    c.decode(view, out2)
    assert c.sync_status() == lic.OK and torch.equal(out1, out2)
    # at most 64 batches live at once
    live = [b] + [c.encode(x) for _ in range(63)]
    with pytest.raises(lic.LicError) as e:
        c.encode(x)
    assert e.value.code == lic.E_BUSY
    live[5].release()
    live[5] = c.encode(x)
    assert live[5].to_bytes() == ref
    for bs in live:
        bs.release()
    c.close()


def test_workspace_estimate_equals_what_encode_and_decode_allocate(W):
    c = lic.Codec(lic.HYPERPRIOR, N, M, W)
    before = c.device_bytes()
    est = c.workspace_bytes(2, 200, 330)
    x = dev(synth.make_frames(2, 200, 330, first=12))
    out = torch.empty_like(x)
    bs = c.encode(x)
    c.decode(bs, out)
    assert c.sync_status() == lic.OK
    assert c.device_bytes() - before == est
    c.close()


def test_mma_rate_probe_orders_the_types():
    """The tensor-pipe probe: dense rates are positive, and per MMA the
    narrower types do more work in the same time (tf32 < bf16 < e4m3)."""
    r = [lic.mma_rate(k, 4000) for k in range(3)]
    assert all(x > 50.0 for x in r), r
    assert r[0] < r[1] < r[2], r
    with pytest.raises(lic.LicError):
        lic.mma_rate(3)


def test_graph_replay_matches_direct_launches(W):
    """The calls are stream-ordered and allocate nothing once a batch size has
    been seen, so an encode and a decode captured as CUDA graphs replay the
    same kernels on the same inputs: bitstreams and frames bit-identical to
    direct launches (how the benchmark times its step), and the bytes equal
    the oracle's coding of the symbols."""
    B, H, Wd = 2, 128, 192
    c = lic.Codec(lic.HYPERPRIOR, N, M, W)
    oc = O.Codec(lic.HYPERPRIOR, N, M, W)
    x = dev(synth.make_frames(B, H, Wd, first=30))
    out_d = torch.empty(B, 3, H, Wd, device="cuda")
    out_g = torch.empty_like(out_d)
    s = torch.cuda.Stream()
    sid = s.cuda_stream
    with torch.cuda.stream(s):
        for _ in range(2):   # warm-up: every buffer sized
            bs = c.encode(x, stream=sid)
            c.decode(bs, out_d, stream=sid)
            bs.release()
        bs = c.encode(x, stream=sid)
        c.decode(bs, out_d, stream=sid)
    assert c.sync_status(sid) == lic.OK
    direct = bs.to_bytes()
    bs.release()
    ge, gd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(ge, stream=s):
        gb = c.encode(x, stream=sid)
    with torch.cuda.graph(gd, stream=s):
        c.decode(gb, out_g, stream=sid)
    with torch.cuda.stream(s):
        for _ in range(3):
            out_g.zero_()
            ge.replay()
            gd.replay()
    torch.cuda.synchronize()
    assert c.sync_status(sid) == lic.OK
    assert gb.to_bytes() == direct
    assert torch.equal(out_g, out_d)
    assert gb.to_bytes() == oracle_containers(c, oc, B, H, Wd)
    gb.release()
    c.close()
