"""lic_encode_latents_noalloc: the entropy encoder for callers that cannot
allocate device memory while they encode (a streaming thread that must not
stall in cudaMalloc/cudaFree, a host whose allocator owns all device memory,
a plugin handed its buffers).  Its containers must equal, byte for byte,
those of lic_encode_latents on the same symbols -- the bit-exact bar of the
integer stages -- on two calls in a row through the one shared working
array, and an oversized batch must be refused before anything runs.

Kept in a file of its own, collected last."""
import numpy as np
import pytest
import torch

import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu

N, M = 128, 192


def frame_cap(kind, Hy, Wy, R=16):
    nb = (Hy + R - 1) // R
    nz = N if kind == 1 else 0
    nsub = nz + M * nb
    nmax = min(R, Hy) * Wy
    if kind == 1:
        nmax = max(nmax, (Hy // 4) * (Wy // 4))
    cap_words = 10 * nmax + 64
    return 36 + 4 * (nsub + 1) + 2 * nsub * cap_words + 16


def containers(data, layout, B):
    lay = layout.cpu().numpy()
    raw = data.cpu().numpy()
    return [raw[lay[b]:lay[b] + lay[B + 1 + b]].tobytes() for b in range(B)]


@pytest.mark.parametrize("kind", [1, 0])
def test_noalloc_matches_encode_latents_twice(kind):
    Wt = synth.make_weights(kind, N, M)
    codec = lic.Codec(kind, N, M, Wt)
    B, H, W = 2, 200, 330                    # pads to 256 x 384
    Hy, Wy = 16, 24
    for call, first in enumerate((40, 50)):  # two calls in a row, different frames
        x = torch.from_numpy(synth.make_frames(B, H, W, first=first)).cuda()
        codec.encode(x)
        codec.sync()
        sy = torch.empty(B, M, Hy, Wy, dtype=torch.int32, device="cuda")
        codec.read_tensor(lic.T_SY, sy)
        idx = sz = None
        if kind == 1:
            idx = torch.empty(B, M, Hy, Wy, dtype=torch.uint8, device="cuda")
            sz = torch.empty(B, N, Hy // 4, Wy // 4, dtype=torch.int32, device="cuda")
            codec.read_tensor(lic.T_IDX, idx)
            codec.read_tensor(lic.T_SZ, sz)
        ref = codec.encode_latents(sy, idx, sz, H, W).to_bytes()
        data = torch.full((B * frame_cap(kind, Hy, Wy),), 0xAB, dtype=torch.uint8, device="cuda")
        layout = torch.full((2 * B + 1,), -1, dtype=torch.int64, device="cuda")
        rc = codec.encode_latents_noalloc(sy, idx, sz, H, W, data, layout)
        assert rc == lic.OK, (call, rc)
        assert codec.sync_status() == lic.OK
        got = containers(data, layout, B)
        assert got == ref, f"call {call}: containers differ from lic_encode_latents"
    codec.close()


def test_noalloc_refuses_oversized_and_short_buffers():
    Wt = synth.make_weights(1, N, M)
    codec = lic.Codec(1, N, M, Wt)
    B, Hy, Wy = 8, 48, 80                    # 8 x 720p: needs ~145 MB of working memory
    sy = torch.zeros(B, M, Hy, Wy, dtype=torch.int32, device="cuda")
    idx = torch.zeros(B, M, Hy, Wy, dtype=torch.uint8, device="cuda")
    sz = torch.zeros(B, N, Hy // 4, Wy // 4, dtype=torch.int32, device="cuda")
    data = torch.zeros(16, dtype=torch.uint8, device="cuda")
    layout = torch.zeros(2 * B + 1, dtype=torch.int64, device="cuda")
    assert codec.encode_latents_noalloc(sy, idx, sz, 720, 1280, data, layout) == lic.E_UNSUPPORTED
    # a batch that fits the working array but not the caller's output buffer
    sy1, idx1, sz1 = sy[:1].contiguous(), idx[:1].contiguous(), sz[:1].contiguous()
    assert codec.encode_latents_noalloc(sy1, idx1, sz1, 720, 1280, data, layout[:3].contiguous()) \
        == lic.E_INVALID_ARG
    assert codec.sync_status() == lic.OK
    codec.close()


def test_noalloc_refuses_host_and_misaligned_buffers():
    """Pointers the kernels could not use are refused before any launch: a
    host output buffer, a container buffer not 16-byte aligned, an offset
    table not 8-byte aligned, and host symbols."""
    Wt = synth.make_weights(1, N, M)
    codec = lic.Codec(1, N, M, Wt)
    B, H, W, Hy, Wy = 1, 64, 64, 4, 4
    sy = torch.zeros(B, M, Hy, Wy, dtype=torch.int32, device="cuda")
    idx = torch.zeros(B, M, Hy, Wy, dtype=torch.uint8, device="cuda")
    sz = torch.zeros(B, N, 1, 1, dtype=torch.int32, device="cuda")
    cap = B * frame_cap(1, Hy, Wy)
    data = torch.zeros(cap + 64, dtype=torch.uint8, device="cuda")
    layout = torch.zeros(2 * B + 2, dtype=torch.int64, device="cuda")
    L = lic.lib()

    def call(sy_p, data_p, cap_, lay_p):
        return L.lic_encode_latents_noalloc(codec.h, sy_p, idx.data_ptr(), sz.data_ptr(), B, H, W, Hy, Wy,
                                            data_p, cap_, lay_p, torch.cuda.current_stream().cuda_stream)

    host_data = np.zeros(cap + 64, np.uint8)
    host_sy = np.zeros(B * M * Hy * Wy, np.int32)
    assert call(sy.data_ptr(), host_data.ctypes.data, cap, layout.data_ptr()) == lic.E_INVALID_ARG
    assert call(sy.data_ptr(), data.data_ptr() + 1, cap, layout.data_ptr()) == lic.E_INVALID_ARG
    assert call(sy.data_ptr(), data.data_ptr(), cap, layout.data_ptr() + 4) == lic.E_INVALID_ARG
    assert call(host_sy.ctypes.data, data.data_ptr(), cap, layout.data_ptr()) == lic.E_INVALID_ARG
    assert call(sy.data_ptr(), data.data_ptr(), cap, layout.data_ptr()) == lic.OK
    assert codec.sync_status() == lic.OK
    codec.close()


def test_noalloc_at_a_new_larger_batch_allocates_nothing():
    """After one call, a call at a batch size the codec has never coded
    leaves the device's free memory and the codec's own count unchanged."""
    Wt = synth.make_weights(1, N, M)
    codec = lic.Codec(1, N, M, Wt)
    H, W, Hy, Wy = 128, 192, 8, 12
    bufs = {}
    for B in (1, 3):
        bufs[B] = (torch.zeros(B, M, Hy, Wy, dtype=torch.int32, device="cuda"),
                   torch.zeros(B, M, Hy, Wy, dtype=torch.uint8, device="cuda"),
                   torch.zeros(B, N, Hy // 4, Wy // 4, dtype=torch.int32, device="cuda"),
                   torch.zeros(B * frame_cap(1, Hy, Wy), dtype=torch.uint8, device="cuda"),
                   torch.zeros(2 * B + 1, dtype=torch.int64, device="cuda"))
    sy, idx, sz, data, layout = bufs[1]
    assert codec.encode_latents_noalloc(sy, idx, sz, H, W, data, layout) == lic.OK
    torch.cuda.synchronize()
    free0, held0 = torch.cuda.mem_get_info()[0], codec.device_bytes()
    sy, idx, sz, data, layout = bufs[3]
    assert codec.encode_latents_noalloc(sy, idx, sz, H, W, data, layout) == lic.OK
    torch.cuda.synchronize()
    assert codec.sync_status() == lic.OK
    assert torch.cuda.mem_get_info()[0] == free0
    assert codec.device_bytes() == held0
    codec.close()
