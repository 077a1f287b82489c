"""The serving form through the C ABI (include/lic_serve.h), marked gpu.

A frame served in a mix -- batched with other frames of its resolution, on
one of several lanes, while other resolutions run concurrently, replayed
from a CUDA graph -- gives the same bitstream size and the same
reconstruction, bit for bit, as the same frame encoded and decoded alone by
a plain codec; the codec's results are per frame.  For the FP32 chain at the
configured width (N=128, M=192), the bitstream of one frame per resolution
is also decoded by the FP64 oracle: its symbols must equal the GPU
decoder's and its reconstruction must lie within 1e-4 of the served frame,
so the served results are pinned to the oracle, not only to the library."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu
N, M = 128, 192
TOL = 1e-4


@pytest.fixture(scope="module")
def W():
    return synth.make_weights(lic.HYPERPRIOR, N, M)


def oracle_check(c, oc, blob, out, H, Wd):
    """The parity rules on one frame's bitstream and reconstruction: the
    oracle decodes the bytes with the GPU decoder's own indices to the GPU
    decoder's symbols (integer stages, exact); those indices differ from the
    FP64 chain's only beside a scale-table edge; the oracle's g_s of the same
    y_hat is within TOL of the served frame (float stage)."""
    hdr = O.unpack_frame(blob)
    n, m, R = hdr["N"], hdr["M"], hdr["R"]
    Hy, Wy = hdr["Hp"] // 16, hdr["Wp"] // 16
    Hz, Wz = Hy // 4, Wy // 4
    sy_g = np.zeros((1, m, Hy, Wy), np.int32)
    sz_g = np.zeros((1, n, Hz, Wz), np.int32)
    idx_g = np.zeros((1, m, Hy, Wy), np.uint8)
    c.read_tensor(lic.T_SY, sy_g)
    c.read_tensor(lic.T_SZ, sz_g)
    c.read_tensor(lic.T_IDX, idx_g)
    subs = hdr["subs"]
    s_z = np.stack([O.rans_decode(subs[ch], Hz * Wz, np.full(Hz * Wz, ch), oc.eb).reshape(Hz, Wz)
                    for ch in range(n)])
    assert np.array_equal(s_z, sz_g[0])
    s_y = np.zeros((m, Hy, Wy), np.int32)
    k = n
    for ch in range(m):
        for r0, r1 in O._bands(Hy, R):
            t = idx_g[0, ch, r0:r1].ravel().astype(np.int32)
            s_y[ch, r0:r1] = O.rans_decode(subs[k], t.size, t, oc.gauss).reshape(r1 - r0, Wy)
            k += 1
    assert np.array_equal(s_y, sy_g[0])
    sig = O.h_s(oc.W, O.dequantize(s_z[None], oc.med))
    bad = O.scale_index(sig.astype(np.float32)) != idx_g
    T = O.scale_table().astype(np.float64)
    sg = sig[bad]
    assert np.all(np.min(np.abs(sg[:, None] - T[None, :]), axis=1) <= TOL * np.maximum(1.0, sg)), int(bad.sum())
    ref = np.clip(O.g_s(oc.W, s_y[None].astype(np.float32)), 0.0, 1.0)[:, :, :H, :Wd]
    err = float(np.abs(out - ref).max())
    assert err <= TOL, f"served frame {H}x{Wd} vs oracle: {err}"


def alone(W, frame, precision, n=N, m=M, oracle=None):
    """(bitstream size, reconstruction) of the frame coded by a plain codec;
    with oracle = an O.Codec, also checks that bitstream against the oracle."""
    c = lic.Codec(lic.HYPERPRIOR, n, m, W, precision=precision)
    x = torch.from_numpy(frame[None]).cuda()
    bs = c.encode(x)
    out = torch.empty_like(x)
    c.decode(bs, out)
    size = bs.sizes()[0]
    if oracle is not None:
        oracle_check(c, oracle, bs.to_bytes()[0], out.cpu().numpy(), *frame.shape[1:])
    c.close()
    return size, out[0].cpu()


@pytest.mark.parametrize("graphs", [True, False])
def test_served_frames_equal_frames_coded_alone(W, graphs):
    oc = O.Codec(lic.HYPERPRIOR, N, M, W) if graphs else None
    shapes = [(64, 96)] * 5 + [(128, 128)] * 3 + [(64, 96)] * 2
    frames = [synth.make_frame(40 + i, h, w) for i, (h, w) in enumerate(shapes)]
    srv = lic.Server(lic.HYPERPRIOR, N, M, W, max_batch=3, lanes=2, graphs=graphs, max_wait_ms=1.0)
    srv.prepare(64, 96)
    srv.prepare(128, 128)
    dev = [torch.from_numpy(f).cuda() for f in frames]
    outs = [torch.empty_like(d) for d in dev]
    tickets = [srv.submit(i % 4, d, o) for i, (d, o) in enumerate(zip(dev, outs))]
    assert tickets == list(range(len(frames)))
    srv.drain(60000)
    res = {r["ticket"]: r for r in srv.poll(64)}
    assert sorted(res) == tickets
    st = srv.stats()
    assert st["completed"] == len(frames) and st["buckets"] == 2 and st["device_bytes"] > 0
    if graphs:
        assert st["graph_replays"] >= 1
    else:
        assert st["graph_replays"] == 0
    checked = set()
    for i, f in enumerate(frames):
        r = res[i]
        assert r["status"] == 0 and (r["H"], r["W"]) == shapes[i] and r["stream_id"] == i % 4
        assert r["t_submit_ms"] <= r["t_start_ms"] <= r["t_done_ms"]
        first_of_shape = oc is not None and shapes[i] not in checked
        checked.add(shapes[i])
        size, x = alone(W, f, lic.FP32, oracle=oc if first_of_shape else None)
        assert r["bytes"] == size, i
        assert torch.equal(outs[i].cpu(), x), i
    srv.close()


def test_served_bf16_frames_equal_alone():
    """The BF16 precision form (N=128, M=192), pinned host frames in and out."""
    W = synth.make_weights(lic.HYPERPRIOR, 128, 192)
    frames = [synth.make_frame(60 + i, 64, 128) for i in range(4)]
    srv = lic.Server(lic.HYPERPRIOR, 128, 192, W, precision=lic.BF16, max_batch=4, lanes=1, max_wait_ms=50.0)
    hosts = [torch.from_numpy(f).pin_memory() for f in frames]
    outs = [torch.empty(f.shape).pin_memory() for f in frames]
    for i, (h, o) in enumerate(zip(hosts, outs)):
        srv.submit(0, h, o)
    srv.drain(60000)
    res = {r["ticket"]: r for r in srv.poll(16)}
    assert all(r["batch"] == 4 for r in res.values())
    for i, f in enumerate(frames):
        size, x = alone(W, f, lic.BF16, 128, 192)
        assert res[i]["bytes"] == size
        assert torch.equal(outs[i], x)
    srv.close()


def test_server_admission(W):
    f = torch.from_numpy(synth.make_frame(80, 64, 64)).cuda()
    tiny = lic.Server(lic.HYPERPRIOR, N, M, W, hbm_budget=1)
    with pytest.raises(lic.LicError) as e:
        tiny.submit(0, f)
    assert e.value.code == lic.E_OOM
    assert tiny.stats()["refused_budget"] == 1 and tiny.stats()["buckets"] == 0
    tiny.close()
    # the budget is charged what the lanes' codecs count, not the device's
    # free memory: two lanes of one resolution hold at least the estimate of
    # their workspaces, and a budget just below that sum is refused before
    # the workspaces are made
    probe = lic.Codec(lic.HYPERPRIOR, N, M, W)
    per_lane = probe.device_bytes() + probe.workspace_bytes(2, 64, 64) + 2 * 2 * 3 * 64 * 64 * 4
    probe.close()
    srv = lic.Server(lic.HYPERPRIOR, N, M, W, max_batch=2, lanes=2, hbm_budget=2 * per_lane - 1)
    with pytest.raises(lic.LicError) as e:
        srv.prepare(64, 64)
    assert e.value.code == lic.E_OOM
    srv.close()
    srv = lic.Server(lic.HYPERPRIOR, N, M, W, max_batch=2, lanes=2, hbm_budget=4 * per_lane)
    srv.prepare(64, 64)
    held = srv.stats()["device_bytes"]
    assert 2 * per_lane <= held <= 4 * per_lane, (held, per_lane)
    srv.close()
    # one request admitted (it waits in its bucket for a second frame), the next refused
    srv = lic.Server(lic.HYPERPRIOR, N, M, W, max_batch=2, max_pending=1, max_wait_ms=1e7)
    srv.submit(0, f)
    with pytest.raises(lic.LicError) as e:
        srv.submit(1, f)
    assert e.value.code == lic.E_BUSY
    assert srv.stats()["refused_busy"] == 1
    srv.close()   # the queued partial batch runs at shutdown
