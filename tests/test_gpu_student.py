"""The learned form's student synthesis net through the C ABI
(include/lic_student.h) against the FP64 oracle (marked gpu).

Float bar: the gradients of one batch agree with the oracle's chain-rule
backward pass to 1e-4 of each tensor's largest magnitude (float32 sums over
up to B*H*W terms); the forward pass to max-abs 1e-4; Adam, fed the GPU's
own gradients, to 1e-6 of the learning rate.  Decoding with the student
returns exactly the student's (or, on fallback, the teacher's) frames."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu
M, C = 192, 64


@pytest.fixture(scope="module")
def SW():
    return synth.make_student_weights(M, C)


def pools(P, Hy, Wy, seed):
    r = np.random.default_rng(seed)
    yp = np.rint(r.standard_normal((P, M, Hy, Wy)) * 2.0).astype(np.float32)
    xp = r.uniform(0.0, 1.0, (P, 3, 16 * Hy, 16 * Wy)).astype(np.float32)
    return yp, xp


def test_student_gradients_match_oracle(SW):
    """Loss and every parameter gradient of a 3-crop batch of 96 x 96 crops
    (latent windows 6 x 6 out of a 2-frame 8 x 10 pool): split-K slices of
    the weight gradient end ragged, the 3-channel layer takes the scalar
    path, and the input-gradient convolutions span several tiles.

    The forward activations match to max-abs 1e-4.  A ReLU decision is a
    float deciding a bit: a pre-activation within rounding of 0 may fall
    either way (this case has a few dozen within 1e-5), so the GPU's
    decisions must equal the oracle's wherever the oracle's pre-activation is
    farther than 1e-4 from 0, and the oracle's backward pass then takes the
    GPU's decisions -- the rest of the chain is compared exactly as is."""
    yp, xp = pools(2, 8, 10, seed=1)
    crops = np.array([[0, 0, 0], [1, 2, 4], [1, 1, 3]], np.int32)
    st = lic.Student(SW, M, C, max_batch=4, crop=96)
    loss = st.grad(torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda(), crops)
    ys, xs = O.student_crops(yp, xp, crops, 96)
    hs, _ = O.student_forward(SW, ys)
    masks = {}
    for l in (1, 2, 3):
        h = st.activation(l, 3).transpose(0, 3, 1, 2)
        assert np.abs(h - hs[l]).max() <= 1e-4, l
        z = O.deconv2d(hs[l - 1], SW[f"student.deconv{l - 1}.weight"], SW[f"student.deconv{l - 1}.bias"], 2)
        clear = np.abs(z) > 1e-4
        assert np.array_equal((h > 0)[clear], (z > 0)[clear]), l
        masks[l] = h > 0
    oloss, ograds = O.student_loss_grads(SW, ys, xs, masks=masks)
    assert abs(loss - oloss) <= 1e-5 * oloss
    for name, og in ograds.items():
        g = st.read(name, lic.STUDENT_GRAD)
        err = np.abs(g - og).max()
        assert err <= 1e-4 * np.abs(og).max() + 1e-9, (name, err, np.abs(og).max())
    st.close()


def test_student_adam_step_matches_oracle(SW):
    """One lic_student_step: the new weights and both moments equal the
    oracle's Adam applied to the GPU's own gradients (stage-wise parity)."""
    yp, xp = pools(1, 6, 6, seed=2)
    crops = np.array([[0, 0, 0], [0, 1, 2]], np.int32)
    lr = 1e-3
    st = lic.Student(SW, M, C, max_batch=2, crop=64, lr=lr)
    dy, dx = torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda()
    P = {k: v.astype(np.float64) for k, v in SW.items()}
    m = {k: np.zeros(v.shape) for k, v in SW.items()}
    v = {k: np.zeros(x.shape) for k, x in SW.items()}
    for t in (1, 2):
        st.step(dy, dx, crops)
        G = {k: st.read(k, lic.STUDENT_GRAD) for k in SW}
        # the hyper-parameters cross the C ABI as float32: the oracle takes those values
        f32 = lambda q: float(np.float32(q))
        O.adam_step(P, G, m, v, t, lr=f32(lr), beta1=f32(0.9), beta2=f32(0.999), eps=f32(1e-8))
        for k in SW:
            assert np.abs(st.read(k) - P[k]).max() <= 1e-6 * lr + 1e-7 * np.abs(P[k]).max(), (k, t)
            assert np.abs(st.read(k, lic.STUDENT_ADAM_M) - m[k]).max() <= 1e-6 * np.abs(m[k]).max() + 1e-12
            assert np.abs(st.read(k, lic.STUDENT_ADAM_V) - v[k]).max() <= 1e-5 * np.abs(v[k]).max() + 1e-16
        P = {k: st.read(k).astype(np.float64) for k in SW}   # continue from the GPU's own weights
    assert st.steps() == 2
    st.close()


def test_student_forward_matches_oracle(SW):
    """Full-frame inference on a ragged 6 x 9 latent plane (B = 2)."""
    r = np.random.default_rng(3)
    yhat = np.rint(r.standard_normal((2, M, 6, 9)) * 2).astype(np.float32)
    st = lic.Student(SW, M, C, max_batch=1, crop=32)
    x = torch.empty(2, 3, 96, 144, device="cuda")
    st.forward(torch.from_numpy(yhat).cuda(), x)
    torch.cuda.synchronize()
    _, want = O.student_forward(SW, yhat)
    assert np.abs(x.cpu().numpy() - want).max() <= 1e-4
    # host buffers through the same call
    xh = np.zeros((2, 3, 96, 144), np.float32)
    st.forward(yhat, xh)
    assert np.array_equal(xh, x.cpu().numpy())
    st.close()


def test_student_training_lowers_loss(SW):
    """Thirty Adam steps on one fixed batch lower its loss."""
    yp, xp = pools(1, 8, 8, seed=4)
    crops = np.array([[0, 0, 0], [0, 2, 2]], np.int32)
    st = lic.Student(SW, M, C, max_batch=2, crop=96, lr=1e-3)
    dy, dx = torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda()
    l0 = st.grad(dy, dx, crops)
    for _ in range(30):
        st.step(dy, dx, crops)
    assert st.grad(dy, dx, crops) < 0.7 * l0
    st.close()


def test_student_rejects_bad_crops(SW):
    yp, xp = pools(1, 6, 6, seed=5)
    st = lic.Student(SW, M, C, max_batch=2, crop=64)
    dy, dx = torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda()
    for bad in ([[1, 0, 0]], [[0, 3, 0]], [[0, 0, -1]], [[0, 0, 0]] * 3):
        with pytest.raises(lic.LicError) as e:
            st.grad(dy, dx, np.array(bad, np.int32))
        assert e.value.code == lic.E_INVALID_ARG
    with pytest.raises(lic.LicError):   # host pools are refused
        st.grad(yp, xp, np.array([[0, 0, 0]], np.int32))
    st.close()


def test_decode_with_student(SW):
    """Factorized 128 x 128 codec (N=128, M=192) decoding with the student:
    unchecked decode = the student's output on the decoded y_hat (clamped,
    cropped); checked with an unreachable bar = the teacher's frames exactly,
    all counted as fallbacks; checked with a bar of -inf dB = the unchecked
    frames exactly; the reported PSNRs match the oracle's."""
    W = synth.make_weights(0, 128, M)
    codec = lic.Codec(0, 128, M, W)
    st = lic.Student(SW, M, C, max_batch=1, crop=32)
    x = synth.make_frames(2, 120, 100, first=11)
    bs = codec.encode(torch.from_numpy(x).cuda())
    teacher = torch.empty(2, 3, 120, 100, device="cuda")
    codec.decode(bs, teacher)
    sy = np.zeros((2, M, 8, 8), np.int32)
    codec.read_tensor(lic.T_SY, sy)
    oc = O.Codec(0, 128, M, W)
    yhat_np = O.dequantize(sy, oc.med)
    yhat_gpu = np.zeros((2, M, 8, 8), np.float32)
    codec.read_tensor(lic.T_YHAT, yhat_gpu)
    assert np.array_equal(yhat_gpu, yhat_np.astype(np.float32))
    _, xs = O.student_forward(SW, yhat_np)
    want_s = np.clip(xs, 0, 1)[:, :, :120, :100]

    codec.set_student(st)
    got_s = torch.empty_like(teacher)
    codec.decode(bs, got_s)
    torch.cuda.synchronize()
    assert np.abs(got_s.cpu().numpy() - want_s).max() <= 1e-4

    codec.set_student(st, min_psnr_db=1000.0, checked=True)
    fb = torch.empty_like(teacher)
    codec.decode(bs, fb)
    torch.cuda.synchronize()
    assert torch.equal(fb, teacher)
    frames, falls, ps = codec.student_report()
    assert (frames, falls) == (2, 2)
    t = teacher.cpu().numpy().astype(np.float64)
    for b in range(2):
        mse = np.mean((np.clip(xs[b, :, :120, :100], 0, 1) - t[b]) ** 2)
        assert abs(ps[b] - 10 * np.log10(1 / mse)) <= 1e-2

    codec.set_student(st, min_psnr_db=-np.inf, checked=True)
    ok = torch.empty_like(teacher)
    codec.decode(bs, ok)
    torch.cuda.synchronize()
    assert torch.equal(ok, got_s)
    assert codec.student_report()[:2] == (2, 0)

    codec.set_student(None)
    back = torch.empty_like(teacher)
    codec.decode(bs, back)
    torch.cuda.synchronize()
    assert torch.equal(back, teacher)
    codec.close()
    st.close()


# ---------------------------------------------------------------------------
# BF16 form: the 64-channel transposed convs and their input gradients on the
# tcgen05 bf16 kernel, bf16 storage of y_hat, h_1, h_2, dz_0..dz_2
# ---------------------------------------------------------------------------

def bf16(a):
    """Round float values to bfloat16 (nearest even), returned as float64."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_student_forward(P, yhat):
    """The BF16 form's forward pass as defined: bf16 y_hat, bf16 weights of the
    three 64-channel layers, bf16 storage of h_1 and h_2, float h_3 and a
    float 3-channel layer (the oracle's float64 arithmetic in between)."""
    h = bf16(yhat)
    for l in range(4):
        w = P[f"student.deconv{l}.weight"]
        z = O.deconv2d(h, bf16(w) if l < 3 else w, P[f"student.deconv{l}.bias"], 2)
        if l == 3:
            return z
        h = O.relu(z)
        if l < 2:
            h = bf16(h)


def test_bf16_student_forward_matches_its_definition(SW):
    r = np.random.default_rng(13)
    yhat = np.rint(r.standard_normal((2, M, 6, 9)) * 2).astype(np.float32)
    st = lic.Student(SW, M, C, max_batch=1, crop=32, precision=lic.BF16)
    x = torch.empty(2, 3, 96, 144, device="cuda")
    st.forward(torch.from_numpy(yhat).cuda(), x)
    torch.cuda.synchronize()
    got = x.cpu().numpy()
    want = bf16_student_forward(SW, yhat)
    assert np.abs(got - want).max() <= 2e-3
    # against the float64 student: the error bf16 storage costs
    _, exact = O.student_forward(SW, yhat)
    assert np.abs(got - exact).max() <= 5e-2
    st.close()


def test_bf16_student_gradients_close_to_oracle(SW):
    """BF16 gradients against the float64 chain rule (taking the GPU's ReLU
    decisions): relative L2 error of every tensor below 3e-2, loss within
    1e-2; an index or sign mistake anywhere gives O(1)."""
    yp, xp = pools(2, 8, 10, seed=1)
    crops = np.array([[0, 0, 0], [1, 2, 4], [1, 1, 3]], np.int32)
    st = lic.Student(SW, M, C, max_batch=4, crop=96, precision=lic.BF16)
    loss = st.grad(torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda(), crops)
    ys, xs = O.student_crops(yp, xp, crops, 96)
    masks = {l: st.activation(l, 3).transpose(0, 3, 1, 2) > 0 for l in (1, 2, 3)}
    oloss, ograds = O.student_loss_grads(SW, ys, xs, masks=masks)
    assert abs(loss - oloss) <= 1e-2 * oloss
    for name, og in ograds.items():
        g = st.read(name, lic.STUDENT_GRAD)
        rel = np.linalg.norm(g - og) / np.linalg.norm(og)
        assert rel <= 3e-2, (name, rel)
    st.close()


def test_bf16_student_training_and_decode(SW):
    yp, xp = pools(1, 8, 8, seed=4)
    crops = np.array([[0, 0, 0], [0, 2, 2]], np.int32)
    st = lic.Student(SW, M, C, max_batch=2, crop=96, lr=1e-3, precision=lic.BF16)
    dy, dx = torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda()
    l0 = st.grad(dy, dx, crops)
    for _ in range(30):
        st.step(dy, dx, crops)
    assert st.grad(dy, dx, crops) < 0.7 * l0
    # the decoder running this student returns its forward pass, clamped and cropped
    W = synth.make_weights(0, 128, M)
    codec = lic.Codec(0, 128, M, W)
    x = synth.make_frames(2, 120, 100, first=21)
    bs = codec.encode(torch.from_numpy(x).cuda())
    codec.set_student(st)
    got = torch.empty(2, 3, 120, 100, device="cuda")
    codec.decode(bs, got)
    yhat = torch.empty(2, M, 8, 8, device="cuda")
    codec.read_tensor(lic.T_YHAT, yhat)
    ref = torch.empty(2, 3, 128, 128, device="cuda")
    st.forward(yhat, ref)
    torch.cuda.synchronize()
    assert torch.equal(got, ref.clamp(0, 1)[:, :, :120, :100])
    codec.close()
    st.close()


@pytest.mark.parametrize("precision", [lic.FP32, lic.BF16])
def test_student_halo_window_gradients(SW, precision):
    """halo = 1: the student runs on 8 x 8 latent windows, the loss covers the
    central 96 x 96 output pixels (zero gradient outside)."""
    yp, xp = pools(2, 9, 10, seed=8)
    crops = np.array([[0, 0, 0], [1, 1, 2]], np.int32)
    st = lic.Student(SW, M, C, max_batch=2, crop=96, halo=1, precision=precision)
    loss = st.grad(torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda(), crops)
    ys, xs = O.student_crops(yp, xp, crops, 96, halo=1)
    assert ys.shape[-1] == 8 and xs.shape[-1] == 96
    masks = {l: st.activation(l, 2).transpose(0, 3, 1, 2) > 0 for l in (1, 2, 3)}
    oloss, ograds = O.student_loss_grads(SW, ys, xs, masks=masks)
    tol = 1e-5 if precision == lic.FP32 else 1e-2
    assert abs(loss - oloss) <= tol * oloss
    for name, og in ograds.items():
        g = st.read(name, lic.STUDENT_GRAD)
        if precision == lic.FP32:
            assert np.abs(g - og).max() <= 1e-4 * np.abs(og).max() + 1e-9, name
        else:
            assert np.linalg.norm(g - og) / np.linalg.norm(og) <= 3e-2, name
    with pytest.raises(lic.LicError):   # the window must fit: 2 + 8 > 9 rows
        st.grad(torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda(), np.array([[0, 2, 0]], np.int32))
    st.close()


def test_trained_student_gain_over_teacher_and_untrained(SW):
    """What the trained network gains: after 400 Adam steps on pairs the
    factorized codec generates, the student reconstructs the teacher's frames
    far better than before training (>= 8 dB), and decoding with it costs
    less than a third of g_s's multiply-adds per frame."""
    W = synth.make_weights(0, 128, M)
    codec = lic.Codec(0, 128, M, W)
    P, H, Wd = 4, 256, 256
    pool_y = torch.empty(P, M, H // 16, Wd // 16, device="cuda")
    pool_x = torch.empty(P, 3, H, Wd, device="cuda")
    for i in range(P):
        fr = torch.from_numpy(synth.make_frames(1, H, Wd, first=600 + i)).cuda()
        out = torch.empty_like(fr)
        codec.decode(codec.encode(fr), out)
        codec.read_tensor(lic.T_YHAT, pool_y[i:i + 1])
        codec.read_tensor(lic.T_XPRE, pool_x[i:i + 1])
    val = torch.from_numpy(synth.make_frames(2, H, Wd, first=700)).cuda()
    bs = codec.encode(val)
    teacher = torch.empty_like(val)
    codec.profile(True)
    codec.decode(bs, teacher)
    gs_flop = sum(r["flop"] for r in codec.profile_report() if r["name"].startswith("g_s."))
    codec.profile(False)

    st = lic.Student(SW, M, C, max_batch=8, crop=128, lr=1e-3, precision=lic.BF16)

    def psnr_vs_teacher():
        codec.set_student(st, min_psnr_db=99.0, checked=True)
        codec.decode(bs, torch.empty_like(val))
        ps = codec.student_report()[2]
        codec.set_student(None)
        return float(np.mean(ps))

    before = psnr_vs_teacher()
    for k in range(400):
        st.step(pool_y, pool_x, synth.draw_crops(k, 8, P, H // 16, Wd // 16, 8))
    after = psnr_vs_teacher()
    print(f"[student gain] PSNR vs teacher {before:.2f} dB untrained -> {after:.2f} dB after 400 steps")
    assert after >= before + 8.0, (before, after)
    st.profile(True)
    st.forward(torch.empty(2, M, H // 16, Wd // 16, device="cuda"), torch.empty(2, 3, H, Wd, device="cuda"))
    stu_flop = sum(r["flop"] for r in st.profile_report())
    st.profile(False)
    print(f"[student gain] decoder synthesis work {stu_flop / 1e9:.2f} GFLOP (student) vs {gs_flop / 1e9:.2f} (g_s)")
    assert stu_flop < gs_flop / 3, (stu_flop, gs_flop)
    codec.close()
    st.close()


def test_bf16_weight_gradients_on_tensor_cores_sum_exactly(SW):
    """The BF16 form's weight gradients of the three 64-channel layers come
    from the tcgen05 kernel (bf16 operands as stored, float32 sums in TMEM,
    pixel slices added in order).  Against the oracle's weight gradient of a
    transposed conv evaluated in float64 on the GPU's own stored h_l and dz_l
    they agree to 1e-5 of each tensor's largest magnitude: only the float32
    summation differs.  The 7 x 7, 14 x 14 and 28 x 28 grids (crop 80, halo
    1) leave ragged 64-pixel tiles, and the 28 x 28 layer runs 21 slices."""
    yp, xp = pools(2, 9, 10, seed=21)
    crops = np.array([[0, 0, 0], [1, 2, 3], [1, 1, 1]], np.int32)
    B = len(crops)
    st = lic.Student(SW, M, C, max_batch=4, crop=80, halo=1, precision=lic.BF16)
    st.grad(torch.from_numpy(yp).cuda(), torch.from_numpy(xp).cuda(), crops)
    for l in range(3):
        x = st.activation(l, B).transpose(0, 3, 1, 2)
        dz = st.output_grad(l, B).transpose(0, 3, 1, 2)
        assert x.shape[-1] == 7 << l and dz.shape[-1] == 14 << l
        want = O.deconv2d_wgrad(x, dz)
        got = st.read(f"student.deconv{l}.weight", lic.STUDENT_GRAD)
        assert np.abs(want).max() > 0
        err = np.abs(got - want).max()
        assert err <= 1e-5 * np.abs(want).max(), (l, err, np.abs(want).max())
    st.close()
