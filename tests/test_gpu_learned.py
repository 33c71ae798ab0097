"""The learned kernel surrogate on the GPU against the FP64 oracle.

Forward and backward at the batch sizes the path runs (400, 512), with FP32 and with BF16
weights (the oracle evaluated at the same BF16-rounded weights, so the check covers the FP32
accumulation): element by element within 1e-4 of each tensor's largest magnitude (BF16
gradients at He weights: bit-identical to the FP32 mode at the same rounded weights);
gradients and training bit-reproducible; Adam against the oracle's step; the
spatial least squares across stamps and the background fit against library
least-squares solutions; a short training run lowers the loss; the per-frame
learned fit falls back to the least-squares fit when its chi2 is worse.
"""
import numpy as np
import pytest
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300 import synth
from paper_2207_14304_gb300.learned import NPX, KernelNet
from paper_2207_14304_gb300.synth import pitch_for

pytestmark = pytest.mark.gpu


def _tensors(n=200_961):
    o = 0
    names = [("W1", 64), ("b1", 32)]
    for l in range(4):
        names += [(f"W{l + 2}", 49 * 1024), (f"b{l + 2}", 32)]
    names += [("W6", 32), ("b6", 1)]
    out = []
    for nm, k in names:
        out.append((nm, slice(o, o + k)))
        o += k
    assert o == n
    return out


def _test_weights(seed):
    """He-normal weights and small biases drawn by the test (never read back from the
    library), FP32."""
    rng = np.random.default_rng(seed)
    fan = {"W1": 2, "W6": 32, **{f"W{l + 2}": 49 * 32 for l in range(4)}}
    out = np.empty(200_961, np.float32)
    for nm, sl in _tensors():
        n = sl.stop - sl.start
        out[sl] = (rng.normal(0, np.sqrt(2.0 / fan[nm]), n) if nm in fan else rng.normal(0, 0.01, n))
    return out


@pytest.fixture(scope="module")
def net():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    k = KernelNet(max_batch=8, seed=7)
    yield k
    k.close()


@pytest.fixture(scope="module")
def bignet():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    k = KernelNet(max_batch=512, seed=7)
    yield k
    k.close()


# element-wise bars (fraction of the largest magnitude of the compared tensor): the oracle runs
# at the weights the GPU computes with (BF16-rounded on the host for the BF16 case), so both
# cases differ only by FP32 accumulation order over <= 1568-term sums
EW_TOL = 1e-4


def _tie_free_weights(seed):
    """Weights whose ReLU decisions no rounding can change: biases of +1 or -1 (random per
    channel) and weights at 1/20 of the He scale, so every pre-activation of a conv layer is
    within ~0.1 of +-1 and half the channels are on, half off.  (With He weights some
    pre-activation lies within FP32 rounding of zero: the FP32 kernels and the FP64 oracle
    then switch that unit differently, and one flipped unit moves a bias gradient by a few
    per cent; measured on these inputs with the BF16-rounded weights.)"""
    rng = np.random.default_rng(seed)
    fan = {"W1": 2, "W6": 32, **{f"W{l + 2}": 49 * 32 for l in range(4)}}
    out = np.empty(200_961, np.float32)
    for nm, sl in _tensors():
        n = sl.stop - sl.start
        if nm in fan:
            out[sl] = rng.normal(0, np.sqrt(2.0 / fan[nm]) * (1.0 if nm in ("W1", "W6") else 0.05), n)
        elif nm in ("b1", "b6"):
            out[sl] = rng.normal(0, 0.01, n)
        else:
            out[sl] = rng.choice([-1.0, 1.0], n)
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16_split"])
@pytest.mark.parametrize("batch,sample", [(400, (0, 1, 133, 262, 399)), (512, (0, 97, 255, 256, 511)),
                                          (7, (0, 3, 6))])
@pytest.mark.parametrize("weights", ["tie_free", "he"])
def test_cnn_forward_backward_parity(ora, bignet, prec, batch, sample, weights):
    """Forward and backward at the batch sizes the path uses (400 stamps per frame, 512 per
    training step), so the kernels' batch tiling is the one that runs: every output of the
    sampled images element by element, and the whole gradient with the loss gradient dy
    nonzero only on the sampled images (the other images then contribute exactly zero, so the
    oracle needs only the sampled ones).  Gradients element by element, except with He weights
    (what training starts from) and BF16: there a pre-activation within FP32 rounding of zero
    may switch its ReLU differently in the kernels and in the oracle (one such unit moves a
    bias gradient by a few per cent), so the BF16 gradient must instead equal, bit for bit,
    the FP32 mode's at the same rounded weights, which meets the element-wise bar here.
    bf16_split (the forward on the tensor cores, activations as BF16 hi + lo): the forward
    element by element against the oracle at the BF16-rounded weights; its gradient (the 7x7
    layers' data gradients also on the tensor cores, with BF16 hi + lo gradient planes; the
    weight gradients on the CUDA cores, on the tensor-core forward's activations) element by
    element with tie-free weights."""
    net = bignet
    w32 = _tie_free_weights(11) if weights == "tie_free" else _test_weights(11)
    net.tensors()[0].copy_(torch.from_numpy(w32).cuda())          # the test's weights into the network
    net.set_precision(prec)                                          # refreshes the BF16 copy from them
    if prec != "fp32":   # the oracle gets the BF16-rounded weights the GPU computes with, rounded on the host
        w32 = torch.from_numpy(w32).to(torch.bfloat16).to(torch.float32).numpy()
    master = w32.astype(np.float64)
    rng = np.random.default_rng(batch)
    x = rng.normal(0, 1, (batch, NPX, 2)).astype(np.float32)
    dy = np.zeros((batch, NPX), np.float32)
    sl = list(sample)
    dy[sl] = rng.normal(0, 1e-3, (len(sl), NPX)).astype(np.float32)
    yo, acts = ora.cnn_forward(master, x[sl].astype(np.float64))
    go = ora.cnn_backward(master, x[sl].astype(np.float64), acts, dy[sl].astype(np.float64))
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((batch, NPX), device="cuda")
    B.argus_cnn_forward(net.net, xd, batch, y)
    g = torch.empty(master.size, device="cuda")
    B.argus_cnn_backward(net.net, xd, torch.from_numpy(dy).cuda(), batch, g)
    assert B.argus_cnn_status(net.net) == 0
    yg = y.cpu().numpy()[sl]
    ey = np.abs(yg - yo).max() / np.abs(yo).max()
    assert ey < EW_TOL, ey
    gg = g.cpu().numpy()
    if weights == "he" and prec == "bf16_split":
        print(f"\n[cnn bf16_split he batch {batch}] forward max |dy| {ey:.2e}")
        return
    if weights == "he" and prec == "bf16":
        net.tensors()[0].copy_(torch.from_numpy(w32).cuda())        # the rounded weights as FP32 master
        net.set_precision("fp32")
        y32 = torch.empty_like(y)
        g32 = torch.empty_like(g)
        B.argus_cnn_forward(net.net, xd, batch, y32)
        B.argus_cnn_backward(net.net, xd, torch.from_numpy(dy).cuda(), batch, g32)
        torch.cuda.synchronize()
        assert torch.equal(y32, y) and torch.equal(g32, g)
        print(f"\n[cnn bf16 he batch {batch}] forward max |dy| {ey:.2e}, gradient = FP32 mode's bit for bit")
        return
    worst = 0.0
    for nm, s in _tensors():
        e = np.abs(gg[s] - go[s]).max() / max(np.abs(go[s]).max(), 1e-30)
        assert e < EW_TOL, (prec, nm, e)
        worst = max(worst, e)
    print(f"\n[cnn {prec} {weights} batch {batch}] forward max |dy| {ey:.2e}, worst gradient element {worst:.2e}")


@pytest.mark.parametrize("prec", ["bf16", "bf16_split"])
def test_cnn_gradients_and_training_are_reproducible(prec):
    """No float atomics in the gradient: the same batch gives the same gradient bit for bit,
    and two short trainings from one seed give the same weights bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g0 = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand((96, NPX, 2), generator=g0, device="cuda") / NPX
    t = torch.rand((96, NPX), generator=g0, device="cuda") / NPX
    dy = torch.randn((96, NPX), generator=g0, device="cuda") * 1e-3
    finals = []
    for rep in range(2):
        k = KernelNet(max_batch=96, seed=3, precision=prec)
        try:
            ga = torch.empty(200_961, device="cuda")
            gb = torch.empty(200_961, device="cuda")
            B.argus_cnn_backward(k.net, x, dy, 96, ga)
            B.argus_cnn_backward(k.net, x, dy, 96, gb)
            torch.cuda.synchronize()
            assert torch.equal(ga, gb)
            k.fit(x, t, epochs=5, batch=32, lr=1e-3)
            assert B.argus_cnn_status(k.net) == 0
            finals.append(k.tensors()[0].clone())
        finally:
            k.close()
    assert torch.equal(finals[0], finals[1])


def test_cnn_adam_step_matches_oracle(ora, net):
    """Parameters, moments, step and gradient all drawn by the test and loaded into the
    network; one library Adam step against the oracle's."""
    rng = np.random.default_rng(2)
    n = 200_961
    p0 = _test_weights(3)
    m0 = rng.normal(0, 1e-3, n).astype(np.float32)
    v0 = rng.uniform(0, 1e-5, n).astype(np.float32)
    step0 = 7
    for t, a in zip(net.tensors(), (p0, m0, v0)):
        t.copy_(torch.from_numpy(a).cuda())
    B.argus_cnn_set_state(net.net, net.precision, step0)
    gr = rng.normal(0, 1e-2, n).astype(np.float32)
    B.argus_cnn_adam(net.net, torch.from_numpy(gr).cuda(), 1e-3)
    torch.cuda.synchronize()
    p, mm, vv = p0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64)
    ora.adam(p, mm, vv, gr.astype(np.float64), lr=1e-3, step=step0 + 1)
    after = net.tensors()[0].cpu().numpy()
    np.testing.assert_allclose(after, p, rtol=1e-5, atol=1e-8)


def test_cnn_training_lowers_loss():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    k = KernelNet(max_batch=64, seed=3)
    try:
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.rand((64, NPX, 2), generator=g, device="cuda") / NPX
        # target: a fixed Gaussian kernel, the task a surrogate must at least learn
        u = torch.arange(21, device="cuda", dtype=torch.float32) - 10
        G = torch.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2 * 1.5 ** 2))
        t = (G / G.sum()).reshape(1, NPX).repeat(64, 1).contiguous()
        hist = k.fit(x, t, epochs=300, batch=64, lr=2e-3)
        assert hist[-1] < 0.2 * hist[0], hist
    finally:
        k.close()


def test_learned_spatial_least_squares(ora):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    W, H, n = 900, 700, 60
    rng = np.random.default_rng(4)
    cen = np.stack([rng.integers(20, W - 20, n), rng.integers(20, H - 20, n)], 1).astype(np.int32)
    Ktrue = rng.normal(0, 1, (6, NPX))
    P = np.array([ora.spatial_terms(x, y, W, H, 2) for x, y in cen])
    y = (P @ Ktrue).astype(np.float32)
    ctx = B.argus_create(0, 1 << 16, 64, 64, 1 << 10)
    try:
        K = torch.empty((6, NPX), device="cuda")
        B.argus_learned_kernel(ctx, torch.from_numpy(y).cuda(), torch.from_numpy(cen).cuda(),
                               torch.tensor([n, 0, 0, 0], dtype=torch.int32, device="cuda"), n, W, H, 2, K)
        torch.cuda.synchronize()
        want = np.linalg.lstsq(P, y.astype(np.float64), rcond=None)[0]
        np.testing.assert_allclose(K.cpu().numpy(), want, rtol=1e-5, atol=1e-5)
    finally:
        B.argus_destroy(ctx)


def test_fit_background_matches_library_least_squares(ora):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, h = 300, 260
    cat = synth.star_catalog(300, w, h, seed=8, flux_min=1e3, flux_max=1e5)
    R = synth.render(cat, w, h, 1.2, sky=300.0).numpy().astype(np.float32)
    rng = np.random.default_rng(5)
    I = (R + rng.normal(0, 5, R.shape)).astype(np.float32)
    V = np.full_like(I, 25.0)
    fl = np.zeros((h, w), np.uint8)
    K = (rng.normal(0, 1e-3, (6, 21, 21))).astype(np.float32)
    K[0, 10, 10] += 1.0
    cen = np.array([(60, 60), (150, 80), (240, 200), (100, 180), (200, 120)], np.int32)
    xy = np.array([(x, y) for xs, ys in cen for y in range(ys - 10, ys + 11) for x in range(xs - 10, xs + 11)],
                  np.int32)
    D0, _ = ora.subtract_at(xy, I, V, R, np.zeros_like(V), fl, K.astype(np.float64), np.zeros(6), sdeg=2, bgdeg=2)
    Pb = np.array([ora.spatial_terms(x, y, w, h, 2) for x, y in xy])
    wgt = 1.0 / 25.0
    bg_want = np.linalg.lstsq(Pb, D0, rcond=None)[0]
    chi_want = wgt * ((D0 - Pb @ bg_want) ** 2).sum()
    pitch = pitch_for(w)
    ctx = B.argus_create(0, h * pitch, 64, 64, 1 << 10)
    try:
        def dev(a):
            t = torch.zeros((h, pitch), dtype=torch.from_numpy(a).dtype)
            t[:, :w] = torch.from_numpy(a)
            return t.cuda()
        bg = torch.zeros(6, dtype=torch.float64, device="cuda")
        st = torch.zeros(128, dtype=torch.uint8, device="cuda")
        B.argus_fit_background(ctx, dev(I), dev(V), dev(R), dev(fl), B.argus_shape(w, h, pitch),
                               torch.from_numpy(cen).cuda(), torch.tensor([5, 0, 0, 0], dtype=torch.int32).cuda(), 5,
                               21, torch.from_numpy(K.reshape(-1)).cuda(), 21, 2, 2, bg, st)
        torch.cuda.synchronize()
        s = B.fit_stats_from_bytes(st)
        # the model convolution runs in FP32 (FP64 sums): the background agrees to
        # 1e-4 of the 5 e- noise and chi2 to 1e-5 relative
        np.testing.assert_allclose(bg.cpu().numpy(), bg_want, rtol=0, atol=5e-4)
        assert abs(s["chi2"] / chi_want - 1) < 1e-5 and s["n_pix"] == len(xy)
    finally:
        B.argus_destroy(ctx)


def test_fit_scale_background_recovers_scales(ora):
    """A kernel given at the wrong flux scale per spatial term is rescaled by the joint
    least squares: I = sum_k p_k R (x) (s_k K_k) + bg exactly, so the fit returns s_k, bg
    and chi2 = 0 (FP32-model level)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, h = 300, 260
    cat = synth.star_catalog(300, w, h, seed=8, flux_min=1e3, flux_max=1e5)
    R = synth.render(cat, w, h, 1.2, sky=300.0).numpy().astype(np.float32)
    rng = np.random.default_rng(6)
    K = (rng.normal(0, 1e-3, (6, 21, 21))).astype(np.float32)
    K[0, 10, 10] += 1.0
    scales = np.array([1.02, 0.97, 1.05, 0.9, 1.1, 0.95])
    bg_true = np.array([3.0, 1.0, -0.5, 0.7, 0.2, -0.3])
    cen = np.array([(60, 60), (150, 80), (240, 200), (100, 180), (200, 120), (60, 200)], np.int32)
    # science = the exact model with the true scales (oracle, FP64)
    Ktrue = (K * scales[:, None, None]).astype(np.float64)
    I0 = np.zeros((h, w), np.float32)
    xy = np.array([(x, y) for y in range(h) for x in range(w)], np.int32)
    D, _ = ora.subtract_at(xy, I0, np.ones_like(I0), R, np.zeros_like(R), np.zeros((h, w), np.uint8), Ktrue,
                           bg_true, sdeg=2, bgdeg=2)
    I = (-D).reshape(h, w).astype(np.float32)          # I = model (D = 0 - model)
    V = np.full_like(I, 25.0)
    fl = np.zeros((h, w), np.uint8)
    pitch = pitch_for(w)
    ctx = B.argus_create(0, h * pitch, 64, 64, 1 << 10)
    try:
        def dev(a):
            t = torch.zeros((h, pitch), dtype=torch.from_numpy(a).dtype)
            t[:, :w] = torch.from_numpy(a)
            return t.cuda()
        bg = torch.zeros(6, dtype=torch.float64, device="cuda")
        st = torch.zeros(128, dtype=torch.uint8, device="cuda")
        dK = torch.from_numpy(K.reshape(-1).copy()).cuda()
        B.argus_fit_scale_background(ctx, dev(I), dev(V), dev(R), dev(fl), B.argus_shape(w, h, pitch),
                                     torch.from_numpy(cen).cuda(), torch.tensor([6, 0, 0, 0], dtype=torch.int32).cuda(),
                                     6, 21, dK, 21, 2, 2, bg, st)
        torch.cuda.synchronize()
        s = B.fit_stats_from_bytes(st)
        assert s["status"] == 0 and s["n_coeffs"] == 12 and s["dof"] == s["n_pix"] - 12
        Kout = dK.cpu().numpy().reshape(6, 21, 21)
        np.testing.assert_allclose(Kout, K * scales[:, None, None], rtol=1e-4, atol=1e-7)
        np.testing.assert_allclose(bg.cpu().numpy(), bg_true, atol=2e-3)
        assert s["chi2"] < 1e-4 * s["n_pix"]
    finally:
        B.argus_destroy(ctx)


def test_learned_fit_falls_back_to_least_squares():
    """An untrained network's kernel is far worse than the least-squares fit, so the
    per-frame learned fit must judge it by chi2 and use the plain fit instead; with
    the chi2 check disabled (ratio = inf) the learned kernel is used and subtraction runs."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_14304_gb300.learned import LearnedFit
    from paper_2207_14304_gb300.pipeline import FramePipeline
    w = h = 320
    cat = synth.star_catalog(900, w, h, seed=21)
    R, Vr = synth.reference_image(synth.render(cat, w, h, 1.2, sky=300.0), 30, 1.7, 22)
    cal = synth.make_calib(w, h, seed=23)
    raw = synth.expose(synth.render(cat, w, h, 1.8, sky=305.0), cal, seed=24)
    basis = B.make_basis(21, (0.7, 1.5, 3.0), (6, 4, 2), 1, 1)
    pipe = FramePipeline(w, h, basis=basis, grid=(4, 4))
    net = KernelNet(max_batch=16, seed=5)
    try:
        def dev(a):
            t = torch.zeros((h, pipe.pitch), dtype=a.dtype)
            t[:, :w] = a
            return t.cuda()
        d_raw, d_R, d_Vr = dev(raw), dev(R), dev(Vr)
        calib = B.make_calib(cal.bias, dev(cal.dark), dev(cal.flat), dev(cal.bpm), cal.gain, cal.read_noise, cal.sat)
        lf = LearnedFit(pipe, net)
        assert lf.run(d_raw, calib, d_R, d_Vr) is True        # first frame: plain fit sets the reference chi2
        assert lf.plain_chi2_dof is not None and lf.plain_chi2_dof < 5
        assert lf.run(d_raw, calib, d_R, d_Vr) is True        # untrained network: judged worse, fallback
        assert lf.n_fallback == 1 and lf.n_learned == 0
        lf.ratio = float("inf")
        assert lf.run(d_raw, calib, d_R, d_Vr) is False       # judge off: learned kernel used
        torch.cuda.synchronize()
        assert B.argus_sync_status(pipe.ctx) == 0
        assert torch.isfinite(pipe.diff).all()
    finally:
        net.close()
        pipe.close()
