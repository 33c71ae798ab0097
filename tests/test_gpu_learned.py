"""The learned kernel surrogate on the GPU against the FP64 oracle.

Forward and backward per tensor: relative error (2-norm) <= 1e-4 with FP32
weights and <= 2e-2 with BF16 weights (the oracle evaluated at the same
BF16-rounded weights, so the check covers the FP32 accumulation); Adam against the oracle's step; the
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


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("bf16", 2e-2)])
def test_cnn_forward_backward_parity(ora, net, prec, tol):
    w32 = _test_weights(11)
    net.tensors()[0].copy_(torch.from_numpy(w32).cuda())          # the test's weights into the network
    net.set_precision(prec)                                          # refreshes the BF16 copy from them
    if prec == "bf16":   # the oracle gets the BF16-rounded weights the GPU computes with, rounded on the host
        w32 = torch.from_numpy(w32).to(torch.bfloat16).to(torch.float32).numpy()
    master = w32.astype(np.float64)
    rng = np.random.default_rng(1)
    x = rng.normal(0, 1, (3, NPX, 2)).astype(np.float32)
    dy = rng.normal(0, 1e-3, (3, NPX)).astype(np.float32)
    yo, acts = ora.cnn_forward(master, x.astype(np.float64))
    go = ora.cnn_backward(master, x.astype(np.float64), acts, dy.astype(np.float64))
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((3, NPX), device="cuda")
    B.argus_cnn_forward(net.net, xd, 3, y)
    g = torch.empty(master.size, device="cuda")
    B.argus_cnn_backward(net.net, xd, torch.from_numpy(dy).cuda(), 3, g)
    torch.cuda.synchronize()
    yg = y.cpu().numpy()
    assert np.linalg.norm(yg - yo) / np.linalg.norm(yo) < tol
    gg = g.cpu().numpy()
    worst = 0.0
    for nm, sl in _tensors():
        e = np.linalg.norm(gg[sl] - go[sl]) / max(np.linalg.norm(go[sl]), 1e-30)
        worst = max(worst, e)
        assert e < tol, (prec, nm, e)
    print(f"\n[cnn {prec}] forward rel {np.linalg.norm(yg - yo) / np.linalg.norm(yo):.2e}, worst grad tensor {worst:.2e}")


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
