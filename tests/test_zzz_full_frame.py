"""Full-size parity: one 9576x6388 frame (150,000 stars, PSF 1.3-2.2 px across
the field, 21x21 kernel with degree-2 spatial variation, 400 stamps) through the
path in the launch configuration the benchmark times, against the FP64 oracle.

* calibration: every pixel (flags bit-exact, I and V within 4 float ulps);
* stamp selection: every centre, bit-exact;
* kernel fit (TF32 normal equations, as benchmarked; then FP32, BF16 split and
  BF16 at their bars): every kernel pixel within 1e-3 of max|K| and chi2 within
  1e-4 (the GPU fits its own calibrated frame, which is within 4 ulps of the
  oracle's); the oracle fits the oracle's calibrated frame;
* subtraction: the same entry point on the oracle's calibrated frame and
  kernel, 20,000 sampled pixels plus whole strips across the 128-pixel work
  tiles against the oracle evaluated pixel by pixel (the unit-test bars);
* detection: on the pipeline's own difference image, properties that hold at
  any size -- the mask is the float threshold of S = D / sqrt(V_D), the
  components are the 8-connected equal-sign components (scipy's labelling),
  each source's peak is its component's max |S| (ties to the lowest (y, x)),
  npix its size, and the list is ordered by (py, px).

The file sorts last so that the per-kernel parity files run first; it needs
about 3 GB of device memory and half a minute of oracle time on 16 cores.
"""
import numpy as np
import pytest
import torch

from paper_2207_14304_gb300 import _binding as B
from tests.gpu_helpers import F32_EPS, VD_RTOL, assert_rel, assert_variance, check_detection_properties, tile_rule_allowance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


def _calib_scale(n, cal):
    """Per-pixel magnitude of the calibration operands (the 4-ulp bar's scale)."""
    flat, dark = cal["flat"], cal["dark"]
    ng = np.abs(n.astype(np.float64) * cal["gain"])
    with np.errstate(divide="ignore", invalid="ignore"):
        ok = np.isfinite(flat) & (flat > 0)
        sI = np.where(ok, (ng + np.abs(dark)) / np.abs(flat), 1.0)
        sV = np.where(ok, (ng + cal["rn"] ** 2) / flat.astype(np.float64) ** 2, 1.0)
    return sI, sV


def test_full_frame_path_against_the_oracle(ora):
    import bench
    from paper_2207_14304_gb300.pipeline import FramePipeline
    from paper_2207_14304_gb300.synth import pitch_for
    W, H, ks, sdeg, bgdeg = bench.W, bench.H, bench.KSIZE, bench.SDEG, bench.BGDEG
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    raw_d, R_d, Vr_d, cal_d = bench.make_inputs(device, seed=2)
    pitch = pitch_for(W)

    def pad(a):
        t = torch.zeros((H, pitch), dtype=a.dtype, device=device)
        t[:, :W] = a
        return t

    raw, R, Vr = raw_d.cpu().numpy(), R_d.cpu().numpy(), Vr_d.cpu().numpy()
    cal = {"bias": cal_d.bias, "dark": cal_d.dark.cpu().numpy(), "flat": cal_d.flat.cpu().numpy(),
           "bpm": cal_d.bpm.cpu().numpy(), "gain": cal_d.gain, "rn": cal_d.read_noise, "sat": cal_d.sat}

    # --- the benchmark's pipeline, one frame
    basis = B.make_basis(ks, (0.7, 1.5, 3.0), (6, 4, 2), sdeg, bgdeg)
    pipe = FramePipeline(W, H, basis=basis, stamp=bench.STAMP, grid=bench.GRID, precision="tf32",
                         psf_sigma=1.8, device=0)
    try:
        dR, dVr = pad(R_d), pad(Vr_d)
        calib = B.make_calib(cal_d.bias, pad(cal_d.dark), pad(cal_d.flat), pad(cal_d.bpm), cal_d.gain,
                             cal_d.read_noise, cal_d.sat)
        pipe.run(pad(raw_d), calib, dR, dVr)
        torch.cuda.synchronize()
        assert pipe.status() == 0
        del raw_d, cal_d
        g_I, g_V, g_fl = (t[:, :W].cpu().numpy() for t in (pipe.img, pipe.var, pipe.flags))

        # --- calibration, every pixel
        I, V, fl, nn = ora.calibrate(raw, bias=cal["bias"], dark=cal["dark"], flat=cal["flat"], bpm=cal["bpm"],
                                     gain=cal["gain"], read_noise=cal["rn"], sat=cal["sat"])
        np.testing.assert_array_equal(g_fl, fl)
        sI, sV = _calib_scale(nn, cal)
        assert_rel(g_I, I, sI, 4 * F32_EPS, "I")
        assert_rel(g_V, V, sV, 4 * F32_EPS, "V")
        del g_I, g_V, sI, sV
        I32, V32 = I.astype(np.float32), V.astype(np.float32)
        del I, V

        # --- stamp selection, every centre
        cen = ora.select_stamps(R, fl, bench.GRID[0], bench.GRID[1], bench.STAMP, ks // 2, 3.0e4)
        n = int(pipe.n_stamps[0].item())
        assert n == len(cen) and n >= 300
        np.testing.assert_array_equal(pipe.centers[:n].cpu().numpy(), cen)

        # --- kernel fit
        b = ora.Basis(ksize=ks, spatial_degree=sdeg, bg_degree=bgdeg)
        res = ora.fit(I32, V32, R, fl, cen, bench.STAMP, b)
        assert res.status == 0
        Ko, bgo = ora.expand(b, res.coeffs)
        st = pipe.fit_stats()
        Kg = pipe.K.cpu().numpy().reshape(-1, ks, ks)
        kerr = np.abs(Kg - Ko).max() / np.abs(Ko).max()
        print(f"\n[full frame] stamps {n}  kernel-pixel err {kerr:.2e}  chi2 {st['chi2']:.9g} vs {res.chi2:.9g}")
        assert st["status"] == 0 and st["n_stamps_used"] == n and st["dof"] == res.dof
        assert kerr < 1e-3
        assert abs(st["chi2"] / res.chi2 - 1) < 1e-4
        np.testing.assert_allclose(pipe.bg.cpu().numpy(), bgo, rtol=0, atol=1e-3 * max(1.0, np.abs(bgo).max()))
        # the other normal-equation precisions on the same frame and stamps (the oracle's fit of its own
        # calibrated frame, as above): the bar of each precision
        from tests.test_gpu_parity import CHIBAR, KBAR
        for prec in ("fp32", "bf16_split", "bf16"):
            pipe.precision = prec
            pipe.fit(dR)
            torch.cuda.synchronize()
            assert pipe.status() == 0
            stp = pipe.fit_stats()
            Kp = pipe.K.cpu().numpy().reshape(-1, ks, ks)
            kp = np.abs(Kp - Ko).max() / np.abs(Ko).max()
            print(f"[full frame] {prec}: kernel-pixel err {kp:.2e}  chi2 rel {stp['chi2'] / res.chi2 - 1:+.2e}")
            assert stp["status"] == 0 and stp["refine_iters"] == 1
            assert kp < KBAR[prec]
            assert abs(stp["chi2"] / res.chi2 - 1) < max(CHIBAR[prec], 1e-4)
        pipe.precision = "tf32"
        pipe.fit(dR)

        # --- subtraction: the entry point on the oracle's frame and kernel
        K32 = Ko.astype(np.float32)
        dK = torch.from_numpy(K32.reshape(-1)).to(device)
        dbg = torch.from_numpy(np.asarray(bgo, np.float64)).to(device)
        dI, dV, dfl = (pad(torch.from_numpy(a).to(device)) for a in (I32, V32, fl))
        D2 = torch.full((H, pitch), -9.0, device=device)
        VD2 = torch.full((H, pitch), -9.0, device=device)
        B.argus_subtract(pipe.ctx, dI, dV, dR, dVr, dfl, pipe.shape, W, H, 0, 0, ks, sdeg, dK, bgdeg, dbg, D2, VD2)
        torch.cuda.synchronize()
        assert pipe.status() == 0
        del dI, dV, dfl
        rng = np.random.default_rng(7)
        xs = [rng.integers(0, W, 20000)]
        ys = [rng.integers(0, H, 20000)]
        for y0 in (0, 127, 128, 2000, H - 11, H - 1):        # whole rows across every 128-column strip
            xs.append(np.arange(W)); ys.append(np.full(W, y0))
        for x0 in (0, 10, 127, 128, 4095, W - 1):             # whole columns across every 128-row band
            xs.append(np.full(H, x0)); ys.append(np.arange(H))
        xy = np.stack([np.concatenate(xs), np.concatenate(ys)], 1).astype(np.int32)
        Do, Vo = ora.subtract_at(xy, I32, V32, R, Vr, fl, K32.astype(np.float64), bgo, sdeg=sdeg, bgdeg=bgdeg)
        Kabs = np.abs(K32.astype(np.float64)).sum(0, keepdims=True)
        Cn, _ = ora.subtract_at(xy, np.zeros_like(I32), V32, np.abs(R), Vr, fl, Kabs, [0.0], sdeg=0, bgdeg=0)
        Dg = D2[:, :W].cpu().numpy()[xy[:, 1], xy[:, 0]]
        Vg = VD2[:, :W].cpu().numpy()[xy[:, 1], xy[:, 0]]
        zero = (Do == 0) & (Vo == 0)
        np.testing.assert_array_equal(Dg[zero], 0.0)
        np.testing.assert_array_equal(Vg[zero], 0.0)
        scale = np.maximum(np.maximum(np.abs(I32[xy[:, 1], xy[:, 0]]), -Cn), 1.0)
        assert assert_rel(Dg, Do, scale, 1e-4, "D") < 1e-5
        # V_D: the exact per-pixel definition, within FP32 arithmetic plus the tile rule's
        # allowance at every sampled pixel, and within the detection-margin bar overall
        ev = assert_variance(Vg, Vo, tile_rule_allowance(K32, sdeg, Vr, xy, (W, H)))
        print(f"[full frame] V_D worst |dV| / V_D {ev:.2e}")
        assert ev <= VD_RTOL
        del D2, VD2

        # --- detection on the pipeline's own difference image
        D, VD, mask = (t[:, :W].cpu().numpy() for t in (pipe.diff, pipe.diff_var, pipe.mask))
        src, nf = pipe.sources_host()
        assert nf <= pipe.src_cap and nf > 0
        n_p, n_n = check_detection_properties(D, VD, g_fl, mask, src, nf, pipe.nsigma)
        print(f"[full frame] sources {nf} (+{n_p} / -{n_n})")
        del D, VD, mask

        # --- the one-call path the benchmark captures (argus_dia_frame): bit for bit the separate
        # calls' outputs
        fused = FramePipeline(W, H, basis=basis, stamp=bench.STAMP, grid=bench.GRID, precision="tf32",
                              psf_sigma=1.8, device=0)
        try:
            pipe.precision = "tf32"
            pipe.run(pad(torch.from_numpy(raw).to(device)), calib, dR, dVr)
            fused.run_fused(pad(torch.from_numpy(raw).to(device)), calib, dR, dVr)
            torch.cuda.synchronize()
            assert fused.status() == 0
            for name in ("coeffs", "diff", "diff_var", "mask"):
                assert torch.equal(getattr(pipe, name), getattr(fused, name)), name
            s1, n1 = pipe.sources_host()
            s2, n2 = fused.sources_host()
            assert n1 == n2 and s1.tobytes() == s2.tobytes()
        finally:
            fused.close()
    finally:
        pipe.close()
