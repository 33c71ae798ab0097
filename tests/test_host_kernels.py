"""The kernels' own arithmetic on the CPU: the FFT butterflies and Stockham
passes (csrc/fft.cuh) and the per-frequency steps of ZOGY and the proper
coadd (csrc/proper.cu) are host-callable; small drivers (tests/host_drivers)
compiled by nvcc as host code run them thread by thread with the kernels'
load/store mapping, against numpy's FFT and the FP64 proper-image oracle
(ZOGY, Sec. 4.2; proper coadd, Sec. 4.1.3); the background-map kernels'
per-thread code (box medians by radix select, mesh filter, bilinear map;
Table 2) and the HEALPix resampler's per-pixel code (Sec. 3.3) likewise
against their oracles.  Needs nvcc, no GPU."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2207_14304_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
DRV = os.path.join(ROOT, "tests", "host_drivers")
F32 = 2.0 ** -24
TILE_DTYPE = [("x0", "<i4"), ("y0", "<i4"), ("Fn", "<f4"), ("Fr", "<f4"), ("sn", "<f4"), ("sr", "<f4")]


@pytest.fixture(scope="module")
def drivers(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("host_drivers")
    for name in ("host_fft", "host_zogy", "host_coadd", "host_background", "host_healpix", "host_segscale"):
        subprocess.check_call([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-I", CSRC, "-I", INCLUDE, "-I", DRV, "-o", str(d / name),
                               os.path.join(DRV, name + ".cu")])
    return d


@pytest.mark.parametrize("T", [256, 512])
@pytest.mark.parametrize("dbl", [0, 1])
def test_fft_passes_match_numpy(drivers, T, dbl):
    rng = np.random.default_rng(T + dbl)
    dt = np.complex128 if dbl else np.complex64
    x = (rng.normal(size=(2, T, T)) + 1j * rng.normal(size=(2, T, T))).astype(dt)
    x.tofile(drivers / "in.bin")
    for sign in (-1, 1):
        subprocess.check_call([str(drivers / "host_fft"), str(T), str(dbl), "2", str(sign),
                               str(drivers / "in.bin"), str(drivers / "out.bin")])
        y = np.fromfile(drivers / "out.bin", dtype=dt).reshape(2, T, T)
        x64 = x.astype(np.complex128)
        ref = np.fft.fft2(x64) if sign < 0 else np.fft.ifft2(x64) * T * T
        err = np.abs(y - ref).max() / np.abs(ref).max()
        # FP32: a few ulps times log2(T^2); FP64 the same in double
        assert err < 8 * (2.0 ** -53 if dbl else F32) * math.log2(T * T), (sign, err)


def _gauss(sig, half=15):
    u = np.arange(-half, half + 1)
    g = np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2 * sig * sig))
    return (g / g.sum()).astype(np.float32)


@pytest.mark.parametrize("T,spec", [(256, (1.05, 1.0, 18.0, 3.3, 2.0, 1.2)), (256, (0.9, 1.1, 10.0, 4.0, 1.3, 1.6)),
                                    (256, (1.0, 1.0, 5.0, 0.0, 1.5, 1.5)), (256, (1.0, 1.0, 4.0, 2.0, 3.5, 3.0)),
                                    (512, (1.0, 1.0, 12.0, 3.0, 1.8, 1.3))])
def test_zogy_step_matches_the_oracle(drivers, T, spec):
    """D within 8 e, S within 8 e F_D ||P_D||_1, P_D within 64 ulps of its maximum,
    sigma_S within 1e-6 (the bars of the GPU test; e is its FP32 error unit).
    Includes a noiseless reference and PSFs wide enough for the frequency floor."""
    from oracle import proper
    Fn, Fr, sn, sr, gn, gr = spec
    rng = np.random.default_rng(T + int(10 * gn))
    pn, pr = _gauss(gn), _gauss(gr)
    sky = np.zeros((T, T))
    n = T * T // 130
    np.add.at(sky, (rng.integers(0, T, n), rng.integers(0, T, n)), 1e2 * 1e4 ** rng.random(n))
    conv = lambda img, P: np.fft.ifft2(np.fft.fft2(img) * np.fft.fft2(proper.psf_on_tile(P, img.shape))).real
    N = (Fn * conv(sky, pn) + rng.normal(0, max(sn, 1.0), (T, T))).astype(np.float32)
    R = (Fr * conv(sky, pr) + rng.normal(0, max(sr, 0.5), (T, T))).astype(np.float32)
    d = drivers / f"zogy_{T}_{gn}_{sr}"
    d.mkdir(exist_ok=True)
    np.array([31, 0], np.int32).tofile(d / "hdr.bin")
    rec = np.zeros(1, TILE_DTYPE)
    rec[0] = (0, 0, Fn, Fr, sn, sr)
    rec.tofile(d / "tile.bin")
    for name, a in (("N", N), ("R", R), ("pn", pn), ("pr", pr)):
        a.tofile(d / f"{name}.bin")
    subprocess.check_call([str(drivers / "host_zogy"), str(T), str(d)])
    D = np.fromfile(d / "D.bin", np.float32).reshape(T, T)
    S = np.fromfile(d / "S.bin", np.float32).reshape(T, T)
    P = np.fromfile(d / "P.bin", np.float32).reshape(T, T)
    sig = np.fromfile(d / "sig.bin", np.float64)[0]
    f = lambda v: float(np.float32(v))
    o = proper.zogy(N, R, pn.astype(np.float64), pr.astype(np.float64), f(Fn), f(Fr), f(sn), f(sr))
    e = F32 * math.log2(T * T) * (np.linalg.norm(N) / sn + (np.linalg.norm(R) / sr if sr > 0 else 0.0)) / T
    sS = e * o["F_D"] * np.abs(o["P_D"]).sum()
    print(f"\n[zogy T={T}] |dD| = {np.abs(D - o['D']).max() / e:.2f} e  |dS| = {np.abs(S - o['S']).max() / sS:.2f} e_S")
    assert np.abs(D - o["D"]).max() <= 8 * e
    assert np.abs(S - o["S"]).max() <= 8 * sS
    assert np.abs(P - o["P_D"]).max() <= 64 * F32 * np.abs(o["P_D"]).max()
    assert abs(sig / o["sigma_S"] - 1) < 1e-6


def test_zogy_psf_reuse_rule(drivers):
    """A ZOGY call without PSFs reuses what the plan holds: per-tile pairs for at least as many
    tiles (held >= n_tiles >= 1), or the one shared pair (held = -1).  A shared pair never serves
    a per-tile call, and an empty plan (held = 0) serves nothing."""
    out = subprocess.check_output([str(drivers / "host_zogy"), "reuse"]).decode().split("\n")
    seen = 0
    for line in filter(None, out):
        held, per, n, ok = map(int, line.split())
        want = (held >= n) if per else (held == -1)
        assert ok == int(want), (held, per, n, ok)
        seen += 1
    assert seen == 5 * 2 * 4


@pytest.mark.parametrize("T,J,eps_psf", [(256, 3, False), (256, 4, True), (512, 2, False)])
def test_proper_coadd_step_matches_the_oracle(drivers, T, J, eps_psf):
    """R within 8 e_R, e_R = u log2(T^2) sum_j ||M_j||_2 / s_j / T (the quotient's gain is at
    most 1/s_j per frame); S within 8 e_S, e_S = u log2(T^2) (sum_j F_j/s_j^2 ||P_j||_1 ||M_j||_2
    + ||R||_2) / T (the last term: S and R share one inverse transform);
    P_R within 64 ulps of its maximum; F_R and sigma_S within 1e-6.  An odd frame count
    exercises the unpaired last frame; eps_psf adds wide PSFs so the frequency floor acts."""
    from oracle import proper
    rng = np.random.default_rng(T + J)
    sky = np.zeros((T, T))
    n = T * T // 150
    np.add.at(sky, (rng.integers(0, T, n), rng.integers(0, T, n)), 1e2 * 1e4 ** rng.random(n))
    conv = lambda img, P: np.fft.ifft2(np.fft.fft2(img) * np.fft.fft2(proper.psf_on_tile(P, img.shape))).real
    sig_psf = [1.2, 1.9, 1.5, 2.4][:J] if not eps_psf else [3.4, 3.8, 1.3, 3.1][:J]
    Ps = [_gauss(g) for g in sig_psf]
    F = np.array([1.0, 0.8, 1.2, 0.95][:J], np.float32)
    sg = np.array([5.0, 9.0, 4.0, 6.0][:J], np.float32)
    Ms = [(f * conv(sky, P) + rng.normal(0, s, (T, T))).astype(np.float32) for P, f, s in zip(Ps, F, sg)]
    d = drivers / f"coadd_{T}_{J}_{int(eps_psf)}"
    d.mkdir(exist_ok=True)
    np.array([J, 31], np.int32).tofile(d / "hdr.bin")
    np.stack(Ms).tofile(d / "M.bin")
    np.stack(Ps).tofile(d / "P.bin")
    F.tofile(d / "F.bin")
    sg.tofile(d / "sig.bin")
    subprocess.check_call([str(drivers / "host_coadd"), str(T), str(d)])
    S = np.fromfile(d / "S.bin", np.float32).reshape(T, T)
    R = np.fromfile(d / "R.bin", np.float32).reshape(T, T)
    PR = np.fromfile(d / "PR.bin", np.float32).reshape(T, T)
    FR, sigS = np.fromfile(d / "norms.bin", np.float64)
    o = proper.proper_coadd(Ms, [P.astype(np.float64) for P in Ps], [float(f) for f in F], [float(s) for s in sg])
    lg = F32 * math.log2(T * T) / T
    eR = lg * sum(np.linalg.norm(M) / s for M, s in zip(Ms, sg))
    # S shares the inverse transform with R, whose rounding (about ||R||_2 / T) it also carries
    eS = lg * (sum(f / s ** 2 * np.abs(P).sum() * np.linalg.norm(M) for M, P, f, s in zip(Ms, Ps, F, sg))
               + np.linalg.norm(o["R"]))
    print(f"\n[coadd T={T} J={J}] |dR| = {np.abs(R - o['R']).max() / eR:.2f} e_R  |dS| = "
          f"{np.abs(S - o['S']).max() / eS:.2f} e_S")
    assert np.abs(R - o["R"]).max() <= 8 * eR
    assert np.abs(S - o["S"]).max() <= 8 * eS
    assert np.abs(PR - o["P_R"]).max() <= 64 * F32 * np.abs(o["P_R"]).max()
    assert abs(FR / o["F_R"] - 1) < 1e-6 and abs(sigS / o["sigma_S"] - 1) < 1e-6


@pytest.mark.parametrize("w,h,box,filt,frac,use_flags", [
    (640, 384, 64, 3, 0.5, True), (1000, 37, 64, 3, 0.5, True), (517, 300, 32, 5, 0.5, True),
    (130, 129, 9, 1, 0.5, True), (64, 64, 64, 3, 0.5, False), (8, 8, 8, 7, 0.5, True), (400, 300, 32, 3, 0.99, False),
    (400, 300, 32, 3, 0.5, "left")])
def test_background_steps_match_the_oracle(drivers, w, h, box, filt, frac, use_flags):
    """Box medians and the filtered mesh bit-exact, the FP32 map within 8 ulps of the
    largest mesh value ("left": the left 150 columns flagged, so boxes without a value
    take the filter's neighbours or the fill)."""
    from oracle import background as bgo
    rng = np.random.default_rng(w + h + box)
    y, x = np.mgrid[0:h, 0:w]
    img = (300 + 0.01 * x - 0.02 * y + rng.normal(0, 15, (h, w))).astype(np.float32)
    for _ in range(w * h // 500):
        cy, cx = rng.integers(0, h), rng.integers(0, w)
        img[max(0, cy - 2):cy + 3, max(0, cx - 2):cx + 3] += rng.uniform(100, 3e4)
    img.flat[3::997] = np.nan
    img.flat[5::1999] = np.inf
    img.flat[7::1499] = -0.0
    fl = (rng.random((h, w)) < 0.02).astype(np.uint8)
    if use_flags == "left":
        fl[:] = 0
        fl[:, :150] = 1
    elif not use_flags:
        fl[:] = 0
    d = drivers / f"bg_{w}_{h}_{box}_{filt}_{frac}_{use_flags}"
    d.mkdir(exist_ok=True)
    np.array([w, h, box, filt, 1 if use_flags else 0], np.int32).tofile(d / "hdr.bin")
    np.array([frac], np.float32).tofile(d / "frac.bin")
    img.tofile(d / "img.bin")
    fl.tofile(d / "flags.bin")
    subprocess.check_call([str(drivers / "host_background"), str(d)])
    ny, nx = -(-h // box), -(-w // box)
    raw = np.fromfile(d / "raw.bin").reshape(ny, nx)
    mesh = np.fromfile(d / "mesh.bin").reshape(ny, nx)
    m = np.fromfile(d / "map.bin", np.float32).reshape(h, w)
    f = fl if use_flags else None
    np.testing.assert_array_equal(raw, bgo.box_medians(img, f, box, frac))
    omesh, omap = bgo.background_map(img, f, box=box, filt=filt, min_frac=frac)
    np.testing.assert_array_equal(mesh, omesh)
    assert np.abs(m - omap).max() <= 8 * F32 * np.abs(omesh).max()


def _segments_in_view(wcs, w, h, nside_seg, n, rng):
    """n random segments whose centres fall inside the frame (found from the oracle's
    own pixel centres at nside_seg)."""
    from oracle import healpix as hp
    p = np.arange(12 * nside_seg * nside_seg)
    x, y = hp.gnomonic(hp.xyf2vec(*hp.nest2xyf(p, nside_seg)[:2], hp.nest2xyf(p, nside_seg)[2], nside_seg), *wcs)
    ok = np.isfinite(x)
    inside = p[ok & (x > 0) & (y > 0) & (x < w - 1) & (y < h - 1)]
    edge = p[ok & (x > -3) & (x < 0) & (y > 0) & (y < h - 1)]          # centre just off the left edge
    return np.concatenate([rng.choice(inside, size=min(n, inside.size), replace=False), edge[:1]])


@pytest.mark.parametrize("nside_seg,k,delta0,use_flags", [(64, 4, 0.4, True), (32, 5, 1.45, False),
                                                          (128, 3, -0.7, True), (256, 6, 0.3, True),
                                                          (128, 7, -0.5, False), (64, 6, 1.2, True),
                                                          (256, 9, 0.1, False)])
def test_healpix_resampling_matches_the_oracle(drivers, nside_seg, k, delta0, use_flags):
    """Coverage bit-exact and values within 4 ulps of the largest frame value, for segments
    around and across the frame edge (a polar-cap field at delta0 = 1.45 included); k >= 6
    takes the row path (cubic between exact nodes) in the equatorial belt."""
    from oracle import healpix as hp
    rng = np.random.default_rng(nside_seg + k)
    w, h = 700, 500
    scale = 2.0 * math.sqrt(4 * math.pi / (12.0 * (nside_seg << k) ** 2))        # ~2 segment pixels per frame pixel
    wcs = (0.9, delta0, scale, 0.25, (w - 1) / 2 + 0.3, (h - 1) / 2 - 0.2)
    yy, xx = np.mgrid[0:h, 0:w]
    frame = (300 + 0.05 * xx + rng.normal(0, 10, (h, w))).astype(np.float32)
    frame.flat[11::701] = np.nan
    fl = (rng.random((h, w)) < 0.01).astype(np.uint8) if use_flags else np.zeros((h, w), np.uint8)
    segs = _segments_in_view(wcs, w, h, nside_seg, 6, rng).astype(np.int64)
    d = drivers / f"hp_{nside_seg}_{k}_{delta0}"
    d.mkdir(exist_ok=True)
    np.array([w, h, nside_seg, k, segs.size, 1 if use_flags else 0], np.int32).tofile(d / "hdr.bin")
    np.array(wcs, np.float64).tofile(d / "wcs.bin")
    segs.tofile(d / "segs.bin")
    frame.tofile(d / "frame.bin")
    fl.tofile(d / "flags.bin")
    subprocess.check_call([str(drivers / "host_healpix"), str(d)])
    m = 1 << k
    out = np.fromfile(d / "out.bin", np.float32).reshape(-1, m, m)
    cov = np.fromfile(d / "cov.bin", np.uint8).reshape(-1, m, m)
    tol = 4 * F32 * float(np.nanmax(np.abs(frame)))
    for i, s in enumerate(segs):
        o, oc = hp.resample_segment(frame, fl if use_flags else None, int(s), nside_seg, k, wcs)
        np.testing.assert_array_equal(cov[i], oc)
        assert np.abs(out[i] - o).max() <= tol
    assert cov[:-1].any() and cov[-1].any() and not cov[-1].all()     # the edge segment is partly covered


def test_segment_fit_fp16_range_scale(drivers):
    """The batched segment fit scales each segment's reference (and the basis) by the power of
    two that puts its largest |value| in [2^13, 2^14), so that the FP16 hi part can never
    overflow (FP16's largest finite value is 65504) and the lo part keeps 11 more bits; zero,
    infinite or NaN maxima leave the data unscaled; maxima below 2^-50 are scaled by 2^64 at
    most, so that scales and their products stay finite."""
    rng = np.random.default_rng(3)
    m = np.concatenate([10.0 ** rng.uniform(-14, 37, 2000), 2.0 ** np.arange(-40, 120, 1.0),
                        [1.0, 8192.0, 16383.99, 16384.0, 65504.0, 3.0e38, 1e-20, 1e-38, 1e-44,
                         0.0, -0.0, np.inf, np.nan]]).astype(np.float32)
    m.tofile(drivers / "scale_in.bin")
    subprocess.check_call([str(drivers / "host_segscale"), str(drivers / "scale_in.bin"),
                           str(drivers / "scale_out.bin")])
    s = np.fromfile(drivers / "scale_out.bin", dtype=np.float32)
    assert s.shape == m.shape and np.all(np.isfinite(s)) and np.all(s > 0)
    frac, _ = np.frexp(s.astype(np.float64))
    assert np.all(frac == 0.5)                               # powers of two: scaling is exact
    ok = np.isfinite(m) & (m > 0)
    big = ok & (m >= 2.0 ** -50)
    ms = m[big].astype(np.float64) * s[big]
    assert np.all((ms >= 2.0 ** 13) & (ms < 2.0 ** 14)), (m[big][~((ms >= 2 ** 13) & (ms < 2 ** 14))])
    assert np.all(s[ok & (m < 2.0 ** -50)] == 2.0 ** 64)
    assert np.all(s[~ok] == 1.0)
    assert np.all(m[big].astype(np.float64) * s[big] * (1 + 2.0 ** -11) < 65504.0)
