"""Pins of the proper-image oracle (ZOGY subtraction, Sec. 4.2; proper
coaddition, Sec. 4.1.3) against closed forms, textbook special cases, brute
force and noise statistics -- never against its own formulas.  CPU only."""
import math

import numpy as np
import pytest

from oracle import proper


def _gauss(sig, half=None, dx=0.0, dy=0.0):
    half = half or int(math.ceil(6 * sig))
    u = np.arange(-half, half + 1)
    g = np.exp(-((u[None, :] - dx) ** 2 + (u[:, None] - dy) ** 2) / (2 * sig * sig))
    return g / g.sum()


def _delta():
    return np.ones((1, 1))


def _source(shape, psf, q, flux):
    """flux * psf centred on pixel q of a periodic tile (no FFT)."""
    h, w = shape
    ph, pw = psf.shape
    img = np.zeros(shape)
    for j in range(ph):
        for i in range(pw):
            img[(q[1] + j - ph // 2) % h, (q[0] + i - pw // 2) % w] += flux * psf[j, i]
    return img


# --------------------------------------------------------------------------- ZOGY
def test_zogy_delta_psfs_give_the_weighted_difference():
    """P_n = P_r = delta: D = (F_r N - F_n R) / sqrt(s_n^2 F_r^2 + s_r^2 F_n^2), plain
    image arithmetic; P_D = delta; S = F_D D."""
    rng = np.random.default_rng(1)
    N = rng.normal(0, 3, (24, 20))
    R = rng.normal(0, 1, (24, 20))
    Fn, Fr, sn, sr = 0.8, 1.3, 3.0, 1.0
    out = proper.zogy(N, R, _delta(), _delta(), Fn, Fr, sn, sr)
    den = math.sqrt(sn * sn * Fr * Fr + sr * sr * Fn * Fn)
    np.testing.assert_allclose(out["D"], (Fr * N - Fn * R) / den, rtol=0, atol=1e-12)
    assert out["F_D"] == pytest.approx(Fr * Fn / den, rel=1e-15)
    pd = np.zeros((24, 20)); pd[0, 0] = 1.0
    np.testing.assert_allclose(out["P_D"], pd, atol=1e-14)
    np.testing.assert_allclose(out["S"], out["F_D"] * out["D"], atol=1e-12)


def test_zogy_static_scene_cancels_and_transient_is_its_psf():
    """N = F_n P_n (x) (T + a delta_q), R = F_r P_r (x) T with different PSFs:
    D = a F_D P_D(x - q) and the static scene T leaves nothing."""
    shape = (64, 48)
    rng = np.random.default_rng(2)
    Pn, Pr = _gauss(2.1, dx=0.4, dy=-0.3), _gauss(1.2, dx=-0.2)     # asymmetric: a conj slip shows
    Fn, Fr, sn, sr = 1.1, 0.9, 5.0, 2.0
    T = [(int(rng.integers(0, 48)), int(rng.integers(0, 64)), float(rng.uniform(50, 500))) for _ in range(30)]
    N = sum(_source(shape, Pn, (x, y), Fn * f) for x, y, f in T)
    R = sum(_source(shape, Pr, (x, y), Fr * f) for x, y, f in T)
    q, a = (17, 40), 250.0
    N = N + _source(shape, Pn, q, Fn * a)
    out = proper.zogy(N, R, Pn, Pr, Fn, Fr, sn, sr)
    expect = a * out["F_D"] * np.roll(out["P_D"], (q[1], q[0]), axis=(0, 1))
    np.testing.assert_allclose(out["D"], expect, rtol=0, atol=1e-9 * a * out["F_D"])
    assert out["P_D"].sum() == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("sn,sr", [(4.0, 0.0), (0.0, 3.0), (4.0, 3.0)])
def test_zogy_detection_snr_textbook_limits(sn, sr):
    """S(q)/sigma_S for a transient of flux a: with a noiseless reference it is the
    matched-filter S/N of the new image alone, a F_n ||P_n|| / s_n; with a noiseless
    new image it is the reference's a F_r ||P_r|| / s_r (the difference flux is only
    as well known as the reference flux); with equal PSFs the inverse squares add."""
    shape = (64, 64)
    Fn, Fr, a, q = 1.2, 0.7, 100.0, (30, 21)
    if sn and sr:
        Pn = Pr = _gauss(1.7)
    else:
        Pn, Pr = _gauss(1.9), _gauss(1.3)
    N = _source(shape, Pn, q, Fn * a)
    out = proper.zogy(N, np.zeros(shape), Pn, Pr, Fn, Fr, sn, sr)
    snr = out["S"][q[1], q[0]] / out["sigma_S"]
    assert np.unravel_index(np.argmax(out["S"]), shape) == (q[1], q[0])
    nn, nr = np.sqrt((Pn ** 2).sum()), np.sqrt((Pr ** 2).sum())
    if sr == 0:
        ref = a * Fn * nn / sn
    elif sn == 0:
        ref = a * Fr * nr / sr
    else:
        ref = 1.0 / math.sqrt((sn / (a * Fn * nn)) ** 2 + (sr / (a * Fr * nr)) ** 2)
    assert snr == pytest.approx(ref, rel=1e-9)


def test_zogy_score_is_the_direct_correlation_of_d_with_its_psf():
    """S(x) = F_D sum_u P_D(u) D(x + u), cyclic, by brute-force loops (asymmetric PSFs)."""
    rng = np.random.default_rng(10)
    h, w = 12, 10
    N, R = rng.normal(0, 2, (h, w)), rng.normal(0, 1, (h, w))
    out = proper.zogy(N, R, _gauss(1.1, 4, dx=0.5), _gauss(0.8, 3, dy=0.4), 1.0, 1.2, 2.0, 1.0)
    D, PD = out["D"], out["P_D"]
    S = np.zeros((h, w))
    for y in range(h):
        for x in range(w):
            S[y, x] = out["F_D"] * sum(PD[j, i] * D[(y + j) % h, (x + i) % w] for j in range(h) for i in range(w))
    np.testing.assert_allclose(out["S"], S, atol=1e-12)


def test_zogy_noise_is_white_with_unit_variance():
    """Pure background noise with different PSFs: D has per-pixel variance 1 and a
    flat power spectrum; S has standard deviation sigma_S."""
    shape = (256, 256)
    rng = np.random.default_rng(3)
    sn, sr = 7.0, 2.5
    N = rng.normal(0, sn, shape)
    R = rng.normal(0, sr, shape)
    out = proper.zogy(N, R, _gauss(2.4), _gauss(1.1), 1.0, 1.4, sn, sr)
    assert out["D"].var() == pytest.approx(1.0, abs=0.03)
    p = np.abs(np.fft.fft2(out["D"])) ** 2 / out["D"].size
    k = np.hypot(*np.meshgrid(np.fft.fftfreq(256), np.fft.fftfreq(256)))
    assert p[(k > 0.02) & (k < 0.15)].mean() == pytest.approx(1.0, abs=0.05)
    assert p[k > 0.35].mean() == pytest.approx(1.0, abs=0.05)
    assert out["S"].std() == pytest.approx(out["sigma_S"], rel=0.05)


def test_zogy_frequencies_below_the_floor_carry_nothing():
    """Wide PSFs on a 256^2 tile: where both PSF transforms are below eps the
    difference has no power; elsewhere its noise stays white with unit variance,
    so the per-pixel variance is the kept fraction of the frequencies."""
    shape = (256, 256)
    rng = np.random.default_rng(11)
    sn, sr = 5.0, 2.0
    Pn, Pr = _gauss(3.2), _gauss(2.8)
    out = proper.zogy(rng.normal(0, sn, shape), rng.normal(0, sr, shape), Pn, Pr, 1.0, 1.0, sn, sr)
    big = np.maximum(np.abs(np.fft.fft2(proper.psf_on_tile(Pn, shape))),
                     np.abs(np.fft.fft2(proper.psf_on_tile(Pr, shape)))) >= 1e-8
    kept = big.mean()
    assert 0.2 < kept < 0.9
    Dh = np.fft.fft2(out["D"])
    assert np.abs(Dh[~big]).max() < 1e-9 * np.abs(Dh).max()
    assert np.abs(np.fft.fft2(out["P_D"])[~big]).max() < 1e-12
    assert out["D"].var() == pytest.approx(kept, abs=0.03)


def test_zogy_swapping_images_negates_the_difference():
    rng = np.random.default_rng(4)
    N, R = rng.normal(0, 2, (32, 40)), rng.normal(0, 1, (32, 40))
    a = proper.zogy(N, R, _gauss(1.8), _gauss(1.0), 1.1, 0.8, 2.0, 1.0)
    b = proper.zogy(R, N, _gauss(1.0), _gauss(1.8), 0.8, 1.1, 1.0, 2.0)
    np.testing.assert_allclose(b["D"], -a["D"], atol=1e-12)
    np.testing.assert_allclose(b["P_D"], a["P_D"], atol=1e-14)
    assert b["F_D"] == pytest.approx(a["F_D"], rel=1e-15)


def test_zogy_cyclic_shift_equivariance():
    rng = np.random.default_rng(5)
    N, R = rng.normal(0, 2, (32, 40)), rng.normal(0, 1, (32, 40))
    a = proper.zogy(N, R, _gauss(1.5), _gauss(1.2), 1.0, 1.0, 2.0, 1.0)
    b = proper.zogy(np.roll(N, (5, -7), (0, 1)), np.roll(R, (5, -7), (0, 1)), _gauss(1.5), _gauss(1.2),
                    1.0, 1.0, 2.0, 1.0)
    np.testing.assert_allclose(b["D"], np.roll(a["D"], (5, -7), (0, 1)), atol=1e-12)


# --------------------------------------------------------------------------- proper coadd
def test_coadd_delta_psfs_give_the_inverse_variance_combination():
    """Delta PSFs: S = sum F_j M_j / s_j^2 and R = S / sqrt(sum F_j^2 / s_j^2)."""
    rng = np.random.default_rng(6)
    M = [rng.normal(0, s, (20, 28)) for s in (1.0, 2.0, 0.5)]
    F, sig = [1.0, 0.7, 1.3], [1.0, 2.0, 0.5]
    out = proper.proper_coadd(M, [_delta()] * 3, F, sig)
    S = sum(f / (s * s) * m for m, f, s in zip(M, F, sig))
    FR = math.sqrt(sum(f * f / (s * s) for f, s in zip(F, sig)))
    np.testing.assert_allclose(out["S"], S, atol=1e-12)
    np.testing.assert_allclose(out["R"], S / FR, atol=1e-12)
    assert out["F_R"] == pytest.approx(FR, rel=1e-15)


@pytest.mark.parametrize("psf_sigma", [1.0, 1.3])
def test_coadd_single_image_is_itself_in_noise_units(psf_sigma):
    """One image with a centred Gaussian PSF (positive real transform): R = M / s,
    P_R = P, F_R = F / s.  (Wider PSFs make the transform ~1e-11 at the corner
    frequencies, where the FFT's own rounding sets the phase: the identity then
    holds only to ~1e-9.)"""
    rng = np.random.default_rng(7)
    M = rng.normal(0, 3, (40, 36))
    P = _gauss(psf_sigma)
    out = proper.proper_coadd([M], [P], [0.9], [3.0])
    np.testing.assert_allclose(out["R"], M / 3.0, atol=1e-12)
    np.testing.assert_allclose(out["P_R"], proper.psf_on_tile(P, M.shape), atol=1e-12)
    assert out["F_R"] == pytest.approx(0.3, rel=1e-15)


def test_coadd_score_is_the_direct_correlation_sum():
    """S(x) = sum_j F_j / s_j^2 sum_u P_j(u) M_j(x + u), cyclic, by brute-force loops."""
    rng = np.random.default_rng(8)
    h, w = 14, 11
    M = [rng.normal(0, 1, (h, w)) for _ in range(2)]
    P = [rng.uniform(0, 1, (5, 5)), rng.uniform(0, 1, (3, 7))]
    P = [p / p.sum() for p in P]
    F, sig = [1.2, 0.6], [1.5, 0.8]
    out = proper.proper_coadd(M, P, F, sig)
    S = np.zeros((h, w))
    for m, p, f, s in zip(M, P, F, sig):
        ph, pw = p.shape
        for y in range(h):
            for x in range(w):
                acc = 0.0
                for j in range(ph):
                    for i in range(pw):
                        acc += p[j, i] * m[(y + j - ph // 2) % h, (x + i - pw // 2) % w]
                S[y, x] += f / (s * s) * acc
    np.testing.assert_allclose(out["S"], S, atol=1e-12)


def test_coadd_point_source_psf_and_snr_add_in_quadrature():
    """Noiseless source of flux a in every frame (different PSFs): R = a F_R P_R(x - q)
    and S(q) / sigma_S = sqrt(sum_j (a F_j ||P_j|| / s_j)^2)."""
    shape = (64, 64)
    q, a = (9, 50), 40.0
    P = [_gauss(s) for s in (1.1, 1.8, 2.6)]
    F, sig = [1.0, 0.8, 1.2], [1.0, 1.5, 2.0]
    M = [_source(shape, p, q, f * a) for p, f in zip(P, F)]
    out = proper.proper_coadd(M, P, F, sig)
    np.testing.assert_allclose(out["R"], a * out["F_R"] * np.roll(out["P_R"], (q[1], q[0]), (0, 1)),
                               atol=1e-10 * a * out["F_R"])
    snr = out["S"][q[1], q[0]] / out["sigma_S"]
    ref = math.sqrt(sum((a * f * np.sqrt((p ** 2).sum()) / s) ** 2 for p, f, s in zip(P, F, sig)))
    # sigma_S is the noise of S; the signal in S at q is a sum_j F_j^2 ||P_j||^2 / s_j^2
    assert snr == pytest.approx(ref, rel=1e-9)


def test_coadd_noise_is_white_with_unit_variance():
    rng = np.random.default_rng(9)
    sig = [1.0, 3.0, 2.0, 0.7]
    M = [rng.normal(0, s, (192, 192)) for s in sig]
    out = proper.proper_coadd(M, [_gauss(s) for s in (1.2, 2.2, 1.6, 2.9)], [1.0, 0.9, 1.1, 1.3], sig)
    assert out["R"].var() == pytest.approx(1.0, abs=0.03)
    assert out["S"].std() == pytest.approx(out["sigma_S"], rel=0.05)


def test_coadd_depth_gain_of_thirty_frames():
    """Sec. 4.1.3: 30 x 30-s frames reach m_g = 19.8 against 17.8 for one frame.  Equal
    frames gain sqrt(30) in S/N, 2.5 log10 sqrt(30) = 1.85 mag, within 0.2 mag of the
    2.0 mag the paper quotes (its figures include the sky and seeing of its site)."""
    shape = (48, 48)
    P, q, a = _gauss(1.8), (20, 30), 10.0
    one = proper.proper_coadd([_source(shape, P, q, a)], [P], [1.0], [4.0])
    many = proper.proper_coadd([_source(shape, P, q, a)] * 30, [P] * 30, [1.0] * 30, [4.0] * 30)
    s1 = one["S"][q[1], q[0]] / one["sigma_S"]
    s30 = many["S"][q[1], q[0]] / many["sigma_S"]
    assert s30 / s1 == pytest.approx(math.sqrt(30), rel=1e-12)
    assert abs(2.5 * math.log10(s30 / s1) - (19.8 - 17.8)) < 0.2
