"""FP64 oracle of the proper-image statistics named by the paper (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU legs may import this
module; the product library never calls it.  numpy's FFT is the one library
primitive used; everything else is the definition written out.

* ZOGY subtraction (Sec. 4.2 "Transient Alerts": ZOGY at base cadence and in
  deep coadds; Zackay, Ofek & Gal-Yam 2016): the proper difference image D,
  its PSF P_D and flux zero point F_D, and the point-source score S.
* Proper coaddition (Sec. 4.1.3 "Deep Coaddition in Sky Segments": a per-image
  matched filter; Zackay & Ofek 2017): the score coadd S, the proper coadd R,
  its PSF P_R and flux zero point F_R.

Conventions (readings of the method, shared by the GPU path):
- images are background-subtracted, registered tiles with background-
  dominated white noise of standard deviation sigma (a scalar per image);
- a tile is periodic: every convolution is the cyclic one the DFT defines;
- a PSF is a small odd-sized stamp, centred, with unit sum; it is placed on
  the tile with its centre at pixel (0, 0) (wrapping around);
- a zero point F scales the PSF: a source of flux a appears as a F P(x - q);
- transforms are numpy's unnormalised forward FFT and its inverse, so a
  unit-sum PSF has P_hat(0) = 1 and white noise of per-pixel variance v has
  E|eps_hat(k)|^2 = v * npix;
- a frequency where every PSF transform has modulus below eps (default 1e-8;
  the PSFs have unit sum, so |P(0)| = 1) carries no proper statistic: D,
  P_D and the ZOGY score S, and the proper coadd R and its PSF P_R, are 0
  there (the score coadd, a plain correlation, keeps every frequency).  Below that floor the transforms of sampled PSFs are
  set by the FFT's own rounding (about 1e-16 in FP64, 1e-7 in FP32), so the
  quotient is not a property of the inputs; the floor makes it one.
"""
from __future__ import annotations

import numpy as np


def psf_on_tile(psf, shape):
    """Place an odd-sized centred PSF stamp on a tile of `shape` with its centre
    at (0, 0), wrapping around (the cyclic convolution kernel of the tile)."""
    psf = np.asarray(psf, np.float64)
    ph, pw = psf.shape
    if ph % 2 == 0 or pw % 2 == 0 or ph > shape[0] or pw > shape[1]:
        raise ValueError("PSF stamp must be odd-sized and fit in the tile")
    t = np.zeros(shape)
    t[:ph, :pw] = psf
    return np.roll(t, (-(ph // 2), -(pw // 2)), axis=(0, 1))


def _safe_div(num, den):
    out = np.zeros(np.broadcast(num, den).shape, dtype=np.result_type(num, den))
    nz = den != 0
    np.divide(num, den, out=out, where=nz)
    return out


def zogy(N, R, Pn, Pr, Fn, Fr, sn, sr, eps=1e-8):
    """Proper image subtraction of a new image N against a reference R.

    With hats for DFTs and the PSFs placed on the tile:
      den(k) = sqrt(sn^2 Fr^2 |Pr(k)|^2 + sr^2 Fn^2 |Pn(k)|^2)
      D      = IDFT[(Fr Pr N - Fn Pn R) / den]     (unit-variance white noise)
      F_D    = Fr Fn / sqrt(sn^2 Fr^2 + sr^2 Fn^2)
      P_D    = IDFT[Fr Fn Pr Pn / (F_D den)]        (unit sum)
      S      = IDFT[F_D D conj(P_D)]               (matched filter of D with its PSF)
      sigma_S = F_D sqrt(sum P_D^2)                (per-pixel standard deviation of S)
    A source of flux a at q in N alone gives D = a F_D P_D(x - q) and
    S(q) / sigma_S = a F_D ||P_D||_2, the optimal detection S/N.
    Returns a dict of float64 arrays / scalars: D, P_D, F_D, S, sigma_S.
    """
    N = np.asarray(N, np.float64)
    R = np.asarray(R, np.float64)
    shape = N.shape
    Pn_h = np.fft.fft2(psf_on_tile(Pn, shape))
    Pr_h = np.fft.fft2(psf_on_tile(Pr, shape))
    N_h = np.fft.fft2(N)
    R_h = np.fft.fft2(R)
    den = np.sqrt(sn * sn * Fr * Fr * np.abs(Pr_h) ** 2 + sr * sr * Fn * Fn * np.abs(Pn_h) ** 2)
    den[np.maximum(np.abs(Pn_h), np.abs(Pr_h)) < eps] = 0.0          # no statistic below the floor
    D_h = _safe_div(Fr * Pr_h * N_h - Fn * Pn_h * R_h, den)
    F_D = Fr * Fn / np.sqrt(sn * sn * Fr * Fr + sr * sr * Fn * Fn)
    PD_h = _safe_div(Fr * Fn * Pr_h * Pn_h, F_D * den)
    D = np.fft.ifft2(D_h).real
    P_D = np.fft.ifft2(PD_h).real
    S = np.fft.ifft2(F_D * D_h * np.conj(PD_h)).real
    sigma_S = F_D * np.sqrt(np.sum(P_D * P_D))
    return {"D": D, "P_D": P_D, "F_D": F_D, "S": S, "sigma_S": sigma_S}


def proper_coadd(images, psfs, F, sigma, eps=1e-8):
    """Proper coaddition of registered images M_j with PSFs P_j, zero points F_j
    and background noise sigma_j.

      S       = IDFT[sum_j (F_j / sigma_j^2) conj(P_j) M_j]      (score coadd)
      den(k)  = sqrt(sum_j F_j^2 / sigma_j^2 |P_j(k)|^2)
      R       = IDFT[DFT(S) / den]                               (unit-variance white noise)
      F_R     = sqrt(sum_j F_j^2 / sigma_j^2)
      P_R     = IDFT[den / F_R]                                  (unit sum)
      sigma_S = sqrt(sum_j F_j^2 / sigma_j^2 sum P_j^2)           (per-pixel standard deviation of S)
    A noiseless source of flux a at q gives R = a F_R P_R(x - q); its S/N in
    S is sqrt(sum_j a^2 F_j^2 ||P_j||^2 / sigma_j^2).
    Returns a dict: S, R, F_R, P_R, sigma_S.
    """
    images = [np.asarray(m, np.float64) for m in images]
    shape = images[0].shape
    S_h = np.zeros(shape, np.complex128)
    den2 = np.zeros(shape)
    pmax = np.zeros(shape)
    varS = 0.0
    for M, P, f, s in zip(images, psfs, F, sigma):
        P_t = psf_on_tile(P, shape)
        P_h = np.fft.fft2(P_t)
        S_h += (f / (s * s)) * np.conj(P_h) * np.fft.fft2(M)
        den2 += (f * f) / (s * s) * np.abs(P_h) ** 2
        pmax = np.maximum(pmax, np.abs(P_h))
        varS += (f * f) / (s * s) * np.sum(P_t * P_t)
    den = np.sqrt(den2)
    den[pmax < eps] = 0.0                                             # no statistic below the floor
    F_R = float(np.sqrt(sum((f * f) / (s * s) for f, s in zip(F, sigma))))
    return {"S": np.fft.ifft2(S_h).real, "R": np.fft.ifft2(_safe_div(S_h, den)).real, "F_R": F_R,
            "P_R": np.fft.ifft2(den / F_R).real, "sigma_S": float(np.sqrt(varS))}
