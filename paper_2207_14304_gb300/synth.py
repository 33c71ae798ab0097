"""Seeded synthetic IMX455-like star fields.

This module makes test and benchmark inputs only.  It renders star catalogues
into expected electron counts, draws detector noise and quantises to 16-bit
ADU.  It contains none of the difference-imaging arithmetic (no calibration,
no kernel convolution, no fitting, no clipping, no detection): both the CUDA
path and the CPU oracle receive the arrays made here as plain inputs.

Detector model (paper, Table 1: IMX455, 16-bit data, 1.7 e- read noise):
  expected_e = flat * (sky + stars) + dark
  raw = clamp(round(Poisson(expected_e) / gain + bias + N(0, rn/gain)), 0, 65535)

Star fluxes follow dN/dF proportional to F**index (index -1.5) between
flux_min and flux_max, drawn by the inverse CDF.  Stars are pixel-integrated
circular Gaussians (differences of the normal CDF), so a star's total flux on
an unbounded grid is exact.

Every draw takes an explicit integer seed; catalogues are drawn on the CPU so
that a seed means the same catalogue on every device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

SQRT2 = math.sqrt(2.0)


def _gen(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


@dataclass
class Catalog:
    x: torch.Tensor      # float64 [n], pixel x of the star centre
    y: torch.Tensor      # float64 [n]
    flux: torch.Tensor   # float64 [n], total electrons

    def __len__(self):
        return int(self.x.numel())


def power_law_fluxes(n: int, seed: int, flux_min=1e2, flux_max=1e6, index=-1.5):
    """Inverse-CDF draw of dN/dF ~ F**index on [flux_min, flux_max]."""
    g = _gen(seed)
    u = torch.rand(n, generator=g, dtype=torch.float64)
    e = index + 1.0
    if abs(e) < 1e-12:
        return flux_min * (flux_max / flux_min) ** u
    a, b = flux_min ** e, flux_max ** e
    return (a + u * (b - a)) ** (1.0 / e)


def star_catalog(n: int, w: int, h: int, seed: int, flux_min=1e2, flux_max=1e6,
                 index=-1.5, border=5.0) -> Catalog:
    """Uniform positions over the frame (plus a border) with power-law fluxes."""
    g = _gen(seed * 7919 + 17)
    x = torch.rand(n, generator=g, dtype=torch.float64) * (w + 2 * border) - border
    y = torch.rand(n, generator=g, dtype=torch.float64) * (h + 2 * border) - border
    f = power_law_fluxes(n, seed * 7919 + 29, flux_min, flux_max, index)
    return Catalog(x, y, f)


def _phi(z):
    return 0.5 * (1.0 + torch.erf(z / SQRT2))


def render(cat: Catalog, w: int, h: int, sigma, *, shift=(0.0, 0.0), sky=0.0,
           device="cpu", dtype=torch.float64, half=None, chunk=65536) -> torch.Tensor:
    """Expected electrons per pixel of a star field (no noise).

    sigma: a float, or a callable (x, y) -> sigma per star (float64 tensors).
    shift: the scene is displaced by (sx, sy) pixels (a star at catalogue
      position p lands at p + shift).
    half: footprint half-width in pixels (default ceil(5 * max sigma)).
    """
    dev = torch.device(device)
    img = torch.full((h * w,), float(sky), dtype=dtype, device=dev)
    n = len(cat)
    if n == 0:
        return img.view(h, w)
    xs = cat.x.to(dev) + shift[0]
    ys = cat.y.to(dev) + shift[1]
    fl = cat.flux.to(dev)
    if callable(sigma):
        sg = sigma(xs, ys).to(torch.float64)
    else:
        sg = torch.full_like(xs, float(sigma))
    if half is None:
        half = int(math.ceil(5.0 * float(sg.max())))
    offs = torch.arange(-half, half + 1, device=dev, dtype=torch.float64)
    L = offs.numel()
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        x0 = torch.floor(xs[s:e] + 0.5)
        y0 = torch.floor(ys[s:e] + 0.5)
        px = x0[:, None] + offs[None, :]            # [m, L]
        py = y0[:, None] + offs[None, :]
        sgi = sg[s:e, None]
        fx = _phi((px + 0.5 - xs[s:e, None]) / sgi) - _phi((px - 0.5 - xs[s:e, None]) / sgi)
        fy = _phi((py + 0.5 - ys[s:e, None]) / sgi) - _phi((py - 0.5 - ys[s:e, None]) / sgi)
        val = fl[s:e, None, None] * fy[:, :, None] * fx[:, None, :]   # [m, L(y), L(x)]
        pxi = px.to(torch.int64)
        pyi = py.to(torch.int64)
        okx = (pxi >= 0) & (pxi < w)
        oky = (pyi >= 0) & (pyi < h)
        ok = oky[:, :, None] & okx[:, None, :]
        idx = pyi[:, :, None] * w + pxi[:, None, :]
        img.index_add_(0, idx[ok], val[ok].to(dtype))
    return img.view(h, w)


@dataclass
class Calib:
    """Calibration frames of one camera (paper: darks, flats, bad-pixel masks)."""
    bias: int            # scalar bias in ADU
    dark: torch.Tensor   # float32 [h, w], electrons in the exposure
    flat: torch.Tensor   # float32 [h, w], relative response
    bpm: torch.Tensor    # uint8   [h, w], nonzero = bad pixel
    gain: float          # e- / ADU
    read_noise: float    # e- rms
    sat: int             # raw level treated as saturated


def make_calib(w: int, h: int, seed: int, *, bias=100, gain=1.0, read_noise=1.7,
               dark_level=0.5, hot_frac=1e-4, bad_frac=1e-4, flat_rms=0.01,
               sat=65535, device="cpu") -> Calib:
    """Dark (with hot pixels), vignetted flat with pixel response scatter, sparse BPM."""
    g = _gen(seed * 104729 + 3)
    dark = torch.full((h, w), dark_level, dtype=torch.float32)
    hot = torch.rand(h, w, generator=g) < hot_frac
    dark[hot] += (torch.rand(int(hot.sum()), generator=g) * 200.0 + 20.0)
    yy = (torch.arange(h, dtype=torch.float32) - (h - 1) / 2) / max(h, 1)
    xx = (torch.arange(w, dtype=torch.float32) - (w - 1) / 2) / max(w, 1)
    r2 = yy[:, None] ** 2 + xx[None, :] ** 2
    flat = (1.0 - 0.2 * r2) * (1.0 + flat_rms * torch.randn(h, w, generator=g))
    bpm = (torch.rand(h, w, generator=g) < bad_frac).to(torch.uint8)
    d = torch.device(device)
    return Calib(int(bias), dark.to(d), flat.to(torch.float32).to(d), bpm.to(d),
                 float(gain), float(read_noise), int(sat))


def expose(expected_sky_e: torch.Tensor, calib: Calib, seed: int, *,
           cosmic_frac=0.0, cosmic_range=(1e3, 3e4)) -> torch.Tensor:
    """Draw one raw uint16 frame from the expected electrons falling on the sky side.

    expected_sky_e: [h, w] expected electrons before the flat (sky + stars).
    Cosmic rays (single pixels, log-uniform amplitude) are added in electrons.
    """
    dev = expected_sky_e.device
    g = _gen(seed, dev)
    lam = expected_sky_e.to(torch.float32) * calib.flat.to(dev) + calib.dark.to(dev)
    lam = torch.clamp(lam, min=0.0)
    e = torch.poisson(lam, generator=g)
    if cosmic_frac > 0:
        hit = torch.rand(lam.shape, generator=g, device=dev) < cosmic_frac
        lo, hi = math.log(cosmic_range[0]), math.log(cosmic_range[1])
        amp = torch.exp(lo + (hi - lo) * torch.rand(lam.shape, generator=g, device=dev))
        e = e + hit.to(e.dtype) * amp
    adu = e / calib.gain + calib.bias + torch.randn(lam.shape, generator=g, device=dev) * (
        calib.read_noise / calib.gain)
    adu = torch.clamp(torch.round(adu), 0, 65535)
    return adu.to(torch.int32).to(torch.uint16)


def reference_image(expected_e: torch.Tensor, n_ref: int, read_noise: float, seed: int):
    """A deep reference: expected electrons plus noise of an n_ref-frame average.

    Returns (R float32, V_ref float32) with V_ref = (expected + rn^2) / n_ref.
    """
    dev = expected_e.device
    g = _gen(seed, dev)
    var = (torch.clamp(expected_e, min=0.0) + read_noise ** 2) / n_ref
    r = expected_e + torch.randn(expected_e.shape, generator=g, device=dev,
                                 dtype=expected_e.dtype) * torch.sqrt(var)
    return r.to(torch.float32), var.to(torch.float32)


def field_sigma(w: int, h: int, s_center: float, s_corner: float):
    """PSF width varying as s_center + (s_corner - s_center) * rhat**2 across the field."""
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    rmax2 = cx * cx + cy * cy

    def f(x, y):
        r2 = ((x - cx) ** 2 + (y - cy) ** 2) / rmax2
        return s_center + (s_corner - s_center) * torch.clamp(r2, 0.0, 1.0)
    return f


def uniform_shifts(n: int, seed: int, amp=0.5) -> torch.Tensor:
    """Per-frame sub-pixel shifts uniform in [-amp, amp]^2, float32 [n, 2]."""
    g = _gen(seed * 31 + 5)
    return ((torch.rand(n, 2, generator=g, dtype=torch.float64) * 2 - 1) * amp).to(torch.float32)


def pitch_for(w: int, align_elems: int = 16) -> int:
    """Row pitch (elements) with every row 16-byte aligned for 1-, 2- and 4-byte types."""
    return (w + align_elems - 1) // align_elems * align_elems


def pad_pitch(a: torch.Tensor, pitch: int) -> torch.Tensor:
    """Copy [h, w] into a zero-padded [h, pitch] contiguous tensor."""
    h, w = a.shape
    if pitch == w:
        return a.contiguous()
    out = torch.zeros((h, pitch), dtype=a.dtype, device=a.device)
    out[:, :w] = a
    return out


def calibrated_image(expected_e: torch.Tensor, read_noise: float, seed: int):
    """An already-calibrated science image: Poisson(expected) + N(0, rn), and its
    variance map expected + rn^2 (float32 pair)."""
    dev = expected_e.device
    g = _gen(seed, dev)
    lam = torch.clamp(expected_e.to(torch.float32), min=0.0)
    img = torch.poisson(lam, generator=g) + torch.randn(lam.shape, generator=g, device=dev) * read_noise
    return img.to(torch.float32), (lam + read_noise ** 2).to(torch.float32)


def segment_sides(n: int, seed: int, smin=64, smax=512):
    """Square segment sides log-uniform on [smin, smax] (rounded)."""
    g = _gen(seed * 613 + 11)
    u = torch.rand(n, generator=g, dtype=torch.float64)
    return torch.round(smin * (smax / smin) ** u).to(torch.int64).tolist()


def segment_origins(sides, w: int, h: int, seed: int):
    """Uniform top-left corners of squares of the given sides inside a w x h frame."""
    g = _gen(seed * 977 + 5)
    s = torch.as_tensor(list(sides), dtype=torch.float64)
    u = torch.rand(len(s), 2, generator=g, dtype=torch.float64)
    x0 = torch.floor(u[:, 0] * (w - s + 1)).to(torch.int64).tolist()
    y0 = torch.floor(u[:, 1] * (h - s + 1)).to(torch.int64).tolist()
    return list(zip(x0, y0))


def transient_catalog(n: int, w: int, h: int, seed: int, sigma: float, noise: float, snr=(5.0, 20.0),
                      border=30.0):
    """Point-like transients to inject into a science frame: uniform positions at least
    `border` px from the edges, fluxes giving a peak-pixel S/N log-uniform in `snr` for a
    Gaussian PSF of width sigma over per-pixel noise `noise` (peak = F / (2 pi sigma^2)).
    Returns (Catalog, peak S/N float64 [n])."""
    g = _gen(seed * 104729 + 3)
    u = torch.rand(n, 3, generator=g, dtype=torch.float64)
    x = border + u[:, 0] * (w - 1 - 2 * border)
    y = border + u[:, 1] * (h - 1 - 2 * border)
    s = torch.exp(math.log(snr[0]) + u[:, 2] * (math.log(snr[1]) - math.log(snr[0])))
    flux = s * noise * 2.0 * math.pi * sigma * sigma
    return Catalog(x, y, flux), s
