"""Shared helpers of the GPU parity tests: pitched device copies and tolerances."""
import numpy as np
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300.synth import pitch_for

F32_EPS = 2.0 ** -24


def dev_pitched(a: np.ndarray, pitch: int | None = None, fill=0) -> torch.Tensor:
    """Copy a [h, w] host array into a [h, pitch] CUDA tensor; padding is `fill`."""
    h, w = a.shape
    pitch = pitch or pitch_for(w)
    t = torch.full((h, pitch), fill, dtype=torch.from_numpy(np.ascontiguousarray(a)).dtype)
    t[:, :w] = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda()


def host(t: torch.Tensor, w: int) -> np.ndarray:
    return t[:, :w].cpu().numpy()


def ctx_for(w, h, max_stamps=64, max_coeffs=320, det_cap=1 << 20):
    return B.argus_create(0, h * pitch_for(w), max_stamps, max_coeffs, det_cap)


def assert_rel(gpu, ref, scale, rtol, what=""):
    """|gpu - ref| <= rtol * scale elementwise, reporting the worst offender."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(gpu - ref) / np.maximum(scale, 1e-300)
    i = int(np.argmax(err)) if err.size else 0
    assert err.size == 0 or err.flat[i] <= rtol, (
        f"{what}: worst rel err {err.flat[i]:.3e} > {rtol:.1e} at {np.unravel_index(i, err.shape)}: "
        f"gpu {gpu.flat[i]!r} ref {ref.flat[i]!r}")
    return float(err.max()) if err.size else 0.0


def check_detection_properties(D, VD, fl, mask, src, n_found, nsigma):
    """Detection checked by properties that hold at any size, on host arrays (float32 D,
    VD; uint8 fl, mask): the mask is the float threshold of S = D / sqrt(V_D) on the valid
    pixels; the components are scipy's 8-connected equal-sign components; each source's
    peak is its component's max |S| (ties to the lowest (y, x)), npix its size, peak_snr
    its S; the list is ordered by (py, px).  Returns the positive and negative counts."""
    import scipy.ndimage as ndi
    valid = (fl == 0) & (VD > 0) & np.isfinite(D) & np.isfinite(VD)
    with np.errstate(divide="ignore", invalid="ignore"):
        S = np.where(valid, D / np.sqrt(VD), np.float32(0)).astype(np.float32)
    m = np.where(valid, (S >= nsigma) * B.ARGUS_MASK_POS + (S <= -nsigma) * B.ARGUS_MASK_NEG,
                 B.ARGUS_MASK_INVALID).astype(np.uint8)
    np.testing.assert_array_equal(mask, m)
    eight = np.ones((3, 3), bool)
    lab_p, n_p = ndi.label(m == B.ARGUS_MASK_POS, structure=eight)
    lab_n, n_n = ndi.label(m == B.ARGUS_MASK_NEG, structure=eight)
    assert n_found == n_p + n_n
    keys = list(zip(src["py"], src["px"]))
    assert keys == sorted(keys)
    A = np.abs(S)
    for lab, sign in ((lab_p, 1), (lab_n, -1)):
        sel = src[src["sign"] == sign]
        if len(sel) == 0:
            continue
        ids = lab[sel["py"], sel["px"]]
        assert (ids > 0).all()
        sizes = np.bincount(lab.ravel())
        np.testing.assert_array_equal(sel["npix"], sizes[ids])
        peaks = ndi.maximum_position(A, lab, ids)     # first maximum in raster order
        np.testing.assert_array_equal(np.array(peaks, dtype=np.int64).reshape(-1, 2),
                                      np.stack([sel["py"], sel["px"]], 1))
        np.testing.assert_array_equal(sel["peak_snr"], S[sel["py"], sel["px"]])
    return n_p, n_n


# The difference variance on the GPU takes, for every pixel, the kernel at the centre of
# the 128 x 128 frame tile holding it (an approximation: the exact kernel at the pixel is
# quadratic in the spatial terms).  Its deviation from the exact V_D at a pixel is
#   sum_{u,v} (K_c(u,v)^2 - K_xy(u,v)^2) V_ref(x - u, y - v),
# bounded in absolute value by the same sum of |K_c^2 - K_xy^2| V_ref.  The tensor-core
# variance also rounds V_ref and K_c^2 to BF16 once each (one product): at most 2^-8 of
# sum K_c^2 V_ref, the convolved-reference term.
BF16_VAR = 2.0 ** -8 * 1.01
VAR_TILE = 128
# V_D bar of the tests: a relative error e in V_D moves S = D / sqrt(V_D) by about e / 2,
# and the detection mask is compared outside a band of 1e-3 of the threshold, so 1e-3
# leaves every decision outside the band unchanged (and moves flux_err by 5e-4 at most).
VD_RTOL = 1e-3


def _terms(xt, yt, sdeg):
    return np.stack([xt ** i * yt ** j for i in range(sdeg + 1) for j in range(sdeg + 1 - i)], -1)


def tile_rule_allowance(K, sdeg, Vr, xy, frame, origin=(0, 0)):
    """sum |K_c^2 - K_xy^2| V_ref + BF16_VAR sum K_c^2 V_ref at the listed pixels xy [n][2]
    (local x, y) of an image whose local (0, 0) is frame pixel `origin` of a W x H frame;
    K [Ks][ks][ks].  Pixels within r of the image edge get 0 (they have no variance)."""
    K = np.asarray(K, np.float64)
    ks = K.shape[-1]
    r = (ks - 1) // 2
    h, w = Vr.shape
    W, H = frame
    ox, oy = origin
    xy = np.asarray(xy)
    out = np.zeros(len(xy))
    Kf = K.reshape(K.shape[0], -1)
    dv, du = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1), indexing="ij")
    Vr64 = np.asarray(Vr, np.float64)
    xt = lambda x: (2.0 * x - (W - 1)) / (W - 1) if W > 1 else 0.0 * x
    yt = lambda y: (2.0 * y - (H - 1)) / (H - 1) if H > 1 else 0.0 * y
    for s in range(0, len(xy), 8192):
        x = xy[s:s + 8192, 0].astype(np.int64)
        y = xy[s:s + 8192, 1].astype(np.int64)
        ok = (x >= r) & (x <= w - 1 - r) & (y >= r) & (y <= h - 1 - r)
        x, y = x[ok], y[ok]
        fx, fy = x + ox, y + oy
        cx = (fx // VAR_TILE) * VAR_TILE + 0.5 * (VAR_TILE - 1)
        cy = (fy // VAR_TILE) * VAR_TILE + 0.5 * (VAR_TILE - 1)
        Kxy = _terms(xt(fx.astype(np.float64)), yt(fy.astype(np.float64)), sdeg) @ Kf
        Kc = _terms(xt(cx), yt(cy), sdeg) @ Kf
        win = Vr64[y[:, None] - dv.ravel()[None, :], x[:, None] - du.ravel()[None, :]]
        e = np.zeros(len(xy[s:s + 8192]))
        e[ok] = (np.abs(Kc ** 2 - Kxy ** 2) * win).sum(1) + BF16_VAR * (Kc ** 2 * win).sum(1)
        out[s:s + 8192] = e
    return out


def assert_variance(Vg, Vo, allowance, what="V_D"):
    """The GPU's V_D against the oracle's exact one: within 1e-5 relative (FP32 arithmetic)
    plus the allowance of the tile rule and the BF16 rounding.  Returns the worst error
    relative to V_D."""
    Vg = np.asarray(Vg, np.float64).ravel()
    Vo = np.asarray(Vo, np.float64).ravel()
    a = np.asarray(allowance, np.float64).ravel()
    err = np.abs(Vg - Vo)
    bad = err > 1e-5 * np.maximum(Vo, 1e-6) + a * (1 + 1e-6)
    i = int(np.argmax(err - 1e-5 * np.maximum(Vo, 1e-6) - a)) if err.size else 0
    assert not bad.any(), f"{what}: |dV| {err[i]:.3e} > allowance {a[i]:.3e} + 1e-5 V ({Vo[i]:.3e}) at {i}"
    pos = Vo > 0
    return float((err[pos] / Vo[pos]).max()) if pos.any() else 0.0


def psf_matching_field(ks, W, H, sig_ref=1.2, s0=1.3, s1=0.9, n=25):
    """Degree-2 kernel field of a W x H frame whose science PSF widens from s0 at the centre
    to s0 + s1 at the corners (sigma = s0 + s1 r^2, r the radius over the corner radius),
    against a reference PSF of sig_ref: at n x n points the unit-sum Gaussian of variance
    sigma^2 - sig_ref^2 (ks x ks taps), each tap fitted by least squares with the six terms
    1, y, y^2, x, x y, x^2 of the normalised frame coordinates.  Returns K [6][ks][ks]."""
    r = (ks - 1) // 2
    u = np.arange(-r, r + 1)
    t = np.linspace(-1, 1, n)
    X, Y = np.meshgrid(t, t)
    rr = (X ** 2 + Y ** 2) / 2.0
    sk2 = (s0 + s1 * rr) ** 2 - sig_ref ** 2
    G = np.exp(-(u[None, None, None, :] ** 2 + u[None, None, :, None] ** 2) / (2 * sk2[..., None, None]))
    G /= G.sum(axis=(-1, -2), keepdims=True)
    A = _terms(X.ravel(), Y.ravel(), 2)
    coef, *_ = np.linalg.lstsq(A, G.reshape(n * n, -1), rcond=None)
    return coef.reshape(6, ks, ks)
