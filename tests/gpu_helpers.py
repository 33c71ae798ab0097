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
