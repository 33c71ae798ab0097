"""FP64 oracle of HEALPix segmentation and resampling (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU legs may import this
module; the product library never calls it.

The paper reprojects each full-frame image into HEALPix NSIDE=256 segments
(Sec. 3.3 "Image Segmentation"; Table 2, GPU stage "Image segmentation and
resampling to HEALPix grid") and names the HEALPix scheme of Gorski et al.
(2005) for it.  Readings taken here:

* a segment image is the 2^k x 2^k grid of the HEALPix pixels at
  NSIDE_seg 2^k that lie inside one NSIDE_seg pixel (nested scheme): image
  column c and row r are the face coordinates ix = X 2^k + c, iy = Y 2^k + r,
  with (X, Y) the segment's own face coordinates; each image pixel takes the
  value at its HEALPix pixel centre;
* the frame's sky-to-pixel map is a gnomonic (tangent-plane) projection about
  a centre (alpha0, delta0) with a pixel scale, a rotation and a reference
  pixel -- the form an astrometric solution of a small field takes;
* the value at a frame position is the bilinear interpolation of the frame
  written as nested lerps (the coadd's rule): a position is covered when it
  lies in [0, w-1] x [0, h-1] and every neighbour with a nonzero weight is
  unflagged and finite; uncovered pixels are 0 with coverage 0.
"""
from __future__ import annotations

import numpy as np

# base-face ring and longitude offsets of the nested layout (faces 0-3 north,
# 4-7 equatorial, 8-11 south)
JRLL = np.array([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4])
JPLL = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7])


def xyf2vec(ix, iy, face, nside):
    """Unit vectors of the centres of the pixels (ix, iy) of base face `face` at
    NSIDE `nside` (arrays broadcast).  Returns (..., 3) float64."""
    ix = np.asarray(ix, np.int64)
    iy = np.asarray(iy, np.int64)
    face = np.asarray(face, np.int64)
    ix, iy, face = np.broadcast_arrays(ix, iy, face)
    n = np.int64(nside)
    jr = JRLL[face] * n - ix - iy - 1                    # ring index, 1 at the north pole
    north, south = jr < n, jr > 3 * n
    nr = np.where(north, jr, np.where(south, 4 * n - jr, n))
    # distance from the nearer pole in z, exact for the caps
    cap = nr.astype(np.float64) ** 2 / (3.0 * float(n) ** 2)
    z = np.where(north, 1.0 - cap, np.where(south, -1.0 + cap, (2 * n - jr) * 2.0 / (3.0 * n)))
    sin_t = np.where(north | south, np.sqrt(cap * (2.0 - cap)), np.sqrt((1.0 - z) * (1.0 + z)))
    kshift = np.where(north | south, 0, (jr - n) & 1)
    jp = (JPLL[face] * nr + ix - iy + 1 + kshift) // 2
    jp = np.where(jp > 4 * nr, jp - 4 * nr, jp)
    jp = np.where(jp < 1, jp + 4 * nr, jp)
    phi = (jp - (kshift + 1) * 0.5) * (np.pi / 2.0) / nr
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), z], axis=-1)


def nest2xyf(pix, nside):
    """Face and face coordinates of a nested pixel index: ix from the even bits
    of the in-face index, iy from the odd bits."""
    pix = np.asarray(pix, np.int64)
    face = pix // (nside * nside)
    ipf = pix - face * nside * nside
    ix = np.zeros_like(ipf)
    iy = np.zeros_like(ipf)
    for b in range(int(np.log2(nside)) + 1):
        ix |= ((ipf >> (2 * b)) & 1) << b
        iy |= ((ipf >> (2 * b + 1)) & 1) << b
    return ix, iy, face


def segment_vectors(seg, nside_seg, k):
    """[2^k][2^k][3] unit vectors of the image pixel centres of segment `seg`
    (nested index at nside_seg): row r, column c is face pixel
    (X 2^k + c, Y 2^k + r) at NSIDE nside_seg 2^k."""
    X, Y, f = nest2xyf(seg, nside_seg)
    m = 1 << k
    c = np.arange(m)
    return xyf2vec(int(X) * m + c[None, :], int(Y) * m + c[:, None], int(f), nside_seg * m)


def gnomonic(v, alpha0, delta0, scale, rot, cx, cy):
    """Frame pixel coordinates (x, y) of unit vectors v (..., 3); NaN where the
    direction is not in front of the tangent plane.  Tangent-plane coordinates
    xi (east), eta (north) about (alpha0, delta0); x = cx + (cos rot xi +
    sin rot eta) / scale, y = cy + (-sin rot xi + cos rot eta) / scale."""
    v = np.asarray(v, np.float64)
    ca, sa, cd, sd = np.cos(alpha0), np.sin(alpha0), np.cos(delta0), np.sin(delta0)
    n = np.array([cd * ca, cd * sa, sd])
    e = np.array([-sa, ca, 0.0])
    u = np.array([-sd * ca, -sd * sa, cd])
    d = v @ n
    with np.errstate(divide="ignore", invalid="ignore"):
        xi = np.where(d > 0, (v @ e) / d, np.nan)
        eta = np.where(d > 0, (v @ u) / d, np.nan)
    cr, sr = np.cos(rot), np.sin(rot)
    return cx + (cr * xi + sr * eta) / scale, cy + (-sr * xi + cr * eta) / scale


def bilinear(frame, flags, x, y):
    """Nested-lerp bilinear value at (x, y) and coverage (see the module notes)."""
    frame = np.asarray(frame, np.float32)
    h, w = frame.shape
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    out = np.zeros(x.shape)
    cov = np.zeros(x.shape, np.uint8)
    inside = np.isfinite(x) & np.isfinite(y) & (x >= 0) & (y >= 0) & (x <= w - 1) & (y <= h - 1)
    for idx in zip(*np.nonzero(inside)):
        xx, yy = x[idx], y[idx]
        x0, y0 = int(np.floor(xx)), int(np.floor(yy))
        tx, ty = xx - x0, yy - y0
        need = [(y0, x0, True), (y0, x0 + 1, tx > 0), (y0 + 1, x0, ty > 0), (y0 + 1, x0 + 1, tx > 0 and ty > 0)]
        ok = True
        vals = {}
        for (j, i, used) in need:
            if not used:
                vals[(j, i)] = 0.0
                continue
            v = float(frame[j, i])
            if not np.isfinite(v) or (flags is not None and flags[j, i]):
                ok = False
                break
            vals[(j, i)] = v
        if not ok:
            continue
        v00, v01 = vals[(y0, x0)], vals[(y0, x0 + 1)]
        v10, v11 = vals[(y0 + 1, x0)], vals[(y0 + 1, x0 + 1)]
        top = v00 + tx * (v01 - v00)
        bot = v10 + tx * (v11 - v10)
        out[idx] = top + ty * (bot - top)
        cov[idx] = 1
    return out, cov


def resample_segment(frame, flags, seg, nside_seg, k, wcs):
    """Segment image ([2^k][2^k] float64) and coverage (u8) of a frame with
    gnomonic WCS (alpha0, delta0, scale, rot, cx, cy)."""
    v = segment_vectors(seg, nside_seg, k)
    x, y = gnomonic(v, *wcs)
    return bilinear(frame, flags, x, y)
