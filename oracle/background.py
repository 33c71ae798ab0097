"""FP64 oracle of the median-filtered background map (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU legs may import this
module; the product library never calls it.

The paper lists a "median-filtered background map" among its GPU stages
(Table 2, GPU timing: 1.7 ms per 61-Mpix frame) and keeps background maps
with the calibration frames (Sec. 3.2), but gives no procedure.  The reading
taken here is the usual mesh estimate:

1. mesh: boxes of box x box pixels from (0, 0); the last row and column of
   boxes hold the pixels that exist;
2. box value: the median of the box's valid pixels (flag 0 and finite; an
   even count takes the mean of the two middle values); a box with fewer than
   min_frac of its pixels valid has no value;
3. median filter: each box takes the median of the values that exist in the
   filt x filt neighbourhood of boxes around it (clipped at the mesh edges);
   boxes with no value in reach take the median of all box values (0 if none);
4. map: bilinear interpolation between box centres (the centre of a box is
   the mean coordinate of its pixels), constant beyond the outermost centres.
"""
from __future__ import annotations

import numpy as np


def _median(v):
    v = np.sort(np.asarray(v, np.float64))
    n = v.size
    return 0.5 * (v[(n - 1) // 2] + v[n // 2])


def box_medians(img, flags, box, min_frac=0.5):
    """Step 2: [ny][nx] box medians, NaN where a box has too few valid pixels."""
    img = np.asarray(img, np.float32)
    h, w = img.shape
    ny, nx = -(-h // box), -(-w // box)
    out = np.full((ny, nx), np.nan)
    for by in range(ny):
        for bx in range(nx):
            b = img[by * box:(by + 1) * box, bx * box:(bx + 1) * box].astype(np.float64)
            ok = np.isfinite(b)
            if flags is not None:
                ok &= np.asarray(flags)[by * box:(by + 1) * box, bx * box:(bx + 1) * box] == 0
            if ok.sum() >= min_frac * b.size and ok.any():
                out[by, bx] = _median(b[ok])
    return out


def median_filter_mesh(mesh, filt):
    """Step 3: filt x filt median of the existing values, clipped at the edges."""
    ny, nx = mesh.shape
    r = filt // 2
    out = np.empty_like(mesh)
    have = mesh[np.isfinite(mesh)]
    fill = _median(have) if have.size else 0.0
    for y in range(ny):
        for x in range(nx):
            nb = mesh[max(0, y - r):y + r + 1, max(0, x - r):x + r + 1]
            nb = nb[np.isfinite(nb)]
            out[y, x] = _median(nb) if nb.size else fill
    return out


def box_centres(n, box):
    """Mean pixel coordinate of each box along one axis of n pixels."""
    starts = np.arange(0, n, box)
    ends = np.minimum(starts + box, n)
    return (starts + ends - 1) / 2.0


def interpolate(mesh, w, h, box):
    """Step 4: bilinear between box centres, clamped beyond the outermost ones."""
    cx, cy = box_centres(w, box), box_centres(h, box)

    def axis(c, n):
        p = np.arange(n, dtype=np.float64)
        if c.size == 1:
            return np.zeros(n, int), np.zeros(n, int), np.zeros(n)
        i = np.clip(np.searchsorted(c, p, side="right") - 1, 0, c.size - 2)
        t = np.clip((p - c[i]) / (c[i + 1] - c[i]), 0.0, 1.0)
        return i, i + 1, t

    x0, x1, tx = axis(cx, w)
    y0, y1, ty = axis(cy, h)
    m00 = mesh[np.ix_(y0, x0)]
    m01 = mesh[np.ix_(y0, x1)]
    m10 = mesh[np.ix_(y1, x0)]
    m11 = mesh[np.ix_(y1, x1)]
    top = m00 + (m01 - m00) * tx[None, :]
    bot = m10 + (m11 - m10) * tx[None, :]
    return top + (bot - top) * ty[:, None]


def background_map(img, flags, box=64, filt=3, min_frac=0.5):
    """The whole map: returns (filtered mesh [ny][nx], map [h][w]), FP64."""
    img = np.asarray(img)
    h, w = img.shape
    mesh = median_filter_mesh(box_medians(img, flags, box, min_frac), filt)
    return mesh, interpolate(mesh, w, h, box)
