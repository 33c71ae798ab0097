"""Pins of the HEALPix segmentation oracle (Sec. 3.3 "Image Segmentation";
Table 2 GPU stage "Image segmentation and resampling to HEALPix grid")
against the closed forms of the HEALPix geometry, the definition of the
gnomonic projection and exact interpolation cases.  CPU only."""
import math

import numpy as np
import pytest

from oracle import healpix as hp


def test_base_pixel_centres():
    """NSIDE = 1: faces 0-3 at z = 2/3, phi = pi/4 + f pi/2; 4-7 on the equator at
    phi = (f - 4) pi/2; 8-11 at z = -2/3, phi = pi/4 + (f - 8) pi/2."""
    v = hp.xyf2vec(0, 0, np.arange(12), 1)
    z_expect = np.array([2 / 3] * 4 + [0.0] * 4 + [-2 / 3] * 4)
    phi_expect = np.array([math.pi / 4 + f * math.pi / 2 for f in range(4)] + [f * math.pi / 2 for f in range(4)]
                          + [math.pi / 4 + f * math.pi / 2 for f in range(4)])
    np.testing.assert_allclose(v[:, 2], z_expect, atol=1e-15)
    np.testing.assert_allclose(np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * math.pi), phi_expect, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)


def _interleave(ix, iy, order):
    p = 0
    for b in range(order):
        p |= ((ix >> b) & 1) << (2 * b)
        p |= ((iy >> b) & 1) << (2 * b + 1)
    return p


@pytest.mark.parametrize("nside", [4, 8, 16])
def test_ring_structure_and_equal_spacing(nside):
    """4 N - 1 rings; ring i has 4 i pixels (i < N) or 4 N (N <= i <= 3 N); ring z is
    1 - i^2/(3 N^2) in the caps and 4/3 - 2 i/(3 N) in the equatorial belt; the
    longitudes of a ring are equally spaced; the vectors sum to zero."""
    n = nside
    v = hp.xyf2vec(*hp.nest2xyf(np.arange(12 * n * n), n)[:2], hp.nest2xyf(np.arange(12 * n * n), n)[2], n)
    z = v[:, 2]
    zs = np.unique(np.round(z, 12))[::-1]
    assert zs.size == 4 * n - 1
    for i, zi in enumerate(zs, start=1):
        ring = np.abs(z - zi) < 1e-11
        m = 4 * i if i < n else (4 * n if i <= 3 * n else 4 * (4 * n - i))
        assert ring.sum() == m
        ze = 1 - i * i / (3 * n * n) if i <= n else (4 / 3 - 2 * i / (3 * n) if i <= 3 * n
                                                     else -1 + (4 * n - i) ** 2 / (3 * n * n))
        assert abs(zi - ze) < 1e-12
        phi = np.sort(np.mod(np.arctan2(v[ring, 1], v[ring, 0]), 2 * math.pi))
        np.testing.assert_allclose(np.diff(phi), 2 * math.pi / m, atol=1e-12)
    np.testing.assert_allclose(v.sum(axis=0), 0.0, atol=1e-11)


def test_nested_index_round_trip():
    rng = np.random.default_rng(1)
    n, order = 256, 8
    ix, iy, f = rng.integers(0, n, 500), rng.integers(0, n, 500), rng.integers(0, 12, 500)
    p = np.array([fi * n * n + _interleave(int(a), int(b), order) for a, b, fi in zip(ix, iy, f)])
    gx, gy, gf = hp.nest2xyf(p, n)
    np.testing.assert_array_equal(gx, ix)
    np.testing.assert_array_equal(gy, iy)
    np.testing.assert_array_equal(gf, f)


def test_children_lie_around_their_parent():
    """The 4 children (ix, iy) -> (2ix + a, 2iy + b) of every NSIDE-8 pixel have centres
    within one parent pixel size of the parent centre, and their mean is closer still."""
    n = 8
    ix, iy, f = hp.nest2xyf(np.arange(12 * n * n), n)
    parent = hp.xyf2vec(ix, iy, f, n)
    size = math.sqrt(4 * math.pi / (12 * n * n))
    kids = np.stack([hp.xyf2vec(2 * ix + a, 2 * iy + b, f, 2 * n) for a in (0, 1) for b in (0, 1)])
    ang = np.arccos(np.clip(np.einsum("kpi,pi->kp", kids, parent), -1, 1))
    assert ang.max() < size
    mean = kids.mean(axis=0)
    mean /= np.linalg.norm(mean, axis=1, keepdims=True)
    assert np.arccos(np.clip(np.einsum("pi,pi->p", mean, parent), -1, 1)).max() < 0.25 * size


def test_gnomonic_centre_scale_and_round_trip():
    a0, d0, scale, rot, cx, cy = 1.1, 0.4, 6.7e-6, 0.3, 4787.5, 3193.5
    ca, sa, cd, sd = math.cos(a0), math.sin(a0), math.cos(d0), math.sin(d0)
    n = np.array([cd * ca, cd * sa, sd])
    e = np.array([-sa, ca, 0.0])
    u = np.array([-sd * ca, -sd * sa, cd])
    x, y = hp.gnomonic(n, a0, d0, scale, rot, cx, cy)
    assert abs(x - cx) < 1e-9 and abs(y - cy) < 1e-9
    rng = np.random.default_rng(2)
    xi, eta = rng.uniform(-0.03, 0.03, 50), rng.uniform(-0.03, 0.03, 50)
    v = n[None, :] + xi[:, None] * e[None, :] + eta[:, None] * u[None, :]     # a point of the tangent plane
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x, y = hp.gnomonic(v, a0, d0, scale, rot, cx, cy)
    np.testing.assert_allclose(x, cx + (math.cos(rot) * xi + math.sin(rot) * eta) / scale, atol=1e-6)
    np.testing.assert_allclose(y, cy + (-math.sin(rot) * xi + math.cos(rot) * eta) / scale, atol=1e-6)
    assert np.isnan(hp.gnomonic(-n, a0, d0, scale, rot, cx, cy)[0])


def test_bilinear_exact_cases():
    h, w = 20, 30
    const = np.full((h, w), 7.25, np.float32)
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-1, w, 400), rng.uniform(-1, h, 400)
    out, cov = hp.bilinear(const, None, x, y)
    inside = (x >= 0) & (y >= 0) & (x <= w - 1) & (y <= h - 1)
    np.testing.assert_array_equal(cov, inside.astype(np.uint8))
    assert (out[inside] == 7.25).all() and (out[~inside] == 0).all()
    yy, xx = np.mgrid[0:h, 0:w]
    ramp = (3.0 + 2.0 * xx - 0.5 * yy).astype(np.float32)
    out, cov = hp.bilinear(ramp, None, x, y)
    np.testing.assert_allclose(out[inside], 3.0 + 2.0 * x[inside] - 0.5 * y[inside], atol=1e-12)
    fl = np.zeros((h, w), np.uint8)
    fl[5, 6] = 1
    # pixel (row 5, column 6) flagged: needed at x = 6 or 5 < x < 7 with row 5 in use
    _, c = hp.bilinear(ramp, fl, np.array([5.0, 5.5, 6.0, 5.0, 6.0, 6.5]), np.array([5.0, 5.0, 5.0, 4.5, 4.5, 5.5]))
    np.testing.assert_array_equal(c, [1, 0, 0, 1, 0, 0])


def test_segment_pixels_surround_the_segment_centre():
    """The mean of a segment image's pixel centres is the segment's own centre to well
    under one segment pixel, and neighbouring image pixels are about one image pixel apart."""
    nside_seg, k = 256, 5
    for seg in (0, 123456, 12 * 256 * 256 - 1, 400000):
        v = hp.segment_vectors(seg, nside_seg, k)
        X, Y, f = hp.nest2xyf(seg, nside_seg)
        c = hp.xyf2vec(X, Y, f, nside_seg)
        m = v.reshape(-1, 3).mean(axis=0)
        m /= np.linalg.norm(m)
        pix = math.sqrt(4 * math.pi / (12 * (nside_seg << k) ** 2))
        assert math.acos(min(1.0, float(m @ c))) < 0.5 * pix
        step = np.arccos(np.clip(np.einsum("rci,rci->rc", v[:, 1:], v[:, :-1]), -1, 1))
        assert 0.5 * pix < step.mean() < 1.5 * pix
