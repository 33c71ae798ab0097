"""Pins of the median-filtered background oracle (Table 2 "Median-filtered
background map"; background maps kept with the calibration frames, Sec. 3.2)
against exact cases, numpy's median and scipy's grid interpolation.  CPU only."""
import numpy as np
import pytest
import scipy.interpolate

from oracle import background as bgo


def test_constant_sky_with_sparse_stars_is_exact():
    """Stars cover well under half of every box, so every box median is the sky."""
    rng = np.random.default_rng(1)
    h, w, box = 200, 300, 32
    img = np.full((h, w), 312.5, np.float32)
    ys, xs = rng.integers(0, h, 400), rng.integers(0, w, 400)
    for y, x in zip(ys, xs):
        img[max(0, y - 1):y + 2, max(0, x - 1):x + 2] += rng.uniform(50, 5000)
    mesh, m = bgo.background_map(img, None, box=box, filt=3)
    assert (mesh == 312.5).all() and (m == 312.5).all()


@pytest.mark.parametrize("w,h,box", [(256, 192, 32), (250, 170, 32), (97, 61, 16)])
def test_linear_ramp_is_reproduced(w, h, box):
    """img = 100 + x + 2 y: a box median is the ramp at the box centre (the pixel
    set is symmetric about its mean), so with no filter the map is the ramp
    between the outermost centres and constant beyond; the 3 x 3 filter keeps
    interior boxes (their neighbourhoods are symmetric too)."""
    y, x = np.mgrid[0:h, 0:w]
    img = (100 + x + 2 * y).astype(np.float32)
    cx, cy = bgo.box_centres(w, box), bgo.box_centres(h, box)
    mesh = bgo.box_medians(img, None, box)
    np.testing.assert_array_equal(mesh, 100 + cx[None, :] + 2 * cy[:, None])
    _, m = bgo.background_map(img, None, box=box, filt=1)
    ramp = 100 + np.clip(x, cx[0], cx[-1]) + 2 * np.clip(y, cy[0], cy[-1])
    np.testing.assert_allclose(m, ramp, rtol=0, atol=1e-9)
    fm = bgo.median_filter_mesh(mesh, 3)
    np.testing.assert_array_equal(fm[1:-1, 1:-1], mesh[1:-1, 1:-1])


def test_single_box_is_numpy_median_of_valid_pixels():
    rng = np.random.default_rng(2)
    img = rng.normal(500, 30, (40, 50)).astype(np.float32)
    img[3, 4] = np.nan
    img[7, 8] = np.inf
    flags = (rng.random((40, 50)) < 0.2).astype(np.uint8)
    img[flags == 1] += 1e6                     # flagged pixels must not count
    mesh, m = bgo.background_map(img, flags, box=64, filt=3)
    ok = (flags == 0) & np.isfinite(img)
    assert mesh.shape == (1, 1)
    assert mesh[0, 0] == np.median(img[ok].astype(np.float64))
    assert (m == mesh[0, 0]).all()


def test_bright_box_and_sparse_box_are_replaced_by_the_filter():
    """A box filled by a bright galaxy, and a box with 60 % flagged pixels (no
    value), both take the median of their neighbourhood."""
    h, w, box = 128, 128, 32
    img = np.full((h, w), 50.0, np.float32)
    img[32:64, 32:64] = 900.0
    flags = np.zeros((h, w), np.uint8)
    flags[64:96, 96:128].flat[: int(0.6 * 32 * 32)] = 1
    raw = bgo.box_medians(img, flags, box)
    assert raw[1, 1] == 900.0 and np.isnan(raw[2, 3])
    mesh, m = bgo.background_map(img, flags, box=box, filt=3)
    assert (mesh == 50.0).all() and (m == 50.0).all()


def test_interpolation_matches_scipy_grid_interpolator():
    """Piecewise-constant boxes, no filter: the map is scipy's bilinear grid
    interpolation of the box values at the box centres, with clamped coordinates."""
    rng = np.random.default_rng(3)
    h, w, box = 90, 140, 20
    ny, nx = -(-h // box), -(-w // box)
    vals = rng.uniform(0, 100, (ny, nx))
    img = np.repeat(np.repeat(vals, box, 0), box, 1)[:h, :w].astype(np.float32)
    mesh, m = bgo.background_map(img, None, box=box, filt=1)
    np.testing.assert_array_equal(mesh, vals.astype(np.float32).astype(np.float64))
    cx, cy = bgo.box_centres(w, box), bgo.box_centres(h, box)
    f = scipy.interpolate.RegularGridInterpolator((cy, cx), mesh, method="linear")
    y, x = np.mgrid[0:h, 0:w]
    pts = np.stack([np.clip(y, cy[0], cy[-1]).ravel(), np.clip(x, cx[0], cx[-1]).ravel()], 1)
    np.testing.assert_allclose(m, f(pts).reshape(h, w), rtol=0, atol=1e-10)


def test_empty_mesh_falls_back_to_zero():
    img = np.full((20, 20), np.nan, np.float32)
    mesh, m = bgo.background_map(img, None, box=8, filt=3)
    assert (mesh == 0).all() and (m == 0).all()
