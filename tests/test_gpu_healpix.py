"""HEALPix segmentation on the GPU (Sec. 3.3; Table 2 GPU stage "Image
segmentation and resampling to HEALPix grid") against the FP64 oracle:
coverage bit-exact, values within 4 ulps of the largest frame value, on both
the exact per-pixel path (k < 6, polar-cap rows) and the row path (k >= 6 in
the equatorial belt).

The kernel has not run on a GPU yet, so the file is skipped until it has.
"""
import math

import numpy as np
import pytest
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300.synth import pitch_for
from tests.gpu_helpers import F32_EPS, dev_pitched

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


@pytest.mark.parametrize("nside_seg,k,delta0", [(64, 4, 0.4), (256, 6, -0.3), (32, 5, 1.45), (256, 9, 0.2),
                                               (128, 7, 1.1)])
def test_healpix_resample_parity(ora, nside_seg, k, delta0):
    from oracle import healpix as hp
    rng = np.random.default_rng(nside_seg + k)
    w, h = 900, 700
    scale = 1.2 * math.sqrt(4 * math.pi / (12.0 * (nside_seg << k) ** 2))
    wcs = (2.1, delta0, scale, -0.4, (w - 1) / 2, (h - 1) / 2)
    yy, xx = np.mgrid[0:h, 0:w]
    frame = (300 + 0.05 * xx - 0.02 * yy + rng.normal(0, 10, (h, w))).astype(np.float32)
    frame.flat[11::701] = np.nan
    fl = (rng.random((h, w)) < 0.01).astype(np.uint8)
    p = np.arange(12 * nside_seg * nside_seg)
    ix, iy, f = hp.nest2xyf(p, nside_seg)
    x, y = hp.gnomonic(hp.xyf2vec(ix, iy, f, nside_seg), *wcs)
    near = p[np.isfinite(x) & (x > -20) & (y > -20) & (x < w + 20) & (y < h + 20)]
    segs = rng.choice(near, size=min(8, near.size), replace=False).astype(np.int64)
    m = 1 << k
    out = torch.full((segs.size, m, m), -7.0, device="cuda")
    cov = torch.full((segs.size, m, m), 7, dtype=torch.uint8, device="cuda")
    B.argus_healpix_resample(dev_pitched(frame), dev_pitched(fl), B.argus_shape(w, h, pitch_for(w)), wcs,
                             nside_seg, k, torch.from_numpy(segs).cuda(), segs.size, out, cov)
    torch.cuda.synchronize()
    out, cov = out.cpu().numpy(), cov.cpu().numpy()
    tol = 4 * F32_EPS * float(np.nanmax(np.abs(frame)))
    for i, s in enumerate(segs):
        o, oc = hp.resample_segment(frame, fl, int(s), nside_seg, k, wcs)
        np.testing.assert_array_equal(cov[i], oc)
        assert np.abs(out[i] - o).max() <= tol
