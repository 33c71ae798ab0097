"""The basis convolution on the stamps (a4, argus_stamp_basis) against the FP64
oracle (ora_stamp_basis) element by element: at the fit's launch configuration
(400 stamps of 21 x 21 pixels with the 49 images of the 21 x 21 Alard-Lupton
basis, the tensor-core kernel), with 64 and with one image, with fewer stamps
than SMs, and on the shapes that run on the CUDA cores.

Tolerance: |X - X_oracle| <= 3e-5 S per element, S = sum over the taps of
|image| |ref| (the oracle's convolution of |ref| with |image|): FP32-level sums
of products (the tensor-core path rounds each operand to FP16 hi + lo, ~2^-21
per product, and accumulates 1,323 products in FP32).
"""
import numpy as np
import pytest
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300 import synth
from paper_2207_14304_gb300.synth import pitch_for
from tests.gpu_helpers import ctx_for, dev_pitched

pytestmark = pytest.mark.gpu

XTOL = 3e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


def _field(w, h, seed):
    rng = np.random.default_rng(seed)
    cat = synth.star_catalog(max(10, w * h // 300), w, h, seed=seed, flux_min=1e2, flux_max=3e6)
    R = synth.render(cat, w, h, 1.2, sky=300.0).numpy() + rng.normal(0, 5, (h, w))
    return R.astype(np.float32)


def _centres(n, w, h, stamp, ks, seed):
    """n stamp centres, about one in eight with its window leaving the frame."""
    rng = np.random.default_rng(seed)
    m = stamp // 2 + ks // 2
    x = rng.integers(m, w - m, n)
    y = rng.integers(m, h - m, n)
    edge = rng.random(n) < 0.125
    x[edge] = rng.integers(0, m + 1, int(edge.sum()))        # window crosses the left edge (or just fits)
    y[::11] = h - 1 - rng.integers(0, m + 1, len(y[::11]))   # and the bottom edge
    return np.stack([x, y], 1).astype(np.int32)


@pytest.mark.parametrize("case,w,h,stamp,ks,nb,n,max_stamps", [
    ("tensor cores, fit configuration", 1500, 1100, 21, 21, 49, 400, 416),
    ("tensor cores, 64 images, fewer stamps than SMs", 700, 500, 21, 21, 64, 37, 64),
    ("tensor cores, one image, one stamp", 200, 150, 21, 21, 1, 1, 4),
    ("CUDA cores, 11x11 images", 600, 400, 21, 11, 49, 50, 64),
    ("CUDA cores, 15x15 stamps, 9x9 images", 500, 300, 15, 9, 20, 30, 32),
])
def test_stamp_basis_parity(ora, case, w, h, stamp, ks, nb, n, max_stamps):
    R = _field(w, h, seed=w + nb)
    cen = _centres(n, w, h, stamp, ks, seed=n + ks)
    if nb == 49:
        imgs, _ = ora.basis(ora.Basis(ksize=ks, spatial_degree=0, bg_degree=0))
        imgs = imgs.reshape(nb, ks * ks)
    else:
        imgs = np.random.default_rng(nb).standard_normal((nb, ks * ks))
    imgs = imgs.astype(np.float32)
    assert imgs.shape == (nb, ks * ks)
    Xo = ora.stamp_conv(R, cen, stamp, imgs)                               # [n][ss][nb]
    So = ora.stamp_conv(np.abs(R), cen, stamp, np.abs(imgs))
    ss = stamp * stamp
    ctx = ctx_for(w, h, max_stamps=max_stamps)
    try:
        dR = dev_pitched(R)
        dcen = torch.zeros((max_stamps, 2), dtype=torch.int32, device="cuda")
        dcen[:n] = torch.from_numpy(cen).cuda()
        ns = torch.tensor([n, 0, 0, 0], dtype=torch.int32, device="cuda")
        dimg = torch.from_numpy(imgs).cuda().contiguous()
        X = torch.full((max_stamps, nb, ss), -7.0, dtype=torch.float32, device="cuda")
        B.argus_stamp_basis(ctx, dR, B.argus_shape(w, h, pitch_for(w)), dcen, ns, max_stamps, stamp, dimg, nb, ks, X)
        torch.cuda.synchronize()
        assert B.argus_sync_status(ctx) == 0
        Xg = X.cpu().numpy().astype(np.float64)
    finally:
        B.argus_destroy(ctx)
    assert (Xg[n:] == -7.0).all(), "stamps past n_stamps are not written"
    Xg = Xg[:n].transpose(0, 2, 1)                                         # [n][ss][nb]
    skipped = np.all(So == 0.0, axis=(1, 2))
    assert skipped.any() and not skipped.all() or n < 8
    assert (Xg[skipped] == 0.0).all(), "stamps whose window leaves the frame are zero"
    err = np.abs(Xg - Xo) / np.maximum(So, 1e-30)
    i = np.unravel_index(int(np.argmax(err)), err.shape)
    print(f"\n[stamp basis: {case}] worst |X - X_oracle| / S = {err[i]:.2e} at {i}")
    assert err[i] <= XTOL, f"{case}: {err[i]:.3e} at {i}: gpu {Xg[i]!r} oracle {Xo[i]!r}"
