"""Sparse segment products on the GPU (sm_103a, through the C ABI) against the
FP64 oracle: minipix stamping (Sec. 3.3 "Sparse Image Segments") and the
low-resolution map (Sec. 2, segments at 10x reduced resolution).

Tolerances: the stamped image, the keep map, the kept-cell list and the packed
cells are bit-exact (copies and zeros); the low-resolution map is within
(2 f + 1) 2^-24 mean|v| of the FP64 block mean (FP32 sums of f column sums of
f pixels each, then one division).
"""
import numpy as np
import pytest
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300.synth import pitch_for
from tests.gpu_helpers import F32_EPS, ctx_for, dev_pitched, host

pytestmark = pytest.mark.gpu

SRC_DT = np.dtype([("x", "<f4"), ("y", "<f4"), ("flux", "<f4"), ("flux_err", "<f4"), ("peak_snr", "<f4"),
                   ("npix", "<i4"), ("sign", "<i4"), ("px", "<i4"), ("py", "<i4")])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


def _image(w, h, seed):
    rng = np.random.default_rng(seed)
    img = rng.normal(300, 20, (h, w)).astype(np.float32)
    img.flat[7::997] = np.nan
    img.flat[11::1999] = -np.inf
    img.flat[5::1013] = -0.0
    return img


def _sources(pxy):
    a = np.zeros(len(pxy), SRC_DT)
    if len(pxy):
        a["px"], a["py"] = np.asarray(pxy)[:, 0], np.asarray(pxy)[:, 1]
    return a


def _run_minipix(img, cell, targets, srcs, n_found, sources_cap, cap, want_out=True, want_pack=True):
    h, w = img.shape
    pitch = pitch_for(w)
    ncx, ncy = -(-w // cell), -(-h // cell)
    ctx = ctx_for(w, h)
    try:
        d_img = dev_pitched(img)
        d_t = torch.from_numpy(np.ascontiguousarray(np.asarray(targets, np.int32).reshape(-1, 2))).cuda()
        nt = d_t.shape[0]
        d_src = torch.from_numpy(srcs.view(np.uint8).copy()).cuda() if len(srcs) else None
        d_nf = torch.tensor([n_found, 0, 0, 0], dtype=torch.int32, device="cuda")
        keep = torch.full((ncy, ncx), 0xEE, dtype=torch.uint8, device="cuda")
        out = torch.full((h, pitch), -7.0, device="cuda") if want_out else None
        packed = torch.full((max(cap, 1), cell * cell), -7.0, device="cuda") if want_pack else None
        cidx = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda") if want_pack else None
        nk = torch.full((4,), -7, dtype=torch.int32, device="cuda")
        B.argus_minipix(ctx, d_img, B.argus_shape(w, h, pitch), cell, d_t if nt else None, nt, d_src,
                        d_nf if sources_cap else None, sources_cap, keep, out, packed, cidx, cap if want_pack else 0,
                        nk)
        torch.cuda.synchronize()
        st = B.argus_sync_status(ctx)
        return (st, keep.cpu().numpy(), None if out is None else out.cpu().numpy(),
                None if packed is None else packed.cpu().numpy(), None if cidx is None else cidx.cpu().numpy(),
                int(nk[0].item()))
    finally:
        B.argus_destroy(ctx)


def _packed_from_oracle(o_out, keep, cell):
    """Kept cells in ascending index order, cut from the oracle's stamped image
    (zero-padded past the right and bottom edges)."""
    h, w = o_out.shape
    ncy, ncx = keep.shape
    pad = np.zeros((ncy * cell, ncx * cell), np.float32)
    pad[:h, :w] = o_out
    idx = np.flatnonzero(keep.ravel())
    cells = pad.reshape(ncy, cell, ncx, cell).transpose(0, 2, 1, 3).reshape(ncy * ncx, cell * cell)
    return idx, cells[idx]


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


@pytest.mark.parametrize("w,h,cell,nt,ns,n_found,cap", [
    (1000, 37, 9, 40, 16, 12, 1 << 12),     # ragged both ways, fewer detections than the list holds
    (777, 515, 8, 300, 64, 90, 1 << 12),    # more detections than sources_cap: only the first 64 count
    (64, 64, 16, 0, 0, 0, 16),              # no targets at all
    (33, 1, 1, 5, 3, 3, 8),                 # one row, one-pixel cells
    (2049, 130, 256, 4, 0, 0, 4),           # largest cell
])
def test_minipix_parity(ora, w, h, cell, nt, ns, n_found, cap):
    rng = np.random.default_rng(w * 7 + h)
    img = _image(w, h, seed=w + h)
    targets = np.stack([rng.integers(-5, w + 5, nt), rng.integers(-5, h + 5, nt)], 1).astype(np.int32)
    pxy = np.stack([rng.integers(0, w, ns), rng.integers(0, h, ns)], 1)
    srcs = _sources(pxy)
    used = pxy[: min(ns, n_found)]
    o_out, o_keep, o_n = ora.minipix(img, cell, np.concatenate([targets.reshape(-1, 2), used.reshape(-1, 2)]))
    st, keep, out, packed, cidx, nk = _run_minipix(img, cell, targets, srcs, n_found, ns, cap)
    assert st == 0
    np.testing.assert_array_equal(keep, o_keep)
    assert nk == o_n
    np.testing.assert_array_equal(_bits(out[:, :w]), _bits(o_out))
    assert not out[:, w:].any()
    idx, cells = _packed_from_oracle(o_out, o_keep, cell)
    np.testing.assert_array_equal(cidx[:o_n], idx)
    np.testing.assert_array_equal(_bits(packed[:o_n]), _bits(cells))


def test_minipix_capacity_and_optional_outputs(ora):
    w, h, cell = 300, 200, 10
    img = _image(w, h, seed=5)
    targets = np.array([[x, y] for y in range(0, h, 20) for x in range(0, w, 20)], np.int32)
    o_out, o_keep, o_n = ora.minipix(img, cell, targets)
    cap = o_n // 3
    st, keep, out, packed, cidx, nk = _run_minipix(img, cell, targets, _sources([]), 0, 0, cap)
    assert st == B.ARGUS_ERR_CAPACITY and nk == o_n
    idx, cells = _packed_from_oracle(o_out, o_keep, cell)
    np.testing.assert_array_equal(cidx[:cap], idx[:cap])
    np.testing.assert_array_equal(_bits(packed[:cap]), _bits(cells[:cap]))
    np.testing.assert_array_equal(_bits(out[:, :w]), _bits(o_out))
    # keep map and count only: no stamped image, no list, no capacity error
    st, keep, out, packed, cidx, nk = _run_minipix(img, cell, targets, _sources([]), 0, 0, 0, want_out=False,
                                                   want_pack=False)
    assert st == 0 and nk == o_n
    np.testing.assert_array_equal(keep, o_keep)


def test_minipix_full_frame(ora):
    """9576 x 6388 frame, 9-pixel minipix cells, 2500 catalogue targets and 400
    detections: every pixel, cell and packed value checked."""
    w, h, cell = 9576, 6388, 9
    rng = np.random.default_rng(11)
    img = rng.normal(300, 20, (h, w)).astype(np.float32)
    targets = np.stack([rng.integers(0, w, 2500), rng.integers(0, h, 2500)], 1).astype(np.int32)
    pxy = np.stack([rng.integers(0, w, 400), rng.integers(0, h, 400)], 1)
    o_out, o_keep, o_n = ora.minipix(img, cell, np.concatenate([targets, pxy]))
    st, keep, out, packed, cidx, nk = _run_minipix(img, cell, targets, _sources(pxy), 400, 400, 1 << 13)
    assert st == 0 and nk == o_n
    np.testing.assert_array_equal(keep, o_keep)
    np.testing.assert_array_equal(_bits(out[:, :w]), _bits(o_out))
    idx, cells = _packed_from_oracle(o_out, o_keep, cell)
    np.testing.assert_array_equal(cidx[:o_n], idx)
    np.testing.assert_array_equal(_bits(packed[:o_n]), _bits(cells))


def _run_lowres(img, flags, f, out_pitch=None):
    h, w = img.shape
    pitch = pitch_for(w)
    ow, oh = -(-w // f), -(-h // f)
    op = out_pitch or pitch_for(ow)
    ctx = ctx_for(w, h)
    try:
        d_img = dev_pitched(img, fill=np.nan)
        d_fl = dev_pitched(flags) if flags is not None else None
        out = torch.full((oh, op), -7.0, device="cuda")
        B.argus_lowres(ctx, d_img, d_fl, B.argus_shape(w, h, pitch), f, out, op)
        torch.cuda.synchronize()
        assert B.argus_sync_status(ctx) == 0
        return out.cpu().numpy(), ow
    finally:
        B.argus_destroy(ctx)


def _check_lowres(ora, img, flags, f, got):
    ref = ora.lowres(img, flags, f)
    mag = ora.lowres(np.abs(img), flags, f)
    tol = (2 * f + 1) * F32_EPS * mag + 1e-30
    err = np.abs(got.astype(np.float64) - ref)
    i = int(np.argmax(err / tol))
    assert (err <= tol).all(), (np.unravel_index(i, err.shape), got.flat[i], ref.flat[i], tol.flat[i])


@pytest.mark.parametrize("w,h,f,use_flags", [
    (1000, 37, 10, True), (1021, 203, 10, False), (517, 77, 3, True), (130, 9, 1, True), (300, 200, 64, True),
    (4096, 21, 7, False)])
def test_lowres_parity(ora, w, h, f, use_flags):
    rng = np.random.default_rng(w + 3 * h + f)
    img = _image(w, h, seed=w * h)
    img.flat[13::1777] = np.inf
    flags = (rng.random((h, w)) < 0.04).astype(np.uint8) if use_flags else None
    got, ow = _run_lowres(img, flags, f)
    _check_lowres(ora, img, flags, f, got[:, :ow])
    assert (got[:, ow:] == -7.0).all()


def test_lowres_fully_masked_blocks_and_out_pitch(ora):
    w, h, f = 95, 41, 10
    img = _image(w, h, seed=1)
    flags = np.zeros((h, w), np.uint8)
    flags[:10, :10] = 1                      # block (0, 0) fully flagged
    img[30:, 90:] = np.nan                   # the bottom-right partial block fully non-finite
    got, ow = _run_lowres(img, flags, f, out_pitch=16)
    assert got[0, 0] == 0.0 and got[4, 9] == 0.0
    _check_lowres(ora, img, flags, f, got[:, :ow])


def test_lowres_full_frame(ora):
    """9576 x 6388 calibrated-like frame to the 13.8 arcsec grid (factor 10)."""
    w, h, f = 9576, 6388, 10
    rng = np.random.default_rng(12)
    img = rng.normal(300, 20, (h, w)).astype(np.float32)
    flags = (rng.random((h, w)) < 0.01).astype(np.uint8)
    got, ow = _run_lowres(img, flags, f)
    _check_lowres(ora, img, flags, f, got[:, :ow])
