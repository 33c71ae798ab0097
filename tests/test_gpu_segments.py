"""Batched segments (persistent kernels + CUDA graph) against the FP64 oracle.

Each segment is fitted over its whole interior (oracle: fit_rect), expanded,
subtracted and searched for sources; the GPU batch does the same for all
segments at once in a packed atlas.  Nothing the GPU computes is fed to the
oracle: the GPU's coefficients are expanded by the library's own expansion
and compared in kernel space (every pixel within 1e-3 of max |K|); the
difference image and its variance are compared with the oracle's own (made
with the oracle's kernel) within the unit-test bars (1e-4 of max(|I|,
|R (x) K|, 1); 1e-5 relative) plus what the kernel and background bars allow
(|dK| <= 1e-3 max|K| per pixel times the window sums of |R| and of V_ref);
detection is checked on the GPU's own atlas by properties that hold at any
size (threshold mask, 8-connected components, peaks, sizes, order).  The
batched subtraction alone, given the oracle's kernels, is compared at the
unit-test bars (argus_segments_subtract).
"""

import numpy as np
import pytest
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300 import synth
from paper_2207_14304_gb300.segments import SegmentBatch
from tests.gpu_helpers import check_detection_properties

pytestmark = pytest.mark.gpu


def _frame(w, h, seed):
    cat = synth.star_catalog(w * h // 150, w, h, seed=seed, flux_min=3e2, flux_max=3e5)
    R, Vr = synth.reference_image(synth.render(cat, w, h, 1.2, sky=300.0), 30, 1.7, seed + 1)
    sig = synth.field_sigma(w, h, 1.5, 2.1)
    I, V = synth.calibrated_image(synth.render(cat, w, h, sig, sky=305.0, shift=(0.3, -0.2)), 1.7, seed + 2)
    rng = np.random.default_rng(seed)
    fl = (rng.random((h, w)) < 0.001).astype(np.uint8)
    return I.numpy(), V.numpy(), R.numpy(), Vr.numpy(), fl


SMALL = (640, 480, [40, 57, 64, 90, 111, 128, 48, 70, 45, 81], 256)
# the batched workload's size range: squares of 64 to 512 px, uneven sides (a ragged atlas of
# several shelves), the largest one pixel short of and exactly at 512
LARGE = (1400, 1100, [512, 256, 300, 77, 64, 419, 128, 511, 97, 333], 1024)


@pytest.mark.parametrize("use_graph,case", [(True, SMALL), (False, SMALL), (True, LARGE)],
                         ids=["graph-small", "direct-small", "graph-large"])
def test_segments_parity(ora, use_graph, case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, h, sides, width = case
    I, V, R, Vr, fl = _frame(w, h, seed=31 + w)
    origins = synth.segment_origins(sides, w, h, seed=3)
    ks = 15
    basis = B.make_basis(ks, (0.7, 1.5, 3.0), (6, 4, 2), 0, 0)
    batch = SegmentBatch(sides, basis=basis, width=width, cfg=B.argus_seg_config(32, 1, 4, 0), src_cap=16384)
    try:
        for i, ((x0, y0), s) in enumerate(zip(origins, sides)):
            sl = (slice(y0, y0 + s), slice(x0, x0 + s))
            for t, a in ((batch.sci, I), (batch.var, V), (batch.ref, R), (batch.ref_var, Vr), (batch.flags, fl)):
                batch.view(t, i).copy_(torch.from_numpy(np.ascontiguousarray(a[sl])))
        for rep in range(2):   # the second run replays the graph (or re-enqueues)
            batch.diff.zero_(); batch.diff_var.zero_()
            batch.run(use_graph=use_graph)
            torch.cuda.synchronize()
            assert B.argus_sync_status(batch.ctx) == 0
        stats = batch.stats_host()
        src, nsrc = batch.sources_host()
        ob = ora.Basis(ksize=ks, spatial_degree=0, bg_degree=0)
        r = ks // 2
        Kd = torch.empty(ks * ks, device="cuda")
        bgd = torch.empty(1, dtype=torch.float64, device="cuda")
        ones = np.ones((1, ks, ks))
        worst = 0.0
        for i, ((x0, y0), s) in enumerate(zip(origins, sides)):
            sl = (slice(y0, y0 + s), slice(x0, x0 + s))
            Is, Vs, Rs, Vrs, Fs = (np.ascontiguousarray(a[sl]) for a in (I, V, R, Vr, fl))
            res = ora.fit_rect(Is, Vs, Rs, Fs, (r, r, s - 1 - r, s - 1 - r), ob)
            assert res.status == 0
            Ko, bgo = ora.expand(ob, res.coeffs)
            # the GPU's coefficients expanded by the library
            B.argus_expand_kernel(batch.ctx, basis, batch.coeffs[i].contiguous(), Kd, bgd)
            torch.cuda.synchronize()
            Kg, bgg = Kd.cpu().numpy().reshape(1, ks, ks), bgd.cpu().numpy()
            kmax = np.abs(Ko).max()
            kerr = np.abs(Kg - Ko).max() / kmax
            worst = max(worst, kerr)
            assert kerr < 1e-3, (i, s, kerr)
            # the background trades off against the kernel sum times the sky level
            sky = float(np.median(Rs))
            dbg = 1e-3 * (abs(bgo[0]) + sky * abs(Ko.sum()))
            assert abs(bgg[0] - bgo[0]) < dbg, (i, bgg, bgo)
            assert stats[i]["status"] == 0
            assert stats[i]["n_pix"] == res.dof + ob.ncoeffs
            # chi2 from the normal equations (t'Wt - 2 c'b + c'Mc) cancels to ~1e-4
            assert abs(stats[i]["chi2"] / res.chi2 - 1) < 1e-3, (i, stats[i]["chi2"], res.chi2)
            # difference and variance against the oracle's, made with the oracle's kernel
            Do, VDo = ora.subtract(Is, Vs, Rs, Vrs, Fs, Ko.astype(np.float32).astype(np.float64), bgo,
                                   sdeg=0, bgdeg=0)
            Dg = batch.view(batch.diff, i).cpu().numpy()
            VDg = batch.view(batch.diff_var, i).cpu().numpy()
            z = np.zeros_like(Is)
            Cabs, _ = ora.subtract(z, Vs, np.abs(Rs), Vrs, Fs, np.abs(Ko), [0.0], sdeg=0, bgdeg=0, with_var=False)
            boxR, _ = ora.subtract(z, Vs, np.abs(Rs), Vrs, Fs, ones, [0.0], sdeg=0, bgdeg=0, with_var=False)
            boxV, _ = ora.subtract(z, Vs, Vrs, Vrs, Fs, ones, [0.0], sdeg=0, bgdeg=0, with_var=False)
            dK = 1e-3 * kmax
            scale = np.maximum(np.maximum(np.abs(Is), -Cabs), 1.0)
            edge = (Do == 0) & (VDo == 0)
            np.testing.assert_array_equal(Dg[edge], 0.0)
            np.testing.assert_array_equal(VDg[edge], 0.0)
            assert (np.abs(Dg - Do) <= 1e-4 * scale + dK * (-boxR) + dbg).all(), i
            assert (np.abs(VDg - VDo) <= 1e-5 * VDo + dK * (2 * kmax + dK) * (-boxV)).all(), i
        # detection on the GPU's own atlas
        assert nsrc <= 16384
        n_p, n_n = check_detection_properties(batch.diff.cpu().numpy(), batch.diff_var.cpu().numpy(),
                                              batch.flags.cpu().numpy(), batch.mask.cpu().numpy(), src, nsrc, 5.0)
        n_checked = n_p + n_n
        print(f"\n[segments graph={use_graph}] {len(sides)} segments, {nsrc} sources, checked {n_checked}, "
              f"worst kernel error {worst:.2e} of max |K|")
    finally:
        batch.close()


def test_segments_subtract_with_the_oracles_kernels(ora):
    """The batched subtraction alone, given the oracle's kernels and backgrounds, against
    the oracle's difference and variance at the unit-test bars (1e-4 of max(|I|,
    |R (x) K|, 1); 1e-5 relative)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, h = 640, 480
    I, V, R, Vr, fl = _frame(w, h, seed=32)
    sides = [40, 57, 64, 90, 111, 128, 48, 70]
    origins = synth.segment_origins(sides, w, h, seed=4)
    ks = 15
    r = ks // 2
    basis = B.make_basis(ks, (0.7, 1.5, 3.0), (6, 4, 2), 0, 0)
    ob = ora.Basis(ksize=ks, spatial_degree=0, bg_degree=0)
    batch = SegmentBatch(sides, basis=basis, width=256, cfg=B.argus_seg_config(32, 1, 4, 0), src_cap=4096)
    try:
        Ks, bgs = [], []
        for i, ((x0, y0), s) in enumerate(zip(origins, sides)):
            sl = (slice(y0, y0 + s), slice(x0, x0 + s))
            for t, a in ((batch.sci, I), (batch.var, V), (batch.ref, R), (batch.ref_var, Vr), (batch.flags, fl)):
                batch.view(t, i).copy_(torch.from_numpy(np.ascontiguousarray(a[sl])))
            res = ora.fit_rect(*(np.ascontiguousarray(a[sl]) for a in (I, V, R)), np.ascontiguousarray(fl[sl]),
                               (r, r, s - 1 - r, s - 1 - r), ob)
            Ko, bgo = ora.expand(ob, res.coeffs)
            Ks.append(Ko.astype(np.float32).reshape(-1))
            bgs.append(float(bgo[0]))
        dK = torch.from_numpy(np.stack(Ks)).cuda()
        dbg = torch.tensor(bgs, dtype=torch.float64, device="cuda")
        batch.diff.fill_(-9.0)
        batch.diff_var.fill_(-9.0)
        B.argus_segments_subtract(batch.plan, batch.sci, batch.var, batch.ref, batch.ref_var, batch.flags, dK, dbg,
                                  batch.diff, batch.diff_var)
        torch.cuda.synchronize()
        assert B.argus_sync_status(batch.ctx) == 0
        for i, ((x0, y0), s) in enumerate(zip(origins, sides)):
            sl = (slice(y0, y0 + s), slice(x0, x0 + s))
            Is, Vs, Rs, Vrs, Fs = (np.ascontiguousarray(a[sl]) for a in (I, V, R, Vr, fl))
            K64 = Ks[i].reshape(1, ks, ks).astype(np.float64)
            Do, VDo = ora.subtract(Is, Vs, Rs, Vrs, Fs, K64, [bgs[i]], sdeg=0, bgdeg=0)
            Cabs, _ = ora.subtract(np.zeros_like(Is), Vs, np.abs(Rs), Vrs, Fs, np.abs(K64), [0.0], sdeg=0, bgdeg=0,
                                   with_var=False)
            Dg = batch.view(batch.diff, i).cpu().numpy()
            VDg = batch.view(batch.diff_var, i).cpu().numpy()
            scale = np.maximum(np.maximum(np.abs(Is), -Cabs), 1.0)
            assert (np.abs(Dg - Do) / scale).max() < 1e-4, i
            assert (np.abs(VDg - VDo) / np.maximum(VDo, 1e-6)).max() < 1e-5, i
    finally:
        batch.close()
