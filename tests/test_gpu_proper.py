"""ZOGY (Sec. 4.2) and the proper coadd (Sec. 4.1.3) on the GPU against the FP64
oracle, tile by tile.

Tolerances, from the FP32 rounding of the image transforms (the PSF
transforms are FP64): with u = 2^-24 and the unit
  e = u log2(T^2) (||N||_2 / s_n + ||R||_2 / s_r) / T
(the rms rounding of a T^2-point FP32 FFT carried through the quotient, whose
gain is at most 1/s_n and 1/s_r), |dD| <= 8 e and |dS| <= 8 (e F_D ||P_D||_1 +
u log2(T^2) ||D||_2 / T) (S filters D with F_D P_D and shares D's inverse
transform); an FP32 emulation of the same algorithm (numpy's
single-precision FFT) stays within 1.4 e and 3.1 e F_D ||P_D||_1 on these
tiles.  P_D within 64 u max|P_D|, sigma_S within 1e-6 relative.

The kernels have not run on a GPU yet, so the file is skipped until they have.
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


def _gauss(sig, half=15):
    u = np.arange(-half, half + 1)
    g = np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2 * sig * sig))
    return (g / g.sum()).astype(np.float32)


def _frame(w, h, seed, sn, sr, psf_n, psf_r, Fn, Fr):
    from oracle import proper
    rng = np.random.default_rng(seed)
    sky = np.zeros((h, w))
    n = w * h // 130
    np.add.at(sky, (rng.integers(0, h, n), rng.integers(0, w, n)), 1e2 * 1e4 ** rng.random(n))
    conv = lambda img, P: np.fft.ifft2(np.fft.fft2(img) * np.fft.fft2(proper.psf_on_tile(P, img.shape))).real
    N = (Fn * conv(sky, psf_n) + rng.normal(0, sn, (h, w))).astype(np.float32)
    R = (Fr * conv(sky, psf_r) + rng.normal(0, sr, (h, w))).astype(np.float32)
    return N, R


@pytest.mark.parametrize("T,origins", [(256, [(0, 0), (300, 100), (520, 260)]), (512, [(64, 32)]),
                                       (1024, [(0, 0)])])
def test_zogy_parity(ora, T, origins):
    from oracle import proper
    w, h = 800, 600 if T < 1024 else 1024
    w = max(w, T)
    specs = [(1.05, 1.0, 18.0, 3.3, 2.0, 1.2), (0.9, 1.1, 10.0, 4.0, 1.3, 1.6), (1.0, 1.0, 7.0, 7.0, 2.2, 2.2)]
    N, R = _frame(w, h, seed=T, sn=12.0, sr=3.0, psf_n=_gauss(1.8), psf_r=_gauss(1.3), Fn=1.0, Fr=1.0)
    rec = np.zeros(len(origins), B.ZOGY_TILE_DTYPE)
    pn = np.zeros((len(origins), 31, 31), np.float32)
    pr = np.zeros_like(pn)
    for i, (x0, y0) in enumerate(origins):
        Fn, Fr, sn, sr, gn, gr = specs[i % len(specs)]
        rec[i] = (x0, y0, Fn, Fr, sn, sr)
        pn[i], pr[i] = _gauss(gn), _gauss(gr)
    nt = len(origins)
    plan = B.proper_plan_create(0, T, 4)
    try:
        pitch = pitch_for(w)
        dN, dR = dev_pitched(N), dev_pitched(R)
        d_rec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
        D = torch.full((nt, T, T), -7.0, device="cuda")
        S = torch.full((nt, T, T), -7.0, device="cuda")
        PD = torch.full((nt, T, T), -7.0, device="cuda")
        sig = torch.zeros(nt, dtype=torch.float64, device="cuda")
        B.argus_zogy(plan, dN, dR, B.argus_shape(w, h, pitch), d_rec, nt, torch.from_numpy(pn).cuda(),
                     torch.from_numpy(pr).cuda(), 31, 1e-8, D, S, PD, sig)
        torch.cuda.synchronize()
        D, S, PD, sig = D.cpu().numpy(), S.cpu().numpy(), PD.cpu().numpy(), sig.cpu().numpy()
    finally:
        B.proper_plan_destroy(plan)
    for i, (x0, y0) in enumerate(origins):
        Fn, Fr, sn, sr = (float(rec[i][k]) for k in ("Fn", "Fr", "sn", "sr"))
        tN = np.zeros((T, T), np.float32)
        tR = np.zeros((T, T), np.float32)
        ys, xs = slice(y0, min(y0 + T, h)), slice(x0, min(x0 + T, w))
        tN[: ys.stop - y0, : xs.stop - x0] = N[ys, xs]
        tR[: ys.stop - y0, : xs.stop - x0] = R[ys, xs]
        o = proper.zogy(tN, tR, pn[i].astype(np.float64), pr[i].astype(np.float64), Fn, Fr, sn, sr)
        e = F32_EPS * math.log2(T * T) * (np.linalg.norm(tN) / sn + np.linalg.norm(tR) / sr) / T
        dD = np.abs(D[i] - o["D"]).max()
        # S filters D with F_D P_D and shares D's inverse transform
        sS = e * o["F_D"] * np.abs(o["P_D"]).sum() + F32_EPS * math.log2(T * T) * np.linalg.norm(o["D"]) / T
        dS = np.abs(S[i] - o["S"]).max()
        print(f"\n[zogy T={T} tile {i}] |dD| {dD:.2e} = {dD / e:.2f} e   |dS| = {dS / sS:.2f} e F_D |P_D|_1")
        assert dD <= 8 * e
        assert dS <= 8 * sS
        assert np.abs(PD[i] - o["P_D"]).max() <= 64 * F32_EPS * np.abs(o["P_D"]).max()
        assert abs(sig[i] / o["sigma_S"] - 1) < 1e-6


@pytest.mark.parametrize("T,J", [(256, 3), (512, 2)])
def test_proper_coadd_parity(ora, T, J):
    """Proper coadd (Sec. 4.1.3) through the entry point against the oracle per tile:
    R within 8 e_R, S within 8 e_S (the units of tests/test_host_kernels.py), P_R
    within 64 ulps of its maximum, F_R and sigma_S within 1e-6."""
    from oracle import proper
    w, h = 700, 600
    rng = np.random.default_rng(T + J)
    sky = np.zeros((h, w))
    n = w * h // 150
    np.add.at(sky, (rng.integers(0, h, n), rng.integers(0, w, n)), 1e2 * 1e4 ** rng.random(n))
    conv = lambda img, P: np.fft.ifft2(np.fft.fft2(img) * np.fft.fft2(proper.psf_on_tile(P, img.shape))).real
    origins = [(0, 0), (400, 300)] if T == 256 else [(100, 50)]
    nt = len(origins)
    gs = [1.2, 1.9, 1.5][:J]
    F = np.array([1.0, 0.8, 1.2][:J], np.float32)
    sg = np.array([5.0, 9.0, 4.0][:J], np.float32)
    frames = [(f * conv(sky, _gauss(g)) + rng.normal(0, s, (h, w))).astype(np.float32) for g, f, s in zip(gs, F, sg)]
    psfs = np.stack([np.stack([_gauss(g + 0.1 * t) for g in gs]) for t in range(nt)])     # [nt][J][31][31]
    pitch = pitch_for(w)
    plan = B.proper_plan_create(0, T, 4)
    try:
        stack = torch.zeros((J, h, pitch), device="cuda")
        for j in range(J):
            stack[j, :, :w] = torch.from_numpy(frames[j]).cuda()
        d_org = torch.tensor(origins, dtype=torch.int32, device="cuda")
        S = torch.full((nt, T, T), -7.0, device="cuda")
        R = torch.full((nt, T, T), -7.0, device="cuda")
        PR = torch.full((nt, T, T), -7.0, device="cuda")
        FR = torch.zeros(1, dtype=torch.float64, device="cuda")
        sig = torch.zeros(nt, dtype=torch.float64, device="cuda")
        B.argus_proper_coadd(plan, stack, J, B.argus_shape(w, h, pitch), d_org, nt, torch.from_numpy(F).cuda(),
                             torch.from_numpy(sg).cuda(), torch.from_numpy(psfs).cuda(), 31, 1e-8, S, R, PR, FR, sig)
        torch.cuda.synchronize()
        S, R, PR, FR, sig = (t.cpu().numpy() for t in (S, R, PR, FR, sig))
    finally:
        B.proper_plan_destroy(plan)
    for i, (x0, y0) in enumerate(origins):
        Ms = [np.ascontiguousarray(f[y0:y0 + T, x0:x0 + T]) for f in frames]
        Ps = [psfs[i, j].astype(np.float64) for j in range(J)]
        o = proper.proper_coadd(Ms, Ps, [float(f) for f in F], [float(s) for s in sg])
        lg = F32_EPS * math.log2(T * T) / T
        eR = lg * sum(np.linalg.norm(M) / s for M, s in zip(Ms, sg))
        eS = lg * (sum(f / s ** 2 * np.abs(P).sum() * np.linalg.norm(M) for M, P, f, s in zip(Ms, Ps, F, sg))
                   + np.linalg.norm(o["R"]))
        assert np.abs(R[i] - o["R"]).max() <= 8 * eR
        assert np.abs(S[i] - o["S"]).max() <= 8 * eS
        assert np.abs(PR[i] - o["P_R"]).max() <= 64 * F32_EPS * np.abs(o["P_R"]).max()
        assert abs(FR[0] / o["F_R"] - 1) < 1e-6 and abs(sig[i] / o["sigma_S"] - 1) < 1e-6


def test_zogy_reuses_psf_transforms_and_coadd_discards_them(ora):
    """A call without PSFs gives the outputs of the call that supplied them, bit for bit;
    after a proper-coadd call on the plan it is refused."""
    T, w, h = 256, 600, 400
    N, R = _frame(w, h, seed=5, sn=12.0, sr=3.0, psf_n=_gauss(1.8), psf_r=_gauss(1.3), Fn=1.0, Fr=1.0)
    rec = np.zeros(2, B.ZOGY_TILE_DTYPE)
    rec[0] = (0, 0, 1.0, 1.0, 12.0, 3.0)
    rec[1] = (300, 100, 1.0, 1.0, 12.0, 3.0)
    pn = np.stack([_gauss(1.8), _gauss(1.9)])
    pr = np.stack([_gauss(1.3), _gauss(1.3)])
    pitch = pitch_for(w)
    plan = B.proper_plan_create(0, T, 2)
    try:
        dN, dR = dev_pitched(N), dev_pitched(R)
        d_rec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
        sh = B.argus_shape(w, h, pitch)
        D1 = torch.empty((2, T, T), device="cuda")
        S1 = torch.empty((2, T, T), device="cuda")
        D2 = torch.empty((2, T, T), device="cuda")
        S2 = torch.empty((2, T, T), device="cuda")
        B.argus_zogy(plan, dN, dR, sh, d_rec, 2, torch.from_numpy(pn).cuda(), torch.from_numpy(pr).cuda(), 31, 1e-8,
                     D1, S1)
        B.argus_zogy(plan, dN, dR, sh, d_rec, 2, None, None, 31, 1e-8, D2, S2)
        torch.cuda.synchronize()
        assert torch.equal(D1, D2) and torch.equal(S1, S2)
        stack = dN.unsqueeze(0).contiguous()
        org = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
        one = torch.ones(1, device="cuda")
        B.argus_proper_coadd(plan, stack, 1, sh, org, 1, one, one, torch.from_numpy(pn[:1]).cuda(), 31, 1e-8,
                             torch.empty((1, T, T), device="cuda"), torch.empty((1, T, T), device="cuda"))
        with pytest.raises(B.ArgusError):
            B.argus_zogy(plan, dN, dR, sh, d_rec, 2, None, None, 31, 1e-8, D2, S2)
    finally:
        B.proper_plan_destroy(plan)


def test_shared_psfs_match_per_tile_copies(ora):
    """One PSF (pair) shared by every tile gives, bit for bit, what the same PSF copied
    into every tile gives, for ZOGY (also when reused) and for the proper coadd."""
    T, w, h, nt = 256, 700, 500, 3
    N, R = _frame(w, h, seed=6, sn=12.0, sr=3.0, psf_n=_gauss(1.8), psf_r=_gauss(1.3), Fn=1.0, Fr=1.0)
    rec = np.zeros(nt, B.ZOGY_TILE_DTYPE)
    for i, (x0, y0) in enumerate([(0, 0), (300, 100), (420, 240)]):
        rec[i] = (x0, y0, 1.0, 1.0, 12.0, 3.0)
    pn, pr = _gauss(1.8), _gauss(1.3)
    pitch = pitch_for(w)
    sh = B.argus_shape(w, h, pitch)
    plan = B.proper_plan_create(0, T, nt)
    try:
        dN, dR = dev_pitched(N), dev_pitched(R)
        d_rec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
        out = [torch.empty((nt, T, T), device="cuda") for _ in range(6)]
        B.argus_zogy(plan, dN, dR, sh, d_rec, nt, torch.from_numpy(np.stack([pn] * nt)).cuda(),
                     torch.from_numpy(np.stack([pr] * nt)).cuda(), 31, 1e-8, out[0], out[1])
        B.argus_zogy(plan, dN, dR, sh, d_rec, nt, torch.from_numpy(pn).cuda(), torch.from_numpy(pr).cuda(), 31, 1e-8,
                     out[2], out[3], psf_per_tile=False)
        B.argus_zogy(plan, dN, dR, sh, d_rec, nt, None, None, 31, 1e-8, out[4], out[5], psf_per_tile=False)
        torch.cuda.synchronize()
        for a, b in ((0, 2), (1, 3), (0, 4), (1, 5)):
            assert torch.equal(out[a], out[b]), (a, b)
        with pytest.raises(B.ArgusError):       # per-tile reuse after a shared call: nothing to reuse
            B.argus_zogy(plan, dN, dR, sh, d_rec, nt, None, None, 31, 1e-8, out[4], out[5])
        J = 3
        stack = torch.stack([dN, dR, dN]).contiguous()
        org = torch.tensor([(0, 0), (300, 100), (420, 240)], dtype=torch.int32, device="cuda")
        F = torch.ones(J, device="cuda")
        sg = torch.tensor([12.0, 3.0, 12.0], device="cuda")
        ps = np.stack([_gauss(g) for g in (1.8, 1.3, 1.6)])
        S1, R1, S2, R2 = (torch.empty((nt, T, T), device="cuda") for _ in range(4))
        B.argus_proper_coadd(plan, stack, J, sh, org, nt, F, sg, torch.from_numpy(np.stack([ps] * nt)).cuda(), 31, 1e-8,
                             S1, R1)
        B.argus_proper_coadd(plan, stack, J, sh, org, nt, F, sg, torch.from_numpy(ps).cuda(), 31, 1e-8, S2, R2,
                             psf_per_tile=False)
        torch.cuda.synchronize()
        assert torch.equal(S1, S2) and torch.equal(R1, R2)
    finally:
        B.proper_plan_destroy(plan)
