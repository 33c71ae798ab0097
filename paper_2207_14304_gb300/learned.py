"""Learned PSF-matching kernel surrogate over the C ABI (marshalling only).

KernelNet wraps the library's CNN object (argus_cnn_*): parameters live on the
device and every forward, backward, loss and Adam step is a library kernel.
`training_set` makes seeded stamp pairs and their targets with the plain
method (one least-squares kernel per stamp window through the batched
segment path), `KernelNet.fit` trains on them, and `LearnedFit` runs the
per-frame learned fit with the least-squares fit as fallback and judge:

  argus_cnn_prepare -> argus_cnn_forward -> argus_learned_kernel (spatial LS
  across stamps) -> argus_fit_scale_background (one flux scale per spatial
  term and the background by least squares, chi2 on the stamps); if chi2/dof >
  1.1 x the last plain fit's chi2/dof, argus_fit_kernel runs.
"""
from __future__ import annotations

import math
import struct

import numpy as np
import torch

from . import _binding as B
from . import synth
from .segments import SegmentBatch

STAMP = 21
NPX = STAMP * STAMP
WIN = STAMP + 20            # fit window of a stamp: 21x21 interior for a 21x21 kernel
CKPT_MAGIC = b"ARGUSCNN"


class _DevArray:
    """__cuda_array_interface__ view of a library-owned device buffer."""

    def __init__(self, ptr, n, typestr="<f4"):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


class KernelNet:
    """precision: "bf16_split" (BF16 weights, the forward on the tensor cores with
    activations as BF16 hi + lo parts), "bf16" (BF16 weights, CUDA-core kernels) or
    "fp32"; the backward runs on the CUDA cores in every mode."""

    def __init__(self, device=0, max_batch=1024, seed=1, precision="bf16_split"):
        self.device = torch.device("cuda", device)
        self.max_batch = int(max_batch)
        self.net = B.argus_cnn_create(device, max_batch, seed)
        self.precision = precision
        B.argus_cnn_set_state(self.net, precision, 0)

    def close(self):
        if self.net is not None:
            B.argus_cnn_destroy(self.net)
            self.net = None

    def tensors(self):
        """(master, adam_m, adam_v) as torch views of the library's device memory."""
        (pm, pa, pv), n, _ = B.argus_cnn_params(self.net)
        return tuple(torch.as_tensor(_DevArray(p, n), device=self.device) for p in (pm, pa, pv))

    @property
    def step(self):
        return B.argus_cnn_params(self.net)[2]

    def set_precision(self, precision):
        self.precision = precision
        B.argus_cnn_set_state(self.net, precision, self.step)

    # checkpoint: magic, u32 version, u64 count, u32 step, then master, m, v (little-endian FP32)
    def save(self, path):
        master, m, v = (t.cpu().numpy() for t in self.tensors())
        with open(path, "wb") as f:
            f.write(CKPT_MAGIC + struct.pack("<IQI", 1, master.size, self.step))
            for a in (master, m, v):
                f.write(a.astype("<f4").tobytes())

    def load(self, path):
        with open(path, "rb") as f:
            if f.read(8) != CKPT_MAGIC:
                raise ValueError("not an argus CNN checkpoint")
            ver, n, step = struct.unpack("<IQI", f.read(16))
            arrs = [np.frombuffer(f.read(4 * n), dtype="<f4") for _ in range(3)]
        for dst, a in zip(self.tensors(), arrs):
            if dst.numel() != n:
                raise ValueError("parameter count mismatch")
            dst.copy_(torch.from_numpy(a.copy()))
        B.argus_cnn_set_state(self.net, self.precision, step)

    def forward(self, x, y=None):
        n = x.shape[0]
        y = y if y is not None else torch.empty((n, NPX), dtype=torch.float32, device=self.device)
        for s in range(0, n, self.max_batch):
            e = min(n, s + self.max_batch)
            B.argus_cnn_forward(self.net, x[s:e], e - s, y[s:e])
        return y

    def fit(self, x, target, *, epochs=10, batch=512, lr=1e-3, lr_end=None, seed=0, log=None):
        """Minibatch Adam on the library kernels; returns the per-epoch mean loss.
        With lr_end the rate follows a cosine from lr to lr_end over all steps."""
        n = x.shape[0]
        total = max(1, epochs * (n // batch))
        step = 0
        g = torch.Generator(device=self.device)
        g.manual_seed(seed)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        hist = []
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g, device=self.device)
            tot = torch.zeros((), dtype=torch.float64, device=self.device)
            nb = 0
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                xb = x.index_select(0, idx).contiguous()
                tb = target.index_select(0, idx).contiguous()
                rate = lr if lr_end is None else lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * step / total))
                B.argus_cnn_train_step(self.net, xb, tb, batch, rate, loss)
                step += 1
                tot += loss[0]
                nb += 1
            hist.append(float(tot.item()) / max(nb, 1))
            if log:
                log(f"epoch {ep}: loss {hist[-1]:.4e}")
        return hist


TRAIN_CHUNK = 32768   # pairs per batched-segment run (one run's per-segment scratch)


def training_set(n, seed=5, device=0, sky=300.0, flux=(1e4, 1e6), sig_ref=1.0, sig_range=(1.0, 3.0),
                 jump_p=0.1, ctx=None, crowd=None):
    """Seeded stamp pairs and plain-method targets, generated in chunks of at most
    TRAIN_CHUNK pairs (chunk c uses seed + 1000 c); see `_training_chunk`.

    crowd: None (one star per window) or (mean count, flux_min, flux_max, index):
    each window also holds Poisson(mean count) field stars at uniform positions
    (over the window and a 5-px border) with dN/dF ~ F**index fluxes, rendered in
    both images."""
    xs, ts, sigs = [], [], []
    for c, s0 in enumerate(range(0, n, TRAIN_CHUNK)):
        x, t, sg = _training_chunk(min(TRAIN_CHUNK, n - s0), seed + 1000 * c, device, sky, flux, sig_ref,
                                   sig_range, jump_p, ctx, crowd)
        xs.append(x)
        ts.append(t)
        sigs.append(sg)
    if len(xs) == 1:
        return xs[0], ts[0], sigs[0]
    return torch.cat(xs), torch.cat(ts), np.concatenate(sigs)


def field_stars(n, seed, mean, flux_min, flux_max, index, border=5.0, device="cpu"):
    """Field stars for n windows of WIN x WIN pixels: Poisson(mean) per window,
    positions uniform over the window plus `border` pixels, power-law fluxes.
    Returns (window index [m] int64, x [m], y [m], flux [m]) as float64 tensors."""
    g = torch.Generator().manual_seed(seed)
    cnt = torch.poisson(torch.full((n,), float(mean), dtype=torch.float64), generator=g).to(torch.int64)
    m = int(cnt.sum())
    widx = torch.repeat_interleave(torch.arange(n, dtype=torch.int64), cnt)
    pos = torch.rand(m, 2, generator=g, dtype=torch.float64) * (WIN + 2 * border) - border
    f = synth.power_law_fluxes(m, seed + 1, flux_min, flux_max, index)
    dev = torch.device(device)
    return widx.to(dev), pos[:, 0].to(dev), pos[:, 1].to(dev), f.to(dev)


def render_field(n, stars, sigma, device="cpu"):
    """Expected electrons of field stars in n windows (FP32 [n, WIN, WIN]):
    pixel-integrated Gaussians of width sigma (a float or a per-window array).
    Stars are added in passes of at most one star per window (the k-th star of
    every window in pass k), so the sums do not depend on scheduling."""
    widx, x, y, f = stars
    dev = torch.device(device)
    img = torch.zeros((n, WIN, WIN), dtype=torch.float32, device=dev)
    if widx.numel() == 0:
        return img
    sig = torch.as_tensor(sigma, dtype=torch.float64, device=dev)
    if sig.dim() == 0:
        sig = sig.expand(n)
    order = torch.argsort(widx, stable=True)
    widx, x, y, f = widx[order], x[order], y[order], f[order]
    rank = torch.arange(widx.numel(), device=widx.device) - torch.searchsorted(widx, widx)
    ax = torch.arange(WIN, dtype=torch.float64, device=dev)
    phi = lambda z: 0.5 * (1 + torch.erf(z / math.sqrt(2)))
    for k in range(int(rank.max()) + 1):
        sel = rank == k
        w, cx, cy, fl = widx[sel], x[sel][:, None], y[sel][:, None], f[sel]
        sw = sig[w][:, None]
        fx = phi((ax + 0.5 - cx) / sw) - phi((ax - 0.5 - cx) / sw)
        fy = phi((ax + 0.5 - cy) / sw) - phi((ax - 0.5 - cy) / sw)
        img[w] += (fl[:, None, None] * fy[:, :, None] * fx[:, None, :]).to(torch.float32)
    return img


def _training_chunk(n, seed, device, sky, flux, sig_ref, sig_range, jump_p, ctx, crowd=None):
    """Seeded stamp pairs and plain-method targets.

    Each pair is a 41x41 window with one star near its centre (plus, with crowd,
    the field stars of `field_stars`); the science PSF
    width follows a sequence with seeing jumps (redrawn from U(1, 3) px with
    probability jump_p per stamp), the reference is at 1 px with the noise of a
    30-frame average.  The target is the 21x21 least-squares kernel fitted over
    the window's 21x21 interior by the batched segment path (Alard-Lupton basis,
    degree 0).  Returns (x [n, 441, 2], target [n, 441]) on the device.
    """
    dev = torch.device("cuda", device)
    g = torch.Generator().manual_seed(seed)
    sig = np.empty(n)
    cur = float(torch.empty(1).uniform_(*sig_range, generator=g))
    jumps = torch.rand(n, generator=g).numpy()
    redraw = torch.empty(n).uniform_(*sig_range, generator=g).numpy()
    for i in range(n):
        if jumps[i] < jump_p:
            cur = float(redraw[i])
        sig[i] = cur
    lf = torch.empty(n, dtype=torch.float64).uniform_(math.log(flux[0]), math.log(flux[1]), generator=g)
    F = torch.exp(lf).to(dev)
    off = (torch.rand(n, 2, generator=g, dtype=torch.float64) - 0.5).to(dev)
    ax = torch.arange(WIN, dtype=torch.float64, device=dev)

    def render(s):
        s = torch.as_tensor(s, dtype=torch.float64, device=dev)[:, None]
        cx = (WIN - 1) / 2 + off[:, 0:1]
        cy = (WIN - 1) / 2 + off[:, 1:2]
        phi = lambda z: 0.5 * (1 + torch.erf(z / math.sqrt(2)))
        fx = phi((ax + 0.5 - cx) / s) - phi((ax - 0.5 - cx) / s)
        fy = phi((ax + 0.5 - cy) / s) - phi((ax - 0.5 - cy) / s)
        return (F[:, None, None] * fy[:, :, None] * fx[:, None, :]).to(torch.float32)

    Rexp = render(np.full(n, sig_ref)) + sky
    Iexp = render(sig) + sky
    if crowd is not None:
        stars = field_stars(n, seed + 13, *crowd, device=dev)
        Rexp += render_field(n, stars, sig_ref, device=dev)
        Iexp += render_field(n, stars, sig, device=dev)
        del stars
    R, Vr = synth.reference_image(Rexp, 30, 1.7, seed + 11)
    I, V = synth.calibrated_image(Iexp, 1.7, seed + 12)
    basis = B.make_basis(STAMP, (0.7, 1.5, 3.0), (6, 4, 2), 0, 0)
    batch = SegmentBatch([WIN] * n, basis=basis, width=2016, ctx=ctx, cfg=B.argus_seg_config(8, 1, 4, 0))
    try:
        per = 2016 // 48
        rows = (n + per - 1) // per

        def place(dst, src):
            buf = torch.zeros((rows * per, 48, 48), dtype=src.dtype, device=dev)
            buf[:n, :WIN, :WIN] = src
            dst[: rows * 48, :2016].copy_(buf.view(rows, per, 48, 48).permute(0, 2, 1, 3).reshape(rows * 48, 2016))

        place(batch.sci, I)
        place(batch.var, V)
        place(batch.ref, R)
        place(batch.ref_var, Vr)
        batch.run(use_graph=False, detect=False)
        K = torch.empty((n, NPX), dtype=torch.float32, device=dev)
        B.argus_segments_kernels(batch.plan, K, None)
        cen = torch.tensor([(c + WIN // 2, r + WIN // 2) for r, c in batch.pos], dtype=torch.int32, device=dev)
        cnt = torch.tensor([n, 0, 0, 0], dtype=torch.int32, device=dev)
        x = torch.empty((n, NPX, 2), dtype=torch.float32, device=dev)
        B.argus_cnn_prepare(batch.sci, batch.ref, B.argus_shape(batch.pitch, batch.atlas_h, batch.pitch), cen, cnt,
                            n, x)
        torch.cuda.synchronize(dev)
        st = batch.stats_host()
        ok = torch.from_numpy(st["status"] == 0).to(dev)
        return x[ok].contiguous(), K[ok].contiguous(), sig[st["status"] == 0]
    finally:
        batch.close()


class LearnedFit:
    """Per-frame learned kernel with the least-squares fit as fallback and judge."""

    def __init__(self, pipe, net: KernelNet, *, ratio=1.1, fit_scale=True):
        self.pipe = pipe              # a FramePipeline (its basis must have ksize 21)
        self.net = net
        self.ratio = float(ratio)
        self.fit_scale = bool(fit_scale)   # fit one flux scale per spatial term with the background
        if pipe.basis.ksize != STAMP:
            raise ValueError("the learned kernel is 21x21")
        self.x = torch.zeros((pipe.max_stamps, NPX, 2), dtype=torch.float32, device=pipe.device)
        self.y = torch.zeros((pipe.max_stamps, NPX), dtype=torch.float32, device=pipe.device)
        self.stats = torch.zeros(128, dtype=torch.uint8, device=pipe.device)
        self.plain_chi2_dof = None
        self.n_learned = 0
        self.n_fallback = 0

    def learned_kernel(self, ref, stream=None):
        """CNN kernels -> K_k and background; returns nothing (results on the device)."""
        p = self.pipe
        B.argus_cnn_prepare(p.img, ref, p.shape, p.centers, p.n_stamps, p.max_stamps, self.x, stream)
        B.argus_cnn_forward(self.net.net, self.x, p.max_stamps, self.y, stream)
        B.argus_learned_kernel(p.ctx, self.y, p.centers, p.n_stamps, p.max_stamps, p.w, p.h,
                               p.basis.spatial_degree, p.K, stream)
        fit = B.argus_fit_scale_background if self.fit_scale else B.argus_fit_background
        fit(p.ctx, p.img, p.var, ref, p.flags, p.shape, p.centers, p.n_stamps, p.max_stamps, p.stamp, p.K,
            p.basis.ksize, p.basis.spatial_degree, p.basis.bg_degree, p.bg, self.stats, stream)

    def plain(self, ref, stream=None):
        self.pipe.fit(ref, stream)
        st = self.pipe.fit_stats()
        self.plain_chi2_dof = st["chi2"] / max(st["dof"], 1)
        return st

    def run(self, raw, calib, ref, ref_var, stream=None):
        """One frame: learned kernel unless its chi2/dof exceeds ratio x the last plain fit's."""
        p = self.pipe
        p.calibrate(raw, calib, stream)
        p.select_stamps(ref, stream)
        used_plain = False
        if self.plain_chi2_dof is None:
            self.plain(ref, stream)
            used_plain = True
        else:
            self.learned_kernel(ref, stream)
            st = B.fit_stats_from_bytes(self.stats)
            c2 = st["chi2"] / max(st["dof"], 1)
            if st["status"] != 0 or not (c2 <= self.ratio * self.plain_chi2_dof):
                self.n_fallback += 1
                self.plain(ref, stream)
                used_plain = True
            else:
                self.n_learned += 1
        p.subtract(ref, ref_var, stream)
        p.detect(stream)
        return used_plain
