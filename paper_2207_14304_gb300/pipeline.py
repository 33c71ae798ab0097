"""Per-frame difference-imaging pipeline over the C ABI (marshalling only).

FramePipeline owns the device buffers of one camera's frame path and calls the
library entry points in the order of the paper's per-frame reduction
(Sec. 4: calibration on the GPU, then -- here also on the GPU -- the kernel
fit, subtraction and detection of Sec. 4.2):

  argus_calibrate -> argus_select_stamps -> argus_fit_kernel ->
  argus_expand_kernel -> argus_subtract -> argus_detect

All buffers are allocated once, in __init__, like the reference and
calibration frames the paper pre-allocates per pointing; run() allocates
nothing, and capture() records it as one CUDA graph (the frame's ~50 kernel
launches replayed without host launch gaps).
"""
from __future__ import annotations

import torch

from . import _binding as B
from .synth import pitch_for


class FramePipeline:
    def __init__(self, w: int, h: int, *, basis: B.argus_basis, stamp: int = 21, grid=(8, 8),
                 precision: str = "fp32", nsigma: float = 5.0, psf_sigma: float = 1.8,
                 max_peak: float = 3.0e4, iso: int = 10, iso_frac: float = 0.1,
                 src_cap: int = 1 << 16, det_cap: int = 1 << 22, device: int = 0, ctx=None):
        self.w, self.h = int(w), int(h)
        self.pitch = pitch_for(self.w)
        self.shape = B.argus_shape(self.w, self.h, self.pitch)
        self.basis = basis
        self.nb, self.Ks, self.Kb, self.Nc = B.basis_counts(basis)
        self.stamp = int(stamp)
        self.grid = tuple(grid)
        self.max_stamps = grid[0] * grid[1]
        self.precision = precision
        self.nsigma, self.psf_sigma = float(nsigma), float(psf_sigma)
        self.max_peak, self.iso, self.iso_frac = float(max_peak), int(iso), float(iso_frac)
        self.src_cap = int(src_cap)
        dev = torch.device("cuda", device)
        self.device = dev
        hp = (self.h, self.pitch)
        self.img = torch.zeros(hp, dtype=torch.float32, device=dev)
        self.var = torch.zeros(hp, dtype=torch.float32, device=dev)
        self.flags = torch.zeros(hp, dtype=torch.uint8, device=dev)
        self.diff = torch.zeros(hp, dtype=torch.float32, device=dev)
        self.diff_var = torch.zeros(hp, dtype=torch.float32, device=dev)
        self.mask = torch.zeros(hp, dtype=torch.uint8, device=dev)
        self.centers = torch.zeros((self.max_stamps, 2), dtype=torch.int32, device=dev)
        self.n_stamps = torch.zeros(4, dtype=torch.int32, device=dev)
        self.coeffs = torch.zeros(self.Nc, dtype=torch.float64, device=dev)
        self.stats = torch.zeros(128, dtype=torch.uint8, device=dev)
        ks = basis.ksize
        self.K = torch.zeros(self.Ks * ks * ks, dtype=torch.float32, device=dev)
        self.bg = torch.zeros(max(self.Kb, 1), dtype=torch.float64, device=dev)
        self.sources = torch.zeros(self.src_cap * B.SOURCE_BYTES, dtype=torch.uint8, device=dev)
        self.n_found = torch.zeros(4, dtype=torch.int32, device=dev)
        self.ctx = ctx if ctx is not None else B.argus_create(
            device, self.h * self.pitch, self.max_stamps, max(self.Nc, 64), det_cap)
        self._own_ctx = ctx is None

    def close(self):
        if self._own_ctx and self.ctx is not None:
            B.argus_destroy(self.ctx)
            self.ctx = None

    def calibrate(self, raw, calib, stream=None):
        B.argus_calibrate(self.ctx, raw, self.shape, calib, self.img, self.var, self.flags, stream)

    def select_stamps(self, ref, stream=None):
        B.argus_select_stamps(self.ctx, ref, self.flags, self.shape, self.grid[0], self.grid[1],
                              self.stamp, (self.basis.ksize - 1) // 2, self.max_peak, self.iso,
                              self.iso_frac, self.centers, self.n_stamps, stream)

    def fit(self, ref, stream=None):
        B.argus_fit_kernel(self.ctx, self.img, self.var, ref, self.flags, self.shape, self.centers,
                           self.n_stamps, self.max_stamps, self.stamp, self.basis, self.precision,
                           self.coeffs, self.stats, stream)
        B.argus_expand_kernel(self.ctx, self.basis, self.coeffs, self.K, self.bg, stream)

    def subtract(self, ref, ref_var, stream=None):
        B.argus_subtract(self.ctx, self.img, self.var, ref, ref_var, self.flags, self.shape, self.w,
                         self.h, 0, 0, self.basis.ksize, self.basis.spatial_degree, self.K,
                         self.basis.bg_degree, self.bg, self.diff, self.diff_var, stream)

    def subtract_variance(self, ref_var, stream=None):
        """The difference variance alone (the first half of `subtract`)."""
        B.argus_subtract(self.ctx, None, self.var, None, ref_var, self.flags, self.shape, self.w,
                         self.h, 0, 0, self.basis.ksize, self.basis.spatial_degree, self.K,
                         self.basis.bg_degree, self.bg, None, self.diff_var, stream)

    def subtract_difference(self, ref, ref_var, stream=None):
        """The difference image alone (the second half of `subtract`)."""
        B.argus_subtract(self.ctx, self.img, self.var, ref, ref_var, self.flags, self.shape, self.w,
                         self.h, 0, 0, self.basis.ksize, self.basis.spatial_degree, self.K,
                         self.basis.bg_degree, self.bg, self.diff, None, stream)

    def detect(self, stream=None):
        B.argus_detect(self.ctx, self.diff, self.diff_var, self.flags, self.shape, self.nsigma,
                       self.psf_sigma, self.mask, self.sources, self.src_cap, self.n_found, stream)

    def run_fused(self, raw, calib, ref, ref_var, stream=None):
        """The same frame through argus_dia_frame: one library call for the whole path."""
        B.argus_dia_frame(self.ctx, raw, self.shape, calib, ref, ref_var, self.grid[0], self.grid[1], self.stamp,
                          self.max_peak, self.iso, self.iso_frac, self.basis, self.precision, self.nsigma,
                          self.psf_sigma, self.img, self.var, self.flags, self.centers, self.n_stamps, self.coeffs,
                          self.stats, self.K, self.bg, self.diff, self.diff_var, self.mask, self.sources,
                          self.src_cap, self.n_found, stream)

    def run(self, raw, calib, ref, ref_var, stream=None, select=True):
        """One frame through the whole path; all outputs stay on the device."""
        self.calibrate(raw, calib, stream)
        if select:
            self.select_stamps(ref, stream)
        self.fit(ref, stream)
        self.subtract(ref, ref_var, stream)
        self.detect(stream)

    def capture(self, raw, calib, ref, ref_var, stream, select=True, pre=None, post=None, fused=False):
        """Record one frame of run() as a CUDA graph on `stream` (a side stream, not the
        default one), after at least one eager run() with the same arguments (the basis is
        prepared then).  pre() and post() are recorded before and after the frame (e.g. the
        host-to-device copy of the raw frame and the copy of the sources back).  Replaying
        the graph (graph.replay() under torch.cuda.stream(s)) repeats the whole path with
        the same buffers and launches; fused=True records run_fused (argus_dia_frame) instead.
        Returns (graph, library kernel launches per frame)."""
        g = torch.cuda.CUDAGraph()
        n0 = B.argus_launch_count()
        with torch.cuda.graph(g, stream=stream):
            if pre is not None:
                pre()
            if fused:
                self.run_fused(raw, calib, ref, ref_var, stream)
            else:
                self.run(raw, calib, ref, ref_var, stream, select=select)
            if post is not None:
                post()
        return g, B.argus_launch_count() - n0

    # host-side readers (synchronising)
    def fit_stats(self) -> dict:
        return B.fit_stats_from_bytes(self.stats)

    def sources_host(self):
        n = int(self.n_found[0].item())
        return B.sources_from_bytes(self.sources, min(n, self.src_cap)), n

    def status(self, stream=None) -> int:
        return B.argus_sync_status(self.ctx, stream)
