"""Batched uneven segments over the C ABI: atlas packing, batch runner, autotuner.

The paper parallelises direct subtraction over image segments (Sec. 5) cut
from HEALPix-resampled frames (Sec. 4.1.1).  Here many square cutouts of
uneven size are packed into one pitched "atlas" per quantity and processed by
argus_segments_run (persistent fit and subtraction kernels, per-segment FP64
solves and atlas-wide detection, replayed as one CUDA graph).  This module only
packs, allocates and marshals; the autotuner times candidate launch shapes of
the library and keeps the fastest in a JSON table.
"""
from __future__ import annotations

import json
import os

import torch

from . import _binding as B

TUNE_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_segments.json")


def pack_shelves(sides, width=2048, align=16):
    """Shelf packing of squares into an atlas of the given width (largest first).

    Returns (positions [(row0, col0)] in input order, atlas height).  Positions
    are multiples of `align`.
    """
    up = lambda v: (v + align - 1) // align * align
    order = sorted(range(len(sides)), key=lambda i: -sides[i])
    pos = [None] * len(sides)
    row0, col, shelf_h = 0, 0, 0
    for i in order:
        s = int(sides[i])
        if s > width:
            raise ValueError("segment wider than the atlas")
        if col + s > width:
            row0 += up(shelf_h)
            col, shelf_h = 0, 0
        pos[i] = (row0, col)
        col = up(col + s)
        shelf_h = max(shelf_h, s)
    return pos, up(row0 + shelf_h)


class SegmentBatch:
    """Device atlas buffers and plan of one batch of segments."""

    def __init__(self, sides, *, basis: B.argus_basis, width=2048, cfg=None, src_cap=1 << 20,
                 det_cap=1 << 22, device=0, ctx=None, nsigma=5.0, psf_sigma=1.8):
        self.sides = [int(s) for s in sides]
        self.n = len(self.sides)
        self.pos, self.atlas_h = pack_shelves(self.sides, width)
        self.pitch = width
        self.basis = basis
        self.nb, self.Ks, self.Kb, self.Nc = B.basis_counts(basis)
        dev = torch.device("cuda", device)
        self.device = dev
        hp = (self.atlas_h, self.pitch)
        f32 = dict(dtype=torch.float32, device=dev)
        self.sci = torch.zeros(hp, **f32)
        self.var = torch.zeros(hp, **f32)
        self.ref = torch.zeros(hp, **f32)
        self.ref_var = torch.zeros(hp, **f32)
        self.flags = torch.zeros(hp, dtype=torch.uint8, device=dev)
        self.diff = torch.zeros(hp, **f32)
        self.diff_var = torch.zeros(hp, **f32)
        self.mask = torch.zeros(hp, dtype=torch.uint8, device=dev)
        self.coeffs = torch.zeros((self.n, self.Nc), dtype=torch.float64, device=dev)
        self.stats = torch.zeros(self.n * C_SIZE_STATS, dtype=torch.uint8, device=dev)
        self.src_cap = int(src_cap)
        self.sources = torch.zeros(self.src_cap * B.SOURCE_BYTES, dtype=torch.uint8, device=dev)
        self.n_found = torch.zeros(4, dtype=torch.int32, device=dev)
        self.nsigma, self.psf_sigma = float(nsigma), float(psf_sigma)
        self.ctx = ctx if ctx is not None else B.argus_create(device, self.atlas_h * self.pitch, 16, 64, det_cap)
        self._own_ctx = ctx is None
        self.table = [(r, c, s) for (r, c), s in zip(self.pos, self.sides)]
        self.cfg = cfg
        self.plan = B.argus_segments_plan(self.ctx, self.table, self.pitch, self.atlas_h, basis, cfg)

    def view(self, t: torch.Tensor, i: int) -> torch.Tensor:
        r, c = self.pos[i]
        s = self.sides[i]
        return t[r:r + s, c:c + s]

    def replan(self, cfg):
        if self.plan is not None:
            B.argus_segments_destroy(self.plan)
            self.plan = None
        self.cfg = cfg
        self.plan = B.argus_segments_plan(self.ctx, self.table, self.pitch, self.atlas_h, self.basis, cfg)

    def run(self, use_graph=True, detect=True, stream=None):
        B.argus_segments_run(self.plan, self.sci, self.var, self.ref, self.ref_var, self.flags, self.diff,
                             self.diff_var, self.mask if detect else None, self.coeffs, self.stats,
                             self.nsigma, self.psf_sigma, self.sources, self.src_cap,
                             self.n_found if detect else None, use_graph, stream)

    def stats_host(self):
        import numpy as np
        raw = self.stats.cpu().numpy().view(np.uint8)
        dt = np.dtype([("chi2", "<f8"), ("n_pix", "<i4"), ("status", "<i4")])
        return raw[: self.n * dt.itemsize].view(dt).copy()

    def sources_host(self):
        n = int(self.n_found[0].item())
        return B.sources_from_bytes(self.sources, min(n, self.src_cap)), n

    def segment_of(self, px, py):
        """Index of the segment holding atlas pixel (px, py), or -1."""
        for i, ((r, c), s) in enumerate(zip(self.pos, self.sides)):
            if r <= py < r + s and c <= px < c + s:
                return i
        return -1

    def close(self):
        if self.plan is not None:
            B.argus_segments_destroy(self.plan)
            self.plan = None
        if self._own_ctx and self.ctx is not None:
            B.argus_destroy(self.ctx)
            self.ctx = None


C_SIZE_STATS = 16


def candidate_configs():
    """Launch shapes the autotuner tries: rows per fit work unit (the tensor-core fit of
    kernel sides <= 15; one CTA per SM), persistent CTAs per SM of the CUDA-core fit
    (side 21, 8-row units) and of the subtraction kernels."""
    out = []
    for band in (32, 64, 128):
        for scta in (4, 8):
            out.append((band, 1, scta))
    for scta in (4, 8):
        out.append((8, 2, scta))
    return out


def autotune(batch: SegmentBatch, key: str, repeats=2, configs=None, table_path=TUNE_FILE, log=None):
    """Time each candidate launch shape on the batch and keep the fastest.

    The result is stored under `key` in a JSON table and returned as an
    argus_seg_config.  Configurations the library rejects (shared memory) are
    skipped.
    """
    results = {}
    best, best_ms = None, float("inf")
    for band, fcta, scta in configs or candidate_configs():
        cfg = B.argus_seg_config(band, fcta, scta, 0)
        try:
            batch.replan(cfg)
        except B.ArgusError:
            continue
        batch.run(use_graph=False, detect=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            batch.run(use_graph=False, detect=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / repeats
        results[f"{band},{fcta},{scta}"] = round(ms, 3)
        if log:
            log(f"autotune {key}: band {band} fit/SM {fcta} sub/SM {scta}: {ms:.2f} ms")
        if ms < best_ms:
            best, best_ms = (band, fcta, scta), ms
    if best is None:
        raise RuntimeError("no segment launch configuration was accepted")
    table = {}
    if os.path.exists(table_path):
        try:
            table = json.load(open(table_path))
        except Exception:
            table = {}
    table[key] = {"fit_band": best[0], "fit_ctas_per_sm": best[1], "sub_ctas_per_sm": best[2],
                  "ms": round(best_ms, 3), "tried": results}
    with open(table_path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    cfg = B.argus_seg_config(best[0], best[1], best[2], 0)
    batch.replan(cfg)
    return cfg


def tuned_config(key: str, table_path=TUNE_FILE):
    """The stored best configuration for `key`, or None."""
    if not os.path.exists(table_path):
        return None
    try:
        e = json.load(open(table_path)).get(key)
    except Exception:
        return None
    if not e:
        return None
    return B.argus_seg_config(int(e["fit_band"]), int(e["fit_ctas_per_sm"]), int(e["sub_ctas_per_sm"]), 0)
