"""Seeded synthetic workload of the batched-segment path.

`cameras` frames of the full IMX455 geometry are rendered on the device with
the full-frame recipe (one catalogue per camera, seed base + camera), and
`per_camera` square cutouts of log-uniform side (64-512 px) at uniform
positions are copied into a packed atlas: calibrated science and variance,
reference and reference variance, flags.  Input generation only.
"""
from __future__ import annotations

import torch

from . import synth


def fill_batch(batch, cameras: int, per_camera: int, seed: int = 4, w: int = 9576, h: int = 6388,
               stars: int = 150_000, log=None):
    dev = batch.device
    sides_all = batch.sides
    k = 0
    for cam in range(cameras):
        sd = seed + cam
        cat = synth.star_catalog(stars, w, h, seed=sd)
        R, Vr = synth.reference_image(synth.render(cat, w, h, 1.2, sky=300.0, device=dev, dtype=torch.float32),
                                      30, 1.7, sd + 1)
        sig = synth.field_sigma(w, h, 1.3, 2.2)
        I, V = synth.calibrated_image(synth.render(cat, w, h, sig, sky=305.0, device=dev, dtype=torch.float32),
                                      1.7, sd + 2)
        g = torch.Generator(device=dev).manual_seed(sd * 31 + 7)
        fl = (torch.rand((h, w), generator=g, device=dev) < 1e-4).to(torch.uint8)
        sides = sides_all[k:k + per_camera]
        origins = synth.segment_origins(sides, w, h, seed=sd)
        for j, ((x0, y0), s) in enumerate(zip(origins, sides)):
            i = k + j
            for dst, src in ((batch.sci, I), (batch.var, V), (batch.ref, R), (batch.ref_var, Vr),
                             (batch.flags, fl)):
                batch.view(dst, i).copy_(src[y0:y0 + s, x0:x0 + s])
        k += len(sides)
        del R, Vr, I, V, fl
        if log:
            log(f"camera {cam}: {len(sides)} segments")
    torch.cuda.synchronize(dev)
