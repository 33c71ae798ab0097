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


def main(argv=None):
    """Run the batched-segment workload once at a given size and launch shape and print its
    time: `cameras` x 512 cutouts (64-512 px), 15x15 kernels, detection off (the fit, solves
    and subtraction).  A short stand-alone run of what the benchmark times, for profiling."""
    import argparse
    import time

    from . import _binding as B
    from .segments import SegmentBatch
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--cameras", type=int, default=2)
    ap.add_argument("--band", type=int, default=64, help="rows per fit work unit")
    ap.add_argument("--sub-ctas", type=int, default=8, help="subtraction CTAs per SM")
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--repeats", type=int, default=1)
    args = ap.parse_args(argv)
    per = 512
    sides = synth.segment_sides(args.cameras * per, seed=4)
    basis = B.make_basis(15, (0.7, 1.5, 3.0), (6, 4, 2), 0, 0)
    batch = SegmentBatch(sides, basis=basis, width=2048, cfg=B.argus_seg_config(args.band, 1, args.sub_ctas, 0),
                         device=0)
    try:
        fill_batch(batch, args.cameras, per)
        for _ in range(args.warmup):
            batch.run(use_graph=False, detect=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.time()
        e0.record()
        for _ in range(args.repeats):
            batch.run(use_graph=False, detect=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.repeats
        st = B.argus_sync_status(batch.ctx, 0)
    finally:
        batch.close()
    px = sum(s * s for s in sides)
    print(f"segments {len(sides)} pixels {px} ms {ms:.3f} Mpix/s {px / 1e3 / ms:.1f} status {st} "
          f"wall {time.time() - t0:.2f} s")
    return 0 if st == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
