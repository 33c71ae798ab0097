"""Benchmark of the full-frame difference-imaging step on GB300.

One step = one 9576 x 6388 IMX455 frame through the whole per-frame path:
calibration, stamp selection (20 x 20 grid), kernel fit (21 x 21 Alard-Lupton
basis, degree-2 spatial variation, 295 unknowns, FP32 normal equations, FP64
Cholesky + one refinement), kernel expansion, subtraction with the difference
variance, and 5-sigma detection.  Inputs are seeded synthetic star fields with
the recipe of the paper's IMX455 frames (150,000 stars, PSF 1.3-2.2 px across
the field, 300 e- sky, 1.7 e- read noise).  Every input is resident in HBM;
per step the raw frame (122 MB), reference and variances (~490 MB) are read, so
the working set is larger than the 129 MB L2 and no flush is needed.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(a bounded sample of the same workload on the host cores).  Under torchrun
with N > 1 every rank runs its own frame stream on its own GPU (replicas: the
path shards by frame with no collective); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpix/s differenced per GB300 (plain vs learned/BF16), % HBM roofline"
W, H = 9576, 6388
N_STARS = 150_000
KSIZE, SDEG, BGDEG = 21, 2, 2
GRID = (20, 20)
STAMP = 21
# algorithmic traffic of the fused frame path, bytes per pixel: raw 2, dark 4, flat 4,
# bpm 1, ref 4, ref var 4 in; D 4, V_D 4, mask 1 out; calibrated image, variance and
# flags (9 B) are written and read back once between the calibration and subtraction
# kernels and are not counted (a fused kernel would not move them).
BYTES_PER_PX = 2 + 4 + 4 + 1 + 4 + 4 + 4 + 4 + 1
# DRAM traffic of one launch of the tensor-core subtraction kernel, bytes per frame
# pixel: dram__bytes_read.sum + dram__bytes_write.sum of an ncu capture of a 4096x4096
# launch, scaled by pixels to the frame (the kernel streams its bands once, so traffic
# grows in proportion).  It holds only for the kernel sources it was taken on (None
# until a capture of these sources is recorded here).
SUBTRACT_TRAFFIC = {"bytes_per_px": 11.4422, "sources_sha1": "b88d70334bc10c960f3a5630a72c35fb9f6525bc",
                    "sources": ("subtract_tc.cu", "subtract_tile.cuh", "tc_ptx.cuh")}
# the same for the difference-variance kernel (V_I, V_ref and flags in, V_D out)
VARIANCE_TRAFFIC = {"bytes_per_px": 11.4747, "sources_sha1": "9332ad8c9b092988cc87fafc1738f66d06951598",
                    "sources": ("subtract_tc.cu", "subtract_tile.cuh", "tc_ptx.cuh", "subtract.cu")}


def traffic_bytes(rec):
    import hashlib
    h = hashlib.sha1()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_2207_14304_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if rec["bytes_per_px"] is None or h.hexdigest() != rec["sources_sha1"]:
        return None
    return int(rec["bytes_per_px"] * W * H)


def workload_config(precision="tf32"):
    return {"workload": f"full-frame plain DIA, {W}x{H} uint16 IMX455 frame + float32 reference",
            "frame": [W, H], "stars": N_STARS, "psf_sigma": "1.3-2.2 px (science), 1.2 px (reference)",
            "kernel": KSIZE, "spatial_degree": SDEG, "bg_degree": BGDEG, "basis": "3 Gaussians x degrees (6,4,2)",
            "stamps": GRID[0] * GRID[1], "stamp": STAMP, "normal_equations": precision, "nsigma": 5.0,
            "l2": (f"working set {W * H * 10 / 1e6:.0f} MB per step (raw {W * H * 2 / 1e6:.0f} MB + reference and "
                   f"variances {W * H * 8 / 1e6:.0f} MB) against the 129 MB L2; no flush")}


# --------------------------------------------------------------------------- distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    """MAX of a float over all ranks (identity on one rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: float, elapsed_s: float, dist, device=None):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    ws = dist.get_world_size() if dist is not None else 1
    tmax = max_over_ranks(dist, elapsed_s, device)
    return units_per_rank * ws / tmax, tmax


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        return parse_clocks(self.path)


def parse_clocks(path):
    """Median SM clock, max clock and the throttle reasons seen, from the sampler's CSV."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        p = [x.strip() for x in line.split(",")]
        if len(p) < 9:
            continue
        try:
            sm.append(float(p[1]))
            mx.append(float(p[2]))
        except ValueError:
            continue
        for n, v in zip(names, p[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


# --------------------------------------------------------------------------- GPU arm
def make_inputs(device, seed=2):
    import torch
    from paper_2207_14304_gb300 import synth
    cat = synth.star_catalog(N_STARS, W, H, seed=seed)
    Rexp = synth.render(cat, W, H, 1.2, sky=300.0, device=device, dtype=torch.float32)
    R, Vr = synth.reference_image(Rexp, 30, 1.7, seed + 1)
    del Rexp
    sig = synth.field_sigma(W, H, 1.3, 2.2)
    Iexp = synth.render(cat, W, H, sig, sky=305.0, device=device, dtype=torch.float32)
    cal = synth.make_calib(W, H, seed=seed + 2, device=device)
    raw = synth.expose(Iexp, cal, seed=seed + 3)
    del Iexp
    return raw, R, Vr, cal


def run_gpu(args):
    import torch
    from paper_2207_14304_gb300 import _binding as B
    from paper_2207_14304_gb300.pipeline import FramePipeline

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = dist_init(ws, "nccl")

    raw, R, Vr, cal = make_inputs(device, seed=2 + rank)
    basis = B.make_basis(KSIZE, (0.7, 1.5, 3.0), (6, 4, 2), SDEG, BGDEG)
    pipe = FramePipeline(W, H, basis=basis, stamp=STAMP, grid=GRID, precision=args.precision,
                         psf_sigma=1.8, device=local)
    pitch = pipe.pitch
    # frames in flight: each has its own pipeline (buffers and library context) and stream,
    # so one frame's latency-bound fit overlaps the next frame's calibration and selection
    nfl = max(1, args.frames_in_flight)
    pipes = [pipe] + [FramePipeline(W, H, basis=basis, stamp=STAMP, grid=GRID, precision=args.precision,
                                    psf_sigma=1.8, device=local) for _ in range(nfl - 1)]

    def pad(a):
        t = torch.zeros((H, pitch), dtype=a.dtype, device=device)
        t[:, :W] = a
        return t

    d_raw, d_R, d_Vr = pad(raw), pad(R), pad(Vr)
    d_dark, d_flat, d_bpm = pad(cal.dark), pad(cal.flat), pad(cal.bpm)
    calib = B.make_calib(cal.bias, d_dark, d_flat, d_bpm, cal.gain, cal.read_noise, cal.sat)
    del raw, R, Vr
    stream = torch.cuda.current_stream(device)

    def step():
        pipe.run(d_raw, calib, d_R, d_Vr, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(device)
    st = pipe.status(stream)
    if st != 0:
        raise RuntimeError(f"device status {st} ({B.status_string(st)}) after warm-up")

    # per-stage times (untimed pass, for the report)
    stage = {}
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    evs[0].record(stream); pipe.calibrate(d_raw, calib, stream)
    evs[1].record(stream); pipe.select_stamps(d_R, stream)
    evs[2].record(stream); pipe.fit(d_R, stream)
    evs[3].record(stream); pipe.subtract(d_R, d_Vr, stream)
    evs[4].record(stream); pipe.detect(stream)
    evs[5].record(stream)
    torch.cuda.synchronize(device)
    for i, k in enumerate(["calibrate", "select_stamps", "fit", "subtract", "detect"]):
        stage[k] = round(evs[i].elapsed_time(evs[i + 1]), 4)

    streams = [stream] + [torch.cuda.Stream(device) for _ in range(nfl - 1)]
    for p, s in zip(pipes[1:], streams[1:]):   # warm the other pipelines too
        p.run(d_raw, calib, d_R, d_Vr, s)
    torch.cuda.synchronize(device)
    # each in-flight pipeline's frame as one CUDA graph on a side stream of its own
    gstreams = [torch.cuda.Stream(device) for _ in range(nfl)]
    graphs, per_frame = [], 0
    for p, s in zip(pipes, gstreams):
        with torch.cuda.stream(s):
            (p.run_fused if args.fused else p.run)(d_raw, calib, d_R, d_Vr, s)
        torch.cuda.synchronize(device)
        g, per_frame = p.capture(d_raw, calib, d_R, d_Vr, s, fused=args.fused)
        graphs.append(g)
    torch.cuda.synchronize(device)

    # timed region: K steps, frame i on pipeline and stream i mod nfl
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local, os.path.join(tempfile.gettempdir(), f"argus_clocks_rank{rank}_{os.getpid()}.csv")) \
        if args.clocks else None
    barrier(dist, device)
    torch.cuda.synchronize(device)
    t0.record(stream)
    for s in gstreams:
        s.wait_event(t0)
    for i in range(args.steps):
        with torch.cuda.stream(gstreams[i % nfl]):
            graphs[i % nfl].replay()
    for s in gstreams:
        stream.wait_stream(s)
    t1.record(stream)
    torch.cuda.synchronize(device)
    launches = per_frame * args.steps   # graph replays: the frame's launches, counted at capture
    barrier(dist, device)
    clk = clocks.stop() if clocks else None
    elapsed = t0.elapsed_time(t1) / 1e3
    for p in pipes:
        st = p.status(stream)
        if st != 0:
            raise RuntimeError(f"device status {st} ({B.status_string(st)}) in the timed region")
    mpix = W * H / 1e6
    value, tmax = aggregate(mpix * args.steps, elapsed, dist, device)

    # the two subtraction kernels timed on their own: the same steps on one stream (with
    # frames in flight their launches share the GPU with the next frame's work), events
    # around each kernel on its stream
    kk = max(5, args.steps // 4)
    var_s = [torch.cuda.Event(enable_timing=True) for _ in range(kk)]
    sub_s = [torch.cuda.Event(enable_timing=True) for _ in range(kk)]
    sub_e = [torch.cuda.Event(enable_timing=True) for _ in range(kk)]
    torch.cuda.synchronize(device)
    for i in range(kk):
        pipe.calibrate(d_raw, calib, stream)
        pipe.select_stamps(d_R, stream)
        pipe.fit(d_R, stream)
        var_s[i].record(stream)
        pipe.subtract_variance(d_Vr, stream)
        sub_s[i].record(stream)
        pipe.subtract_difference(d_R, d_Vr, stream)
        sub_e[i].record(stream)
        pipe.detect(stream)
    torch.cuda.synchronize(device)
    tc_ms = statistics.mean(sub_s[i].elapsed_time(sub_e[i]) for i in range(kk))
    ktiming = f"CUDA events around the launch on its stream, mean of {kk} steps of the workload on one stream"
    var_ms = statistics.mean(var_s[i].elapsed_time(sub_s[i]) for i in range(kk))

    # end to end through the public API: pinned host raw frame in, detection list out
    raw_host = d_raw.cpu().pin_memory()
    d_raws = [d_raw] + [torch.empty_like(d_raw) for _ in range(nfl - 1)]
    out_host = [torch.empty(pipe.sources.numel(), dtype=torch.uint8).pin_memory() for _ in range(nfl)]
    nf_hosts = [torch.empty(4, dtype=torch.int32).pin_memory() for _ in range(nfl)]
    ke = max(3, args.steps // 4)
    # one graph per in-flight pipeline: pinned raw frame in, the frame, sources and count out
    egraphs = []
    for j, (p, s) in enumerate(zip(pipes, gstreams)):
        def pre(j=j):
            d_raws[j].copy_(raw_host, non_blocking=True)

        def post(j=j, p=p):
            nf_hosts[j].copy_(p.n_found, non_blocking=True)
            out_host[j].copy_(p.sources, non_blocking=True)
        with torch.cuda.stream(s):
            pre()
            (p.run_fused if args.fused else p.run)(d_raws[j], calib, d_R, d_Vr, s)
            post()
        torch.cuda.synchronize(device)
        egraphs.append(p.capture(d_raws[j], calib, d_R, d_Vr, s, pre=pre, post=post, fused=args.fused)[0])
    barrier(dist, device)
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in gstreams:
        s.wait_event(e0)
    for i in range(ke):
        with torch.cuda.stream(gstreams[i % nfl]):
            egraphs[i % nfl].replay()
    for s in gstreams:
        stream.wait_stream(s)
    e1.record(stream)
    nf_host = nf_hosts[(ke - 1) % nfl]
    torch.cuda.synchronize(device)
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_value, _ = aggregate(mpix * ke, e2e_s, dist, device)
    n_found = int(nf_host[0].item())

    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    step_s = tmax / args.steps
    hbm_frac = BYTES_PER_PX * W * H / step_s / 1e9 / hbm
    kernels = kernel_rooflines(tc_ms, var_ms, ktiming, peaks)
    # the step against the compute roof: algorithmic FLOPs of its dense contractions (the
    # difference image 2 x 6 x 441, the variance 2 x 441 per pixel; the fit's stamp
    # convolutions and normal equations per frame) over the step time, against the
    # sustained cuBLAS BF16 rate (the step is a long run)
    nst = GRID[0] * GRID[1]
    nunk = 1 + (49 - 1) * 6 + 6
    fit_flop = 2.0 * nst * STAMP * STAMP * 49 * KSIZE * KSIZE + 2.0 * nst * STAMP * STAMP * (nunk + 1) * (nunk + 2) / 2
    step_flop_px = 2 * 6 * KSIZE * KSIZE + 2 * KSIZE * KSIZE + fit_flop / (W * H)
    bf16_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    step_tflops = step_flop_px * W * H / step_s / 1e12
    compute_roofline = {"flop_per_px": round(step_flop_px, 1), "achieved": round(step_tflops, 2),
                        "peak": bf16_peak, "unit": "TFLOP/s", "frac": round(step_tflops / bf16_peak, 4),
                        "algorithmic": "difference image 2x6x441 + variance 2x441 FLOP/px, with the fit's stamp "
                                       "convolutions (400 x 441 px x 49 x 441 taps) and normal equations "
                                       "(400 x 441 rows, 296 columns, upper triangle) per frame",
                        "peak_source": ("measured, MEASURED_PEAKS.json bf16_tflops_sustained"
                                        if "bf16_tflops_sustained" in peaks
                                        else "fallback, 1.7 PFLOP/s sustained from an earlier GB300 measurement")}

    var = {}
    if args.variants and ws == 1:
        # whole frames, one at a time, with each normal-equation precision (fp32 included, for
        # comparison on equal terms); fit_ms is the fit stage alone
        for prec in ("fp32", "tf32", "bf16", "bf16_split"):
            pv = FramePipeline(W, H, basis=basis, stamp=STAMP, grid=GRID, precision=prec, psf_sigma=1.8,
                               device=local, ctx=pipe.ctx)
            for _ in range(2):
                pv.run(d_raw, calib, d_R, d_Vr, stream)
            torch.cuda.synchronize(device)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            kv = max(3, args.steps // 4)
            a0.record(stream)
            for _ in range(kv):
                pv.run(d_raw, calib, d_R, d_Vr, stream)
            a1.record(stream)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(kv):
                pv.fit(d_R, stream)
            f1.record(stream)
            torch.cuda.synchronize(device)
            var[prec] = {"mpix_s": round(mpix * kv / (a0.elapsed_time(a1) / 1e3), 2),
                         "fit_ms": round(f0.elapsed_time(f1) / kv, 4)}
            if pv.status(stream) != 0:
                var[prec] = None

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(tmax / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(args.precision), "frames_in_flight": nfl,
                   "launch": ("each frame one argus_dia_frame call" if args.fused
                              else "each frame the separate calls argus_calibrate .. argus_detect")
                             + ", captured once per in-flight pipeline as a CUDA graph and replayed"},
        # the dominant kernel of the step (the larger of the two subtraction kernels)
        "roofline": dict(kernels["subtract_tc"] if tc_ms >= var_ms else kernels["variance"]),
        "kernels": kernels,
        "hbm_roofline_frac": round(hbm_frac, 4),
        "hbm_bytes_per_px": BYTES_PER_PX,
        "compute_roofline": compute_roofline,
        "stage_ms": stage, "subtract_ms": round(tc_ms + var_ms, 4),
        "subtract_detect_mpix_s": round(W * H / 1e6 / ((stage["subtract"] + stage["detect"]) / 1e3), 1),
        "e2e": {"value": round(e2e_value, 2), "unit": "Mpix/s", "h2d_bytes_per_step": int(raw_host.numel() * 2),
                "d2h_bytes_per_step": int(out_host[0].numel() + nf_host.numel() * 4)},
        "gpu_launches": int(launches), "sources_last_frame": n_found,
        "variants": var, "clocks": clk,
    }
    pipe.close()
    del d_raw, d_R, d_Vr
    torch.cuda.empty_cache()
    if args.extras and ws == 1:
        extras = {}
        wanted = set(x for x in args.extras.split(",") if x)
        for name, fn in (("coadd", lambda: bench_coadd(device, stream, args.steps, hbm)),
                         ("segments", lambda: bench_segments(device, stream, args.segment_cameras)),
                         ("learned", lambda: bench_learned(device, stream, args.train_pairs, args.train_epochs,
                                                              crowd=args.train_crowd == "frame")),
                         ("sparse", lambda: bench_sparse(device, stream, hbm)),
                         ("background", lambda: bench_background(device, stream, hbm)),
                         ("healpix", lambda: bench_healpix(device, stream, hbm)),
                         ("zogy", lambda: bench_zogy(device, stream, hbm)),
                         ("proper_coadd", lambda: bench_proper_coadd(device, stream, hbm))):
            if name not in wanted:
                continue
            try:
                extras[name] = fn()
            except Exception as e:   # an extra never invalidates the headline line
                extras[name] = {"error": repr(e)[:300]}
            torch.cuda.empty_cache()
        result["workloads"] = extras
    if rank == 0 and args.cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


VAR_BYTES_PER_PX = 4 + 4 + 1 + 4      # V_I, V_ref, flags read; V_D written


def kernel_rooflines(tc_ms, var_ms, ktiming, peaks):
    """Roofline entries of the two subtraction kernels of one full frame.

    Difference image: NK * KS^2 multiply-adds per pixel against 13 bytes (I, R,
    flags in, D out), 407 FLOP/B at 21x21 and degree 2 -- above the ridge of the
    measured peaks (1719.5 TFLOP/s / 6777 GB/s = 254 FLOP/B), so the tensor roof
    binds.  The MMAs execute more (BF16 hi/lo x three products, K padded 21 -> 24,
    one M=128 x N=16*ceil((KS-1+4)*NK/16) MMA group per source row, source rows in
    blocks of 4 with 2R halo rows per 128-row band), reported beside it.
    Variance: KS^2 multiply-adds per pixel against 13 bytes, 68 FLOP/B -- below
    the ridge, so the HBM roof binds: achieved = 13 B/px / kernel time."""
    nk = (SDEG + 1) * (SDEG + 2) // 2
    conv_flops = 2 * nk * KSIZE * KSIZE * W * H
    achieved = conv_flops / (tc_ms / 1e3) / 1e12
    bands = [min(128, H - y0) for y0 in range(0, H, 128)]
    n_mma = 16 * (((KSIZE - 1 + 4) * nk + 15) // 16)
    k_row = 16 if KSIZE <= 16 else 24          # taps 16..23 of a row pair share one K = 16 MMA
    src_rows = ((W + 127) // 128) * sum(4 * ((b + KSIZE - 1 + 3) // 4) for b in bands)
    executed = 3 * 2 * 128 * n_mma * k_row * src_rows
    # the variance: one term of width N1 = 16*ceil((KS-1+4)/16), MMAs of width 2 N1 (hi*hi, hi*lo)
    # and N1 (lo*hi)
    n1 = 16 * ((KSIZE - 1 + 4 + 15) // 16)
    executed_var = 2 * 128 * 3 * n1 * k_row * src_rows
    tensor_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    hbm = peaks.get("hbm_gbs", 6800.0)
    var_tflops = 2 * KSIZE * KSIZE * W * H / (var_ms / 1e3) / 1e12
    var_gbs = VAR_BYTES_PER_PX * W * H / (var_ms / 1e3) / 1e9
    return {
        "subtract_tc": {"bound": "tensor", "kernel": "subtract_tc (reference convolution, difference image)",
                        "achieved": round(achieved, 3), "peak": round(tensor_peak, 1), "unit": "TFLOP/s",
                        "frac": round(achieved / tensor_peak, 4), "traffic": traffic_bytes(SUBTRACT_TRAFFIC),
                        "traffic_unit": "bytes per launch (ncu DRAM read+write)",
                        "peak_source": "measured, MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS BF16 GEMM, sustained)",
                        "algorithmic": f"{2 * nk * KSIZE * KSIZE} FLOP/px ({nk} spatial terms x {KSIZE}x{KSIZE} taps)",
                        "executed_tflops": round(executed / (tc_ms / 1e3) / 1e12, 1),
                        "kernel_ms": round(tc_ms, 4), "kernel_timing": ktiming},
        "variance": {"bound": "hbm", "kernel": "subtract_tc variance (tile-centre kernel squared (x) V_ref)",
                     "achieved": round(var_gbs, 1), "peak": round(hbm, 1), "unit": "GB/s",
                     "frac": round(var_gbs / hbm, 4), "traffic": traffic_bytes(VARIANCE_TRAFFIC),
                     "traffic_unit": "bytes per launch (ncu DRAM read+write)",
                     "peak_source": "measured, MEASURED_PEAKS.json hbm_gbs (STREAM-style copy)",
                     "algorithmic": (f"{VAR_BYTES_PER_PX} B/px (V_I, V_ref, flags in; V_D out); "
                                     f"{2 * KSIZE * KSIZE} FLOP/px ({KSIZE}x{KSIZE} squared taps)"),
                     "tflops": round(var_tflops, 3), "tensor_frac": round(var_tflops / tensor_peak, 4),
                     "executed_tflops": round(executed_var / (var_ms / 1e3) / 1e12, 1),
                     "kernel_ms": round(var_ms, 4), "kernel_timing": ktiming},
    }


def timed_ms(fn, n, stream, device):
    import torch
    fn()
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        fn()
    e1.record(stream)
    torch.cuda.synchronize(device)
    return e0.elapsed_time(e1) / n


def call_ms(fn, n, stream, device):
    """Median over n calls of one call's device time (CUDA events on the launching
    stream, the device synchronised before each call)."""
    import torch
    fn()
    ts = []
    for _ in range(n):
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(device)
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def bench_coadd(device, stream, steps, hbm):
    """30 x 9576x6388 uint16 frames (one 15-min ratchet at 30 s), shifts up to 0.5 px,
    1 % cosmic rays, 3-sigma clipped mean with fused calibration."""
    import torch
    from paper_2207_14304_gb300 import _binding as B
    from paper_2207_14304_gb300 import synth
    nf = 30
    pitch = synth.pitch_for(W)
    cat = synth.star_catalog(N_STARS, W, H, seed=3)
    cal = synth.make_calib(W, H, seed=5, device=device)
    sh = synth.uniform_shifts(nf, seed=3)
    stack = torch.zeros((nf, H, pitch), dtype=torch.uint16, device=device)
    for f in range(nf):
        e = synth.render(cat, W, H, 1.5, sky=300.0, shift=(-float(sh[f, 0]), -float(sh[f, 1])), device=device,
                         dtype=torch.float32)
        stack[f, :, :W] = synth.expose(e, cal, seed=300 + f, cosmic_frac=0.01)
        del e

    def pad(a):
        t = torch.zeros((H, pitch), dtype=a.dtype, device=device)
        t[:, :W] = a
        return t
    d_dark, d_flat, d_bpm = pad(cal.dark), pad(cal.flat), pad(cal.bpm)
    calib = B.make_calib(cal.bias, d_dark, d_flat, d_bpm, cal.gain, cal.read_noise, cal.sat)
    co = torch.zeros((H, pitch), device=device)
    va = torch.zeros((H, pitch), device=device)
    nu = torch.zeros((H, pitch), dtype=torch.uint8, device=device)
    ctx = B.argus_create(device.index, H * pitch, 16, 64, 1 << 10)
    try:
        shifts = sh.to(device)
        ms = timed_ms(lambda: B.argus_coadd(ctx, stack, nf, B.argus_shape(W, H, pitch), shifts, calib, 3.0, 5, co,
                                            va, nu, stream), max(3, steps // 10), stream, device)
        st = B.argus_sync_status(ctx, stream)
    finally:
        B.argus_destroy(ctx)
    bpp = nf * 2 + 9 + 9
    return {"workload": f"30 x {W}x{H} uint16, shifts <= 0.5 px, 1% cosmic rays, kappa 3, 5 iterations",
            "ms": round(ms, 3), "value": round(W * H / 1e6 / (ms / 1e3), 1), "unit": "Mpix/s (output)",
            "hbm_bytes_per_px": bpp, "hbm_frac": round(bpp * W * H / (ms / 1e3) / 1e9 / hbm, 4), "status": st}


def bench_segments(device, stream, cameras, log=None):
    """38 cameras x 512 square cutouts (64-512 px, log-uniform) with their own fitted 15x15
    kernels, through one CUDA-graph launch of the persistent kernels."""
    import torch
    from paper_2207_14304_gb300 import _binding as B
    from paper_2207_14304_gb300 import synth
    from paper_2207_14304_gb300.segment_workload import fill_batch
    from paper_2207_14304_gb300.segments import SegmentBatch, autotune, tuned_config
    per = 512
    sides = synth.segment_sides(cameras * per, seed=4)
    basis = B.make_basis(15, (0.7, 1.5, 3.0), (6, 4, 2), 0, 0)
    key = f"segments_{cameras}x{per}_ks15"
    cfg = tuned_config(key)
    batch = SegmentBatch(sides, basis=basis, width=2048, cfg=cfg or B.argus_seg_config(64, 1, 8, 0),
                         device=device.index)
    try:
        t0 = time.time()
        fill_batch(batch, cameras, per)
        gen_s = time.time() - t0
        if cfg is None:
            cfg = autotune(batch, key, repeats=1)
        ms = timed_ms(lambda: batch.run(use_graph=True, stream=stream), 3, stream, device)
        st = B.argus_sync_status(batch.ctx, stream)
        nsrc = int(batch.n_found[0].item())
        fit_items, sub_items = B.argus_segments_items(batch.plan)
    finally:
        batch.close()
    px = sum(s * s for s in sides)
    return {"workload": f"{cameras} cameras x {per} segments, 64-512 px log-uniform, 15x15 kernel per segment",
            "segments": len(sides), "pixels": px, "ms": round(ms, 3), "value": round(px / 1e6 / (ms / 1e3), 1),
            "unit": "Mpix/s", "config": {"fit_band": cfg.fit_band, "fit_ctas_per_sm": cfg.fit_ctas_per_sm,
                                         "sub_ctas_per_sm": cfg.sub_ctas_per_sm},
            "work_units": {"fit": fit_items, "subtract": sub_items}, "sources": nsrc, "status": st,
            "generation_s": round(gen_s, 1)}


def bench_sparse(device, stream, hbm):
    """Minipix stamping (9-pixel cells ~ the NSIDE=16384 minipix at 1.38 arcsec/px,
    4600 catalogue targets ~ 1e7 sources over 19,370 sq deg seen by one 9 sq deg
    camera, 400 detections) and the 10x low-resolution map of one 9576x6388 frame."""
    import torch
    from paper_2207_14304_gb300 import _binding as B
    from paper_2207_14304_gb300 import synth
    cell, factor, n_cat, n_det = 9, 10, 4600, 400
    pitch = synth.pitch_for(W)
    cat = synth.star_catalog(N_STARS, W, H, seed=21)
    g = torch.Generator(device=device)
    g.manual_seed(21)
    img = torch.zeros((H, pitch), device=device)
    img[:, :W] = synth.render(cat, W, H, 1.5, sky=300.0, device=device, dtype=torch.float32)
    img[:, :W] += torch.randn((H, W), generator=g, device=device) * 18.0
    flags = torch.zeros((H, pitch), dtype=torch.uint8, device=device)
    flags[:, :W] = (torch.rand((H, W), generator=g, device=device) < 1e-4).to(torch.uint8)
    tx = cat.x[:n_cat].round().clamp(0, W - 1).to(torch.int32)
    ty = cat.y[:n_cat].round().clamp(0, H - 1).to(torch.int32)
    targets = torch.stack([tx, ty], 1).contiguous().to(device)
    src = torch.zeros((n_det, B.SOURCE_BYTES // 4), dtype=torch.int32, device=device)
    src[:, 7] = torch.randint(0, W, (n_det,), generator=g, device=device, dtype=torch.int32)   # px
    src[:, 8] = torch.randint(0, H, (n_det,), generator=g, device=device, dtype=torch.int32)   # py
    n_src = torch.tensor([n_det], dtype=torch.int32, device=device)
    ncx, ncy = -(-W // cell), -(-H // cell)
    cap = 1 << 14
    keep = torch.zeros((ncy, ncx), dtype=torch.uint8, device=device)
    out = torch.empty((H, pitch), device=device)
    packed = torch.empty((cap, cell * cell), device=device)
    cidx = torch.empty(cap, dtype=torch.int32, device=device)
    nk = torch.zeros(4, dtype=torch.int32, device=device)
    ow, oh = -(-W // factor), -(-H // factor)
    lpitch = synth.pitch_for(ow)
    low = torch.empty((oh, lpitch), device=device)
    shape = B.argus_shape(W, H, pitch)
    ctx = B.argus_create(device.index, H * pitch, 16, 64, 1 << 10)
    try:
        # inputs (245 MB image) exceed L2, so successive calls do not reuse cached pixels
        mp_ms = call_ms(lambda: B.argus_minipix(ctx, img, shape, cell, targets, n_cat, src, n_src, n_det, keep, out,
                                                packed, cidx, cap, nk, stream), 20, stream, device)
        lr_ms = call_ms(lambda: B.argus_lowres(ctx, img, flags, shape, factor, low, lpitch, stream), 20, stream,
                        device)
        st = B.argus_sync_status(ctx, stream)
        kept = int(nk[0].item())
    finally:
        B.argus_destroy(ctx)
    npx = H * pitch
    kept_px = kept * cell * cell
    mp_bytes = 4 * npx + 8 * kept_px + ncx * ncy * 4      # out write, kept reads + packed writes, keep map
    lr_bytes = 5 * npx + 4 * oh * ow                      # image + flags read, map written
    return {"workload": f"{W}x{H} frame, {cell}-px minipix cells, {n_cat} catalogue targets + {n_det} detections; "
                        f"{factor}x low-resolution map",
            "minipix": {"ms": round(mp_ms, 4), "value": round(W * H / 1e6 / (mp_ms / 1e3), 1), "unit": "Mpix/s",
                        "kept_cells": kept, "kept_frac": round(kept / (ncx * ncy), 5),
                        "hbm_bytes": mp_bytes, "hbm_frac": round(mp_bytes / (mp_ms / 1e3) / 1e9 / hbm, 4)},
            "lowres": {"ms": round(lr_ms, 4), "value": round(W * H / 1e6 / (lr_ms / 1e3), 1), "unit": "Mpix/s",
                       "hbm_bytes": lr_bytes, "hbm_frac": round(lr_bytes / (lr_ms / 1e3) / 1e9 / hbm, 4)},
            "status": st}


def _star_frame(device, seed, sigma=1.5, sky=300.0, noise=18.0):
    """A rendered 9576x6388 star field with Gaussian noise, pitched, and sparse flags."""
    import torch
    from paper_2207_14304_gb300 import synth
    pitch = synth.pitch_for(W)
    cat = synth.star_catalog(N_STARS, W, H, seed=seed)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    img = torch.zeros((H, pitch), device=device)
    img[:, :W] = synth.render(cat, W, H, sigma, sky=sky, device=device, dtype=torch.float32)
    img[:, :W] += torch.randn((H, W), generator=g, device=device) * noise
    flags = torch.zeros((H, pitch), dtype=torch.uint8, device=device)
    flags[:, :W] = (torch.rand((H, W), generator=g, device=device) < 1e-4).to(torch.uint8)
    return img, flags, pitch


def bench_background(device, stream, hbm):
    """Median-filtered background map of one 9576x6388 frame: 64-px boxes, 3x3 mesh filter.
    Opt-in (--extras background)."""
    import torch
    from paper_2207_14304_gb300 import _binding as B
    img, flags, pitch = _star_frame(device, 31)
    box = 64
    mesh = torch.zeros((-(-H // box), -(-W // box)), dtype=torch.float64, device=device)
    bmap = torch.empty((H, pitch), device=device)
    ctx = B.argus_create(device.index, H * pitch, 16, 64, 1 << 10)
    try:
        ms = call_ms(lambda: B.argus_background(ctx, img, flags, B.argus_shape(W, H, pitch), box, 3, 0.5, mesh, bmap,
                                                stream), 20, stream, device)
        st = B.argus_sync_status(ctx, stream)
    finally:
        B.argus_destroy(ctx)
    nbytes = (4 + 1 + 4) * H * pitch                     # image and flags read, map written
    return {"workload": f"{W}x{H} frame, {box}-px boxes, 3x3 mesh median filter, bilinear map",
            "ms": round(ms, 4), "value": round(W * H / 1e6 / (ms / 1e3), 1), "unit": "Mpix/s",
            "hbm_bytes": nbytes, "hbm_frac": round(nbytes / (ms / 1e3) / 1e9 / hbm, 4), "status": st}


def bench_healpix(device, stream, hbm):
    """Every NSIDE=256 segment whose centre falls in a 9576x6388 frame at 1.38 arcsec/px
    (gnomonic WCS at RA 60 deg, Dec 30 deg), resampled to 512x512 segment images (k = 9).
    Opt-in (--extras healpix)."""
    import math
    import torch
    from paper_2207_14304_gb300 import _binding as B
    img, flags, pitch = _star_frame(device, 32)
    nside, k = 256, 9
    shape = B.argus_shape(W, H, pitch)
    wcs = (math.radians(60.0), math.radians(30.0), math.radians(1.38 / 3600.0), 0.1, (W - 1) / 2, (H - 1) / 2)
    # the segments whose centre falls in the frame: resample every NSIDE-256 pixel at k = 0
    every = torch.arange(12 * nside * nside, dtype=torch.int64, device=device)
    centre = torch.empty(every.numel(), device=device)
    ccov = torch.empty(every.numel(), dtype=torch.uint8, device=device)
    B.argus_healpix_resample(img, None, shape, wcs, nside, 0, every, every.numel(), centre, ccov, stream)
    torch.cuda.synchronize(device)
    d_segs = every[ccov.bool()].contiguous()
    n_seg = int(d_segs.numel())
    m = 1 << k
    out = torch.empty((n_seg, m, m), device=device)
    cov = torch.empty((n_seg, m, m), dtype=torch.uint8, device=device)
    ms = call_ms(lambda: B.argus_healpix_resample(img, flags, shape, wcs, nside, k, d_segs, n_seg, out, cov, stream),
                 10, stream, device)
    covered = float(cov.float().mean().item())
    npx = n_seg * m * m
    nbytes = npx * (4 + 1) + (4 + 1) * W * H              # outputs written, the frame and flags read once
    return {"workload": f"{n_seg} NSIDE-{nside} segments of {m}x{m} (k = {k}) from a {W}x{H} frame at 1.38 arcsec/px",
            "ms": round(ms, 4), "value": round(npx / 1e6 / (ms / 1e3), 1), "unit": "Mpix/s (segment pixels)",
            "covered_frac": round(covered, 4), "hbm_bytes": nbytes,
            "hbm_frac": round(nbytes / (ms / 1e3) / 1e9 / hbm, 4)}


def _gauss_psf(sig, half=15):
    import numpy as np
    u = np.arange(-half, half + 1)
    g = np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / (2 * sig * sig))
    return (g / g.sum()).astype(np.float32)


def bench_zogy(device, stream, hbm):
    """ZOGY on 512x512 tiles covering a 9576x6388 frame (18 x 12 tiles), per-tile Gaussian PSFs
    (new 1.3-2.2 px, reference 1.2 px). Opt-in (--extras zogy)."""
    import numpy as np
    import torch
    from paper_2207_14304_gb300 import _binding as B
    N, _, pitch = _star_frame(device, 33, sigma=1.8)
    R, _, _ = _star_frame(device, 33, sigma=1.2, noise=3.0)
    T = 512
    org = [(x, y) for y in range(0, H - T + 1, T) for x in range(0, W - T + 1, T)]
    nt = len(org)
    rec = np.zeros(nt, B.ZOGY_TILE_DTYPE)
    pn = np.zeros((nt, 31, 31), np.float32)
    pr = np.zeros_like(pn)
    for i, (x0, y0) in enumerate(org):
        rec[i] = (x0, y0, 1.0, 1.0, 18.0, 3.0)
        pn[i] = _gauss_psf(1.3 + 0.9 * i / max(nt - 1, 1))
        pr[i] = _gauss_psf(1.2)
    plan = B.proper_plan_create(device.index, T, nt)
    try:
        d_rec = torch.from_numpy(rec.view(np.uint8).copy()).to(device)
        dpn, dpr = torch.from_numpy(pn).to(device), torch.from_numpy(pr).to(device)
        D = torch.empty((nt, T, T), device=device)
        S = torch.empty((nt, T, T), device=device)
        sig = torch.empty(nt, dtype=torch.float64, device=device)
        ms = call_ms(lambda: B.argus_zogy(plan, N, R, B.argus_shape(W, H, pitch), d_rec, nt, dpn, dpr, 31, 1e-8, D, S,
                                          None, sig, stream), 5, stream, device)
        # the same frame with the pointing's PSF transforms kept from the previous call
        ms_reuse = call_ms(lambda: B.argus_zogy(plan, N, R, B.argus_shape(W, H, pitch), d_rec, nt, None, None, 31, 1e-8,
                                                D, S, None, sig, stream), 5, stream, device)
    finally:
        B.proper_plan_destroy(plan)
    npx = nt * T * T
    return {"workload": f"{nt} tiles of {T}x{T} from a {W}x{H} frame, per-tile PSFs", "ms": round(ms, 3),
            "value": round(npx / 1e6 / (ms / 1e3), 1), "unit": "Mpix/s", "ms_per_tile": round(ms / nt, 4),
            "ms_psf_reused": round(ms_reuse, 3), "value_psf_reused": round(npx / 1e6 / (ms_reuse / 1e3), 1)}


def bench_proper_coadd(device, stream, hbm):
    """Proper coadd of 30 frames on 512x512 tiles of a 9576x6388 field (18 x 12 tiles).
    Opt-in (--extras proper_coadd)."""
    import numpy as np
    import torch
    from paper_2207_14304_gb300 import _binding as B
    J, T = 30, 512
    frames = []
    for j in range(J):
        f, _, pitch = _star_frame(device, 40 + j, sigma=1.4 + 0.02 * j)
        frames.append(f)
    stack = torch.stack(frames)
    del frames
    org = [(x, y) for y in range(0, H - T + 1, T) for x in range(0, W - T + 1, T)]
    nt = len(org)
    psfs = np.stack([_gauss_psf(1.4 + 0.02 * j) for j in range(J)])          # one PSF per frame, shared by the tiles
    plan = B.proper_plan_create(device.index, T, nt)
    try:
        d_org = torch.tensor(org, dtype=torch.int32, device=device)
        F = torch.ones(J, device=device)
        sg = torch.full((J,), 18.0, device=device)
        d_psf = torch.from_numpy(psfs).to(device)
        S = torch.empty((nt, T, T), device=device)
        R = torch.empty((nt, T, T), device=device)
        ms = call_ms(lambda: B.argus_proper_coadd(plan, stack, J, B.argus_shape(W, H, pitch), d_org, nt, F, sg, d_psf,
                                                  31, 1e-8, S, R, None, None, None, stream, psf_per_tile=False),
                     3, stream, device)
    finally:
        B.proper_plan_destroy(plan)
    npx = nt * T * T
    return {"workload": f"{J} frames x {nt} tiles of {T}x{T}, one PSF per frame", "ms": round(ms, 3),
            "value": round(npx / 1e6 / (ms / 1e3), 1), "unit": "Mpix/s (coadd pixels)"}


def score_injections(src, n_found, inj, snr, radius=2.0):
    """Injected transients recovered by a detection list: an injection counts as found when a
    positive source's peak pixel lies within `radius` px of it.  Returns the recovered fraction
    per peak-S/N bin, and the detections matched to no injection (positive / negative)."""
    import numpy as np
    n = min(int(n_found), len(src))
    px = src["px"][:n].astype(np.float64)
    py = src["py"][:n].astype(np.float64)
    sign = src["sign"][:n]
    ix, iy = inj.x.numpy(), inj.y.numpy()
    found = np.zeros(len(ix), bool)
    matched = np.zeros(n, bool)
    # sources sorted by (py, px): candidates of an injection lie in a row window
    order_y = py
    for k in range(len(ix)):
        lo = np.searchsorted(order_y, iy[k] - radius, "left")
        hi = np.searchsorted(order_y, iy[k] + radius, "right")
        for j in range(lo, hi):
            if (px[j] - ix[k]) ** 2 + (py[j] - iy[k]) ** 2 <= radius * radius:
                matched[j] = True
                if sign[j] > 0:
                    found[k] = True
    s = snr.numpy()
    bins = [(5, 7), (7, 10), (10, 20.0001)]
    rec = {f"snr_{a}_{int(b)}": round(float(found[(s >= a) & (s < b)].mean()), 4) if ((s >= a) & (s < b)).any() else None
           for a, b in bins}
    return {"recovered": rec, "recovered_all": round(float(found.mean()), 4),
            "unmatched_pos": int(((~matched) & (sign > 0)).sum()), "unmatched_neg": int(((~matched) & (sign < 0)).sum())}


def bench_learned(device, stream, train_pairs, epochs, log=None, crowd=False):
    """Learned kernel vs least-squares fit on a 1-s frame (sky 10 e-, reference 1 px PSF):
    CNN trained on plain-method fits, judged by chi2/dof against the plain fit.
    crowd: the training windows also hold the test frame's field stars (its
    density and flux law)."""
    import torch
    from paper_2207_14304_gb300 import _binding as B
    from paper_2207_14304_gb300 import synth
    from paper_2207_14304_gb300.learned import WIN, KernelNet, LearnedFit, training_set
    from paper_2207_14304_gb300.pipeline import FramePipeline
    t0 = time.time()
    # training pairs from the test frames' domain: 1-s exposures (sky 10 e-), the
    # bright isolated stars that stamp selection picks (1e3-3e4 e-), reference PSF 1 px
    field = None
    if crowd:
        # the frame's catalogue: N_STARS uniform over the frame and a 5-px border, fluxes
        # dN/dF ~ F^-1.5 on [1e2/30, 1e6/30]; a window's field covers it and a 5-px border
        field = (N_STARS / ((W + 10) * (H + 10)) * (WIN + 10) ** 2, 1e2 / 30, 1e6 / 30, -1.5)
    x, t, _ = training_set(train_pairs, seed=5, device=device.index, sky=10.0, flux=(1e3, 3e4), crowd=field)
    net = KernelNet(device=device.index, max_batch=512, seed=5)
    hist = net.fit(x, t, epochs=epochs, batch=512, lr=2e-3, lr_end=1e-4)
    train_s = time.time() - t0
    del x, t
    g = torch.Generator().manual_seed(50)
    sig = float(torch.empty(1).uniform_(1.0, 3.0, generator=g))
    cat = synth.star_catalog(N_STARS, W, H, seed=50, flux_min=1e2 / 30, flux_max=1e6 / 30)
    R, Vr = synth.reference_image(synth.render(cat, W, H, 1.0, sky=10.0, device=device, dtype=torch.float32),
                                  30, 1.7, 51)
    cal = synth.make_calib(W, H, seed=52, device=device)
    # 300 injected transients (science frame only) at peak S/N 5-20 over the sky + read noise
    inj, inj_snr = synth.transient_catalog(300, W, H, seed=54, sigma=sig, noise=math.sqrt(10.0 + 1.7 ** 2))
    Iexp = synth.render(cat, W, H, sig, sky=10.0, device=device, dtype=torch.float32)
    Iexp += synth.render(inj, W, H, sig, device=device, dtype=torch.float32)
    raw = synth.expose(Iexp, cal, seed=53)
    del Iexp
    basis = B.make_basis(KSIZE, (0.7, 1.5, 3.0), (6, 4, 2), SDEG, BGDEG)
    pipe = FramePipeline(W, H, basis=basis, stamp=STAMP, grid=GRID, psf_sigma=sig, max_peak=3.0e4, device=device.index,
                         src_cap=1 << 18, precision="tf32")
    try:
        pitch = pipe.pitch

        def pad(a):
            z = torch.zeros((H, pitch), dtype=a.dtype, device=device)
            z[:, :W] = a
            return z
        d_raw, d_R, d_Vr = pad(raw), pad(R), pad(Vr)
        calib = B.make_calib(cal.bias, pad(cal.dark), pad(cal.flat), pad(cal.bpm), cal.gain, cal.read_noise, cal.sat)
        del raw, R, Vr
        lf = LearnedFit(pipe, net)
        pipe.calibrate(d_raw, calib, stream)
        pipe.select_stamps(d_R, stream)
        plain_ms = timed_ms(lambda: pipe.fit(d_R, stream), 3, stream, device)
        plain = pipe.fit_stats()
        learned_ms = timed_ms(lambda: lf.learned_kernel(d_R, stream), 3, stream, device)
        lst = B.fit_stats_from_bytes(lf.stats)
        ratio = (lst["chi2"] / max(lst["dof"], 1)) / (plain["chi2"] / max(plain["dof"], 1))
        lf.plain_chi2_dof = plain["chi2"] / max(plain["dof"], 1)
        lf.ratio = float("inf")     # learned path as measured: the chi2 check keeps the learned kernel
        frame_ms = timed_ms(lambda: lf.run(d_raw, calib, d_R, d_Vr, stream), 3, stream, device)
        n_learned_src = int(pipe.n_found[0].item())
        src_l, nf_l = pipe.sources_host()
        score_learned = score_injections(src_l, nf_l, inj, inj_snr)
        lf.ratio = 1.1
        used_plain = lf.run(d_raw, calib, d_R, d_Vr, stream)
        judged = "plain (fallback)" if used_plain else "learned"
        plain_frame_ms = timed_ms(lambda: pipe.run(d_raw, calib, d_R, d_Vr, stream), 3, stream, device)
        n_plain_src = int(pipe.n_found[0].item())
        src_p, nf_p = pipe.sources_host()
        score_plain = score_injections(src_p, nf_p, inj, inj_snr)
        st = pipe.status(stream)
    finally:
        pipe.close()
        net.close()
    mpix = W * H / 1e6
    return {"workload": f"{W}x{H} 1-s frame (sky 10 e-), science PSF {sig:.2f} px, reference 1.0 px, 400 stamps",
            "train": {"pairs": train_pairs, "epochs": epochs, "loss_first": hist[0], "loss_last": hist[-1],
                      "seconds": round(train_s, 1),
                      "windows": "one star + the frame's field stars" if crowd else "one star"},
            "fit_ms": {"plain": round(plain_ms, 3), "learned": round(learned_ms, 3)},
            "chi2_per_dof": {"plain": plain["chi2"] / max(plain["dof"], 1), "learned": lst["chi2"] / max(lst["dof"], 1),
                             "ratio": round(ratio, 4)},
            "judge_at_ratio_1.1": judged,
            "sources_5sigma": {"learned_kernel": n_learned_src, "plain_kernel": n_plain_src},
            "injected_transients": {"n": 300, "peak_snr": [5, 20], "match_radius_px": 2.0,
                                    "plain_kernel": score_plain, "learned_kernel": score_learned},
            "frame_mpix_s": {"learned_path": round(mpix / (frame_ms / 1e3), 1),
                             "plain_path": round(mpix / (plain_frame_ms / 1e3), 1)},
            "equal_chi2_within_2pct": bool(abs(ratio - 1) <= 0.02), "status": st}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


# --------------------------------------------------------------------------- CPU oracle arm
def oracle_sample(band_rows=48, seed=2, threads=None):
    """Time the FP64 oracle on a bounded sample of the full-frame workload.

    The kernel fit runs in full (400 stamps, 295 unknowns); calibration,
    subtraction and detection run on a band of `band_rows` full-width rows in
    the middle of the frame (the fit's kernel, frame geometry and spatial terms
    of the full frame).  Frame throughput is extrapolated linearly:
    T_frame = T_fit + T_band * H / band_rows.
    """
    import numpy as np
    import torch

    import oracle
    from paper_2207_14304_gb300 import synth
    if threads:
        oracle.set_threads(threads)
    cores = oracle.num_threads()
    cat = synth.star_catalog(N_STARS, W, H, seed=seed)
    # only the rows the sample touches are rendered: the fit stamps' rows and the band
    y0 = H // 2 - band_rows // 2
    ob = oracle.Basis(ksize=KSIZE, spatial_degree=SDEG, bg_degree=BGDEG)
    Rexp = synth.render(cat, W, H, 1.2, sky=300.0, dtype=torch.float32)
    R, Vr = synth.reference_image(Rexp, 30, 1.7, seed + 1)
    sig = synth.field_sigma(W, H, 1.3, 2.2)
    Iexp = synth.render(cat, W, H, sig, sky=305.0, dtype=torch.float32)
    cal = synth.make_calib(W, H, seed=seed + 2)
    raw = synth.expose(Iexp, cal, seed=seed + 3).numpy()
    R, Vr = R.numpy(), Vr.numpy()
    dark, flat, bpm = cal.dark.numpy(), cal.flat.numpy(), cal.bpm.numpy()
    # fit: calibrate and select on the full frame is part of the per-pixel cost; the
    # oracle's stamp selection runs on the full frame once (timed)
    t0 = time.perf_counter()
    I, V, fl, _ = oracle.calibrate(raw, bias=cal.bias, dark=dark, flat=flat, bpm=bpm, gain=cal.gain,
                                   read_noise=cal.read_noise, sat=cal.sat)
    t_cal_full = time.perf_counter() - t0
    t0 = time.perf_counter()
    cen = oracle.select_stamps(R, fl, GRID[0], GRID[1], STAMP, KSIZE // 2, 3.0e4)
    t_sel = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = oracle.fit(I.astype(np.float32), V.astype(np.float32), R, fl, cen, STAMP, ob)
    K, bg = oracle.expand(ob, res.coeffs)
    t_fit = time.perf_counter() - t0
    # band: subtract + detect with the full-frame geometry
    r = KSIZE // 2
    ys = slice(y0 - r, y0 + band_rows + r)
    t0 = time.perf_counter()
    Db, Vb = oracle.subtract(I[ys].astype(np.float32), V[ys].astype(np.float32), R[ys], Vr[ys], fl[ys], K, bg,
                             sdeg=SDEG, bgdeg=BGDEG, frame=(W, H), origin=(0, y0 - r))
    mask, src, n = oracle.detect(Db[r:-r].astype(np.float32), Vb[r:-r].astype(np.float32), fl[ys][r:-r], 5.0, 1.8)
    t_band = time.perf_counter() - t0
    t_frame = t_cal_full + t_sel + t_fit + t_band * H / band_rows
    return {"value": round(W * H / 1e6 / t_frame, 4), "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "sample": (f"full calibration ({t_cal_full:.2f} s), stamp selection ({t_sel:.2f} s) and 400-stamp "
                       f"kernel fit ({t_fit:.2f} s) of one {W}x{H} frame, subtraction+detection on a "
                       f"{band_rows}-row band ({t_band:.2f} s) scaled x{H / band_rows:.1f} to the frame"),
            "seconds": round(t_cal_full + t_sel + t_fit + t_band, 2)}


def cpu_baseline(args):
    try:
        return oracle_sample(band_rows=args.band_rows)
    except Exception as e:   # the GPU line stays valid without the baseline
        return {"value": None, "unit": "Mpix/s", "cores": None, "kind": "oracle", "sample": f"failed: {e!r}"}


def run_reference(args):
    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return
    import oracle
    oracle.build()
    vals, secs = [], []
    last = None
    for _ in range(max(1, args.steps)):
        last = oracle_sample(band_rows=args.band_rows)
        vals.append(last["value"])
        secs.append(last["seconds"])
    v = statistics.median(vals)
    # each step runs a bounded sample (a band of rows for the subtraction and detection);
    # ms_per_step is the full frame's time extrapolated from it, not the sample's wall time
    out = {"metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(W * H / 1e6 / v * 1e3, 2),
           "ms_per_step_kind": "extrapolated from the sample to the full frame",
           "sample_seconds_per_step": round(statistics.median(secs), 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config("fp64"), "impl": "reference",
           "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": last["cores"], "kind": "oracle",
                            "sample": last["sample"]},
           "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    # TF32 normal equations on the tensor cores by default: they meet the 1e-3 kernel-pixel bar
    # on the full frame; --precision fp32 / bf16 / bf16_split select the others
    ap.add_argument("--precision", default="tf32", choices=["fp32", "tf32", "bf16", "bf16_split"])
    ap.add_argument("--band-rows", type=int, default=48)
    ap.add_argument("--frames-in-flight", type=int, default=4,
                    help="frames processed concurrently, each on its own pipeline and stream")
    ap.add_argument("--no-fused", dest="fused", action="store_false",
                    help="capture the separate calls (argus_calibrate .. argus_detect) instead of argus_dia_frame")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-clocks", dest="clocks", action="store_false")
    ap.add_argument("--extras", default="coadd,segments,learned,sparse,background,healpix,zogy,proper_coadd",
                    help="comma list of the extra workloads to measure after the headline")
    ap.add_argument("--no-extras", dest="extras", action="store_const", const="")
    ap.add_argument("--frame", type=int, nargs=2, metavar=("W", "H"), default=None,
                    help="smaller frame for profiling captures (star count scaled by area)")
    ap.add_argument("--segment-cameras", type=int, default=38)
    ap.add_argument("--train-pairs", type=int, default=100_000)
    ap.add_argument("--train-epochs", type=int, default=16)
    ap.add_argument("--train-crowd", default="none", choices=["none", "frame"],
                    help="field stars in the learned kernel's training windows: none, or the test frame's")
    args = ap.parse_args(argv)
    if args.frame:
        global W, H, N_STARS
        fw, fh = args.frame
        N_STARS = max(1, int(N_STARS * fw * fh / (W * H)))
        W, H = fw, fh
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        args.steps = min(args.steps, 3)
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
