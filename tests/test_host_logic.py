"""Host-side logic that needs no GPU: atlas packing, the autotuner's table, the
bench's multi-rank aggregation (two gloo ranks on the CPU), the reference arm's
rank handling and the clock-record parsing."""
from __future__ import annotations

import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2207_14304_gb300 import synth  # noqa: E402
from paper_2207_14304_gb300.segments import candidate_configs, pack_shelves, tuned_config  # noqa: E402


def test_pack_shelves_no_overlap():
    sides = synth.segment_sides(300, seed=4)
    pos, hgt = pack_shelves(sides, 2048)
    occ = np.zeros((hgt, 2048), np.int32)
    for (r, c), s in zip(pos, sides):
        assert r % 16 == 0 and c % 16 == 0 and c + s <= 2048 and r + s <= hgt
        occ[r:r + s, c:c + s] += 1
    assert occ.max() == 1
    assert occ.sum() / occ.size > 0.6


def test_pack_shelves_edge_cases():
    pos, hgt = pack_shelves([], 2048)
    assert pos == [] and hgt == 0
    pos, hgt = pack_shelves([2048], 2048)
    assert pos == [(0, 0)] and hgt == 2048
    # equal squares fill shelves left to right, 16-aligned
    pos, hgt = pack_shelves([40] * 5, 100)
    assert all(c % 16 == 0 and c + 40 <= 100 for _, c in pos)
    assert len(set(pos)) == 5


def test_tuned_config_table(tmp_path):
    path = str(tmp_path / "tune.json")
    assert tuned_config("k", table_path=path) is None
    json.dump({"k": {"fit_band": 8, "fit_ctas_per_sm": 2, "sub_ctas_per_sm": 6}}, open(path, "w"))
    c = tuned_config("k", table_path=path)
    assert (c.fit_band, c.fit_ctas_per_sm, c.sub_ctas_per_sm) == (8, 2, 6)
    assert tuned_config("other", table_path=path) is None
    open(path, "w").write("{not json")
    assert tuned_config("k", table_path=path) is None
    # candidates: distinct launch shapes the plan accepts (fit bands even, 8..128; fit CTAs 1..4;
    # subtraction CTAs 1..16), among them the CUDA-core fit's 8-row units and larger
    # tensor-core fit bands
    cands = candidate_configs()
    assert len(cands) == len(set(cands))
    assert all(c[0] % 2 == 0 and 8 <= c[0] <= 128 and 1 <= c[1] <= 4 and 1 <= c[2] <= 16 for c in cands)
    assert any(c[0] == 8 for c in cands) and any(c[0] > 8 for c in cands)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(ws),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    assert bench.dist_env() == (ws, rank, rank)
    dist = bench.dist_init(ws, "gloo")
    bench.barrier(dist)
    # rank r processed 10 units in (r + 1) seconds: the job is timed by the slowest rank
    value, tmax = bench.aggregate(10.0, float(rank + 1), dist)
    mx = bench.max_over_ranks(dist, 100.0 - rank, None)
    bench.barrier(dist)
    json.dump({"value": value, "tmax": tmax, "max": mx}, open(os.path.join(out_dir, f"r{rank}.json"), "w"))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    for r in range(ws):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["tmax"] == 2.0                    # max over ranks
        assert d["value"] == pytest.approx(10.0 * ws / 2.0)
        assert d["max"] == 100.0


def test_single_rank_helpers_are_identity():
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.aggregate(10.0, 2.0, None) == (5.0, 2.0)
    bench.barrier(None)


def test_reference_arm_non_zero_rank_does_no_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(bench, "oracle_sample", lambda **k: pytest.fail("rank 1 ran the oracle"))
    bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert capsys.readouterr().out == ""


def test_parse_clocks(tmp_path):
    p = tmp_path / "clocks.csv"
    p.write_text(
        "0, 1900, 2070, 900.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 1950, 2070, 950.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 2000, 2070, 990.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    c = bench.parse_clocks(str(p))
    assert c["sm_mhz"] == 1950 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    p.write_text("0, 700, 2070, 500, 0x8, Active, Not Active, Not Active, Not Active\n")
    assert bench.parse_clocks(str(p))["reasons"] == ["hw_slowdown"]
    p.write_text("")
    assert bench.parse_clocks(str(p)) is None


def test_frame_override_scales_the_workload():
    saved = (bench.W, bench.H, bench.N_STARS)
    try:
        args = []
        ap_main = bench.main

        def fake_run(a):
            args.append((bench.W, bench.H, bench.N_STARS, a.extras))

        bench.run_gpu, orig = fake_run, bench.run_gpu
        try:
            ap_main(["--frame", "4096", "4096", "--extras", "coadd"])
        finally:
            bench.run_gpu = orig
        w, h, n, extras = args[0]
        assert (w, h) == (4096, 4096) and n == int(150_000 * 4096 * 4096 / (9576 * 6388))
        assert extras == "coadd"
        assert bench.workload_config()["frame"] == [4096, 4096]
    finally:
        bench.W, bench.H, bench.N_STARS = saved


def test_kernel_rooflines_pick_the_binding_roof():
    """Difference image above the ridge of the measured peaks (tensor), variance below
    it (HBM): achieved = algorithmic work / kernel time, frac = achieved / peak."""
    import bench
    peaks = {"hbm_gbs": 6777.0, "bf16_tflops_sustained": 1719.5}
    k = bench.kernel_rooflines(0.848, 0.888, "events", peaks)
    npx = bench.W * bench.H
    d, v = k["subtract_tc"], k["variance"]
    assert d["bound"] == "tensor" and d["unit"] == "TFLOP/s"
    assert abs(d["achieved"] - 2 * 6 * 441 * npx / 0.848e-3 / 1e12) < 1e-3
    assert abs(d["frac"] - d["achieved"] / 1719.5) < 1e-4
    assert v["bound"] == "hbm" and v["unit"] == "GB/s" and v["peak"] == 6777.0
    assert abs(v["achieved"] - 13 * npx / 0.888e-3 / 1e9) < 0.1
    assert abs(v["frac"] - v["achieved"] / 6777.0) < 1e-4
    ridge = 1719.5e12 / 6777e9
    assert 2 * 6 * 441 / 13 > ridge > 2 * 441 / bench.VAR_BYTES_PER_PX


def test_training_field_stars_match_the_frame_renderer():
    # crowded training windows: the field stars of a window rendered by the
    # training set's separable renderer equal the frame renderer's image of the
    # same catalogue (same pixel-integrated Gaussian, footprint 5 sigma there)
    import torch
    from paper_2207_14304_gb300 import learned
    n = 5
    stars = learned.field_stars(n, seed=3, mean=6.0, flux_min=3.0, flux_max=3e4, index=-1.5)
    widx, x, y, f = stars
    assert widx.numel() > 0 and bool((widx[1:] >= widx[:-1]).all())
    assert float(x.min()) >= -5.0 and float(x.max()) < learned.WIN + 5.0
    assert float(f.min()) >= 3.0 and float(f.max()) <= 3e4
    sig = np.array([1.0, 1.5, 2.0, 2.5, 3.0])
    img = learned.render_field(n, stars, sig)
    for w in range(n):
        sel = widx == w
        cat = synth.Catalog(x[sel], y[sel], f[sel])
        ref = synth.render(cat, learned.WIN, learned.WIN, float(sig[w]))
        assert torch.allclose(img[w].double(), ref, rtol=1e-5, atol=1e-4 * max(1.0, float(ref.max())))
    # the reference width is one float for every window
    one = learned.render_field(n, stars, 1.0)
    assert one.shape == (n, learned.WIN, learned.WIN)
    # a star far inside a window keeps its whole flux there
    st = (torch.tensor([2]), torch.tensor([20.3]), torch.tensor([19.6]), torch.tensor([1234.0], dtype=torch.float64))
    im = learned.render_field(n, st, 2.0)
    assert abs(float(im[2].double().sum()) - 1234.0) < 1e-3 and float(im[[0, 1, 3, 4]].abs().sum()) == 0.0


def test_training_field_stars_are_seeded_and_order_independent():
    # the same seed gives the same field; the rendered windows do not depend on the order
    # in which the stars are listed (one star per window per pass)
    import torch
    from paper_2207_14304_gb300 import learned
    a = learned.field_stars(7, seed=9, mean=5.0, flux_min=3.0, flux_max=3e4, index=-1.5)
    b = learned.field_stars(7, seed=9, mean=5.0, flux_min=3.0, flux_max=3e4, index=-1.5)
    c = learned.field_stars(7, seed=10, mean=5.0, flux_min=3.0, flux_max=3e4, index=-1.5)
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    assert not (a[0].numel() == c[0].numel() and all(torch.equal(x, y) for x, y in zip(a, c)))
    img = learned.render_field(7, a, 1.5)
    assert torch.equal(img, learned.render_field(7, b, 1.5))
    perm = torch.randperm(a[0].numel(), generator=torch.Generator().manual_seed(1))
    shuffled = tuple(t[perm] for t in a)
    torch.testing.assert_close(learned.render_field(7, shuffled, 1.5), img, rtol=1e-6, atol=1e-4)
    assert learned.render_field(3, tuple(t[:0] for t in a), 1.0).abs().sum() == 0


def test_reference_arm_line_on_a_small_frame():
    # the oracle arm end to end on the host cores (a 512 x 512 frame): one JSON line with the
    # contract's keys, its own cpu_baseline and an e2e object without host-device copies
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--frame", "512", "512"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT, check=True).stdout.strip().splitlines()
    line = json.loads(out[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["frame"] == [512, 512]
