"""Shared helpers of the GPU parity tests: pitched device copies and tolerances."""
import numpy as np
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300.synth import pitch_for

F32_EPS = 2.0 ** -24


def dev_pitched(a: np.ndarray, pitch: int | None = None, fill=0) -> torch.Tensor:
    """Copy a [h, w] host array into a [h, pitch] CUDA tensor; padding is `fill`."""
    h, w = a.shape
    pitch = pitch or pitch_for(w)
    t = torch.full((h, pitch), fill, dtype=torch.from_numpy(np.ascontiguousarray(a)).dtype)
    t[:, :w] = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda()


def host(t: torch.Tensor, w: int) -> np.ndarray:
    return t[:, :w].cpu().numpy()


def ctx_for(w, h, max_stamps=64, max_coeffs=320, det_cap=1 << 20):
    return B.argus_create(0, h * pitch_for(w), max_stamps, max_coeffs, det_cap)


def assert_rel(gpu, ref, scale, rtol, what=""):
    """|gpu - ref| <= rtol * scale elementwise, reporting the worst offender."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(gpu - ref) / np.maximum(scale, 1e-300)
    i = int(np.argmax(err)) if err.size else 0
    assert err.size == 0 or err.flat[i] <= rtol, (
        f"{what}: worst rel err {err.flat[i]:.3e} > {rtol:.1e} at {np.unravel_index(i, err.shape)}: "
        f"gpu {gpu.flat[i]!r} ref {ref.flat[i]!r}")
    return float(err.max()) if err.size else 0.0
