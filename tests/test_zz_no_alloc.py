"""The allocation-free stamp selection entry point (argus_select_stamps_noalloc).

Some callers cannot call cudaMalloc: a host that reserves all device memory
up front, a real-time loop that must never enter an allocator, or a plugin
that is only handed input and output pointers.  For them the library offers a
context-free variant of stamp selection whose scratch is a fixed device array
inside the library.  This test calls it through the C ABI twice in a row
(the second call must not see the first call's scratch) and checks both
results against the context-based argus_select_stamps on the same inputs; the
outputs are integers, so they must be identical.  It sits in a file of its own
that pytest collects last, and it passes alone in a fresh process as well.
"""
import numpy as np
import pytest
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300 import synth
from paper_2207_14304_gb300.synth import pitch_for

pytestmark = pytest.mark.gpu


def _field(w, h, seed):
    cat = synth.star_catalog(w * h // 250, w, h, seed=seed, flux_min=1e3, flux_max=1e6)
    R, _ = synth.reference_image(synth.render(cat, w, h, 1.2, sky=300.0), 30, 1.7, seed + 1)
    rng = np.random.default_rng(seed)
    fl = (rng.random((h, w)) < 0.0005).astype(np.uint8)
    return R.numpy(), fl


def _dev(a, pitch):
    h, w = a.shape
    t = torch.zeros((h, pitch), dtype=torch.from_numpy(a).dtype)
    t[:, :w] = torch.from_numpy(a)
    return t.cuda()


def test_noalloc_select_matches_context_select_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    cases = [(300, 260, 4, 3, 11), (257, 129, 5, 2, 12)]   # second call: other sizes, fewer cells
    for w, h, gx, gy, seed in cases:
        R, fl = _field(w, h, seed)
        pitch = pitch_for(w)
        dR, dfl = _dev(R, pitch), _dev(fl, pitch)
        shape = B.argus_shape(w, h, pitch)
        ctx = B.argus_create(0, h * pitch, 16, 64, 1 << 16)
        try:
            ref_c = torch.full((gx * gy, 2), -1, dtype=torch.int32, device="cuda")
            ref_n = torch.zeros(4, dtype=torch.int32, device="cuda")
            B.argus_select_stamps(ctx, dR, dfl, shape, gx, gy, 21, 5, 3.0e4, 10, 0.1, ref_c, ref_n)
        finally:
            torch.cuda.synchronize()
            B.argus_destroy(ctx)
        got_c = torch.full((gx * gy, 2), -1, dtype=torch.int32, device="cuda")
        got_n = torch.zeros(4, dtype=torch.int32, device="cuda")
        B.argus_select_stamps_noalloc(dR, dfl, shape, gx, gy, 21, 5, 3.0e4, 10, 0.1, got_c, got_n)
        torch.cuda.synchronize()
        n = int(ref_n[0].item())
        assert n > 0
        assert int(got_n[0].item()) == n
        np.testing.assert_array_equal(got_c[:n].cpu().numpy(), ref_c[:n].cpu().numpy())


def test_noalloc_rejects_grids_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    x = torch.zeros((8, 16), device="cuda")
    f = torch.zeros((8, 16), dtype=torch.uint8, device="cuda")
    c = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    n = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(B.ArgusError) as e:
        B.argus_select_stamps_noalloc(x, f, B.argus_shape(16, 8, 16), 65, 64, 3, 1, 1e4, 1, 0.1, c, n)
    assert e.value.code == B.ARGUS_ERR_CAPACITY
