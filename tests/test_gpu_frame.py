"""argus_dia_frame: the whole per-frame path from the raw frame in one call, against
the same steps called one by one (argus_calibrate .. argus_detect, each checked
against the oracle in tests/test_gpu_parity.py): every output is compared bit for
bit.  The calibrated flags and the stamp centres are also checked
against the oracle here, and the detection by properties that hold at any size."""
import numpy as np
import pytest
import torch

from paper_2207_14304_gb300 import _binding as B
from paper_2207_14304_gb300.pipeline import FramePipeline
from tests.gpu_helpers import check_detection_properties, dev_pitched
from tests.test_gpu_parity import _fit_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()


@pytest.mark.parametrize("w,h,ks,sdeg,grid,prec", [(700, 500, 21, 2, (5, 4), "tf32"),      # tensor cores, 256-row bands
                                                   (512, 384, 11, 0, (4, 4), "fp32"),      # tensor cores, one term
                                                   (400, 300, 15, 1, (4, 3), "bf16_split")])  # FP32 subtraction
def test_dia_frame_equals_the_separate_calls(ora, w, h, ks, sdeg, grid, prec):
    R, Vr, I, V, fl, raw, cal = _fit_field(w, h, seed=w + ks, sdeg=sdeg)
    basis = B.make_basis(ks, (0.7, 1.5, 3.0), (6, 4, 2), sdeg, sdeg)
    kw = dict(basis=basis, stamp=21, grid=grid, precision=prec, psf_sigma=1.8)
    a, b = FramePipeline(w, h, **kw), FramePipeline(w, h, **kw)
    try:
        d_raw, d_R, d_Vr = dev_pitched(raw), dev_pitched(R), dev_pitched(Vr)
        calib = B.make_calib(cal.bias, dev_pitched(cal.dark.numpy()), dev_pitched(cal.flat.numpy()),
                             dev_pitched(cal.bpm.numpy()), cal.gain, cal.read_noise, cal.sat)
        for p in (a, b):   # garbage in the outputs first: everything must be written
            for t in (p.diff, p.diff_var):
                t.fill_(-7.0)
            p.mask.fill_(0xEE)
        a.run(d_raw, calib, d_R, d_Vr)
        b.run_fused(d_raw, calib, d_R, d_Vr)
        torch.cuda.synchronize()
        assert a.status() == 0 and b.status() == 0
        for name in ("img", "var", "flags", "centers", "n_stamps", "coeffs", "K", "bg", "diff", "diff_var", "mask"):
            ta, tb = getattr(a, name), getattr(b, name)
            assert torch.equal(ta, tb), name
        sa, na = a.sources_host()
        sb, nb = b.sources_host()
        assert na == nb and sa.tobytes() == sb.tobytes()
        # anchors to the oracle: calibration flags and stamp centres are exact
        fo = fl                                   # the oracle's flags of this raw frame
        np.testing.assert_array_equal(b.flags[:, :w].cpu().numpy(), fo)
        cen = ora.select_stamps(R, fo, grid[0], grid[1], 21, ks // 2, 3.0e4)
        n = int(b.n_stamps[0].item())
        assert n == len(cen) and (b.centers[:n].cpu().numpy() == cen).all()
        D, VD, M = (t[:, :w].cpu().numpy() for t in (b.diff, b.diff_var, b.mask))
        n_p, n_n = check_detection_properties(D, VD, fo, M, sb, nb, 5.0)
        print(f"\n[dia_frame {w}x{h} ks{ks} sdeg{sdeg} {prec}] stamps {n}, sources {nb} (+{n_p} / -{n_n})")
    finally:
        a.close()
        b.close()
