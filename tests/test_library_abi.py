"""The C-ABI library loads (no GPU needed) and exports every entry point that
include/*.h declares; the binding's struct layouts match the header."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(argus_\w+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2207_14304_gb300 import _binding as B
    lib = B.load()
    names = declared_symbols()
    assert len(names) >= 11
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    for n in names:
        assert n in B.SIGNATURES or n in getattr(B, "EXTRA_SIGNATURES", {}), f"binding lacks {n}"


def test_status_strings_and_struct_sizes():
    from paper_2207_14304_gb300 import _binding as B
    B.load()
    assert B.status_string(0) == "ok"
    assert "positive definite" in B.status_string(-5)
    assert C.sizeof(B.argus_source) == 36
    assert C.sizeof(B.argus_fit_stats) == 64
    assert C.sizeof(B.argus_shape) == 16


def test_host_argument_checks_need_no_gpu():
    """Argument errors are returned before any CUDA call."""
    from paper_2207_14304_gb300 import _binding as B
    lib = B.load()
    assert lib.argus_create(None, 0, 1, 1, 16, 1) == B.ARGUS_ERR_ARG
    assert lib.argus_destroy(None) == B.ARGUS_ERR_ARG
    sh = B.argus_shape(10, 10, 10)   # pitch not a multiple of 16
    cal = B.make_calib()
    assert lib.argus_calibrate(None, None, sh, C.byref(cal), None, None, None, None) == B.ARGUS_ERR_ARG
    sh = B.argus_shape(64, 8, 64)
    # sparse products: NULL context, bad cell size / factor
    assert lib.argus_minipix(None, None, sh, 9, None, 0, None, None, 0, None, None, None, None, 0, None,
                             None) == B.ARGUS_ERR_ARG
    assert lib.argus_lowres(None, None, None, sh, 10, None, 16, None) == B.ARGUS_ERR_ARG
    assert lib.argus_background(None, None, None, sh, 64, 3, 0.5, None, None, None) == B.ARGUS_ERR_ARG
    plan = C.c_void_p()
    assert lib.argus_proper_plan_create(0, 300, 4, C.byref(plan)) == B.ARGUS_ERR_ARG      # tile not a power of two
    assert lib.argus_proper_plan_destroy(None) == B.ARGUS_ERR_ARG
    assert lib.argus_zogy(None, None, None, sh, None, 1, None, None, 31, 1, 1e-8, None, None, None, None,
                          None) == B.ARGUS_ERR_ARG
    assert C.sizeof(C.c_int) * 2 + C.sizeof(C.c_float) * 4 == np_zogy_tile_itemsize()


def np_zogy_tile_itemsize():
    import numpy as np
    from paper_2207_14304_gb300 import _binding as B
    return np.dtype(B.ZOGY_TILE_DTYPE).itemsize


def test_proper_coadd_argument_checks_need_no_gpu():
    from paper_2207_14304_gb300 import _binding as B
    lib = B.load()
    sh = B.argus_shape(64, 8, 64)
    assert lib.argus_proper_coadd(None, None, 2, sh, None, 1, None, None, None, 31, 1, 1e-8, None, None, None, None,
                                  None, None) == B.ARGUS_ERR_ARG


def test_healpix_argument_checks_need_no_gpu():
    from paper_2207_14304_gb300 import _binding as B
    lib = B.load()
    sh = B.argus_shape(64, 8, 64)
    wcs = B.argus_wcs(0.0, 0.0, 1e-5, 0.0, 32.0, 4.0)
    assert lib.argus_healpix_resample(None, None, sh, wcs, 256, 9, None, 1, None, None, None) == B.ARGUS_ERR_ARG
    assert C.sizeof(B.argus_wcs) == 48


def test_binding_argument_counts_match_the_header():
    """Every entry point the binding declares takes as many arguments as its prototype."""
    from paper_2207_14304_gb300 import _binding as B
    txt = ""
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt += re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(argus_\w+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S):
        params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        protos[m.group(1)] = len(params)
    checked = 0
    for name, (args, _) in B.SIGNATURES.items():
        if name in protos:
            assert protos[name] == len(args), (name, protos[name], len(args))
            checked += 1
    assert checked >= 30
