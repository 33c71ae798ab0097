"""GB300-native (sm_103a) difference-image-analysis path of the Argus Array
Hierarchical Data Processing System (Corbett et al. 2022, arXiv:2207.14304).

The computation lives in libargusdia.so (hand-written CUDA behind the C ABI of
include/argus_dia.h); this package only loads it, marshals arguments
(``_binding``), composes the per-frame path (``pipeline``) and generates seeded
synthetic inputs (``synth``).  There is no CPU fallback: without the library
every call raises.
"""
from . import _binding as binding  # noqa: F401
from ._binding import (ArgusError, argus_calibrate, argus_coadd, argus_create, argus_destroy,  # noqa: F401
                       argus_detect, argus_expand_kernel, argus_fit_kernel, argus_select_stamps,
                       argus_subtract, argus_sync_status, load, make_basis, make_calib, shape_of)
