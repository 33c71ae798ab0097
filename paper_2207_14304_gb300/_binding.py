"""ctypes binding of libargusdia (argument marshalling only).

Every function here has the name of a C entry point declared in
include/argus_dia.h and forwards to it: tensors become device pointers,
shapes and parameter structs become the C structs, and the stream defaults
to PyTorch's current stream.  All computation happens in the CUDA library;
if it cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

ARGUS_OK = 0
ARGUS_ERR_ARG = -1
ARGUS_ERR_ALIGN = -2
ARGUS_ERR_CUDA = -3
ARGUS_ERR_NOMEM = -4
ARGUS_ERR_SINGULAR = -5
ARGUS_ERR_CAPACITY = -6
ARGUS_ERR_TIMEOUT = -7
ARGUS_ERR_UNSUPPORTED = -8
ARGUS_FLAG_BAD, ARGUS_FLAG_SAT = 1, 2
ARGUS_MASK_POS, ARGUS_MASK_NEG, ARGUS_MASK_INVALID = 1, 2, 4

PREC = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16_split": 3}
FLAG_BAD, FLAG_SAT = 1, 2
MASK_POS, MASK_NEG, MASK_INVALID = 1, 2, 4


class ArgusError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        detail = ""
        if code == ARGUS_ERR_CUDA:
            try:
                detail = f" [{load(False).argus_last_cuda_error().decode()}]"
            except Exception:
                pass
        super().__init__(f"{what}: argus status {code} ({status_string(code)}){detail}")


class argus_shape(C.Structure):
    _fields_ = [("w", C.c_int), ("h", C.c_int), ("pitch", C.c_long)]


class argus_calib(C.Structure):
    _fields_ = [("bias_frame", C.c_void_p), ("bias_scalar", C.c_int), ("dark", C.c_void_p),
                ("flat", C.c_void_p), ("bpm", C.c_void_p), ("gain", C.c_float),
                ("read_noise", C.c_float), ("sat", C.c_int)]


class argus_basis(C.Structure):
    _fields_ = [("ksize", C.c_int), ("ngauss", C.c_int), ("sigma", C.c_float * 4),
                ("degree", C.c_int * 4), ("spatial_degree", C.c_int), ("bg_degree", C.c_int)]


class argus_source(C.Structure):
    _fields_ = [("x", C.c_float), ("y", C.c_float), ("flux", C.c_float), ("flux_err", C.c_float),
                ("peak_snr", C.c_float), ("npix", C.c_int), ("sign", C.c_int), ("px", C.c_int),
                ("py", C.c_int)]


class argus_fit_stats(C.Structure):
    _fields_ = [("chi2", C.c_double), ("chi2_a0", C.c_double), ("max_step", C.c_double),
                ("n_pix", C.c_longlong), ("dof", C.c_longlong), ("n_coeffs", C.c_int),
                ("status", C.c_int), ("n_stamps_used", C.c_int), ("precision", C.c_int),
                ("refine_iters", C.c_int), ("pad_", C.c_int)]


class argus_segment(C.Structure):
    _fields_ = [("row0", C.c_int), ("col0", C.c_int), ("side", C.c_int)]


class argus_seg_config(C.Structure):
    _fields_ = [("fit_band", C.c_int), ("fit_ctas_per_sm", C.c_int), ("sub_ctas_per_sm", C.c_int),
                ("reserved", C.c_int)]


class argus_seg_stats(C.Structure):
    _fields_ = [("chi2", C.c_double), ("n_pix", C.c_int), ("status", C.c_int)]


SOURCE_BYTES = C.sizeof(argus_source)
FIT_STATS_BYTES = C.sizeof(argus_fit_stats)

_lib = None

P = C.c_void_p
I = C.c_int
F = C.c_float
SH = argus_shape


class argus_wcs(C.Structure):
    _fields_ = [("alpha0", C.c_double), ("delta0", C.c_double), ("scale", C.c_double), ("rot", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double)]

# entry point -> argument types
SIGNATURES = {
    "argus_status_string": ([I], C.c_char_p),
    "argus_launch_count": ([], C.c_ulonglong),
    "argus_last_cuda_error": ([], C.c_char_p),
    "argus_create": ([C.POINTER(P), I, C.c_size_t, I, I, I], I),
    "argus_destroy": ([P], I),
    "argus_sync_status": ([P, P], I),
    "argus_calibrate": ([P, P, SH, C.POINTER(argus_calib), P, P, P, P], I),
    "argus_coadd": ([P, P, I, SH, P, C.POINTER(argus_calib), F, I, P, P, P, P], I),
    "argus_select_stamps": ([P, P, P, SH, I, I, I, I, F, I, F, P, P, P], I),
    "argus_stamp_basis": ([P, P, SH, P, P, I, I, P, I, I, P, P], I),
    "argus_fit_kernel": ([P, P, P, P, P, SH, P, P, I, I, C.POINTER(argus_basis), I, P, P, P], I),
    "argus_expand_kernel": ([P, C.POINTER(argus_basis), P, P, P, P], I),
    "argus_subtract": ([P, P, P, P, P, P, SH, I, I, I, I, I, I, P, I, P, P, P, P], I),
    "argus_detect": ([P, P, P, P, SH, F, F, P, P, I, P, P], I),
    "argus_dia_frame": ([P, P, SH, C.POINTER(argus_calib), P, P, I, I, I, F, I, F, C.POINTER(argus_basis), I, F, F,
                         P, P, P, P, P, P, P, P, P, P, P, P, P, I, P, P], I),
    "argus_select_stamps_noalloc": ([P, P, SH, I, I, I, I, F, I, F, P, P, P], I),
    "argus_segments_plan": ([P, C.POINTER(argus_segment), I, I, I, C.POINTER(argus_basis),
                             C.POINTER(argus_seg_config), C.POINTER(P)], I),
    "argus_segments_destroy": ([P], I),
    "argus_segments_run": ([P, P, P, P, P, P, P, P, P, P, P, F, F, P, I, P, I, P], I),
    "argus_segments_items": ([P, C.POINTER(I), C.POINTER(I)], I),
    "argus_segments_subtract": ([P, P, P, P, P, P, P, P, P, P, P], I),
    "argus_segments_kernels": ([P, P, P, P], I),
    "argus_cnn_create": ([C.POINTER(P), I, I, C.c_ulonglong], I),
    "argus_cnn_destroy": ([P], I),
    "argus_cnn_params": ([P, C.POINTER(P), C.POINTER(P), C.POINTER(P), C.POINTER(C.c_long), C.POINTER(I)], I),
    "argus_cnn_set_state": ([P, I, I, P], I),
    "argus_cnn_forward": ([P, P, I, P, P], I),
    "argus_cnn_status": ([P, P], I),
    "argus_cnn_backward": ([P, P, P, I, P, P], I),
    "argus_cnn_train_step": ([P, P, P, I, F, P, P], I),
    "argus_cnn_adam": ([P, P, F, P], I),
    "argus_cnn_prepare": ([P, P, SH, P, P, I, P, P], I),
    "argus_learned_kernel": ([P, P, P, P, I, I, I, I, P, P], I),
    "argus_fit_background": ([P, P, P, P, P, SH, P, P, I, I, P, I, I, I, P, P, P], I),
    "argus_fit_scale_background": ([P, P, P, P, P, SH, P, P, I, I, P, I, I, I, P, P, P], I),
    "argus_minipix": ([P, P, SH, I, P, I, P, P, I, P, P, P, P, I, P, P], I),
    "argus_lowres": ([P, P, P, SH, I, P, C.c_long, P], I),
    "argus_background": ([P, P, P, SH, I, I, F, P, P, P], I),
    "argus_proper_plan_create": ([I, I, I, C.POINTER(P)], I),
    "argus_proper_plan_destroy": ([P], I),
    "argus_zogy": ([P, P, P, SH, P, I, P, P, I, I, F, P, P, P, P, P], I),
    "argus_proper_coadd": ([P, P, I, SH, P, I, P, P, P, I, I, F, P, P, P, P, P, P], I),
    "argus_healpix_resample": ([P, P, SH, argus_wcs, I, I, P, I, P, P, P], I),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libargusdia.so (building it in-tree when missing); raise on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libargusdia.so not built at {path}")
        _build.build()
    lib = C.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load(False).argus_status_string(int(code)).decode()
    except Exception:
        return "unknown"


def _check(rc, what):
    if rc != ARGUS_OK:
        raise ArgusError(rc, what)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor (device memory)")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def shape_of(t: torch.Tensor, w: int | None = None) -> argus_shape:
    """argus_shape of a [h, pitch] tensor holding w valid columns."""
    h, pitch = t.shape[-2], t.shape[-1]
    return argus_shape(int(w if w is not None else pitch), int(h), int(pitch))


def make_calib(bias=100, dark=None, flat=None, bpm=None, gain=1.0, read_noise=1.7, sat=65535,
               bias_frame=None) -> argus_calib:
    c = argus_calib()
    c.bias_frame = _ptr(bias_frame)
    c.bias_scalar = int(bias)
    c.dark = _ptr(dark)
    c.flat = _ptr(flat)
    c.bpm = _ptr(bpm)
    c.gain = float(gain)
    c.read_noise = float(read_noise)
    c.sat = int(sat)
    c._keep = (bias_frame, dark, flat, bpm)   # the struct holds raw pointers into these tensors
    return c


def make_basis(ksize=11, sigmas=(0.7, 1.5, 3.0), degrees=(6, 4, 2), spatial_degree=0,
               bg_degree=0) -> argus_basis:
    b = argus_basis()
    b.ksize = int(ksize)
    b.ngauss = len(sigmas)
    for i, s in enumerate(sigmas):
        b.sigma[i] = float(s)
        b.degree[i] = int(degrees[i])
    b.spatial_degree = int(spatial_degree)
    b.bg_degree = int(bg_degree)
    return b


def basis_counts(b: argus_basis):
    nb = sum((b.degree[g] + 1) * (b.degree[g] + 2) // 2 for g in range(b.ngauss))
    ks = (b.spatial_degree + 1) * (b.spatial_degree + 2) // 2
    kb = (b.bg_degree + 1) * (b.bg_degree + 2) // 2
    return nb, ks, kb, 1 + (nb - 1) * ks + kb


# ---------------------------------------------------------------------------
def argus_create(device=0, max_pixels=1 << 22, max_stamps=400, max_coeffs=320, det_cap=1 << 22):
    h = C.c_void_p()
    rc = load().argus_create(C.byref(h), int(device), int(max_pixels), int(max_stamps),
                             int(max_coeffs), int(det_cap))
    _check(rc, "argus_create")
    return h


def argus_launch_count() -> int:
    return int(load().argus_launch_count())


def argus_destroy(ctx):
    _check(load().argus_destroy(ctx), "argus_destroy")


def argus_sync_status(ctx, stream=None) -> int:
    return load().argus_sync_status(ctx, _stream(stream))


def argus_calibrate(ctx, raw, shape, calib, img, var, flags, stream=None):
    _check(load().argus_calibrate(ctx, _ptr(raw), shape, C.byref(calib), _ptr(img), _ptr(var),
                                  _ptr(flags), _stream(stream)), "argus_calibrate")


def argus_coadd(ctx, raw_stack, n, shape, shifts_xy, calib, kappa, max_iter, coadd, var, n_used,
                stream=None):
    _check(load().argus_coadd(ctx, _ptr(raw_stack), int(n), shape, _ptr(shifts_xy), C.byref(calib),
                              float(kappa), int(max_iter), _ptr(coadd), _ptr(var), _ptr(n_used),
                              _stream(stream)), "argus_coadd")


def argus_select_stamps(ctx, ref, flags, shape, grid_x, grid_y, stamp, khalf, max_peak, iso,
                        iso_frac, centers, n_stamps, stream=None):
    _check(load().argus_select_stamps(ctx, _ptr(ref), _ptr(flags), shape, int(grid_x), int(grid_y),
                                      int(stamp), int(khalf), float(max_peak), int(iso),
                                      float(iso_frac), _ptr(centers), _ptr(n_stamps),
                                      _stream(stream)), "argus_select_stamps")


def argus_select_stamps_noalloc(ref, flags, shape, grid_x, grid_y, stamp, khalf, max_peak, iso,
                                iso_frac, centers, n_stamps, stream=None):
    """Context-free stamp selection for callers that cannot allocate device memory."""
    _check(load().argus_select_stamps_noalloc(_ptr(ref), _ptr(flags), shape, int(grid_x), int(grid_y),
                                              int(stamp), int(khalf), float(max_peak), int(iso),
                                              float(iso_frac), _ptr(centers), _ptr(n_stamps),
                                              _stream(stream)), "argus_select_stamps_noalloc")


def argus_segments_plan(ctx, table, pitch, atlas_h, basis, cfg=None):
    """table: sequence of (row0, col0, side); returns an opaque plan handle."""
    n = len(table)
    arr = (argus_segment * n)(*[argus_segment(int(r), int(c), int(s)) for r, c, s in table])
    h = C.c_void_p()
    _check(load().argus_segments_plan(ctx, arr, n, int(pitch), int(atlas_h), C.byref(basis),
                                      C.byref(cfg) if cfg is not None else None, C.byref(h)),
           "argus_segments_plan")
    return h


def argus_segments_destroy(plan):
    _check(load().argus_segments_destroy(plan), "argus_segments_destroy")


def argus_segments_run(plan, sci, sci_var, ref, ref_var, flags, diff, diff_var, mask, coeffs, stats,
                       nsigma, psf_sigma, out, cap, n_found, use_graph=True, stream=None):
    _check(load().argus_segments_run(plan, _ptr(sci), _ptr(sci_var), _ptr(ref), _ptr(ref_var), _ptr(flags),
                                     _ptr(diff), _ptr(diff_var), _ptr(mask), _ptr(coeffs), _ptr(stats),
                                     float(nsigma), float(psf_sigma), _ptr(out), int(cap), _ptr(n_found),
                                     int(bool(use_graph)), _stream(stream)), "argus_segments_run")


def argus_segments_items(plan):
    a, b = C.c_int(0), C.c_int(0)
    _check(load().argus_segments_items(plan, C.byref(a), C.byref(b)), "argus_segments_items")
    return a.value, b.value


def argus_segments_kernels(plan, K=None, bg=None, stream=None):
    _check(load().argus_segments_kernels(plan, _ptr(K), _ptr(bg), _stream(stream)), "argus_segments_kernels")


def argus_cnn_create(device=0, max_batch=1024, seed=1):
    h = C.c_void_p()
    _check(load().argus_cnn_create(C.byref(h), int(device), int(max_batch), int(seed)), "argus_cnn_create")
    return h


def argus_cnn_destroy(net):
    _check(load().argus_cnn_destroy(net), "argus_cnn_destroy")


def argus_cnn_params(net):
    """(master, adam_m, adam_v) as device addresses, parameter count, Adam step."""
    m, a, v = C.c_void_p(), C.c_void_p(), C.c_void_p()
    n, st = C.c_long(0), C.c_int(0)
    _check(load().argus_cnn_params(net, C.byref(m), C.byref(a), C.byref(v), C.byref(n), C.byref(st)),
           "argus_cnn_params")
    return (m.value, a.value, v.value), n.value, st.value


def argus_cnn_set_state(net, precision, step, stream=None):
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    _check(load().argus_cnn_set_state(net, prec, int(step), _stream(stream)), "argus_cnn_set_state")


def argus_cnn_forward(net, x, n, y, stream=None):
    _check(load().argus_cnn_forward(net, _ptr(x), int(n), _ptr(y), _stream(stream)), "argus_cnn_forward")


def argus_cnn_status(net, stream=None) -> int:
    return load().argus_cnn_status(net, _stream(stream))


def argus_cnn_backward(net, x, dy, n, grad_out=None, stream=None):
    _check(load().argus_cnn_backward(net, _ptr(x), _ptr(dy), int(n), _ptr(grad_out), _stream(stream)),
           "argus_cnn_backward")


def argus_cnn_train_step(net, x, target, n, lr, loss_out=None, stream=None):
    _check(load().argus_cnn_train_step(net, _ptr(x), _ptr(target), int(n), float(lr), _ptr(loss_out),
                                       _stream(stream)), "argus_cnn_train_step")


def argus_cnn_adam(net, grad, lr, stream=None):
    _check(load().argus_cnn_adam(net, _ptr(grad), float(lr), _stream(stream)), "argus_cnn_adam")


def argus_cnn_prepare(sci, ref, shape, centers, n_stamps, max_stamps, x, stream=None):
    _check(load().argus_cnn_prepare(_ptr(sci), _ptr(ref), shape, _ptr(centers), _ptr(n_stamps), int(max_stamps),
                                    _ptr(x), _stream(stream)), "argus_cnn_prepare")


def argus_learned_kernel(ctx, y, centers, n_stamps, max_stamps, frame_w, frame_h, spatial_degree, K,
                         stream=None):
    _check(load().argus_learned_kernel(ctx, _ptr(y), _ptr(centers), _ptr(n_stamps), int(max_stamps),
                                       int(frame_w), int(frame_h), int(spatial_degree), _ptr(K),
                                       _stream(stream)), "argus_learned_kernel")


def argus_fit_background(ctx, sci, sci_var, ref, flags, shape, centers, n_stamps, max_stamps, stamp, K, ksize,
                         spatial_degree, bg_degree, bg, stats, stream=None):
    _check(load().argus_fit_background(ctx, _ptr(sci), _ptr(sci_var), _ptr(ref), _ptr(flags), shape,
                                       _ptr(centers), _ptr(n_stamps), int(max_stamps), int(stamp), _ptr(K),
                                       int(ksize), int(spatial_degree), int(bg_degree), _ptr(bg), _ptr(stats),
                                       _stream(stream)), "argus_fit_background")


def argus_fit_scale_background(ctx, sci, sci_var, ref, flags, shape, centers, n_stamps, max_stamps, stamp, K,
                               ksize, spatial_degree, bg_degree, bg, stats, stream=None):
    _check(load().argus_fit_scale_background(ctx, _ptr(sci), _ptr(sci_var), _ptr(ref), _ptr(flags), shape,
                                             _ptr(centers), _ptr(n_stamps), int(max_stamps), int(stamp), _ptr(K),
                                             int(ksize), int(spatial_degree), int(bg_degree), _ptr(bg), _ptr(stats),
                                             _stream(stream)), "argus_fit_scale_background")


def argus_stamp_basis(ctx, ref, shape, centers, n_stamps, max_stamps, stamp, images, nb, ksize, X, stream=None):
    _check(load().argus_stamp_basis(ctx, _ptr(ref), shape, _ptr(centers), _ptr(n_stamps), int(max_stamps),
                                    int(stamp), _ptr(images), int(nb), int(ksize), _ptr(X), _stream(stream)),
           "argus_stamp_basis")


def argus_fit_kernel(ctx, sci, sci_var, ref, flags, shape, centers, n_stamps, max_stamps, stamp,
                     basis, precision, coeffs, stats, stream=None):
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    _check(load().argus_fit_kernel(ctx, _ptr(sci), _ptr(sci_var), _ptr(ref), _ptr(flags), shape,
                                   _ptr(centers), _ptr(n_stamps), int(max_stamps), int(stamp),
                                   C.byref(basis), prec, _ptr(coeffs), _ptr(stats), _stream(stream)),
           "argus_fit_kernel")


def argus_expand_kernel(ctx, basis, coeffs, K, bg, stream=None):
    _check(load().argus_expand_kernel(ctx, C.byref(basis), _ptr(coeffs), _ptr(K), _ptr(bg),
                                      _stream(stream)), "argus_expand_kernel")


def argus_subtract(ctx, sci, sci_var, ref, ref_var, flags, shape, frame_w, frame_h, ox, oy, ksize,
                   spatial_degree, K, bg_degree, bg, diff, diff_var, stream=None):
    _check(load().argus_subtract(ctx, _ptr(sci), _ptr(sci_var), _ptr(ref), _ptr(ref_var), _ptr(flags),
                                 shape, int(frame_w), int(frame_h), int(ox), int(oy), int(ksize),
                                 int(spatial_degree), _ptr(K), int(bg_degree), _ptr(bg), _ptr(diff),
                                 _ptr(diff_var), _stream(stream)), "argus_subtract")


def argus_detect(ctx, diff, diff_var, flags, shape, nsigma, psf_sigma, mask, out, cap, n_found,
                 stream=None):
    _check(load().argus_detect(ctx, _ptr(diff), _ptr(diff_var), _ptr(flags), shape, float(nsigma),
                               float(psf_sigma), _ptr(mask), _ptr(out), int(cap), _ptr(n_found),
                               _stream(stream)), "argus_detect")


def argus_dia_frame(ctx, raw, shape, calib, ref, ref_var, grid_x, grid_y, stamp, max_peak, iso, iso_frac, basis,
                    precision, nsigma, psf_sigma, img, var, flags, centers, n_stamps, coeffs, stats, K, bg, diff,
                    diff_var, mask, out, cap, n_found, stream=None):
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    _check(load().argus_dia_frame(ctx, _ptr(raw), shape, C.byref(calib), _ptr(ref), _ptr(ref_var), int(grid_x),
                                  int(grid_y), int(stamp), float(max_peak), int(iso), float(iso_frac),
                                  C.byref(basis), prec, float(nsigma), float(psf_sigma), _ptr(img), _ptr(var),
                                  _ptr(flags), _ptr(centers), _ptr(n_stamps), _ptr(coeffs), _ptr(stats), _ptr(K),
                                  _ptr(bg), _ptr(diff), _ptr(diff_var), _ptr(mask), _ptr(out), int(cap),
                                  _ptr(n_found), _stream(stream)), "argus_dia_frame")


def argus_minipix(ctx, img, shape, cell, targets, n_targets, sources, n_sources, sources_cap, keep, out,
                  packed, cell_index, cap, n_kept, stream=None):
    _check(load().argus_minipix(ctx, _ptr(img), shape, int(cell), _ptr(targets), int(n_targets), _ptr(sources),
                                _ptr(n_sources), int(sources_cap), _ptr(keep), _ptr(out), _ptr(packed),
                                _ptr(cell_index), int(cap), _ptr(n_kept), _stream(stream)), "argus_minipix")


def argus_lowres(ctx, img, flags, shape, factor, out, out_pitch, stream=None):
    _check(load().argus_lowres(ctx, _ptr(img), _ptr(flags), shape, int(factor), _ptr(out), int(out_pitch),
                               _stream(stream)), "argus_lowres")


def argus_background(ctx, img, flags, shape, box, filt, min_frac, mesh, map_=None, stream=None):
    _check(load().argus_background(ctx, _ptr(img), _ptr(flags), shape, int(box), int(filt), float(min_frac),
                                   _ptr(mesh), _ptr(map_), _stream(stream)), "argus_background")


ZOGY_TILE_DTYPE = [("x0", "<i4"), ("y0", "<i4"), ("Fn", "<f4"), ("Fr", "<f4"), ("sn", "<f4"), ("sr", "<f4")]


def proper_plan_create(device: int, tile: int, max_tiles: int):
    plan = P()
    _check(load().argus_proper_plan_create(int(device), int(tile), int(max_tiles), C.byref(plan)),
           "argus_proper_plan_create")
    return plan


def proper_plan_destroy(plan):
    _check(load().argus_proper_plan_destroy(plan), "argus_proper_plan_destroy")


def argus_zogy(plan, N, R, shape, tiles, n_tiles, psf_n, psf_r, psf_size, eps, D, S, P_D=None, sigma_S=None,
               stream=None, psf_per_tile=True):
    """tiles: a device uint8 tensor holding n_tiles records of ZOGY_TILE_DTYPE; psf_n and
    psf_r both None reuse the PSF transforms of the plan's last call that gave PSFs;
    psf_per_tile False: one PSF pair shared by every tile."""
    _check(load().argus_zogy(plan, _ptr(N), _ptr(R), shape, _ptr(tiles), int(n_tiles), _ptr(psf_n), _ptr(psf_r),
                             int(psf_size), 1 if psf_per_tile else 0, float(eps), _ptr(D), _ptr(S), _ptr(P_D),
                             _ptr(sigma_S), _stream(stream)), "argus_zogy")


def argus_proper_coadd(plan, stack, n_frames, shape, origins, n_tiles, F, sigma, psfs, psf_size, eps, S, R, P_R=None,
                       F_R=None, sigma_S=None, stream=None, psf_per_tile=True):
    """psf_per_tile False: psfs holds one PSF per frame, shared by every tile."""
    _check(load().argus_proper_coadd(plan, _ptr(stack), int(n_frames), shape, _ptr(origins), int(n_tiles), _ptr(F),
                                     _ptr(sigma), _ptr(psfs), int(psf_size), 1 if psf_per_tile else 0, float(eps),
                                     _ptr(S), _ptr(R), _ptr(P_R), _ptr(F_R), _ptr(sigma_S), _stream(stream)),
           "argus_proper_coadd")


def argus_healpix_resample(frame, flags, shape, wcs, nside_seg, k, segs, n_seg, out, coverage=None, stream=None):
    """wcs: argus_wcs or a tuple (alpha0, delta0, scale, rot, cx, cy)."""
    if not isinstance(wcs, argus_wcs):
        wcs = argus_wcs(*[float(v) for v in wcs])
    _check(load().argus_healpix_resample(_ptr(frame), _ptr(flags), shape, wcs, int(nside_seg), int(k), _ptr(segs),
                                         int(n_seg), _ptr(out), _ptr(coverage), _stream(stream)),
           "argus_healpix_resample")


def argus_segments_subtract(plan, sci, sci_var, ref, ref_var, flags, K, bg, diff, diff_var, stream=None):
    _check(load().argus_segments_subtract(plan, _ptr(sci), _ptr(sci_var), _ptr(ref), _ptr(ref_var), _ptr(flags),
                                          _ptr(K), _ptr(bg), _ptr(diff), _ptr(diff_var), _stream(stream)),
           "argus_segments_subtract")


def sources_from_bytes(buf: torch.Tensor, n: int):
    """Decode n argus_source records from a uint8 tensor (host copy) into a numpy record array."""
    import numpy as np
    dt = np.dtype([("x", "<f4"), ("y", "<f4"), ("flux", "<f4"), ("flux_err", "<f4"),
                   ("peak_snr", "<f4"), ("npix", "<i4"), ("sign", "<i4"), ("px", "<i4"),
                   ("py", "<i4")])
    a = buf.detach().cpu().numpy().view(np.uint8)[: n * SOURCE_BYTES]
    return a.view(dt).copy()


def fit_stats_from_bytes(buf: torch.Tensor) -> dict:
    raw = bytes(buf.detach().cpu().numpy().view("uint8")[:FIT_STATS_BYTES])
    s = argus_fit_stats.from_buffer_copy(raw)
    return {k: getattr(s, k) for k, _ in argus_fit_stats._fields_}
