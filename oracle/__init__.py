"""FP64 CPU oracle of the difference-imaging hot path (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The product library never calls it.  The arithmetic lives in
``argus_oracle.c`` (plain C, FP64, direct loops); this module compiles it with
gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "argus_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

BAD, SAT = 1, 2
MPOS, MNEG, MINV = 1, 2, 4

SOURCE_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("flux", "<f4"), ("flux_err", "<f4"),
                         ("peak_snr", "<f4"), ("npix", "<i4"), ("sign", "<i4"),
                         ("px", "<i4"), ("py", "<i4")])


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, no fast-math)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-std=c11", "-o", _OUT + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_OUT + ".tmp", _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


P = C.c_void_p
I = C.c_int
D = C.c_double
F = C.c_float
L = C.c_long


def _declare(l):
    l.ora_calibrate.argtypes = [I, I, P, P, I, P, P, P, D, D, I, P, P, P, P]
    l.ora_basis_count.argtypes = [I, P]
    l.ora_basis.argtypes = [I, I, P, P, P, P]
    l.ora_nterms.argtypes = [I]
    l.ora_spatial_terms.argtypes = [D, D, I, I, I, P]
    l.ora_ncoeffs.argtypes = [I, I, I]
    l.ora_select_stamps.argtypes = [I, I, P, P, I, I, I, I, F, I, F, P]
    l.ora_cholesky.argtypes = [I, P, P]
    l.ora_cholesky_solve.argtypes = [I, P, P, P]
    l.ora_stamp_basis.argtypes = [I, I, P, P, I, I, P, I, I, P]
    l.ora_stamp_basis.restype = None
    l.ora_fit.argtypes = [I, I, P, P, P, P, P, I, I, I, I, P, P, I, I, P, P, P, P, P]
    l.ora_expand.argtypes = [I, I, P, P, I, I, P, P, P]
    l.ora_fit_rect.argtypes = [I, I, P, P, P, P, I, I, I, I, I, I, P, P, I, I, P, P, P, P, P]
    l.ora_subtract.argtypes = [I, I, I, I, I, I, P, P, P, P, P, I, I, P, I, P, P, P]
    l.ora_subtract_at.argtypes = [I, I, I, I, I, I, P, P, P, P, P, I, I, P, I, P, I, P, P, P]
    l.ora_detect.argtypes = [I, I, P, P, P, F, D, P, P, I]
    l.ora_coadd.argtypes = [I, I, I, P, P, I, P, P, P, D, D, I, D, I, P, P, P, P]
    l.ora_cnn_nparams.restype = L
    l.ora_cnn_forward.argtypes = [I, P, P, P, P]
    l.ora_cnn_forward.restype = None
    l.ora_cnn_backward.argtypes = [I, P, P, P, P, P]
    l.ora_cnn_backward.restype = None
    l.ora_cnn_mse.argtypes = [L, P, P, P]
    l.ora_cnn_mse.restype = D
    l.ora_adam.argtypes = [L, P, P, P, P, D, D, D, D, I]
    l.ora_adam.restype = None
    l.ora_num_threads.restype = I
    l.ora_set_threads.argtypes = [I]
    l.ora_minipix.argtypes = [I, I, P, I, P, I, P, P]
    l.ora_minipix.restype = I
    l.ora_lowres.argtypes = [I, I, P, P, I, P]


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle inputs must be C-contiguous"
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return lib().ora_num_threads()


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


# --------------------------------------------------------------------------- #
def calibrate(raw, *, bias=100, bias_frame=None, dark=None, flat=None, bpm=None,
              gain=1.0, read_noise=1.7, sat=65535):
    """Returns (I f64, V f64, flags u8, n i32) for a [h, w] uint16 frame."""
    raw = _c(raw, np.uint16)
    h, w = raw.shape
    img = np.empty((h, w)); var = np.empty((h, w))
    fl = np.empty((h, w), np.uint8); n = np.empty((h, w), np.int32)
    lib().ora_calibrate(w, h, _p(raw), _p(_c(bias_frame, np.uint16)), int(bias),
                        _p(_c(dark, np.float32)), _p(_c(flat, np.float32)),
                        _p(_c(bpm, np.uint8)), float(gain), float(read_noise), int(sat),
                        _p(img), _p(var), _p(fl), _p(n))
    return img, var, fl, n


class Basis:
    """Alard-Lupton basis specification (kernel size, Gaussian widths, degrees)."""

    def __init__(self, ksize=11, sigmas=(0.7, 1.5, 3.0), degrees=(6, 4, 2), spatial_degree=0,
                 bg_degree=0):
        self.ksize = int(ksize)
        self.sigmas = np.ascontiguousarray(sigmas, dtype=np.float64)
        self.degrees = np.ascontiguousarray(degrees, dtype=np.int32)
        self.spatial_degree = int(spatial_degree)
        self.bg_degree = int(bg_degree)

    @property
    def ngauss(self):
        return int(self.sigmas.size)

    @property
    def nb(self):
        return lib().ora_basis_count(self.ngauss, _p(self.degrees))

    @property
    def ncoeffs(self):
        return lib().ora_ncoeffs(self.nb, self.spatial_degree, self.bg_degree)

    @property
    def nterms(self):
        return lib().ora_nterms(self.spatial_degree)

    @property
    def nbg(self):
        return lib().ora_nterms(self.bg_degree)


def basis(b: Basis):
    """Returns (B [nb, ks, ks] f64, gpq [nb, 3] int)."""
    nb = b.nb
    B = np.empty((nb, b.ksize, b.ksize))
    pq = np.empty((nb, 3), np.int32)
    lib().ora_basis(b.ksize, b.ngauss, _p(b.sigmas), _p(b.degrees), _p(B), _p(pq))
    return B, pq


def spatial_terms(x, y, W, H, deg):
    out = np.empty(max(lib().ora_nterms(deg), 1))
    lib().ora_spatial_terms(float(x), float(y), int(W), int(H), int(deg), _p(out))
    return out[: lib().ora_nterms(deg)]


def cholesky(M):
    M = _c(M, np.float64)
    n = M.shape[0]
    Lm = np.empty_like(M)
    st = lib().ora_cholesky(n, _p(M), _p(Lm))
    return st, Lm


def cholesky_solve(Lm, b):
    Lm = _c(Lm, np.float64); b = _c(b, np.float64)
    x = np.empty_like(b)
    lib().ora_cholesky_solve(Lm.shape[0], _p(Lm), _p(b), _p(x))
    return x


def select_stamps(R, flags, gx, gy, stamp, khalf, max_peak, iso=10, iso_frac=0.1):
    R = _c(R, np.float32); flags = _c(flags, np.uint8)
    h, w = R.shape
    cen = np.empty((gx * gy, 2), np.int32)
    n = lib().ora_select_stamps(w, h, _p(R), _p(flags), gx, gy, stamp, khalf,
                                float(max_peak), int(iso), float(iso_frac), _p(cen))
    return cen[:n].copy()


def stamp_conv(R, centers, stamp, images):
    """The basis convolution of ora_stamp_basis with given images [nb][ks*ks]
    (FP64 sums): X [n_stamps][stamp^2][nb], zero for stamps whose window
    leaves the frame."""
    R = _c(R, np.float32); cen = _c(centers, np.int32)
    img = _c(images, np.float64)
    nb, kk = img.shape
    ks = int(round(kk ** 0.5))
    h, w = R.shape
    X = np.empty((cen.shape[0], stamp * stamp, nb))
    lib().ora_stamp_basis(w, h, _p(R), _p(cen), cen.shape[0], stamp, _p(img), nb, ks, _p(X))
    return X


def stamp_basis(R, centers, stamp, b: Basis):
    R = _c(R, np.float32); cen = _c(centers, np.int32)
    h, w = R.shape
    B, _ = basis(b)
    X = np.empty((cen.shape[0], stamp * stamp, b.nb))
    lib().ora_stamp_basis(w, h, _p(R), _p(cen), cen.shape[0], stamp, _p(B), b.nb, b.ksize, _p(X))
    return X


class FitResult:
    def __init__(self, status, coeffs, M, b, chi2, dof):
        self.status, self.coeffs, self.M, self.b, self.chi2, self.dof = status, coeffs, M, b, chi2, dof


def fit(sci, sci_var, ref, flags, centers, stamp, b: Basis) -> FitResult:
    sci = _c(sci, np.float32); sv = _c(sci_var, np.float32); R = _c(ref, np.float32)
    fl = _c(flags, np.uint8); cen = _c(centers, np.int32)
    h, w = sci.shape
    Nc = b.ncoeffs
    a = np.zeros(Nc); M = np.empty((Nc, Nc)); bv = np.empty(Nc)
    chi2 = C.c_double(0.0); dof = C.c_long(0)
    st = lib().ora_fit(w, h, _p(sci), _p(sv), _p(R), _p(fl), _p(cen), cen.shape[0], stamp,
                       b.ksize, b.ngauss, _p(b.sigmas), _p(b.degrees), b.spatial_degree,
                       b.bg_degree, _p(a), _p(M), _p(bv), C.byref(chi2), C.byref(dof))
    return FitResult(st, a, M, bv, chi2.value, dof.value)


def fit_rect(sci, sci_var, ref, flags, rect, b: Basis) -> FitResult:
    """Least-squares kernel fit over every pixel of rect = (x0, y0, x1, y1) (inclusive)."""
    sci = _c(sci, np.float32); sv = _c(sci_var, np.float32); R = _c(ref, np.float32)
    fl = _c(flags, np.uint8)
    h, w = sci.shape
    Nc = b.ncoeffs
    a = np.zeros(Nc); M = np.empty((Nc, Nc)); bv = np.empty(Nc)
    chi2 = C.c_double(0.0); dof = C.c_long(0)
    x0, y0, x1, y1 = (int(v) for v in rect)
    st = lib().ora_fit_rect(w, h, _p(sci), _p(sv), _p(R), _p(fl), x0, y0, x1, y1, b.ksize, b.ngauss,
                            _p(b.sigmas), _p(b.degrees), b.spatial_degree, b.bg_degree, _p(a), _p(M),
                            _p(bv), C.byref(chi2), C.byref(dof))
    return FitResult(st, a, M, bv, chi2.value, dof.value)


def expand(b: Basis, coeffs):
    """Returns (K [Ks, ks, ks] f64, bg [Kb] f64)."""
    a = _c(coeffs, np.float64)
    K = np.empty((b.nterms, b.ksize, b.ksize)); bg = np.empty(max(b.nbg, 1))
    lib().ora_expand(b.ksize, b.ngauss, _p(b.sigmas), _p(b.degrees), b.spatial_degree,
                     b.bg_degree, _p(a), _p(K), _p(bg))
    return K, bg[: b.nbg]


def subtract(sci, sci_var, ref, ref_var, flags, K, bg, *, sdeg, bgdeg, frame=None, origin=(0, 0),
             with_var=True):
    """Full-image D (and V_D = V_I + sum K_xy^2 V_ref with the kernel K_xy at each pixel).
    K [Ks, ks, ks], bg [Kb]; frame = (W, H) for spatial terms."""
    sci = _c(sci, np.float32); sv = _c(sci_var, np.float32); R = _c(ref, np.float32)
    Rv = _c(ref_var, np.float32); fl = _c(flags, np.uint8)
    K = _c(K, np.float64); bg = _c(np.atleast_1d(bg), np.float64)
    h, w = sci.shape
    W, H = frame if frame is not None else (w, h)
    Dd = np.empty((h, w)); Vd = np.empty((h, w)) if with_var else None
    lib().ora_subtract(w, h, W, H, origin[0], origin[1], _p(sci), _p(sv), _p(R), _p(Rv), _p(fl),
                       K.shape[-1], sdeg, _p(K), bgdeg, _p(bg), _p(Dd), _p(Vd))
    return Dd, Vd


def subtract_at(xy, sci, sci_var, ref, ref_var, flags, K, bg, *, sdeg, bgdeg, frame=None,
                origin=(0, 0)):
    sci = _c(sci, np.float32); sv = _c(sci_var, np.float32); R = _c(ref, np.float32)
    Rv = _c(ref_var, np.float32); fl = _c(flags, np.uint8)
    K = _c(K, np.float64); bg = _c(np.atleast_1d(bg), np.float64); xy = _c(xy, np.int32)
    h, w = sci.shape
    W, H = frame if frame is not None else (w, h)
    n = xy.shape[0]
    Dd = np.empty(n); Vd = np.empty(n)
    lib().ora_subtract_at(w, h, W, H, origin[0], origin[1], _p(sci), _p(sv), _p(R), _p(Rv),
                          _p(fl), K.shape[-1], sdeg, _p(K), bgdeg, _p(bg), n, _p(xy),
                          _p(Dd), _p(Vd))
    return Dd, Vd


def detect(D, VD, flags, nsigma=5.0, psf_sigma=1.8, cap=1 << 20):
    """Returns (mask u8, sources structured array, total count)."""
    Dd = _c(D, np.float32); Vd = _c(VD, np.float32); fl = _c(flags, np.uint8)
    h, w = Dd.shape
    mask = np.empty((h, w), np.uint8)
    out = np.zeros(cap, SOURCE_DTYPE)
    n = lib().ora_detect(w, h, _p(Dd), _p(Vd), _p(fl), float(nsigma), float(psf_sigma), _p(mask),
                         _p(out), cap)
    return mask, out[: min(n, cap)].copy(), n


def coadd(raw_stack, shifts, *, bias=100, dark=None, flat=None, bpm=None, gain=1.0,
          read_noise=1.7, sat=65535, kappa=3.0, max_iter=5):
    """Returns (coadd f64, var f64, n_used u8, margin f64)."""
    rs = _c(raw_stack, np.uint16); sh = _c(shifts, np.float32)
    nf, h, w = rs.shape
    co = np.empty((h, w)); va = np.empty((h, w)); nu = np.empty((h, w), np.uint8)
    mg = np.empty((h, w))
    lib().ora_coadd(nf, w, h, _p(rs), _p(sh), int(bias), _p(_c(dark, np.float32)),
                    _p(_c(flat, np.float32)), _p(_c(bpm, np.uint8)), float(gain),
                    float(read_noise), int(sat), float(kappa), int(max_iter), _p(co), _p(va),
                    _p(nu), _p(mg))
    return co, va, nu, mg


# --------------------------------------------------------------------------- learned surrogate
CNN_S, CNN_C = 21, 32


def cnn_nparams() -> int:
    return int(lib().ora_cnn_nparams())


def cnn_forward(params, x):
    """params [P] f64, x [B, 441, 2] -> (y [B, 441], acts [5, B, 441, 32])."""
    prm = _c(params, np.float64); x = _c(x, np.float64)
    B = x.shape[0]
    acts = np.empty((5, B, CNN_S * CNN_S, CNN_C)); y = np.empty((B, CNN_S * CNN_S))
    lib().ora_cnn_forward(B, _p(prm), _p(x), _p(acts), _p(y))
    return y, acts


def cnn_backward(params, x, acts, dy):
    prm = _c(params, np.float64); x = _c(x, np.float64); acts = _c(acts, np.float64); dy = _c(dy, np.float64)
    g = np.empty(cnn_nparams())
    lib().ora_cnn_backward(x.shape[0], _p(prm), _p(x), _p(acts), _p(dy), _p(g))
    return g


def cnn_mse(y, t):
    y = _c(y, np.float64); t = _c(t, np.float64)
    dy = np.empty_like(y)
    loss = lib().ora_cnn_mse(y.size, _p(y), _p(t), _p(dy))
    return loss, dy


def adam(p, m, v, g, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, step=1):
    """In-place Adam step on float64 arrays p, m, v."""
    g = _c(g, np.float64)
    lib().ora_adam(p.size, _p(p), _p(m), _p(v), _p(g), float(lr), float(b1), float(b2), float(eps), int(step))


def minipix(img, cell, targets):
    """Sparse stamping: (out f32 [h][w], keep u8 [ceil(h/cell)][ceil(w/cell)], kept cells)."""
    img = _c(img, np.float32)
    h, w = img.shape
    t = _c(np.asarray(targets, np.int32).reshape(-1, 2), np.int32)
    out = np.empty((h, w), np.float32)
    keep = np.empty(((h + cell - 1) // cell, (w + cell - 1) // cell), np.uint8)
    n = lib().ora_minipix(w, h, _p(img), int(cell), _p(t), t.shape[0], _p(out), _p(keep))
    return out, keep, n


def lowres(img, flags, f):
    """Block mean of the valid pixels, FP64 [ceil(h/f)][ceil(w/f)]."""
    img = _c(img, np.float32)
    h, w = img.shape
    fl = None if flags is None else _c(flags, np.uint8)
    out = np.empty(((h + f - 1) // f, (w + f - 1) // f))
    lib().ora_lowres(w, h, _p(img), None if fl is None else _p(fl), int(f), _p(out))
    return out
