"""Python binding of libsfft (``include/sfft.h``): argument marshalling only.

Every function here has the name of the C entry point it wraps and passes device pointers
(``torch.Tensor.data_ptr()`` or plain integers) straight through; all arithmetic runs in
the CUDA kernels of ``libsfft.so``.  If the library has not been built this module raises
``SfftError`` on first use -- there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsfft.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_SPD, ERR_NO_CONVERGENCE, ERR_TIMEOUT, ERR_UNSUPPORTED = range(8)
F32, F64 = 0, 1
PREC_FP32, PREC_SPLIT, PREC_FP64 = 0, 1, 2
SOLVE_CHOLESKY, SOLVE_PCG = 0, 1

EXPORTED = ("sfft_plan", "sfft_destroy", "sfft_n_unknowns", "sfft_workspace_size", "sfft_set_stream",
            "sfft_normal", "sfft_fit", "sfft_subtract", "sfft_sync_status", "sfft_batch",
            "sfft_batch_create", "sfft_batch_run", "sfft_batch_info", "sfft_batch_destroy",
            "sfft_tuning_get", "sfft_tuning_set", "sfft_autotune", "sfft_tuning_save", "sfft_tuning_load",
            "sfft_profile", "sfft_stage_times", "sfft_launch_count", "sfft_subtract_noalloc",
            "sfft_cross_convolve", "sfft_resample", "sfft_align_psf", "sfft_decorrelation_kernel",
            "sfft_forced_photometry",
            "sfft_status_string", "sfft_last_error",
            "sfft_cnn_create", "sfft_cnn_destroy", "sfft_cnn_param_count", "sfft_cnn_set_params",
            "sfft_cnn_get_params", "sfft_cnn_forward", "sfft_cnn_gradients", "sfft_cnn_train_step",
            "sfft_cnn_train", "sfft_cnn_warm_start", "sfft_cnn_save", "sfft_cnn_load", "sfft_cnn_last_error",
            "sfft_cnn_set_stream")
NSTAGES = 8
STAGES = ("segment_fft", "moments", "ycorr", "lag_tables", "assemble", "solve", "subtract", "refine")


class SfftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class sfft_desc(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("nx", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("L", ctypes.c_int32), ("dk", ctypes.c_int32), ("db", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("precision", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("workspace_cap", ctypes.c_size_t),
                ("seg", ctypes.c_int32), ("refine", ctypes.c_int32), ("spin_limit", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class sfft_fit_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("fallback", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("start_residual", ctypes.c_double), ("pcg_status", ctypes.c_int32),
                ("reserved_i", ctypes.c_int32), ("reserved", ctypes.c_double * 1)]


class sfft_pair(ctypes.Structure):
    _fields_ = [("sci", ctypes.c_void_p), ("tmpl", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("x0", ctypes.c_void_p), ("coeffs", ctypes.c_void_p), ("diff", ctypes.c_void_p),
                ("ny", ctypes.c_int32), ("nx", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("psf_stamps", ctypes.c_void_p),
                ("sci_host", ctypes.c_void_p), ("tmpl_host", ctypes.c_void_p), ("mask_host", ctypes.c_void_p),
                ("coeffs_host", ctypes.c_void_p), ("diff_host", ctypes.c_void_p)]


class sfft_tuning(ctypes.Structure):
    _fields_ = [("ycorr_bins", ctypes.c_int32), ("ycorr_split", ctypes.c_int32),
                ("ycorr_scalar", ctypes.c_int32), ("subtract_ctas", ctypes.c_int32),
                ("pcg_cluster", ctypes.c_int32), ("ycorr_direct", ctypes.c_int32),
                ("ycorr_sets", ctypes.c_int32), ("subtract_fft", ctypes.c_int32)]


class sfft_warp(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("reserved", ctypes.c_int32), ("x_ref", ctypes.c_double),
                ("y_ref", ctypes.c_double), ("cu", ctypes.c_double * 10), ("cv", ctypes.c_double * 10)]


class sfft_phot_job(ctypes.Structure):
    _fields_ = [("image", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("psf", ctypes.c_void_p), ("x", ctypes.c_double), ("y", ctypes.c_double),
                ("ny", ctypes.c_int32), ("nx", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("dtype", ctypes.c_int32)]


BATCH_GRAPH, BATCH_AUTOTUNE = 1, 2
LANCZOS3, BILINEAR = 0, 1
RESAMPLE_FLUX, RESAMPLE_ZERO_OUTSIDE = 1, 2
PHOT_BACKGROUND = 1

_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libsfft.so (built by ``paper_2509_18544_gb300.build``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise SfftError(ERR_UNSUPPORTED, "libsfft.so not built at %s (run __graft_entry__.build())" % path)
        lib = ctypes.CDLL(path)
        P, I32 = ctypes.c_void_p, ctypes.c_int32
        lib.sfft_plan.argtypes = [ctypes.POINTER(P), ctypes.POINTER(sfft_desc), P]
        lib.sfft_destroy.argtypes = [P]
        lib.sfft_destroy.restype = None
        lib.sfft_n_unknowns.argtypes = [P, ctypes.POINTER(I32)]
        lib.sfft_workspace_size.argtypes = [ctypes.POINTER(sfft_desc), ctypes.POINTER(ctypes.c_size_t)]
        lib.sfft_set_stream.argtypes = [P, P]
        lib.sfft_normal.argtypes = [P, P, P, P, P, P]
        lib.sfft_fit.argtypes = [P, P, P, P, P, P, ctypes.POINTER(sfft_fit_info)]
        lib.sfft_subtract.argtypes = [P, P, P, P, P]
        lib.sfft_sync_status.argtypes = [P]
        lib.sfft_batch.argtypes = [ctypes.POINTER(sfft_desc), I32, I32, ctypes.POINTER(sfft_pair), P,
                                   ctypes.POINTER(sfft_fit_info), P]
        lib.sfft_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(sfft_desc), ctypes.POINTER(sfft_pair),
                                          I32, I32, I32, P, P]
        lib.sfft_batch_run.argtypes = [P]
        lib.sfft_batch_info.argtypes = [P, ctypes.POINTER(sfft_fit_info)]
        lib.sfft_batch_destroy.argtypes = [P]
        lib.sfft_batch_destroy.restype = None
        lib.sfft_tuning_get.argtypes = [ctypes.POINTER(sfft_desc), ctypes.POINTER(sfft_tuning), ctypes.POINTER(I32)]
        lib.sfft_tuning_set.argtypes = [ctypes.POINTER(sfft_desc), ctypes.POINTER(sfft_tuning)]
        lib.sfft_autotune.argtypes = [ctypes.POINTER(sfft_desc), P, P, P, I32, ctypes.POINTER(sfft_tuning),
                                      ctypes.POINTER(ctypes.c_double)]
        lib.sfft_tuning_save.argtypes = [ctypes.c_char_p]
        lib.sfft_tuning_load.argtypes = [ctypes.c_char_p]
        lib.sfft_subtract_noalloc.argtypes = [ctypes.POINTER(sfft_desc), P, P, P, P, P]
        lib.sfft_cross_convolve.argtypes = [I32, I32, I32, I32, I32, P, P, P, P, P, P, P]
        D = ctypes.c_double
        lib.sfft_resample.argtypes = [ctypes.POINTER(sfft_warp), I32, I32, I32, I32, I32, I32, P, P, I32, I32, I32,
                                      P, P, P]
        lib.sfft_align_psf.argtypes = [ctypes.POINTER(sfft_warp), D, D, I32, P, P, P]
        lib.sfft_decorrelation_kernel.argtypes = [I32, I32, I32, I32, P, D, D, I32, P, P, D, D, I32, P, P, P]
        lib.sfft_forced_photometry.argtypes = [I32, P, I32, I32, P, P]
        lib.sfft_profile.argtypes = [P, I32]
        lib.sfft_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I32)]
        lib.sfft_launch_count.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        lib.sfft_status_string.argtypes = [I32]
        lib.sfft_status_string.restype = ctypes.c_char_p
        lib.sfft_last_error.argtypes = [P]
        lib.sfft_last_error.restype = ctypes.c_char_p
        lib.sfft_cnn_create.argtypes = [ctypes.POINTER(P), I32, I32, P]
        lib.sfft_cnn_destroy.argtypes = [P]
        lib.sfft_cnn_destroy.restype = None
        lib.sfft_cnn_param_count.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        lib.sfft_cnn_set_params.argtypes = [P, P]
        lib.sfft_cnn_get_params.argtypes = [P, P]
        lib.sfft_cnn_forward.argtypes = [P, P, I32, P]
        lib.sfft_cnn_gradients.argtypes = [P, P, P, I32, P, P, P]
        lib.sfft_cnn_train_step.argtypes = [P, P, P, I32, ctypes.c_float, P]
        lib.sfft_cnn_train.argtypes = [P, P, P, I32, I32, I32, ctypes.c_float, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_float)]
        lib.sfft_cnn_warm_start.argtypes = [P, P, I32, I32, P]
        lib.sfft_cnn_save.argtypes = [P, ctypes.c_char_p]
        lib.sfft_cnn_set_stream.argtypes = [P, P]
        lib.sfft_cnn_load.argtypes = [P, ctypes.c_char_p]
        lib.sfft_cnn_last_error.argtypes = [P]
        lib.sfft_cnn_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("sfft_destroy", "sfft_status_string", "sfft_last_error", "sfft_cnn_destroy",
                            "sfft_cnn_last_error", "sfft_batch_destroy"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _check(rc, handle=None):
    if rc != OK:
        lib = load_library()
        msg = lib.sfft_last_error(handle).decode(errors="replace") or lib.sfft_status_string(rc).decode()
        raise SfftError(rc, msg)


class Plan:
    """Owns one ``sfft_plan_t``; created by :func:`sfft_plan`."""

    def __init__(self, handle, desc):
        self.handle = handle
        self.desc = desc

    @property
    def n(self) -> int:
        return sfft_n_unknowns(self)

    def close(self):
        if self.handle:
            load_library().sfft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def make_desc(ny, nx, L, dk, db, dtype=F32, precision=PREC_SPLIT, solver=SOLVE_CHOLESKY, pitch=0,
              max_iter=0, tol=0.0, workspace_cap=0, seg=0, refine=0, spin_limit=0) -> sfft_desc:
    d = sfft_desc()
    d.ny, d.nx, d.pitch, d.L, d.dk, d.db = ny, nx, pitch, L, dk, db
    d.dtype, d.precision, d.solver = dtype, precision, solver
    d.max_iter, d.tol, d.workspace_cap, d.seg, d.refine = max_iter, tol, workspace_cap, seg, refine
    d.spin_limit = spin_limit
    return d


def sfft_plan(desc: sfft_desc, stream=None) -> Plan:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.sfft_plan(ctypes.byref(h), ctypes.byref(desc), _stream(stream)))
    return Plan(h.value, desc)


def sfft_destroy(plan: Plan):
    plan.close()


def sfft_n_unknowns(plan: Plan) -> int:
    n = ctypes.c_int32()
    _check(load_library().sfft_n_unknowns(plan.handle, ctypes.byref(n)), plan.handle)
    return n.value


def sfft_workspace_size(desc: sfft_desc) -> int:
    v = ctypes.c_size_t()
    _check(load_library().sfft_workspace_size(ctypes.byref(desc), ctypes.byref(v)))
    return v.value


def sfft_set_stream(plan: Plan, stream):
    _check(load_library().sfft_set_stream(plan.handle, _stream(stream)), plan.handle)


def sfft_normal(plan: Plan, sci, tmpl, mask, N, b):
    _check(load_library().sfft_normal(plan.handle, _ptr(sci), _ptr(tmpl), _ptr(mask), _ptr(N), _ptr(b)),
           plan.handle)


def sfft_fit(plan: Plan, sci, tmpl, mask, x0, coeffs, want_info: bool = True):
    """Queue the fit; with ``want_info`` synchronise and return the sfft_fit_info (raises on
    a device-side failure such as a non-positive-definite normal matrix)."""
    info = sfft_fit_info() if want_info else None
    rc = load_library().sfft_fit(plan.handle, _ptr(sci), _ptr(tmpl), _ptr(mask), _ptr(x0), _ptr(coeffs),
                                 ctypes.byref(info) if info is not None else None)
    _check(rc, plan.handle)
    return info


def sfft_subtract(plan: Plan, sci, tmpl, coeffs, diff):
    _check(load_library().sfft_subtract(plan.handle, _ptr(sci), _ptr(tmpl), _ptr(coeffs), _ptr(diff)),
           plan.handle)


def sfft_sync_status(plan: Plan):
    _check(load_library().sfft_sync_status(plan.handle), plan.handle)


def make_pair(sci, tmpl, mask, coeffs, diff, ny, nx, pitch=0, x0=None, host=None, stamps=None) -> sfft_pair:
    """host: optional dict of pinned host tensors (sci, tmpl, mask, coeffs, diff) that a run
    copies in before the fit and out after the subtraction; stamps: the pair's 18 x 32 x 32
    float PSF stamps on the device (read when the batch has a warm-start network)."""
    q = sfft_pair()
    q.sci, q.tmpl, q.mask, q.x0 = _ptr(sci), _ptr(tmpl), _ptr(mask), _ptr(x0)
    q.psf_stamps = _ptr(stamps)
    q.coeffs, q.diff = _ptr(coeffs), _ptr(diff)
    q.ny, q.nx, q.pitch = ny, nx, pitch
    if host:
        q.sci_host, q.tmpl_host = _ptr(host.get("sci")), _ptr(host.get("tmpl"))
        q.mask_host, q.coeffs_host, q.diff_host = _ptr(host.get("mask")), _ptr(host.get("coeffs")), _ptr(host.get("diff"))
    return q


def _pairs(pairs):
    return (sfft_pair * len(pairs))(*pairs)


def sfft_batch(desc: sfft_desc, n_sci: int, n_tmpl: int, pairs, want_info=True, stream=None, cnn=None):
    """One-shot run of all S x T pairs (science-major list of sfft_pair); returns the infos."""
    infos = (sfft_fit_info * len(pairs))() if want_info else None
    _check(load_library().sfft_batch(ctypes.byref(desc), n_sci, n_tmpl, _pairs(pairs),
                                     cnn.handle if cnn is not None else None, infos, _stream(stream)))
    return list(infos) if infos is not None else None


class Batch:
    """Owns one ``sfft_batch_t``; created by :func:`sfft_batch_create`."""

    def __init__(self, handle, npairs):
        self.handle, self.npairs = handle, npairs

    def close(self):
        if self.handle:
            load_library().sfft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def sfft_batch_create(desc: sfft_desc, pairs, lanes: int = 0, flags: int = 0, stream=None, cnn=None) -> Batch:
    """cnn: a warm-start network (Cnn) evaluated on the pairs' stamps at every run."""
    h = ctypes.c_void_p()
    _check(load_library().sfft_batch_create(ctypes.byref(h), ctypes.byref(desc), _pairs(pairs), len(pairs), lanes,
                                            flags, cnn.handle if cnn is not None else None, _stream(stream)))
    return Batch(h.value, len(pairs))


def sfft_batch_run(batch: Batch):
    _check(load_library().sfft_batch_run(batch.handle))


def sfft_batch_info(batch: Batch, raise_on_error: bool = False):
    infos = (sfft_fit_info * batch.npairs)()
    rc = load_library().sfft_batch_info(batch.handle, infos)
    if raise_on_error or rc not in (OK, ERR_NOT_SPD):
        _check(rc)
    return list(infos)


def sfft_batch_destroy(batch: Batch):
    batch.close()


def sfft_tuning_get(desc: sfft_desc):
    t = sfft_tuning()
    cached = ctypes.c_int32()
    _check(load_library().sfft_tuning_get(ctypes.byref(desc), ctypes.byref(t), ctypes.byref(cached)))
    return t, bool(cached.value)


def sfft_tuning_set(desc: sfft_desc, t: sfft_tuning):
    _check(load_library().sfft_tuning_set(ctypes.byref(desc), ctypes.byref(t)))


def sfft_autotune(desc: sfft_desc, sci, tmpl, mask, trials: int = 3):
    t = sfft_tuning()
    ms = ctypes.c_double()
    _check(load_library().sfft_autotune(ctypes.byref(desc), _ptr(sci), _ptr(tmpl), _ptr(mask), trials,
                                        ctypes.byref(t), ctypes.byref(ms)))
    return t, ms.value


def sfft_tuning_save(path: str):
    _check(load_library().sfft_tuning_save(path.encode()))


def sfft_tuning_load(path: str):
    _check(load_library().sfft_tuning_load(path.encode()))


def sfft_profile(plan: Plan, enable: bool = True):
    _check(load_library().sfft_profile(plan.handle, 1 if enable else 0), plan.handle)


def sfft_stage_times(plan: Plan):
    """Synchronise; return ({stage: ms summed since the last read}, number of timed calls)."""
    ms = (ctypes.c_double * NSTAGES)()
    calls = ctypes.c_int32()
    _check(load_library().sfft_stage_times(plan.handle, ms, ctypes.byref(calls)), plan.handle)
    return dict(zip(STAGES, list(ms))), calls.value


def sfft_launch_count() -> int:
    v = ctypes.c_uint64()
    _check(load_library().sfft_launch_count(ctypes.byref(v)))
    return v.value


def sfft_cross_convolve(ny: int, nx: int, K: int, sci, tmpl, psf_sci, psf_tmpl, sci_out, tmpl_out, dtype: int = F32,
                        pitch: int = 0, stream=None):
    """sci_out = sci (x) psf_tmpl and tmpl_out = tmpl (x) psf_sci: cyclic convolutions with
    K x K float32 stamps (device); a half whose image, stamp or output is None is skipped."""
    _check(load_library().sfft_cross_convolve(ny, nx, pitch, dtype, K, _ptr(sci), _ptr(tmpl), _ptr(psf_sci),
                                              _ptr(psf_tmpl), _ptr(sci_out), _ptr(tmpl_out), _stream(stream)))


def make_warp(degree: int, cu, cv, x_ref: float = 0.0, y_ref: float = 0.0) -> sfft_warp:
    """Coordinate polynomials u(x, y), v(x, y) about (x_ref, y_ref) (monomial order of sfft.h)."""
    w = sfft_warp()
    w.degree, w.x_ref, w.y_ref = degree, x_ref, y_ref
    for k in range(10):
        w.cu[k] = float(cu[k]) if k < len(cu) else 0.0
        w.cv[k] = float(cv[k]) if k < len(cv) else 0.0
    return w


def sfft_resample(warp: sfft_warp, src, out, src_mask=None, out_mask=None, method: int = LANCZOS3, flags: int = 0,
                  dtype: int = F32, in_shape=None, out_shape=None, in_pitch: int = 0, out_pitch: int = 0,
                  stream=None):
    """Resample the template (device) onto the science grid; shapes default to the tensors'."""
    iny, inx = in_shape if in_shape is not None else tuple(src.shape)
    ony, onx = out_shape if out_shape is not None else tuple(out.shape)
    _check(load_library().sfft_resample(ctypes.byref(warp), method, flags, iny, inx, in_pitch, dtype, _ptr(src),
                                        _ptr(src_mask), ony, onx, out_pitch, _ptr(out), _ptr(out_mask),
                                        _stream(stream)))


def sfft_align_psf(warp: sfft_warp, x: float, y: float, psf_in, psf_out, stream=None):
    """The template PSF stamp (device, K x K float32) aligned to the science grid at (x, y)."""
    _check(load_library().sfft_align_psf(ctypes.byref(warp), x, y, psf_in.shape[0], _ptr(psf_in), _ptr(psf_out),
                                         _stream(stream)))


def sfft_decorrelation_kernel(ny: int, nx: int, L: int, dk: int, coeffs, x: float, y: float, psf_sci, psf_tmpl,
                              sigma_sci: float, sigma_tmpl: float, phi, psf_out=None, stream=None):
    """Decorrelation kernel phi (device M x M float32; M = phi.shape[0]) at pixel (x, y) and,
    optionally, the decorrelated science PSF."""
    _check(load_library().sfft_decorrelation_kernel(ny, nx, L, dk, _ptr(coeffs), x, y, psf_sci.shape[0],
                                                    _ptr(psf_sci), _ptr(psf_tmpl), sigma_sci, sigma_tmpl,
                                                    phi.shape[0], _ptr(phi), _ptr(psf_out), _stream(stream)))


def phot_jobs(jobs) -> "ctypes.Array":
    """Host array of sfft_phot_job from dicts (image, psf, x, y, [weight, mask, ny, nx, pitch, dtype])."""
    arr = (sfft_phot_job * len(jobs))()
    for a, j in zip(arr, jobs):
        img = j["image"]
        a.image, a.psf = _ptr(img), _ptr(j["psf"])
        a.weight, a.mask = _ptr(j.get("weight")), _ptr(j.get("mask"))
        a.x, a.y = float(j["x"]), float(j["y"])
        a.ny = j.get("ny", img.shape[0] if hasattr(img, "shape") else 0)
        a.nx = j.get("nx", img.shape[1] if hasattr(img, "shape") else 0)
        a.pitch = j.get("pitch", 0)
        a.dtype = j.get("dtype", F64 if getattr(img, "dtype", None) is not None and "64" in str(img.dtype) else F32)
    return arr


def sfft_forced_photometry(jobs_dev, njobs: int, K: int, results, flags: int = 0, stream=None):
    """PSF fluxes of njobs jobs; jobs_dev: device copy of a :func:`phot_jobs` array; results:
    device float64 (njobs, 8)."""
    _check(load_library().sfft_forced_photometry(njobs, _ptr(jobs_dev), K, flags, _ptr(results),
                                                 _stream(stream)))


def sfft_subtract_noalloc(desc: sfft_desc, sci, tmpl, coeffs, diff, stream=None):
    """Plan-free difference image whose scratch is a fixed device array (no allocation)."""
    _check(load_library().sfft_subtract_noalloc(ctypes.byref(desc), _ptr(sci), _ptr(tmpl), _ptr(coeffs),
                                                _ptr(diff), _stream(stream)))


# ---------------------------------------------------------------------------------------
# warm-start network

def _check_cnn(rc, handle):
    if rc != OK:
        lib = load_library()
        msg = lib.sfft_cnn_last_error(handle).decode(errors="replace") or lib.sfft_status_string(rc).decode()
        raise SfftError(rc, msg)


class Cnn:
    """Owns one ``sfft_cnn_t``; created by :func:`sfft_cnn_create`."""

    def __init__(self, handle, n_out, max_batch):
        self.handle, self.n_out, self.max_batch = handle, n_out, max_batch

    def close(self):
        if self.handle:
            load_library().sfft_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def sfft_cnn_create(n_out: int, max_batch: int, stream=None) -> Cnn:
    h = ctypes.c_void_p()
    _check_cnn(load_library().sfft_cnn_create(ctypes.byref(h), n_out, max_batch, _stream(stream)), None)
    return Cnn(h.value, n_out, max_batch)


def sfft_cnn_destroy(cnn: Cnn):
    cnn.close()


def sfft_cnn_param_count(cnn: Cnn) -> int:
    v = ctypes.c_int64()
    _check_cnn(load_library().sfft_cnn_param_count(cnn.handle, ctypes.byref(v)), cnn.handle)
    return v.value


def sfft_cnn_set_params(cnn: Cnn, params):
    """params: a float32 device tensor, or a host buffer address (int)."""
    _check_cnn(load_library().sfft_cnn_set_params(cnn.handle, _ptr(params)), cnn.handle)


def sfft_cnn_get_params(cnn: Cnn, params):
    _check_cnn(load_library().sfft_cnn_get_params(cnn.handle, _ptr(params)), cnn.handle)


def sfft_cnn_save(cnn: Cnn, path: str):
    """Write the network's parameters to a file (see sfft_cnn_save in include/sfft.h)."""
    _check_cnn(load_library().sfft_cnn_save(cnn.handle, os.fsencode(path)), cnn.handle)


def sfft_cnn_load(cnn: Cnn, path: str):
    """Replace the parameters with a file written by sfft_cnn_save for the same output width."""
    _check_cnn(load_library().sfft_cnn_load(cnn.handle, os.fsencode(path)), cnn.handle)


def sfft_cnn_forward(cnn: Cnn, stamps, batch: int, out):
    _check_cnn(load_library().sfft_cnn_forward(cnn.handle, _ptr(stamps), batch, _ptr(out)), cnn.handle)


def sfft_cnn_gradients(cnn: Cnn, stamps, targets, batch: int, grad, grad_in=None, loss=None):
    _check_cnn(load_library().sfft_cnn_gradients(cnn.handle, _ptr(stamps), _ptr(targets), batch, _ptr(grad),
                                                 _ptr(grad_in), _ptr(loss)), cnn.handle)


def sfft_cnn_train_step(cnn: Cnn, stamps, targets, batch: int, lr: float, loss=None):
    _check_cnn(load_library().sfft_cnn_train_step(cnn.handle, _ptr(stamps), _ptr(targets), batch, lr, _ptr(loss)),
               cnn.handle)


def sfft_cnn_train(cnn: Cnn, stamps, targets, n: int, batch: int, epochs: int, lr: float, seed: int):
    """Returns the list of per-epoch mean losses."""
    losses = (ctypes.c_float * epochs)()
    _check_cnn(load_library().sfft_cnn_train(cnn.handle, _ptr(stamps), _ptr(targets), n, batch, epochs, lr,
                                             seed, losses), cnn.handle)
    return list(losses)


def sfft_cnn_warm_start(cnn: Cnn, stamps, batch: int, n_stride: int, x0):
    _check_cnn(load_library().sfft_cnn_warm_start(cnn.handle, _ptr(stamps), batch, n_stride, _ptr(x0)),
               cnn.handle)
