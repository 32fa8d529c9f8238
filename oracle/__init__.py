"""FP64 CPU oracle for the SFFT fit and subtraction.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` are the only callers.  The CUDA library never imports, links or calls it,
and it shares no code with the CUDA path.

The arithmetic lives in ``sfft_oracle.c`` (plain C, FP64, OpenMP, Neumaier-compensated
direct spatial sums, no FFT).  This module only compiles that file with gcc and marshals
numpy arrays through ctypes.  The statement of the problem that the C file implements is
in its header comment: a delta-basis matching kernel with a degree-DK spatial polynomial
per lag plus a degree-DB polynomial background, fitted by least squares on the masked
frames and applied to the unmasked template (the SFFT subtraction step, Sec. "Pipeline
steps", step 6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfft_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_OOM, ERR_NOT_SPD = 0, 1, 3, 4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/lib/liboracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    # -O2 without -ffast-math: the compensated sums must not be re-associated.
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.oracle_lag_tables.argtypes = [I, I, P, P, P, I, I, I, P, P, P, P, P]
        lib.oracle_lag_tables_band.argtypes = [I, I, P, P, P, I, I, I, I, I, P, P, P, P, P]
        lib.oracle_normal.argtypes = [I, I, P, P, P, I, I, I, P, P]
        lib.oracle_brute_normal.argtypes = [I, I, P, P, P, I, I, I, P, P]
        lib.oracle_normal_entries.argtypes = [I, I, P, P, P, I, I, I, I, P, P, P]
        lib.oracle_assemble.argtypes = [I, I, I, P, P, P, P, P, P, P]
        lib.oracle_cholesky_solve.argtypes = [I, P, P, P]
        lib.oracle_fit.argtypes = [I, I, P, P, P, I, I, I, P]
        lib.oracle_subtract.argtypes = [I, I, P, P, I, I, I, P, P]
        lib.oracle_subtract_pixels.argtypes = [I, I, P, P, I, I, I, P, I, P, P]
        lib.oracle_n_unknowns.argtypes = [I, I, I]
        lib.oracle_convolve.argtypes = [I, I, P, I, P, P]
        lib.oracle_npoly.argtypes = [I]
        lib.oracle_mono_pq.argtypes = [I, P, P]
        for name in ("oracle_lag_tables", "oracle_lag_tables_band", "oracle_normal", "oracle_brute_normal",
                     "oracle_normal_entries", "oracle_assemble", "oracle_cholesky_solve",
                     "oracle_fit", "oracle_subtract", "oracle_subtract_pixels",
                     "oracle_n_unknowns", "oracle_npoly", "oracle_num_threads", "oracle_convolve"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mask(m, shape):
    if m is None:
        return None
    m = np.ascontiguousarray(m, dtype=np.uint8)
    if m.shape != shape:
        raise ValueError("mask shape %r != image shape %r" % (m.shape, shape))
    return m


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc == ERR_NOT_SPD:
        raise OracleError("%s: normal matrix is not symmetric positive definite" % what)
    if rc != OK:
        raise OracleError("%s failed with code %d" % (what, rc))


def npoly(d: int) -> int:
    return (d + 1) * (d + 2) // 2 if d >= 0 else 0


def n_unknowns(L: int, dk: int, db: int) -> int:
    return L * L * npoly(dk) + npoly(db)


def mono_pq(idx: int):
    lib = _load()
    p, q = ctypes.c_int(), ctypes.c_int()
    lib.oracle_mono_pq(idx, ctypes.byref(p), ctypes.byref(q))
    return p.value, q.value


def num_threads() -> int:
    return _load().oracle_num_threads()


def lag_tables(S, T, mask, L, dk, db):
    """Lag tables by direct sums: dict with Cww, Cwg, Cws, Ggg, Ggs (see sfft_oracle.c)."""
    lib = _load()
    S, T = _f64(S), _f64(T)
    ny, nx = S.shape
    m = _mask(mask, S.shape)
    nk, nb, Lw = npoly(dk), npoly(db), 2 * L - 1
    out = dict(Cww=np.zeros((nk * (nk + 1) // 2, Lw, Lw)), Cwg=np.zeros((nk, nb, L, L)),
               Cws=np.zeros((nk, L, L)), Ggg=np.zeros((nb, nb)), Ggs=np.zeros(nb))
    rc = lib.oracle_lag_tables(ny, nx, _ptr(S), _ptr(T), _ptr(m), L, dk, db,
                               *[_ptr(out[k]) for k in ("Cww", "Cwg", "Cws", "Ggg", "Ggs")])
    _check(rc, "oracle_lag_tables")
    return out


def lag_tables_band(S, T, mask, L, dk, db, y0, y1):
    """The lag tables of ``lag_tables`` with the sums restricted to rows y0 <= y < y1 of the
    first factor; tables of bands that cover every row add up to the full tables."""
    lib = _load()
    S, T = _f64(S), _f64(T)
    ny, nx = S.shape
    m = _mask(mask, S.shape)
    nk, nb, Lw = npoly(dk), npoly(db), 2 * L - 1
    out = dict(Cww=np.zeros((nk * (nk + 1) // 2, Lw, Lw)), Cwg=np.zeros((nk, nb, L, L)),
               Cws=np.zeros((nk, L, L)), Ggg=np.zeros((nb, nb)), Ggs=np.zeros(nb))
    rc = lib.oracle_lag_tables_band(ny, nx, _ptr(S), _ptr(T), _ptr(m), L, dk, db, int(y0), int(y1),
                                    *[_ptr(out[k]) for k in ("Cww", "Cwg", "Cws", "Ggg", "Ggs")])
    _check(rc, "oracle_lag_tables_band")
    return out


def assemble(tables, L, dk, db):
    lib = _load()
    n = n_unknowns(L, dk, db)
    N, b = np.zeros((n, n)), np.zeros(n)
    t = {k: _f64(v) for k, v in tables.items()}
    rc = lib.oracle_assemble(L, dk, db, *[_ptr(t[k]) for k in ("Cww", "Cwg", "Cws", "Ggg", "Ggs")],
                             _ptr(N), _ptr(b))
    _check(rc, "oracle_assemble")
    return N, b


def normal_equations(S, T, mask, L, dk, db):
    """(N, b) from the lag tables (direct sums, FP64)."""
    lib = _load()
    S, T = _f64(S), _f64(T)
    ny, nx = S.shape
    m = _mask(mask, S.shape)
    n = n_unknowns(L, dk, db)
    N, b = np.zeros((n, n)), np.zeros(n)
    _check(lib.oracle_normal(ny, nx, _ptr(S), _ptr(T), _ptr(m), L, dk, db, _ptr(N), _ptr(b)),
           "oracle_normal")
    return N, b


def brute_normal_equations(S, T, mask, L, dk, db):
    """(N, b) from materialised basis images and explicit dot products (tiny frames)."""
    lib = _load()
    S, T = _f64(S), _f64(T)
    ny, nx = S.shape
    m = _mask(mask, S.shape)
    n = n_unknowns(L, dk, db)
    N, b = np.zeros((n, n)), np.zeros(n)
    _check(lib.oracle_brute_normal(ny, nx, _ptr(S), _ptr(T), _ptr(m), L, dk, db, _ptr(N), _ptr(b)),
           "oracle_brute_normal")
    return N, b


def normal_entries(S, T, mask, L, dk, db, rows, cols):
    """Entries <basis_row, basis_col> by definition; col == n selects S_m (the RHS b)."""
    lib = _load()
    S, T = _f64(S), _f64(T)
    ny, nx = S.shape
    m = _mask(mask, S.shape)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.zeros(len(rows))
    _check(lib.oracle_normal_entries(ny, nx, _ptr(S), _ptr(T), _ptr(m), L, dk, db, len(rows),
                                     _ptr(rows), _ptr(cols), _ptr(out)), "oracle_normal_entries")
    return out


def cholesky_solve(N, b):
    lib = _load()
    N, b = _f64(N), _f64(b)
    x = np.zeros(len(b))
    _check(lib.oracle_cholesky_solve(len(b), _ptr(N), _ptr(b), _ptr(x)), "oracle_cholesky_solve")
    return x


def fit(S, T, mask, L, dk, db):
    """theta = N^{-1} b (FP64 Cholesky on the lag-table normal equations)."""
    lib = _load()
    S, T = _f64(S), _f64(T)
    ny, nx = S.shape
    m = _mask(mask, S.shape)
    theta = np.zeros(n_unknowns(L, dk, db))
    _check(lib.oracle_fit(ny, nx, _ptr(S), _ptr(T), _ptr(m), L, dk, db, _ptr(theta)), "oracle_fit")
    return theta


def subtract(S, T, theta, L, dk, db):
    """Difference image on the unmasked frames, by direct spatial sums."""
    lib = _load()
    S, T, theta = _f64(S), _f64(T), _f64(theta)
    ny, nx = S.shape
    D = np.zeros((ny, nx))
    _check(lib.oracle_subtract(ny, nx, _ptr(S), _ptr(T), L, dk, db, _ptr(theta), _ptr(D)),
           "oracle_subtract")
    return D


def subtract_pixels(S, T, theta, L, dk, db, flat_idx):
    lib = _load()
    S, T, theta = _f64(S), _f64(T), _f64(theta)
    ny, nx = S.shape
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.zeros(len(idx))
    _check(lib.oracle_subtract_pixels(ny, nx, _ptr(S), _ptr(T), L, dk, db, _ptr(theta), len(idx),
                                      _ptr(idx), _ptr(out)), "oracle_subtract_pixels")
    return out


def convolve(X, P):
    """Cyclic convolution of the image X with the odd-sized square stamp P (centred on its
    middle element), by direct FP64 sums: the cross-convolution of the pipeline."""
    lib = _load()
    X, P = _f64(X), _f64(P)
    ny, nx = X.shape
    K = P.shape[0]
    if P.shape != (K, K):
        raise ValueError("stamp must be square")
    out = np.zeros((ny, nx))
    _check(lib.oracle_convolve(ny, nx, _ptr(X), K, _ptr(P), _ptr(out)), "oracle_convolve")
    return out
