"""TEST INFRASTRUCTURE -- not part of the product path.

Python access to the plain CPU oracle in ``hankel_oracle.c``: the direct
O(N^2) FP64 evaluation of Eq. (2) of Townsend, arXiv:1501.01652,

    f_k = sum_{n=1}^{N} c_n J_nu(r_k omega_n),

with Kahan summation and its own Bessel evaluator, plus a double-double
brute force for N <= 64. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package. It shares no code
with the CUDA library and never imports it.

Tasks (Section 1): ``"schlomilch"`` (omega_n = (n+gamma)pi, Section 4),
``"fourier_bessel"`` (omega_n = j_{0,n}, Section 5) and ``"dht"``
(r_k = j_{0,k}/j_{0,N+1}, omega_n = j_{0,n}, Section 6). ``grid=0`` samples
tasks 0 and 1 at r_k = (k-1)/(N-1); ``grid=1`` at the paper's r_k = k/N.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hankel_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
TASKS = {"schlomilch": 0, "fourier_bessel": 1, "dht": 2}
_lib = None


def build(force=False):
    """Compile the oracle with gcc (no fast-math, no FMA contraction) and return the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i64, dbl, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_int64)
    lib.orc_besselj.restype = dbl
    lib.orc_besselj.argtypes = [i32, dbl]
    lib.orc_besselj_pi.restype = dbl
    lib.orc_besselj_pi.argtypes = [i32, i64, i64, dbl]
    lib.orc_besselj_dd.restype = dbl
    lib.orc_besselj_dd.argtypes = [i32, dbl]
    lib.orc_j0_zero_offsets.restype = i32
    lib.orc_j0_zero_offsets.argtypes = [i64, dp]
    lib.orc_j0_zero_offsets_dd.restype = i32
    lib.orc_j0_zero_offsets_dd.argtypes = [i64, dp]
    lib.orc_transform.restype = i32
    lib.orc_transform.argtypes = [i32, i32, i32, i64, i64, i32, dp, i64, lp, i64, dp, i64, i32]
    lib.orc_transform_dd.restype = i32
    lib.orc_transform_dd.argtypes = [i32, i32, i32, i64, i64, i32, dp, i64, dp, i64]
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def besselj(nu, z):
    """J_nu(z) in FP64 (series / Miller / Hankel by regime)."""
    return _load().orc_besselj(int(nu), float(z))


def besselj_pi(nu, P, Q, delta=0.0):
    """J_nu(pi*P/Q + delta) with the large-z phase reduced exactly in integers."""
    return _load().orc_besselj_pi(int(nu), int(P), int(Q), float(delta))


def besselj_dd(nu, z):
    """J_nu(z) computed in double-double and rounded to FP64."""
    return _load().orc_besselj_dd(int(nu), float(z))


def j0_zero_offsets(count):
    """b_n = j_{0,n} - (n-1/4)pi for n = 1..count (Lemma 3.2), FP64."""
    b = np.empty(int(count), dtype=np.float64)
    _load().orc_j0_zero_offsets(int(count), _dptr(b))
    return b


def j0_zero_offsets_dd(count):
    """b_n from double-double Newton iterations (count <= 4096)."""
    b = np.empty(int(count), dtype=np.float64)
    if _load().orc_j0_zero_offsets_dd(int(count), _dptr(b)) != 0:
        raise ValueError("count out of range")
    return b


def _gamma(task, nu, gamma):
    if gamma is None:
        return int(nu) if task == "schlomilch" else 0
    return int(gamma)


def transform(task, nu, N, c, rows=None, grid=0, gamma=None, nthreads=0):
    """Direct O(N^2) sum for the listed 0-based rows (default: all).

    ``c`` has shape (N,) or (nrhs, N); the result has shape (nrows,) or
    (nrhs, nrows) to match.
    """
    c = np.ascontiguousarray(c, dtype=np.float64)
    single = c.ndim == 1
    c2 = c.reshape(1, -1) if single else c
    if c2.shape[1] != N:
        raise ValueError("c has the wrong length")
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    f = np.zeros((c2.shape[0], rows.size), dtype=np.float64)
    rc = _load().orc_transform(TASKS[task], int(nu), int(grid), _gamma(task, nu, gamma), int(N),
                               c2.shape[0], _dptr(c2), int(N),
                               rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rows.size,
                               _dptr(f), rows.size, int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return f[0] if single else f


def transform_dd(task, nu, N, c, grid=0, gamma=None):
    """Double-double brute force of the same sum, all rows, N <= 64."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    single = c.ndim == 1
    c2 = c.reshape(1, -1) if single else c
    f = np.zeros((c2.shape[0], N), dtype=np.float64)
    rc = _load().orc_transform_dd(TASKS[task], int(nu), int(grid), _gamma(task, nu, gamma), int(N),
                                  c2.shape[0], _dptr(c2), int(N), _dptr(f), int(N))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return f[0] if single else f
