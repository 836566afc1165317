"""ctypes front end of oracle/cwilson.c, the plain-C FP64 Wilson operator.

Test infrastructure only.  `build()` compiles the C file with gcc into
oracle/_build/ (OpenMP when the compiler has it); the functions below build
on first use when the shared object is missing or older than the source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cwilson.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle_wilson.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile cwilson.c into a shared object and return its path.
    (Test infrastructure: builds the C form of the Sec. 2 operator.)"""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        lib.oracle_wilson.argtypes = [dp, dp, dp, ip, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.oracle_wilson.restype = None
        lib.oracle_wilson_sites.argtypes = [dp, dp, dp, ip, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, lp, ctypes.c_long]
        lib.oracle_wilson_sites.restype = None
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def apply_D(U, psi, kappa, dims, bc_t=1, dagger=False):
    """D psi (or D^dagger psi) for one spinor of shape (V, 4, 3) or (V*12,).
    (Sec. 2: the Wilson matrix M (D here), written as plain C site loops.)"""
    lib = _load()
    U = np.ascontiguousarray(U, dtype=np.complex128)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    lib.oracle_wilson(_dp(U), _dp(psi), _dp(out), d, float(kappa), int(bc_t), int(bool(dagger)))
    return out


def apply_D_sites(U, psi, kappa, dims, sites, bc_t=1, dagger=False):
    """(D psi)(s) for the listed sites only; returns (len(sites), 4, 3).
    (Sec. 2: the Wilson matrix M (D here), written as plain C site loops.)"""
    lib = _load()
    U = np.ascontiguousarray(U, dtype=np.complex128)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    lib.oracle_wilson_sites(_dp(U), _dp(psi), _dp(out), d, float(kappa), int(bc_t),
                            int(bool(dagger)), sites.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                            len(sites))
    return out


def _g5(x):
    y = np.array(x, dtype=np.complex128, copy=True).reshape(-1, 4, 3)
    y[:, 2:, :] *= -1.0
    return y.reshape(np.shape(x))


def operator(U, kappa, dims, which="D", bc_t=1):
    """Flat-vector closure x -> A x, which in {'D', 'Ddag', 'Q', 'DdagD'}.

    gamma5 = diag(1, 1, -1, -1) in the chiral basis (a property checked by
    the tests against the product gamma1 gamma2 gamma3 gamma4).
    (Sec. 2: the Wilson matrix M (D here), written as plain C site loops.)
    """
    V = int(np.prod(dims))

    def D(x):
        return apply_D(U, x.reshape(V, 4, 3), kappa, dims, bc_t).reshape(-1)

    def Dd(x):
        return apply_D(U, x.reshape(V, 4, 3), kappa, dims, bc_t, dagger=True).reshape(-1)

    if which == "D":
        return D
    if which == "Ddag":
        return Dd
    def Q(x):
        y = D(x)
        y.reshape(-1, 4, 3)[:, 2:, :] *= -1.0     # gamma5 in place on the fresh output
        return y

    if which == "Q":
        return Q
    if which == "DdagD":
        return lambda x: Dd(D(x))
    raise ValueError(which)
