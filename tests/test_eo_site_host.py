"""The even-odd site functions of the CUDA path (csrc/wilson_eo_site.cuh), built for the
host and run site by site on the CPU (tests/eo_site_host.cu), against the even-odd
oracle (oracle/evenodd.py): H_oe, H_eo, Dhat, Dhat^dagger and Qhat in FP64 and FP32
on lattices of several shapes and both time boundaries.  Not in the paper: the first
step of the even-odd form of the Wilson matrix."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle import evenodd as eo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("eo") / "libeo_site_host.so")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_0901_3163_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "eo_site_host.cu"), "-o", out], check=True, capture_output=True)
    L = ctypes.CDLL(out)
    vp, ip = ctypes.c_void_p, ctypes.c_int
    L.eo_hop_f64.argtypes = [ip, vp, ip, vp, vp, vp]
    L.eo_hop_f32.argtypes = [ip, vp, ip, vp, vp, vp]
    L.eo_dhat_f64.argtypes = [ip, vp, ip, ctypes.c_double, vp, vp, vp, vp]
    L.eo_dhat_f32.argtypes = [ip, vp, ip, ctypes.c_float, vp, vp, vp, vp]
    return L


def _planes64(psi_half):                      # (Vh, 4, 3) -> double2[12][Vh]
    return np.ascontiguousarray(psi_half.reshape(-1, 12).T, dtype=np.complex128)


def _unplanes64(p):
    return p.T.reshape(-1, 4, 3)


def _planes32(psi_half):                      # (Vh, 4, 3) -> float4[6][Vh]
    return np.ascontiguousarray(psi_half.reshape(-1, 6, 2).transpose(1, 0, 2), dtype=np.complex64)


def _unplanes32(p):
    return p.transpose(1, 0, 2).reshape(-1, 4, 3).astype(np.complex128)


def _links64(U):                              # (4, V, 3, 3) -> double2[4][9][V]
    return np.ascontiguousarray(U.reshape(4, -1, 9).transpose(0, 2, 1), dtype=np.complex128)


def _links32(U):                              # rows 0 and 1 -> float4[4][3][V]
    return np.ascontiguousarray(U.reshape(4, -1, 9)[:, :, :6].reshape(4, -1, 3, 2).transpose(0, 2, 1, 3),
                                dtype=np.complex64)


def _dims(d):
    return (ctypes.c_int * 4)(*d)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), 1), ((4, 4, 4, 4), -1), ((2, 4, 2, 6), -1),
                                       ((6, 2, 4, 2), 1)])
def test_eo_hops_and_schur_operator(lib, dims, bc_t):
    V = synth.volume(dims)
    Vh = V // 2
    U = synth.su3_links(dims, 21)
    kappa = 0.19
    full = synth.gaussian_spinor(dims, 22)
    xe, xo = eo.split(full, dims)
    U64, U32 = _links64(U), _links32(U)
    d = _dims(dims)
    # H_oe x_e (odd output) and H_eo x_o (even output)
    for par, src, want in [(1, xe, eo.hop_oe(U, xe, dims, bc_t)), (0, xo, eo.hop_eo(U, xo, dims, bc_t))]:
        out = np.empty((12, Vh), dtype=np.complex128)
        inp = _planes64(src)
        lib.eo_hop_f64(par, d, bc_t, inp.ctypes.data, U64.ctypes.data, out.ctypes.data)
        assert _rel(_unplanes64(out), want) < 1e-14
        out32 = np.empty((6, Vh, 2), dtype=np.complex64)
        inp32 = _planes32(src)
        lib.eo_hop_f32(par, d, bc_t, inp32.ctypes.data, U32.ctypes.data, out32.ctypes.data)
        assert _rel(_unplanes32(out32), want) < 3e-6
    # Dhat, Dhat^dagger, Qhat
    oracle = [eo.apply_Dhat, eo.apply_Dhatdag, eo.apply_Qhat]
    for which, f in enumerate(oracle):
        want = f(U, xe, kappa, dims, bc_t)
        t = np.empty((12, Vh), dtype=np.complex128)
        out = np.empty((12, Vh), dtype=np.complex128)
        x = _planes64(xe)
        lib.eo_dhat_f64(which, d, bc_t, kappa, x.ctypes.data, U64.ctypes.data, t.ctypes.data, out.ctypes.data)
        assert _rel(_unplanes64(out), want) < 1e-14
        t32 = np.empty((6, Vh, 2), dtype=np.complex64)
        out32 = np.empty((6, Vh, 2), dtype=np.complex64)
        x32 = _planes32(xe)
        lib.eo_dhat_f32(which, d, bc_t, kappa, x32.ctypes.data, U32.ctypes.data, t32.ctypes.data,
                        out32.ctypes.data)
        assert _rel(_unplanes32(out32), want) < 3e-6


def test_checkerboard_index_is_half_the_site_index():
    """The site order of the oracle's even and odd fields is the kernels' cb = s >> 1."""
    for dims in [(4, 4, 4, 4), (2, 4, 2, 6), (6, 2, 4, 2)]:
        ev, od = eo.sites(dims)
        assert np.array_equal(ev >> 1, np.arange(len(ev)))
        assert np.array_equal(od >> 1, np.arange(len(od)))
