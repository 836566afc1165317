"""The block walk of the batched FP32 stencils (csrc/slab_walk.cuh), built for the host:
every site of a lattice (or of one parity of an even-odd field) is visited by exactly one
block, blocks hold at most 128 contiguous sites of one slab, and the slab the library
chooses is the largest divisor of Lz within its traffic budget (DLZ_SLAB fixes it)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("slab") / "libslab_walk_host.so")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_0901_3163_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "slab_walk_host.cu"), "-o", out], check=True, capture_output=True)
    L = ctypes.CDLL(out)
    L.slab_choice.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_void_p]
    L.slab_blocks_of.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p, ctypes.c_void_p]
    return L


def _walk(lib, plane, Lz, Lt, bz):
    V = plane * Lz * Lt
    cap = (V // 128 + 4) * (Lz + 1)
    s0 = np.zeros(cap, dtype=np.int32)
    nb = np.zeros(cap, dtype=np.int32)
    n = lib.slab_blocks_of(plane, Lz, Lt, bz, s0.ctypes.data, nb.ctypes.data)
    return s0[:n], nb[:n]


@pytest.mark.parametrize("plane,Lz,Lt", [(576, 24, 48), (288, 24, 48), (256, 16, 32), (16, 6, 8),
                                         (64, 8, 8), (6, 5, 3), (1, 1, 1)])
@pytest.mark.parametrize("bz", [1, 2, 3, 4, 5, 8, 24])
def test_every_site_once(lib, plane, Lz, Lt, bz):
    V = plane * Lz * Lt
    s0, nb = _walk(lib, plane, Lz, Lt, bz)
    seen = np.zeros(V, dtype=np.int32)
    b = min(bz, Lz)
    for a, n in zip(s0, nb):
        assert 0 <= n <= 128
        if n == 0:
            continue
        assert 0 <= a and a + n <= V
        # a block lies inside one slab: one t, z-planes [z0, z0 + b)
        t0, t1 = a // (plane * Lz), (a + n - 1) // (plane * Lz)
        z0, z1 = (a // plane) % Lz, ((a + n - 1) // plane) % Lz
        assert t0 == t1 and z0 // b == z1 // b
        seen[a:a + n] += 1
    assert np.all(seen == 1)


def test_choice_is_the_largest_divisor_within_budget(lib, monkeypatch):
    monkeypatch.delenv("DLZ_SLAB", raising=False)
    out = np.zeros(3, dtype=np.int64)
    # 24^3 x 48, 16 RHS, the CGNR kernels' ~900 B per site and RHS: 36 MB / (576 x 16 x 900) = 4.3
    lib.slab_choice(576, 24, 48, 16, 900.0, out.ctypes.data)
    assert out[0] == 4 and out[1] == 18 and out[2] == 18 * 48 * 6
    # a small lattice fits whole: the plain order
    lib.slab_choice(16, 6, 8, 3, 900.0, out.ctypes.data)
    assert out[0] == 6
    # 7 planes fit the budget, the largest divisor of 24 below is 6
    lib.slab_choice(576, 24, 48, 16, 36.0e6 / (576 * 16 * 7.5), out.ctypes.data)
    assert out[0] == 6
    monkeypatch.setenv("DLZ_SLAB", "5")
    lib.slab_choice(576, 24, 48, 16, 900.0, out.ctypes.data)
    assert out[0] == 5
