"""The tensor-core products of FP32 basis vectors (dlz_basis_combine, dlz_basis_dots:
the kernels of the FP32 Rayleigh-Ritz restart and of the batched Galerkin projection)
against FP64 products of the same FP32 inputs, through the C ABI.

Tolerance: the operands are split into two TF32 parts and hi*hi + hi*lo + lo*hi is
accumulated in FP32, so each output is within a few FP32 roundings of the exact sum:
|err| <= 4e-6 (combine; 1e-5 for the long dot products) times sum_i |c_i| |v_i|
elementwise; a single TF32 product (10-bit mantissa)
would miss that by two orders of magnitude, which the assertions rule out too."""
import numpy as np
import pytest

from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    return dlz()


@pytest.mark.parametrize("nin,nout,length", [(121, 61, 24 * 1000), (201, 151, 24 * 96), (7, 3, 4 * 333)])
def test_basis_combine_real_coefficients(m, nin, nout, length):
    rng = np.random.default_rng(nin)
    V = rng.standard_normal((nin, length)).astype(np.float32)
    P = rng.standard_normal((nin, nout))
    out = m.basis_combine(torch.from_numpy(V).cuda(), P).cpu().numpy()
    ref = P.T @ V.astype(np.float64)
    bound = 4e-6 * (np.abs(P).T @ np.abs(V.astype(np.float64)))
    assert np.all(np.abs(out - ref) <= bound)


def test_basis_combine_complex_coefficients(m):
    rng = np.random.default_rng(5)
    nin, nout, L = 60, 16, 12 * 800
    V = (rng.standard_normal((nin, L)) + 1j * rng.standard_normal((nin, L))).astype(np.complex64)
    C = rng.standard_normal((nin, nout)) + 1j * rng.standard_normal((nin, nout))
    out = m.basis_combine(torch.from_numpy(V).cuda(), C).cpu().numpy()
    ref = C.T @ V.astype(np.complex128)
    bound = 8e-6 * (np.abs(C).T @ np.abs(V.astype(np.complex128)))
    assert np.all(np.abs(out - ref) <= bound)


@pytest.mark.parametrize("nin,nq,L", [(60, 16, 12 * 4096), (128, 1, 16 * 1000), (5, 3, 16 * 7)])
def test_basis_dots(m, nin, nq, L):
    rng = np.random.default_rng(nin + nq)
    V = (rng.standard_normal((nin, L)) + 1j * rng.standard_normal((nin, L))).astype(np.complex64)
    R = (rng.standard_normal((nq, L)) + 1j * rng.standard_normal((nq, L))).astype(np.complex64)
    C = m.basis_dots(torch.from_numpy(V).cuda(), torch.from_numpy(R).cuda())
    V64, R64 = V.astype(np.complex128), R.astype(np.complex128)
    ref = np.conj(V64) @ R64.T                      # [nin, nq]
    bound = 1e-5 * (np.abs(V64) @ np.abs(R64).T) + 1e-30
    assert np.all(np.abs(C.T - ref) <= bound)


def test_basis_products_reject_shapes_outside_the_tiles(m):
    V = torch.zeros((129, 32), dtype=torch.complex64, device="cuda")
    R = torch.zeros((1, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(m.DlzError):
        m.basis_dots(V, R)
    with pytest.raises(m.DlzError):
        m.basis_combine(torch.zeros((2, 32), dtype=torch.float32, device="cuda"), np.zeros((2, 257)))
