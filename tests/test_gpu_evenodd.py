"""The even-odd (Schur complement) operator on the GPU against the FP64 oracle
(oracle/evenodd.py), through the C ABI: Dhat, Dhat^dag, Qhat and Dhat^dag Dhat element
by element on three lattice shapes and both time boundaries, the preparation of the
even right-hand side and the reconstruction of the full solution, and the deflated
solvers run on the even sites (Lan-DR + D-CG in FP64 and FP32, MinRes-DR + D-MinRes
in FP64), whose reconstructed full solutions must reach ||b - D x|| / ||b|| <= 1e-10
by the oracle's own full-lattice operator.

Tolerances: FP64 operator 1e-14 of the largest element; FP32 3e-6 (the FP32 stencil
with 12-real links against the FP64 oracle on FP32-rounded input)."""
import numpy as np
import pytest

import synth
from oracle import evenodd as EO
from oracle import wilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAMES = {"Dhat": 0, "Dhatdag": 1, "Qhat": 2, "DhatdagDhat": 3}


@pytest.fixture(scope="module")
def m():
    return dlz()


@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), 1), ((4, 4, 4, 8), -1), ((6, 4, 2, 8), 1)])
def test_evenodd_operator_elementwise(m, dims, bc_t):
    U = synth.su3_links(dims, 11)
    kappa = 0.21
    op = m.create_operator_eo(dims, torch.from_numpy(U).cuda(), kappa, bc_t=bc_t)
    Vh = synth.volume(dims) // 2
    assert op.volume == Vh
    X = synth.gaussian_spinors(dims, [5, 6])[:, ::2].copy()        # any even-site vectors
    X = X.reshape(2, Vh, 4, 3)
    for name, which in NAMES.items():
        A = EO.operator(U, kappa, dims, name, bc_t)
        ref = np.stack([A(X[i].reshape(-1)).reshape(Vh, 4, 3) for i in range(2)])
        got = m.apply(op, which, torch.from_numpy(X).cuda()).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max(), name
        X32 = X.astype(np.complex64)
        ref32 = np.stack([A(X32[i].astype(np.complex128).reshape(-1)).reshape(Vh, 4, 3) for i in range(2)])
        got32 = m.apply(op, which, torch.from_numpy(X32).cuda()).cpu().numpy()
        assert np.abs(got32 - ref32).max() <= 3e-6 * np.abs(ref32).max(), name


def test_evenodd_prepare_and_reconstruct(m):
    dims, kappa = (4, 4, 4, 8), 0.2
    U = synth.su3_links(dims, 12)
    op = m.create_operator_eo(dims, torch.from_numpy(U).cuda(), kappa)
    b = synth.gaussian_spinors(dims, [7, 8])
    be = m.eo_prepare(op, torch.from_numpy(b).cuda()).cpu().numpy()
    for i in range(2):
        ref = EO.prepare(U, b[i], kappa, dims)
        assert np.abs(be[i] - ref).max() <= 1e-14 * np.abs(ref).max()
    xe = synth.gaussian_spinors(dims, [9, 10])[:, ::2].copy().reshape(2, -1, 4, 3)
    x = m.eo_reconstruct(op, torch.from_numpy(xe).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    for i in range(2):
        ref = EO.reconstruct(U, xe[i], b[i], kappa, dims)
        assert np.abs(x[i] - ref).max() <= 1e-14 * np.abs(ref).max()


def _full_residual(U, kappa, dims, x, b):
    D = wilson.operator(U, kappa, dims, "D")
    return np.linalg.norm(b.reshape(-1) - D(x.reshape(-1))) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_evenodd_landr_dcg_reconstructed_solutions(m, prec):
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 1)
    kappa = synth.kappa_for(dims, 1)            # the sigma_min = 1e-3 workload kappa
    op = m.create_operator_eo(dims, torch.from_numpy(U).cuda(), kappa)
    B = synth.gaussian_spinors(dims, [0, 1, 2, 3])
    Bd = torch.from_numpy(B).cuda()
    Be = m.eo_prepare(op, Bd)
    pr = m.F64 if prec == "f64" else m.F32
    p = m.params_default(m=40, k=10, tol=1e-10, max_cycles=2000, precision=pr, finish=1)
    xe0, defl, st = m.landr(op, Be[0].contiguous(), p)
    assert st.converged == 1 and st.true_residual <= 1e-10
    Xe, sts = m.dcg(op, defl, Be[1:].contiguous(), m.params_default(m=40, k=10, tol=1e-10, precision=pr))
    xe = torch.cat([xe0[None], Xe])
    X = m.eo_reconstruct(op, xe.contiguous(), Bd).cpu().numpy()
    for i in range(4):
        assert _full_residual(U, kappa, dims, X[i], B[i]) <= 1.01e-10
    for s in sts:
        assert s.converged == 1
    # the same solutions as the direct dense solve of the full D (sigma_min = 1e-3)
    n = synth.volume(dims) * 12
    Dm = wilson.dense(wilson.operator(U, kappa, dims, "D"), n)
    for i in range(4):
        xo = np.linalg.solve(Dm, B[i].reshape(-1))
        assert np.linalg.norm(X[i].reshape(-1) - xo) <= 2.5e-10 * np.linalg.norm(B[i]) / 1e-3


def test_evenodd_minresdr_dminres_fp64_and_fp32_rejected(m):
    dims, kappa = (4, 4, 4, 8), 0.22
    U = synth.su3_links(dims, 13)
    op = m.create_operator_eo(dims, torch.from_numpy(U).cuda(), kappa)
    B = synth.gaussian_spinors(dims, [0, 1, 2])
    Bd = torch.from_numpy(B).cuda()
    Be = m.eo_prepare(op, Bd)
    p = m.params_default(m=40, k=10, tol=1e-10, max_cycles=2000)
    xe0, defl, st = m.minresdr(op, Be[0].contiguous(), p)
    assert st.converged == 1
    Xe, sts = m.dminres(op, defl, Be[1:].contiguous(), p)
    X = m.eo_reconstruct(op, torch.cat([xe0[None], Xe]).contiguous(), Bd).cpu().numpy()
    for i in range(3):
        assert _full_residual(U, kappa, dims, X[i], B[i]) <= 1.01e-10
    # the harmonic Ritz values are those of Qhat: Rayleigh quotients within their residual
    Qh = EO.operator(U, kappa, dims, "Qhat")
    y = np.empty((synth.volume(dims) // 2, 4, 3), dtype=np.complex128)
    val, res = m.defl_get(defl, 0, y)
    qy = Qh(y.reshape(-1))
    assert abs(np.linalg.norm(qy - val * y.reshape(-1)) - res) <= 1e-10
    with pytest.raises(m.DlzError) as e:
        m.dminres(op, defl, Be[1:].contiguous(), m.params_default(m=40, k=10, tol=1e-10, precision=m.F32))
    assert e.value.code == m.ERR_BADARG


def test_evenodd_stencil_at_16x16x16x32(m):
    dims, kappa = (16, 16, 16, 32), 0.27
    U = synth.su3_links(dims, 2)
    op = m.create_operator_eo(dims, torch.from_numpy(U).cuda(), kappa)
    Vh = synth.volume(dims) // 2
    x = synth.gaussian_spinor(dims, 3)[::2].copy().reshape(Vh, 4, 3).astype(np.complex64)
    got = m.apply(op, m.DDAGD, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = EO.operator(U, kappa, dims, "DhatdagDhat")(x.astype(np.complex128).reshape(-1)).reshape(Vh, 4, 3)
    assert np.abs(got - ref).max() <= 3e-6 * np.abs(ref).max()
