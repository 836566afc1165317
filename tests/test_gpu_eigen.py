"""Lan-DR and MinRes-DR as eigensolvers (dlz_params.eig_only; Sec. 2 keeps the k
lowest eigenvectors of the first right-hand side's solve, up to the paper's k = 150
with m = 200), through the C ABI, against dense LAPACK eigensolves of the 4^4 Wilson
matrices and the FP64 oracle's own eigensolver run.

Tolerances: FP64 Ritz values within 1e-8 relative of the exact eigenvalues (every
kept pair, since the cycles stop only when all of them converged); FP32 (kept
residuals to 1e-5 ||A||): within 1e-4 relative."""
import numpy as np
import pytest

import synth
from oracle import krylov as K
from oracle import wilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (4, 4, 4, 4)
KAPPA = 0.2


@pytest.fixture(scope="module")
def m():
    return dlz()


@pytest.fixture(scope="module")
def case(m):
    U = synth.su3_links(DIMS, 1)
    op = m.create_operator(DIMS, torch.from_numpy(U).cuda(), KAPPA)
    n = synth.volume(DIMS) * 12
    Dm = wilson.dense(wilson.operator(U, KAPPA, DIMS, "D"), n)
    g5 = np.diag(np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), synth.volume(DIMS)))
    ev_dd = np.linalg.eigvalsh(Dm.conj().T @ Dm)
    ev_q = np.linalg.eigvalsh(g5 @ Dm)
    b = synth.gaussian_spinor(DIMS, 0)
    return U, op, b, ev_dd, ev_q


def _values(m, defl):
    k, _ = m.defl_count(defl)
    return np.array([m.defl_get(defl, i) for i in range(k)])


@pytest.mark.parametrize("mm,k", [(40, 10), (200, 150)])
def test_landr_eigensolver_fp64_against_dense(m, case, mm, k):
    U, op, b, ev_dd, _ = case
    p = m.params_default(m=mm, k=k, tol=1e-10, eig_only=1, max_cycles=4000)
    _, defl, st = m.landr(op, torch.from_numpy(b).cuda(), p)
    assert st.converged == 1
    vals = _values(m, defl)
    got = np.sort(vals[:, 0])
    exact = ev_dd[:k]
    assert np.all(np.abs(got - exact) <= 1e-8 * exact)
    if k == 10:
        Ad = wilson.operator(U, KAPPA, DIMS, "DdagD")
        bp = wilson.operator(U, KAPPA, DIMS, "Ddag")(b.reshape(-1))
        r = K.landr(Ad, bp, m=mm, k=k, tol=1e-10, eig_only=True, max_cycles=4000)
        assert r.info.converged
        assert np.all(np.abs(got - np.sort(r.ritz_values)) <= 1e-8 * exact)


def test_minresdr_eigensolver_fp64_against_dense(m, case):
    U, op, b, _, ev_q = case
    p = m.params_default(m=40, k=10, tol=1e-10, eig_only=1, max_cycles=4000)
    _, defl, st = m.minresdr(op, torch.from_numpy(b).cuda(), p)
    assert st.converged == 1
    got = np.sort(_values(m, defl)[:, 0])
    exact = np.sort(ev_q[np.argsort(np.abs(ev_q))[:10]])
    assert np.all(np.abs(got - exact) <= 1e-8 * np.abs(exact))


def test_landr_eigensolver_fp32(m, case):
    U, op, b, ev_dd, _ = case
    p = m.params_default(m=60, k=20, tol=1e-10, eig_only=1, max_cycles=4000, precision=m.F32)
    _, defl, st = m.landr(op, torch.from_numpy(b).cuda(), p)
    assert st.converged == 1
    got = np.sort(_values(m, defl)[:, 0])
    assert np.all(np.abs(got - ev_dd[:20]) <= 1e-4 * ev_dd[:20])
