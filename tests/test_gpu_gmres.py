"""GMRES-DR and D-GMRES on D (dlz_gmresdr, dlz_dgmres; FP64) against the oracle
(oracle/gmres.py) and dense LAPACK, through the C ABI.

Tolerances: the first cycle (no restart yet, the same FP64 algorithm) agrees element by
element to 1e-11 of the largest entry; converged solutions reach ||b - D x|| / ||b|| <=
1e-10 by the oracle's own operator and agree with the dense solve within
2.5e-10 ||b|| / sigma_min(D); after the same fixed number of cycles the kept harmonic
Ritz values agree with the oracle's to 1e-8 (relative) and the iterate to 1e-9 of its
largest entry; the best-converged kept pair lies within 10 times its FP64 residual of
an eigenvalue of D."""
import numpy as np
import pytest

import synth
from oracle import gmres as G
from oracle import wilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def m():
    return dlz()


@pytest.fixture(scope="module")
def case(m):
    kappa = 0.21
    U = synth.su3_links(DIMS, 1)
    op = m.create_operator(DIMS, torch.from_numpy(U).cuda(), kappa)
    n = synth.volume(DIMS) * 12
    D = wilson.operator(U, kappa, DIMS, "D")
    Dm = wilson.dense(D, n)
    return U, kappa, op, D, Dm


def test_first_cycle_matches_oracle_elementwise(m, case):
    U, kappa, op, D, Dm = case
    b = synth.gaussian_spinor(DIMS, 0)
    p = m.params_default(m=30, k=8, tol=1e-30, max_cycles=1)
    x, _, st = m.gmresdr(op, torch.from_numpy(b).cuda(), p, deflate=False)
    xo = G.gmresdr(D, b.reshape(-1), m=30, k=8, tol=0.0, max_cycles=1).x
    assert np.abs(x.cpu().numpy().reshape(-1) - xo).max() <= 1e-11 * np.abs(xo).max()
    assert st.cycles == 1 and st.mvps == 31


def test_gmresdr_converges_to_the_direct_solve(m, case):
    U, kappa, op, D, Dm = case
    b = synth.gaussian_spinor(DIMS, 1)
    p = m.params_default(m=40, k=10, tol=1e-10, max_cycles=500)
    x, defl, st = m.gmresdr(op, torch.from_numpy(b).cuda(), p)
    assert st.converged == 1 and st.true_residual <= 1e-10
    xg = x.cpu().numpy().reshape(-1)
    bf = b.reshape(-1)
    assert np.linalg.norm(bf - D(xg)) <= 1.01e-10 * np.linalg.norm(bf)
    sig = np.linalg.svd(Dm, compute_uv=False)[-1]
    xo = np.linalg.solve(Dm, bf)
    assert np.linalg.norm(xg - xo) <= 2.5e-10 * np.linalg.norm(bf) / sig
    k, which = m.defl_count(defl)
    assert k == 10 and which == m.D
    # the oracle's GMRES-DR reaches the same solution
    ro = G.gmresdr(D, bf, m=40, k=10, tol=1e-10, max_cycles=500)
    assert np.linalg.norm(xg - ro.x) <= 2.5e-10 * np.linalg.norm(bf) / sig


def test_harmonic_ritz_values_match_oracle_and_converge_to_eigenvalues(m, case):
    """The same FP64 algorithm run for a fixed number of cycles on both sides gives the
    same kept harmonic Ritz values and iterate; run past linear convergence (tol far
    below reach), the best-converged pairs sit within their residual of eigenvalues of D."""
    U, kappa, op, D, Dm = case
    b = synth.gaussian_spinor(DIMS, 7)
    p = m.params_default(m=30, k=8, tol=1e-30, max_cycles=6)
    x, defl, st = m.gmresdr(op, torch.from_numpy(b).cuda(), p)
    assert st.cycles == 6 and st.converged == 0
    ro = G.gmresdr(D, b.reshape(-1), m=30, k=8, tol=0.0, max_cycles=6)
    th = np.array([m.defl_value_complex(defl, i) for i in range(8)])
    to = np.sort_complex(ro.theta)
    assert np.all(np.abs(np.sort_complex(th) - to) <= 1e-8 * np.abs(to))
    xo = ro.x
    assert np.abs(x.cpu().numpy().reshape(-1) - xo).max() <= 1e-9 * np.abs(xo).max()
    lam = np.linalg.eigvals(Dm)
    p = m.params_default(m=30, k=8, tol=1e-30, max_cycles=80)
    _, defl, _ = m.gmresdr(op, torch.from_numpy(b).cuda(), p)
    pairs = sorted((m.defl_get(defl, i)[1], m.defl_value_complex(defl, i)) for i in range(8))
    res, t = pairs[0]
    assert res <= 1e-6
    assert np.min(np.abs(lam - t)) <= 10 * res


def test_dgmres_solves_later_rhs_with_fewer_products(m, case):
    U, kappa, op, D, Dm = case
    b0 = synth.gaussian_spinor(DIMS, 2)
    _, defl, st0 = m.gmresdr(op, torch.from_numpy(b0).cuda(), m.params_default(m=40, k=10, tol=1e-10, max_cycles=500))
    B = synth.gaussian_spinors(DIMS, [3, 4, 5])
    pd = m.params_default(m=30, k=10, tol=1e-10, max_iter=100000)
    X, sts = m.dgmres(op, defl, torch.from_numpy(B).cuda(), pd)
    Xp, stp = m.dgmres(op, None, torch.from_numpy(B).cuda(), pd)
    for i in range(3):
        bf = B[i].reshape(-1)
        for XX, ss in ((X, sts), (Xp, stp)):
            assert ss[i].converged == 1
            assert np.linalg.norm(bf - D(XX[i].cpu().numpy().reshape(-1))) <= 1.01e-10 * np.linalg.norm(bf)
        assert sts[i].mvps < stp[i].mvps
    # the oracle's D-GMRES over the oracle's own GMRES-DR space reaches the same x
    ro = G.gmresdr(D, b0.reshape(-1), m=40, k=10, tol=1e-10, max_cycles=500)
    xo, _ = G.dgmres(D, B[0].reshape(-1), ro.V, ro.Hbar, m=30, tol=1e-10)
    sig = np.linalg.svd(Dm, compute_uv=False)[-1]
    assert np.linalg.norm(X[0].cpu().numpy().reshape(-1) - xo) <= 2.5e-10 * np.linalg.norm(B[0]) / sig


def test_gmres_rejects_fp32_and_foreign_sets(m, case):
    U, kappa, op, D, Dm = case
    b = torch.from_numpy(synth.gaussian_spinor(DIMS, 6)).cuda()
    with pytest.raises(m.DlzError) as e:
        m.gmresdr(op, b, m.params_default(m=20, k=5, precision=m.F32))
    assert e.value.code == m.ERR_BADARG
    _, dq, _ = m.minresdr(op, b, m.params_default(m=20, k=5, max_cycles=200))
    with pytest.raises(m.DlzError):
        m.dgmres(op, dq, b[None].contiguous(), m.params_default(m=20, k=5))
