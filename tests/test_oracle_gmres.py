"""Pins of the GMRES-DR / D-GMRES oracle (oracle/gmres.py), the non-hermitian deflated
methods the paper contrasts with (its refs. [1], [2]):

* one cycle is GMRES: the residual minimiser over an explicit Krylov basis;
* cycle 2 is the residual minimiser over span{harmonic Ritz vectors of cycle 1} plus
  the Krylov space of the cycle-1 residual (the defining property of the restart);
* residual norms never increase from cycle to cycle;
* on a hermitian matrix it coincides with MinRes-DR run with full re-orthogonalisation
  (both are GMRES-DR in exact arithmetic), on the paper's indefinite example (Sec. 1);
* on a normal matrix with known complex eigenvalues the kept harmonic Ritz values
  converge to the eigenvalues nearest zero;
* GMRES-DR and D-GMRES on the 4^4 Wilson matrix reach the direct solve, and the
  deflated D-GMRES takes fewer products with D than plain restarted GMRES."""
import numpy as np
import pytest

import synth
from oracle import gmres as G
from oracle import krylov as K
from oracle import wilson


def _dense_op(M):
    return lambda v: M @ v


def _krylov(A, r, j):
    Q = [r / np.linalg.norm(r)]
    while len(Q) < j:
        w = A(Q[-1])
        for _ in range(2):
            for q in Q:
                w = w - np.vdot(q, w) * q
        Q.append(w / np.linalg.norm(w))
    return np.stack(Q, axis=1)


def _nonnormal(n, seed):
    rng = np.random.default_rng(seed)
    M = np.diag(1.0 + rng.random(n) + 0.5j * rng.standard_normal(n))
    M += 0.3 * np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), 1) / np.sqrt(n)
    return M


def test_one_cycle_is_gmres():
    M = _nonnormal(120, 1)
    A = _dense_op(M)
    b = np.random.default_rng(2).standard_normal(120) + 0j
    r = G.gmresdr(A, b, m=25, k=5, tol=0.0, max_cycles=1)
    Q = _krylov(A, b, 25)
    z, *_ = np.linalg.lstsq(M @ Q, b, rcond=None)
    assert np.linalg.norm(r.x - Q @ z) <= 1e-10 * np.linalg.norm(Q @ z)


def test_second_cycle_is_the_augmented_residual_minimiser():
    M = _nonnormal(150, 3)
    A = _dense_op(M)
    b = np.random.default_rng(4).standard_normal(150) + 1j * np.random.default_rng(5).standard_normal(150)
    m, k = 20, 6
    r1 = G.gmresdr(A, b, m=m, k=k, tol=0.0, max_cycles=1)
    r2 = G.gmresdr(A, b, m=m, k=k, tol=0.0, max_cycles=2)
    # cycle-1 harmonic Ritz vectors from an independent run of the first cycle
    V = np.zeros((150, m + 1), dtype=complex)
    H = np.zeros((m + 1, m), dtype=complex)
    V[:, 0] = b / np.linalg.norm(b)
    G._arnoldi(A, V, H, 0, m)
    _, Gk = G.harmonic_ritz(H, m, k)
    res1 = b - M @ r1.x
    S = np.hstack([V[:, :m] @ Gk, _krylov(A, res1, m - k)])
    z, *_ = np.linalg.lstsq(M @ S, res1, rcond=None)
    x_bf = r1.x + S @ z
    assert np.linalg.norm(r2.x - x_bf) <= 1e-9 * np.linalg.norm(x_bf)


def test_residuals_never_increase():
    M = _nonnormal(200, 6)
    b = np.ones(200, dtype=complex)
    r = G.gmresdr(_dense_op(M), b, m=15, k=5, tol=1e-12, max_cycles=40)
    h = np.array(r.info.residuals)
    assert np.all(np.diff(h) <= 1e-12 * h[0])


def test_hermitian_case_equals_minresdr_with_full_reorthogonalisation():
    d, _ = synth.diag_indefinite_1000()
    A = lambda v: d * v  # noqa: E731
    b = np.ones(1000, dtype=complex) / np.sqrt(1000)
    rg = G.gmresdr(A, b, m=40, k=10, tol=0.0, max_cycles=3)
    rm = K.minresdr(A, b, m=40, k=10, tol=0.0, max_cycles=3, full_reorth=True)
    assert np.linalg.norm(rg.x - rm.x) <= 1e-8 * np.linalg.norm(rm.x)


def test_harmonic_ritz_values_converge_to_the_eigenvalues_nearest_zero():
    rng = np.random.default_rng(7)
    lam = (0.05 + np.arange(300)) * np.exp(1j * rng.uniform(-0.6, 0.6, 300))
    A = lambda v: lam * v  # noqa: E731
    b = np.ones(300, dtype=complex)
    r = G.gmresdr(A, b, m=30, k=8, tol=0.0, max_cycles=60)      # run past convergence
    near = lam[np.argsort(np.abs(lam))[:4]]
    for t in near:
        assert np.min(np.abs(r.theta - t)) <= 1e-8 * abs(t)


def test_wilson_gmresdr_and_dgmres_reach_the_direct_solve():
    dims, kappa = (4, 4, 4, 4), 0.2
    U = synth.su3_links(dims, 1)
    D = wilson.operator(U, kappa, dims, "D")
    n = synth.volume(dims) * 12
    Dm = wilson.dense(D, n)
    B = synth.gaussian_spinors(dims, [0, 1]).reshape(2, -1)
    r = G.gmresdr(D, B[0], m=40, k=10, tol=1e-10, max_cycles=200)
    assert r.info.converged
    xo = np.linalg.solve(Dm, B[0])
    assert np.linalg.norm(r.x - xo) <= 1e-8 * np.linalg.norm(xo)
    # the kept space satisfies A V_k = V_{k+1} Hbar_k
    Vk1, Hb = r.V, r.Hbar
    k = Hb.shape[1]
    assert np.linalg.norm(Dm @ Vk1[:, :k] - Vk1 @ Hb) <= 1e-10 * np.linalg.norm(Hb)
    x, info = G.dgmres(D, B[1], Vk1, Hb, m=30, tol=1e-10)
    assert info.converged
    x1 = np.linalg.solve(Dm, B[1])
    assert np.linalg.norm(x - x1) <= 1e-8 * np.linalg.norm(x1)
    # plain restarted GMRES(30) on the same right-hand side, for the count of products
    xp = np.zeros(n, dtype=complex)
    mv = 0
    for _ in range(1000):
        res = B[1] - D(xp)
        mv += 1
        if np.linalg.norm(res) <= 1e-10 * np.linalg.norm(B[1]):
            break
        dx, c = G.gmres_cycle(D, res, 30)
        xp = xp + dx
        mv += c
    assert info.mvps < mv
