"""Pins of the FP64 Krylov oracle (CG, MinRes, Lanczos, Lan-DR, MinRes-DR, D-CG, D-MinRes).

Each routine is checked against something other than itself: brute-force
optimality over an explicit Krylov basis, exact eigenvalues of the paper's
diagonal examples (Sec. 1), the facts the paper states about them
(tests/golden/paper_sec1_examples.json), dense LAPACK eigensolves of a small
Wilson matrix, direct solves, and the exact-arithmetic equivalences
(one Lan-DR cycle = CG, one MinRes-DR cycle = MinRes).
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import krylov as K
from oracle import wilson

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_sec1_examples.json")))


def _rand_herm(n, eigs, seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return (q * eigs) @ q.conj().T


def _krylov_basis(A, b, j):
    """Orthonormal basis of span{b, Ab, ..., A^(j-1) b} by dense Arnoldi with full
    Gram-Schmidt (twice), which spans the Krylov space stably."""
    Q = [b / np.linalg.norm(b)]
    while len(Q) < j:
        w = A @ Q[-1]
        for _ in range(2):
            for q in Q:
                w = w - np.vdot(q, w) * q
        Q.append(w / np.linalg.norm(w))
    return np.stack(Q, axis=1)


def test_cg_iterate_is_the_A_norm_minimiser():
    n = 40
    A = _rand_herm(n, np.linspace(1.0, 6.0, n), seed=1)
    b = np.random.default_rng(2).standard_normal(n) + 0j
    xs = np.linalg.solve(A, b)
    for j in range(1, 9):
        x, info = K.cg(lambda v: A @ v, b, tol=0.0, maxiter=j)
        Kj = _krylov_basis(A, b, j)
        xb = Kj @ np.linalg.solve(Kj.conj().T @ A @ Kj, Kj.conj().T @ b)
        assert np.linalg.norm(x - xb) <= 1e-10 * np.linalg.norm(xs)


def test_minres_iterate_is_the_residual_minimiser():
    n = 40
    eigs = np.concatenate([np.linspace(-3, -0.5, 10), np.linspace(0.7, 5, 30)])
    A = _rand_herm(n, eigs, seed=3)
    b = np.random.default_rng(4).standard_normal(n) + 1j
    for j in range(1, 9):
        x, info = K.minres(lambda v: A @ v, b, tol=0.0, maxiter=j)
        Kj = _krylov_basis(A, b, j)
        c, *_ = np.linalg.lstsq(A @ Kj, b, rcond=None)
        xb = Kj @ c
        assert np.linalg.norm(x - xb) <= 1e-10 * np.linalg.norm(b)
        assert abs(info.residuals[-1] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-12


def test_cgnr_matches_cg_on_normal_equations():
    n = 30
    rng = np.random.default_rng(5)
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 6 * np.eye(n)
    b = rng.standard_normal(n) + 0j
    x1, i1 = K.cgnr(lambda v: M @ v, lambda v: M.conj().T @ v, b, tol=1e-12)
    assert np.linalg.norm(M @ x1 - b) / np.linalg.norm(b) < 1e-11
    assert abs(i1.residuals[-1] - i1.true_residual) < 1e-12


def _diag_op(d):
    return lambda x: d * x


def test_paper_hpd_example_minres_slightly_faster_than_cg():
    g = GOLD["hpd_diagonal"]
    d = synth.diag_hpd_1000()
    assert d.size == g["n"] and d[0] == 0.1 and d[-1] == 999.0
    b = np.ones(g["n"], dtype=complex) / np.sqrt(g["n"])
    _, ic = K.cg(_diag_op(d), b, tol=1e-10)
    _, im = K.minres(_diag_op(d), b, tol=1e-10)
    rc, rm = np.array(ic.residuals), np.array(im.residuals)
    k = min(len(rc), len(rm))
    assert np.all(rm[:k] <= rc[:k] * (1 + 1e-10))          # minimal residual property
    assert im.iterations <= ic.iterations <= im.iterations * 1.2   # "slightly faster"
    assert ic.true_residual < 1e-10 and im.true_residual < 1e-10


def test_paper_indefinite_example():
    g = GOLD["indefinite_diagonal"]
    d, seed = synth.diag_indefinite_1000(g["negatives"])
    assert int((d < 0).sum()) == g["negatives"]
    b = np.ones(g["n"], dtype=complex) / np.sqrt(g["n"])
    _, ic = K.cg(_diag_op(d), b, tol=1e-10, maxiter=5000)
    _, im = K.minres(_diag_op(d), b, tol=1e-10, maxiter=5000)
    rc, rm = np.array(ic.residuals), np.array(im.residuals)
    assert ic.converged and im.converged
    assert im.iterations < ic.iterations                    # MinRes slightly outperforms CG
    assert np.sum(np.diff(rc) > 0) > 20                     # spiked CG residual curve
    assert np.all(np.diff(rm) <= 1e-15 * rm[:-1])           # MinRes residual is monotone
    # deflation knee: where the 25-step log-slope first exceeds 3x the slope on [50, 100]
    ls = np.log10(rm)
    base = (ls[100] - ls[50]) / 50
    knee = next(j for j in range(50, len(ls) - 25) if (ls[j + 25] - ls[j]) / 25 < 3 * base)
    assert 100 <= knee <= 200, knee                          # "after about 125 iterations"
    assert (ls[300] - ls[200]) / 100 < 10 * base             # super-linear afterwards


def test_lanczos_relation_and_orthogonality():
    d = np.linspace(0.5, 20, 300)
    b = np.random.default_rng(1).standard_normal(300) + 0j
    Vm, T, beta0 = K.lanczos(_diag_op(d), b, 40, full_reorth=True)
    assert np.abs(d[:, None] * Vm[:, :40] - Vm @ T).max() < 1e-12 * 20
    assert np.abs(Vm.conj().T @ Vm - np.eye(41)).max() < 1e-12
    assert np.all(np.triu(T, 2) == 0) and np.all(np.tril(T, -2) == 0)
    assert np.all(np.diag(T, -1) > 0)
    # extreme Ritz values approach the extreme eigenvalues
    th = np.linalg.eigvalsh(T[:40, :40])
    assert 20 - 0.05 < th[-1] <= 20 + 1e-12 and th[0] > 0.5 - 1e-12


def test_lanczos_breakdown_on_few_distinct_eigenvalues():
    d = np.repeat([1.0, 2.0, 5.0], 50)
    b = np.ones(150, dtype=complex)
    with pytest.raises(K.LanczosBreakdown) as e:
        K.lanczos(_diag_op(d), b, 10)
    assert e.value.j == 2


def test_one_landr_cycle_is_cg_and_one_minresdr_cycle_is_minres():
    d = np.linspace(0.2, 30, 400)
    b = np.random.default_rng(8).standard_normal(400) + 0j
    m = 25
    r = K.landr(_diag_op(d), b, m=m, k=5, tol=0.0, max_cycles=1, full_reorth=True)
    x_cg, _ = K.cg(_diag_op(d), b, tol=0.0, maxiter=m)
    assert np.linalg.norm(r.x - x_cg) < 1e-10 * np.linalg.norm(x_cg)
    r = K.minresdr(_diag_op(d), b, m=m, k=5, tol=0.0, max_cycles=1, full_reorth=True)
    x_mr, _ = K.minres(_diag_op(d), b, tol=0.0, maxiter=m)
    assert np.linalg.norm(r.x - x_mr) < 1e-10 * np.linalg.norm(x_mr)


@pytest.mark.parametrize("method", ["landr", "minresdr"])
def test_dr_on_paper_hpd_example_finds_lowest_eigenvalues(method):
    d = synth.diag_hpd_1000()
    b = np.ones(1000, dtype=complex) / np.sqrt(1000)
    r = getattr(K, method)(_diag_op(d), b, m=40, k=10, tol=1e-10)
    assert r.info.converged
    assert r.info.true_residual <= 1e-10
    assert np.linalg.norm(r.x - b / d) <= 1e-9 * np.linalg.norm(b / d)
    exact = np.sort(d)[:10]
    assert np.all(np.abs(np.sort(r.ritz_values) - exact) <= 1e-8 * exact)
    assert np.abs(r.Vk.conj().T @ r.Vk - np.eye(10)).max() < 1e-12


@pytest.mark.parametrize("m,k", [(40, 10), (200, 150)])
def test_landr_as_eigensolver_on_paper_hpd_example(m, k):
    """Eigensolver use (Sec. 2's k = 150 with m = 200 included): the linear tolerance
    is unreachable (1e-30), so only the kept pairs can stop the cycles; all k Ritz
    values must be the k smallest eigenvalues 0.1, 1, 2, ... of the Sec. 1 example."""
    d = synth.diag_hpd_1000()
    b = np.ones(1000, dtype=complex) / np.sqrt(1000)
    r = K.landr(_diag_op(d), b, m=m, k=k, tol=1e-30, tol_eig=1e-9, max_cycles=2000, eig_only=True)
    assert r.info.converged
    exact = np.sort(d)[:k]
    assert np.all(np.abs(np.sort(r.ritz_values) - exact) <= 1e-8 * exact)
    assert np.all(r.ritz_residuals <= 1e-10 * d.max())       # ||A|| = 999
    assert np.abs(r.Vk.conj().T @ r.Vk - np.eye(k)).max() < 1e-8


def test_minresdr_as_eigensolver_on_paper_indefinite_example():
    d, _ = synth.diag_indefinite_1000()
    b = np.ones(1000, dtype=complex) / np.sqrt(1000)
    r = K.minresdr(_diag_op(d), b, m=40, k=10, tol=1e-30, tol_eig=1e-9, max_cycles=2000, eig_only=True)
    assert r.info.converged
    exact = d[np.argsort(np.abs(d))[:10]]
    assert np.all(np.abs(np.sort(r.ritz_values) - np.sort(exact)) <= 1e-8 * np.abs(np.sort(exact)))


def test_minresdr_on_paper_indefinite_example():
    d, _ = synth.diag_indefinite_1000()
    b = np.ones(1000, dtype=complex) / np.sqrt(1000)
    r = K.minresdr(_diag_op(d), b, m=40, k=10, tol=1e-10)
    assert r.info.converged and r.info.true_residual <= 1e-10
    hist = np.array(r.info.residuals)
    assert np.all(np.diff(hist) <= 1e-14)                  # residual non-increasing over cycles
    exact = d[np.argsort(np.abs(d))[:10]]
    got = np.sort(r.ritz_values)
    ok = r.ritz_residuals <= 1e-6
    vals = np.sort(r.ritz_values[ok])
    for v in vals:
        assert np.min(np.abs(exact - v) / np.abs(exact)) <= 1e-8
    assert ok.sum() >= 8
    assert np.all(np.abs(got) < 0.1)


def test_deflated_solves_match_direct_and_beat_undeflated():
    d, _ = synth.diag_indefinite_1000()
    b1 = np.ones(1000, dtype=complex) / np.sqrt(1000)
    r = K.minresdr(_diag_op(d), b1, m=40, k=10, tol=1e-10)
    H = K.deflation_space(_diag_op(d), r.Vk)
    b2 = np.random.default_rng(9).standard_normal(1000) + 0j
    x, info = K.dminres(_diag_op(d), b2, r.Vk, H, tol=1e-10)
    _, info0 = K.minres(_diag_op(d), b2, tol=1e-10)
    assert info.true_residual <= 1e-10
    assert np.linalg.norm(x - b2 / d) <= 1e-10 * np.abs(1 / d).max() * np.linalg.norm(b2)
    assert info.iterations < 0.8 * info0.iterations
    # D-CG through the normal equations of a non-hermitian M with the same kept space idea
    dp = np.sqrt(synth.diag_hpd_1000())
    r2 = K.landr(_diag_op(dp * dp), dp * b1, m=40, k=10, tol=1e-10,
                 residual=lambda xx: np.linalg.norm(b1 - dp * xx) / np.linalg.norm(b1))
    H2 = K.deflation_space(_diag_op(dp * dp), r2.Vk)
    x2, i2 = K.dcg(_diag_op(dp), _diag_op(dp), b2, r2.Vk, H2, tol=1e-10)
    _, i20 = K.cgnr(_diag_op(dp), _diag_op(dp), b2, tol=1e-10)
    assert i2.true_residual <= 1e-10 and i2.iterations < 0.8 * i20.iterations


def _harmonic_ritz_vectors(A, Kb, k):
    """k harmonic Ritz vectors of span(Kb) for target 0: (AK)^H (AK) g = theta (AK)^H K g."""
    import scipy.linalg as sla
    AK = A @ Kb
    th, G = sla.eig(AK.conj().T @ AK, AK.conj().T @ Kb)
    return Kb @ G[:, np.argsort(np.abs(th))[:k]]


def _ritz_vectors(A, Kb, k):
    th, G = np.linalg.eigh(Kb.conj().T @ A @ Kb)
    return Kb @ G[:, np.argsort(th)[:k]]


@pytest.mark.parametrize("method", ["landr", "minresdr"])
def test_second_cycle_equals_brute_force_augmented_projection(method):
    """Cycle 2 of Lan-DR / MinRes-DR = Galerkin / minimum-residual projection over
    span{k (harmonic) Ritz vectors of cycle 1, r1, A r1, ..., A^(m-k-1) r1} (FOM-DR / GMRES-DR)."""
    n, m, k = 300, 20, 5
    if method == "landr":
        d = np.linspace(0.01, 5, n)
    else:
        d = np.concatenate([np.linspace(-2, -0.01, 20), np.linspace(0.02, 5, n - 20)])
    A = np.diag(d).astype(complex)
    b = np.random.default_rng(0).standard_normal(n) + 0.5j
    f = getattr(K, method)
    x1 = f(lambda v: d * v, b, m=m, k=k, tol=0, max_cycles=1, full_reorth=True).x
    x2 = f(lambda v: d * v, b, m=m, k=k, tol=0, max_cycles=2, full_reorth=True).x
    Kb = _krylov_basis(A, b, m)
    Y = (_harmonic_ritz_vectors if method == "minresdr" else _ritz_vectors)(A, Kb, k)
    r1 = b - d * x1
    S, _ = np.linalg.qr(np.hstack([Y, _krylov_basis(A, r1, m - k)]))
    if method == "landr":
        xb = x1 + S @ np.linalg.solve(S.conj().T @ A @ S, S.conj().T @ r1)
    else:
        c, *_ = np.linalg.lstsq(A @ S, r1, rcond=None)
        xb = x1 + S @ c
    assert np.linalg.norm(x2 - xb) <= 1e-8 * np.linalg.norm(xb)


@pytest.fixture(scope="module")
def wilson4():
    """4^4 Wilson lattice (gauge seed 1) at kappa = 0.2: a quick dense check case."""
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 1)
    kappa = 0.2
    n = synth.volume(dims) * 12
    Q = wilson.dense(wilson.operator(U, kappa, dims, "Q"), n)
    return dims, U, kappa, np.linalg.eigvalsh(Q)


def _check_ritz_against_spectrum(vals, res, ev, lowest_first):
    """Every Ritz pair (value, residual) against the exact spectrum ev (sorted):
    an eigenvalue lies within the residual, and the best-converged value obeys
    the Kato-Temple bound |theta - lambda| <= res^2 / gap."""
    for v, r in zip(vals, res):
        assert np.min(np.abs(ev - v)) <= r * (1 + 1e-9) + 1e-13
    i = int(np.argmin(res))
    j = int(np.argmin(np.abs(ev - vals[i])))
    gap = np.min(np.abs(np.delete(ev, j) - vals[i]))
    assert abs(vals[i] - ev[j]) <= res[i] ** 2 / gap * (1 + 1e-6) + 1e-14
    assert abs(vals[i] - ev[j]) <= 1e-8 * abs(ev[j])


def test_wilson_4x4x4x4_dr_ritz_pairs_against_dense_eigensolve(wilson4):
    """Lan-DR on D^dagger D and MinRes-DR on Q against LAPACK on the dense matrix."""
    dims, U, kappa, ev = wilson4
    b = synth.gaussian_spinor(dims, 0).reshape(-1)
    m, k = 40, 10
    Aq = wilson.operator(U, kappa, dims, "Q")
    bg = wilson.apply_gamma5(b.reshape(-1, 4, 3)).reshape(-1)
    r = K.minresdr(Aq, bg, m=m, k=k, tol=1e-10, max_cycles=400, oversolve=2.0)
    assert r.info.converged and r.info.true_residual <= 1e-10
    _check_ritz_against_spectrum(r.ritz_values, r.ritz_residuals, ev, lowest_first=False)
    Ad = wilson.operator(U, kappa, dims, "DdagD")
    D = wilson.operator(U, kappa, dims, "D")
    Dd = wilson.operator(U, kappa, dims, "Ddag")
    bn = np.linalg.norm(b)
    r2 = K.landr(Ad, Dd(b), m=m, k=k, tol=1e-10, max_cycles=400, oversolve=2.0,
                 residual=lambda xx: np.linalg.norm(b - D(xx)) / bn)
    assert r2.info.converged and r2.info.true_residual <= 1e-10
    ev2 = np.sort(ev ** 2)
    _check_ritz_against_spectrum(r2.ritz_values, r2.ritz_residuals, ev2, lowest_first=True)
    # Cauchy interlacing: the i-th smallest Ritz value is >= the i-th smallest eigenvalue
    assert np.all(np.sort(r2.ritz_values) >= ev2[:k] - 1e-13)
    # deflated follow-up solves: same x as the undeflated solve, fewer iterations
    for seed in (1, 2):
        bb = synth.gaussian_spinor(dims, seed).reshape(-1)
        bbg = wilson.apply_gamma5(bb.reshape(-1, 4, 3)).reshape(-1)
        x0, i0 = K.minres(Aq, bbg)
        x, info = K.dminres(Aq, bbg, r.Vk, K.deflation_space(Aq, r.Vk))
        cond = np.abs(ev).max() / np.abs(ev).min()
        assert info.true_residual <= 1e-10 and info.iterations < i0.iterations
        assert np.linalg.norm(x - x0) <= cond * 2e-10 * np.linalg.norm(x0)
        x2, info2 = K.dcg(D, Dd, bb, r2.Vk, K.deflation_space(Ad, r2.Vk))
        _, i20 = K.cgnr(D, Dd, bb)
        assert info2.true_residual <= 1e-10 and info2.iterations < i20.iterations
        assert np.linalg.norm(x2 - x0) <= cond * 2e-10 * np.linalg.norm(x0)


def test_kappa_rule_holds_on_the_4x4x4x4_workload():
    import scipy.linalg as sla
    w = synth.WORKLOADS["wilson_4x4x4x4"]
    dims = w["dims"]
    U = synth.su3_links(dims, w["gauge_seed"])
    kappa = synth.kappa_for(dims, w["gauge_seed"])
    n = synth.volume(dims) * 12
    D = wilson.dense(wilson.operator(U, kappa, dims, "D"), n)
    lam = sla.eigvalsh(D.conj().T @ D, subset_by_index=[0, 0])[0]
    assert abs(np.sqrt(lam) / 1e-3 - 1) < 1e-5


def test_kappa_verification_agrees_with_the_dense_eigensolve():
    """The independent re-verification of a stored kappa (a cold-started MinRes-DR
    eigensolve of gamma5 D) on the 4^4 workload: its |rho| lies within its own
    Kato-Temple bound of the dense min |eig(gamma5 D)|, and within the residual."""
    from oracle import kappa as okappa
    w = synth.WORKLOADS["wilson_4x4x4x4"]
    dims = w["dims"]
    U = synth.su3_links(dims, w["gauge_seed"])
    kappa = synth.kappa_for(dims, w["gauge_seed"])
    v = okappa.verify_sigma(U, kappa, dims, seed=99, rel_bound=1e-2, max_cycles=300)
    n = synth.volume(dims) * 12
    ev = np.linalg.eigvalsh(wilson.dense(wilson.operator(U, kappa, dims, "Q"), n))
    exact = np.min(np.abs(ev))
    assert abs(v["sigma"] - exact) <= v["bound"] + 1e-15
    assert abs(v["sigma"] - exact) <= v["residual"]
    assert v["bound"] <= 1e-2 * v["sigma"] and abs(exact / 1e-3 - 1) < 1e-5


def test_iterative_kappa_searches_find_the_dense_crossing():
    """The two searches used past dense size (Illinois on MinRes-DR eigensolves, and
    Newton inside a bracket) run on the 4^4 workload, where the dense eigensolve gives
    the crossing exactly: each returns a kappa whose dense sigma_min meets the rule
    to its tolerance, and a sigma that is the dense one at that kappa to within the
    search's own error estimate."""
    from oracle import kappa as okappa
    w = synth.WORKLOADS["wilson_4x4x4x4"]
    dims = w["dims"]
    U = synth.su3_links(dims, w["gauge_seed"])
    H = okappa._dense_hop(U, dims)
    a, b = 0.2582, 0.2586
    sa, sb = okappa.sigma_min_dense(H, a), okappa.sigma_min_dense(H, b)
    assert sa > 1e-3 > sb
    kap, sig, res, bound, hist = okappa.kappa_newton(U, dims, a, sa, b, sb, rtol=5e-2)
    exact = okappa.sigma_min_dense(H, kap)
    assert abs(exact / 1e-3 - 1) < 5e-2 and abs(sig - exact) <= bound + 1e-15
    assert a < kap < b and hist[-1]["kappa"] == kap
    kap2, sig2, res2 = okappa.kappa_iterative(U, dims, start=0.2583, step=0.0003, rtol=5e-2,
                                              res_tol=1e-4, max_cycles=200)
    exact2 = okappa.sigma_min_dense(H, kap2)
    assert abs(exact2 / 1e-3 - 1) < 5e-2 and abs(sig2 - exact2) <= res2
    # both within the Illinois-refined dense crossing's neighbourhood
    kd = synth.kappa_for(dims, w["gauge_seed"])
    assert abs(kap - kd) < 1e-4 and abs(kap2 - kd) < 1e-4


def test_kappa_rule_free_field_limit():
    """At U = 1 the first crossing of sigma_min = 1e-3 is kappa = (1 - 1e-3)/8."""
    from oracle import kappa as okappa
    dims = (2, 2, 2, 2)
    kap, sig = okappa.kappa_dense(synth.unit_links(dims), dims)
    assert abs(kap - (1 - 1e-3) / 8) < 1e-9
    assert abs(sig / 1e-3 - 1) < 1e-6


def test_landr_past_convergence_keeps_an_orthonormal_positive_kept_space():
    """Lan-DR(40,10) on the 4^4 Wilson D^dag D run 150 cycles, long past linear
    convergence (the over-solve): the kept regular Ritz vectors converge to rounding
    level, and the kept space must stay orthonormal (to 1e-13) with the exact lowest
    eigenvalues.  (Re-orthogonalising only every 10 steps leaves a 1.8e-12 overlap
    here, and on 8^4 with Lan-DR(100,40) gives negative Ritz values after 12 cycles.)"""
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 1)
    A = wilson.operator(U, 0.25, dims, "DdagD")
    Dd = wilson.operator(U, 0.25, dims, "Ddag")
    b = synth.gaussian_spinor(dims, 0).reshape(-1)
    r = K.landr(A, Dd(b), m=40, k=10, tol=1e-10, tol_eig=1e-300, oversolve=50.0, max_cycles=150)
    G = r.Vk.conj().T @ r.Vk
    assert np.abs(G - np.eye(10)).max() <= 1e-13
    exact = np.linalg.eigvalsh(wilson.dense(A, 3072))[:10]
    assert np.allclose(np.sort(r.ritz_values), exact, rtol=1e-8)


def test_landr_refuses_a_reorthogonalisation_period_it_would_not_honour():
    d = synth.diag_hpd_1000()
    b = np.ones(1000, dtype=complex) / np.sqrt(1000)
    with pytest.raises(ValueError):
        K.landr(_diag_op(d), b, m=20, k=5, reorth_period=10, max_cycles=1)
    r = K.landr(_diag_op(d), b, m=20, k=5, reorth_period=0, max_cycles=1)   # off is allowed
    assert r.cycles == 1
