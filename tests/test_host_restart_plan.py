"""The host small problem of a restart cycle (dlz_host_restart_plan, the code the GPU
solvers run between cycles) against the oracle's restart_plan on the same Tbar and c,
taken from every cycle of oracle Lan-DR / MinRes-DR runs (Sec. 1-2).

Eigenvectors are compared through what is unique: the projector onto span(P), the
singular values of the new Tbar block and |c|; values and residuals elementwise after
sorting.  Tolerances: eps-level perturbation bounds, ~1e3 eps ||T|| for values, looser
for subspaces (angle ~ eps ||T|| / gap at the cut; cycles whose cut gap is below 1e-6
are compared by values only)."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import krylov as K
from oracle import wilson
from tests._lib import dlz


def _collect(case):
    recs = []

    def hook(T, c, pl):
        recs.append((T.copy(), c.copy(), {key: np.array(v, copy=True) if isinstance(v, np.ndarray) else v
                                          for key, v in pl.__dict__.items()}))

    if case.startswith("wilson"):
        dims = (4, 4, 4, 4)
        U = synth.su3_links(dims, 1)
        Q = wilson.operator(U, 0.2, dims, "Q")
        b = synth.gaussian_spinor(dims, 0).reshape(-1)
        m, k = 30, 8
        if case == "wilson_minresdr":
            K.minresdr(Q, b, m, k, tol=1e-10, max_cycles=8, plan_hook=hook)
        else:
            K.landr(lambda v: Q(Q(v)), b, m, k, tol=1e-10, max_cycles=8, plan_hook=hook)
    else:
        m, k = 40, 10
        b = np.ones(1000, dtype=complex) / np.sqrt(1000)
        if case == "hpd_diag_landr":
            d = synth.diag_hpd_1000()
            K.landr(lambda v: d * v, b, m, k, tol=1e-10, max_cycles=60, oversolve=2.0, plan_hook=hook)
        else:
            d, _ = synth.diag_indefinite_1000(22)
            K.minresdr(lambda v: d * v, b, m, k, tol=1e-10, max_cycles=60, oversolve=2.0, plan_hook=hook)
    return recs, m, k, case.endswith("minresdr")


def _cut_gap(T, m, k, harmonic):
    """Relative gap between the k-th kept and the first dropped value."""
    Tm = T[:m, :m]
    if harmonic:
        mu = np.sort(np.abs(sla.eigh(Tm, T.T @ T, eigvals_only=True)))[::-1]
        return (mu[k - 1] - mu[k]) / mu[0]
    ev = np.linalg.eigvalsh(Tm)
    return (ev[k] - ev[k - 1]) / np.abs(ev).max()


@pytest.mark.parametrize("case", ["wilson_minresdr", "wilson_landr", "hpd_diag_landr", "indefinite_diag_minresdr"])
def test_host_restart_plan_matches_oracle(case):
    m_ = dlz()
    recs, m, k, harmonic = _collect(case)
    assert len(recs) >= 6
    for T, c, o in recs:
        g = m_.host_restart_plan(T, c, k, harmonic)
        sc = np.abs(T).max()
        # linear-system coefficients (Galerkin or least squares)
        assert np.abs(g["y"] - o["y"]).max() <= 1e-10 * np.abs(o["y"]).max()
        # kept (harmonic) Ritz values and residuals
        assert np.abs(np.sort(g["theta"]) - np.sort(o["theta"])).max() <= 1e-12 * sc
        assert np.abs(np.sort(g["ritz_res"]) - np.sort(o["ritz_res"])).max() <= 1e-12 * sc
        # ||A|| estimate: max |eig T_m|
        an = np.abs(np.linalg.eigvalsh(T[:m, :m])).max()
        assert abs(g["anorm"] - an) <= 1e-13 * an
        # restart matrix: orthonormal columns; its span; the new Tbar and c
        P = g["P"]
        assert np.abs(P.T @ P - np.eye(k + 1)).max() < 1e-13
        Tn = g["Tn"]
        assert np.all(Tn[k + 1:, :] == 0) and np.all(Tn[:, k:] == 0)
        assert np.all(g["cn"][k + 1:] == 0)
        if not harmonic:
            assert np.array_equal(Tn[:k, :k], np.diag(np.diag(Tn[:k, :k])))
        assert np.abs(Tn[:k, :k] - Tn[:k, :k].T).max() == 0
        so = np.linalg.svd(o["Tn"][:k + 1, :k], compute_uv=False)
        sg = np.linalg.svd(Tn[:k + 1, :k], compute_uv=False)
        assert np.abs(so - sg).max() <= 1e-12 * sc
        assert abs(np.linalg.norm(g["cn"]) - np.linalg.norm(o["cn"])) <= 1e-12 * np.linalg.norm(c)
        if _cut_gap(T, m, k, harmonic) > 1e-6:
            Po = o["P"]
            assert np.abs(P @ P.T - Po @ Po.T).max() <= 1e-9


def test_host_restart_plan_arguments():
    m_ = dlz()
    T = np.zeros((5, 4))
    c = np.zeros(5)
    for k in (0, 4):
        with pytest.raises(m_.DlzError):
            m_.host_restart_plan(T, c, k, True)
