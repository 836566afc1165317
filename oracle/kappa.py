"""The kappa rule of the synthetic workloads, FP64 oracle (test infrastructure only).

The paper runs at "essentially kappa critical" (kappa = 0.15720 on its
beta = 6.0 ensemble, Sec. 2).  The synthetic links have a different critical
point, so each synthetic lattice takes the kappa at which
min |eig(gamma5 D)| = sigma_min(D) = 1e-3:

  * lattices of at most 256 sites (dense): scan kappa upward from 0 in
    steps of 0.005 to the first kappa where sigma_min < 1e-3 (sigma_min^2 =
    lowest eigenvalue of D^dagger D from LAPACK), then refine inside that
    bracket by safeguarded false position (Illinois) to
    |sigma_min / 1e-3 - 1| < 1e-6;
  * larger lattices: sigma_min = min |eig(Q)| from MinRes-DR run as an
    eigensolver (the harmonic Ritz pair nearest zero), stepping by 0.003
    from a start value near the expected crossing to bracket it, then
    Illinois to 1e-3 and an independent re-verification.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import cwilson, wilson

TARGET = 1e-3


def _dense_hop(U, dims, bc_t=1):
    """Dense hopping matrix H with D(kappa) = 1 - kappa H (tiny lattices)."""
    n = int(np.prod(dims)) * 12
    D1 = wilson.dense(wilson.operator(U, 1.0, dims, "D", bc_t), n)
    return np.eye(n) - D1


def sigma_min_dense(H, kappa):
    """sigma_min(1 - kappa H) from the lowest eigenvalue of D^dagger D (LAPACK)."""
    D = np.eye(H.shape[0]) - kappa * H
    lam = sla.eigvalsh(D.conj().T @ D, subset_by_index=[0, 0])[0]
    return float(np.sqrt(max(lam, 0.0)))


def _illinois(f, a, fa, b, fb, rtol):
    """Safeguarded false position on a bracket [a, b] with f(a) > 0 > f(b)."""
    side = 0
    for _ in range(200):
        c = b - fb * (b - a) / (fb - fa)
        if not (min(a, b) < c < max(a, b)):
            c = 0.5 * (a + b)
        fc = f(c)
        if abs(fc) < rtol * TARGET:
            return c
        if fc > 0:
            a, fa = c, fc
            if side == -1:
                fb *= 0.5
            side = -1
        else:
            b, fb = c, fc
            if side == 1:
                fa *= 0.5
            side = 1
    raise RuntimeError("kappa refinement did not converge")


def kappa_dense(U, dims, bc_t=1, step=0.005, rtol=1e-6):
    """kappa with sigma_min(D) = 1e-3 on a lattice small enough to be dense."""
    H = _dense_hop(U, dims, bc_t)
    f = lambda kap: sigma_min_dense(H, kap) - TARGET  # noqa: E731
    a, fa = 0.0, f(0.0)
    while True:
        b = a + step
        fb = f(b)
        if fb < 0:
            break
        a, fa = b, fb
    kap = _illinois(f, a, fa, b, fb, rtol)
    return kap, sigma_min_dense(H, kap)


def sigma_min_iterative(U, kappa, dims, v0, res_tol, m=100, k=20, bc_t=1, max_cycles=2000,
                        log=None):
    """min |eig(gamma5 D)| by MinRes-DR used as an eigensolver (harmonic Ritz pairs
    nearest zero), started from v0.  Returns (sigma, eigenvector, residual, mvps)."""
    from .krylov import minresdr
    A = cwilson.operator(U, kappa, dims, "Q", bc_t)

    def progress(cycle, mvps, rel, theta, res):
        if log and cycle % 5 == 0:
            i = int(np.argmin(np.abs(theta)))
            log(f"   cycle {cycle} mvps {mvps} theta {abs(theta[i]):.6e} res {res[i]:.2e}")

    r = minresdr(A, v0, m, k, tol=0.0, max_cycles=max_cycles, eig_stop=res_tol, progress=progress)
    i = int(np.argmin(np.abs(r.ritz_values)))
    return (float(abs(r.ritz_values[i])), r.ritz_vectors[:, i], float(r.ritz_residuals[i]),
            r.info.mvps)


def kappa_iterative(U, dims, start, bc_t=1, step=0.003, rtol=1e-3, res_tol=1e-5, seed=12345,
                    log=None, max_cycles=2000):
    """kappa with sigma_min(D) = 1e-3 on a lattice too large for a dense eigensolve.

    sigma_min is min |eig(Q)|, taken from the harmonic Ritz pair nearest zero of
    MinRes-DR(100, 20) run as an eigensolver and warm-started from the previous
    eigenvector.  From `start` kappa is stepped by `step` (down while
    sigma_min < 1e-3, then up) to bracket the crossing, which is refined by
    Illinois false position to |sigma_min/1e-3 - 1| < rtol, and re-evaluated
    there.  Each eigensolve stops at a harmonic Ritz residual below
    max(res_tol, 5% of |sigma - 1e-3|) or after max_cycles restart cycles
    (the nearest-zero harmonic Ritz value of a capped run is then the
    estimate used).  Returns (kappa, sigma_min, residual of that estimate).
    """
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    state = {"v": rng.standard_normal(V * 12) + 1j * rng.standard_normal(V * 12)}

    def f(kap, res_tol=res_tol):
        # Far from the target only the sign and a rough size of sigma_min - 1e-3
        # are needed: stop once the residual is below 5% of that distance.
        def stop(theta, res):
            return res <= max(res_tol, 0.05 * abs(abs(theta) - TARGET))

        s, y, res, mv = sigma_min_iterative(U, kap, dims, state["v"], stop, bc_t=bc_t, log=log,
                                            max_cycles=max_cycles)
        state["res"] = res
        state["v"] = y + 1e-3 * (rng.standard_normal(V * 12) + 1j * rng.standard_normal(V * 12)) / np.sqrt(V * 12)
        if log:
            log(f"kappa={kap:.10f} sigma_min={s:.10e} res={res:.2e} mvps={mv}")
        return s - TARGET

    a = start
    fa = f(a)
    while fa < 0:
        a -= step
        fa = f(a)
    b = a + step
    fb = f(b)
    while fb > 0:
        a, fa = b, fb
        b = a + step
        fb = f(b)
    kap = _illinois(f, a, fa, b, fb, rtol)
    return kap, f(kap, res_tol) + TARGET, state["res"]
