"""GMRES-DR and D-GMRES for the non-hermitian Wilson matrix D itself, FP64 NumPy oracle
(test infrastructure only).

The paper contrasts its hermitian methods with the non-hermitian deflated methods of
its refs. [1] and [2] (GMRES-DR for the first right-hand side, a deflated GMRES for
the others) and defines neither here; the readings below are the standard forms.

GMRES-DR(m, k) for A x = b (A non-hermitian):
  1. r0 = b, beta = ||r0||, v_1 = r0 / beta, c = beta e_1.
  2. Arnoldi with full Gram-Schmidt (twice) to j = m: A V_m = V_{m+1} Hbar_m,
     Hbar_m ((m+1) x m, complex) upper Hessenberg after the restart block.
  3. y = argmin ||c - Hbar_m y||, x += V_m y, s = c - Hbar_m y (the residual is V_{m+1} s).
  4. Harmonic Ritz pairs: (H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^H) g = theta g; keep the
     k of smallest |theta|.
  5. P_{k+1} = orthonormalise([[G_k; 0], q]) (modified Gram-Schmidt twice, q last), q the
     unit vector spanning range(Hbar_m)^perp (parallel to s, from the complete QR);
     V_{k+1} <- V_{m+1} P_{k+1}, Hbar_k <- P_{k+1}^H Hbar_m P_k ((k+1) x k, full), c <- P^H s.
  6. Arnoldi continues from v_{k+1} against all previous vectors.
  Stop when ||b - A x|| / ||b|| <= tol (checked once per cycle).  The kept space carries
  A V_k = V_{k+1} Hbar_k, which the later right-hand sides use.

D-GMRES(m) over that space for each later right-hand side: from x = 0, repeat
  (a) minimum-residual projection over span(V_k): y = argmin ||V_{k+1}^H r - Hbar_k y||
      (the least squares of ||r - A V_k y|| by the relation A V_k = V_{k+1} Hbar_k),
      x += V_k y, and r = b - A x recomputed;
  (b) one GMRES(m) cycle from r;
  until ||b - A x|| / ||b|| <= tol.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .krylov import SolveInfo, _norm


def _arnoldi(A, V, H, j0, m):
    """Extend an Arnoldi relation A V[:, :j] = V[:, :j+1] H[:j+1, :j] from j0 to m columns
    (full Gram-Schmidt, applied twice).  V is (n, m+1), H is (m+1, m); returns the MVPs."""
    for j in range(j0, m):
        w = A(V[:, j])
        for _ in range(2):
            h = V[:, : j + 1].conj().T @ w
            w = w - V[:, : j + 1] @ h
            H[: j + 1, j] += h
        H[j + 1, j] = _norm(w)
        if H[j + 1, j] == 0.0:
            raise ZeroDivisionError("Arnoldi breakdown")
        V[:, j + 1] = w / H[j + 1, j]
    return m - j0


def _mgs(P):
    """Orthonormalise the columns of P left to right (modified Gram-Schmidt, twice)."""
    Q = np.array(P, dtype=np.complex128, copy=True)
    for j in range(Q.shape[1]):
        for _ in range(2):
            for i in range(j):
                Q[:, j] -= np.vdot(Q[:, i], Q[:, j]) * Q[:, i]
        Q[:, j] /= np.linalg.norm(Q[:, j])
    return Q


def harmonic_ritz(Hbar, m, k):
    """The k harmonic Ritz pairs of smallest |theta| of an (m+1) x m Arnoldi matrix:
    eigenpairs of H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^H (theta ascending in |theta|,
    unit vectors g).
    (The paper's refs. [1], [2]: the non-hermitian deflated methods Sec. 1 contrasts
    with.)"""
    Hm = Hbar[:m, :m]
    em = np.zeros(m, dtype=np.complex128)
    em[m - 1] = 1.0
    f = np.linalg.solve(Hm.conj().T, em)
    B = Hm + abs(Hbar[m, m - 1]) ** 2 * np.outer(f, em)
    theta, G = np.linalg.eig(B)
    order = np.argsort(np.abs(theta), kind="stable")[:k]
    G = G[:, order]
    return theta[order], G / np.linalg.norm(G, axis=0)


@dataclass
class GmresDRResult:
    x: np.ndarray
    V: np.ndarray              # n x (k+1): V_{k+1} of the last restart
    Hbar: np.ndarray           # (k+1) x k: A V_k = V_{k+1} Hbar
    theta: np.ndarray          # the kept harmonic Ritz values
    info: SolveInfo
    cycles: int = 0


def gmresdr(A, b, m, k, tol=1e-10, max_cycles=500, progress=None):
    """GMRES-DR(m, k) for A x = b (module docstring), x0 = 0.
    (The paper's refs. [1], [2]: the non-hermitian deflated methods Sec. 1 contrasts
    with.)"""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    n = b.size
    bn = _norm(b)
    info = SolveInfo()
    x = np.zeros(n, dtype=np.complex128)
    V = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    V[:, 0] = b / bn
    c = np.zeros(m + 1, dtype=np.complex128)
    c[0] = bn
    j0 = 0
    theta = None
    cycles = 0
    for cycle in range(max_cycles):
        cycles += 1
        info.mvps += _arnoldi(A, V, H, j0, m)
        y, *_ = np.linalg.lstsq(H, c, rcond=None)
        x = x + V[:, :m] @ y
        s = c - H @ y
        rel = _norm(b - A(x)) / bn
        info.mvps += 1
        info.residuals.append(rel)
        if progress is not None:
            progress(cycle, info.mvps, rel)
        theta, G = harmonic_ritz(H, m, k)
        # s is orthogonal to range(Hbar_m); its direction is taken from the complete QR
        # of Hbar_m (phase matched to s) so that it stays exact when ||s|| is tiny
        q = np.linalg.qr(H, mode="complete")[0][:, m]
        ph = np.vdot(q, s)
        if abs(ph) > 0:
            q = q * (ph / abs(ph))
        P = _mgs(np.hstack([np.vstack([G, np.zeros((1, k))]), q[:, None]]))
        Vn = V @ P
        Hk = P.conj().T @ H @ P[:m, :k]
        cn = P.conj().T @ s
        V = np.zeros((n, m + 1), dtype=np.complex128)
        V[:, : k + 1] = Vn
        H = np.zeros((m + 1, m), dtype=np.complex128)
        H[: k + 1, :k] = Hk
        c = np.zeros(m + 1, dtype=np.complex128)
        c[: k + 1] = cn
        j0 = k
        if rel <= tol:
            info.converged = True
            break
    info.iterations = info.mvps
    info.true_residual = info.residuals[-1]
    return GmresDRResult(x=x, V=V[:, : k + 1].copy(), Hbar=H[: k + 1, :k].copy(), theta=theta, info=info,
                         cycles=cycles)


def gmres_cycle(A, r, m):
    """One GMRES(m) cycle from residual r: the correction minimising ||r - A dx|| over the
    Krylov space of dimension m (returns dx and the MVPs).
    (The paper's refs. [1], [2]: the non-hermitian deflated methods Sec. 1 contrasts
    with.)"""
    n = r.size
    beta = _norm(r)
    V = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    V[:, 0] = r / beta
    mv = _arnoldi(A, V, H, 0, m)
    c = np.zeros(m + 1, dtype=np.complex128)
    c[0] = beta
    y, *_ = np.linalg.lstsq(H, c, rcond=None)
    return V[:, :m] @ y, mv


def dgmres(A, b, Vk1, Hbar, m, tol=1e-10, max_cycles=1000):
    """D-GMRES(m) over the kept space (V_{k+1}, Hbar_k) of GMRES-DR (module docstring).
    (The paper's refs. [1], [2]: the non-hermitian deflated methods Sec. 1 contrasts
    with.)"""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    bn = _norm(b)
    info = SolveInfo()
    k = Hbar.shape[1]
    x = np.zeros_like(b)
    r = b.copy()
    for cycle in range(max_cycles):
        y, *_ = np.linalg.lstsq(Hbar, Vk1.conj().T @ r, rcond=None)
        x = x + Vk1[:, :k] @ y
        r = b - A(x)
        info.mvps += 1
        if _norm(r) / bn <= tol:
            info.converged = True
            break
        dx, mv = gmres_cycle(A, r, m)
        info.mvps += mv
        x = x + dx
        r = b - A(x)
        info.mvps += 1
        info.residuals.append(_norm(r) / bn)
        if info.residuals[-1] <= tol:
            info.converged = True
            break
    info.iterations = info.mvps
    info.true_residual = _norm(b - A(x)) / bn
    return x, info
