"""Krylov methods of arXiv:0901.3163 in FP64 NumPy (test infrastructure only).

Operators are callables on flat complex128 vectors; inner products are
<u, v> = u^dagger v.  Every routine follows the textbook definition of the
method the paper names, written step by step:

  cg       -- conjugate gradient (Hestenes-Stiefel), the CG implementation of
              Lanczos (Sec. 1);
  cgnr     -- CG on the normal equations M^dagger M x = M^dagger b, tracking
              the residual of M x = b itself, as plotted in Sec. 2;
  minres   -- minimum residual (Paige-Saunders form) (Sec. 1);
  lanczos  -- the three-term Lanczos recurrence A V_m = V_{m+1} Tbar_m;
  landr    -- Lan-DR(m,k): restarted Lanczos, Galerkin (CG-type) solve, k
              regular Ritz vectors kept across restarts (Sec. 1, Sec. 2);
  minresdr -- MinRes-DR(m,k): restarted Lanczos, minimum-residual solve, k
              harmonic Ritz vectors kept across restarts (Sec. 1, Sec. 2);
  deflation_space, galerkin_x0, dcg, dminres -- the Galerkin projection over
              the k vectors at the start, then CG or MinRes (Sec. 2).

The paper leaves the detailed definition of the deflated methods to its
ref. [3]; the readings taken here are the standard thick-restart forms,
each listed in its docstring.  Small dense problems use numpy/scipy
(eigh, lstsq, solve, cholesky) as library steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


def _dot(u, v):
    return np.vdot(u, v)


def _norm(u):
    return float(np.sqrt(np.vdot(u, u).real))


@dataclass
class SolveInfo:
    converged: bool = False
    iterations: int = 0
    mvps: int = 0
    residuals: list = field(default_factory=list)   # relative residual history
    true_residual: float = float("nan")


# --------------------------------------------------------------------------
# CG and MinRes (Sec. 1)
# --------------------------------------------------------------------------

def cg(A, b, x0=None, tol=1e-10, maxiter=10000):
    """Conjugate gradient for hermitian positive definite A.

    r0 = b - A x0, p0 = r0; then alpha = <r,r>/<p,Ap>, x += alpha p,
    r -= alpha A p, beta = <r',r'>/<r,r>, p = r' + beta p.  Stops when
    ||r|| <= tol ||b||.  The residual history is the recursive ||r_j||/||b||.
    (Sec. 1: the CG implementation of Lanczos (Hestenes-Stiefel).)
    """
    b = np.asarray(b, dtype=np.complex128)
    bn = _norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    info = SolveInfo()
    r = b - A(x) if x0 is not None else b.copy()
    if x0 is not None:
        info.mvps += 1
    p = r.copy()
    rr = _dot(r, r).real
    info.residuals.append(np.sqrt(rr) / bn)
    for j in range(maxiter):
        if np.sqrt(rr) <= tol * bn:
            info.converged = True
            break
        q = A(p)
        info.mvps += 1
        alpha = rr / _dot(p, q).real
        x += alpha * p
        r -= alpha * q
        rr_new = _dot(r, r).real
        info.iterations += 1
        info.residuals.append(np.sqrt(rr_new) / bn)
        p = r + (rr_new / rr) * p
        rr = rr_new
    else:
        info.converged = np.sqrt(rr) <= tol * bn
    info.true_residual = _norm(b - A(x)) / bn
    return x, info


def cgnr(M, Mdag, b, x0=None, tol=1e-10, maxiter=10000):
    """CG on M^dagger M x = M^dagger b, stopping on the residual of M x = b.

    Sec. 2 plots the residual of M^{-1} itself, normalised to 1 at x = 0.
    The CG recurrence is the one of `cg` applied to A = M^dagger M; the
    residual s = b - M x of the original system is carried along by
    s -= alpha M p (M p is the first half of A p).  Each iteration is 2 MVPs.
    """
    b = np.asarray(b, dtype=np.complex128)
    bn = _norm(b)
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    s = b - M(x) if x0 is not None else b.copy()
    if x0 is not None:
        info.mvps += 1
    r = Mdag(s)
    info.mvps += 1
    p = r.copy()
    rr = _dot(r, r).real
    sn = _norm(s)
    info.residuals.append(sn / bn)
    for j in range(maxiter):
        if sn <= tol * bn:
            info.converged = True
            break
        mp = M(p)
        q = Mdag(mp)
        info.mvps += 2
        alpha = rr / _dot(p, q).real
        x += alpha * p
        r -= alpha * q
        s -= alpha * mp
        sn = _norm(s)
        rr_new = _dot(r, r).real
        info.iterations += 1
        info.residuals.append(sn / bn)
        p = r + (rr_new / rr) * p
        rr = rr_new
    else:
        info.converged = sn <= tol * bn
    info.true_residual = _norm(b - M(x)) / bn
    return x, info


def minres(A, b, x0=None, tol=1e-10, maxiter=10000):
    """Minimum residual method for hermitian (possibly indefinite) A.

    Lanczos from v1 = r0/beta1; the least-squares problem
    min || beta1 e1 - Tbar_j y || is solved by Givens rotations applied to the
    new column (0, .., beta_j, alpha_j, beta_{j+1}) of Tbar_j; with
    R's column (eps_j, delta_j, gamma_j) the search directions are
    d_j = (v_j - delta_j d_{j-1} - eps_j d_{j-2}) / gamma_j, x_j = x_{j-1} + tau_j d_j,
    tau_j = c_j phibar_j, phibar_{j+1} = -s_j phibar_j and ||r_j|| = |phibar_{j+1}|.
    (Sec. 1: the MinRes implementation of Lanczos (Paige-Saunders).)
    """
    b = np.asarray(b, dtype=np.complex128)
    bn = _norm(b)
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - A(x) if x0 is not None else b.copy()
    if x0 is not None:
        info.mvps += 1
    beta = _norm(r)
    info.residuals.append(beta / bn)
    if beta <= tol * bn:
        info.converged = True
        info.true_residual = beta / bn
        return x, info
    v_prev = np.zeros_like(b)
    v = r / beta
    d_prev2 = np.zeros_like(b)
    d_prev = np.zeros_like(b)
    c_old, s_old = 1.0, 0.0      # rotation j-2
    c, s = 1.0, 0.0              # rotation j-1
    phibar = beta
    beta_j = 0.0                 # beta_j (coupling to v_{j-1})
    for j in range(maxiter):
        w = A(v)
        info.mvps += 1
        w -= beta_j * v_prev
        alpha = _dot(v, w).real
        w -= alpha * v
        beta_next = _norm(w)
        # previous rotations on the new column (beta_j, alpha_j) -> (eps, delta, gammabar)
        eps = s_old * beta_j
        deltabar = c_old * beta_j
        delta = c * deltabar + s * alpha
        gammabar = -s * deltabar + c * alpha
        gamma = np.hypot(gammabar, beta_next)
        c_new, s_new = gammabar / gamma, beta_next / gamma
        tau = c_new * phibar
        phibar = -s_new * phibar
        d = (v - delta * d_prev - eps * d_prev2) / gamma
        x += tau * d
        info.iterations += 1
        info.residuals.append(abs(phibar) / bn)
        d_prev2, d_prev = d_prev, d
        c_old, s_old, c, s = c, s, c_new, s_new
        if abs(phibar) <= tol * bn:
            info.converged = True
            break
        if beta_next == 0.0:
            break
        v_prev, v = v, w / beta_next
        beta_j = beta_next
    info.true_residual = _norm(b - A(x)) / bn
    return x, info


# --------------------------------------------------------------------------
# Lanczos recurrence shared by Lan-DR and MinRes-DR
# --------------------------------------------------------------------------

class LanczosBreakdown(FloatingPointError):
    """beta_j fell below breakdown_tol * |alpha|-scale: span(V_j) is an invariant subspace."""

    def __init__(self, j):
        super().__init__(f"Lanczos breakdown at step {j}: invariant subspace found")
        self.j = j


def lanczos_extend(A, V, T, j0, m, kept=0, reorth_period=10, full_reorth=False,
                   breakdown_tol=1e-14, store=None):
    """Extend A V_j = V_{j+1} Tbar_j from j = j0 to j = m (0-based columns).

    V is a list of orthonormal vectors with len(V) == j0 + 1; T is the
    (m+1) x m array whose columns < j0 and row j0 (left of the diagonal)
    are already known.  For column j:
        w = A v_j - sum_{i<j} T[j,i] v_i        (T is hermitian: T[i,j] = conj(T[j,i]);
                                                 only i = j-1 is nonzero in the
                                                 three-term part; after a restart
                                                 column j0 couples to all kept vectors)
        alpha_j = <v_j, w>,  w -= alpha_j v_j,  beta_j = ||w||,  v_{j+1} = w / beta_j.
    Re-orthogonalisation (Sec. 2: periodic, over the vectors kept at the
    restart): w -= V_kept (V_kept^dag w) at the first new step j = j0 and then
    every `reorth_period` steps; the period is not given by the paper.
    full_reorth=True orthogonalises against all previous vectors (twice) at
    every step instead.  beta_j <= breakdown_tol * max|T| raises
    LanczosBreakdown (span(V_j) is invariant under A).  Returns the number
    of MVPs (one per step).
    """
    mvps = 0
    for j in range(j0, m):
        w = A(V[j])
        mvps += 1
        for i in range(j):
            t = T[j, i]
            if t != 0.0:
                w -= np.conj(t) * V[i]
                T[i, j] = np.conj(t)
        alpha = _dot(V[j], w).real
        w -= alpha * V[j]
        if full_reorth:
            for _ in range(2):
                for i in range(j + 1):
                    w -= _dot(V[i], w) * V[i]
        elif kept > 0 and reorth_period and (j - j0) % reorth_period == 0:
            # w -= V_kept (V_kept^dag w)
            Vk = store[:kept] if store is not None else np.array(V[:kept])
            w -= Vk.T @ (Vk.conj() @ w)
        beta = _norm(w)
        T[j, j] = alpha
        T[j + 1, j] = beta
        if j + 1 < m:
            T[j, j + 1] = beta
        scale = max(abs(alpha), float(np.abs(T[: j + 1, : j + 1]).max()))
        if beta <= breakdown_tol * scale:
            raise LanczosBreakdown(j)
        if store is None:
            V.append(w / beta)
        else:                       # preallocated (m+1) x n basis rows
            np.multiply(w, 1.0 / beta, out=store[j + 1])
            V.append(store[j + 1])
    return mvps


def lanczos(A, r0, m, full_reorth=False):
    """Plain Lanczos: returns (V_{m+1} as an n x (m+1) array, Tbar_m (m+1) x m, beta0).
    (Sec. 1: the Lanczos recurrence under both implementations.)"""
    beta0 = _norm(r0)
    V = [np.asarray(r0, dtype=np.complex128) / beta0]
    T = np.zeros((m + 1, m))
    lanczos_extend(A, V, T, 0, m, full_reorth=full_reorth)
    return np.stack(V, axis=1), T, beta0


def _combine(V, coeffs):
    """sum_j V[j] * coeffs[j] for a list of vectors (coefficient vector or matrix)."""
    Vm = np.stack(V[: coeffs.shape[0]], axis=1)
    return Vm @ coeffs


@dataclass
class DRResult:
    x: np.ndarray
    Vk: np.ndarray               # n x k orthonormal basis of the kept space
    ritz_values: np.ndarray      # theta (Lan-DR) or Rayleigh quotients (MinRes-DR)
    ritz_residuals: np.ndarray   # ||A y_i - value_i y_i|| for unit y_i in span(Vk)
    info: SolveInfo
    cycles: int = 0
    harmonic_theta: np.ndarray | None = None
    ritz_vectors: np.ndarray | None = None  # n x k, unit Rayleigh-Ritz vectors of span(Vk)


def landr(A, b, m, k, tol=1e-10, tol_eig=None, max_cycles=500, reorth_period=1,
          full_reorth=False, residual=None, oversolve=1.0, eig_stop=None, progress=None,
          plan_hook=None, eig_only=False):
    """Lan-DR(m,k) for hermitian positive definite A (Sec. 1, Sec. 2).

    Cycle 1: x0 = 0, r0 = b, v1 = r0/||r0||, Lanczos to j = m.  Each cycle:
      1. Galerkin solve T_m y = c (c = ||r0|| e_1 in cycle 1, rho e_{k+1} later);
         x += V_m y.  The new residual is rho v_{m+1}, rho = -Tbar[m, m-1] y_{m-1}.
      2. eig(T_m); keep the k algebraically smallest theta with orthonormal G_k
         (regular Ritz vectors, Sec. 2: exterior eigenproblem).
      3. Restart: V_{k+1} <- [V_m G_k, v_{m+1}]; the new Tbar has diag(theta) in
         its top k x k block and row k+1 equal to Tbar[m, m-1] * (last row of G_k).
      4. Continue Lanczos from column k (lanczos_extend handles the coupling of
         v_{k+1} to all kept vectors and the periodic re-orthogonalisation).
    Stopping (Sec. 2: the first right-hand side is run past convergence so the
    eigenvectors are accurate, at most doubling the MVPs): stop when the
    linear residual is <= tol AND every kept Ritz residual
    |Tbar[m,m-1] * G[m-1, i]| is <= tol_eig, or when the MVPs spent after the
    linear convergence exceed `oversolve` times those spent before it.
    `residual(x)` gives the relative residual used for the linear test
    (default ||b - A x|| / ||b||, evaluated once per cycle).  `eig_stop`
    turns the routine into an eigensolver: it stops as soon as the lowest
    Ritz pair has a residual <= eig_stop (or, for a callable,
    eig_stop(value, residual) is true).  `eig_only` is the eigensolver use
    of all k kept pairs (Sec. 2: the eigenvectors are the product handed to
    later right-hand sides): it stops as soon as every kept Ritz residual is
    <= tol_eig, whatever the linear residual, and `info.converged` says
    whether they did.
    """
    # Converged kept Ritz vectors attract rounding errors in every new Lanczos
    # vector (the loss of orthogonality grows like eps ||A|| / Ritz residual), so
    # Lan-DR re-orthogonalises against the kept vectors at every step: reorth_period
    # is 1 (every step) or 0 (off); any other value is refused rather than ignored.
    if reorth_period not in (0, 1):
        raise ValueError("Lan-DR re-orthogonalises at every step (reorth_period 1) or not at all (0)")
    return _dr(A, b, m, k, tol, tol_eig, max_cycles, reorth_period, full_reorth,
               residual, oversolve, harmonic=False, eig_stop=eig_stop, progress=progress,
               plan_hook=plan_hook, eig_only=eig_only)


def minresdr(A, b, m, k, tol=1e-10, tol_eig=None, max_cycles=500, reorth_period=10,
             full_reorth=False, residual=None, oversolve=1.0, eig_stop=None, progress=None,
             plan_hook=None, eig_only=False):
    """MinRes-DR(m,k) for hermitian, possibly indefinite A (Sec. 1, Sec. 2).

    Same Lanczos and restart skeleton as Lan-DR, with (GMRES-DR read for a
    hermitian matrix):
      1. Least squares y = argmin || c - Tbar_m y ||; x += V_m y; s = c - Tbar_m y
         so that the residual is V_{m+1} s.
      2. Harmonic Ritz pairs: T_m g = mu (Tbar_m^T Tbar_m) g (a symmetric-definite
         pencil, solved through the Cholesky factor of Tbar^T Tbar), theta = 1/mu;
         keep the k smallest |theta| (Sec. 2: harmonic Ritz vectors).
      3. P_{k+1} = orthonormalise([[G_k; 0], s]) (modified Gram-Schmidt twice,
         s last; s spans the orthogonal complement of range(Tbar_m), and that
         unit direction is used so the step stays exact once ||s|| is tiny); V_{k+1} <- V_{m+1} P_{k+1}; Tbar_k <- P_{k+1}^T Tbar_m P_k
         (k x k block symmetric, not diagonal); c <- P_{k+1}^T s.
    The kept-space values reported are the Rayleigh quotients over span(V_k)
    (eigenvalues of V_k^dag A V_k = top k x k block of Tbar_k); stopping as Lan-DR
    (`eig_only`: every kept harmonic Ritz residual <= tol_eig).
    """
    return _dr(A, b, m, k, tol, tol_eig, max_cycles, reorth_period, full_reorth,
               residual, oversolve, harmonic=True, eig_stop=eig_stop, progress=progress,
               plan_hook=plan_hook, eig_only=eig_only)


def _mgs_columns(P):
    """Orthonormalise the columns of P left to right (modified Gram-Schmidt, twice)."""
    Q = np.array(P, dtype=np.float64, copy=True)
    for j in range(Q.shape[1]):
        for _ in range(2):
            for i in range(j):
                Q[:, j] -= (Q[:, i] @ Q[:, j]) * Q[:, i]
        Q[:, j] /= np.linalg.norm(Q[:, j])
    return Q


@dataclass
class RestartPlan:
    """The small FP64 problem at the end of one DR cycle (Sec. 1-2; readings in
    the landr / minresdr docstrings), given Tbar_m ((m+1) x m) and c (m+1)."""
    y: np.ndarray            # m: x += V_m y
    theta: np.ndarray        # k kept (harmonic) Ritz values
    G: np.ndarray            # m x k, their unit vectors in the V_m basis
    ritz_res: np.ndarray     # k (harmonic) Ritz residuals
    P: np.ndarray            # (m+1) x (k+1): V_{k+1} <- V_{m+1} P
    Tn: np.ndarray           # (m+1) x m: the new Tbar (rows / columns < k+1 filled)
    cn: np.ndarray           # m+1: the new c
    rho: float = 0.0         # Lan-DR: the residual is rho v_{m+1}
    s: np.ndarray | None = None   # MinRes-DR: c - Tbar_m y (the residual is V_{m+1} s)


def restart_plan(T, c, m, k, harmonic):
    """Galerkin solve and regular Ritz pairs (Lan-DR) or least squares and harmonic
    Ritz pairs (MinRes-DR) of one cycle, and the restart matrices P, Tbar_k, c.
    (Sec. 1-2: the small problem at the end of each Lan-DR / MinRes-DR cycle.)"""
    Tm = T[:m, :m]
    if not harmonic:
        y = sla.solve(Tm, c[:m], assume_a="sym")
        rho = -T[m, m - 1] * y[m - 1]
        theta, G = np.linalg.eigh(Tm)
        order = np.argsort(theta, kind="stable")[:k]
        theta_k, G_k = theta[order], G[:, order]
        ritz_res = np.abs(T[m, m - 1] * G_k[m - 1, :])
        P = np.zeros((m + 1, k + 1))
        P[:m, :k] = G_k
        P[m, k] = 1.0
        Tn = np.zeros((m + 1, m))
        Tn[:k, :k] = np.diag(theta_k)
        Tn[k, :k] = T[m, m - 1] * G_k[m - 1, :]
        cn = np.zeros(m + 1)
        cn[k] = rho
        return RestartPlan(y=y, theta=theta_k, G=G_k, ritz_res=ritz_res, P=P, Tn=Tn, cn=cn, rho=rho)
    y, *_ = np.linalg.lstsq(T, c, rcond=None)
    s = c - T @ y
    L = np.linalg.cholesky(T.T @ T)
    Cm = sla.solve_triangular(L, sla.solve_triangular(L, Tm, lower=True).T, lower=True)
    Cm = 0.5 * (Cm + Cm.T)
    mu, Z = np.linalg.eigh(Cm)
    g = sla.solve_triangular(L.T, Z, lower=False)
    order = np.argsort(-np.abs(mu), kind="stable")[:k]
    theta_k = 1.0 / mu[order]
    G_k = g[:, order]
    G_k = G_k / np.linalg.norm(G_k, axis=0)
    Gpad = np.vstack([G_k, np.zeros((1, k))])
    ritz_res = np.linalg.norm(T @ G_k - theta_k * Gpad, axis=0)
    # s is orthogonal to range(Tbar_m); its direction is taken from the
    # complete QR of Tbar_m so that it stays exact when ||s|| is tiny.
    q = np.linalg.qr(T, mode="complete")[0][:, m]
    if q @ s < 0:
        q = -q
    P = _mgs_columns(np.hstack([np.vstack([G_k, np.zeros((1, k))]), q[:, None]]))
    Tk = P.T @ T @ P[:m, :k]
    Tn = np.zeros((m + 1, m))
    Tn[: k + 1, :k] = Tk
    Tn[:k, :k] = 0.5 * (Tn[:k, :k] + Tn[:k, :k].T)
    cn = np.zeros(m + 1)
    cn[: k + 1] = P.T @ s
    return RestartPlan(y=y, theta=theta_k, G=G_k, ritz_res=ritz_res, P=P, Tn=Tn, cn=cn, s=s)


def _rayleigh_ritz(T, k):
    """Eigen-decomposition of the k x k block, for the reported values/residuals."""
    return np.linalg.eigh(T[:k, :k])


def _dr(A, b, m, k, tol, tol_eig, max_cycles, reorth_period, full_reorth, residual,
        oversolve, harmonic, eig_stop=None, progress=None, plan_hook=None, eig_only=False):
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    bn = _norm(b)
    if residual is None:
        def residual(xx):
            return _norm(b - A(xx)) / bn
    info = SolveInfo()
    x = np.zeros_like(b)
    stores = [np.empty((m + 1, n), dtype=np.complex128), np.empty((m + 1, n), dtype=np.complex128)]
    cur = 0
    np.multiply(b, 1.0 / bn, out=stores[cur][0])
    V = [stores[cur][0]]
    T = np.zeros((m + 1, m))
    c = np.zeros(m + 1)
    c[0] = bn
    j0 = 0
    mvps_at_conv = None
    Anorm_est = 0.0
    theta_k = G_k = None
    cycles = 0
    for cycle in range(max_cycles):
        cycles += 1
        info.mvps += lanczos_extend(A, V, T, j0, m, kept=j0, reorth_period=reorth_period,
                                    full_reorth=full_reorth, store=stores[cur])
        Tm = T[:m, :m]
        Anorm_est = max(Anorm_est, float(np.abs(np.linalg.eigvalsh(Tm)).max()))
        if tol_eig is None:
            tol_eig_abs = 1e-10 * Anorm_est
        else:
            tol_eig_abs = tol_eig
        Vs = stores[cur]            # (m+1) x n: the basis as rows, for the products below
        pl = restart_plan(T, c, m, k, harmonic)
        if plan_hook is not None:
            plan_hook(T, c, pl)
        x = x + pl.y @ Vs[:m]
        theta_k, G_k, ritz_res = pl.theta, pl.G, pl.ritz_res
        info.iterations = info.mvps
        rel = residual(x)
        info.residuals.append(rel)
        lin_ok = rel <= tol
        if lin_ok and mvps_at_conv is None:
            mvps_at_conv = info.mvps
        eig_ok = bool(np.all(ritz_res <= tol_eig_abs))
        if progress is not None:
            progress(cycle, info.mvps, rel, theta_k, ritz_res)
        over = mvps_at_conv is not None and (info.mvps - mvps_at_conv) >= oversolve * mvps_at_conv
        last = cycle == max_cycles - 1
        if eig_only:
            info.converged = eig_ok
        elif lin_ok and (eig_ok or over):
            info.converged = True
        if eig_stop is not None:
            # eigenvalue-only use: stop once the pair nearest zero (harmonic) or the
            # lowest pair (regular) has a residual <= eig_stop, whatever the linear residual
            i0 = int(np.argmin(np.abs(theta_k))) if harmonic else 0
            done = (eig_stop(theta_k[i0], ritz_res[i0]) if callable(eig_stop)
                    else ritz_res[i0] <= eig_stop)
            if done:
                info.converged = True
        # restart (always performed so that V[:k] is the kept space on exit)
        nxt = stores[1 - cur]
        np.matmul(pl.P.T.astype(np.complex128), Vs, out=nxt[: k + 1])
        Vnew = [nxt[i] for i in range(k + 1)]
        Tn, cn = pl.Tn, pl.cn
        if not full_reorth and reorth_period:
            # The vector carried across the restart (v_{m+1} -> v_{k+1}) is part
            # of the periodic re-orthogonalisation over the kept vectors (Sec. 2);
            # without it the rounding-level overlap grows from cycle to cycle.
            for i in range(k):
                Vnew[k] -= _dot(Vnew[i], Vnew[k]) * Vnew[i]
            Vnew[k] /= _norm(Vnew[k])
        del Vs
        cur = 1 - cur
        V, T, c, j0 = Vnew, Tn, cn, k
        if info.converged or last:
            break
    Vk = np.array(np.stack(V[:k], axis=1))
    # Rayleigh-Ritz over the kept space (values reported for comparison)
    vals, Z = _rayleigh_ritz(T, k)
    Y = Vk @ Z
    res = np.array([_norm(A(Y[:, i]) - vals[i] * Y[:, i]) for i in range(k)])
    info.true_residual = residual(x)
    return DRResult(x=x, Vk=Vk, ritz_values=vals, ritz_residuals=res, info=info,
                    cycles=cycles, harmonic_theta=theta_k if harmonic else None,
                    ritz_vectors=Y)


# --------------------------------------------------------------------------
# D-CG and D-MinRes (Sec. 2)
# --------------------------------------------------------------------------

def deflation_space(A, Vk):
    """H = V_k^dagger A V_k (k MVPs).
    (Sec. 2: the projected matrix of the Galerkin projection of D-CG / D-MinRes.)"""
    AV = np.stack([A(Vk[:, i]) for i in range(Vk.shape[1])], axis=1)
    H = Vk.conj().T @ AV
    return 0.5 * (H + H.conj().T)


def galerkin_x0(Vk, H, b):
    """x0 = V_k H^{-1} V_k^dagger b: the Galerkin projection over the kept vectors.
    (Sec. 2: the Galerkin projection at the start of D-CG / D-MinRes.)"""
    return Vk @ np.linalg.solve(H, Vk.conj().T @ b)


def dcg(M, Mdag, b, Vk, H, tol=1e-10, maxiter=10000):
    """D-CG: Galerkin projection over V_k at the start, then CG on M^dagger M.

    A = M^dagger M, b' = M^dagger b, x0 = V_k H^{-1} V_k^dagger b', then cgnr
    from x0 (stopping on ||b - M x|| / ||b||).
    (Sec. 2: D-CG.)
    """
    bp = Mdag(b)
    x0 = galerkin_x0(Vk, H, bp)
    x, info = cgnr(M, Mdag, b, x0=x0, tol=tol, maxiter=maxiter)
    info.mvps += 1
    return x, info


def dminres(Q, b_gamma5, Vk, H, tol=1e-10, maxiter=10000):
    """D-MinRes: Galerkin projection over V_k at the start, then MinRes on Q.

    For Q = gamma5 M the right-hand side is b' = gamma5 b and
    ||b' - Q x|| = ||b - M x||, the residual plotted in Sec. 2.
    """
    x0 = galerkin_x0(Vk, H, b_gamma5)
    return minres(Q, b_gamma5, x0=x0, tol=tol, maxiter=maxiter)
