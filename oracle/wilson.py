"""Wilson-Dirac operator, FP64 NumPy oracle (test infrastructure only).

Sec. 2 of the paper uses the Wilson matrix M (written D here), as
M^dagger M for the CG family and as gamma5 M for the MinRes family.  The
paper does not write M out; the standard form is used:

    (D psi)(x) = psi(x) - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                                          + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ]

with periodic boundaries (bc_t = -1 makes the time direction antiperiodic for
the fermion hop), and the chiral Euclidean hermitian gamma basis

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1, 2, 3),
    gamma_4 = [[0, 1], [1, 0]],   gamma5 = gamma1 gamma2 gamma3 gamma4.

Everything is written from the definition: explicit 4x4 spin matrices, one
np.roll per hop, no spin projection, no fusion.  Arrays may carry any number
of leading batch axes: a spinor is (..., V, 4, 3), the gauge field (4, V, 3, 3).
"""
from __future__ import annotations

import numpy as np

_SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def gamma_matrices():
    """(gamma_1, gamma_2, gamma_3, gamma_4, gamma_5) in the chiral basis.
    (Sec. 2: the Wilson matrix M (D here), used as M^dagger M and gamma5 M.)"""
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)
    g = [np.block([[z, -1j * s], [1j * s, z]]) for s in _SIGMA]
    g.append(np.block([[z, one], [one, z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return tuple(g) + (g5,)


_G = gamma_matrices()
_ONE4 = np.eye(4, dtype=np.complex128)


def _lattice_view(psi, dims):
    lx, ly, lz, lt = dims
    return psi.reshape(psi.shape[:-3] + (lt, lz, ly, lx, 4, 3))


# axis of direction mu in the (..., Lt, Lz, Ly, Lx, 4, 3) view (counted from the end)
_AXIS_SPINOR = {0: -3, 1: -4, 2: -5, 3: -6}
# axis of direction mu in the (Lt, Lz, Ly, Lx, 3, 3) view of one link direction
_AXIS_LINK = {0: -3, 1: -4, 2: -5, 3: -6}


def _hop_sum(U, psi, dims, bc_t, sign):
    """sum_mu [ (1 - s g_mu) U_mu(x) psi(x+mu) + (1 + s g_mu) U_mu(x-mu)^dag psi(x-mu) ].

    sign = +1 gives the hopping term of D, sign = -1 that of D^dagger.
    """
    lx, ly, lz, lt = dims
    P = _lattice_view(psi, dims)
    Ul = U.reshape(4, lt, lz, ly, lx, 3, 3)
    acc = np.zeros_like(P)
    for mu in range(4):
        ax = _AXIS_SPINOR[mu]
        # forward hop: psi(x + mu), with the boundary phase on the wrapped slice
        pf = np.roll(P, -1, axis=ax)
        if mu == 3 and bc_t != 1:
            pf[..., lt - 1, :, :, :, :, :] *= bc_t
        hf = np.einsum("...ij,...sj->...si", Ul[mu], pf)
        # backward hop: U_mu(x - mu)^dagger psi(x - mu)
        pb = np.roll(P, 1, axis=ax)
        if mu == 3 and bc_t != 1:
            pb[..., 0, :, :, :, :, :] *= bc_t
        ub = np.roll(Ul[mu], 1, axis=_AXIS_LINK[mu])
        hb = np.einsum("...ji,...sj->...si", ub.conj(), pb)
        acc += np.einsum("ab,...bc->...ac", _ONE4 - sign * _G[mu], hf)
        acc += np.einsum("ab,...bc->...ac", _ONE4 + sign * _G[mu], hb)
    return acc.reshape(psi.shape)


def apply_D(U, psi, kappa, dims, bc_t=1):
    """Wilson matrix D (the paper's M), Sec. 2."""
    return psi - kappa * _hop_sum(U, psi, dims, bc_t, +1)


def apply_Ddag(U, psi, kappa, dims, bc_t=1):
    """D^dagger written out directly (gamma_mu -> -gamma_mu in the hopping term).
    (Sec. 2: the Wilson matrix M (D here), used as M^dagger M and gamma5 M.)"""
    return psi - kappa * _hop_sum(U, psi, dims, bc_t, -1)


def apply_gamma5(psi):
    """gamma5 on the spin index of (..., 4, 3) spinors.
    (Sec. 2: the Wilson matrix M (D here), used as M^dagger M and gamma5 M.)"""
    return np.einsum("ab,...bc->...ac", _G[4], psi)


def apply_Q(U, psi, kappa, dims, bc_t=1):
    """Hermitian indefinite Q = gamma5 D, the MinRes-family operator of Sec. 2."""
    return apply_gamma5(apply_D(U, psi, kappa, dims, bc_t))


def apply_DdagD(U, psi, kappa, dims, bc_t=1):
    """Hermitian positive definite D^dagger D, the CG-family operator of Sec. 2."""
    return apply_Ddag(U, apply_D(U, psi, kappa, dims, bc_t), kappa, dims, bc_t)


def dense(apply, n, chunk=256):
    """Dense n x n matrix of a linear map on flat complex vectors (tiny lattices).
    (Sec. 2: the Wilson matrix M (D here), used as M^dagger M and gamma5 M.)"""
    out = np.empty((n, n), dtype=np.complex128)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        e = np.zeros((c1 - c0, n), dtype=np.complex128)
        e[np.arange(c1 - c0), np.arange(c0, c1)] = 1.0
        out[:, c0:c1] = apply(e).T
    return out


def operator(U, kappa, dims, which="D", bc_t=1):
    """Flat-vector closure x -> A x for which in {'D', 'Ddag', 'Q', 'DdagD'}.
    (Sec. 2: the Wilson matrix M (D here), used as M^dagger M and gamma5 M.)"""
    V = int(np.prod(dims))
    f = {"D": apply_D, "Ddag": apply_Ddag, "Q": apply_Q, "DdagD": apply_DdagD}[which]

    def A(x):
        x = np.asarray(x)
        lead = x.shape[:-1]
        y = f(U, x.reshape(lead + (V, 4, 3)), kappa, dims, bc_t)
        return y.reshape(lead + (V * 12,))

    return A


def free_spectrum_Q(kappa, dims, bc_t=1):
    """Closed-form eigenvalues of Q = gamma5 D at U = 1 (each with multiplicity 6).

    For a plane wave with lattice momenta p_mu = 2 pi n_mu / L_mu (n_t + 1/2
    for antiperiodic time), D acts as a(p) - i*kappa*2 sum gamma_mu sin p_mu
    up to sign with a(p) = 1 - 2 kappa sum cos p_mu, so eigenvalues of Q are
    +-sqrt(a(p)^2 + 4 kappa^2 sum sin^2 p_mu).  Returns them sorted.
    (Sec. 2: the Wilson matrix M (D here), used as M^dagger M and gamma5 M.)
    """
    lx, ly, lz, lt = dims
    ps = []
    for L, anti in ((lx, False), (ly, False), (lz, False), (lt, bc_t == -1)):
        n = np.arange(L) + (0.5 if anti else 0.0)
        ps.append(2 * np.pi * n / L)
    P = np.meshgrid(*ps, indexing="ij")
    a = 1 - 2 * kappa * sum(np.cos(p) for p in P)
    b2 = 4 * kappa ** 2 * sum(np.sin(p) ** 2 for p in P)
    e = np.sqrt(a ** 2 + b2).ravel()
    ev = np.concatenate([np.repeat(e, 6), -np.repeat(e, 6)])
    return np.sort(ev)
