"""Even-odd (Schur complement) form of the Wilson operator, FP64 NumPy oracle (test
infrastructure only).

Not in the paper: the standard reduction to the even sites that the deflated
methods of Sec. 2 apply to unchanged.  The hopping term H of D = 1 - kappa H
(oracle/wilson.py) only links sites of opposite parity (x + y + z + t even or
odd), so with the even sites first

    D = [[1, -kappa H_eo], [-kappa H_oe, 1]],

and D x = b is solved through the Schur complement on the even sites:

    Dhat x_e = b_e + kappa H_eo b_o,   Dhat = 1 - kappa^2 H_eo H_oe,
    x_o = b_o + kappa H_oe x_e.

det D = det Dhat.  Dhat^dagger has the same form with the hopping term of
D^dagger, and gamma5 Dhat gamma5 = Dhat^dagger, so Qhat = gamma5 Dhat is
hermitian.  Every lattice extent must be even (the checkerboard must be
consistent across the periodic wrap).  Even-site vectors hold the even sites in
increasing site order: (..., V/2, 4, 3).
"""
from __future__ import annotations

import numpy as np

from . import wilson


def parity(dims):
    """(x + y + z + t) mod 2 for every site s = ((t Lz + z) Ly + y) Lx + x.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    if any(int(L) % 2 for L in dims):
        raise ValueError("even-odd splitting needs every lattice extent even")
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1)


def sites(dims):
    """(even site indices, odd site indices), each increasing.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    p = parity(dims)
    return np.flatnonzero(p == 0), np.flatnonzero(p == 1)


def split(psi, dims):
    """Full-lattice spinor (..., V, 4, 3) -> (even part, odd part).
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    ev, od = sites(dims)
    return psi[..., ev, :, :], psi[..., od, :, :]


def join(psi_e, psi_o, dims):
    """(even part, odd part) -> full-lattice spinor.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    ev, od = sites(dims)
    V = int(np.prod(dims))
    lead = psi_e.shape[:-3] if psi_e is not None else psi_o.shape[:-3]
    out = np.zeros(lead + (V, 4, 3), dtype=np.complex128)
    if psi_e is not None:
        out[..., ev, :, :] = psi_e
    if psi_o is not None:
        out[..., od, :, :] = psi_o
    return out


def hop_oe(U, psi_e, dims, bc_t=1, sign=+1):
    """H_oe psi_e: the hopping term applied to an even-site vector, read on the odd
    sites (sign = -1: the hopping term of D^dagger).
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    full = wilson._hop_sum(U, join(psi_e, None, dims), dims, bc_t, sign)
    return split(full, dims)[1]


def hop_eo(U, psi_o, dims, bc_t=1, sign=+1):
    """H_eo psi_o: the hopping term applied to an odd-site vector, read on the even sites.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    full = wilson._hop_sum(U, join(None, psi_o, dims), dims, bc_t, sign)
    return split(full, dims)[0]


def apply_Dhat(U, psi_e, kappa, dims, bc_t=1):
    """Schur complement Dhat = 1 - kappa^2 H_eo H_oe on the even sites.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    return psi_e - kappa * kappa * hop_eo(U, hop_oe(U, psi_e, dims, bc_t), dims, bc_t)


def apply_Dhatdag(U, psi_e, kappa, dims, bc_t=1):
    """Dhat^dagger = 1 - kappa^2 H'_eo H'_oe with H' the hopping term of D^dagger.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    return psi_e - kappa * kappa * hop_eo(U, hop_oe(U, psi_e, dims, bc_t, -1), dims, bc_t, -1)


def apply_Qhat(U, psi_e, kappa, dims, bc_t=1):
    """Hermitian Qhat = gamma5 Dhat.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    return wilson.apply_gamma5(apply_Dhat(U, psi_e, kappa, dims, bc_t))


def apply_DhatdagDhat(U, psi_e, kappa, dims, bc_t=1):
    """Hermitian positive definite Dhat^dagger Dhat.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    return apply_Dhatdag(U, apply_Dhat(U, psi_e, kappa, dims, bc_t), kappa, dims, bc_t)


def prepare(U, b, kappa, dims, bc_t=1):
    """Right-hand side of the even-site system: b_e + kappa H_eo b_o.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    b_e, b_o = split(b, dims)
    return b_e + kappa * hop_eo(U, b_o, dims, bc_t)


def reconstruct(U, x_e, b, kappa, dims, bc_t=1):
    """Full solution from the even part: x_o = b_o + kappa H_oe x_e.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    _, b_o = split(b, dims)
    return join(x_e, b_o + kappa * hop_oe(U, x_e, dims, bc_t), dims)


def operator(U, kappa, dims, which="Dhat", bc_t=1):
    """Flat closure on even-site vectors (6 V complex values) for which in
    {'Dhat', 'Dhatdag', 'Qhat', 'DhatdagDhat'}.
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    Vh = int(np.prod(dims)) // 2
    f = {"Dhat": apply_Dhat, "Dhatdag": apply_Dhatdag, "Qhat": apply_Qhat,
         "DhatdagDhat": apply_DhatdagDhat}[which]

    def A(x):
        x = np.asarray(x)
        lead = x.shape[:-1]
        return f(U, x.reshape(lead + (Vh, 4, 3)), kappa, dims, bc_t).reshape(lead + (Vh * 12,))

    return A


def free_spectrum_Dhat(kappa, dims, bc_t=1):
    """Closed-form eigenvalues of Dhat at U = 1: with C = sum_mu cos p_mu and
    S = (sum_mu sin^2 p_mu)^(1/2), the hopping term at momentum p has the eigenvalues
    h = 2 C -/+ 2 i S (gamma_mu anticommute, so (sum_mu gamma_mu sin p_mu)^2 = S^2),
    each twice in spin and three times in colour; p and p + (pi, pi, pi, pi) give
    h and -h, the same h^2, so Dhat has 1 - kappa^2 h^2 for every momentum of the
    lattice and both signs, each three times (6 V values).
    (Not in the paper: the even-odd reduction that the methods of Sec. 1-2 apply to
    unchanged.)"""
    axes = []
    for mu, L in enumerate(dims):
        shift = 0.5 if (mu == 3 and bc_t == -1) else 0.0
        axes.append(2.0 * np.pi * (np.arange(L) + shift) / L)
    P = np.meshgrid(*axes, indexing="ij")
    C = sum(np.cos(p) for p in P).reshape(-1)
    S = np.sqrt(sum(np.sin(p) ** 2 for p in P)).reshape(-1)
    vals = []
    for sgn in (+1.0, -1.0):
        h = 2.0 * C + sgn * 2.0j * S
        vals.append(1.0 - kappa * kappa * h * h)
    return np.repeat(np.concatenate(vals), 3)
