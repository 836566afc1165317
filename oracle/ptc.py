"""Gauge-covariant parallel-transport convolution (PTC) network, FP64 NumPy
oracle (test infrastructure only).

The learned deflation seed is not in the paper (Sec. 2 computes the deflation
space with Lan-DR / MinRes-DR only).  The layer used here moves colour only with
the gauge links, so it commutes with gauge transformations:

    out[c'](x) = sum_o sum_c  W[o, c', c] (T_o in[c])(x),

with nine offsets o = 0, +mu, -mu (index 0, 1 + 2 mu, 2 + 2 mu; mu = x, y, z, t),
the parallel transports

    (T_0 psi)(x)   = psi(x)
    (T_+mu psi)(x) = U_mu(x) psi(x + mu)
    (T_-mu psi)(x) = U_mu(x - mu)^dagger psi(x - mu)

(periodic boundaries) and a complex 4x4 spin matrix W[o, c', c] per offset and
channel pair.  With one channel, W[0] = 1, W[+mu] = -kappa (1 - gamma_mu) and
W[-mu] = -kappa (1 + gamma_mu) the layer is the Wilson matrix D.

Gradients use the convention G(z) = dL/dRe z + i dL/dIm z for a real loss L
(twice the Wirtinger derivative dL/dconj(z)).  For out = W t:
G(W) = sum over sites and colours of G(out) t^dagger, and G(in) = L^dagger G(out),
where the adjoint layer has weights W^H on the opposite offsets.

Everything is written from these definitions with np.roll and einsum, one offset
at a time.  Arrays: a field of C channels is (C, V, 4, 3) complex; weights of a
layer (9, C_out, C_in, 4, 4); the gauge field (4, V, 3, 3).
"""
from __future__ import annotations

import numpy as np

from .wilson import _AXIS_LINK, _AXIS_SPINOR, _lattice_view

N_OFFSETS = 9


def offset_index(mu: int, sign: int) -> int:
    """Index of offset +mu (sign = +1) or -mu (sign = -1); 0 is the site itself.
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    return 1 + 2 * mu + (0 if sign > 0 else 1)


def opposite(o: int) -> int:
    """Index of the offset opposite to o (0 is its own opposite).
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    if o == 0:
        return 0
    return o + 1 if (o - 1) % 2 == 0 else o - 1


def transport(U, psi, dims, o):
    """T_o psi for a field psi (..., V, 4, 3).
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    if o == 0:
        return psi.copy()
    mu, fwd = (o - 1) // 2, (o - 1) % 2 == 0
    lx, ly, lz, lt = dims
    P = _lattice_view(psi, dims)
    Ul = U.reshape(4, lt, lz, ly, lx, 3, 3)
    ax = _AXIS_SPINOR[mu]
    if fwd:
        pf = np.roll(P, -1, axis=ax)
        out = np.einsum("...ij,...sj->...si", Ul[mu], pf)
    else:
        pb = np.roll(P, 1, axis=ax)
        ub = np.roll(Ul[mu], 1, axis=_AXIS_LINK[mu])
        out = np.einsum("...ji,...sj->...si", ub.conj(), pb)
    return out.reshape(psi.shape)


def layer(W, U, x, dims):
    """out[c'] = sum_o sum_c W[o, c', c] (T_o x[c]); x (C_in, V, 4, 3).
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    W = np.asarray(W, dtype=np.complex128)
    nout = W.shape[1]
    out = np.zeros((nout,) + x.shape[1:], dtype=np.complex128)
    for o in range(N_OFFSETS):
        t = transport(U, x, dims, o)                       # (C_in, V, 4, 3)
        out += np.einsum("pqab,qvbc->pvac", W[o], t)
    return out


def adjoint_weights(W):
    """Weights of the adjoint layer: W'[o, c, c'] = W[opp(o), c', c]^H.
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    W = np.asarray(W, dtype=np.complex128)
    Wa = np.empty((W.shape[0], W.shape[2], W.shape[1], 4, 4), dtype=np.complex128)
    for o in range(N_OFFSETS):
        Wa[o] = np.conj(np.transpose(W[opposite(o)], (1, 0, 3, 2)))
    return Wa


def layer_adjoint(W, U, g, dims):
    """L^dagger g for the layer L with weights W.
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    return layer(adjoint_weights(W), U, g, dims)


def layer_weight_grad(U, x, g, dims):
    """G(W)[o, c', c] = sum_{sites, colours} g[c'] (T_o x[c])^dagger (spin 4x4).
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    G = np.empty((N_OFFSETS, g.shape[0], x.shape[0], 4, 4), dtype=np.complex128)
    for o in range(N_OFFSETS):
        t = transport(U, x, dims, o)
        G[o] = np.einsum("pvac,qvbc->pqab", g, t.conj())
    return G


def forward(Ws, U, eta, dims):
    """Network output and the inputs of every layer (for the backward pass).

    eta: (V, 4, 3) one input vector; returns (f (V, 4, 3), [layer inputs]).
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)
    """
    x = np.asarray(eta, dtype=np.complex128)[None]
    inputs = []
    for W in Ws:
        inputs.append(x)
        x = layer(W, U, x, dims)
    return x[0], inputs


def backward(Ws, U, inputs, g_out, dims):
    """Weight gradients of every layer and G(eta), given G(f) = g_out (V, 4, 3).
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    g = np.asarray(g_out, dtype=np.complex128)[None]
    grads = [None] * len(Ws)
    for li in range(len(Ws) - 1, -1, -1):
        grads[li] = layer_weight_grad(U, inputs[li], g, dims)
        g = layer_adjoint(Ws[li], U, g, dims)
    return grads, g[0]


def subspace_loss(Vk, f):
    """||(1 - V V^dag) f||^2 / ||f||^2 for orthonormal columns Vk (n, k), and G(f).
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    f = np.asarray(f, dtype=np.complex128).reshape(-1)
    h = Vk.conj().T @ f
    perp = f - Vk @ h
    nf = np.vdot(f, f).real
    L = np.vdot(perp, perp).real / nf
    g = 2.0 * (perp - L * f) / nf
    return L, g


def wilson_weights(kappa):
    """Weights of the one-channel layer that equals the Wilson matrix D.
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    from .wilson import gamma_matrices
    G = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    W = np.zeros((N_OFFSETS, 1, 1, 4, 4), dtype=np.complex128)
    W[0, 0, 0] = one
    for mu in range(4):
        W[offset_index(mu, +1), 0, 0] = -kappa * (one - G[mu])
        W[offset_index(mu, -1), 0, 0] = -kappa * (one + G[mu])
    return W


def round_bf16(a):
    """Round real and imaginary parts to bfloat16 (nearest even), returned as complex128.
    (Not in the paper: the learned seed for the deflation space of Sec. 2.)"""
    a = np.asarray(a, dtype=np.complex128)

    def r(x):
        b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32).astype(np.float64)

    return r(a.real) + 1j * r(a.imag)
