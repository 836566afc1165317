"""Pins of the FP64 Wilson oracle against facts outside the oracle itself.

The Wilson matrix M of Sec. 2 (D here) is checked against: the Clifford
algebra, closed-form free-field and constant-U(1) spectra, plane waves,
hermiticity of gamma5 D, the adjoint written out independently, gauge
covariance, and a pure-gauge field.  A wrong sign of a projector, a
transposed or un-conjugated backward link, a link taken at the wrong site or
a mixed-up axis fails at least one of them.
"""
import numpy as np
import pytest

import synth
from oracle import cwilson, wilson

G = wilson.gamma_matrices()


def test_gamma_clifford_and_gamma5():
    for a in range(4):
        assert np.allclose(G[a], G[a].conj().T)
        for b in range(4):
            assert np.allclose(G[a] @ G[b] + G[b] @ G[a], 2.0 * (a == b) * np.eye(4))
        assert np.allclose(G[4] @ G[a] + G[a] @ G[4], 0)
    assert np.allclose(G[4], np.diag([1, 1, -1, -1]))


def test_links_are_su3():
    U = synth.su3_links((3, 2, 4, 2), seed=9)
    uu = np.einsum("...ji,...jk->...ik", U.conj(), U)
    assert np.abs(uu - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


@pytest.mark.parametrize("dims,bc_t", [((2, 2, 2, 2), 1), ((2, 2, 2, 4), -1), ((3, 2, 2, 2), 1)])
def test_free_field_spectrum_closed_form(dims, bc_t):
    kappa = 0.11
    n = synth.volume(dims) * 12
    Q = wilson.dense(wilson.operator(synth.unit_links(dims), kappa, dims, "Q", bc_t), n)
    ev = np.linalg.eigvalsh(Q)
    assert np.abs(ev - wilson.free_spectrum_Q(kappa, dims, bc_t)).max() < 1e-13


def _plane_wave(dims, nvec, chi, theta_t=0.0):
    lx, ly, lz, lt = dims
    x, y, z, t = np.meshgrid(np.arange(lx), np.arange(ly), np.arange(lz), np.arange(lt),
                             indexing="ij")
    p = [2 * np.pi * nvec[0] / lx, 2 * np.pi * nvec[1] / ly, 2 * np.pi * nvec[2] / lz,
         (2 * np.pi * nvec[3] + theta_t) / lt]
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    ph = np.transpose(ph, (3, 2, 1, 0)).reshape(-1)      # site order x fastest
    return ph[:, None, None] * chi[None, :, :], p


def test_plane_wave_symbol():
    """D e^{ipx} chi = [1 - 2 kappa sum cos p + 2 i kappa sum gamma_mu sin p] e^{ipx} chi."""
    dims = (4, 3, 2, 5)
    kappa = 0.137
    rng = np.random.default_rng(3)
    chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi, p = _plane_wave(dims, (1, 2, 1, 3), chi)
    sym = (1 - 2 * kappa * sum(np.cos(q) for q in p)) * np.eye(4) \
        + 2j * kappa * sum(G[m] * np.sin(p[m]) for m in range(4))
    want = psi[:, :, :] * 0
    want = (np.einsum("ab,bc->ac", sym, chi))[None] * (psi[:, 0, 0] / chi[0, 0])[:, None, None]
    got = wilson.apply_D(synth.unit_links(dims), psi, kappa, dims)
    assert np.abs(got - want).max() < 1e-13


def test_constant_u1_phase_shifts_momentum():
    """U_mu = exp(i th_mu) 1 acts on a plane wave like the shift p_mu -> p_mu + th_mu."""
    dims = (4, 3, 2, 5)
    kappa = 0.121
    th = [0.3, -0.7, 1.1, 0.45]
    U = synth.unit_links(dims) * np.exp(1j * np.array(th))[:, None, None, None]
    rng = np.random.default_rng(4)
    chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi, p = _plane_wave(dims, (1, 0, 1, 2), chi)
    q = [p[m] + th[m] for m in range(4)]
    sym = (1 - 2 * kappa * sum(np.cos(v) for v in q)) * np.eye(4) \
        + 2j * kappa * sum(G[m] * np.sin(q[m]) for m in range(4))
    want = (np.einsum("ab,bc->ac", sym, chi))[None] * (psi[:, 0, 0] / chi[0, 0])[:, None, None]
    got = wilson.apply_D(U, psi, kappa, dims)
    assert np.abs(got - want).max() < 1e-13


def test_antiperiodic_time_is_a_half_momentum_shift():
    dims = (2, 3, 2, 4)
    kappa = 0.1
    rng = np.random.default_rng(5)
    chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi, p = _plane_wave(dims, (1, 1, 0, 1), chi, theta_t=np.pi)
    sym = (1 - 2 * kappa * sum(np.cos(v) for v in p)) * np.eye(4) \
        + 2j * kappa * sum(G[m] * np.sin(p[m]) for m in range(4))
    want = (np.einsum("ab,bc->ac", sym, chi))[None] * (psi[:, 0, 0] / chi[0, 0])[:, None, None]
    got = wilson.apply_D(synth.unit_links(dims), psi, kappa, dims, bc_t=-1)
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("bc_t", [1, -1])
def test_gamma5_D_is_hermitian_and_adjoint_is_consistent(bc_t):
    dims = (3, 4, 2, 5)
    U = synth.su3_links(dims, seed=11)
    kappa = 0.2
    rng = np.random.default_rng(2)
    V = synth.volume(dims)
    u = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    v = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    Qv = wilson.apply_Q(U, v, kappa, dims, bc_t)
    Qu = wilson.apply_Q(U, u, kappa, dims, bc_t)
    nrm = np.linalg.norm(u) * np.linalg.norm(v)
    assert abs(np.vdot(u, Qv) - np.vdot(Qu, v)) / nrm < 1e-14
    Dv = wilson.apply_D(U, v, kappa, dims, bc_t)
    Ddu = wilson.apply_Ddag(U, u, kappa, dims, bc_t)
    assert abs(np.vdot(u, Dv) - np.vdot(Ddu, v)) / nrm < 1e-14
    # D^dagger = gamma5 D gamma5
    g5Dg5 = wilson.apply_gamma5(wilson.apply_D(U, wilson.apply_gamma5(u), kappa, dims, bc_t))
    assert np.abs(g5Dg5 - Ddu).max() < 1e-14


def test_dense_Q_hermitian_small_lattice():
    dims = (2, 2, 2, 4)
    U = synth.su3_links(dims, seed=1)
    n = synth.volume(dims) * 12
    Q = wilson.dense(wilson.operator(U, 0.15, dims, "Q", -1), n)
    assert np.abs(Q - Q.conj().T).max() < 1e-15


def _gauge_transform(U, g, dims):
    """U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger."""
    lx, ly, lz, lt = dims
    gl = g.reshape(lt, lz, ly, lx, 3, 3)
    out = np.empty_like(U)
    for mu, ax in zip(range(4), (3, 2, 1, 0)):
        gf = np.roll(gl, -1, axis=ax).reshape(-1, 3, 3)
        out[mu] = g @ U[mu] @ np.conj(np.swapaxes(gf, -1, -2))
    return out


def test_gauge_covariance():
    dims = (3, 2, 4, 3)
    U = synth.su3_links(dims, seed=21)
    g = synth.random_su3_gauge_transform(dims, seed=22)
    Up = _gauge_transform(U, g, dims)
    V = synth.volume(dims)
    rng = np.random.default_rng(7)
    psi = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    gpsi = np.einsum("sij,saj->sai", g, psi)
    for bc in (1, -1):
        lhs = wilson.apply_D(Up, gpsi, 0.17, dims, bc)
        rhs = np.einsum("sij,saj->sai", g, wilson.apply_D(U, psi, 0.17, dims, bc))
        assert np.abs(lhs - rhs).max() < 1e-13


def test_pure_gauge_reproduces_free_spectrum():
    dims = (2, 2, 2, 2)
    g = synth.random_su3_gauge_transform(dims, seed=31)
    U = _gauge_transform(synth.unit_links(dims), g, dims)
    n = synth.volume(dims) * 12
    Q = wilson.dense(wilson.operator(U, 0.09, dims, "Q"), n)
    assert np.abs(np.linalg.eigvalsh(Q) - wilson.free_spectrum_Q(0.09, dims)).max() < 1e-13


@pytest.mark.parametrize("dims", [(3, 5, 4, 6), (4, 6, 2, 8)])
def test_c_oracle_matches_numpy_oracle(dims):
    U = synth.su3_links(dims, seed=5)
    psi = synth.gaussian_spinor(dims, 7)
    for bc in (1, -1):
        a = wilson.apply_D(U, psi, 0.13, dims, bc)
        b = cwilson.apply_D(U, psi, 0.13, dims, bc)
        assert np.abs(a - b).max() < 1e-14
        a = wilson.apply_Ddag(U, psi, 0.13, dims, bc)
        b = cwilson.apply_D(U, psi, 0.13, dims, bc, dagger=True)
        assert np.abs(a - b).max() < 1e-14
        sites = np.array([0, 1, synth.volume(dims) // 2, synth.volume(dims) - 1])
        c = cwilson.apply_D_sites(U, psi, 0.13, dims, sites, bc)
        assert np.abs(c - wilson.apply_D(U, psi, 0.13, dims, bc)[sites]).max() < 1e-14
