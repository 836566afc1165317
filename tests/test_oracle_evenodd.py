"""Pins of the even-odd (Schur complement) oracle (oracle/evenodd.py): against the
full Wilson operator (direct solve, determinant, adjoint), the closed-form free-field
spectrum, and the reduction in CG iterations."""
import numpy as np
import pytest

import synth
from oracle import evenodd as eo
from oracle import krylov as K
from oracle import wilson


def _unit_links(V):
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)
    for a in range(3):
        U[..., a, a] = 1.0
    return U


@pytest.mark.parametrize("dims,bc_t", [((2, 2, 2, 4), 1), ((4, 2, 2, 2), -1)])
def test_schur_solve_equals_direct_solve_and_determinants_agree(dims, bc_t):
    V = int(np.prod(dims))
    U = synth.su3_links(dims, 5)
    kappa = 0.12
    b = synth.gaussian_spinor(dims, 1)
    D = wilson.dense(wilson.operator(U, kappa, dims, "D", bc_t), 12 * V)
    x = np.linalg.solve(D, b.reshape(-1))
    Dh = wilson.dense(eo.operator(U, kappa, dims, "Dhat", bc_t), 6 * V)
    xe = np.linalg.solve(Dh, eo.prepare(U, b, kappa, dims, bc_t).reshape(-1)).reshape(V // 2, 4, 3)
    xf = eo.reconstruct(U, xe, b, kappa, dims, bc_t).reshape(-1)
    assert np.linalg.norm(xf - x) <= 1e-13 * np.linalg.norm(x)
    s1, l1 = np.linalg.slogdet(D)
    s2, l2 = np.linalg.slogdet(Dh)
    assert abs(l1 - l2) < 1e-11 and abs(s1 - s2) < 1e-12


def test_adjoint_and_hermitian_forms():
    dims = (2, 2, 2, 4)
    V = 32
    U = synth.su3_links(dims, 7)
    Dh = wilson.dense(eo.operator(U, 0.2, dims, "Dhat", -1), 6 * V)
    Dhd = wilson.dense(eo.operator(U, 0.2, dims, "Dhatdag", -1), 6 * V)
    Qh = wilson.dense(eo.operator(U, 0.2, dims, "Qhat", -1), 6 * V)
    assert np.abs(Dhd - Dh.conj().T).max() < 1e-14
    assert np.abs(Qh - Qh.conj().T).max() < 1e-14
    # on a larger lattice, by random vectors: <u, Dhat v> = <Dhat^dag u, v>, gamma5 Dhat gamma5 = Dhat^dag
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 8)
    u = synth.gaussian_spinor(dims, 2)[:128]
    v = synth.gaussian_spinor(dims, 3)[:128]
    lhs = np.vdot(u, eo.apply_Dhat(U, v, 0.2, dims))
    rhs = np.vdot(eo.apply_Dhatdag(U, u, 0.2, dims), v)
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(u) * np.linalg.norm(v)
    g5 = wilson.apply_gamma5
    assert np.abs(g5(eo.apply_Dhat(U, g5(v), 0.2, dims)) - eo.apply_Dhatdag(U, v, 0.2, dims)).max() < 1e-14


@pytest.mark.parametrize("bc_t", [1, -1])
def test_free_field_spectrum(bc_t):
    dims = (4, 4, 4, 4)
    V = 256
    Dh = wilson.dense(eo.operator(_unit_links(V), 0.11, dims, "Dhat", bc_t), 6 * V)
    ev = np.linalg.eigvals(Dh)
    cf = eo.free_spectrum_Dhat(0.11, dims, bc_t)
    assert ev.size == cf.size == 6 * V
    # as multisets: real parts, imaginary parts and moduli, each sorted
    assert np.abs(np.sort(ev.real) - np.sort(cf.real)).max() < 1e-12
    assert np.abs(np.sort(ev.imag) - np.sort(cf.imag)).max() < 1e-12
    assert np.abs(np.sort(np.abs(ev)) - np.sort(np.abs(cf))).max() < 1e-12


def test_cg_on_the_schur_complement_takes_fewer_iterations():
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 9)
    kappa = 0.2
    b = synth.gaussian_spinor(dims, 4)
    D = wilson.operator(U, kappa, dims, "D")
    Ddag = wilson.operator(U, kappa, dims, "Ddag")
    x_full, i_full = K.cgnr(D, Ddag, b.reshape(-1), tol=1e-10, maxiter=20000)
    Dh = eo.operator(U, kappa, dims, "Dhat")
    Dhd = eo.operator(U, kappa, dims, "Dhatdag")
    bh = eo.prepare(U, b, kappa, dims).reshape(-1)
    xe, i_eo = K.cgnr(Dh, Dhd, bh, tol=1e-10, maxiter=20000)
    x = eo.reconstruct(U, xe.reshape(128, 4, 3), b, kappa, dims).reshape(-1)
    assert i_full.converged and i_eo.converged
    assert np.linalg.norm(b.reshape(-1) - D(x)) <= 1e-9 * np.linalg.norm(b)
    assert np.linalg.norm(x - x_full) <= 1e-8 * np.linalg.norm(x_full)
    assert i_eo.iterations < 0.75 * i_full.iterations


def test_odd_extent_is_rejected():
    with pytest.raises(ValueError):
        eo.parity((3, 4, 4, 4))


def test_deflated_solves_on_the_schur_complement():
    """MinRes-DR on Qhat = gamma5 Dhat for the first right-hand side, D-MinRes over its
    deflation set for a second one: both reconstruct the full solution of D x = b, and
    the deflated solve takes fewer iterations than plain MinRes on Qhat."""
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 10)
    kappa = 0.2
    D = wilson.operator(U, kappa, dims, "D")
    Qh = eo.operator(U, kappa, dims, "Qhat")
    g5 = wilson.apply_gamma5
    b1, b2 = synth.gaussian_spinor(dims, 11), synth.gaussian_spinor(dims, 12)
    r = K.minresdr(Qh, g5(eo.prepare(U, b1, kappa, dims)).reshape(-1), 30, 8, tol=1e-10, max_cycles=200,
                   oversolve=2.0)
    assert r.info.converged
    x1 = eo.reconstruct(U, r.x.reshape(128, 4, 3), b1, kappa, dims).reshape(-1)
    assert np.linalg.norm(b1.reshape(-1) - D(x1)) <= 1e-9 * np.linalg.norm(b1)
    H = K.deflation_space(Qh, r.Vk)
    rhs = g5(eo.prepare(U, b2, kappa, dims)).reshape(-1)
    xd, info_d = K.dminres(Qh, rhs, r.Vk, H, tol=1e-10)
    _, info_0 = K.minres(Qh, rhs, tol=1e-10)
    x2 = eo.reconstruct(U, xd.reshape(128, 4, 3), b2, kappa, dims).reshape(-1)
    assert np.linalg.norm(b2.reshape(-1) - D(x2)) <= 1e-9 * np.linalg.norm(b2)
    assert info_d.iterations < info_0.iterations
