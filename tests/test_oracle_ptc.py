"""Pins of the PTC-network oracle (oracle/ptc.py) against facts fixed by the
definitions: the one-channel layer with Wilson weights is the (already pinned)
Wilson matrix; forward-then-backward transport is the identity for unitary
links; the layer commutes with gauge transformations; the adjoint layer
satisfies <a, L b> = <L^dag a, b>; the network's weight and input gradients and
the subspace loss's gradient match central finite differences (step 1e-5,
complex directions, FP64, 1e-7 relative) on a 4^4 lattice with widths
1 -> 2 -> 2 -> 1; bfloat16 rounding matches hand-worked ties and torch."""
import numpy as np
import pytest

import synth
from oracle import ptc, wilson

DIMS = (4, 4, 4, 4)


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _gauge_transform(U, g, dims):
    """U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger."""
    lx, ly, lz, lt = dims
    gl = g.reshape(lt, lz, ly, lx, 3, 3)
    out = np.empty_like(U)
    for mu, ax in zip(range(4), (3, 2, 1, 0)):
        gf = np.roll(gl, -1, axis=ax).reshape(-1, 3, 3)
        out[mu] = g @ U[mu] @ np.conj(np.swapaxes(gf, -1, -2))
    return out


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_wilson_weights_give_the_wilson_matrix(dims):
    U = synth.su3_links(dims, 4)
    psi = synth.gaussian_spinor(dims, 9)
    kappa = 0.137
    out = ptc.layer(ptc.wilson_weights(kappa), U, psi[None], dims)[0]
    ref = wilson.apply_D(U, psi, kappa, dims)
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()


def test_opposite_transports_cancel():
    U = synth.su3_links(DIMS, 5)
    psi = synth.gaussian_spinor(DIMS, 1)
    for mu in range(4):
        for s in (+1, -1):
            o = ptc.offset_index(mu, s)
            back = ptc.transport(U, ptc.transport(U, psi, DIMS, o), DIMS, ptc.opposite(o))
            assert np.abs(back - psi).max() <= 1e-13
    # and a forward transport is a genuine hop: on the free field it is a shift
    one = synth.unit_links(DIMS)
    t = ptc.transport(one, psi, DIMS, ptc.offset_index(0, +1)).reshape(4, 4, 4, 4, 4, 3)
    assert np.array_equal(t, np.roll(psi.reshape(4, 4, 4, 4, 4, 3), -1, axis=3))


def test_layer_is_gauge_covariant():
    rng = np.random.default_rng(3)
    U = synth.su3_links(DIMS, 6)
    g = synth.random_su3_gauge_transform(DIMS, 23)
    W = _rand_c(rng, (9, 3, 2, 4, 4))
    x = _rand_c(rng, (2, 256, 4, 3))
    Up = _gauge_transform(U, g, DIMS)
    gx = np.einsum("vij,cvsj->cvsi", g, x)
    lhs = ptc.layer(W, Up, gx, DIMS)
    rhs = np.einsum("vij,cvsj->cvsi", g, ptc.layer(W, U, x, DIMS))
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


def test_adjoint_layer():
    rng = np.random.default_rng(4)
    U = synth.su3_links(DIMS, 7)
    W = _rand_c(rng, (9, 3, 2, 4, 4))
    a = _rand_c(rng, (3, 256, 4, 3))
    b = _rand_c(rng, (2, 256, 4, 3))
    lhs = np.vdot(a, ptc.layer(W, U, b, DIMS))
    rhs = np.vdot(ptc.layer_adjoint(W, U, a, DIMS), b)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _net_loss(Ws, U, eta, Vk):
    f, _ = ptc.forward(Ws, U, eta, DIMS)
    return ptc.subspace_loss(Vk, f)[0]


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(8)
    U = synth.su3_links(DIMS, 8)
    widths = (1, 2, 2, 1)
    Ws = [0.3 * _rand_c(rng, (9, widths[i + 1], widths[i], 4, 4)) for i in range(3)]
    eta = _rand_c(rng, (256, 4, 3))
    # a subspace holding about half of f, so that the loss has O(1) sensitivity
    f0 = ptc.forward(Ws, U, eta, DIMS)[0].reshape(-1)
    noise = _rand_c(rng, 3072) * np.linalg.norm(f0) / np.sqrt(3072)
    Vk, _ = np.linalg.qr(np.stack([f0 + noise, _rand_c(rng, 3072), _rand_c(rng, 3072)], axis=1))
    f, inputs = ptc.forward(Ws, U, eta, DIMS)
    L, gf = ptc.subspace_loss(Vk, f)
    grads, geta = ptc.backward(Ws, U, inputs, gf.reshape(256, 4, 3), DIMS)
    h = 1e-5         # central differences: O(h^2) truncation ~1e-10, rounding ~1e-11
    # weights: three random complex directions per layer
    for li in range(3):
        for _ in range(3):
            d = _rand_c(rng, Ws[li].shape)
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[li] = Ws[li] + h * d
            Wm[li] = Ws[li] - h * d
            fd = (_net_loss(Wp, U, eta, Vk) - _net_loss(Wm, U, eta, Vk)) / (2 * h)
            an = np.real(np.vdot(grads[li], d))          # Re(conj(G) . d)
            assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3 * L)
    # input: two random complex directions
    for _ in range(2):
        d = _rand_c(rng, eta.shape)
        fd = (_net_loss(Ws, U, eta + h * d, Vk) - _net_loss(Ws, U, eta - h * d, Vk)) / (2 * h)
        an = np.real(np.vdot(geta, d))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3 * L)


def test_subspace_loss_values():
    rng = np.random.default_rng(9)
    Vk, _ = np.linalg.qr(_rand_c(rng, (50, 4)))
    inside = Vk @ _rand_c(rng, 4)
    assert ptc.subspace_loss(Vk, inside)[0] <= 1e-28
    perp = _rand_c(rng, 50)
    perp -= Vk @ (Vk.conj().T @ perp)
    L, g = ptc.subspace_loss(Vk, perp)
    assert abs(L - 1.0) <= 1e-14
    # scale invariance: the gradient is orthogonal to f
    f = _rand_c(rng, 50)
    L, g = ptc.subspace_loss(Vk, f)
    assert abs(np.vdot(f, g).real) <= 1e-12 * np.linalg.norm(f) * np.linalg.norm(g)


def test_round_bf16():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-3])
    r = ptc.round_bf16(x).real
    assert r[0] == 1.0
    assert r[1] == 1.0                       # tie -> even
    assert r[2] == 1.0 + 2.0 ** -6           # tie -> even
    assert r[3] == -2.5
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    v = rng.standard_normal(1000) * 10.0 ** rng.uniform(-5, 5, 1000)
    t = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ptc.round_bf16(v).real, t)
