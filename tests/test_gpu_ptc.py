"""GPU parity of the PTC network (forward, backward, subspace loss) and of the
Rayleigh-Ritz seed, against the FP64 oracle (oracle/ptc.py, oracle/krylov.py).

The oracle gets the weights rounded to bfloat16 on the host (oracle.ptc.round_bf16),
which must equal the bfloat16 weights the kernels use (checked bit for bit); what
remains is FP32 arithmetic: forward outputs within 1e-5 of the largest output,
gradients within 2e-4 of the largest gradient entry."""
import numpy as np
import pytest

import synth
from oracle import ptc, wilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    return dlz()


def _rand_weights(widths, seed, scale=0.25):
    rng = np.random.default_rng(seed)
    return [scale * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(9 * shp[2] * 4)
            for shp in [(9, widths[i + 1], widths[i], 4, 4) for i in range(len(widths) - 1)]]


def _setup(m, dims, widths, seed):
    U = synth.su3_links(dims, seed)
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), 0.2)
    Ws = _rand_weights(widths, seed + 100)
    net = m.net_create(op, widths, Ws)
    Wr = [ptc.round_bf16(w.astype(np.complex64)) for w in Ws]
    return U, op, net, Wr


@pytest.mark.parametrize("dims,widths", [((4, 4, 4, 4), (1, 3, 2, 1)), ((4, 2, 6, 4), (1, 4, 8, 1)),
                                         ((4, 4, 4, 4), (1, 12, 16, 1))])
def test_forward_matches_oracle(m, dims, widths):
    U, op, net, Wr = _setup(m, dims, widths, 2)
    # the kernels use exactly the host-rounded bfloat16 weights
    for a, b in zip(m.net_get(net, 2), Wr):
        assert np.array_equal(a.astype(np.complex128), b)
    X = synth.gaussian_spinors(dims, [1, 2, 3])
    f = m.net_forward(net, torch.from_numpy(X.astype(np.complex64)).cuda()).cpu().numpy()
    for i in range(3):
        ref, _ = ptc.forward(Wr, U, X[i], dims)
        assert np.abs(f[i] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_wilson_weights_reproduce_the_stencil(m):
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 3)
    kappa = 0.125                        # -kappa (1 -+ gamma) entries are exact in bfloat16
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    net = m.net_create(op, (1, 1), [ptc.wilson_weights(kappa)])
    x = synth.gaussian_spinor(dims, 4)
    f = m.net_forward(net, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    ref = wilson.apply_D(U, x, kappa, dims)
    assert np.abs(f - ref).max() <= 2e-6 * np.abs(ref).max()


@pytest.mark.parametrize("widths", [(1, 3, 2, 1), (1, 12, 16, 1)])
def test_backward_matches_oracle(m, widths):
    dims = (4, 4, 4, 4)
    U, op, net, Wr = _setup(m, dims, widths, 5)
    X = synth.gaussian_spinors(dims, [7, 8])
    G = synth.gaussian_spinors(dims, [9, 10])
    m.net_forward(net, torch.from_numpy(X.astype(np.complex64)).cuda())
    m.net_zero_grad(net)
    gin = m.net_backward(net, torch.from_numpy(G.astype(np.complex64)).cuda(), want_input_grad=True).cpu().numpy()
    grads = m.net_get(net, 1)
    ref_w = [np.zeros_like(w) for w in Wr]
    for i in range(2):
        _, inputs = ptc.forward(Wr, U, X[i], dims)
        gw, gx = ptc.backward(Wr, U, inputs, G[i], dims)
        for li in range(len(Wr)):
            ref_w[li] += gw[li]
        assert np.abs(gin[i] - gx).max() <= 1e-5 * np.abs(gx).max()
    for a, b in zip(grads, ref_w):
        assert np.abs(a - b).max() <= 2e-4 * np.abs(b).max()
    # a second backward adds to the gradients; zero_grad clears them
    m.net_backward(net, torch.from_numpy(G.astype(np.complex64)).cuda())
    for a, b in zip(m.net_get(net, 1), ref_w):
        assert np.abs(a - 2 * b).max() <= 4e-4 * np.abs(b).max()
    m.net_zero_grad(net)
    assert all(np.count_nonzero(a) == 0 for a in m.net_get(net, 1))


def test_seed_deflation_and_subspace_loss_match_oracle(m):
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 6)
    kappa = 0.2
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    F = synth.gaussian_spinors(dims, list(range(20, 26)))
    defl = m.seed_deflation(op, torch.from_numpy(F).cuda(), which=m.DDAGD)
    A = wilson.operator(U, kappa, dims, "DdagD")
    Qo, _ = np.linalg.qr(F.reshape(6, -1).T)
    H = Qo.conj().T @ np.stack([A(Qo[:, i]) for i in range(6)], axis=1)
    ref = np.linalg.eigvalsh(0.5 * (H + H.conj().T))
    vals = np.array([m.defl_get(defl, i)[0] for i in range(6)])
    assert np.allclose(np.sort(vals), ref, rtol=1e-10, atol=0)
    # subspace loss of other vectors against that span
    Fx = synth.gaussian_spinors(dims, [40, 41, 42]).astype(np.complex64)
    loss, g = m.subspace_loss(defl, torch.from_numpy(Fx).cuda())
    g = g.cpu().numpy()
    for i in range(3):
        L, gr = ptc.subspace_loss(Qo, Fx[i].astype(np.complex128))
        assert abs(loss[i] - L) <= 1e-6 * L
        assert np.abs(g[i].reshape(-1) - gr).max() <= 1e-5 * np.abs(gr).max()
    # vectors inside the span have zero loss
    inside = (Qo @ (np.arange(6) + 1j)).reshape(256, 4, 3).astype(np.complex64)
    li, _ = m.subspace_loss(defl, torch.from_numpy(inside).cuda(), want_grad=False)
    assert li[0] <= 1e-12


def test_adam_step_and_training_lower_the_loss(m):
    """Adam on the master weights (checked against the textbook update on the
    host), and a short training run that lowers the subspace loss of the network's
    outputs against a fixed deflation set."""
    dims = (4, 4, 4, 4)
    U, op, net, _ = _setup(m, dims, (1, 4, 4, 1), 7)
    F = synth.gaussian_spinors(dims, list(range(60, 64)))
    defl = m.seed_deflation(op, torch.from_numpy(F).cuda(), which=m.DDAGD)
    X = torch.from_numpy(synth.gaussian_spinors(dims, [70, 71]).astype(np.complex64)).cuda()
    w0 = [w.astype(np.complex128) for w in m.net_get(net, 0)]
    f = m.net_forward(net, X)
    loss0, g = m.subspace_loss(defl, f)
    m.net_backward(net, g)
    gr = [w.astype(np.complex128) for w in m.net_get(net, 1)]
    m.net_adam_step(net, 1e-3)
    w1 = m.net_get(net, 0)
    for a, b, gg in zip(w1, w0, gr):
        # first Adam step: w - lr * g / (|g| + eps), per real component
        exp = b - 1e-3 * (gg.real / (np.abs(gg.real) + 1e-8) + 1j * gg.imag / (np.abs(gg.imag) + 1e-8))
        assert np.abs(a - exp).max() <= 1e-6
    assert all(np.count_nonzero(a) == 0 for a in m.net_get(net, 1))
    for _ in range(60):
        f = m.net_forward(net, X)
        loss, g = m.subspace_loss(defl, f)
        m.net_backward(net, g)
        m.net_adam_step(net, 3e-3)
    assert loss.mean() < 0.9 * loss0.mean()
