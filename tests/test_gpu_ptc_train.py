"""The learned seed end to end on a small lattice: Lan-DR eigenvectors of
training fields, Adam training through the library's kernels, and the seeded
versus plain Lan-DR deflation sets on held-out fields (what the trained network
gains over the untrained one, and the fallback rule)."""
import numpy as np
import pytest

import synth
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (8, 8, 8, 8)
KAPPA = 0.2
M, K = 30, 10


@pytest.fixture(scope="module")
def m():
    return dlz()


def _field(m, seed):
    op = m.create_operator(DIMS, torch.from_numpy(synth.su3_links(DIMS, seed)).cuda(), KAPPA)
    b = torch.from_numpy(synth.gaussian_spinor(DIMS, 0)).cuda()
    _, d, st = m.landr(op, b, m.params_default(m=M, k=K, tol=1e-10, max_cycles=200, precision=m.F32))
    assert st.converged == 1
    return op, d


def test_training_lowers_held_out_loss_and_fallback_rule(m):
    from paper_0901_3163_gb300 import ptc_train as T
    train = [_field(m, 300 + i) for i in range(4)]
    held = [_field(m, 400 + i) for i in range(2)]
    widths = T.default_widths()
    W0 = T.init_weights(widths, 1)
    net = m.net_create(train[0][0], widths, W0)
    net0 = m.net_create(held[0][0], widths, W0)          # untrained copy

    def held_loss(n):
        tot = []
        for op, d in held:
            m.net_bind(n, op)
            g = torch.Generator(device="cuda")
            g.manual_seed(5)
            f = m.net_forward(n, T.noise(torch, op, 4, g))
            tot.append(m.subspace_loss(d, f, want_grad=False)[0].mean())
        return float(np.mean(tot))

    before = held_loss(net)
    hist = T.train(torch, net, [o for o, _ in train], [d for _, d in train], steps=120, nvec=4, lr=3e-3)
    assert np.mean(hist[-20:]) < np.mean(hist[:20])
    after = held_loss(net)
    assert after < before
    op, _ = held[0]
    bl = [torch.from_numpy(synth.gaussian_spinor(DIMS, s)).cuda() for s in (10, 11, 12)]
    r = T.evaluate(torch, net, op, bl, M, K, net_untrained=net0)
    print("learned seed vs plain Lan-DR at equal MVPs:", {k_: r[k_] for k_ in (
        "seed_mvps", "plain_equal_mvps", "ritz_median_seed", "ritz_median_plain", "ritz_median_untrained",
        "dcg_iters_seed", "dcg_iters_plain_equal", "cg_iters_undeflated", "chosen")})
    assert r["converged"]
    # the two sets cost the same budget: 2k applications of D or D^dag against
    # 2(k+1) + 2 (Lanczos steps, D^dag b and the true residual)
    assert abs(r["plain_equal_mvps"] - r["seed_mvps"]) <= 4
    assert r["ritz_median_seed"] < r["ritz_median_untrained"]
    assert r["chosen"] == ("seed" if r["ritz_median_seed"] <= r["ritz_median_plain"] else "plain Lan-DR")
    # what training gains over the method without it, at the same budget: nothing here.
    # One Lan-DR(k+1, k) cycle's Krylov space beats the trained network's outputs (median
    # Ritz residual 0.46 against 1.01 on GB300, a factor 2.2), so the fallback keeps
    # plain Lan-DR; the assertion holds that margin with room for run-to-run noise
    assert r["ritz_median_plain"] * 1.5 <= r["ritz_median_seed"]
    assert r["chosen"] == "plain Lan-DR"
    # deflation by either set never costs iterations over undeflated CG
    assert max(r["dcg_iters_plain_cycle"]) <= max(r["cg_iters_undeflated"])
