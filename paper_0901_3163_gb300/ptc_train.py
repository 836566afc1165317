"""Training and use of the learned deflation seed (the PTC network of dlz.h).

The network maps complex Gaussian noise to vectors that should lie in the
low-eigenvector space of D^dagger D.  Training minimises the mean subspace
residual ||(1 - V V^dag) f||^2 / ||f||^2 of its outputs against the k
eigenvectors V that Lan-DR computed on each training field; every step runs
the library's kernels (forward, subspace loss, backward, Adam).  The seed of a
new field is the Rayleigh-Ritz set over k network outputs
(dlz_seed_deflation); plain Lan-DR stays the fallback, chosen whenever its
Ritz residuals are lower (arXiv:0901.3163 itself builds the deflation space
with Lan-DR only, Sec. 2).
"""
from __future__ import annotations

import time

import numpy as np

from . import dlz


def default_widths():
    """Three layers, 1 -> 12 -> 16 -> 1 complex spinor channels."""
    return (1, 12, 16, 1)


def init_weights(widths, seed, scale=1.0):
    """Complex Gaussian weights scaled so each layer roughly preserves the norm;
    the site term starts near the identity (a network that begins as a mild filter)."""
    rng = np.random.default_rng(seed)
    Ws = []
    for shp in dlz.net_weight_shapes(widths):
        w = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) * (scale / np.sqrt(2 * 9 * shp[2] * 4))
        for c in range(min(shp[1], shp[2])):
            w[0, c, c] += np.eye(4) / np.sqrt(max(shp[2], 1))
        if shp[1] > shp[2]:
            for c in range(shp[2], shp[1]):
                w[0, c, c % shp[2]] += np.eye(4) / np.sqrt(shp[1])
        Ws.append(w)
    return Ws


def noise(torch, op, nvec, gen):
    """nvec complex Gaussian vectors [nvec, V, 4, 3] (complex64) on the operator's device."""
    shape = (nvec, op.volume, 4, 3)
    re = torch.randn(shape, generator=gen, device="cuda")
    im = torch.randn(shape, generator=gen, device="cuda")
    return torch.complex(re, im)


def train(torch, net, ops, defls, steps, nvec=4, lr=3e-3, seed=0, log=None):
    """Adam on the mean subspace loss; each step draws one training field (in a
    seeded order) and nvec noise inputs.  Returns the per-step mean losses."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    hist = []
    for it in range(steps):
        i = int(rng.integers(len(ops)))
        dlz.net_bind(net, ops[i])
        x = noise(torch, ops[i], nvec, gen)
        f = dlz.net_forward(net, x)
        loss, g = dlz.subspace_loss(defls[i], f, grad_scale=1.0 / nvec)   # gradient of the mean
        dlz.net_backward(net, g)
        dlz.net_adam_step(net, lr)
        hist.append(float(loss.mean()))
        if log and (it % 50 == 0 or it == steps - 1):
            log(f"step {it} loss {hist[-1]:.4f}")
    return hist


def seed_set(torch, net, op, k, seed=0, which=dlz.DDAGD):
    """The Rayleigh-Ritz deflation set over k network outputs on noise."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    dlz.net_bind(net, op)
    x = noise(torch, op, k, gen)
    f = dlz.net_forward(net, x)
    return dlz.seed_deflation(op, f, which=which)


def ritz_residual_median(defl):
    k, _ = dlz.defl_count(defl)
    return float(np.median([dlz.defl_get(defl, i)[1] for i in range(k)]))


def evaluate(torch, net, op, b_list, m, k, seed=0, net_untrained=None):
    """Seeded vs plain Lan-DR deflation sets on one field, at an equal MVP budget.

    seeded: Rayleigh-Ritz over k network outputs (k products with D^dag D);
    plain (equal budget): one Lan-DR(k+1, k) cycle on the first right-hand side
    (k+1 products with D^dag D), the Krylov-space set the same budget buys;
    plain (context): one Lan-DR(m, k) cycle (m products).  The set used for the
    remaining solves is the seeded one unless the equal-budget plain set's median
    Ritz residual is lower (fallback).  Returns the medians, the MVPs (applications
    of D or D^dag) each set cost, D-CG iterations to 1e-10 on b_list[1:] for each
    set and undeflated, and which set the rule picks."""
    p_eq = dlz.params_default(m=k + 1, k=k, tol=1e-10, max_cycles=1)
    _, d_eq, st_eq = dlz.landr(op, b_list[0], p_eq)
    p1 = dlz.params_default(m=m, k=k, tol=1e-10, max_cycles=1)
    _, d_plain, st_plain = dlz.landr(op, b_list[0], p1)
    t0 = time.perf_counter()
    d_seed = seed_set(torch, net, op, k, seed)
    torch.cuda.synchronize()
    t_seed = time.perf_counter() - t0
    out = {"seed_mvps": 2 * k, "plain_equal_mvps": int(st_eq.mvps), "plain_m_mvps": int(st_plain.mvps),
           "ritz_median_seed": ritz_residual_median(d_seed),
           "ritz_median_plain": ritz_residual_median(d_eq),
           "ritz_median_plain_m_cycle": ritz_residual_median(d_plain), "seed_seconds": t_seed}
    if net_untrained is not None:
        out["ritz_median_untrained"] = ritz_residual_median(seed_set(torch, net_untrained, op, k, seed))
    pd = dlz.params_default(m=m, k=k, tol=1e-10, max_iter=100000)
    B = torch.stack(list(b_list[1:]))
    _, s_seed = dlz.dcg(op, d_seed, B, pd)
    _, s_eq = dlz.dcg(op, d_eq, B, pd)
    _, s_plain = dlz.dcg(op, d_plain, B, pd)
    _, s_none = dlz.dcg(op, None, B, pd)
    out["dcg_iters_seed"] = [s.iterations for s in s_seed]
    out["dcg_iters_plain_equal"] = [s.iterations for s in s_eq]
    out["dcg_iters_plain_cycle"] = [s.iterations for s in s_plain]
    out["cg_iters_undeflated"] = [s.iterations for s in s_none]
    out["converged"] = all(s.converged == 1 for s in list(s_seed) + list(s_eq) + list(s_plain) + list(s_none))
    out["chosen"] = "seed" if out["ritz_median_seed"] <= out["ritz_median_plain"] else "plain Lan-DR"
    return out
