"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws random numbers and applies the input recipe for the gauge
links; it holds none of the deflated-Lanczos arithmetic (no Wilson operator, no
Krylov step).  Both the CPU oracle and the CUDA path take their inputs from
here, so the two sides see bit-identical inputs.

Conventions (shared by every consumer, implemented separately by each):
  * lattice dims = (Lx, Ly, Lz, Lt); site s = ((t*Lz + z)*Ly + y)*Lx + x,
    x fastest;
  * a spinor is complex128 of shape (V, 4, 3): 4 spins x 3 colours, component
    a = 3*spin + colour;
  * a gauge field is complex128 of shape (4, V, 3, 3): U[mu][s] is the link
    from s to s+mu_hat (mu = 0..3 <-> x, y, z, t), row-major.

The paper's own lattice workload (a quenched beta=6.0 20^3x32 configuration
at kappa=0.15720, Sec. 2) is not available; the near-free random SU(3) links
below stand in for it.
"""
from __future__ import annotations

import json
import os

import numpy as np

__all__ = [
    "volume", "su3_links", "unit_links", "random_su3_gauge_transform",
    "gaussian_spinor", "gaussian_spinors", "point_source", "kappa_for",
    "diag_hpd_1000", "diag_indefinite_1000", "WORKLOADS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
KAPPA_TABLE = os.path.join(_HERE, "kappa_table.json")


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def _expi_hermitian(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*h) for a stack of hermitian 3x3 matrices, by eigendecomposition."""
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ik,...k,...jk->...ij", v, ph, v.conj())


def su3_links(dims, seed: int, eps: float = 0.3) -> np.ndarray:
    """SU(3) links U = exp(i*eps*H), H hermitian traceless with Gaussian entries.

    For each (mu, s) in index order a 3x3 matrix A with independent
    re, im ~ N(0,1) entries is drawn from numpy's default_rng(seed);
    H = (A + A^dagger)/2 - tr(H)/3.  Returns complex128 of shape (4, V, 3, 3).
    """
    V = volume(dims)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((4, V, 3, 3, 2))
    a = g[..., 0] + 1j * g[..., 1]
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    return _expi_hermitian(h, eps)


def unit_links(dims) -> np.ndarray:
    """The free field U = 1."""
    V = volume(dims)
    u = np.zeros((4, V, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def random_su3_gauge_transform(dims, seed: int) -> np.ndarray:
    """One random SU(3) matrix g(x) per site, shape (V, 3, 3) (same recipe, eps=1)."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((V, 3, 3, 2))
    a = g[..., 0] + 1j * g[..., 1]
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    return _expi_hermitian(h, 1.0)


def gaussian_spinor(dims, seed: int) -> np.ndarray:
    """Complex Gaussian spinor (re, im ~ N(0,1) per component), shape (V, 4, 3)."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((V, 4, 3, 2))
    return g[..., 0] + 1j * g[..., 1]


def gaussian_spinors(dims, seeds) -> np.ndarray:
    """Stack of gaussian_spinor(dims, s) for s in seeds, shape (N, V, 4, 3)."""
    return np.stack([gaussian_spinor(dims, s) for s in seeds])


def point_source(dims, spin: int, colour: int, site: int = 0) -> np.ndarray:
    """Unit vector at one site, spin and colour (the origin by default)."""
    V = volume(dims)
    b = np.zeros((V, 4, 3), dtype=np.complex128)
    b[site, spin, colour] = 1.0
    return b


def kappa_for(dims, seed: int) -> float:
    """kappa with min|eig(gamma5 D)| = 1e-3 for the links su3_links(dims, seed).

    The values are computed by the FP64 oracle (synth/make_kappa_table.py) and
    stored in synth/kappa_table.json; this function only looks them up.
    """
    key = "x".join(str(int(d)) for d in dims) + f"_s{int(seed)}"
    with open(KAPPA_TABLE) as f:
        table = json.load(f)
    if key not in table:
        raise KeyError(f"kappa for {key} not in {KAPPA_TABLE}; run synth/make_kappa_table.py")
    return float(table[key]["kappa"])


def diag_hpd_1000() -> np.ndarray:
    """Diagonal of the positive definite example of Sec. 1: 0.1, 1, 2, ..., 999."""
    return np.concatenate([[0.1], np.arange(1.0, 1000.0)])


def diag_indefinite_1000(negatives: int = 22):
    """Diagonal of the indefinite example of Sec. 1: N(0,1) entries shifted by +2.0.

    The paper does not give the seed; the first seed s = 0, 1, ... of
    default_rng(s).normal(size=1000) + 2.0 with exactly `negatives` negative
    entries is taken.  Returns (diagonal, seed).
    """
    s = 0
    while True:
        d = np.random.default_rng(s).normal(size=1000) + 2.0
        if int((d < 0).sum()) == negatives:
            return d, s
        s += 1


# Named workloads (lattice, seeds, Krylov sizes).  The gauge seed of each
# lattice and the RHS seeds are fixed here; the right-hand-side recipe is
# stated with each entry.
WORKLOADS = {
    # 4^4 Wilson lattice, Lan-DR and MinRes-DR(40,10) on one Gaussian RHS
    # (seed 0), then D-CG and D-MinRes on 4 Gaussian RHS (seeds 1..4).
    "wilson_4x4x4x4": dict(dims=(4, 4, 4, 4), gauge_seed=1, m=40, k=10,
                           first_rhs_seed=0, rhs_seeds=(1, 2, 3, 4)),
    # 16^3x32 lattice, MinRes-DR(100,40) on the point source (spin 0,
    # colour 0) at the origin, D-MinRes on the other 11 spin-colour point
    # sources.
    "wilson_16x16x16x32": dict(dims=(16, 16, 16, 32), gauge_seed=2, m=100, k=40,
                               point_sources=12),
    # 24^3x48 lattice, Lan-DR(120,60) on D^dagger D for one Gaussian RHS (seed 0),
    # then D-CG on 48 Gaussian RHS (seeds 1..48).
    "wilson_24x24x24x48": dict(dims=(24, 24, 24, 48), gauge_seed=3, m=120, k=60,
                               first_rhs_seed=0, rhs_seeds=tuple(range(1, 49))),
    # 64 lattices of uneven size (lattice i: 8^4, 12^4 or 16^4 for i mod 3 = 0, 1, 2;
    # gauge seed 3000 + i); MinRes-DR(40,10) on one Gaussian RHS (seed 0), then
    # D-MinRes on 8 Gaussian RHS (seeds 1..8) per lattice.
    "uneven_64": dict(sizes=((8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16)), lattices=64,
                      gauge_seed0=3000, m=40, k=10, first_rhs_seed=0, rhs_seeds=tuple(range(1, 9))),
}
