"""The library's complex host helpers (GMRES-DR's small problem) against LAPACK through
NumPy, on CPU: eigenvalues of general complex matrices (random, non-normal, with a
cluster, and the harmonic-Ritz matrix of an Arnoldi run), eigenvector residuals, and
complex least squares with the orthogonal-complement vector."""
import numpy as np
import pytest

from tests._lib import dlz


def _match(a, b):
    """max distance between two multisets of complex numbers (greedy nearest pairing)."""
    b = list(b)
    worst = 0.0
    for x in a:
        i = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b[i]))
        b.pop(i)
    return worst


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (40, 3), (121, 4)])
def test_zgeev_random(n, seed):
    m = dlz()
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    w, Z = m.host_zgeev(A)
    ref = np.linalg.eigvals(A)
    assert _match(w, ref) <= 1e-10 * np.abs(ref).max()
    for j in range(n):
        assert np.linalg.norm(A @ Z[:, j] - w[j] * Z[:, j]) <= 1e-10 * np.linalg.norm(A, 2)
        assert abs(np.linalg.norm(Z[:, j]) - 1) < 1e-12


def test_zgeev_nonnormal_and_clustered():
    m = dlz()
    rng = np.random.default_rng(9)
    n = 60
    d = np.concatenate([np.full(5, 1.0 + 0.5j), 2.0 + rng.standard_normal(n - 5) + 1j * rng.standard_normal(n - 5)])
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = S @ np.diag(d) @ np.linalg.inv(S)
    w, Z = m.host_zgeev(A)
    assert _match(w, d) <= 1e-6 * np.abs(d).max()
    for j in range(n):
        assert np.linalg.norm(A @ Z[:, j] - w[j] * Z[:, j]) <= 1e-8 * np.linalg.norm(A, 2)


def test_zgeev_rejects_nonfinite():
    m = dlz()
    A = np.eye(3, dtype=complex)
    A[1, 2] = np.nan
    with pytest.raises(m.DlzError):
        m.host_zgeev(A)


@pytest.mark.parametrize("rows,cols", [(6, 5), (41, 40), (30, 12)])
def test_zlstsq(rows, cols):
    m = dlz()
    rng = np.random.default_rng(rows)
    A = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
    c = rng.standard_normal(rows) + 1j * rng.standard_normal(rows)
    y, q = m.host_zlstsq(A, c)
    ref, *_ = np.linalg.lstsq(A, c, rcond=None)
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    if q is not None:
        assert abs(np.linalg.norm(q) - 1) < 1e-13
        assert np.abs(A.conj().T @ q).max() < 1e-12 * np.abs(A).max()
