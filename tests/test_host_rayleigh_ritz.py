"""The Rayleigh-Ritz step of a deflation set (csrc/solvers.cu, dlz_host_rayleigh_ritz) on
CPU against SciPy's generalized hermitian eigensolver (LAPACK): with the Gram matrix of a
basis that is orthonormal only to FP32 rounding, each value must be the Rayleigh quotient
of its vector V z, and the vectors G-orthonormal; without it, the plain eigenpairs of H.
The test builds V, A and H = V^dag A V, G = V^dag V explicitly, so the pairs are also
checked against the Rayleigh quotients of y = V z computed directly."""
import numpy as np
import pytest

scipy_linalg = pytest.importorskip("scipy.linalg")

from tests._lib import dlz  # noqa: E402


def _hermitian(rng, n, scale=1.0):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return scale * (A + A.conj().T) / 2


@pytest.mark.parametrize("k,n,seed", [(1, 8, 0), (6, 50, 1), (40, 300, 2), (60, 400, 3)])
def test_generalized_pairs_are_rayleigh_quotients(k, n, seed):
    m = dlz()
    rng = np.random.default_rng(seed)
    A = _hermitian(rng, n)
    # an orthonormal basis perturbed at the FP32 level: V^dag V = 1 + O(1e-6)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    V = Q + 1e-6 * (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    H = V.conj().T @ A @ V
    G = V.conj().T @ V
    w, Z = m.host_rayleigh_ritz(H, G)
    ref = scipy_linalg.eigh(H, G, eigvals_only=True)
    scale = max(1.0, np.abs(ref).max())
    assert np.all(np.diff(w) >= -1e-12 * scale)
    assert np.abs(w - ref).max() <= 1e-11 * scale
    # H z = value G z, z^dag G z = 1, and the value is the Rayleigh quotient of y = V z
    assert np.abs(H @ Z - G @ Z * w).max() <= 1e-10 * scale
    assert np.abs(Z.conj().T @ G @ Z - np.eye(k)).max() <= 1e-10
    Y = V @ Z
    rq = np.einsum("ij,ij->j", Y.conj(), A @ Y).real / np.einsum("ij,ij->j", Y.conj(), Y).real
    assert np.abs(rq - w).max() <= 1e-11 * scale
    assert np.abs(np.linalg.norm(Y, axis=0) - 1.0).max() <= 1e-10


def test_without_gram_matrix_the_eigenpairs_of_h():
    m = dlz()
    rng = np.random.default_rng(7)
    H = _hermitian(rng, 30, scale=3.0)
    w, Z = m.host_rayleigh_ritz(H)
    ref, _ = np.linalg.eigh(H)
    assert np.abs(w - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(Z.conj().T @ Z - np.eye(30)).max() <= 1e-12
    assert np.abs(H @ Z - Z * w).max() <= 1e-11 * np.abs(ref).max()


def test_clustered_values_and_an_indefinite_gram_matrix():
    m = dlz()
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 20)) + 1j * rng.standard_normal((20, 20)))
    lam = np.concatenate([np.full(5, 1e-6), np.linspace(1e-3, 2.0, 15)])
    H = (Q * lam) @ Q.conj().T
    H = (H + H.conj().T) / 2
    w, Z = m.host_rayleigh_ritz(H, np.eye(20))
    assert np.abs(w - np.sort(lam)).max() <= 1e-13
    assert np.abs(Z.conj().T @ Z - np.eye(20)).max() <= 1e-12
    G = np.eye(20, dtype=np.complex128)
    G[3, 3] = -1.0
    with pytest.raises(m.DlzError) as e:
        m.host_rayleigh_ritz(H, G)
    assert e.value.code == m.ERR_BREAKDOWN
