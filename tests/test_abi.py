"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and its host-side helpers (small dense solvers of the
restart, argument validation, error names) behave."""
import ctypes

import numpy as np
import pytest

from tests._lib import dlz


def test_library_exports_every_declared_symbol():
    m = dlz()
    syms = m.header_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(m.lib, s), s


def test_every_declared_call_cites_its_passage():
    """Each entry point of include/dlz.h sits under a comment that names the passage
    of the paper defining the operation (a section, or one of the paper's references),
    or says that the paper has no counterpart (interface, checkpoint, measurement)."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dlz.h")
    text = open(path).read()
    body = text[text.index("#ifndef DLZ_H"):]
    cite = re.compile(r"Sec\. ?\d|refs?\. \[\d|no counterpart|not in the paper")
    missing = []
    for m in re.finditer(r"^[a-z][\w \*]*?\b(dlz_\w+)\(", body, re.M):
        before = body[: m.start()]
        end = before.rfind("*/")
        start = before.rfind("/*", 0, end)
        # the comment must belong to this declaration's group: only declarations
        # (and their continuation lines) between it and the call
        between = before[end + 2:]
        assert "{" not in between and "#define" not in between, m.group(1)
        if not cite.search(before[start:end]):
            missing.append(m.group(1))
    assert not missing, missing


def test_params_defaults():
    m = dlz()
    p = m.params_default()
    assert (p.m, p.k, p.tol, p.oversolve, p.reorth_period, p.precision) == (40, 10, 1e-10, 1.0, 10, m.F64)
    assert p.reliable_delta == 1e-2 and p.finish == 0 and p.eig_only == 0


def test_error_names():
    m = dlz()
    for code, name in [(0, "DLZ_OK"), (-1, "DLZ_ERR_BADARG"), (-2, "DLZ_ERR_BAD_GAUGE"),
                       (-4, "DLZ_ERR_NOT_CONVERGED"), (-9, "DLZ_ERR_IO")]:
        assert m.strerror(code) == name


@pytest.mark.parametrize("n", [1, 2, 7, 40, 121])
def test_host_symeig_matches_lapack(n):
    m = dlz()
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w, Z = m.host_symeig(A)
    assert np.abs(w - np.linalg.eigvalsh(A)).max() < 1e-13 * max(1, np.abs(w).max())
    assert np.abs(A @ Z - Z * w).max() < 1e-12 * max(1, np.abs(w).max())
    assert np.abs(Z.T @ Z - np.eye(n)).max() < 1e-13


@pytest.mark.parametrize("scale", [1e-200, 1e200])
def test_host_symeig_extreme_scales(scale):
    """Entries near the ends of the double range: the reduction scales them first."""
    m = dlz()
    rng = np.random.default_rng(4)
    B = rng.standard_normal((30, 30))
    A = (B + B.T) * scale
    w, Z = m.host_symeig(A)
    w0 = np.linalg.eigvalsh(B + B.T) * scale
    assert np.abs(w - w0).max() <= 1e-13 * np.abs(w0).max()
    assert np.abs(Z.T @ Z - np.eye(30)).max() < 1e-13


def test_host_symeig_arrowhead_with_clusters():
    """The Lan-DR restart matrix: diagonal block of Ritz values, one coupling row."""
    m = dlz()
    k, n = 10, 40
    rng = np.random.default_rng(3)
    T = np.zeros((n, n))
    T[:k, :k] = np.diag(np.sort(rng.uniform(1e-6, 1e-3, k)))
    T[k, :k] = T[:k, k] = rng.standard_normal(k) * 1e-9
    for j in range(k, n):
        T[j, j] = rng.uniform(0.5, 4)
        if j + 1 < n:
            T[j, j + 1] = T[j + 1, j] = rng.uniform(0.1, 1)
    w, Z = m.host_symeig(T)
    assert np.abs(w - np.linalg.eigvalsh(T)).max() < 1e-14 * 4


@pytest.mark.parametrize("case", ["dense", "arrowhead", "indefinite", "one", "huge", "tiny"])
def test_host_sym_extremes(case):
    """Smallest and largest eigenvalue by Sturm bisection, against LAPACK."""
    m = dlz()
    rng = np.random.default_rng(11)
    if case == "one":
        A = np.array([[2.5]])
    elif case == "arrowhead":             # the MinRes-DR restart matrix: dense block, then a band
        n, k = 100, 40
        A = np.zeros((n, n))
        B = rng.standard_normal((k + 1, k + 1)) * 1e-3
        A[:k + 1, :k + 1] = B + B.T
        for j in range(k + 1, n):
            A[j, j] = rng.uniform(-2, 2)
            A[j, j - 1] = A[j - 1, j] = rng.uniform(0.1, 1)
    else:
        n = 60
        A = rng.standard_normal((n, n))
        A = A + A.T
        if case == "indefinite":
            A += np.diag(np.linspace(-50, 50, n))
        A *= {"huge": 1e200, "tiny": 1e-200}.get(case, 1.0)
    lo, hi = m.host_sym_extremes(A)
    w = np.linalg.eigvalsh(A)
    scale = np.abs(w).max()
    assert abs(lo - w[0]) <= 1e-13 * scale and abs(hi - w[-1]) <= 1e-13 * scale


@pytest.mark.parametrize("rows,cols", [(5, 4), (41, 40), (101, 100), (30, 12)])
def test_host_lstsq(rows, cols):
    m = dlz()
    rng = np.random.default_rng(rows)
    T = rng.standard_normal((rows, cols))
    c = rng.standard_normal(rows)
    y, q = m.host_lstsq(T, c)
    assert np.abs(y - np.linalg.lstsq(T, c, rcond=None)[0]).max() < 1e-11
    if q is not None:
        assert abs(np.linalg.norm(q) - 1) < 1e-14 and np.abs(T.T @ q).max() < 1e-13


def test_argument_validation_without_gpu():
    m = dlz()
    out = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 0, 4, 4)
    g = np.zeros(16, dtype=np.complex128)
    assert m.lib.dlz_create_operator(bad, g.ctypes.data, 0.1, 1, None, ctypes.byref(out)) == m.ERR_BADARG
    dims = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert m.lib.dlz_create_operator(dims, g.ctypes.data, 0.1, 2, None, ctypes.byref(out)) == m.ERR_BADARG
    assert m.lib.dlz_create_operator(dims, None, 0.1, 1, None, ctypes.byref(out)) == m.ERR_BADARG
    assert m.lib.dlz_create_operator(dims, g.ctypes.data, float("nan"), 1, None, ctypes.byref(out)) == m.ERR_BADARG
    assert m.lib.dlz_destroy_operator(None) == m.ERR_BADARG
    assert m.lib.dlz_apply(None, 0, None, None, 0, 1) == m.ERR_BADARG
    assert m.lib.dlz_defl_count(None, None, None) == m.ERR_BADARG
    assert "null" in m.last_error()
    # even-odd entries: odd extents and null operators are rejected before any GPU work
    odd = (ctypes.c_int * 4)(4, 4, 3, 4)
    assert m.lib.dlz_create_operator_eo(odd, g.ctypes.data, 0.1, 1, None, ctypes.byref(out)) == m.ERR_BADARG
    assert "even" in m.last_error()
    assert m.lib.dlz_eo_prepare(None, None, None, 1) == m.ERR_BADARG
    assert m.lib.dlz_eo_reconstruct(None, None, None, None, 1) == m.ERR_BADARG


def test_argument_validation_of_batch_network_and_noalloc_entries_without_gpu():
    """The multi-lattice, network, seed and no-allocation entry points reject null or
    out-of-range arguments before touching a GPU."""
    m = dlz()
    out = ctypes.c_void_p()
    p = m.params_default()
    z = (ctypes.c_int * 1)(0)
    assert m.lib.dlz_batch_dminres(0, None, None, None, None, z, ctypes.byref(p), None) == m.ERR_BADARG
    ops = (ctypes.c_void_p * 1)(None)
    ptrs = (ctypes.c_void_p * 1)(None)
    one = (ctypes.c_int * 1)(1)
    assert m.lib.dlz_batch_dminres(1, ops, None, ptrs, ptrs, one, ctypes.byref(p), None) == m.ERR_BADARG
    widths = (ctypes.c_int * 4)(1, 12, 16, 1)
    assert m.lib.dlz_net_create(None, 3, widths, None, ctypes.byref(out)) == m.ERR_BADARG
    assert m.lib.dlz_net_forward(None, None, 1, None) == m.ERR_BADARG
    assert m.lib.dlz_net_backward(None, None, 1, None) == m.ERR_BADARG
    assert m.lib.dlz_net_adam_step(None, 1e-3, 0.9, 0.999, 1e-8) == m.ERR_BADARG
    assert m.lib.dlz_net_bind(None, None) == m.ERR_BADARG
    assert m.lib.dlz_subspace_loss(None, None, 1, 1.0, None, None) == m.ERR_BADARG
    assert m.lib.dlz_seed_deflation(None, m.DDAGD, None, m.F64, 4, ctypes.byref(out)) == m.ERR_BADARG
    assert m.lib.dlz_apply_noalloc(None, 0, None, None, m.F64, 1) == m.ERR_BADARG
    bad_params = m.params_default()
    bad_params.finish = 2
    assert m.lib.dlz_batch_dminres(1, ops, None, ptrs, ptrs, one, ctypes.byref(bad_params), None) == m.ERR_BADARG
