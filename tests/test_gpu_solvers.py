"""GPU parity of Lan-DR, MinRes-DR, D-CG and D-MinRes against the FP64 oracle,
through the C ABI (arXiv:0901.3163, Sec. 1-2).

Tolerances: every solve reaches a true relative residual ||b - D x||/||b|| <=
1e-10 verified in FP64; two such solutions differ by at most
2e-10 ||b|| / sigma_min(D); Ritz values of converged pairs agree to 1e-8
relative; the first restart cycle (no restart yet, same FP64 algorithm) agrees
element by element to round-off."""
import numpy as np
import pytest

import synth
from oracle import krylov as K
from oracle import wilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (4, 4, 4, 4)
KAPPA = 0.2       # quick case; the kappa-rule workload is tested below


@pytest.fixture(scope="module")
def m():
    return dlz()


@pytest.fixture(scope="module")
def case(m):
    U = synth.su3_links(DIMS, 1)
    op = m.create_operator(DIMS, torch.from_numpy(U).cuda(), KAPPA)
    b = synth.gaussian_spinor(DIMS, 0)
    return U, op, b


def _g5(x):
    return wilson.apply_gamma5(x.reshape(-1, 4, 3)).reshape(-1)


def _ops(U, kappa):
    return (wilson.operator(U, kappa, DIMS, "Q"), wilson.operator(U, kappa, DIMS, "D"),
            wilson.operator(U, kappa, DIMS, "Ddag"), wilson.operator(U, kappa, DIMS, "DdagD"))


def _params(m, **kw):
    base = dict(m=40, k=10, tol=1e-10, oversolve=2.0, max_cycles=400)
    base.update(kw)
    return m.params_default(**base)


def test_first_cycle_matches_oracle_elementwise(m, case):
    U, op, b = case
    Aq, D, Dd, Ad = _ops(U, KAPPA)
    xg, _, st = m.minresdr(op, torch.from_numpy(b).cuda(), _params(m, max_cycles=1), deflate=False)
    xo = K.minresdr(Aq, _g5(b), m=40, k=10, tol=1e-10, max_cycles=1).x
    assert np.abs(xg.cpu().numpy().reshape(-1) - xo).max() <= 1e-11 * np.abs(xo).max()
    xg, _, st = m.landr(op, torch.from_numpy(b).cuda(), _params(m, max_cycles=1), deflate=False)
    xo = K.landr(Ad, Dd(b.reshape(-1)), m=40, k=10, tol=1e-10, max_cycles=1).x
    assert np.abs(xg.cpu().numpy().reshape(-1) - xo).max() <= 1e-11 * np.abs(xo).max()


def _compare_dr(m, defl, st, r_or, xg, xo, bnorm, sigma):
    assert st.converged == 1 and st.true_residual <= 1e-10
    assert np.linalg.norm(xg - xo) <= 2.5e-10 * bnorm / sigma
    k, _ = m.defl_count(defl)
    vals = np.array([m.defl_get(defl, i) for i in range(k)])
    ov = np.sort(r_or.ritz_values)
    order = np.argsort(vals[:, 0])
    gv, gr = vals[order, 0], vals[order, 1]
    orr = r_or.ritz_residuals[np.argsort(r_or.ritz_values)]
    ok = (gr <= 1e-7) & (orr <= 1e-7)
    # the same FP64 algorithm converges the same pairs on both sides (allowing one pair
    # at the threshold), and every pair converged on both sides agrees to 1e-8
    assert ok.sum() >= max(1, int((orr <= 1e-7).sum()) - 1)
    assert np.all(np.abs(gv[ok] - ov[ok]) <= 1e-8 * np.abs(ov[ok]))
    return gv


def test_minresdr_and_dminres_match_oracle(m, case):
    U, op, b = case
    Aq, D, Dd, Ad = _ops(U, KAPPA)
    bnorm = np.linalg.norm(b)
    xg, defl, st = m.minresdr(op, torch.from_numpy(b).cuda(), _params(m))
    ro = K.minresdr(Aq, _g5(b), m=40, k=10, tol=1e-10, oversolve=2.0, max_cycles=400)
    sigma = np.abs(ro.ritz_values).min()
    _compare_dr(m, defl, st, ro, xg.cpu().numpy().reshape(-1), ro.x, bnorm, sigma)
    # D-MinRes on four more right-hand sides, and plain MinRes for comparison
    B = synth.gaussian_spinors(DIMS, [1, 2, 3, 4])
    Xg, sts = m.dminres(op, defl, torch.from_numpy(B).cuda(), _params(m))
    X0, sts0 = m.dminres(op, None, torch.from_numpy(B).cuda(), _params(m))
    H = K.deflation_space(Aq, ro.Vk)
    for i in range(4):
        xo, io = K.dminres(Aq, _g5(B[i]), ro.Vk, H)
        assert sts[i].converged == 1 and sts[i].true_residual <= 1e-10
        assert sts0[i].converged == 1
        nb = np.linalg.norm(B[i])
        assert np.linalg.norm(Xg[i].cpu().numpy().reshape(-1) - xo) <= 2.5e-10 * nb / sigma
        assert sts[i].iterations < sts0[i].iterations
        assert abs(sts[i].iterations - io.iterations) <= 0.1 * io.iterations + 16


def test_landr_and_dcg_match_oracle(m, case):
    U, op, b = case
    Aq, D, Dd, Ad = _ops(U, KAPPA)
    bf = b.reshape(-1)
    bnorm = np.linalg.norm(b)
    xg, defl, st = m.landr(op, torch.from_numpy(b).cuda(), _params(m))
    ro = K.landr(Ad, Dd(bf), m=40, k=10, tol=1e-10, oversolve=2.0, max_cycles=400,
                 residual=lambda xx: np.linalg.norm(bf - D(xx)) / bnorm)
    sigma = np.sqrt(np.min(ro.ritz_values))
    _compare_dr(m, defl, st, ro, xg.cpu().numpy().reshape(-1), ro.x, bnorm, sigma)
    B = synth.gaussian_spinors(DIMS, [1, 2])
    Xg, sts = m.dcg(op, defl, torch.from_numpy(B).cuda(), _params(m))
    _, sts0 = m.dcg(op, None, torch.from_numpy(B).cuda(), _params(m))
    H = K.deflation_space(Ad, ro.Vk)
    for i in range(2):
        xo, io = K.dcg(D, Dd, B[i].reshape(-1), ro.Vk, H)
        assert sts[i].converged == 1 and sts[i].true_residual <= 1e-10
        assert np.linalg.norm(Xg[i].cpu().numpy().reshape(-1) - xo) <= 2.5e-10 * np.linalg.norm(B[i]) / sigma
        assert sts[i].iterations < sts0[i].iterations


def test_kappa_rule_workload_4x4x4x4(m):
    """The 4^4 workload at the kappa of min|eig(gamma5 D)| = 1e-3, MinRes-DR(40,10)."""
    w = synth.WORKLOADS["wilson_4x4x4x4"]
    dims = w["dims"]
    U = synth.su3_links(dims, w["gauge_seed"])
    kappa = synth.kappa_for(dims, w["gauge_seed"])
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    b = synth.gaussian_spinor(dims, w["first_rhs_seed"])
    p = m.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=2000)
    xg, defl, st = m.minresdr(op, torch.from_numpy(b).cuda(), p)
    assert st.converged == 1 and st.true_residual <= 1e-10
    B = synth.gaussian_spinors(dims, w["rhs_seeds"])
    Xg, sts = m.dminres(op, defl, torch.from_numpy(B).cuda(), p)
    Q = wilson.operator(U, kappa, dims, "Q")
    D = wilson.operator(U, kappa, dims, "D")
    for i in range(len(B)):
        assert sts[i].converged == 1 and sts[i].true_residual <= 1e-10
        xi = Xg[i].cpu().numpy().reshape(-1)
        # the oracle's own residual of the GPU solution, and agreement with the oracle solve
        assert np.linalg.norm(B[i].reshape(-1) - D(xi)) <= 1.01e-10 * np.linalg.norm(B[i])
    xo, io = K.minres(Q, _g5(B[0]), tol=1e-10, maxiter=20000)
    x0 = Xg[0].cpu().numpy().reshape(-1)
    assert np.linalg.norm(x0 - xo) <= 2.5e-10 * np.linalg.norm(B[0]) / 1e-3
    assert sts[0].iterations < io.iterations


def test_error_paths(m, case):
    U, op, b = case
    bad = b.copy()
    bad[3, 1, 2] = np.nan
    with pytest.raises(m.DlzError) as e:
        m.dminres(op, None, torch.from_numpy(bad[None]).cuda(), _params(m))
    assert e.value.code == m.ERR_NONFINITE
    X, sts = m.dminres(op, None, torch.from_numpy(b[None]).cuda(), _params(m, max_iter=5, check_every=1))
    assert sts[0].converged == 0 and np.isfinite(X.cpu().numpy()).all()
    Z, stz = m.dminres(op, None, torch.zeros((1,) + b.shape, dtype=torch.complex128, device="cuda"), _params(m))
    assert stz[0].converged == 1 and float(Z.abs().max()) == 0.0
    with pytest.raises(m.DlzError) as e:
        m.minresdr(op, torch.from_numpy(b).cuda(), _params(m, k=40))
    assert e.value.code == m.ERR_BADARG


def test_deflation_save_load_roundtrip(m, case, tmp_path):
    U, op, b = case
    _, defl, _ = m.minresdr(op, torch.from_numpy(b).cuda(), _params(m))
    path = tmp_path / "defl.bin"
    m.defl_save(defl, path)
    d2 = m.defl_load(op, path)
    assert m.defl_count(d2) == m.defl_count(defl)
    for i in range(m.defl_count(defl)[0]):
        v1, r1 = m.defl_get(defl, i)
        v2, r2 = m.defl_get(d2, i)
        assert abs(v1 - v2) <= 1e-12 * abs(v1)
    y = torch.empty(b.shape, dtype=torch.complex128, device="cuda")
    val, res = m.defl_get(d2, 0, y)
    Q = wilson.operator(U, KAPPA, DIMS, "Q")
    yv = y.cpu().numpy().reshape(-1)
    assert abs(np.linalg.norm(yv) - 1) < 1e-12
    assert abs(np.linalg.norm(Q(yv) - val * yv) - res) < 1e-10
    B = synth.gaussian_spinors(DIMS, [7])
    _, s1 = m.dminres(op, defl, torch.from_numpy(B).cuda(), _params(m))
    _, s2 = m.dminres(op, d2, torch.from_numpy(B).cuda(), _params(m))
    assert s1[0].iterations == s2[0].iterations


@pytest.mark.parametrize("minres", [True, False])
def test_mixed_precision_dsolves_reach_fp64_tolerance(m, case, minres):
    """FP32 stencil and vectors inside FP64 defect correction: the FP64-verified
    residual still reaches 1e-10 and x agrees with the FP64 oracle solve."""
    U, op, b = case
    Aq, D, Dd, Ad = _ops(U, KAPPA)
    fn = m.minresdr if minres else m.landr
    _, defl, _ = fn(op, torch.from_numpy(b).cuda(), _params(m))
    B = synth.gaussian_spinors(DIMS, [5, 6, 7])
    p32 = _params(m, precision=m.F32)
    solve = m.dminres if minres else m.dcg
    X32, s32 = solve(op, defl, torch.from_numpy(B).cuda(), p32)
    X64, s64 = solve(op, defl, torch.from_numpy(B).cuda(), _params(m))
    for i in range(len(B)):
        bi = B[i].reshape(-1)
        assert s32[i].converged == 1 and s32[i].true_residual <= 1e-10
        x32 = X32[i].cpu().numpy().reshape(-1)
        # the oracle's FP64 residual of the mixed-precision solution
        assert np.linalg.norm(bi - D(x32)) <= 1.01e-10 * np.linalg.norm(bi)
        x64 = X64[i].cpu().numpy().reshape(-1)
        rel = np.linalg.norm(x32 - x64) / np.linalg.norm(x64)
        assert rel <= 2.5e-10 * np.linalg.norm(bi) / (0.16 * np.linalg.norm(x64)), rel
        assert s32[i].iterations <= 3 * s64[i].iterations + 64


@pytest.mark.parametrize("method", ["minresdr", "landr"])
def test_mixed_precision_dr_first_rhs(m, case, method):
    """FP32 DR phase (FP32 basis and stencil, FP64 small problem, x and residual)
    followed by FP64 defect correction: the first right-hand side still reaches
    1e-10 and the Rayleigh-Ritz values of the FP32-built deflation set match the
    FP64 oracle's converged ones to their residual level."""
    U, op, b = case
    Aq, D, Dd, Ad = _ops(U, KAPPA)
    bf = b.reshape(-1)
    x32, d32, st = getattr(m, method)(op, torch.from_numpy(b).cuda(), _params(m, precision=m.F32))
    assert st.converged == 1 and st.true_residual <= 1e-10
    xv = x32.cpu().numpy().reshape(-1)
    assert np.linalg.norm(bf - D(xv)) <= 1.01e-10 * np.linalg.norm(bf)
    k, _ = m.defl_count(d32)
    vals = np.array([m.defl_get(d32, i) for i in range(k)])
    if method == "minresdr":
        ro = K.minresdr(Aq, _g5(b), m=40, k=10, tol=1e-10, oversolve=2.0, max_cycles=400)
    else:
        bn = np.linalg.norm(bf)
        ro = K.landr(Ad, Dd(bf), m=40, k=10, tol=1e-10, oversolve=2.0, max_cycles=400,
                     residual=lambda xx: np.linalg.norm(bf - D(xx)) / bn)
    ok = (vals[:, 1] <= 1e-4)
    assert ok.sum() >= 3
    for v, r in vals[ok]:
        # an oracle eigenvalue estimate lies within the pair's residual
        assert np.min(np.abs(ro.ritz_values - v)) <= r + 1e-6 * abs(v)
    # and the FP32-built set still deflates: D-MinRes / D-CG in F32 converge faster than without it
    B = synth.gaussian_spinors(DIMS, [11])
    solve = m.dminres if method == "minresdr" else m.dcg
    _, s1 = solve(op, d32, torch.from_numpy(B).cuda(), _params(m, precision=m.F32))
    _, s0 = solve(op, None, torch.from_numpy(B).cuda(), _params(m, precision=m.F32))
    assert s1[0].converged == 1 and s1[0].iterations < s0[0].iterations


@pytest.mark.parametrize("method", ["minresdr", "landr"])
def test_fp64_dr_capped_then_finished(m, case, method):
    """finish = 1: FP64 restart cycles capped at 3 (short of tol), then D-MinRes /
    D-CG from that x over the deflation set just built.  The result reaches 1e-10
    and agrees with the oracle's undeflated solution within 2e-10 ||b|| / sigma_min;
    with finish = 0 the same cap returns not-converged."""
    U, op, b = case
    Aq, D, Dd, Ad = _ops(U, KAPPA)
    bf = b.reshape(-1)
    fn = getattr(m, method)
    _, _, s0 = fn(op, torch.from_numpy(b).cuda(), _params(m, max_cycles=3), deflate=False)
    assert s0.converged == 0 and s0.true_residual > 1e-10
    xg, d, st = fn(op, torch.from_numpy(b).cuda(), _params(m, max_cycles=3, finish=1))
    assert st.converged == 1 and st.true_residual <= 1e-10 and st.cycles == 3
    assert st.iterations > s0.iterations
    xv = xg.cpu().numpy().reshape(-1)
    assert np.linalg.norm(bf - D(xv)) <= 1.01e-10 * np.linalg.norm(bf)
    xo, _ = K.minres(Aq, _g5(b), tol=1e-12, maxiter=20000)
    sig = np.abs(np.linalg.eigvalsh(wilson.dense(Aq, bf.size))).min()
    assert np.linalg.norm(xv - xo) <= 2e-10 * np.linalg.norm(bf) / sig
    assert m.defl_count(d)[0] == 10


def test_graph_replay_is_bit_identical_to_direct_launches(m, case, tmp_path):
    """The CUDA-graph path (captured Lanczos cycles and MinRes iteration groups)
    gives bit-identical results to plain launches: the reductions have a fixed
    summation order, so only a wrong captured argument could change a bit."""
    import os
    import subprocess
    import sys
    U, op, b = case
    p = _params(m, precision=m.F32)
    x, d, st = m.minresdr(op, torch.from_numpy(b).cuda(), p)
    B = synth.gaussian_spinors(DIMS, [21, 22])
    X, sts = m.dminres(op, d, torch.from_numpy(B).cuda(), p)
    np.save(tmp_path / "ref.npy", np.concatenate([x.cpu().numpy()[None], X.cpu().numpy()]))
    code = f"""
import sys, numpy as np, torch
sys.path.insert(0, {os.path.dirname(os.path.dirname(os.path.abspath(__file__)))!r})
import synth
from paper_0901_3163_gb300 import dlz
dims = {DIMS!r}
op = dlz.create_operator(dims, torch.from_numpy(synth.su3_links(dims, 1)).cuda(), {KAPPA!r})
p = dlz.params_default(m=40, k=10, tol=1e-10, oversolve=2.0, max_cycles=400, precision=dlz.F32)
x, d, st = dlz.minresdr(op, torch.from_numpy(synth.gaussian_spinor(dims, 0)).cuda(), p)
X, sts = dlz.dminres(op, d, torch.from_numpy(synth.gaussian_spinors(dims, [21, 22])).cuda(), p)
np.save(sys.argv[1], np.concatenate([x.cpu().numpy()[None], X.cpu().numpy()]))
"""
    env = dict(os.environ, DLZ_NO_GRAPHS="1")
    subprocess.run([sys.executable, "-c", code, str(tmp_path / "plain.npy")], check=True, env=env)
    ref = np.load(tmp_path / "ref.npy")
    plain = np.load(tmp_path / "plain.npy")
    assert np.array_equal(ref, plain)


def test_mixed_dcg_many_rhs_in_chunks(m, case):
    """18 right-hand sides through the batched FP32 D-CG (chunks of 16 and 2): every
    solution's oracle FP64 residual is below 1e-10, and batching does not change the
    per-RHS iteration count much versus solving one right-hand side alone."""
    U, op, b = case
    Aq, D, Dd, Ad = _ops(U, KAPPA)
    _, defl, _ = m.landr(op, torch.from_numpy(b).cuda(), _params(m))
    B = synth.gaussian_spinors(DIMS, list(range(30, 48)))
    p32 = _params(m, precision=m.F32)
    X, sts = m.dcg(op, defl, torch.from_numpy(B).cuda(), p32)
    _, one = m.dcg(op, defl, torch.from_numpy(B[:1]).cuda(), p32)
    Xn = X.cpu().numpy()
    for i in range(len(B)):
        bi = B[i].reshape(-1)
        assert sts[i].converged == 1
        assert np.linalg.norm(bi - D(Xn[i].reshape(-1))) <= 1.01e-10 * np.linalg.norm(bi)
    assert sts[0].iterations <= one[0].iterations + 24


@pytest.mark.parametrize("planes", ["4", "1"])
def test_mixed_dcg_slab_walk_matches_plain_order(m, monkeypatch, planes):
    """The fused CGNR kernels walk the lattice in slabs of z-planes when a 3-D slice is
    too large for L2 (DLZ_SLAB fixes the slab).  On 4x4x6x8 with slabs of 4 planes
    (one short slab of 2, whose spare block does nothing) or of 1 plane, every FP32 D-CG
    solution still reaches 1e-10 by the oracle's operator, and the iteration count stays
    within 10% of the plain site order's (the orders differ only in the rounding of the
    block sums)."""
    dims = (4, 4, 6, 8)
    U = synth.su3_links(dims, 11)
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), KAPPA)
    D = wilson.operator(U, KAPPA, dims, "D")
    B = synth.gaussian_spinors(dims, [21, 22, 23])
    p32 = _params(m, precision=m.F32)
    monkeypatch.delenv("DLZ_SLAB", raising=False)
    Xp, sp = m.dcg(op, None, torch.from_numpy(B).cuda(), p32)
    monkeypatch.setenv("DLZ_SLAB", planes)
    Xs, ss = m.dcg(op, None, torch.from_numpy(B).cuda(), p32)
    for i in range(len(B)):
        bi = B[i].reshape(-1)
        for X, s in ((Xp, sp), (Xs, ss)):
            assert s[i].converged == 1 and s[i].true_residual <= 1e-10
            assert np.linalg.norm(bi - D(X[i].cpu().numpy().reshape(-1))) <= 1.01e-10 * np.linalg.norm(bi)
        assert abs(ss[i].iterations - sp[i].iterations) <= 0.1 * sp[i].iterations


@pytest.mark.parametrize("planes", [None, "4"])
def test_mixed_dcg_staged_gathers_bit_identical(m, monkeypatch, planes):
    """The fused CGNR kernels copy the gathered field's site ranges into shared memory
    with bulk asynchronous copies before the stencil (DLZ_CG_STAGE=0 reads every
    neighbour from global memory instead).  Both read the same values and do the same
    arithmetic in the same order, so on 4x4x6x8 (every direction wraps somewhere; slabs
    of 4 z-planes leave a short slab) the solutions and iteration counts are identical
    bit for bit."""
    dims = (4, 4, 6, 8)
    U = synth.su3_links(dims, 12)
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), KAPPA)
    B = torch.from_numpy(synth.gaussian_spinors(dims, [31, 32])).cuda()
    p32 = _params(m, precision=m.F32)
    if planes is None:
        monkeypatch.delenv("DLZ_SLAB", raising=False)
    else:
        monkeypatch.setenv("DLZ_SLAB", planes)
    monkeypatch.setenv("DLZ_CG_STAGE", "0")
    Xg, sg = m.dcg(op, None, B, p32)
    monkeypatch.setenv("DLZ_CG_STAGE", "1")
    Xs, ss = m.dcg(op, None, B, p32)
    for i in range(2):
        assert sg[i].converged == 1 and ss[i].converged == 1
        assert sg[i].iterations == ss[i].iterations
    assert torch.equal(Xg, Xs)


def test_mixed_dcg_inner_tolerance_below_the_recurrence_floor(m, case):
    """The fused FP32 CG tracks |s| by a scalar recurrence whose rounding levels off near a
    3e-4 reduction; an inner tolerance far below that (reliable_delta 1e-7) must not keep
    the inner solve running to max_iter (D-CG holds it at 2e-3 or more), and every
    solution still verifies to 1e-10."""
    U, op, b = case
    Aq, D, Dd, Ad = _ops(U, KAPPA)
    B = synth.gaussian_spinors(DIMS, [41, 42])
    p = m.params_default(m=40, k=10, tol=1e-10, max_iter=20000, precision=m.F32, reliable_delta=1e-7)
    X, sts = m.dcg(op, None, torch.from_numpy(B).cuda(), p)
    for i in range(2):
        bi = B[i].reshape(-1)
        assert sts[i].converged == 1 and sts[i].iterations < 20000
        assert np.linalg.norm(bi - D(X[i].cpu().numpy().reshape(-1))) <= 1.01e-10 * np.linalg.norm(bi)
