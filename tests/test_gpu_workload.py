"""The benchmark workloads run exactly as one benchmark step runs them (bench.solve_step
with bench.workload_params, FP32 chosen form), checked by properties that hold at any
size with the oracle's independent FP64 operator (the plain-C Wilson loops): every
solution's ||b - D x|| / ||b||, and, for three of the returned deflation pairs, the
library's residual ||A y - value y|| and the Rayleigh quotient of the unit vector y,
which equals the value to rounding.

  * 24^3x48: Lan-DR(120,60) on D^dagger D for the first Gaussian RHS, D-CG on 48;
  * 16^3x32: MinRes-DR(100,40) + D-MinRes on the 12 spin-colour point sources;
  * the 64 lattices of uneven size (8^4, 12^4, 16^4): one dlz_batch_dminres call on
    8 Gaussian RHS per lattice, each solution checked with its lattice's operator."""
import numpy as np
import pytest

import bench
import synth
from oracle import cwilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _check_pairs(m, defl, k_expect, A, V, picks, name):
    k, _ = m.defl_count(defl)
    assert k == k_expect
    y = np.empty((V, 4, 3), dtype=np.complex128)
    for i in picks(k):
        val, res = m.defl_get(defl, i, y)
        yv = y.reshape(-1)
        ay = A(yv)
        assert abs(np.linalg.norm(ay - val * yv) - res) <= 1e-10 * max(1.0, abs(val))
        rq = np.vdot(yv, ay).real / np.vdot(yv, yv).real
        assert abs(np.linalg.norm(yv) - 1.0) <= 1e-10
        # each reported value is the Rayleigh quotient of its vector (Rayleigh-Ritz with the
        # Gram matrix of the FP32-built basis), so it agrees with the oracle's to rounding
        assert abs(rq - val) <= 1e-12 + 1e-10 * abs(val)
        # the error of each reported value against the oracle (the value is a Rayleigh
        # quotient, within its residual of an eigenvalue of A)
        print(f"{name} pair {i}: value {val:.6e}, oracle Rayleigh quotient {rq:.6e}, "
              f"|difference| {abs(rq - val):.2e}, oracle residual {np.linalg.norm(ay - rq * yv):.2e}")


def _check_solutions(stats, xs, B, D, name):
    worst = 0.0
    for s, x, b in zip(stats, xs, B):
        assert s.converged == 1 and s.true_residual <= 1e-10
        bf = b.reshape(-1)
        rel = np.linalg.norm(bf - D(x.reshape(-1))) / np.linalg.norm(bf)
        assert rel <= 1.01e-10
        worst = max(worst, rel)
    # the error of each solution against the oracle, as its residual by the oracle's operator
    print(f"{name}: {len(xs)} solutions, largest ||b - D x|| / ||b|| by the oracle's operator {worst:.3e}")


def test_c2_workload_against_oracle_operator():
    m = dlz()
    w, dims, U, kappa, B = bench.workload_inputs(name=bench.C2)
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    Bd = torch.from_numpy(B).cuda()
    p_dr, p_d = bench.workload_params(m, w, m.F32, name=bench.C2)
    x0, defl, st = m.minresdr(op, Bd[0].contiguous(), p_dr)
    X, sts = m.dminres(op, defl, Bd[1:].contiguous(), p_d)
    D = cwilson.operator(U, kappa, dims, "D")
    xs = [x0.cpu().numpy()] + [X[i].cpu().numpy() for i in range(B.shape[0] - 1)]
    _check_solutions([st] + list(sts), xs, B, D, "16^3x32")
    Q = cwilson.operator(U, kappa, dims, "Q")
    _check_pairs(m, defl, w["k"], Q, synth.volume(dims), lambda k: (0, k // 2, k - 1), "16^3x32")


def test_c3_step_against_oracle_operator():
    m = dlz()
    w, dims, U, kappa, B = bench.workload_inputs()
    assert B.shape[0] == 49 and dims == (24, 24, 24, 48)
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    Bd = torch.from_numpy(B).cuda()
    p_dr, p_d = bench.workload_params(m, w, m.F32)
    x0, defl, st = m.landr(op, Bd[0].contiguous(), p_dr)
    X, sts = m.dcg(op, defl, Bd[1:].contiguous(), p_d)
    D = cwilson.operator(U, kappa, dims, "D")
    xs = [x0.cpu().numpy()] + [X[i].cpu().numpy() for i in range(B.shape[0] - 1)]
    del X, Bd
    _check_solutions([st] + list(sts), xs, B, D, "24^3x48")
    DD = cwilson.operator(U, kappa, dims, "DdagD")
    _check_pairs(m, defl, w["k"], DD, synth.volume(dims), lambda k: (0, k // 2, k - 1), "24^3x48")


def test_c4_batch_against_oracle_operator():
    m = dlz()
    w = synth.WORKLOADS[bench.C4]
    kap = bench.c4_kappas(w)
    ops, defls, Bs, Us = [], [], [], []
    for i in range(w["lattices"]):
        dims = w["sizes"][i % 3]
        U = synth.su3_links(dims, w["gauge_seed0"] + i)
        op = m.create_operator(dims, torch.from_numpy(U).cuda(), float(kap[i]))
        b0 = torch.from_numpy(synth.gaussian_spinor(dims, w["first_rhs_seed"])).cuda()
        _, d, st = m.minresdr(op, b0, m.params_default(m=w["m"], k=w["k"], tol=1e-10, max_cycles=400,
                                                       precision=m.F32))
        assert st.converged == 1
        ops.append(op)
        defls.append(d)
        Us.append(U)
        Bs.append(synth.gaussian_spinors(dims, w["rhs_seeds"]))
    p32 = m.params_default(m=w["m"], k=w["k"], tol=1e-10, max_iter=100000, precision=m.F32,
                           reliable_delta=1e-5)
    Xs, sts = m.batch_dminres(ops, defls, [torch.from_numpy(b).cuda() for b in Bs], p32)
    for i in range(w["lattices"]):
        dims = w["sizes"][i % 3]
        D = cwilson.operator(Us[i], float(kap[i]), dims, "D")
        X = Xs[i].cpu().numpy()
        _check_solutions(sts[i], [X[j] for j in range(X.shape[0])], Bs[i], D, f"lattice {i} {dims}")
    # deflation pairs of one lattice of each size
    for i in range(3):
        dims = w["sizes"][i]
        Q = cwilson.operator(Us[i], float(kap[i]), dims, "Q")
        _check_pairs(m, defls[i], w["k"], Q, synth.volume(dims), lambda k: (0, k - 1), f"lattice {i} {dims}")
