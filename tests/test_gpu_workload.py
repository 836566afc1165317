"""The 16^3x32 benchmark workload (MinRes-DR(100,40) + D-MinRes, 12 point sources) run
exactly as one benchmark step runs it (bench.workload_params, FP32 chosen form), checked
by properties that hold at any size with the oracle's independent FP64 operator (the
plain-C Wilson loops): every solution's ||b - D x|| / ||b||, and, for three of the 40
returned deflation pairs, the library's residual ||Q y - value y|| and the Rayleigh
quotient of y (which lies within residual / ||y|| of the value)."""
import numpy as np
import pytest

import bench
import synth
from oracle import cwilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_benchmark_workload_against_oracle_operator():
    m = dlz()
    w, dims, U, kappa, B = bench.workload_inputs()
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
    Bd = torch.from_numpy(B).cuda()
    p_dr, p_d = bench.workload_params(m, w, m.F32)
    x0, defl, st = m.minresdr(op, Bd[0].contiguous(), p_dr)
    X, sts = m.dminres(op, defl, Bd[1:].contiguous(), p_d)
    D = cwilson.operator(U, kappa, dims, "D")
    xs = [x0.cpu().numpy()] + [X[i].cpu().numpy() for i in range(B.shape[0] - 1)]
    for s, x, b in zip([st] + list(sts), xs, B):
        assert s.converged == 1 and s.true_residual <= 1e-10
        bf = b.reshape(-1)
        assert np.linalg.norm(bf - D(x.reshape(-1))) <= 1.01e-10 * np.linalg.norm(bf)
    Q = cwilson.operator(U, kappa, dims, "Q")
    k, _ = m.defl_count(defl)
    assert k == w["k"]
    y = np.empty((synth.volume(dims), 4, 3), dtype=np.complex128)
    for i in (0, k // 2, k - 1):
        val, res = m.defl_get(defl, i, y)
        yv = y.reshape(-1)
        qy = Q(yv)
        assert abs(np.linalg.norm(qy - val * yv) - res) <= 1e-10
        rq = np.vdot(yv, qy).real / np.vdot(yv, yv).real
        assert abs(rq - val) <= res / np.linalg.norm(yv) + 1e-12
