"""D-MinRes on several lattices of uneven size at once (dlz_batch_dminres):
every solution reaches ||b - D x|| / ||b|| <= 1e-10 (checked with the FP64 oracle's
own operator) and agrees with that lattice's solve on its own."""
import numpy as np
import pytest

import synth
from oracle import wilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LATS = [((4, 4, 4, 4), 0.18, 11), ((4, 4, 4, 8), 0.2, 12), ((6, 4, 4, 4), 0.21, 13), ((8, 8, 8, 8), 0.19, 14)]


@pytest.fixture(scope="module")
def m():
    return dlz()


@pytest.mark.parametrize("with_defl", [True, False])
def test_batch_dminres_uneven_lattices(m, with_defl):
    ops, defls, Bs, Us = [], [], [], []
    for i, (dims, kappa, seed) in enumerate(LATS):
        U = synth.su3_links(dims, seed)
        op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa)
        b0 = torch.from_numpy(synth.gaussian_spinor(dims, 0)).cuda()
        d = None
        if with_defl:
            _, d, _ = m.minresdr(op, b0, m.params_default(m=30, k=8, tol=1e-10, max_cycles=200))
        ops.append(op); defls.append(d); Us.append(U)
        Bs.append(torch.from_numpy(synth.gaussian_spinors(dims, [1 + i, 2 + i, 3 + i][: 2 + (i % 2)])).cuda())
    p = m.params_default(m=30, k=8, tol=1e-10, max_iter=20000, precision=m.F32)
    Xs, sts = m.batch_dminres(ops, defls, Bs, p)
    alone_max = 0
    for l, (dims, kappa, seed) in enumerate(LATS):
        D = wilson.operator(Us[l], kappa, dims, "D")
        Xl = Xs[l].cpu().numpy()
        Bl = Bs[l].cpu().numpy()
        _, alone = m.dminres(ops[l], defls[l], Bs[l], p)
        alone_max = max(alone_max, max(s.iterations for s in alone))
        for r in range(Bl.shape[0]):
            assert sts[l][r].converged == 1
            b = Bl[r].reshape(-1)
            assert np.linalg.norm(b - D(Xl[r].reshape(-1))) <= 1.01e-10 * np.linalg.norm(b)
    # the slots iterate together until the slowest one is done: the batch takes about
    # as many iterations as the hardest lattice alone
    assert max(s.iterations for ss in sts for s in ss) <= alone_max + 96
    # the plain FP64 form of the same entry point solves them one lattice at a time
    p64 = m.params_default(m=30, k=8, tol=1e-10, max_iter=20000)
    Xs64, sts64 = m.batch_dminres(ops, defls, Bs, p64)
    assert all(s.converged == 1 for ss in sts64 for s in ss)


def test_batch_dminres_tiles_bit_identical(m, monkeypatch):
    """The batched kernels run with 1, 2 or 4 chunks of 128 sites per block (chosen by
    timing, or forced with DLZ_MULTI_TILE); the sums are taken per chunk in a fixed
    order, so every tile gives the same bits."""
    ops, Bs = [], []
    for i, (dims, kappa, seed) in enumerate(LATS):
        U = synth.su3_links(dims, seed)
        ops.append(m.create_operator(dims, torch.from_numpy(U).cuda(), kappa))
        Bs.append(torch.from_numpy(synth.gaussian_spinors(dims, [5 + i, 6 + i])).cuda())
    p = m.params_default(m=30, k=8, tol=1e-10, max_iter=20000, precision=m.F32)
    runs = {}
    for tile in ["1", "2", "4", None]:
        if tile is None:
            monkeypatch.delenv("DLZ_MULTI_TILE", raising=False)
        else:
            monkeypatch.setenv("DLZ_MULTI_TILE", tile)
        Xs, sts = m.batch_dminres(ops, [None] * len(ops), Bs, p)
        assert all(s.converged == 1 for ss in sts for s in ss)
        runs[tile] = ([x.cpu().numpy() for x in Xs], [[s.iterations for s in ss] for ss in sts])
    ref_x, ref_it = runs["1"]
    for tile, (xs, its) in runs.items():
        assert its == ref_it, tile
        for a, b in zip(xs, ref_x):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), tile


def _small_batch(m):
    ops, Bs = [], []
    for i, (dims, kappa, seed) in enumerate(LATS):
        U = synth.su3_links(dims, seed)
        ops.append(m.create_operator(dims, torch.from_numpy(U).cuda(), kappa))
        Bs.append(torch.from_numpy(synth.gaussian_spinors(dims, [5 + i, 6 + i])).cuda())
    return ops, Bs


def test_batch_dminres_persistent_and_graph_forms_bit_identical(m, monkeypatch):
    """The persistent form (one cooperative launch over all slots and iterations, grid
    barriers between the stages) against the graph form and the autotuner's pick: the
    same chunk partials and the same freezing points give the same bits."""
    ops, Bs = _small_batch(m)
    p = m.params_default(m=30, k=8, tol=1e-10, max_iter=20000, precision=m.F32)
    runs = {}
    for form, tile in [("graph", "1"), ("persistent", "1"), ("persistent", "2"), ("persistent", "4"), (None, None)]:
        for var, val in (("DLZ_MULTI_FORM", form), ("DLZ_MULTI_TILE", tile)):
            if val is None:
                monkeypatch.delenv(var, raising=False)
            else:
                monkeypatch.setenv(var, val)
        Xs, sts = m.batch_dminres(ops, [None] * len(ops), Bs, p)
        assert all(s.converged == 1 for ss in sts for s in ss)
        runs[(form, tile)] = ([x.cpu().numpy() for x in Xs], [[s.iterations for s in ss] for ss in sts],
                              m.batch_last_choice(ops[0]))
    ref_x, ref_it, _ = runs[("graph", "1")]
    for key, (xs, its, choice) in runs.items():
        assert its == ref_it, key
        for a, b in zip(xs, ref_x):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), key
    assert runs[("persistent", "2")][2][:2] == (1, 2)
    assert runs[("graph", "1")][2][:2] == (0, 1)


def test_persistent_barrier_wait_limit_returns_device_timeout(m, monkeypatch):
    """Failure detection without a fault: with a wait limit of zero polls, every block
    that has to wait at a grid barrier gives up at once, sets the error word and
    returns; the call reports DLZ_ERR_DEVICE_TIMEOUT and the context stays usable (the
    same call with the default limit then succeeds)."""
    ops, Bs = _small_batch(m)
    p = m.params_default(m=30, k=8, tol=1e-10, max_iter=20000, precision=m.F32)
    monkeypatch.setenv("DLZ_MULTI_FORM", "persistent")
    monkeypatch.setenv("DLZ_MULTI_TILE", "1")
    monkeypatch.setenv("DLZ_WAIT_LIMIT", "0")
    with pytest.raises(m.DlzError) as e:
        m.batch_dminres(ops, [None] * len(ops), Bs, p)
    assert e.value.code == m.ERR_DEVICE_TIMEOUT
    monkeypatch.delenv("DLZ_WAIT_LIMIT")
    Xs, sts = m.batch_dminres(ops, [None] * len(ops), Bs, p)
    assert all(s.converged == 1 for ss in sts for s in ss)
