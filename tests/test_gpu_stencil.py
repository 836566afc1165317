"""GPU parity of the Wilson stencil (D, D^dagger, gamma5 D, D^dagger D) against the
FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import cwilson, wilson
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (3, 5, 4, 6), (1, 2, 3, 4), (8, 4, 6, 10)]
REFS = {"D": wilson.apply_D, "DDAG": wilson.apply_Ddag, "Q": wilson.apply_Q, "DDAGD": wilson.apply_DdagD}


@pytest.fixture(scope="module")
def m():
    return dlz()


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("bc_t", [1, -1])
def test_stencil_fp64_fp32_match_oracle(m, dims, bc_t):
    U = synth.su3_links(dims, 3)
    kappa = 0.137
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa, bc_t)
    psi = synth.gaussian_spinors(dims, [1, 2, 3])
    x64 = torch.from_numpy(psi).cuda()
    x32 = x64.to(torch.complex64)
    for name, ref in REFS.items():
        want = ref(U, psi, kappa, dims, bc_t)
        got = m.apply(op, getattr(m, name), x64).cpu().numpy()
        assert _rel(got, want) < 1e-14, (name, _rel(got, want))
        got32 = m.apply(op, getattr(m, name), x32).cpu().numpy()
        assert _rel(got32, want) < 3e-6, (name, _rel(got32, want))


def test_stencil_host_buffers_and_empty_batch(m):
    dims = (4, 6, 2, 8)
    U = synth.su3_links(dims, 4)
    op = m.create_operator(dims, U, 0.15, 1)          # gauge passed from host memory
    psi = synth.gaussian_spinor(dims, 9)
    got = m.apply(op, m.Q, psi)                       # host in, host out
    assert isinstance(got, np.ndarray)
    assert _rel(got, wilson.apply_Q(U, psi, 0.15, dims)) < 1e-14
    empty = np.zeros((0,) + psi.shape, dtype=np.complex128)
    assert m.apply(op, m.D, empty).shape == empty.shape


def test_stencil_full_size_sampled_sites(m):
    dims = (16, 16, 16, 32)
    V = synth.volume(dims)
    U = synth.su3_links(dims, 2)
    kappa = 0.25
    psi = synth.gaussian_spinor(dims, 5)
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa, 1)
    x = torch.from_numpy(psi).cuda()
    got = m.apply(op, m.D, x).cpu().numpy()
    rng = np.random.default_rng(0)
    lx, ly, lz, lt = dims
    corners = [0, lx - 1, lx * (ly - 1), V - 1, V - lx * ly * lz, lx * ly * lz - 1]
    sites = np.unique(np.concatenate([rng.choice(V, 3000, replace=False), corners]))
    want = cwilson.apply_D_sites(U, psi, kappa, dims, sites)
    assert _rel(got[sites], want) < 1e-14
    got32 = m.apply(op, m.D, x.to(torch.complex64)).cpu().numpy()
    assert _rel(got32[sites], want) < 3e-6


def test_bad_gauge_is_rejected(m):
    dims = (2, 2, 2, 4)
    U = synth.su3_links(dims, 1)
    U[2, 5] *= 1.001
    with pytest.raises(m.DlzError) as e:
        m.create_operator(dims, U, 0.1)
    assert e.value.code == m.ERR_BAD_GAUGE
    U = synth.su3_links(dims, 1)
    U[0, 0, 1, 1] = np.nan
    with pytest.raises(m.DlzError) as e:
        m.create_operator(dims, U, 0.1)
    assert e.value.code == m.ERR_BAD_GAUGE


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 4, 6)])
@pytest.mark.parametrize("bc_t", [1, -1])
def test_stencil_bf16_storage(m, dims, bc_t):
    """bfloat16 storage, FP32 arithmetic: against the FP64 oracle applied to the input
    rounded to bfloat16 on the host, within one bfloat16 rounding of the output (2^-8
    of the largest entry; D^dag D within two); every output value is a bfloat16."""
    from oracle import ptc
    U = synth.su3_links(dims, 3)
    kappa = 0.137
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), kappa, bc_t)
    psi = synth.gaussian_spinors(dims, [1, 2])
    xr = ptc.round_bf16(psi.astype(np.complex64))
    x = torch.from_numpy(psi.astype(np.complex64)).cuda()
    for name, ref in REFS.items():
        want = ref(U, xr, kappa, dims, bc_t)
        got = m.apply(op, getattr(m, name), x, dtype=m.BF16).cpu().numpy()
        assert np.array_equal(ptc.round_bf16(got), got.astype(np.complex128))
        tol = 2.0 ** -8 * (2 if name == "DDAGD" else 1)
        assert _rel(got, want) < tol, (name, _rel(got, want))
