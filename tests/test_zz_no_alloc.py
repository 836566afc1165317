"""dlz_apply_noalloc (library-interface variant of dlz_apply with a static device
scratch; the paper has no counterpart): same results as dlz_apply, bit for bit, on
two calls in a row; rejects lattices beyond the scratch and host pointers.

The file name sorts last so that the test also runs after every other GPU test;
it uses nothing that the other tests leave behind."""
import numpy as np
import pytest

import synth
from tests._lib import dlz

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    return dlz()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 6, 4, 10)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_equals_apply_two_calls_in_a_row(m, dims, prec):
    U = synth.su3_links(dims, 3)
    op = m.create_operator(dims, torch.from_numpy(U).cuda(), 0.21)
    X = synth.gaussian_spinors(dims, [4, 5, 6])
    dt = torch.complex128 if prec == "f64" else torch.complex64
    x = torch.from_numpy(X).to(dt).cuda()
    for which in (m.D, m.DDAG, m.Q, m.DDAGD):
        ref = m.apply(op, which, x)
        first = m.apply_noalloc(op, which, x)
        second = m.apply_noalloc(op, which, x)
        torch.cuda.synchronize()
        assert torch.equal(first, ref)
        assert torch.equal(second, ref)
        assert torch.isfinite(torch.view_as_real(ref)).all()


def test_noalloc_limits(m):
    dims = (16, 16, 16, 32)
    op = m.create_operator(dims, torch.from_numpy(synth.unit_links(dims)).cuda(), 0.12)
    x64 = torch.zeros((1,) + (synth.volume(dims), 4, 3), dtype=torch.complex128, device="cuda")
    # 3 FP64 work vectors of 16^3x32 exceed the 64 MiB scratch: rejected before any work
    with pytest.raises(m.DlzError) as e:
        m.apply_noalloc(op, m.DDAGD, x64)
    assert e.value.code == m.ERR_BADARG
    # 2 vectors fit: same result as dlz_apply
    x64.normal_()
    assert torch.equal(m.apply_noalloc(op, m.Q, x64), m.apply(op, m.Q, x64))
    # host tensors would need staging buffers: rejected
    xh = torch.zeros((4, 4, 4, 4, 4, 3), dtype=torch.complex128)
    op4 = m.create_operator((4, 4, 4, 4), torch.from_numpy(synth.unit_links((4, 4, 4, 4))).cuda(), 0.12)
    with pytest.raises(m.DlzError):
        m.apply_noalloc(op4, m.D, xh.reshape(256, 4, 3), out=torch.zeros_like(xh.reshape(256, 4, 3)))
