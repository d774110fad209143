"""The failure path of the bounded device waits, made to happen on the host side
of the contract: polfed_set_wait_limit lowers the iteration caps so that the
step kernel's mbarrier waits and the batched kernel's grid barrier run out.
The calls must return POLFED_ETIMEOUT (no fault, no hang: the kernels drain the
copies they issued with the full cap and exit), and the next call with the
default caps must compute the same result as before."""
import numpy as np
import pytest

import polfed_inputs as I
from gpu_common import device_basis, lib, torch_dev

pytestmark = pytest.mark.gpu


def test_step_kernel_wait_limit_returns_timeout():
    torch, dev = torch_dev()
    pf = lib()
    m = I.xxz(22, 3.0, 4, 0)
    dim, st = device_basis(pf, torch, dev, m.L)
    X = torch.from_numpy(I.block(dim, 64, 5)).to(dev, torch.float32)
    Y0 = torch.empty_like(X)
    Y1 = torch.empty_like(X)
    b = 1.01 * (m.L * 0.75 + 0.5 * float(np.abs(m.h).sum()))
    pf.cheb_filter(m, st, dim, -b, b, 0.0, 6, X, Y0, 64, pf.F32)
    try:
        pf.set_wait_limit(1)
        with pytest.raises(pf.PolfedError) as e:
            pf.cheb_filter(m, st, dim, -b, b, 0.0, 6, X, Y1, 64, pf.F32)
        assert e.value.code == pf.POLFED_ETIMEOUT
    finally:
        pf.set_wait_limit(0)
    pf.cheb_filter(m, st, dim, -b, b, 0.0, 6, X, Y1, 64, pf.F32)
    assert torch.equal(Y0, Y1)


def test_batched_barrier_wait_limit_returns_timeout():
    torch, dev = torch_dev()
    pf = lib()
    ms = [I.xxz(16, 3.0, 3, 0), I.xxz(18, 2.0, 3, 1)]
    Xs, Y0, Y1 = [], [], []
    for k, m in enumerate(ms):
        dim = pf.basis_build(m.L, m.L // 2)
        Xs.append(torch.from_numpy(I.block(dim, 16, 50 + k)).to(dev))
        Y0.append(torch.empty_like(Xs[-1]))
        Y1.append(torch.empty_like(Xs[-1]))
    bs = [1.01 * (m.L * 0.75 + 0.5 * float(np.abs(m.h).sum())) for m in ms]
    lo, hi = [-b for b in bs], bs
    pf.cheb_filter_batched(ms, lo, hi, [0.0, 0.0], [40, 30], Xs, Y0, 16, pf.DF64)
    try:
        pf.set_wait_limit(1)
        with pytest.raises(pf.PolfedError) as e:
            pf.cheb_filter_batched(ms, lo, hi, [0.0, 0.0], [40, 30], Xs, Y1, 16, pf.DF64)
        assert e.value.code == pf.POLFED_ETIMEOUT
    finally:
        pf.set_wait_limit(0)
    pf.cheb_filter_batched(ms, lo, hi, [0.0, 0.0], [40, 30], Xs, Y1, 16, pf.DF64)
    for a, c in zip(Y0, Y1):
        assert torch.equal(a, c)
