"""The allocation-free filter entry point (polfed_cheb_filter_static).

Callers that cannot allocate device memory while they run use this variant;
it must give the same Y as the allocating polfed_cheb_filter.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

import polfed_inputs as I
from gpu_common import device_basis, lib, torch_dev

pytestmark = pytest.mark.gpu


def _bound(m):
    """A bound on ||H|| of Eq. (1): each bond term is at most |J| (1/2 + |Delta|/4), each field |h_i|/2."""
    nb = m.L if m.periodic else m.L - 1
    return 1.01 * (nb * (abs(m.J1) + abs(m.J2)) * (0.5 + abs(m.Delta) / 4) + 0.5 * float(np.abs(m.h).sum()))


@pytest.mark.parametrize("L,n_b,K,model", [(14, 16, 120, "xxz"), (18, 64, 300, "xxz"), (16, 32, 200, "j1j2"),
                                             (18, 64, 150, "j1j2")])
def test_static_filter_matches_allocating_filter_on_two_calls(L, n_b, K, model):
    torch, dev = torch_dev()
    pf = lib()
    dim, st = device_basis(pf, torch, dev, L)
    # the J1-J2 chain (J2 = 1, Delta = 0.55) runs the next-nearest-neighbour tables and kernels
    m = I.xxz(L, 3.0, 9, 0) if model == "xxz" else I.j1j2(L, 4.0, 9, 1)
    hi = _bound(m)
    lo = -hi
    for dtype, tdt, tol in ((pf.DF64, torch.float64, 1e-12), (pf.F64, torch.float64, 1e-12),
                            (pf.F32, torch.float32, 1e-5)):
        X = torch.from_numpy(I.block(dim, n_b, L + K)).to(dev, tdt)
        Y_ref = torch.empty_like(X)
        pf.cheb_filter(m, st, dim, lo, hi, 0.0, K, X, Y_ref, n_b, dtype)
        scale = float(torch.max(torch.abs(Y_ref)))
        for _ in range(2):  # the shared array keeps the previous call's contents
            Y = torch.full_like(X, float("nan"))
            pf.cheb_filter_static(m, st, dim, lo, hi, 0.0, K, X, Y, n_b, dtype)
            err = float(torch.max(torch.abs(Y.double() - Y_ref.double())))
            assert err <= tol * scale, (dtype, err, scale)


def test_static_filter_rejects_sizes_beyond_the_array():
    torch, dev = torch_dev()
    pf = lib()
    L = 20  # dim 184756: three 128-byte slice buffers alone exceed 32 MiB
    dim, st = device_basis(pf, torch, dev, L)
    X = torch.zeros((dim, 64), dtype=torch.float64, device=dev)
    Y = torch.zeros_like(X)
    with pytest.raises(pf.PolfedError) as e:
        pf.cheb_filter_static(I.xxz(L, 3.0, 9, 0), st, dim, -30.0, 30.0, 0.0, 10, X, Y, 64, pf.DF64)
    assert e.value.code == pf.POLFED_ENOMEM
    assert "32" in str(e.value) or "bytes" in str(e.value)


def test_static_filter_clears_the_previous_error():
    """A successful call leaves no stale message from an earlier failure."""
    torch, dev = torch_dev()
    pf = lib()
    L = 12
    dim, st = device_basis(pf, torch, dev, L)
    m = I.xxz(L, 2.0, 9, 2)
    X = torch.from_numpy(I.block(dim, 8, 3)).to(dev)
    Y = torch.empty_like(X)
    with pytest.raises(pf.PolfedError):
        pf.cheb_filter_static(m, st, dim, 1.0, -1.0, 0.0, 10, X, Y, 8, pf.DF64)  # e_lo > e_hi
    assert pf.last_error() != ""
    pf.cheb_filter_static(m, st, dim, -_bound(m), _bound(m), 0.0, 10, X, Y, 8, pf.DF64)
    assert pf.last_error() == ""
