"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

import polfed_inputs as I


def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch, torch.device("cuda:0")


_BUILT = []


def lib():
    if not _BUILT:
        from paper_2005_09534_gb300 import build
        build.build()
        _BUILT.append(1)
    import paper_2005_09534_gb300 as pf
    pf.load()
    return pf


def device_basis(pf, torch, dev, L):
    dim = pf.basis_build(L, L // 2)
    st = torch.empty(dim, dtype=torch.int32, device=dev)
    pf.basis_build(L, L // 2, st)
    torch.cuda.synchronize()
    return dim, st


def models(L):
    """A few Eq. (1) instances at length L: XXZ and J1-J2, periodic and open, random fields."""
    return [I.xxz(L, 3.0, 7, 0), I.j1j2(L, 4.0, 7, 1), I.xxz(L, 2.0, 7, 2, periodic=False),
            I.Model(L, 0.8, 0.45, 0.7, I.fields(L, 2.5, 7, 3), False, 2.5)]
