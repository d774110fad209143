"""GPU parity of the basis, the matrix-free H~ application and the Chebyshev filter
against the CPU oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle as O
import polfed_inputs as I
from gpu_common import device_basis, lib, models, torch_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [4, 6, 8, 12, 16, 20])
def test_basis_bit_exact(L):
    torch, dev = torch_dev()
    pf = lib()
    dim, st = device_basis(pf, torch, dev, L)
    assert np.array_equal(st.cpu().numpy().view(np.uint32).astype(np.int64), O.basis(L))
    # other magnetization sectors too
    for n_up in (0, 1, L // 2 - 1, L):
        d = pf.basis_build(L, n_up)
        assert d == math.comb(L, n_up)
        t = torch.empty(max(d, 1), dtype=torch.int32, device=dev)
        pf.basis_build(L, n_up, t)
        torch.cuda.synchronize()
        assert np.array_equal(t[:d].cpu().numpy().view(np.uint32).astype(np.int64), O.basis(L, n_up))


@pytest.mark.parametrize("L", [22, 24])
def test_basis_full_size_sampled(L):
    torch, dev = torch_dev()
    pf = lib()
    dim, st = device_basis(pf, torch, dev, L)
    assert dim == math.comb(L, L // 2)
    s = st.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.all(np.diff(s) > 0)
    assert np.all(O.popcount(s) == L // 2)
    for r in I.sample_rows(dim, 200, L):
        assert O.rank_combinatorial(int(s[r])) == r


def _tol(dtype):
    import paper_2005_09534_gb300 as pf
    return {pf.F64: 1e-13, pf.DF64: 1e-12, pf.F32: 3e-6}[dtype]


@pytest.mark.parametrize("L", [4, 6, 8, 10, 14])
@pytest.mark.parametrize("n_b", [1, 3, 16, 33, 64])
def test_h_apply_vs_dense(L, n_b):
    torch, dev = torch_dev()
    pf = lib()
    dim, st = device_basis(pf, torch, dev, L)
    for mi, m in enumerate(models(L)):
        H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)
        X = I.block(dim, n_b, 100 * L + n_b + mi)
        for (lo, hi) in ((0.0, 0.0), (-9.0, 7.5)):
            A = H if lo == hi == 0.0 else O.rescale_matrix(H, lo, hi)
            want = A @ X
            scale = max(1.0, np.abs(want).max())
            for dtype in (pf.F64, pf.DF64, pf.F32):
                tdt = torch.float32 if dtype == pf.F32 else torch.float64
                Xd = torch.from_numpy(X).to(dev, tdt)
                Yd = torch.full_like(Xd, float("nan"))
                pf.h_apply(m, st, dim, lo, hi, Xd, Yd, n_b, dtype)
                got = Yd.double().cpu().numpy()
                err = np.abs(got - want).max() / scale
                assert err < _tol(dtype) * (10 if dtype == pf.F32 else 1) * max(1, L / 4), (mi, lo, dtype, err)


@pytest.mark.parametrize("L,n_b", [(20, 32), (22, 64), (24, 64)])
def test_h_apply_full_size_sampled_rows(L, n_b):
    torch, dev = torch_dev()
    pf = lib()
    dim, st = device_basis(pf, torch, dev, L)
    states = O.basis(L)
    for m in (I.xxz(L, 3.0, 4, 0), I.j1j2(L, 4.0, 2, 0)):
        X = I.block(dim, n_b, L)
        rows = I.sample_rows(dim, 60, L + 1)
        lo, hi = -30.0, 31.0
        want = O.h_apply_rows(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic, states, X, rows, lo, hi)
        for dtype in (pf.F64, pf.DF64, pf.F32):
            tdt = torch.float32 if dtype == pf.F32 else torch.float64
            Xd = torch.from_numpy(X).to(dev, tdt)
            Yd = torch.empty_like(Xd)
            pf.h_apply(m, st, dim, lo, hi, Xd, Yd, n_b, dtype)
            got = Yd[torch.from_numpy(rows).to(dev)].double().cpu().numpy()
            err = np.abs(got - want).max() / max(1.0, np.abs(want).max())
            assert err < (1e-13 if dtype == pf.F64 else (1e-12 if dtype == pf.DF64 else 3e-5)), (dtype, err)


def _spectral(m):
    H, st = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)
    w, V = np.linalg.eigh(H)
    return H, w, V


@pytest.mark.parametrize("L", [8, 12])
@pytest.mark.parametrize("K", [0, 1, 2, 7, 60, 400])
def test_cheb_filter_vs_spectral_definition(L, K):
    torch, dev = torch_dev()
    pf = lib()
    dim, st = device_basis(pf, torch, dev, L)
    for mi, m in enumerate(models(L)[:2]):
        H, w, V = _spectral(m)
        lo, hi = w[0] - 0.05, w[-1] + 0.07
        lt = (2 * w - lo - hi) / (hi - lo)
        for sigma in (0.0, 0.31):
            n_b = 16 if sigma == 0.0 else 5
            X = I.block(dim, n_b, K + 31 * mi)
            want = O.filter_spectral(lt, V, X, sigma, K)
            for dtype in (pf.F64, pf.DF64, pf.F32):
                tdt = torch.float32 if dtype == pf.F32 else torch.float64
                Xd = torch.from_numpy(X).to(dev, tdt)
                Yd = torch.empty_like(Xd)
                pf.cheb_filter(m, st, dim, lo, hi, sigma, K, Xd, Yd, n_b, dtype)
                err = np.abs(Yd.double().cpu().numpy() - want).max() / np.abs(X).max()
                tol = {pf.F64: 1e-13 * (K + 1), pf.DF64: 1e-12 * (K + 1), pf.F32: 2e-7 * (K + 1) + 1e-6}[dtype]
                assert err < tol, (mi, sigma, dtype, err)


def test_cheb_filter_user_coefficients():
    torch, dev = torch_dev()
    pf = lib()
    L = 10
    dim, st = device_basis(pf, torch, dev, L)
    m = models(L)[1]
    H, w, V = _spectral(m)
    lo, hi = w[0] - 0.1, w[-1] + 0.1
    lt = (2 * w - lo - hi) / (hi - lo)
    K = 25
    c = np.random.default_rng(3).standard_normal(K + 1)
    X = I.block(dim, 8, 9)
    want = O.filter_spectral(lt, V, X, 0.0, K, coeffs=c, D=1.0)
    Xd = torch.from_numpy(X).to(dev)
    Yd = torch.empty_like(Xd)
    pf.cheb_filter(m, st, dim, lo, hi, 0.0, K, Xd, Yd, 8, pf.DF64, coeffs=c)
    assert np.abs(Yd.cpu().numpy() - want).max() < 1e-11 * np.abs(c).sum()


def test_cheb_filter_reports_bounds_violation():
    torch, dev = torch_dev()
    pf = lib()
    L = 10
    dim, st = device_basis(pf, torch, dev, L)
    m = models(L)[0]
    H, w, V = _spectral(m)
    X = torch.from_numpy(I.block(dim, 16, 2)).to(dev)
    Y = torch.empty_like(X)
    lo, hi = 0.5 * w[0], 0.5 * w[-1]  # half the spectrum lies outside [lo, hi]
    rc = pf.cheb_filter(m, st, dim, lo, hi, 0.0, 200, X, Y, 16, pf.F64, allow_bounds_error=True)
    assert rc == pf.POLFED_EBOUNDS


def test_filter_properties_full_size():
    """L = 22, n_b = 64: the filter is symmetric, contracts norms, and K = 1 with
    coefficients (0, 1) reproduces the H~ application on sampled rows."""
    torch, dev = torch_dev()
    pf = lib()
    L, n_b = 22, 64
    dim, st = device_basis(pf, torch, dev, L)
    m = I.xxz(L, 3.0, 4, 0)
    lo, hi = -33.0, 33.0
    X = torch.from_numpy(I.block(dim, n_b, 5)).to(dev)
    Z = torch.from_numpy(I.block(dim, n_b, 6)).to(dev)
    PX = torch.empty_like(X)
    PZ = torch.empty_like(X)
    K = 300
    pf.cheb_filter(m, st, dim, lo, hi, 0.0, K, X, PX, n_b, pf.DF64)
    pf.cheb_filter(m, st, dim, lo, hi, 0.0, K, Z, PZ, n_b, pf.DF64)
    a = (Z * PX).sum(0)
    b = (PZ * X).sum(0)
    assert torch.max(torch.abs(a - b)).item() < 1e-10 * torch.max(torch.abs(a)).item() + 1e-8
    assert torch.all(PX.norm(dim=0) <= X.norm(dim=0) * (1 + 1e-12))
    Y1 = torch.empty_like(X)
    pf.cheb_filter(m, st, dim, lo, hi, 0.0, 1, X, Y1, n_b, pf.DF64, coeffs=np.array([0.0, 1.0]))
    Y2 = torch.empty_like(X)
    pf.h_apply(m, st, dim, lo, hi, X, Y2, n_b, pf.F64)
    assert torch.max(torch.abs(Y1 - Y2)).item() < 1e-12 * torch.max(torch.abs(Y2)).item()
    rows = I.sample_rows(dim, 30, 8)
    want = O.h_apply_rows(m.L, m.J1, m.J2, m.Delta, m.h, True, O.basis(L), X.cpu().numpy(), rows, lo, hi)
    assert np.abs(Y1.cpu().numpy()[rows] - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("L,n_b", [(12, 16), (12, 7), (18, 64)])
def test_cheb_filter_per_column_coefficients(L, n_b):
    """polfed_cheb_filter_cols: every column through its own Chebyshev series
    (FP32), against the oracle's matrix three-term recurrence column by column;
    L = 12 runs the generic step kernel, L = 18 with 64 columns the TMA kernel."""
    torch, dev = torch_dev()
    pf = lib()
    import scipy.sparse as sp
    dim, st = device_basis(pf, torch, dev, L)
    m = models(L)[0]
    H, _ = O.sparse_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)
    b = 1.01 * (m.L * 0.75 + 0.5 * float(np.abs(m.h).sum()))
    Ht = sp.csr_matrix(H / b)
    K = 40
    rng = np.random.default_rng(L + n_b)
    C = rng.standard_normal((n_b, K + 1)) / np.sqrt(np.arange(1, K + 2))
    X = I.block(dim, n_b, 77)
    want = np.stack([O.filter_matrix_powers(Ht, X[:, [j]], C[j], 1.0)[:, 0] for j in range(n_b)], axis=1)
    Xd = torch.from_numpy(X).to(dev, torch.float32)
    Yd = torch.empty_like(Xd)
    pf.cheb_filter_cols(m, st, dim, -b, b, C, Xd, Yd, n_b)
    err = np.abs(Yd.double().cpu().numpy() - want).max() / (np.abs(X).max() * np.abs(C).sum(axis=1).max())
    assert err < 2e-7 * (K + 1) + 1e-6, err
    # one column's own series equals the scalar-coefficient filter of that column
    j = n_b // 2
    Y1 = torch.empty_like(Xd)
    pf.cheb_filter(m, st, dim, -b, b, 0.0, K, Xd, Y1, n_b, pf.F32, coeffs=C[j])
    assert torch.allclose(Yd[:, j], Y1[:, j], rtol=0, atol=1e-5 * float(np.abs(C[j]).sum() * np.abs(X).max()))
