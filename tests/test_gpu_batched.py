"""GPU parity of the batched runner.

* polfed_cheb_filter_batched (one cooperative launch for many realizations of
  mixed L, K, sigma) against the oracle's spectral definition of the filter.
* polfed_eigs_batched (rendezvous of many realizations' block-Lanczos runs,
  autotuned block widths) against dense ED: eigenvalues within 1e-10 ||H||,
  residuals <= 1e-8 ||H||, and the same eigenvalues as separate polfed_eigs runs.
"""
import numpy as np
import pytest

import oracle as O
import polfed_inputs as I
from gpu_common import device_basis, lib, torch_dev

pytestmark = pytest.mark.gpu


def _instances():
    # mixed lengths, disorder, orders and targets; XXZ (J2 = 0)
    spec = [(10, 1.0, 0, 0.0), (12, 3.0, 1, 0.0), (14, 8.0, 7, 0.0), (12, 2.0, 60, 0.31),
            (10, 4.0, 150, -0.2), (14, 3.0, 2, 0.0), (12, 6.0, 33, 0.0)]
    out = []
    for k, (L, W, K, sig) in enumerate(spec):
        m = I.xxz(L, W, 21, k)
        H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)
        w, V = np.linalg.eigh(H)
        out.append((m, w, V, K, sig))
    return out


@pytest.mark.parametrize("dtype_name", ["F32", "DF64"])
@pytest.mark.parametrize("n_b", [40, 7])
@pytest.mark.parametrize("ctas", [0, 1])
def test_filter_batched_vs_spectral_definition(dtype_name, n_b, ctas):
    torch, dev = torch_dev()
    pf = lib()
    dtype = getattr(pf, dtype_name)
    tdt = torch.float32 if dtype == pf.F32 else torch.float64
    inst = _instances()
    models, lo, hi, sg, Ks, Xs, Ys, wants, Xh = [], [], [], [], [], [], [], [], []
    for k, (m, w, V, K, sig) in enumerate(inst):
        dim = w.size
        a, b = w[0] - 0.05, w[-1] + 0.07
        X = I.block(dim, n_b, 500 + k)
        wants.append(O.filter_spectral((2 * w - a - b) / (b - a), V, X, sig, K))
        models.append(m)
        lo.append(a)
        hi.append(b)
        sg.append(sig)
        Ks.append(K)
        Xh.append(X)
        Xs.append(torch.from_numpy(X).to(dev, tdt))
        Ys.append(torch.empty((dim, n_b), dtype=tdt, device=dev))
    pf.cheb_filter_batched(models, lo, hi, sg, Ks, Xs, Ys, n_b, dtype, ctas_per_sm=ctas)
    torch.cuda.synchronize()
    for k in range(len(inst)):
        K = Ks[k]
        err = np.abs(Ys[k].double().cpu().numpy() - wants[k]).max() / np.abs(Xh[k]).max()
        tol = {pf.DF64: 1e-12 * (K + 1), pf.F32: 2e-7 * (K + 1) + 1e-6}[dtype]
        assert err < tol, (k, K, err)


def test_filter_batched_j1j2_and_argument_checks():
    torch, dev = torch_dev()
    pf = lib()
    ms = [I.j1j2(12, 4.0, 22, 0), I.j1j2(10, 2.0, 22, 1)]
    Xs, Ys, wants, lo, hi = [], [], [], [], []
    for k, m in enumerate(ms):
        H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)
        w, V = np.linalg.eigh(H)
        a, b = w[0] - 0.1, w[-1] + 0.1
        X = I.block(w.size, 32, 700 + k)
        wants.append((O.filter_spectral((2 * w - a - b) / (b - a), V, X, 0.0, 80), np.abs(X).max()))
        lo.append(a)
        hi.append(b)
        Xs.append(torch.from_numpy(X).to(dev))
        Ys.append(torch.empty_like(Xs[-1]))
    pf.cheb_filter_batched(ms, lo, hi, [0.0, 0.0], [80, 80], Xs, Ys, 32, pf.DF64)
    torch.cuda.synchronize()
    for k in range(2):
        assert np.abs(Ys[k].cpu().numpy() - wants[k][0]).max() / wants[k][1] < 1e-12 * 81
    # J2 = 0 and J2 != 0 cannot share a launch; F64 storage is not batched
    mixed = [ms[0], I.xxz(12, 3.0, 22, 2)]
    with pytest.raises(pf.PolfedError) as e:
        pf.cheb_filter_batched(mixed, lo, hi, [0.0, 0.0], [10, 10], Xs, Ys, 32, pf.DF64)
    assert e.value.code == pf.POLFED_EINVAL
    with pytest.raises(pf.PolfedError) as e:
        pf.cheb_filter_batched(ms, lo, hi, [0.0, 0.0], [10, 10], Xs, Ys, 32, pf.F64)
    assert e.value.code == pf.POLFED_EINVAL
    # an interval that cuts the spectrum is reported, not hidden
    mid = [0.5 * (a + b) for a, b in zip(lo, hi)]
    with pytest.raises(pf.PolfedError) as e:
        pf.cheb_filter_batched(ms, [x - 0.5 for x in mid], [x + 0.5 for x in mid], [0.0, 0.0], [300, 300], Xs, Ys,
                               32, pf.DF64)
    assert e.value.code == pf.POLFED_EBOUNDS


@pytest.mark.parametrize("precision", ["DF64", "F32"])
def test_eigs_batched_against_dense_ed(precision):
    torch, dev = torch_dev()
    pf = lib()
    spec = [(12, 1.0, 20), (14, 3.0, 50), (12, 8.0, 30), (14, 6.0, 40), (12, 2.0, 24), (14, 4.0, 20)]
    models, refs, nevs = [], [], []
    for k, (L, W, n_ev) in enumerate(spec):
        m = I.xxz(L, W, 23, k)
        models.append(m)
        refs.append(O.eigs_nearest(m.L, m.J1, m.J2, m.Delta, m.h, True, 0.5, n_ev))
        nevs.append(n_ev)
    vecs = [torch.empty((n, pf.basis_build(m.L, m.L // 2)), dtype=torch.float64, device=dev)
            for n, m in zip(nevs, models)]
    o = pf.opts_default()
    o.precision = getattr(pf, precision)
    evs, res, sts, status, info, rc = pf.eigs_batched(models, 0.5, nevs, n_b=0, opts=o, d_evecs=vecs,
                                                      allow_fail=True)
    diag = [(k, int(status[k]), sts[k]["n_b"], sts[k]["K"], sts[k]["m"], sts[k]["n_refine"], sts[k]["n_restarts"],
             sts[k]["fallback_df64"], sts[k]["max_resid"] / refs[k]["norm"]) for k in range(len(spec))]
    print("\nbatched", precision, diag)
    assert rc == 0 and list(status) == [0] * len(spec), diag
    assert info["rounds"] > 0 and info["workers"] == len(spec)
    assert info["n_width16"] + info["n_width32"] + info["n_width64"] == len(spec)
    single_calls = sum(s["m"] for s in sts)
    assert info["rounds"] < single_calls  # filter calls of different realizations shared launches
    for k, r in enumerate(refs):
        nrm = r["norm"]
        assert np.max(np.abs(evs[k] - r["evals"])) <= 1e-10 * nrm, (k, np.max(np.abs(evs[k] - r["evals"])) / nrm)
        assert np.max(res[k]) <= 1e-8 * nrm
        V = vecs[k].cpu().numpy().T
        s = np.linalg.svd(r["evecs"].T @ V, compute_uv=False)
        assert s.min() ** 2 >= 1 - 1e-8


def test_eigs_batched_matches_separate_runs_and_fixed_width():
    torch, dev = torch_dev()
    pf = lib()
    models = [I.xxz(14, 3.0, 24, k) for k in range(3)]
    o = pf.opts_default()
    evs, res, sts, status, info, rc = pf.eigs_batched(models, 0.5, 30, n_b=32, opts=o, max_workers=2)
    assert rc == 0 and info["workers"] == 2 and info["n_width32"] == 3
    with pf.Ctx(0) as ctx:
        for k, m in enumerate(models):
            ev, r, st, rc1 = pf.eigs(ctx, m, 0.5, 30, 0, 32, o)
            nrm = max(abs(st["E_min"]), abs(st["E_max"]))
            assert np.max(np.abs(ev - evs[k])) <= 1e-10 * nrm


def test_filter_batched_full_size_matches_single_filters():
    """Realizations of the batched workload's sizes (L = 16 and 18, dim 12870 and
    48620): one batched launch equals separate polfed_cheb_filter calls."""
    torch, dev = torch_dev()
    pf = lib()
    spec = [(16, 2.0, 300), (18, 6.0, 120), (16, 8.0, 37), (18, 1.0, 500)]
    ms, Xs, Ys, Ks, lo, hi = [], [], [], [], [], []
    for k, (L, W, K) in enumerate(spec):
        m = I.xxz(L, W, 25, k)
        dim, st = device_basis(pf, torch, dev, L)
        bound = L * 0.75 + 0.5 * float(np.abs(m.h).sum()) + 0.1  # > ||H||
        ms.append(m)
        Ks.append(K)
        lo.append(-bound)
        hi.append(bound)
        Xs.append(torch.from_numpy(I.block(dim, 16, 900 + k)).to(dev))
        Ys.append(torch.empty_like(Xs[-1]))
    pf.cheb_filter_batched(ms, lo, hi, [0.0] * 4, Ks, Xs, Ys, 16, pf.DF64)
    for k, m in enumerate(ms):
        dim, st = device_basis(pf, torch, dev, m.L)
        Y1 = torch.empty_like(Xs[k])
        pf.cheb_filter(m, st, dim, lo[k], hi[k], 0.0, Ks[k], Xs[k], Y1, 16, pf.DF64)
        err = torch.max(torch.abs(Ys[k] - Y1)).item() / torch.max(torch.abs(Xs[k])).item()
        assert err < 1e-12 * (Ks[k] + 1), (k, err)
