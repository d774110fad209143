"""Observables on the GPU (polfed_gap_ratio, polfed_entanglement_entropy) against
the oracle (section "Entanglement entropy and level statistics"): the mean gap
ratio and the half-chain entanglement entropy averaged over the L cuts."""
import math

import numpy as np
import pytest

import oracle as O
import polfed_inputs as I
from gpu_common import device_basis, lib, torch_dev

pytestmark = pytest.mark.gpu


def test_gap_ratio_matches_oracle():
    torch, dev = torch_dev()
    pf = lib()
    rng = np.random.default_rng(3)
    for n in (3, 17, 1000, 5003):
        e = np.sort(rng.standard_normal(n))
        d = torch.from_numpy(e).to(dev)
        r_d = torch.empty(n - 2, dtype=torch.float64, device=dev)
        got = pf.gap_ratio(d, n, r_d)
        assert abs(got - O.gap_ratio(e)) <= 1e-14
        g = np.diff(e)
        want = np.minimum(g[:-1], g[1:]) / np.maximum(g[:-1], g[1:])
        assert np.max(np.abs(r_d.cpu().numpy() - want)) <= 1e-15
    # by hand: levels 0, 1, 3, 4 -> r = (1/2, 1/2)
    assert abs(pf.gap_ratio(torch.tensor([0.0, 1.0, 3.0, 4.0], dtype=torch.float64, device=dev), 4) - 0.5) < 1e-15


def test_gap_ratio_rejects_unsorted_and_undefined():
    torch, dev = torch_dev()
    pf = lib()
    with pytest.raises(pf.PolfedError) as e:
        pf.gap_ratio(torch.tensor([0.0, 2.0, 1.0, 3.0], dtype=torch.float64, device=dev), 4)
    assert e.value.code == pf.POLFED_EINVAL
    with pytest.raises(pf.PolfedError) as e:
        pf.gap_ratio(torch.tensor([1.0, 1.0, 1.0], dtype=torch.float64, device=dev), 3)
    assert e.value.code == pf.POLFED_EINVAL


@pytest.mark.parametrize("L", [4, 8, 10, 12, 14])
def test_entropy_random_vectors_match_oracle(L):
    """Random normalized sector vectors: every cut and the average, FP64 both sides."""
    torch, dev = torch_dev()
    pf = lib()
    dim, st = device_basis(pf, torch, dev, L)
    states = O.basis(L)
    rng = np.random.default_rng(L)
    nv = 3
    V = rng.standard_normal((nv, dim))
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    Vd = torch.from_numpy(V).to(dev)  # row v = vector v: column-major dim x nv with ld = dim
    with pf.Ctx(0) as ctx:
        per = pf.entanglement_entropy(ctx, L, st, Vd, dim, nv, per_cut=True)
        avg = pf.entanglement_entropy(ctx, L, st, Vd, dim, nv)
    for v in range(nv):
        want = [O.entanglement_entropy_cut(V[v], states, L, x) for x in range(L)]
        assert np.max(np.abs(per[v] - want)) <= 1e-11, (v, per[v], want)
        assert abs(avg[v] - np.mean(want)) <= 1e-11


def test_entropy_product_and_dimer_states():
    """By hand: a product state has S = 0 at every cut; singlets on the bonds
    (0,1), (2,3), (4,5), (6,7) of an L = 8 ring give S = 0 at even cuts (no
    singlet is cut) and 2 ln 2 at odd cuts (two singlets are cut)."""
    torch, dev = torch_dev()
    pf = lib()
    L = 8
    dim, st = device_basis(pf, torch, dev, L)
    states = O.basis(L)
    prod = np.zeros(dim)
    prod[0] = 1.0
    dimer = np.zeros(dim)
    for s_idx, s in enumerate(states):
        amp = 1.0
        for b in range(0, L, 2):
            pair = (int(s) >> b) & 3
            if pair == 0b01:
                amp *= 1.0 / math.sqrt(2)
            elif pair == 0b10:
                amp *= -1.0 / math.sqrt(2)
            else:
                amp = 0.0
        dimer[s_idx] = amp
    assert abs(np.linalg.norm(dimer) - 1.0) < 1e-14
    V = torch.from_numpy(np.stack([prod, dimer])).to(dev)
    with pf.Ctx(0) as ctx:
        per = pf.entanglement_entropy(ctx, L, st, V, dim, 2, per_cut=True)
    assert np.max(np.abs(per[0])) < 1e-13
    want = [0.0 if x % 2 == 0 else 2 * math.log(2) for x in range(L)]
    assert np.max(np.abs(per[1] - want)) < 1e-12


def test_observables_of_polfed_eigenpairs_L14():
    """The 1e-8 observables bar on the method's own output: L = 14 XXZ ring,
    W = 3, N_ev = 50 at eps = 0.5 from the float-float path; the GPU gap ratio
    and the GPU entropies of the GPU eigenvectors are within 1e-8 of the
    oracle's values on the dense-ED eigenpairs."""
    torch, dev = torch_dev()
    pf = lib()
    m = I.xxz(14, 3.0, 1, 0)
    r = O.eigs_nearest(m.L, m.J1, m.J2, m.Delta, m.h, True, 0.5, 50)
    dim, st = device_basis(pf, torch, dev, m.L)
    vecs = torch.empty((50, dim), dtype=torch.float64, device=dev)
    o = pf.opts_default()
    o.precision = pf.DF64
    with pf.Ctx(0) as ctx:
        ev, res, stats, rc = pf.eigs(ctx, m, 0.5, 50, 0, 16, o, d_evecs=vecs)
        S_gpu = pf.entanglement_entropy(ctx, m.L, st, vecs, dim, 50)
    rbar = pf.gap_ratio(torch.from_numpy(ev).to(dev), 50)
    assert abs(rbar - O.gap_ratio(r["evals"])) <= 1e-8
    S_or = np.array([O.entanglement_entropy(r["evecs"][:, i], r["states"], m.L) for i in range(50)])
    assert np.max(np.abs(S_gpu - S_or)) <= 1e-8, np.max(np.abs(S_gpu - S_or))
    # s_E = S_E / S_RMT is well inside (0, 1) at W = 3 (intermediate regime)
    sE = S_gpu.mean() / O.s_rmt(m.L)
    assert 0.05 < sE < 1.0


def test_entropy_L22_sampled_against_oracle():
    """Headline size: two random L = 22 sector vectors (dim 705432), the GPU
    entropy of cut 0 and cut 5 against the oracle's block SVD."""
    torch, dev = torch_dev()
    pf = lib()
    L = 22
    dim, st = device_basis(pf, torch, dev, L)
    states = O.basis(L)
    rng = np.random.default_rng(22)
    V = rng.standard_normal((2, dim))
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    with pf.Ctx(0) as ctx:
        per = pf.entanglement_entropy(ctx, L, st, torch.from_numpy(V).to(dev), dim, 2, per_cut=True)
    for v in range(2):
        for x in (0, 5):
            want = O.entanglement_entropy_cut(V[v], states, L, x)
            assert abs(per[v][x] - want) <= 1e-10, (v, x, per[v][x], want)
        assert abs(per[v][3] - per[v][3 + L // 2]) < 1e-14  # complement: same entropy

