"""Host-only entry points of the library (no GPU needed) against the oracle,
and the symmetry copies the predictor's training set relies on."""
import math

import numpy as np
import pytest

import polfed_inputs as I
from oracle import kpm_oracle as KO
from oracle import polfed_oracle as O


@pytest.fixture(scope="module")
def pf():
    import shutil
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_2005_09534_gb300 import build
    build.build()
    import paper_2005_09534_gb300 as m
    m.load()
    return m


def test_kpm_count_host_matches_oracle(pf):
    m = I.xxz(10, 2.5, 31, 0)
    H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)
    ev = np.linalg.eigvalsh(H)
    lo, hi = ev[0] - 0.1, ev[-1] + 0.1
    mu = KO.trace_moments((2 * ev - lo - hi) / (hi - lo), 200)
    for xa, xb in [(-1.0, 1.0), (-0.2, 0.1), (0.5, 0.51), (-0.9, -0.8)]:
        assert pf.kpm_count(mu, xa, xb) == pytest.approx(KO.count_fraction(mu, xa, xb), abs=1e-13)
    with pytest.raises(pf.PolfedError) as e:
        pf.kpm_count(mu, 0.3, 0.2)
    assert e.value.code == pf.POLFED_EINVAL


def test_predictor_feature_and_target_conventions(pf):
    m = I.j1j2(12, 4.0, 31, 1)
    x = pf.mlp_features(m, 4.0)
    assert x.dtype == np.float32 and np.array_equal(x, np.concatenate([m.h, [4.0]]).astype(np.float32))
    y = pf.mlp_targets(12, [-15.5, 9.25, 0.8])
    assert np.array_equal(y, np.array([-15.5 / 12, 9.25 / 12, math.log(0.8)], dtype=np.float32))
    with pytest.raises(pf.PolfedError):
        pf.mlp_targets(12, [-1.0, 1.0, 0.0])  # the density must be positive


def test_symmetry_copies_share_the_spectrum():
    """Every field vector predictor.symmetric_copies produces (cyclic shifts,
    reflection, h -> -h on a ring; reflection and h -> -h on an open chain) has
    the sector spectrum of the original: the training labels are shared."""
    from paper_2005_09534_gb300.predictor import symmetric_copies
    for periodic, J2 in [(True, 0.0), (True, 1.0), (False, 0.7)]:
        L = 8
        h = I.fields(L, 3.0, 32, int(J2 * 10) + periodic)
        ref = np.linalg.eigvalsh(O.dense_hamiltonian(L, 1.0, J2, 0.55, h, periodic)[0])
        copies = symmetric_copies(h, periodic)
        assert len(copies) == (4 * L if periodic else 4)
        for c in copies:
            ev = np.linalg.eigvalsh(O.dense_hamiltonian(L, 1.0, J2, 0.55, c, periodic)[0])
            assert np.max(np.abs(ev - ref)) < 1e-11


def test_predictor_dataset_rows(pf):
    """dataset() stacks one feature/target row per symmetry copy, with the shared labels."""
    from paper_2005_09534_gb300 import predictor
    ms = [I.xxz(10, 2.0, 33, 0), I.xxz(10, 5.0, 33, 1)]
    labels = np.array([[-9.0, 7.0, 1.1], [-12.0, 10.0, 0.9]])
    X, Y = predictor.dataset(ms, [2.0, 5.0], labels)
    assert X.shape == (2 * 40, 11) and Y.shape == (2 * 40, 3)
    assert np.all(X[:40, 10] == 2.0) and np.all(X[40:, 10] == 5.0)
    assert np.allclose(Y[:40], pf.mlp_targets(10, labels[0])) and np.allclose(Y[40:], pf.mlp_targets(10, labels[1]))
    # every copy's fields are a symmetry image of the original ring's fields
    for k in range(40):
        assert np.isclose(np.sort(np.abs(X[k, :10])), np.sort(np.abs(ms[0].h).astype(np.float32))).all()
