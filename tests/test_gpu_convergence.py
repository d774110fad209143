"""Convergence of POLFED (Supplement, "Convergence of POLFED", Fig. S1): the
number of converged eigenvalues stays near zero until the Lanczos basis holds
about 2 N_ev columns, then rises to N_ev, and a run needs fewer than 2.8 N_ev
columns in all.  The paper shows this for the J1-J2 chain at W = 5.4; here it
is checked on J1-J2 rings of L = 16 and 18 (three realizations each, block size
s = 16, K chosen for N_ev accessible eigenvalues as in the paper, float-float
filter), from the library's record of every convergence check.  The order
rule's scaling K ~ 1 / N_ev (N_ev -> 2 N_ev halves K) is checked on the same
realizations."""
import numpy as np
import pytest

import polfed_inputs as I
from gpu_common import lib, torch_dev

pytestmark = pytest.mark.gpu


def _run(pf, m, n_ev, n_b=16):
    o = pf.opts_default()
    o.precision = pf.DF64
    o.k_margin = 0.0  # the paper's rule: N_ev eigenvalues with P >= p
    with pf.Ctx(0) as ctx:
        ev, res, st, rc = pf.eigs(ctx, m, 0.5, n_ev, 0, n_b, o, allow_noconv=True)
        hist = pf.history(ctx)
    return ev, res, st, rc, hist


@pytest.mark.parametrize("L,n_ev", [(16, 100), (18, 200)])
def test_convergence_onset_and_column_budget(L, n_ev):
    torch, dev = torch_dev()
    pf = lib()
    rows = []
    for r in range(3):
        m = I.j1j2(L, 5.4, 8, r)
        ev, res, st, rc, hist = _run(pf, m, n_ev)
        hist = [h for h in hist if h["attempt"] == hist[-1]["attempt"]]  # the attempt that finished
        assert rc == 0 and len(ev) == n_ev
        hn = max(abs(st["E_min"]), abs(st["E_max"]))
        assert np.max(res) <= 1e-8 * hn
        cols = np.array([h["cols"] for h in hist])
        conv = np.array([h["n_conv"] for h in hist])
        # onset: the first check with at least 5% of N_ev converged
        onset = cols[np.argmax(conv >= 0.05 * n_ev)] if np.any(conv >= 0.05 * n_ev) else cols[-1]
        rows.append((r, st["K"], onset / n_ev, cols[-1] / n_ev, list(zip(cols.tolist(), conv.tolist()))))
        # before the onset almost nothing is converged
        assert np.all(conv[cols < 1.4 * n_ev] <= 0.05 * n_ev), rows[-1]
        assert 1.4 <= onset / n_ev <= 2.6, rows[-1]
        assert cols[-1] < 2.8 * n_ev, rows[-1]
    print(rows)


def test_order_scales_inversely_with_n_ev():
    torch, dev = torch_dev()
    pf = lib()
    m = I.j1j2(16, 5.4, 8, 0)
    o = pf.opts_default()
    o.precision = pf.DF64
    o.k_margin = 0.0
    Ks = []
    for n_ev in (50, 100, 200):
        with pf.Ctx(0) as ctx:
            ev, res, st, rc = pf.eigs(ctx, m, 0.5, n_ev, 0, 16, o, allow_noconv=True)
        assert st["n_restarts"] == 0
        Ks.append(st["K"])
    assert abs(Ks[0] / Ks[1] - 2.0) < 0.05 and abs(Ks[1] / Ks[2] - 2.0) < 0.05, Ks
