"""GPU parity of the density-of-states machinery and of the learned predictor.

* KPM moments (polfed_kpm_moments) against the oracle's moments written
  through the eigen-decomposition, with the same random block.
* polfed_kpm_count against the oracle's damped count.
* polfed_spectral_bounds / polfed_spectral_labels against dense ED.
* MLP forward, gradient and Adam step against the FP64 oracle network.
* polfed_eigs under every DOS rule against dense ED, bounds hints accepted
  and rejected by the Lanczos probe.
* What the trained predictor gains: the K it sets puts the accessible-window
  count closer to the requested (1 + k_margin) N_ev than the paper's
  analytic Gamma rule does.
"""
import math

import numpy as np
import pytest

import oracle as O
import polfed_inputs as I
from gpu_common import device_basis, lib, torch_dev
from oracle import kpm_oracle as KO
from oracle import mlp_oracle as MO

pytestmark = pytest.mark.gpu


def _spectrum(m, pad=1e-3):
    H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)
    ev, V = np.linalg.eigh(H)
    w = ev[-1] - ev[0]
    e_lo, e_hi = ev[0] - pad * w, ev[-1] + pad * w
    return ev, V, e_lo, e_hi, (2 * ev - e_lo - e_hi) / (e_hi - e_lo)


# ------------------------------------------------------------------ KPM

@pytest.mark.parametrize("L,which", [(10, "xxz"), (12, "j1j2"), (12, "obc")])
@pytest.mark.parametrize("dtype,tol", [("F64", 1e-11), ("DF64", 1e-11), ("F32", 2e-4)])
@pytest.mark.parametrize("n_mom", [2, 33, 96])
def test_kpm_moments_parity(L, which, dtype, tol, n_mom):
    torch, dev = torch_dev()
    pf = lib()
    m = {"xxz": I.xxz(L, 3.0, 11, 0), "j1j2": I.j1j2(L, 4.0, 11, 1),
         "obc": I.xxz(L, 2.0, 11, 2, periodic=False)}[which]
    ev, V, e_lo, e_hi, evt = _spectrum(m)
    dim, st = device_basis(pf, torch, dev, L)
    R = 7
    Rb = I.block(dim, R, seed=100 + L)
    want = KO.moments_from_spectrum(evt, V, Rb, n_mom)
    tdt = torch.float32 if dtype == "F32" else torch.float64
    dR = torch.from_numpy(Rb).to(dev, tdt)
    got = pf.kpm_moments(m, st, dim, e_lo, e_hi, n_mom, dR, R, getattr(pf, dtype))
    assert got.shape == (n_mom,)
    assert np.max(np.abs(got - want)) <= tol * want[0], np.max(np.abs(got - want)) / want[0]


def test_kpm_count_matches_oracle_and_bounds_error():
    torch, dev = torch_dev()
    pf = lib()
    m = I.xxz(12, 3.0, 11, 5)
    ev, V, e_lo, e_hi, evt = _spectrum(m)
    mu = KO.trace_moments(evt, 300)
    for xa, xb in [(-1.0, 1.0), (-0.05, 0.05), (-0.4, 0.1), (0.2, 0.9)]:
        assert pf.kpm_count(mu, xa, xb) == pytest.approx(KO.count_fraction(mu, xa, xb), abs=1e-13)
    # an interval that cuts the spectrum makes |mu_n| exceed mu_0
    dim, st = device_basis(pf, torch, dev, 12)
    dR = torch.from_numpy(I.block(dim, 4, seed=3)).to(dev)
    mid = 0.5 * (ev[0] + ev[-1])
    with pytest.raises(pf.PolfedError) as e:
        pf.kpm_moments(m, st, dim, mid - 0.2 * (ev[-1] - ev[0]), mid + 0.2 * (ev[-1] - ev[0]), 200, dR, 4, pf.F64)
    assert e.value.code == pf.POLFED_EBOUNDS


def _exact_rho_eps(evt, ev, e_lo, e_hi, n_mom=256):
    """Oracle value of the label rho_eps: the Jackson-damped exact-trace count of
    the same window around eps = 0.5, per unit eps and per state."""
    mu = KO.trace_moments(evt, n_mom)
    Es = 0.5 * (ev[0] + ev[-1])
    sig = (2 * Es - e_lo - e_hi) / (e_hi - e_lo)
    d = max(0.01, 8.0 / n_mom)
    xa, xb = max(-1.0, sig - d), min(1.0, sig + d)
    f = KO.count_fraction(mu, xa, xb)
    return f / (xb - xa) * 2.0 / (e_hi - e_lo) * (ev[-1] - ev[0])


@pytest.mark.parametrize("m", [I.xxz(14, 3.0, 12, 0), I.j1j2(12, 4.0, 12, 1), I.xxz(14, 1.0, 12, 2)])
def test_spectral_bounds_and_labels(m):
    torch, dev = torch_dev()
    pf = lib()
    ev, V, _, _, _ = _spectrum(m)
    nrm = max(abs(ev[0]), abs(ev[-1]))
    with pf.Ctx(0) as ctx:
        lo, hi, err = pf.spectral_bounds(ctx, m)
        lab = pf.spectral_labels(ctx, m, 0.5, 256, 16)
    assert abs(lo - ev[0]) <= 1e-10 * nrm and abs(hi - ev[-1]) <= 1e-10 * nrm
    assert err <= 1e-10 * nrm
    assert abs(lab[0] - ev[0]) <= 1e-10 * nrm and abs(lab[1] - ev[-1]) <= 1e-10 * nrm
    w = ev[-1] - ev[0]
    pad = 1e-6 * w + 10 * err
    e_lo, e_hi = ev[0] - pad, ev[-1] + pad
    want = _exact_rho_eps((2 * ev - e_lo - e_hi) / (e_hi - e_lo), ev, e_lo, e_hi)
    # stochastic trace with 16 vectors: relative std ~ sqrt(2 / (16 * states in window)) < 3% here
    assert lab[2] == pytest.approx(want, rel=0.12)


# ------------------------------------------------------------------ MLP

def _net_and_params(pf, d_in, H, d_out, seed):
    rng = np.random.default_rng(seed)
    p = MO.glorot_params(d_in, H, d_out, rng).astype(np.float32)
    p[H * d_in:H * d_in + H] = (0.2 * rng.standard_normal(H)).astype(np.float32)
    p[-d_out:] = (0.3 * rng.standard_normal(d_out)).astype(np.float32)
    sc = (rng.normal(size=d_in).astype(np.float32), rng.uniform(0.5, 2, d_in).astype(np.float32),
          rng.normal(size=d_out).astype(np.float32), rng.uniform(0.5, 2, d_out).astype(np.float32))
    net = pf.MLP(d_in, H, d_out, seed=seed)
    net.set_params(p)
    net.set_scaling(*sc)
    sc64 = tuple(np.asarray(v, dtype=np.float64) for v in sc)
    return net, p.astype(np.float64), sc64, rng


@pytest.mark.parametrize("d_in,H,B", [(23, 128, 64), (15, 128, 1), (7, 32, 300)])
def test_mlp_forward_and_gradient_parity(d_in, H, B):
    torch, dev = torch_dev()
    pf = lib()
    d_out = 3
    net, p, sc, rng = _net_and_params(pf, d_in, H, d_out, seed=d_in)
    assert net.num_params == MO.n_params(d_in, H, d_out)
    assert np.array_equal(net.get_params().astype(np.float64), p)
    x = rng.normal(size=(B, d_in)).astype(np.float32)
    t = rng.normal(size=(B, d_out)).astype(np.float32)
    dx = torch.from_numpy(x).to(dev)
    dt = torch.from_numpy(t).to(dev)
    dy = torch.empty((B, d_out), dtype=torch.float32, device=dev)
    net.forward(dx, B, dy)
    want = MO.predict(p, x.astype(np.float64), d_in, H, d_out, sc)
    assert np.max(np.abs(dy.cpu().numpy() - want)) <= 1e-5 * max(1.0, np.max(np.abs(want)))
    g = torch.empty(net.num_params, dtype=torch.float32, device=dev)
    loss = net.grad(dx, dt, B, g)
    wl, wg = MO.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64), d_in, H, d_out, sc)
    assert loss == pytest.approx(wl, rel=1e-5)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gg - wg)) <= 2e-5 * np.max(np.abs(wg)), np.max(np.abs(gg - wg)) / np.max(np.abs(wg))


def test_mlp_adam_steps_parity():
    torch, dev = torch_dev()
    pf = lib()
    d_in, H, d_out, B = 23, 128, 3, 32
    net, p, sc, rng = _net_and_params(pf, d_in, H, d_out, seed=77)
    x = rng.normal(size=(B, d_in)).astype(np.float32)
    t = rng.normal(size=(B, d_out)).astype(np.float32)
    dx, dt = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    lr = 1e-3
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    q = p.copy()
    for step in range(1, 4):
        net.train_step(dx, dt, B, lr)
        _, g = MO.loss_and_grad(q, x.astype(np.float64), t.astype(np.float64), d_in, H, d_out, sc)
        q, m, v = MO.adam_step(q, g, m, v, step, lr)
    got = net.get_params().astype(np.float64)
    # Adam moves each parameter by about lr per step; where |g| is tiny the
    # FP32 gradient's rounding can flip the step, so compare the rest tightly
    big = np.abs(m) > 1e-3 * np.max(np.abs(m))
    assert np.max(np.abs(got - q)[big]) <= 2e-3 * lr * 3
    assert np.max(np.abs(got - q)) <= 3 * 2 * lr


def test_mlp_feature_and_target_conventions():
    torch, dev = torch_dev()
    pf = lib()
    m = I.xxz(16, 2.5, 13, 0)
    x = pf.mlp_features(m, 2.5)
    assert np.array_equal(x, np.concatenate([m.h, [2.5]]).astype(np.float32))
    y = pf.mlp_targets(16, [-20.0, 12.0, 1.7])
    assert np.array_equal(y, np.array([-20.0 / 16, 12.0 / 16, math.log(1.7)], dtype=np.float32))
    net = pf.MLP(17, 128, 3, seed=5)
    out = net.predict(m, 2.5)
    dx = torch.from_numpy(x[None, :]).to(dev)
    dy = torch.empty((1, 3), dtype=torch.float32, device=dev)
    net.forward(dx, 1, dy)
    yy = dy.cpu().numpy()[0].astype(np.float64)
    assert out[0] == pytest.approx(yy[0] * 16, rel=1e-6) and out[1] == pytest.approx(yy[1] * 16, rel=1e-6)
    assert out[2] == pytest.approx(math.exp(yy[2]), rel=1e-6)


def test_mlp_training_kernels_fit_a_smooth_function():
    torch, dev = torch_dev()
    pf = lib()
    from paper_2005_09534_gb300 import predictor
    rng = np.random.default_rng(8)
    X = rng.uniform(-1, 1, size=(2048, 6)).astype(np.float32)
    Y = np.stack([np.sum(X * X, 1), np.sin(2 * X[:, 0]) * X[:, 1], X[:, 2] - X[:, 3]], 1).astype(np.float32)
    net = pf.MLP(6, 64, 3, seed=1)
    net.set_scaling(X.mean(0), X.std(0), Y.mean(0), Y.std(0))
    dX, dY = torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev)
    l0 = net.grad(dX, dY, 2048)
    loss, _ = predictor.fit(net, X, Y, steps=1500, lr=3e-3, batch=256)
    assert loss < l0 / 30, (l0, loss)


# ------------------------------------------------------- DOS rules in polfed_eigs

def _eigs(pf, torch, dev, m, n_ev, n_b, o, allow_noconv=False):
    dim = pf.basis_build(m.L, m.L // 2)
    vecs = torch.empty((n_ev, dim), dtype=torch.float64, device=dev)
    with pf.Ctx(0) as ctx:
        ev, res, st, rc = pf.eigs(ctx, m, 0.5, n_ev, 0, n_b, o, d_evecs=vecs, allow_noconv=allow_noconv)
    return ev, res, st


@pytest.mark.parametrize("rule", ["DOS_MOMENTS", "DOS_GAMMA", "DOS_KPM", "DOS_HINT"])
def test_eigs_under_each_dos_rule(rule):
    torch, dev = torch_dev()
    pf = lib()
    m = I.xxz(14, 3.0, 1, 1)
    r = O.eigs_nearest(m.L, m.J1, m.J2, m.Delta, m.h, True, 0.5, 50)
    o = pf.opts_default()
    o.dos_rule = getattr(pf, rule)
    if rule == "DOS_HINT":
        ev_all = r["spectrum"]
        o.rho_hint = _exact_rho_eps((2 * ev_all - ev_all[0] - ev_all[-1]) / (ev_all[-1] - ev_all[0]), ev_all,
                                    ev_all[0], ev_all[-1])
    ev, res, st = _eigs(pf, torch, dev, m, 50, 16, o)
    nrm = r["norm"]
    assert st["dos_rule"] == o.dos_rule
    assert np.max(np.abs(ev - r["evals"])) <= 1e-10 * nrm
    assert np.max(res) <= 1e-8 * nrm


def test_bounds_hints_are_checked_by_the_probe():
    torch, dev = torch_dev()
    pf = lib()
    m = I.xxz(14, 3.0, 1, 2)
    r = O.eigs_nearest(m.L, m.J1, m.J2, m.Delta, m.h, True, 0.5, 40)
    lo, hi = r["E_min"], r["E_max"]
    w = hi - lo
    for emin, emax, accepted in [(lo - 0.01 * w, hi + 0.01 * w, 1),   # contains the spectrum, 2% looser
                                 (lo + 0.01 * w, hi + 0.01 * w, 0),   # cuts the spectrum: rejected
                                 (lo - 0.2 * w, hi + 0.2 * w, 0)]:    # too loose: rejected
        o = pf.opts_default()
        o.dos_rule = pf.DOS_HINT
        o.rho_hint = 1.0
        o.emin_hint, o.emax_hint = emin, emax
        ev, res, st = _eigs(pf, torch, dev, m, 40, 16, o)
        assert st["bounds_from_hint"] == accepted
        if accepted:
            assert st["e_lo"] == emin and st["e_hi"] == emax
        assert np.max(np.abs(ev - r["evals"])) <= 1e-10 * r["norm"]
        assert np.max(res) <= 1e-8 * r["norm"]


# ---------------------------------------------------------------- the gain

def _realizations(L, n, config, w_lo=1.0, w_hi=8.0):
    out = []
    for k in range(n):
        W = w_lo + (w_hi - w_lo) * ((0.6180339887498949 * (k + 1)) % 1.0)
        h = I.fields(L, W, config, k)
        out.append((I.Model(L, 1.0, 0.0, 1.0, h, True, W), W))
    return out


def test_trained_predictor_sets_K_better_than_the_gamma_rule():
    """Train the network on labels the method produced (Lanczos bounds, KPM
    counts) for 160 L=14 XXZ rings with W in [1, 8]; then, on 12 unseen rings
    at W in {1, 2, 3, 4, 6, 8}, compare the density of states each rule feeds
    to the choice of K against the oracle's (exact eigenvalues, same Jackson
    window), and the POLFED runs those K values lead to.  The library's
    default rule (exact sector moments, Gaussian density) is measured beside
    the two and printed; the assertions compare the network with the paper's
    Gamma rule."""
    torch, dev = torch_dev()
    pf = lib()
    from paper_2005_09534_gb300 import predictor
    L, n_ev, n_b = 14, 50, 16
    train = _realizations(L, 160, config=40)
    with pf.Ctx(0) as ctx:
        labels = predictor.labels_for(ctx, [m for m, _ in train])
    X, Y = predictor.dataset([m for m, _ in train], [W for _, W in train], labels)
    net = pf.MLP(L + 1, 128, 3, seed=3)
    loss, secs = predictor.fit(net, X, Y, steps=6000, lr=2e-3, batch=256)
    rows = []
    for k, W in enumerate([1, 2, 3, 4, 6, 8] * 2):
        h = I.fields(L, W, 41, k)
        m = I.Model(L, 1.0, 0.0, 1.0, h, True, W)
        ev = np.linalg.eigvalsh(O.dense_hamiltonian(L, 1.0, 0.0, 1.0, h, True)[0])
        nrm = max(abs(ev[0]), abs(ev[-1]))
        pred = net.predict(m, W)
        assert abs(pred[0] - ev[0]) < 0.1 * (ev[-1] - ev[0]) and abs(pred[1] - ev[-1]) < 0.1 * (ev[-1] - ev[0])
        row = {"W": W}
        for rule in ("mlp", "gamma", "moments"):
            o = pf.opts_default()
            if rule == "mlp":
                o.dos_rule = pf.DOS_HINT
                o.rho_hint = pred[2]
            elif rule == "gamma":
                o.dos_rule = pf.DOS_GAMMA
            else:
                o.dos_rule = pf.DOS_MOMENTS
            evg, res, st = _eigs(pf, torch, dev, m, n_ev, n_b, o, allow_noconv=True)
            lo, hi = st["e_lo"], st["e_hi"]
            evt = (2 * ev - lo - hi) / (hi - lo)
            rho_true = _exact_rho_eps(evt, ev, lo, hi) * ev.size / (ev[-1] - ev[0]) * 0.5 * (hi - lo)
            row[rule] = {"dos_err": abs(math.log(st["rho_sigma"] / rho_true)), "status": st["status"],
                         "restarts": st["n_restarts"], "matvecs": st["matvec_cols"], "K": st["K"],
                         "resid": float(np.max(res) / nrm) if len(res) else 1.0}
        rows.append(row)
    for r in rows:
        print("W %g" % r["W"] + "".join(
            " | %s: dos err %.3f K %d restarts %d matvecs %d" % (k, r[k]["dos_err"], r[k]["K"], r[k]["restarts"],
                                                                r[k]["matvecs"]) for k in ("mlp", "gamma", "moments")))
    e_mlp = float(np.mean([r["mlp"]["dos_err"] for r in rows]))
    e_gam = float(np.mean([r["gamma"]["dos_err"] for r in rows]))
    e_mom = float(np.mean([r["moments"]["dos_err"] for r in rows]))
    mv = {k: sum(r[k]["matvecs"] for r in rows) for k in ("mlp", "gamma", "moments")}
    rs = {k: sum(r[k]["restarts"] for r in rows) for k in ("mlp", "gamma", "moments")}
    print(f"mean |log(rho_rule / rho_exact)|: MLP {e_mlp:.4f}  Gamma {e_gam:.4f}  moments {e_mom:.4f}; "
          f"matvec columns {mv}; restarts {rs}; train loss {loss:.3e} in {secs:.1f} s")
    for r in rows:
        assert r["moments"]["status"] == 0 and r["moments"]["resid"] <= 1e-8
    for r in rows:
        assert r["mlp"]["status"] == 0 and r["mlp"]["resid"] <= 1e-8
    assert e_mlp < e_gam
    assert sum(r["mlp"]["restarts"] for r in rows) <= sum(r["gamma"]["restarts"] for r in rows)
