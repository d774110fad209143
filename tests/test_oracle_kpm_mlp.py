"""Pins of the density-of-states oracle (KPM, Gaussian rules) and of the MLP oracle.

CPU only.  Each pin checks the oracle against something other than itself:
dense matrix polynomials, brute-force counts, quadrature, finite differences,
closed forms of the Adam update.
"""
import math

import numpy as np
import pytest

import polfed_inputs as pi
from oracle import kpm_oracle as KO
from oracle import mlp_oracle as MO
from oracle import polfed_oracle as O


def _rescaled(m, pad=1e-3):
    H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, m.periodic)
    ev, V = np.linalg.eigh(H)
    w = ev[-1] - ev[0]
    e_lo, e_hi = ev[0] - pad * w, ev[-1] + pad * w
    Ht = O.rescale_matrix(H, e_lo, e_hi)
    evt = (2 * ev - e_lo - e_hi) / (e_hi - e_lo)
    return H, Ht, ev, evt, V


def _dense_cheb(Ht, n_mom):
    """T_n(H~) by the matrix three-term recurrence (not via eigenvalues)."""
    T = [np.eye(Ht.shape[0]), Ht.copy()]
    for _ in range(2, n_mom):
        T.append(2 * Ht @ T[-1] - T[-2])
    return T[:n_mom]


# ----------------------------------------------------------------------- KPM

def test_trace_moments_equal_dense_matrix_polynomials():
    m = pi.xxz(8, 2.0, config=7, realization=1)
    _, Ht, _, evt, _ = _rescaled(m)
    T = _dense_cheb(Ht, 24)
    mu = KO.trace_moments(evt, 24)
    ref = np.array([np.trace(t) for t in T])
    assert np.max(np.abs(mu - ref)) < 1e-10 * Ht.shape[0]


def test_stochastic_moments_equal_quadratic_forms():
    m = pi.j1j2(8, 3.0, config=7, realization=2)
    _, Ht, _, evt, V = _rescaled(m)
    R = pi.block(Ht.shape[0], 3, seed=11)
    T = _dense_cheb(Ht, 20)
    ref = np.array([np.mean([R[:, j] @ t @ R[:, j] for j in range(3)]) for t in T])
    mu = KO.moments_from_spectrum(evt, V, R, 20)
    assert np.max(np.abs(mu - ref)) < 1e-11 * np.abs(ref[0])
    # the identity block turns the stochastic average into the exact trace / dim
    n = Ht.shape[0]
    mu_id = KO.moments_from_spectrum(evt, V, np.eye(n), 20)
    assert np.max(np.abs(mu_id * n - KO.trace_moments(evt, 20))) < 1e-10 * n


def test_jackson_factors_and_kernel_width():
    for N in (16, 64, 257):
        g = KO.jackson(N)
        assert g[0] == pytest.approx(1.0, abs=1e-15)
        assert np.all(g > -1e-15) and np.all(g <= 1.0 + 1e-15)
        assert np.all(np.diff(g) < 1e-15)
    # one eigenvalue at 0: the damped density is a positive bump of unit mass and
    # variance (pi / N)^2 to leading order (Weisse et al., section II.C)
    N = 200
    mu = np.cos(np.arange(N) * math.pi / 2)  # T_n(0)
    x = np.cos(math.pi * (np.arange(20000) + 0.5) / 20000)  # Chebyshev nodes: int f dx = pi/M sum f sqrt(1-x^2)
    rho = KO.kpm_density(mu, x)
    wts = math.pi / 20000 * np.sqrt(1 - x * x)
    assert np.min(rho) > -1e-10
    assert np.sum(rho * wts) == pytest.approx(1.0, abs=1e-9)
    var = np.sum(rho * x * x * wts)
    assert var == pytest.approx((math.pi / N) ** 2, rel=0.05)


def test_indicator_coefficients_match_quadrature():
    M = 400000
    th = math.pi * (np.arange(M) + 0.5) / M
    x = np.cos(th)
    for xa, xb in [(-0.3, 0.2), (0.0, 0.05), (-1.0, 1.0), (0.7, 0.99)]:
        chi = ((x >= xa) & (x <= xb)).astype(float)
        c = KO.indicator_coeffs(40, xa, xb)
        for n in range(40):
            q = (1.0 if n == 0 else 2.0) / M * np.sum(chi * np.cos(n * th))
            assert abs(q - c[n]) < 2e-5, (xa, xb, n)


def test_count_fraction_whole_interval_and_exact_count():
    m = pi.xxz(12, 3.0, config=7, realization=3)
    _, _, _, evt, _ = _rescaled(m)
    mu = KO.trace_moments(evt, 3000)
    assert KO.count_fraction(mu, -1.0, 1.0) == pytest.approx(1.0, abs=1e-12)
    n = evt.size
    for xa, xb in [(-0.1, 0.1), (-0.5, 0.02), (0.3, 0.6)]:
        exact = np.sum((evt >= xa) & (evt <= xb)) / n
        edge = 6 * math.pi / 3000
        slack = (np.sum(np.abs(evt - xa) < edge) + np.sum(np.abs(evt - xb) < edge)) / n
        assert abs(KO.count_fraction(mu, xa, xb) - exact) <= slack + 2e-4


def test_gamma_rule_moments():
    # full 2^L space: mean 0 and variance sum over bonds of J^2 (1/8 + Delta^2/16) + sum h^2 / 4
    for L, J2, periodic in [(8, 0.0, True), (8, 1.0, True), (8, 0.7, False)]:
        h = pi.fields(L, 2.5, config=9, realization=L)
        Hf = O.full_space_hamiltonian(L, 1.0, J2, 0.55, h, periodic)
        d = Hf.shape[0]
        nb1 = L if periodic else L - 1
        nb2 = L if periodic else L - 2
        var = (nb1 + nb2 * J2 ** 2) * (1 / 8 + 0.55 ** 2 / 16) + np.sum(h * h) / 4
        assert np.trace(Hf) / d == pytest.approx(0.0, abs=1e-12)
        assert np.trace(Hf @ Hf) / d == pytest.approx(var, rel=1e-12)
        # sector mean: the centre the rule uses
        H, _ = O.dense_hamiltonian(L, 1.0, J2, 0.55, h, periodic)
        n = H.shape[0]
        mean = -0.55 * (nb1 + nb2 * J2) / (4 * (L - 1))
        assert np.trace(H) / n == pytest.approx(mean, abs=1e-12)
        # gamma_rho is the Gaussian with that centre and width, at its peak
        peak = KO.gamma_rho(mean, L, 1.0, J2, 0.55, h, periodic, n)
        assert peak == pytest.approx(n / math.sqrt(2 * math.pi * var), rel=1e-12)


# ----------------------------------------------------------------------- MLP

def _scaling(d_in, d_out, rng):
    return (rng.normal(size=d_in), rng.uniform(0.5, 2.0, d_in), rng.normal(size=d_out), rng.uniform(0.5, 2.0, d_out))


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    d_in, H, d_out, B = 5, 7, 3, 4
    p = MO.glorot_params(d_in, H, d_out, rng)
    p[H * d_in:H * d_in + H] = rng.normal(size=H) * 0.3  # non-zero b1
    sc = _scaling(d_in, d_out, rng)
    x = rng.normal(size=(B, d_in))
    t = rng.normal(size=(B, d_out))
    _, g = MO.loss_and_grad(p, x, t, d_in, H, d_out, sc)
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = 1e-6
        fd[k] = (MO.loss_and_grad(p + e, x, t, d_in, H, d_out, sc)[0]
                 - MO.loss_and_grad(p - e, x, t, d_in, H, d_out, sc)[0]) / 2e-6
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_mlp_zero_weights_special_case():
    d_in, H, d_out, B = 4, 6, 3, 5
    rng = np.random.default_rng(4)
    p = np.zeros(MO.n_params(d_in, H, d_out))
    b3 = np.array([0.5, -1.0, 2.0])
    p[-3:] = b3
    x = rng.normal(size=(B, d_in))
    t = rng.normal(size=(B, d_out))
    y, _ = MO.forward(p, x, d_in, H, d_out)
    assert np.array_equal(y, np.tile(b3, (B, 1)))
    loss, g = MO.loss_and_grad(p, x, t, d_in, H, d_out)
    assert loss == pytest.approx(0.5 * np.sum((b3 - t) ** 2) / B, rel=1e-14)
    w = MO.unpack(g, d_in, H, d_out)
    assert np.allclose(w["b3"], np.mean(b3 - t, axis=0), atol=1e-15)
    for k in ("W1", "b1", "W2", "b2", "W3"):
        assert np.all(w[k] == 0.0), k


def test_adam_first_step_and_convergence():
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = MO.adam_step(p0, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    # bias-corrected first step: m^ = g, v^ = g^2  ->  step = lr g / (|g| + eps)
    assert np.allclose(p1 - p0, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    target = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 3001):
        p, m, v = MO.adam_step(p, p - target, m, v, t, 1e-2)
    assert np.max(np.abs(p - target)) < 1e-3


def test_mlp_training_with_oracle_adam_fits_a_smooth_function():
    rng = np.random.default_rng(6)
    d_in, H, d_out = 3, 16, 1
    X = rng.uniform(-1, 1, size=(256, d_in))
    Y = (np.sum(X * X, axis=1) - 1.0)[:, None]
    p = MO.glorot_params(d_in, H, d_out, rng)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = MO.loss_and_grad(p, X, Y, d_in, H, d_out)[0]
    for t in range(1, 1501):
        loss, g = MO.loss_and_grad(p, X, Y, d_in, H, d_out)
        p, m, v = MO.adam_step(p, g, m, v, t, 1e-2)
    assert loss < l0 / 50
