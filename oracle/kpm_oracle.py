"""Plain FP64 CPU oracle of the density-of-states estimates that set K.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the GPU
library imports or calls this module.

The paper fixes K from the density of states at the target ("POLFED
algorithm" section; the Supplement's Gaussian estimate of rho(0) with the
width Gamma) and names iterative estimators of it.  The estimator built here is
the kernel polynomial method of Weisse, Wellein, Alvermann and Fehske, Rev.
Mod. Phys. 78, 275 (2006) (section II):
  * ``moments_from_spectrum`` -- mu_n = (1/R) sum_r sum_i (v_i . r)^2 T_n(lambda_i):
                                 the stochastic moments written through the
                                 eigen-decomposition (a different algorithm from
                                 the GPU's three-term recurrence on vectors).
  * ``trace_moments``         -- mu_n = Tr T_n(H~) = sum_i T_n(lambda_i).
  * ``jackson``               -- damping factors g_n, their Eq. (71).
  * ``indicator_coeffs``      -- Chebyshev coefficients of the indicator of
                                 [x_a, x_b]: c_n = (2 - delta_{n0}) / pi times the
                                 integral of cos(n th) over [arccos x_b, arccos x_a].
  * ``count_fraction``        -- sum_n g_n c_n mu_n / mu_0, the damped fraction of
                                 the spectrum inside [x_a, x_b].
  * ``gaussian_rho`` / ``gamma_rho`` -- the Gaussian estimates the paper uses.
"""
from __future__ import annotations

import math

import numpy as np


def cheb_T_table(n_mom: int, x: np.ndarray) -> np.ndarray:
    """[n_mom, len(x)] table of T_n(x) = cos(n arccos x) for x in [-1, 1]."""
    x = np.clip(np.asarray(x, dtype=np.float64), -1.0, 1.0)
    th = np.arccos(x)
    return np.cos(np.outer(np.arange(n_mom), th))


def moments_from_spectrum(evals_t: np.ndarray, evecs: np.ndarray, R_block: np.ndarray, n_mom: int) -> np.ndarray:
    """mu_n = (1/R) sum_r r^T T_n(H~) r with H~ = V diag(evals_t) V^T and the R
    columns r of R_block (dim x R)."""
    w = (evecs.T @ np.asarray(R_block, dtype=np.float64)) ** 2  # [n_states, R]
    weights = w.sum(axis=1) / R_block.shape[1]
    return cheb_T_table(n_mom, evals_t) @ weights


def trace_moments(evals_t: np.ndarray, n_mom: int) -> np.ndarray:
    """mu_n = Tr T_n(H~) = sum_i T_n(lambda_i)."""
    return cheb_T_table(n_mom, evals_t).sum(axis=1)


def jackson(n_mom: int) -> np.ndarray:
    """g_n = [(N - n + 1) cos(pi n / (N + 1)) + sin(pi n / (N + 1)) cot(pi / (N + 1))] / (N + 1), N = n_mom."""
    N = n_mom
    n = np.arange(N)
    q = math.pi / (N + 1)
    return ((N - n + 1) * np.cos(q * n) + np.sin(q * n) / math.tan(q)) / (N + 1)


def indicator_coeffs(n_mom: int, x_a: float, x_b: float) -> np.ndarray:
    """c_n of chi_[x_a, x_b](x) = sum_n c_n T_n(x): with x = cos th,
    c_n = (2 - delta_{n0}) / pi * int_{th_b}^{th_a} cos(n th) d th."""
    ta, tb = math.acos(max(-1.0, min(1.0, x_a))), math.acos(max(-1.0, min(1.0, x_b)))
    c = np.empty(n_mom)
    c[0] = (ta - tb) / math.pi
    n = np.arange(1, n_mom)
    c[1:] = 2.0 / math.pi * (np.sin(n * ta) - np.sin(n * tb)) / n
    return c


def count_fraction(mu: np.ndarray, x_a: float, x_b: float) -> float:
    """Jackson-damped fraction of the spectrum in [x_a, x_b]."""
    mu = np.asarray(mu, dtype=np.float64)
    N = mu.size
    return float(np.sum(jackson(N) * indicator_coeffs(N, x_a, x_b) * mu) / mu[0])


def kpm_density(mu: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Jackson-damped density (per unit x, normalized to 1):
    rho(x) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(x)] / (pi sqrt(1 - x^2) mu_0)."""
    mu = np.asarray(mu, dtype=np.float64)
    N = mu.size
    g = jackson(N)
    coef = g * mu
    coef[1:] *= 2.0
    x = np.asarray(x, dtype=np.float64)
    return (coef @ cheb_T_table(N, x)) / (math.pi * np.sqrt(1.0 - x * x) * mu[0])


def gaussian_rho(E: float, mean: float, var: float, dim: int) -> float:
    """Gaussian density of states (states per unit energy) with the given moments."""
    return dim / math.sqrt(2.0 * math.pi * var) * math.exp(-0.5 * (E - mean) ** 2 / var)


def gamma_rho(E: float, L: int, J1: float, J2: float, Delta: float, h, periodic: bool, dim: int) -> float:
    """The paper's analytic estimate: Gamma^2 = L [(1+J2^2)/8 + Delta^2 (1+J2^2)/16 + W^2/12]
    (Supplement, J1 = 1), written per bond and per realization (nb_l terms of
    class l; sum h_i^2 / 4 for L W^2 / 12), centred at the S^z = 0 sector mean
    (<S^z_i S^z_j> = -1 / (4 (L - 1)) there for i != j)."""
    nb1 = L if periodic else L - 1
    nb2 = L if periodic else L - 2
    h = np.asarray(h, dtype=np.float64)
    var = (nb1 * J1 ** 2 + nb2 * J2 ** 2) * (1.0 / 8.0 + Delta ** 2 / 16.0) + float(np.sum(h * h)) / 4.0
    mean = -Delta * (nb1 * J1 + nb2 * J2) / (4.0 * (L - 1))
    return gaussian_rho(E, mean, var, dim)
