"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: an
independent construction (Kronecker products on the full 2^L space), closed
forms (Dirichlet kernel, trace identity, infinite-temperature variance),
exactly solvable limits (free fermions, the 4-site Heisenberg ring), symmetry
invariants, brute force on tiny inputs, or values worked by hand.
"""
import math

import numpy as np
import pytest

import oracle as O
import polfed_inputs as I


def rnd_model(L, seed, periodic=True, J2=None, Delta=None):
    rng = np.random.default_rng(seed)
    J1 = 1.0 + 0.3 * rng.standard_normal()
    J2 = rng.uniform(0.2, 1.2) if J2 is None else J2
    Delta = rng.uniform(0.3, 1.5) if Delta is None else Delta
    h = rng.uniform(-2.5, 2.5, L)
    return J1, J2, Delta, h, periodic


# --------------------------------------------------------------------- basis

@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 14, 16])
def test_basis_dimension_and_order(L):
    st = O.basis(L)
    assert len(st) == math.comb(L, L // 2)
    assert np.all(np.diff(st) > 0)
    assert np.all(O.popcount(st) == L // 2)


def test_basis_matches_brute_force_enumeration():
    L = 10
    brute = sorted(s for s in range(1 << L) if bin(s).count("1") == L // 2)
    assert O.basis(L).tolist() == brute


def test_paper_full_ed_limit():
    # "full ED ... limited to N <~ 5*10^4 corresponding to L=18" (section "Calculation of eigenpairs")
    assert math.comb(18, 9) == 48620 < 5e4 < math.comb(20, 10)


@pytest.mark.parametrize("L", [8, 12])
def test_rank_combinatorial_number_system(L):
    st = O.basis(L)
    for idx, s in enumerate(st):
        assert O.rank_combinatorial(int(s)) == idx


# ------------------------------------------------------------ Hamiltonian Eq. (1)

@pytest.mark.parametrize("L", [4, 6, 8])
@pytest.mark.parametrize("periodic", [True, False])
def test_sector_equals_full_space_restriction(L, periodic):
    J1, J2, Delta, h, _ = rnd_model(L, 11 * L + periodic, periodic)
    Hs, st = O.dense_hamiltonian(L, J1, J2, Delta, h, periodic)
    Hf = O.full_space_hamiltonian(L, J1, J2, Delta, h, periodic)
    assert np.allclose(Hs, Hf[np.ix_(st, st)], atol=1e-13)
    # S^z conservation: no element couples the S^z = 0 sector to the rest
    rest = np.setdiff1d(np.arange(1 << L), st)
    assert np.max(np.abs(Hf[np.ix_(st, rest)])) < 1e-14


@pytest.mark.parametrize("L", [4, 6])
def test_all_sectors_reproduce_full_spectrum(L):
    J1, J2, Delta, h, _ = rnd_model(L, 5, True)
    full = np.linalg.eigvalsh(O.full_space_hamiltonian(L, J1, J2, Delta, h, True))
    parts = []
    for n_up in range(L + 1):
        H, _ = O.dense_hamiltonian(L, J1, J2, Delta, h, True, n_up=n_up)
        parts.append(np.linalg.eigvalsh(H))
    assert np.allclose(np.sort(np.concatenate(parts)), full, atol=1e-12)


def test_heisenberg_ring_L4_ground_state():
    H, _ = O.dense_hamiltonian(4, 1.0, 0.0, 1.0, np.zeros(4), True)
    assert abs(np.linalg.eigvalsh(H)[0] + 2.0) < 1e-13


@pytest.mark.parametrize("L", [6, 8, 10, 12, 14])
def test_trace_identity(L):
    # Tr_{S^z=0} H = -N Delta L (J1 + J2) / (4 (L - 1)) for periodic chains: the
    # field terms vanish by symmetry and a given pair is parallel with
    # probability (L-2)/(2(L-1)).
    J1, J2, Delta, h, _ = rnd_model(L, L, True)
    st = O.basis(L)
    d = O.diagonal(L, J1, J2, Delta, h, True, st)
    want = -len(st) * Delta * L * (J1 + J2) / (4.0 * (L - 1))
    assert abs(d.sum() - want) < 1e-9 * max(1.0, abs(want))


@pytest.mark.parametrize("L", [6, 8, 10])
def test_infinite_temperature_variance_matches_gamma(L):
    # Var(H) over the full space = L[(J1^2+J2^2)/8 + Delta^2 (J1^2+J2^2)/16] + sum h^2/4,
    # which is Gamma^2 of the Supplement when J1 = 1 and sum h^2/4 -> L W^2/12.
    J1, J2, Delta, h, _ = rnd_model(L, 3 * L, True)
    J1 = 1.0
    Hf = O.full_space_hamiltonian(L, J1, J2, Delta, h, True)
    n = Hf.shape[0]
    var = np.trace(Hf @ Hf) / n - (np.trace(Hf) / n) ** 2
    want = L * ((J1 ** 2 + J2 ** 2) / 8 + Delta ** 2 * (J1 ** 2 + J2 ** 2) / 16) + np.sum(h ** 2) / 4
    assert abs(var - want) < 1e-10 * want
    W = 2.0
    hh = np.full(L, W / math.sqrt(3.0))  # h^2 = W^2/3 = E[h^2] for U[-W, W]
    assert abs(O.gamma_paper(L, J2, Delta, W) ** 2 - (want - np.sum(h ** 2) / 4 + np.sum(hh ** 2) / 4)) < 1e-10


@pytest.mark.parametrize("L", [4, 6, 8, 10])
@pytest.mark.parametrize("periodic", [True, False])
def test_free_fermions(L, periodic):
    h = np.random.default_rng(L + 17 * periodic).uniform(-3, 3, L)
    H, _ = O.dense_hamiltonian(L, 1.0, 0.0, 0.0, h, periodic)
    ed = np.linalg.eigvalsh(H)
    ff = O.free_fermion_energies(L, 1.0, h, periodic)
    assert np.allclose(ed, ff, atol=1e-12)


def test_spectrum_symmetries():
    L = 10
    J1, J2, Delta, h, _ = rnd_model(L, 99, True)
    base = np.linalg.eigvalsh(O.dense_hamiltonian(L, J1, J2, Delta, h, True)[0])
    for hh in (np.roll(h, 3), h[::-1], -h):
        other = np.linalg.eigvalsh(O.dense_hamiltonian(L, J1, J2, Delta, hh, True)[0])
        assert np.allclose(base, other, atol=1e-11)


def test_sparse_and_rowwise_apply_match_dense():
    L = 10
    J1, J2, Delta, h, per = rnd_model(L, 4, False)
    H, st = O.dense_hamiltonian(L, J1, J2, Delta, h, per)
    Hs, st2 = O.sparse_hamiltonian(L, J1, J2, Delta, h, per)
    assert np.array_equal(st, st2)
    assert np.allclose(Hs.toarray(), H, atol=1e-14)
    X = I.block(len(st), 3, 1)
    rows = I.sample_rows(len(st), 20, 2)
    lo, hi = -7.0, 9.0
    want = (O.rescale_matrix(H, lo, hi) @ X)[rows]
    got = O.h_apply_rows(L, J1, J2, Delta, h, per, st, X, rows, lo, hi)
    assert np.allclose(got, want, atol=1e-13)
    assert np.allclose(O.h_apply_rows(L, J1, J2, Delta, h, per, st, X, rows), (H @ X)[rows], atol=1e-13)


# ------------------------------------------------------------ Eq. (2) filter

@pytest.mark.parametrize("K", [2, 10, 22, 100])
def test_dirichlet_closed_form_at_center(K):
    # At sigma = 0 with K even, (1/D) sum c_n T_n(sin u) = sin((K+1)u) / ((K+1) sin u).
    u = np.linspace(-1.5, 1.5, 301)
    u = u[np.abs(u) > 1e-6]
    got = O.P_scalar(np.sin(u), 0.0, K)
    want = np.sin((K + 1) * u) / ((K + 1) * np.sin(u))
    assert np.allclose(got, want, atol=1e-12)
    c, D = O.cheb_coeffs(0.0, K)
    assert abs(D - (1 + 2 * (K // 2))) < 1e-12
    assert np.allclose(c[1::2], 0.0, atol=1e-14 * K)  # cos(n pi / 2) in floating point


@pytest.mark.parametrize("sigma", [-0.6, -0.1, 0.3, 0.85])
@pytest.mark.parametrize("K", [7, 40])
def test_general_sigma_closed_form(sigma, K):
    # sum_{n=0}^K c_n T_n(cos t) with c_0 = 1, c_n = 2 cos(n phi), phi = arccos(sigma):
    # = 1 + sum_{n>=1} [cos n(t-phi) + cos n(t+phi)] = Dk(t-phi) + Dk(t+phi) - 1,
    # Dk(a) = sin((K+1/2)a) / (2 sin(a/2)) + 1/2 (Lagrange's trigonometric identity).
    phi = math.acos(sigma)
    t = np.linspace(0.01, math.pi - 0.01, 157)
    t = t[np.abs(t - phi) > 1e-4]

    def Dk(a):
        return np.sin((K + 0.5) * a) / (2 * np.sin(a / 2)) + 0.5

    S = Dk(t - phi) + Dk(t + phi) - 1.0
    c, D = O.cheb_coeffs(sigma, K)
    assert np.allclose(O.P_scalar(np.cos(t), sigma, K) * D, S, atol=1e-10)
    assert abs(O.P_scalar(np.array([sigma]), sigma, K)[0] - 1.0) < 1e-13
    # normalization: D = S(t = phi) = Dk(0) + Dk(2 phi) - 1 = K + Dk(2 phi)
    assert abs(D - (K + Dk(np.array([2 * phi]))[0])) < 1e-9


def test_filter_spectral_equals_matrix_recurrence():
    L = 8
    J1, J2, Delta, h, _ = rnd_model(L, 21, True)
    H, st = O.dense_hamiltonian(L, J1, J2, Delta, h, True)
    w, V = np.linalg.eigh(H)
    lo, hi = w[0] - 0.1, w[-1] + 0.2
    Ht = O.rescale_matrix(H, lo, hi)
    lt = (2 * w - lo - hi) / (hi - lo)
    X = I.block(len(st), 4, 3)
    for sigma, K in ((0.0, 16), (0.27, 31)):
        c, D = O.cheb_coeffs(sigma, K)
        a = O.filter_spectral(lt, V, X, sigma, K, c, D)
        b = O.filter_matrix_powers(Ht, X, c, D)
        assert np.allclose(a, b, atol=1e-11)
        # an eigenvector is mapped to P(lambda~) times itself
        v = V[:, [5]]
        pv = O.filter_spectral(lt, V, v, sigma, K, c, D)
        assert np.allclose(pv, O.P_scalar(lt[5:6], sigma, K) * v, atol=1e-12)


@pytest.mark.parametrize("K", [22, 100, 1000])
def test_lobe_halfwidth_closed_form(K):
    # Dirichlet kernel: P(sin u) = sin((K+1)u)/((K+1) sin u) >= p for |u| <= u*, the
    # first root; for large K, (K+1) u* -> y*, the root of sin(y)/y = p.
    from scipy.optimize import brentq
    ustar = brentq(lambda u: math.sin((K + 1) * u) / ((K + 1) * math.sin(u)) - O.P_THRESHOLD,
                   1e-9, math.pi / (K + 1))
    xl, xr = O.lobe_halfwidth(0.0, K)
    assert abs(xr - math.sin(ustar)) < 1e-10
    assert abs(xl + xr) < 1e-10
    ystar = brentq(lambda y: math.sin(y) / y - O.P_THRESHOLD, 1.0, 3.0)
    assert abs(ystar - 2.6704) < 1e-3
    assert abs((K + 1) * ustar - ystar) < 3.0 / (K + 1)


def test_fig1_sidelobes_below_p():
    # Fig. 1(b) / Supplement: outside the main lobe P^{K=22}_0 stays below p; the
    # secondary extrema (about +0.13 and -0.22 at K = 22, tending to +0.128 and
    # -0.217 as K grows) come from the Dirichlet closed form.
    K = 22
    u = np.linspace(1e-4, math.pi / 2, 20001)
    P = O.P_scalar(np.sin(u), 0.0, K)
    closed = np.sin((K + 1) * u) / ((K + 1) * np.sin(u))
    first_zero = math.pi / (K + 1)
    side = P[u > first_zero]
    assert side.max() < O.P_THRESHOLD
    assert abs(side.max() - closed[u > first_zero].max()) < 1e-12
    assert abs(side.min() - closed[u > first_zero].min()) < 1e-12
    assert abs(side.max() - 0.1284) < 4e-3 and abs(side.min() + 0.2172) < 4e-3


# ------------------------------------------------------------ selection, observables

def test_select_nearest_by_hand():
    ev = np.array([-3.0, -1.0, 0.2, 0.5, 2.0, 4.0])
    V = np.eye(6)
    got, vec = O.select_nearest(ev, V, 0.4, 3)
    assert got.tolist() == [-1.0, 0.2, 0.5]
    assert np.array_equal(vec, V[:, [1, 2, 3]])
    assert O.target_energy(ev, 0.5) == 0.5
    assert O.target_energy(ev, 0.0) == -3.0


def test_gap_ratio_by_hand_and_poisson():
    assert abs(O.gap_ratio(np.array([0.0, 1.0, 3.0, 4.0])) - 0.5) < 1e-15
    assert abs(O.gap_ratio(np.array([0.0, 1.0, 4.0])) - 1.0 / 3.0) < 1e-15
    lv = np.sort(np.random.default_rng(1).uniform(0, 1, 200001))
    assert abs(O.gap_ratio(lv) - (2 * math.log(2) - 1)) < 5e-3


def test_entropy_product_and_dimer_states():
    L = 4
    st = O.basis(L)
    prod = np.zeros(len(st))
    prod[0] = 1.0  # |0011>, a product state
    assert abs(O.entanglement_entropy(prod, st, L)) < 1e-12
    # singlets on bonds (0,1) and (2,3): (|01>-|10>)/sqrt2 (x) (|01>-|10>)/sqrt2
    vec = np.zeros(len(st))
    for a, sa in ((0b01, 1), (0b10, -1)):
        for b, sb in ((0b01, 1), (0b10, -1)):
            s = a | (b << 2)
            vec[np.searchsorted(st, s)] += 0.5 * sa * sb
    # cuts x=0,2 keep both singlets whole (S=0); x=1,3 cut both (S = 2 ln 2)
    assert abs(O.entanglement_entropy_cut(vec, st, L, 0)) < 1e-12
    assert abs(O.entanglement_entropy_cut(vec, st, L, 1) - 2 * math.log(2)) < 1e-12
    assert abs(O.entanglement_entropy(vec, st, L) - math.log(2)) < 1e-12


def test_random_sector_state_near_s_rmt():
    L = 12
    st = O.basis(L)
    rng = np.random.default_rng(5)
    vals = []
    for _ in range(3):
        v = rng.standard_normal(len(st))
        v /= np.linalg.norm(v)
        vals.append(O.entanglement_entropy_cut(v, st, L, 0))
    assert abs(np.mean(vals) - O.s_rmt(L)) < 0.03


def test_eigs_nearest_small_chain():
    m = I.xxz(8, 2.0, 1, 0)
    r = O.eigs_nearest(m.L, m.J1, m.J2, m.Delta, m.h, True, 0.5, 6)
    H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, True)
    assert np.all(O.residual_norms(H, r["evals"], r["evecs"]) < 1e-12)
    d = np.abs(r["spectrum"] - r["target"])
    assert np.max(np.abs(r["evals"] - r["target"])) <= np.sort(d)[5] + 1e-15


def test_input_generator_is_deterministic():
    a = I.fields(22, 3.0, 4, 1)
    b = I.fields(22, 3.0, 4, 1)
    assert np.array_equal(a, b) and np.all(np.abs(a) <= 3.0)
    assert not np.array_equal(a, I.fields(22, 3.0, 4, 2))
    # splitmix64 reference values for seed 0 (published test vector of the generator)
    assert I.splitmix64_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ------------------------------------------------- order selection ("POLFED algorithm")

def test_sector_moments_match_the_spectrum():
    # traces give the spectrum's mean and variance without an eigen-solve
    m = I.j1j2(10, 3.0, 2, 0)
    H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, True)
    w = np.linalg.eigvalsh(H)
    mean, var = O.sector_moments(H)
    assert abs(mean - w.mean()) < 1e-12 and abs(var - w.var()) < 1e-11
    Hs, _ = O.sparse_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, True)
    ms, vs = O.sector_moments(Hs)
    assert abs(ms - mean) < 1e-12 and abs(vs - var) < 1e-11


def test_gaussian_rho_normalization():
    # a density of states integrates to the number of states
    x = np.linspace(-40.0, 40.0, 400001)
    r = np.array([O.gaussian_rho(1000, 1.5, 9.0, e) for e in x[::100]])
    assert abs(np.trapezoid(r, x[::100]) - 1000.0) < 1e-6


@pytest.mark.parametrize("rho_t,n_target", [(2.0e4, 60.0), (5.0e4, 120.0), (3.0e5, 600.0)])
def test_order_for_window_fills_the_main_lobe(rho_t, n_target):
    # the chosen even K holds n_target values in its lobe; K + 2 no longer does.
    # The lobe is measured by scanning P itself (lobe_halfwidth), not by the
    # Dirichlet closed form that order_for_window uses.
    K = O.order_for_window(rho_t, n_target)
    assert K % 2 == 0
    assert O.n_accessible(rho_t, 0.0, K) >= n_target * (1 - 1e-9)
    assert O.n_accessible(rho_t, 0.0, K + 2) < n_target
    # large-K limit: K + 1 -> 2 y* rho / n_target with sin(y*)/y* = p
    assert abs((K + 1) / (2 * 2.6704 * rho_t / n_target) - 1.0) < 2.0 / (K + 1) + 2e-4


def test_order_for_window_counts_a_real_window():
    # L = 14 XXZ ring, W = 3: with the Gaussian density of the exact moments,
    # the window of the chosen K holds about the requested number of eigenvalues
    m = I.xxz(14, 3.0, 1, 0)
    H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, True)
    w = np.linalg.eigvalsh(H)
    lo, hi = w[0], w[-1]
    mean, var = O.sector_moments(H)
    Es = 0.5 * (lo + hi)
    rho_t = O.gaussian_rho(len(w), mean, var, Es) * 0.5 * (hi - lo)
    K = O.order_for_window(rho_t, 60.0)
    lt = (2 * w - lo - hi) / (hi - lo)
    n_in = int(np.sum(O.P_scalar(lt, 0.0, K) >= O.P_THRESHOLD))
    assert 40 <= n_in <= 80, (K, n_in)


def test_extreme_eigenvalues_match_dense():
    m = I.j1j2(12, 4.0, 2, 1)
    Hs, _ = O.sparse_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, True)
    H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, True)
    w = np.linalg.eigvalsh(H)
    lo, hi = O.extreme_eigenvalues(Hs)
    assert abs(lo - w[0]) < 1e-9 and abs(hi - w[-1]) < 1e-9


def test_residual_norms_two_level_closed_form():
    # u = cos(t) v_i + sin(t) v_j with eigenvectors v_i, v_j: the Rayleigh value is
    # e = cos^2 l_i + sin^2 l_j and ||H u - e u|| = |sin t cos t| |l_i - l_j|
    m = I.xxz(8, 2.0, 1, 3)
    H, _ = O.dense_hamiltonian(m.L, m.J1, m.J2, m.Delta, m.h, True)
    w, V = np.linalg.eigh(H)
    i, j = 3, 17
    us, es, want = [], [], []
    for t in (0.0, 0.1, 0.7):
        us.append(math.cos(t) * V[:, i] + math.sin(t) * V[:, j])
        es.append(math.cos(t) ** 2 * w[i] + math.sin(t) ** 2 * w[j])
        want.append(abs(math.sin(t) * math.cos(t)) * abs(w[i] - w[j]))
    got = O.residual_norms(H, np.array(es), np.stack(us, axis=1))
    assert np.allclose(got, want, atol=1e-12)
