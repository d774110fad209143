"""Plain, slow, FP64 CPU oracle for POLFED (Sierant, Lewenstein, Zakrzewski,
"Polynomially filtered exact diagonalization approach to many-body
localization", arXiv:2005.09534).

TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library imports or calls this
module; the two share no code.  Only the seeded input generator
(``polfed_inputs``) serves both.

What each function follows (paper's numbering):
  * ``basis``                 -- S^z = 0 sector, dim C(L, L/2) ("Benchmark models").
  * ``dense_hamiltonian``     -- Eq. (1), built literally bond by bond.
  * ``full_space_hamiltonian``-- Eq. (1) from Kronecker products of spin matrices
                                 on the whole 2^L space (independent construction).
  * ``rescale``               -- H~ = [2H - (E0+E1)]/(E1-E0) ("POLFED algorithm").
  * ``cheb_coeffs``/``P_scalar`` -- Eq. (2): c_n = sqrt(4-3 delta_{0n}) cos(n arccos sigma),
                                 T_n(x) = cos(n arccos x), D such that P(sigma) = 1.
  * ``filter_spectral``       -- P(H~) X = V diag(P(lambda~)) V^T X (definition of a
                                 matrix function; a different algorithm from Clenshaw).
  * ``gamma_paper``, ``sector_moments``, ``gaussian_rho``, ``lobe_halfwidth``,
    ``n_accessible``, ``order_for_window`` -- order selection from the density of
                                 states with p = 0.17 ("POLFED algorithm"; Suppl.
                                 "Convergence of POLFED").
  * ``extreme_eigenvalues``   -- E_min, E_max of a sparse H (the Lanczos bounds of the
                                 "POLFED algorithm" paragraph, by ARPACK).
  * ``eigs_nearest``          -- the result POLFED reaches: the N_ev eigenpairs nearest
                                 the target (the text after Eqs. (3)-(4)).
  * ``gap_ratio``             -- mean gap ratio r (section "Entanglement entropy and
                                 level statistics").
  * ``entanglement_entropy``  -- S_E averaged over cuts [x, x+L/2) (same section).
  * ``free_fermion_energies`` -- exact sector spectrum at Delta = 0, J2 = 0 (textbook
                                 Jordan-Wigner mapping; a check, not from the paper).

Conventions: site i (0-based) <-> bit i of the state; bit = 1 <-> spin up
(S^z = +1/2); basis in ascending integer order; the S^z = 0 sector has L/2 up
spins.  Energies are in units of J1.
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, Optional, Tuple

import numpy as np

P_THRESHOLD = 0.17  # accessible-eigenvalue threshold p (section "POLFED algorithm")


# ----------------------------------------------------------------------------
# Basis and ranking ("Benchmark models": S^z = 0 sector, N = C(L, L/2))
# ----------------------------------------------------------------------------

def popcount(a: np.ndarray) -> np.ndarray:
    """Number of set bits of each entry (plain loop over 64 bit positions)."""
    a = np.asarray(a, dtype=np.int64)
    c = np.zeros(a.shape, dtype=np.int64)
    for b in range(63):
        c += (a >> b) & 1
    return c


def basis(L: int, n_up: Optional[int] = None) -> np.ndarray:
    """All L-bit integers with ``n_up`` set bits (default L/2), ascending."""
    if n_up is None:
        n_up = L // 2
    states = np.arange(1 << L, dtype=np.int64)
    return states[popcount(states) == n_up]


def rank_lookup(states: np.ndarray, s) -> np.ndarray:
    """Rank of state(s) s = position in the ascending basis list."""
    idx = np.searchsorted(states, s)
    assert np.all(states[np.minimum(idx, len(states) - 1)] == s), "state not in basis"
    return idx


def rank_combinatorial(s: int) -> int:
    """Rank via the combinatorial number system: sum_k C(p_k, k+1) over the set
    bits p_0 < p_1 < ... of s (counts the same-popcount states below s)."""
    r, k = 0, 0
    for p in range(64):
        if (s >> p) & 1:
            r += math.comb(p, k + 1)
            k += 1
    return r


# ----------------------------------------------------------------------------
# Hamiltonian, Eq. (1)
# ----------------------------------------------------------------------------

def bonds(L: int, periodic: bool, J1: float, J2: float):
    """(i, j, J_l) for every term of the double sum in Eq. (1).

    The sum runs over l = 1, 2 and i = 1..L literally; with periodic boundaries
    j = (i + l) mod L, with open boundaries the terms with i + l > L are dropped.
    Terms with J_l = 0 are skipped.
    """
    out = []
    for l, J in ((1, J1), (2, J2)):
        if J == 0.0:
            continue
        for i in range(L):
            j = i + l
            if j >= L:
                if not periodic:
                    continue
                j -= L
            out.append((i, j, J))
    return out


def diagonal(L: int, J1: float, J2: float, Delta: float, h: np.ndarray,
             periodic: bool, states: np.ndarray) -> np.ndarray:
    """Diagonal of Eq. (1) in the S^z basis: sum J_l Delta S^z_i S^z_j + sum h_i S^z_i."""
    d = np.zeros(len(states))
    for i, j, J in bonds(L, periodic, J1, J2):
        zi = ((states >> i) & 1) - 0.5
        zj = ((states >> j) & 1) - 0.5
        d += J * Delta * zi * zj
    for i in range(L):
        d += h[i] * (((states >> i) & 1) - 0.5)
    return d


def dense_hamiltonian(L: int, J1: float, J2: float, Delta: float, h, periodic: bool = True,
                      n_up: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Dense sector matrix of Eq. (1) and its basis.

    S^x_i S^x_j + S^y_i S^y_j = (S^+_i S^-_j + S^-_i S^+_j)/2 flips an
    antiparallel pair with amplitude 1/2, so the off-diagonal element between
    s and s ^ (2^i | 2^j) is J_l / 2 (the paper's H_ij = 1/2 at J_l = 1).
    Returns (H, states).
    """
    h = np.asarray(h, dtype=np.float64)
    states = basis(L, n_up)
    n = len(states)
    H = np.zeros((n, n))
    H[np.arange(n), np.arange(n)] = diagonal(L, J1, J2, Delta, h, periodic, states)
    for i, j, J in bonds(L, periodic, J1, J2):
        bi = (states >> i) & 1
        bj = (states >> j) & 1
        rows = np.nonzero(bi != bj)[0]
        flipped = states[rows] ^ ((1 << i) | (1 << j))
        cols = rank_lookup(states, flipped)
        np.add.at(H, (cols, rows), 0.5 * J)
    return H, states


def sparse_hamiltonian(L: int, J1: float, J2: float, Delta: float, h, periodic: bool = True):
    """Same matrix as ``dense_hamiltonian`` in scipy CSR form (for L up to ~24)."""
    import scipy.sparse as sp
    h = np.asarray(h, dtype=np.float64)
    states = basis(L)
    n = len(states)
    rows_all = [np.arange(n)]
    cols_all = [np.arange(n)]
    vals_all = [diagonal(L, J1, J2, Delta, h, periodic, states)]
    for i, j, J in bonds(L, periodic, J1, J2):
        bi = (states >> i) & 1
        bj = (states >> j) & 1
        rows = np.nonzero(bi != bj)[0]
        cols = rank_lookup(states, states[rows] ^ ((1 << i) | (1 << j)))
        rows_all.append(cols)
        cols_all.append(rows)
        vals_all.append(np.full(len(rows), 0.5 * J))
    H = sp.coo_matrix((np.concatenate(vals_all), (np.concatenate(rows_all), np.concatenate(cols_all))),
                      shape=(n, n)).tocsr()
    H.sum_duplicates()
    return H, states


def h_apply_rows(L: int, J1: float, J2: float, Delta: float, h, periodic: bool,
                 states: np.ndarray, X: np.ndarray, rows, e_lo: float = 0.0, e_hi: float = 0.0):
    """Rows ``rows`` of H~ X (or H X when e_lo == e_hi == 0), one row at a time.

    For each sampled row r: (H X)[r] = d_r X[r] + sum over flippable pairs of
    (J_l/2) X[rank(s_r ^ mask)].  Then the rescaling of the "POLFED algorithm"
    paragraph is applied.
    """
    h = np.asarray(h, dtype=np.float64)
    bl = bonds(L, periodic, J1, J2)
    out = np.zeros((len(rows), X.shape[1]))
    for t, r in enumerate(rows):
        s = int(states[r])
        d = 0.0
        acc = np.zeros(X.shape[1])
        for i, j, J in bl:
            bi, bj = (s >> i) & 1, (s >> j) & 1
            d += J * Delta * (bi - 0.5) * (bj - 0.5)
            if bi != bj:
                c = int(rank_lookup(states, s ^ ((1 << i) | (1 << j))))
                acc += 0.5 * J * X[c]
        for i in range(L):
            d += h[i] * (((s >> i) & 1) - 0.5)
        hx = d * X[r] + acc
        if e_lo == e_hi == 0.0:
            out[t] = hx
        else:
            out[t] = (2.0 * hx - (e_lo + e_hi) * X[r]) / (e_hi - e_lo)
    return out


def full_space_hamiltonian(L: int, J1: float, J2: float, Delta: float, h, periodic: bool = True) -> np.ndarray:
    """Eq. (1) on the full 2^L space from Kronecker products of spin-1/2 matrices.

    Independent of the bit-flip construction above: each operator is the
    tensor product with S^a on site i and identities elsewhere; site i is the
    factor whose index bit is bit i (so the ordering matches the bit convention).
    """
    sx = np.array([[0.0, 0.5], [0.5, 0.0]])
    sy = np.array([[0.0, -0.5j], [0.5j, 0.0]])
    # basis order |0> = down (bit 0), |1> = up (bit 1)
    sz = np.array([[-0.5, 0.0], [0.0, 0.5]])
    eye = np.eye(2)

    def site_op(op, i):
        # kron ordering: the last factor is the least significant bit (site 0)
        m = np.array([[1.0 + 0j]])
        for k in reversed(range(L)):
            m = np.kron(m, op if k == i else eye)
        return m

    dim = 1 << L
    H = np.zeros((dim, dim), dtype=complex)
    S = {(a, i): site_op(op, i) for a, op in (("x", sx), ("y", sy), ("z", sz)) for i in range(L)}
    for l, J in ((1, J1), (2, J2)):
        for i in range(L):
            j = i + l
            if j >= L:
                if not periodic:
                    continue
                j -= L
            H += J * (S[("x", i)] @ S[("x", j)] + S[("y", i)] @ S[("y", j)] + Delta * S[("z", i)] @ S[("z", j)])
    for i in range(L):
        H += h[i] * S[("z", i)]
    assert np.max(np.abs(H.imag)) < 1e-12
    return H.real


# ----------------------------------------------------------------------------
# Rescaling and the polynomial spectral transformation, Eq. (2)
# ----------------------------------------------------------------------------

def rescale_matrix(H: np.ndarray, e_lo: float, e_hi: float) -> np.ndarray:
    """H~ = [2H - (E0 + E1)] / (E1 - E0) with E0 = e_lo, E1 = e_hi."""
    n = H.shape[0]
    return (2.0 * H - (e_lo + e_hi) * np.eye(n)) / (e_hi - e_lo)


def cheb_T(n: int, x):
    """Chebyshev polynomial of the first kind, T_n(x) = cos(n arccos x) for |x| <= 1,
    cosh(n arccosh |x|) * sign^n outside."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(n * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** n * np.cosh(n * np.arccosh(np.abs(xo)))
    return out


def cheb_coeffs(sigma: float, K: int) -> Tuple[np.ndarray, float]:
    """Eq. (2): c_n = sqrt(4 - 3 delta_{0n}) cos(n arccos sigma), n = 0..K, and the
    normalization D = sum_n c_n T_n(sigma) that makes P(sigma) = 1."""
    n = np.arange(K + 1)
    c = np.sqrt(4.0 - 3.0 * (n == 0)) * np.cos(n * np.arccos(sigma))
    D = float(sum(c[k] * cheb_T(k, np.array([sigma]))[0] for k in range(K + 1)))
    return c, D


def P_scalar(x, sigma: float, K: int, coeffs: Optional[np.ndarray] = None, D: Optional[float] = None):
    """P^K_sigma(x) = (1/D) sum_{n=0}^K c_n T_n(x), summed term by term."""
    if coeffs is None:
        coeffs, D = cheb_coeffs(sigma, K)
    x = np.asarray(x, dtype=np.float64)
    s = np.zeros_like(x)
    for k in range(len(coeffs)):
        s += coeffs[k] * cheb_T(k, x)
    return s / D


def filter_spectral(evals_t: np.ndarray, evecs: np.ndarray, X: np.ndarray, sigma: float, K: int,
                    coeffs: Optional[np.ndarray] = None, D: Optional[float] = None) -> np.ndarray:
    """P(H~) X = V diag(P(lambda~)) V^T X from the eigendecomposition of H~."""
    p = P_scalar(evals_t, sigma, K, coeffs, D)
    return evecs @ (p[:, None] * (evecs.T @ X))


def filter_matrix_powers(Ht: np.ndarray, X: np.ndarray, coeffs: np.ndarray, D: float) -> np.ndarray:
    """(1/D) sum c_n T_n(H~) X with T_n(H~)X built by the matrix three-term
    recurrence T_{n+1} = 2 H~ T_n - T_{n-1} (the identity quoted in the
    Supplement, "Technical details").  A second, independent route to the
    filter for small matrices."""
    t_prev = X.copy()
    acc = coeffs[0] * t_prev
    if len(coeffs) == 1:
        return acc / D
    t = Ht @ X
    acc = acc + coeffs[1] * t
    for n in range(2, len(coeffs)):
        t_next = 2.0 * (Ht @ t) - t_prev
        t_prev, t = t, t_next
        acc = acc + coeffs[n] * t
    return acc / D


# ----------------------------------------------------------------------------
# Order K from the density of states (section "POLFED algorithm",
# Supplement "Convergence of POLFED")
# ----------------------------------------------------------------------------

def gamma_paper(L: int, J2: float, Delta: float, W: float) -> float:
    """Gamma = sqrt(L [(1+J2^2)/8 + Delta^2 (1+J2^2)/16 + W^2/12]) (Supplement, J1 = 1)."""
    return math.sqrt(L * ((1.0 + J2 ** 2) / 8.0 + Delta ** 2 * (1.0 + J2 ** 2) / 16.0 + W ** 2 / 12.0))


def lobe_halfwidth(sigma: float, K: int, p: float = P_THRESHOLD, coeffs=None, D=None) -> Tuple[float, float]:
    """Interval [x_L, x_R] around sigma on which P^K_sigma(x) >= p (main lobe),
    found by scanning P on a fine grid and bisecting the two crossings."""
    if coeffs is None:
        coeffs, D = cheb_coeffs(sigma, K)

    def f(x):
        return float(P_scalar(np.array([x]), sigma, K, coeffs, D)[0]) - p

    step = 0.25 / (K + 1)
    ends = []
    for direction in (-1.0, 1.0):
        a = sigma
        b = sigma + direction * step
        while abs(b) <= 1.0 and f(b) > 0:
            a, b = b, b + direction * step
        b = max(-1.0, min(1.0, b))
        for _ in range(80):
            m = 0.5 * (a + b)
            if f(m) > 0:
                a = m
            else:
                b = m
        ends.append(0.5 * (a + b))
    return ends[0], ends[1]


def n_accessible(rho_t: float, sigma: float, K: int, p: float = P_THRESHOLD) -> float:
    """Expected number of eigenvalues of H~ with P^K_sigma >= p for a locally flat
    density of states rho~ (eigenvalues per unit of the rescaled axis)."""
    xl, xr = lobe_halfwidth(sigma, K, p)
    return rho_t * (xr - xl)


def sector_moments(H) -> Tuple[float, float]:
    """Mean and variance of the spectrum of the sector matrix from traces:
    Tr H / N and Tr H^2 / N - mean^2 (H dense or scipy sparse; no eigen-solve)."""
    n = H.shape[0]
    if hasattr(H, "multiply"):
        t1 = float(H.diagonal().sum())
        t2 = float(H.multiply(H).sum())
    else:
        t1 = float(np.trace(H))
        t2 = float(np.sum(H * H))
    mean = t1 / n
    return mean, t2 / n - mean * mean


def gaussian_rho(n_states: int, mean: float, var: float, E: float) -> float:
    """Gaussian density of states per unit of energy at E with the spectrum's
    mean and variance (the Supplement's estimate of the density, with the
    width taken from the exact moments)."""
    g = math.sqrt(var)
    return n_states / (math.sqrt(2.0 * math.pi) * g) * math.exp(-0.5 * (E - mean) ** 2 / var)


def dirichlet_halfwidth(K: int, p: float = P_THRESHOLD) -> float:
    """At sigma = 0 and even K, P(sin u) = sin((K+1)u) / ((K+1) sin u): the main
    lobe P >= p is |x| <= sin(u*) with u* the first root of that ratio = p."""
    a, b = 1e-12, math.pi / (K + 1)
    for _ in range(200):
        m = 0.5 * (a + b)
        if math.sin((K + 1) * m) / ((K + 1) * math.sin(m)) > p:
            a = m
        else:
            b = m
    return math.sin(0.5 * (a + b))


def order_for_window(rho_t: float, n_target: float, p: float = P_THRESHOLD) -> int:
    """Order K of the transform at sigma = 0 ("POLFED algorithm": K is chosen so
    that about n_target eigenvalues have P >= p): the largest even K whose main
    lobe holds at least n_target eigenvalues of a locally flat density rho_t
    (eigenvalues per unit of the rescaled axis), lobe from ``dirichlet_halfwidth``."""
    def holds(K):
        return 2.0 * dirichlet_halfwidth(K, p) * rho_t >= n_target
    if not holds(2):
        return 2
    lo, hi = 2, 4
    while holds(hi):
        lo, hi = hi, 2 * hi
    while hi - lo > 2:  # even K: holds(lo), not holds(hi)
        mid = (lo + hi) // 2
        mid -= mid % 2
        if holds(mid):
            lo = mid
        else:
            hi = mid
    return lo


def extreme_eigenvalues(H) -> Tuple[float, float]:
    """Lowest and highest eigenvalue of a sparse symmetric H (ARPACK Lanczos,
    scipy.sparse.linalg.eigsh), the spectral bounds E0, E1 of the "POLFED
    algorithm" paragraph."""
    from scipy.sparse.linalg import eigsh
    lo = eigsh(H, k=1, which="SA", return_eigenvectors=False, tol=1e-12)[0]
    hi = eigsh(H, k=1, which="LA", return_eigenvectors=False, tol=1e-12)[0]
    return float(lo), float(hi)


# ----------------------------------------------------------------------------
# Eigenpairs nearest a target: the result POLFED reaches (text after Eqs. (3)-(4))
# ----------------------------------------------------------------------------

def target_energy(evals: np.ndarray, eps: float) -> float:
    """E* = E_min + eps (E_max - E_min) for the rescaled energy eps in [0, 1]."""
    return float(evals.min() + eps * (evals.max() - evals.min()))


def select_nearest(evals: np.ndarray, evecs: Optional[np.ndarray], target: float, n_ev: int):
    """The n_ev eigenpairs whose eigenvalues are nearest ``target``, ascending."""
    order = np.argsort(np.abs(evals - target), kind="stable")[:n_ev]
    order = np.sort(order)
    return evals[order], (None if evecs is None else evecs[:, order])


def eigs_nearest(L, J1, J2, Delta, h, periodic, eps, n_ev):
    """Dense ED of the S^z = 0 block of Eq. (1) and selection of the n_ev
    eigenpairs nearest E* = E_min + eps (E_max - E_min).

    Returns dict with evals (ascending), evecs (columns), E_min, E_max, norm
    (max |E|), target and the full spectrum.
    """
    H, states = dense_hamiltonian(L, J1, J2, Delta, h, periodic)
    w, V = np.linalg.eigh(H)
    tgt = target_energy(w, eps)
    ev, vec = select_nearest(w, V, tgt, n_ev)
    return dict(evals=ev, evecs=vec, E_min=float(w[0]), E_max=float(w[-1]),
                norm=float(max(abs(w[0]), abs(w[-1]))), target=tgt, spectrum=w, states=states)


def residual_norms(H: np.ndarray, evals: np.ndarray, evecs: np.ndarray) -> np.ndarray:
    """||H u_i - e_i u_i|| per column (the residual check after Eqs. (3)-(4))."""
    R = H @ evecs - evecs * evals[None, :]
    return np.linalg.norm(R, axis=0)


# ----------------------------------------------------------------------------
# Free fermions (exact check at Delta = 0, J2 = 0; textbook, not from the paper)
# ----------------------------------------------------------------------------

def free_fermion_energies(L: int, J1: float, h, periodic: bool) -> np.ndarray:
    """All S^z = 0 energies of the XX chain with fields, ascending.

    Jordan-Wigner: S^z_i = n_i - 1/2, (S^+_i S^-_j + h.c.)/2 -> hopping J1/2.
    With N = L/2 fermions the periodic wrap-around hop carries (-1)^(N+1).
    Sector energies = sum over the occupied single-particle levels minus
    sum(h)/2, over all subsets of L/2 levels.
    """
    h = np.asarray(h, dtype=np.float64)
    T = np.diag(h.copy())
    for i in range(L - 1):
        T[i, i + 1] = T[i + 1, i] = 0.5 * J1
    if periodic:
        sgn = (-1.0) ** (L // 2 + 1)
        T[0, L - 1] += sgn * 0.5 * J1
        T[L - 1, 0] += sgn * 0.5 * J1
    eps = np.linalg.eigvalsh(T)
    occ = basis(L)
    bits = ((occ[:, None] >> np.arange(L)[None, :]) & 1).astype(np.float64)
    E = bits @ eps - 0.5 * h.sum()
    return np.sort(E)


# ----------------------------------------------------------------------------
# Observables (section "Entanglement entropy and level statistics")
# ----------------------------------------------------------------------------

def gap_ratio(evals_sorted: np.ndarray) -> float:
    """Mean of r_i = min(g_i, g_{i+1}) / max(g_i, g_{i+1}), g_i = E_{i+1} - E_i."""
    e = np.sort(np.asarray(evals_sorted, dtype=np.float64))
    g = np.diff(e)
    r = np.minimum(g[:-1], g[1:]) / np.maximum(g[:-1], g[1:])
    return float(np.mean(r))


def s_rmt(L: int) -> float:
    """S_RMT(L) = (L/2) ln 2 + (1/2 + ln(1/2))/2 - 1/2."""
    return (L / 2.0) * math.log(2.0) + (0.5 + math.log(0.5)) / 2.0 - 0.5


def entanglement_entropy_cut(vec: np.ndarray, states: np.ndarray, L: int, x: int) -> float:
    """S_E = -sum alpha^2 ln alpha^2 for the bipartition [x, x+L/2) | rest (sites mod L).

    The vector is embedded in the full 2^L space, the amplitude tensor is
    reshaped with subsystem A's sites as row index, and the Schmidt
    coefficients are its singular values.
    """
    half = L // 2
    A = [(x + k) % L for k in range(half)]
    B = [s for s in range(L) if s not in A]
    states = np.asarray(states, dtype=np.int64)
    a = np.zeros(len(states), dtype=np.int64)  # index of each state's configuration of A
    b = np.zeros(len(states), dtype=np.int64)  # and of B
    for k, site in enumerate(A):
        a |= ((states >> site) & 1) << k
    for k, site in enumerate(B):
        b |= ((states >> site) & 1) << k
    M = np.zeros((1 << half, 1 << (L - half)))
    np.add.at(M, (a, b), np.asarray(vec, dtype=np.float64))
    sv = np.linalg.svd(M, compute_uv=False)
    a2 = sv ** 2
    a2 = a2[a2 > 1e-300]
    return float(-np.sum(a2 * np.log(a2)))


def entanglement_entropy(vec: np.ndarray, states: np.ndarray, L: int) -> float:
    """S_E averaged over the L cut positions x = 0..L-1."""
    return float(np.mean([entanglement_entropy_cut(vec, states, L, x) for x in range(L)]))
