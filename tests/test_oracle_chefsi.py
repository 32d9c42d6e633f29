"""Pins of the oracle's CheFSI pass, Fermi level, density and D&C assembly against closed
forms (Chebyshev polynomials, FD plane-wave spectrum), brute-force dense diagonalisation,
an independent root finder and invariants (trace of rho, orthonormality, D&C = undivided)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as sopt

import synth
from oracle import chefsi, dc, fd, fermi, pseudo
from oracle.operator import SubdomainHamiltonian


class Diagonal:
    """H = diag(d): the filter acts on each coordinate as the scalar polynomial."""

    def __init__(self, d):
        self.d = np.asarray(d, dtype=float)
        self.N = len(self.d)

    def apply(self, Y):
        return np.atleast_2d(Y) * self.d


def chebyshev_T(m, t):
    t = np.asarray(t, dtype=float)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1
    out[inside] = np.cos(m * np.arccos(t[inside]))
    s = np.sign(t[~inside])
    out[~inside] = np.cosh(m * np.arccosh(np.abs(t[~inside]))) * s ** m
    return out


@pytest.mark.parametrize("m", [1, 2, 7, 16, 24])
def test_filter_is_scaled_chebyshev_on_diagonal_operator(m):
    rng = np.random.default_rng(m)
    d = np.sort(rng.uniform(-1.0, 60.0, 200))
    a, b, a0 = 5.0, 60.5, -1.2
    X = rng.standard_normal((3, d.size))
    got = chefsi.chebyshev_filter(Diagonal(d), X, m, a, b, a0)
    e, c = (b - a) / 2, (b + a) / 2
    factor = chebyshev_T(m, (d - c) / e) / chebyshev_T(m, np.array([(a0 - c) / e]))[0]
    np.testing.assert_allclose(got, X * factor, rtol=1e-12, atol=1e-13)


def test_lanczos_bound_above_spectrum_and_tight():
    rng = np.random.default_rng(3)
    d = rng.uniform(-2.0, 40.0, 500)
    b = chefsi.lanczos_upper_bound(Diagonal(d), synth.lanczos_start(d.size))
    assert b >= d.max()
    assert b < d.max() + 0.5 * (d.max() - d.min())


def test_generalized_eig_matches_lapack_and_invariants():
    rng = np.random.default_rng(4)
    B = rng.standard_normal((30, 30))
    Ms = B @ B.T + 30 * np.eye(30)
    Hs = rng.standard_normal((30, 30))
    Hs = Hs + Hs.T
    lam, Y = chefsi.generalized_eig(Hs, Ms)
    np.testing.assert_allclose(lam, sla.eigh(Hs, Ms, eigvals_only=True), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(Y.T @ Ms @ Y, np.eye(30), atol=1e-11)
    np.testing.assert_allclose(Y.T @ Hs @ Y, np.diag(lam), atol=1e-10)
    assert np.all(np.diff(lam) >= 0)


def test_chefsi_converges_to_fd_laplacian_spectrum():
    """V = 0, no projectors, periodic grid: the lowest eigenvalues of -1/2 Delta_h are
    1/2 sum_axes s(2 pi j/n) (closed form), including their degeneracies."""
    n, h = 12, 0.45
    H = SubdomainHamiltonian((n, n, n), (h, h, h), (True,) * 3, np.zeros((n, n, n)), [])
    s = fd.symbol_1d(2 * math.pi * np.fft.fftfreq(n), h)
    exact = np.sort((0.5 * (s[:, None, None] + s[None, :, None] + s[None, None, :])).ravel())
    Psi0 = synth.psi0_block(7, H.N, 40)
    lam, Psi, b = chefsi.run_chefsi(H, Psi0, m=20, n_passes=25, v0=synth.lanczos_start(H.N))
    # 33 = 1 + 6 + 12 + 8 + ... lowest shells; compare the first 27 (complete shells 1+6+12+8)
    np.testing.assert_allclose(lam[:27], exact[:27], atol=1e-10)
    np.testing.assert_allclose(Psi @ Psi.T, np.eye(40), atol=1e-11)


def _small_si(periodic=True):
    """8-atom Si cell on a coarse 12^3 grid (h = 0.855): dense H fits in memory."""
    w = synth.workload(0)
    w.n = (12, 12, 12)
    norms = pseudo.projector_norms(w)
    V = pseudo.local_potential(w)
    if periodic:
        s = dc.partition(w)[0]
    else:
        s = dc.Subdomain(start=np.array([2, -3, 1]), size=np.array([10, 12, 9]), periodic=np.array([False, True, False]),
                         core_lo=np.array([0, 0, 0]), core_n=np.array([10, 12, 9]), core_global_lo=np.array([2, -3, 1]))
    return w, dc.subdomain_operator(w, s, V, norms)


@pytest.mark.parametrize("periodic", [True, False])
def test_chefsi_matches_dense_diagonalisation(periodic):
    w, H = _small_si(periodic)
    D = H.dense()
    exact = np.linalg.eigvalsh(D)
    Psi0 = synth.psi0_block(11, H.N, 28)
    lam, Psi, b = chefsi.run_chefsi(H, Psi0, m=16, n_passes=40, v0=synth.lanczos_start(H.N))
    assert b >= exact[-1]
    np.testing.assert_allclose(lam[:20], exact[:20], atol=1e-10)
    # residuals of the converged vectors
    R = H.apply(Psi[:20]) - lam[:20, None] * Psi[:20]
    assert np.abs(R).max() < 1e-6


def test_fermi_function_and_entropy():
    x = np.array([-800.0, -30.0, -1.0, 0.0, 0.5, 30.0, 800.0])
    g = fermi.fermi(x)
    assert np.all(np.isfinite(g))
    np.testing.assert_allclose(g[1:-1], 1.0 / (1.0 + np.exp(x[1:-1])), rtol=1e-14)
    np.testing.assert_allclose(fermi.fermi(-x), 1.0 - g, atol=1e-16)
    s = fermi.entropy_s(np.array([0.0, 1.0, 0.5, 0.25]))
    np.testing.assert_allclose(s, [0.0, 0.0, math.log(0.5), 0.25 * math.log(0.25) + 0.75 * math.log(0.75)])


def test_fermi_level_bisection_against_brent():
    rng = np.random.default_rng(9)
    lam = np.sort(rng.uniform(-0.5, 1.0, 300))
    c = rng.uniform(0.0, 1.0, 300)
    ne = 0.8 * 2 * c.sum()
    mu = fermi.fermi_level(lam, c, 0.01, ne)
    ref = sopt.brentq(lambda m: fermi.electron_count(m, lam, c, 0.01) - ne, -2, 2, xtol=1e-15, rtol=1e-15)
    assert abs(mu - ref) < 1e-12
    assert fermi.electron_count(mu, lam, c, 0.01) == pytest.approx(ne, rel=1e-12)
    with pytest.raises(fermi.NoBracket):
        fermi.fermi_level(lam, c, 0.01, 2 * c.sum() + 1.0)


def test_energies_definitions_on_two_levels():
    lam = np.array([0.0, 0.1])
    c = np.array([1.0, 0.5])
    mu, kT = 0.05, 0.02
    g = 1 / (1 + np.exp((lam - mu) / kT))
    assert fermi.band_energy(lam, c, mu, kT) == pytest.approx(2 * np.sum(g * c * lam), rel=1e-15)
    eS = fermi.entropy_energy(lam, c, mu, kT)
    assert eS > 0                                          # -2kT sum c s with s <= 0
    de = fermi.dos(lam, c, np.linspace(-1, 1, 20001), 0.01)
    assert np.trapezoid(de, dx=2 / 20000) == pytest.approx(2 * c.sum(), rel=1e-6)


@pytest.mark.slow
def test_config0_invariants():
    w = synth.workload(0)
    V = pseudo.local_potential(w)
    sub = dc.partition(w)[0]
    r = dc.run(w, V, [synth.psi0_block(w.psi_seed, sub.N, 24)])
    lam, Psi = r.lam[0], r.Psi[0]
    np.testing.assert_allclose(Psi @ Psi.T, np.eye(24), atol=1e-11)
    np.testing.assert_allclose(r.c[0], 1.0, atol=1e-12)      # core = whole cell
    assert r.rho.sum() * np.prod(w.h) == pytest.approx(32.0, rel=1e-12)
    assert np.all(r.rho >= 0)
    assert r.e_entropy >= 0
    assert np.all(np.diff(lam) >= 0)


@pytest.mark.slow
def test_dc_with_covering_buffer_equals_undivided():
    """Two subdomains whose buffers cover the (periodic) cell reproduce the undivided result.
    A small smearing keeps the unconverged top states of the block unoccupied."""
    w = synth.workload(0)
    w.n = (12, 12, 12)
    w2 = synth.Workload("pair", (2 * w.L[0], w.L[1], w.L[2]), (24, 12, 12),
                        np.concatenate([w.pos, w.pos + [w.L[0], 0, 0]]), np.zeros(16, int), [synth.SI],
                        core_lo=np.array([[0, 0, 0], [12, 0, 0]]), core_n=np.array([[12, 12, 12]] * 2),
                        buf=np.array([[6, 0, 0]] * 2), n_states=np.array([44, 44]), degree=20, n_passes=30,
                        psi_seed=5, kT=0.005)
    whole = synth.Workload("whole", w2.L, w2.n, w2.pos, w2.species_index, w2.species,
                           core_lo=np.zeros((1, 3), int), core_n=np.array([[24, 12, 12]]),
                           buf=np.zeros((1, 3), int), n_states=np.array([44]), degree=20, n_passes=30, psi_seed=6,
                           kT=0.005)
    V = pseudo.local_potential(w2)
    subs = dc.partition(w2)
    assert all(s.periodic.all() for s in subs)
    r2 = dc.run(w2, V, [synth.psi0_block(5, s.N, 44, k * 10 ** 6) for k, s in enumerate(subs)])
    r1 = dc.run(whole, V, [synth.psi0_block(6, 24 * 12 * 12, 44)])
    np.testing.assert_allclose(r2.lam[0][:36], r1.lam[0][:36], atol=1e-9)
    np.testing.assert_allclose(r2.lam[1][:36], r1.lam[0][:36], atol=1e-9)
    assert r2.mu == pytest.approx(r1.mu, abs=1e-9)
    # vectors converge as the square root of the Ritz values: rho agrees to ~1e-6 here
    assert np.linalg.norm(r2.rho - r1.rho) < 3e-6 * np.linalg.norm(r1.rho)
    assert r2.e_band == pytest.approx(r1.e_band, abs=1e-7)


def test_interior_weights_count_core_points_only():
    """c_n sums psi_n^2 over the core box alone (Sec. 5.A.4): with one unit vector per grid point
    (x fastest), the weights are 1 exactly on the points of the core box and 0 on the buffer."""
    s = dc.Subdomain(start=np.array([-2, -1, -3]), size=np.array([9, 8, 7]), periodic=np.zeros(3, bool),
                     core_lo=np.array([2, 1, 3]), core_n=np.array([4, 5, 2]), core_global_lo=np.zeros(3, int))
    c = dc.interior_weights(np.eye(s.N), s)
    want = np.zeros(s.N)
    for k in range(7):
        for j in range(8):
            for i in range(9):
                if 2 <= i < 6 and 1 <= j < 6 and 3 <= k < 5:
                    want[i + 9 * (j + 8 * k)] = 1.0
    np.testing.assert_array_equal(c, want)
    assert c.sum() == 4 * 5 * 2
