"""Pins of the oracle's SCF pieces: LDA (Slater + Perdew-Zunger 1981) against closed forms,
continuity and the potential as the derivative of the energy density; the ion self-energy
against numerical quadrature; the Kerker preconditioner against the real-space FD operator;
Pulay mixing against its exactness on linear fixed-point maps."""
import math

import numpy as np
import pytest

import synth
from oracle import fd, pseudo, scf


def rho_of_rs(rs):
    return 3.0 / (4.0 * math.pi * np.asarray(rs, dtype=np.float64) ** 3)


def test_slater_exchange_closed_form():
    """eps_x = -(3/(4 pi)) (9 pi / 4)^(1/3) / r_s for the uniform gas (the textbook form in r_s)."""
    rs = np.array([0.3, 0.9, 1.0, 2.0, 5.0, 12.0])
    eps, _ = scf.lda_pz81(rho_of_rs(rs))
    ec = np.where(rs >= 1.0, scf.PZ_GAMMA / (1.0 + scf.PZ_BETA1 * np.sqrt(rs) + scf.PZ_BETA2 * rs),
                  scf.PZ_A * np.log(rs) + scf.PZ_B + scf.PZ_C * rs * np.log(rs) + scf.PZ_D * rs)
    ex = eps - ec
    np.testing.assert_allclose(ex * rs, -(3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0), rtol=1e-13)
    # known value of the exchange constant, 0.458165...
    assert abs((3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0) - 0.4581652932831429) < 1e-15


def test_pz81_correlation_joins_at_rs_one():
    """The two branches of the Perdew-Zunger fit meet at r_s = 1 (value to 1e-4 Ha, the fit's
    own matching accuracy) and the potential has no jump larger than that either."""
    lo, hi = rho_of_rs(1.0 - 1e-9), rho_of_rs(1.0 + 1e-9)
    e_lo, v_lo = scf.lda_pz81(np.array([lo]))
    e_hi, v_hi = scf.lda_pz81(np.array([hi]))
    assert abs(e_lo[0] - e_hi[0]) < 1e-4
    assert abs(v_lo[0] - v_hi[0]) < 2e-3


@pytest.mark.parametrize("rs", [0.2, 0.6, 0.95, 1.05, 2.0, 4.0, 10.0])
def test_xc_potential_is_derivative_of_energy_density(rs):
    """v_xc = d(rho eps_xc)/d rho, by a central difference of the energy density."""
    rho = rho_of_rs(rs)
    d = rho * 1e-5
    e_p, _ = scf.lda_pz81(np.array([rho + d]))
    e_m, _ = scf.lda_pz81(np.array([rho - d]))
    _, v = scf.lda_pz81(np.array([rho]))
    fd_v = ((rho + d) * e_p[0] - (rho - d) * e_m[0]) / (2 * d)
    assert abs(fd_v - v[0]) < 1e-8 * max(1.0, abs(v[0]))


def test_xc_zero_density():
    eps, v = scf.lda_pz81(np.array([0.0, -1e-12]))
    assert np.all(eps == 0.0) and np.all(v == 0.0)


def test_self_energy_matches_quadrature():
    """1/2 int b V for b = -Z pi^-3/2 rc^-3 exp(-r^2/rc^2), V = -Z erf(r/rc)/r, by quadrature."""
    from scipy import integrate, special
    w = synth.workload(0)
    sp = w.species[0]
    Z, rc = sp.Zv, sp.rc_loc
    f = lambda r: (-Z * math.pi ** -1.5 * rc ** -3 * math.exp(-r * r / rc ** 2)) * (-Z * special.erf(r / rc) / r) * 4 * math.pi * r * r
    val, _ = integrate.quad(f, 0.0, 40.0 * rc, limit=200)
    assert abs(scf.self_energy(w) - 0.5 * val * len(w.pos)) < 1e-10 * abs(scf.self_energy(w))


def test_kerker_matches_real_space_operator():
    """(-Delta_h + kappa^2) P R = -Delta_h R with the real-space FD Laplacian."""
    rng = np.random.default_rng(5)
    n = (14, 16, 18)
    h = (0.41, 0.43, 0.45)
    R = rng.standard_normal((n[2], n[1], n[0]))
    PR = scf.kerker(R, h, 0.5)
    lhs = -fd.laplacian(PR, h, (True, True, True)) + 0.25 * PR
    rhs = -fd.laplacian(R, h, (True, True, True))
    np.testing.assert_allclose(lhs, rhs, atol=1e-10 * np.abs(rhs).max())
    assert abs(PR.mean()) < 1e-12


def test_pulay_exact_on_linear_map():
    """Anderson/Pulay extrapolation at every step (period 1, no preconditioner, beta 1) on a
    linear contraction g(x) = A x + c in n dimensions reaches the fixed point after n + 1 steps
    (its iterates are those of GMRES on (I - A) x = c)."""
    rng = np.random.default_rng(11)
    n = 8
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(rng.uniform(-0.5, 0.9, n)) @ Q.T
    c = rng.standard_normal(n)
    xs = np.linalg.solve(np.eye(n) - A, c)
    m = scf.Mixer(h=(1.0, 1.0, 1.0), shape=(2, 2, 2), beta=1.0, kappa=None, history=n, period=1)
    x = np.zeros(n)
    for _ in range(n + 1):
        x = m.step(x, A @ x + c)
    assert np.linalg.norm(x - xs) < 1e-9 * np.linalg.norm(xs)
    # plain linear mixing is far from it after the same number of steps
    y = np.zeros(n)
    for _ in range(n + 1):
        y = y + 1.0 * ((A @ y + c) - y)
    assert np.linalg.norm(y - xs) > 1e-3 * np.linalg.norm(xs)


def test_periodic_pulay_alternates_linear_and_extrapolated_steps():
    """With period 2 the odd steps are plain preconditioned linear mixing."""
    rng = np.random.default_rng(3)
    n = 8
    A = np.diag(rng.uniform(0.0, 0.8, n))
    c = rng.standard_normal(n)
    m = scf.Mixer(h=(1.0, 1.0, 1.0), shape=(2, 2, 2), beta=0.3, kappa=None, history=7, period=2)
    x0 = rng.standard_normal(n)
    x1 = m.step(x0, A @ x0 + c)          # k = 0: linear
    np.testing.assert_allclose(x1, x0 + 0.3 * (A @ x0 + c - x0), rtol=1e-14)
    x2 = m.step(x1, A @ x1 + c)          # k = 1: extrapolated
    assert np.linalg.norm(x2 - (x1 + 0.3 * (A @ x1 + c - x1))) > 1e-6
