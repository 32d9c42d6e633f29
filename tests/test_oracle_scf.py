"""Pins of the oracle's SCF pieces: LDA (Slater + Perdew-Zunger 1981) against closed forms,
continuity and the potential as the derivative of the energy density; the ion self-energy
against numerical quadrature; the Kerker preconditioner against the real-space FD operator;
Pulay mixing against its exactness on linear fixed-point maps."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import fd, pseudo, scf


def rho_of_rs(rs):
    return 3.0 / (4.0 * math.pi * np.asarray(rs, dtype=np.float64) ** 3)


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lda_limits.txt")


def golden_limits():
    """name -> (value, kind, tolerance) from tests/golden/lda_limits.txt."""
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        name, rest = line.split(":")
        val, kind, tol = rest.split()
        out[name.strip()] = (float(val), kind, float(tol))
    return out


def check_golden(name, got):
    val, kind, tol = golden_limits()[name]
    bound = tol * abs(val) if kind == "rel" else tol
    assert abs(got - val) <= bound, f"{name}: {got} vs {val} (tolerance {bound})"


SLATER = (3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0)   # 0.458165...


def eps_c(rs):
    """Correlation energy per electron of the oracle's LDA: eps_xc minus the exchange closed form."""
    rs = np.asarray(rs, dtype=np.float64)
    eps, _ = scf.lda_pz81(rho_of_rs(rs))
    return eps + SLATER / rs


def test_slater_exchange_high_density_limit():
    """r_s eps_xc -> -(3/(4 pi)) (9 pi / 4)^(1/3) as r_s -> 0, where the logarithmic correlation
    energy is negligible against the 1/r_s exchange: pins the exchange without the correlation."""
    rs = np.array([1e-10, 1e-9, 1e-8])
    eps, _ = scf.lda_pz81(rho_of_rs(rs))
    np.testing.assert_allclose(eps * rs, -SLATER, rtol=1e-7)
    # known value of the exchange constant, 0.458165...
    assert abs(SLATER - 0.4581652932831429) < 1e-15


def test_pz81_high_density_expansion():
    """Slope of eps_c against ln r_s at r_s -> 0 is the exact (1 - ln 2)/pi^2; the constant term
    is Gell-Mann and Brueckner's (both from the oracle's function values, not its constants)."""
    r1, r2 = 1e-7, 1e-6
    e1, e2 = eps_c([r1, r2])
    slope = (e2 - e1) / (math.log(r2) - math.log(r1))
    check_golden("hd_log_coefficient", slope)
    assert abs(slope - (1.0 - math.log(2.0)) / math.pi ** 2) < 1e-3 * slope
    check_golden("hd_constant", e1 - slope * math.log(r1))


def test_pz81_correlation_joins_smoothly_at_rs_one():
    """The two branches of the Perdew-Zunger fit meet at r_s = 1 in value and in slope (C and D
    are defined by that), within the precision of the printed constants; a wrong C or D by 1e-3
    breaks one of the two."""
    e_lo, e_hi = eps_c([1.0 - 1e-12, 1.0 + 1e-12])
    check_golden("join_value", e_hi - e_lo)
    d = 1e-6
    lo = eps_c([1.0 - 2 * d, 1.0 - d])        # one-sided slopes inside each branch
    hi = eps_c([1.0 + d, 1.0 + 2 * d])
    check_golden("join_slope", (hi[1] - hi[0]) / d - (lo[1] - lo[0]) / d)
    # and the potential has no jump larger than the slope mismatch allows
    _, v_lo = scf.lda_pz81(np.array([rho_of_rs(1.0 - 1e-9)]))
    _, v_hi = scf.lda_pz81(np.array([rho_of_rs(1.0 + 1e-9)]))
    assert abs(v_lo[0] - v_hi[0]) < 1e-4


def test_pz81_low_density_wigner_limit():
    """r_s eps_c = L + C r_s^-1/2 + O(1/r_s) at r_s -> infinity, against the Wigner-crystal
    energy minus exchange."""
    r1, r2 = 1e8, 4e8
    y1, y2 = eps_c([r1, r2]) * np.array([r1, r2])
    C = (y1 - y2) / (r1 ** -0.5 - r2 ** -0.5)
    L = y1 - C * r1 ** -0.5
    check_golden("ld_inverse_rs", L)
    check_golden("ld_inverse_rs_three_halves", C)


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
    x3 = m.step(x2, A @ x2 + c)          # k = 2: linear again, with a history to extrapolate from
    np.testing.assert_allclose(x3, x2 + 0.3 * (A @ x2 + c - x2), rtol=1e-14)
    x4 = m.step(x3, A @ x3 + c)          # k = 3: extrapolated
    assert np.linalg.norm(x4 - (x3 + 0.3 * (A @ x3 + c - x3))) > 1e-6


def _si2_cell():
    """Two displaced Si atoms in a cubic 8.55 bohr cell (20^3 points, h = 0.4275 bohr), 10 states."""
    a = 8.55
    pos = np.array([[0.3, 0.2, 0.1], [2.1375 + 0.3, 2.1375 + 0.1, 2.1375 - 0.2]])
    return synth.Workload("si2_20cube", (a, a, a), (20, 20, 20), pos, np.zeros(2, int), [synth.SI],
                          core_lo=np.zeros((1, 3), int), core_n=np.full((1, 3), 20), buf=np.zeros((1, 3), int),
                          n_states=np.array([10]), degree=16, n_passes=1, psi_seed=1000)


def _converged_scf(w, n_electrons, tol=1e-10, max_steps=80):
    """(free energy, mu) of the oracle's SCF run to a density residual below tol."""
    from oracle import dc
    b = pseudo.pseudocharge(w)
    n_pts = int(np.prod(w.n))
    dV = float(np.prod(w.h))
    rho0 = (w.n_electrons / (n_pts * dV) - b) * (n_electrons / w.n_electrons)
    sub = dc.partition(w)[0]
    st = scf.start(w, rho0, [synth.psi0_block(w.psi_seed, sub.N, int(w.n_states[0]))])
    for k in range(max_steps):
        res, energy, mu, _ = scf.step(w, st, n_passes=2 if k == 0 else 1, n_electrons=n_electrons)
        if res < tol:
            return energy, mu
    raise AssertionError(f"SCF did not reach {tol} (last residual {res:.2e})")


@pytest.mark.slow
def test_scf_energy_derivative_is_chemical_potential():
    """Janak's theorem for the Mermin free energy: at self-consistency dF/dN = mu.  The SCF
    energy assembly (E_band + E_xc - sum v_xc rho + 1/2 sum (b - rho) phi - E_self - E_entropy)
    is pinned by F(N + d) - F(N - d) = integral of mu dN (Simpson's rule over three converged
    runs) on a cell with a partly filled level (7 electrons, 8 valence), where mu(N) is smooth.
    A flipped entropy or Hartree sign, or a dropped -sum v_xc rho term, moves the difference by
    more than 1e-3 Ha; the pin holds to 1e-8."""
    w = _si2_cell()
    N, d = 7.0, 0.1
    F_m, mu_m = _converged_scf(w, N - d)
    _, mu_0 = _converged_scf(w, N)
    F_p, mu_p = _converged_scf(w, N + d)
    assert abs((F_p - F_m) - d / 3.0 * (mu_m + 4.0 * mu_0 + mu_p)) < 1e-7
    assert abs(F_p - F_m) > 1e-3          # a non-trivial energy change
