"""Fermi level, density and energies from local eigenpairs (Sec. 5.A.4-5).

  g(lambda; mu, sigma) = 1 / (1 + exp((lambda - mu)/sigma))              (Eq. dm_global)
  N_e(mu) = 2 sum_alpha sum_n g(lambda_n^alpha) c_n^alpha                 (Sec. 5.A.5, chemical potential)
  rho(x) = sum_alpha p^alpha(x) 2 sum_n g_n |psi_n^alpha(x)|^2            (Eq. density)
  E_band = 2 sum sum g c lambda,  E_entropy = -2 kT sum sum c s(lambda),
  s = g log g + (1 - g) log(1 - g)                                       (Sec. 5.A.4)

Readings: vectors are Euclidean-normalised on the grid (sum_g psi^2 = 1), so the density
on a grid point is (2/dV) sum_n g_n psi_n(g)^2 and c_n = sum over core points of psi_n^2;
mu is found by bisection on [min lambda - 1, max lambda + 1] (the paper's own solver is a
histogram + Newton scheme; any bracketing root finder gives the same mu).
"""
from __future__ import annotations

import numpy as np


def fermi(x: np.ndarray) -> np.ndarray:
    """1/(1 + e^x), evaluated as e^-x/(1 + e^-x) for x > 0 so that nothing overflows."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x > 0
    ex = np.exp(-x[pos])
    out[pos] = ex / (1.0 + ex)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def entropy_s(g: np.ndarray) -> np.ndarray:
    """g log g + (1 - g) log(1 - g) with 0 log 0 = 0."""
    g = np.asarray(g, dtype=np.float64)
    a = np.where(g > 0, g * np.log(np.where(g > 0, g, 1.0)), 0.0)
    q = 1.0 - g
    b = np.where(q > 0, q * np.log(np.where(q > 0, q, 1.0)), 0.0)
    return a + b


def occupations(lam, mu: float, kT: float) -> np.ndarray:
    return fermi((np.asarray(lam, dtype=np.float64) - mu) / kT)


def electron_count(mu: float, lam, c, kT: float) -> float:
    return float(2.0 * np.sum(occupations(lam, mu, kT) * np.asarray(c)))


class NoBracket(ValueError):
    """N_e lies outside [N_e(min lambda - 1), N_e(max lambda + 1)]: no Fermi level exists."""


def fermi_level(lam, c, kT: float, n_electrons: float, tol: float = 1e-14, max_iter: int = 200) -> float:
    """mu with N_e(mu) = n_electrons by bisection until the bracket is narrower than tol."""
    lam = np.asarray(lam, dtype=np.float64).ravel()
    c = np.asarray(c, dtype=np.float64).ravel()
    lo, hi = float(lam.min()) - 1.0, float(lam.max()) + 1.0
    if not (electron_count(lo, lam, c, kT) <= n_electrons <= electron_count(hi, lam, c, kT)):
        raise NoBracket(f"N_e={n_electrons} outside [{electron_count(lo, lam, c, kT)}, "
                        f"{electron_count(hi, lam, c, kT)}]")
    for _ in range(max_iter):
        if hi - lo <= tol:
            break
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if electron_count(mid, lam, c, kT) < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def band_energy(lam, c, mu: float, kT: float) -> float:
    lam = np.asarray(lam, dtype=np.float64)
    return float(2.0 * np.sum(occupations(lam, mu, kT) * np.asarray(c) * lam))


def entropy_energy(lam, c, mu: float, kT: float) -> float:
    s = entropy_s(occupations(lam, mu, kT))
    return float(-2.0 * kT * np.sum(np.asarray(c) * s))


def point_density(Psi_rows: np.ndarray, g: np.ndarray, dV: float) -> np.ndarray:
    """(2/dV) sum_n g_n psi_n(x)^2 for the given rows of vectors (shape (N_s, n_points))."""
    return (2.0 / dV) * np.einsum("n,ng->g", g, Psi_rows * Psi_rows)


def dos(lam, c, energies: np.ndarray, width: float) -> np.ndarray:
    """Eq. dos with the delta function broadened to a normalised Gaussian of the given width."""
    lam = np.asarray(lam, dtype=np.float64).ravel()
    c = np.asarray(c, dtype=np.float64).ravel()
    d = energies[:, None] - lam[None, :]
    k = np.exp(-0.5 * (d / width) ** 2) / (width * np.sqrt(2.0 * np.pi))
    return 2.0 * k @ c
