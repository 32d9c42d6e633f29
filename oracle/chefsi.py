"""Chebyshev-filtered subspace iteration on one subdomain (Sec. 5.A.3, steps (1)-(4)).

A block has one vector per row: Psi has shape (N_s, N_d).  In the paper's column
notation Psi is N_d x N_s; M_s = Psi^T Psi becomes Psi @ Psi.T here.

Readings (the paper names the method, Zhou et al. 2006, but gives no bounds or scaling):
  * filter: the scaled three-term recurrence that yields C_m((H-c)/e) / C_m((a0-c)/e) applied
    to Psi, with e = (b-a)/2, c = (b+a)/2; a scalar multiple of the paper's p_m(H), which the
    generalised eigenproblem of step (3) does not see;
  * bounds: b = Lanczos upper bound (k steps from a given random start vector, largest Ritz
    value plus the final residual norm); a = largest and a0 = smallest Ritz value of the
    previous pass, and of the unfiltered start block for the first pass;
  * projection: H_s symmetrised, (H_s + H_s^T)/2;
  * eigensolve: Cholesky M_s = L L^T, A = L^-1 H_s L^-T, A = Z diag(lambda) Z^T ascending,
    Y = L^-T Z; each column of Z signed so that its largest-magnitude entry is positive.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def lanczos_upper_bound(H, v0: np.ndarray, k: int = 10) -> float:
    """Upper bound of the spectrum of H: max eig of the k-step Lanczos matrix T_k started
    from v0, plus the norm of the final residual f_k."""
    v = np.asarray(v0, dtype=np.float64).reshape(1, H.N)
    v = v / np.linalg.norm(v)
    alpha = np.zeros(k)
    beta = np.zeros(k)
    f = H.apply(v)
    alpha[0] = float(np.sum(v * f))
    f = f - alpha[0] * v
    steps = 1
    for j in range(1, k):
        beta[j] = float(np.linalg.norm(f))
        v_prev, v = v, f / beta[j]
        f = H.apply(v) - beta[j] * v_prev
        alpha[j] = float(np.sum(v * f))
        f = f - alpha[j] * v
        steps += 1
    T = np.diag(alpha[:steps]) + np.diag(beta[1:steps], 1) + np.diag(beta[1:steps], -1)
    return float(np.linalg.eigvalsh(T)[-1] + np.linalg.norm(f))


def filter_coefficients(m: int, a: float, b: float, a0: float) -> list:
    """Per-step (scale, c, shift) of the scaled recurrence: Y_1 = scale_1 (H - c) Y_0 and
    Y_{k+1} = scale_{k+1} (H - c) Y_k - shift_{k+1} Y_{k-1}."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    sigma1 = e / (a0 - c)
    sigma = sigma1
    coef = [(sigma1 / e, c, 0.0)]
    for _ in range(2, m + 1):
        sigma2 = 1.0 / (2.0 / sigma1 - sigma)
        coef.append((2.0 * sigma2 / e, c, sigma * sigma2))
        sigma = sigma2
    return coef


def chebyshev_filter(H, X: np.ndarray, m: int, a: float, b: float, a0: float) -> np.ndarray:
    """Step (1): Psi_f = C_m((H - c)/e) X / C_m((a0 - c)/e) by the three-term recurrence."""
    coef = filter_coefficients(m, a, b, a0)
    scale, c, _ = coef[0]
    Y = scale * (H.apply(X) - c * X)
    for scale, c, shift in coef[1:]:
        Y_new = scale * (H.apply(Y) - c * Y) - shift * X
        X, Y = Y, Y_new
    return Y


def projection(H, Psi_f: np.ndarray):
    """Step (2): M_s = Psi_f^T Psi_f and H_s = Psi_f^T (H Psi_f), symmetrised."""
    HPsi = H.apply(Psi_f)
    Ms = Psi_f @ Psi_f.T
    Hs = Psi_f @ HPsi.T
    return Ms, 0.5 * (Hs + Hs.T)


def generalized_eig(Hs: np.ndarray, Ms: np.ndarray):
    """Step (3): H_s y = lambda M_s y via Cholesky reduction; returns (lambda ascending, Y)."""
    Lc = np.linalg.cholesky(Ms)
    W = sla.solve_triangular(Lc, Hs, lower=True)            # L^-1 H_s
    A = sla.solve_triangular(Lc, W.T, lower=True)           # L^-1 (L^-1 H_s)^T = L^-1 H_s L^-T
    A = 0.5 * (A + A.T)
    lam, Z = np.linalg.eigh(A)
    piv = np.argmax(np.abs(Z), axis=0)
    Z = Z * np.sign(Z[piv, np.arange(Z.shape[1])])
    Y = sla.solve_triangular(Lc.T, Z, lower=False)          # L^-T Z
    return lam, Y


def rotate(Psi_f: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Step (4): Psi = Psi_f Y (rows: Psi_new = Y^T Psi_f)."""
    return Y.T @ Psi_f


def ritz_values(H, Psi: np.ndarray) -> np.ndarray:
    """Ritz values of H on span(Psi) (used to bound the first pass)."""
    Ms, Hs = projection(H, Psi)
    return generalized_eig(Hs, Ms)[0]


def chefsi_pass(H, Psi: np.ndarray, m: int, a: float, b: float, a0: float):
    """One CheFSI iteration: filter, project, solve, rotate.  Returns (lambda, Psi)."""
    Psi_f = chebyshev_filter(H, Psi, m, a, b, a0)
    Ms, Hs = projection(H, Psi_f)
    lam, Y = generalized_eig(Hs, Ms)
    return lam, rotate(Psi_f, Y)


def run_chefsi(H, Psi0: np.ndarray, m: int, n_passes: int, b: float | None = None,
               lam_prev: np.ndarray | None = None, v0: np.ndarray | None = None):
    """n_passes CheFSI iterations from Psi0 with the bound rules above.  Returns (lambda, Psi, b).
    b defaults to the Lanczos bound from v0 (the caller's random start vector)."""
    if b is None:
        b = lanczos_upper_bound(H, v0)
    lam = ritz_values(H, Psi0) if lam_prev is None else lam_prev
    Psi = Psi0
    for _ in range(n_passes):
        lam, Psi = chefsi_pass(H, Psi, m, a=float(lam[-1]), b=b, a0=float(lam[0]))
    return lam, Psi, b
