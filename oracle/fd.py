"""12th-order central finite-difference Laplacian (Sec. 5.B.2: a 2*n0-order stencil with
n0 = 6, 3 * 2 * n0 = 36 neighbours plus the centre, fixed weights w_p).

The weights are the standard central-difference weights of the second derivative,
    w_p = 2 (-1)^(p+1) (n0!)^2 / (p^2 (n0-p)! (n0+p)!),   w_0 = -2 sum_p w_p,
so that f''(x_i) ~ (1/h^2) [w_0 f_i + sum_{p=1..n0} w_p (f_{i+p} + f_{i-p})].
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

N0 = 6


def fd_weights_exact(n0: int = N0) -> list:
    """[w_0, w_1, ..., w_n0] as exact fractions."""
    w = [Fraction(0)] * (n0 + 1)
    for p in range(1, n0 + 1):
        w[p] = Fraction(2 * (-1) ** (p + 1) * factorial(n0) ** 2,
                        p * p * factorial(n0 - p) * factorial(n0 + p))
    w[0] = -2 * sum(w[1:])
    return w


def fd_weights(n0: int = N0) -> np.ndarray:
    return np.array([float(x) for x in fd_weights_exact(n0)])


def _shift(f: np.ndarray, axis: int, p: int, periodic: bool) -> np.ndarray:
    """g[i] = f[i + p] along `axis`; outside the box: periodic wrap or zero (Dirichlet)."""
    if periodic:
        return np.roll(f, -p, axis=axis)
    g = np.zeros_like(f)
    n = f.shape[axis]
    src = [slice(None)] * f.ndim
    dst = [slice(None)] * f.ndim
    if p >= 0:
        src[axis] = slice(p, n)
        dst[axis] = slice(0, max(n - p, 0))
    else:
        src[axis] = slice(0, max(n + p, 0))
        dst[axis] = slice(-p, n)
    g[tuple(dst)] = f[tuple(src)]
    return g


def second_derivative(f: np.ndarray, axis: int, h: float, periodic: bool, n0: int = N0) -> np.ndarray:
    """(1/h^2)[w_0 f_i + sum_p w_p (f_{i+p} + f_{i-p})] along one axis."""
    w = fd_weights(n0)
    out = w[0] * f
    for p in range(1, n0 + 1):
        out = out + w[p] * (_shift(f, axis, p, periodic) + _shift(f, axis, -p, periodic))
    return out / (h * h)


def laplacian(f: np.ndarray, h, periodic, n0: int = N0) -> np.ndarray:
    """Delta_h f for f of shape (..., nz, ny, nx); h and periodic are (x, y, z) triples."""
    out = np.zeros_like(f)
    for d in range(3):                       # d = 0: x (last axis) ... d = 2: z
        out += second_derivative(f, f.ndim - 1 - d, h[d], bool(periodic[d]), n0)
    return out


def symbol_1d(theta: np.ndarray, h: float, n0: int = N0) -> np.ndarray:
    """Eigenvalue of -(d^2/dx^2)_h on the plane wave exp(i theta j): -(w_0 + 2 sum w_p cos p theta)/h^2."""
    w = fd_weights(n0)
    s = w[0] + sum(2.0 * w[p] * np.cos(p * theta) for p in range(1, n0 + 1))
    return -s / (h * h)
