"""Local pseudopotential by pseudocharge electrostatics and Kleinman-Bylander projectors.

Electrostatics (Eq. poisson, Sec. 5.A.1): -(1/4 pi) lap(phi) = rho + b with the total
pseudocharge b = sum_I b_I, b_I = -(1/4 pi) lap(V_I).  For V_I(r) = -Z erf(r/r_c)/r the
pseudocharge is the normalised Gaussian b_I(r) = -Z pi^{-3/2} r_c^{-3} exp(-r^2/r_c^2).
Reading (the paper gives V only through Eq. poisson): the local potential of a fixed
geometry is phi[b] with rho = 0 on the periodic grid, solved with the discrete (FD) Laplacian,
the pseudocharge renormalised to -sum Z and its mean removed (neutralising background),
phi(G = 0) = 0.

Nonlocal part (Sec. 5.B.2: projectors grouped by atom): per atom an s and three p
projectors chi_s = exp(-r^2/2w^2), chi_p_a = (x - R)_a exp(-r^2/2w^2), zero for r >= r_cut,
minimum periodic image.  Reading (normalisation not given): each chi is normalised on the
global grid, sum_g chi^2 dV = 1, and V_nl = sum_I sum_l E_l |chi_Il><chi_Il| with
<chi|psi> = sum_g chi psi dV.
"""
from __future__ import annotations

import math

import numpy as np

from . import fd


def pseudocharge(w) -> np.ndarray:
    """Total pseudocharge b on the global grid (nz, ny, nx), renormalised to -sum Z, mean removed."""
    n = np.asarray(w.n)
    h = w.h
    L = np.asarray(w.L, dtype=np.float64)
    dV = float(np.prod(h))
    b = np.zeros((n[2], n[1], n[0]))
    for I, R in enumerate(w.pos):
        sp = w.species[w.species_index[I]]
        rc = sp.rc_loc
        g1 = []
        for d in range(3):
            x = np.arange(n[d]) * h[d]
            kmax = int(math.ceil(12.0 * rc / L[d])) + 1
            acc = np.zeros(n[d])
            for k in range(-kmax, kmax + 1):           # periodic images: separable Gaussian
                acc += np.exp(-((x - R[d] - k * L[d]) ** 2) / rc ** 2)
            g1.append(acc)
        b += -sp.Zv * math.pi ** -1.5 * rc ** -3 * np.einsum("k,j,i->kji", g1[2], g1[1], g1[0])
    Ztot = sum(w.species[s].Zv for s in w.species_index)
    b *= -Ztot / (b.sum() * dV)
    return b - b.mean()


def solve_poisson_periodic(f: np.ndarray, h, n0: int = fd.N0) -> np.ndarray:
    """phi with -Delta_h phi = 4 pi f on the periodic grid (FD symbol), phi(G=0) = 0."""
    nz, ny, nx = f.shape
    th = [2.0 * math.pi * np.fft.fftfreq(m) for m in (nx, ny, nz)]
    sx = fd.symbol_1d(th[0], h[0], n0)
    sy = fd.symbol_1d(th[1], h[1], n0)
    sz = fd.symbol_1d(th[2], h[2], n0)
    S = sz[:, None, None] + sy[None, :, None] + sx[None, None, :]
    F = np.fft.fftn(4.0 * math.pi * f)
    S[0, 0, 0] = 1.0
    P = F / S
    P[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(P))


def local_potential(w) -> np.ndarray:
    """V_loc = phi[b] on the global grid (rho = 0)."""
    return solve_poisson_periodic(pseudocharge(w), w.h)


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def _chi(dz, dy, dx, wdt):
    """Unnormalised [chi_s, chi_px, chi_py, chi_pz] on displacement arrays."""
    g = np.exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * wdt * wdt))
    return np.stack([g, dx * g, dy * g, dz * g])


def projector_norms(w) -> np.ndarray:
    """(n_atoms, 4) factors N_Il with sum over the global periodic grid of (N chi)^2 dV = 1."""
    n = np.asarray(w.n)
    h = w.h
    L = np.asarray(w.L, dtype=np.float64)
    dV = float(np.prod(h))
    out = np.zeros((len(w.pos), 4))
    for I, R in enumerate(w.pos):
        sp = w.species[w.species_index[I]]
        dd = [_min_image(np.arange(n[d]) * h[d] - R[d], L[d]) for d in range(3)]
        dz, dy, dx = np.meshgrid(dd[2], dd[1], dd[0], indexing="ij")
        inside = (dx * dx + dy * dy + dz * dz) < sp.r_cut ** 2
        chi = _chi(dz, dy, dx, sp.w_proj) * inside
        out[I] = 1.0 / np.sqrt((chi ** 2).sum(axis=(1, 2, 3)) * dV)
    return out


def subdomain_projectors(w, start, size, norms) -> list:
    """Projector table of the subdomain whose point (i, j, k) sits at global index start+(i, j, k)
    (positions (start + i) h, unwrapped).  One entry per atom whose sphere meets the subdomain:
    (flat subdomain indices of the support, chi (4, n_supp) normalised, E (4,))."""
    h = w.h
    L = np.asarray(w.L, dtype=np.float64)
    size = np.asarray(size)
    table = []
    for I, R in enumerate(w.pos):
        sp = w.species[w.species_index[I]]
        idx, dis = [], []
        for d in range(3):
            x = (start[d] + np.arange(size[d])) * h[d]
            dd = _min_image(x - R[d], L[d])
            m = np.abs(dd) < sp.r_cut
            idx.append(np.nonzero(m)[0])
            dis.append(dd[m])
        if any(len(i) == 0 for i in idx):
            continue
        dz, dy, dx = np.meshgrid(dis[2], dis[1], dis[0], indexing="ij")
        inside = (dx * dx + dy * dy + dz * dz) < sp.r_cut ** 2
        if not inside.any():
            continue
        kz, ky, kx = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
        flat = (kx + size[0] * (ky + size[1] * kz))[inside]
        chi = _chi(dz, dy, dx, sp.w_proj)[:, inside] * norms[I][:, None]
        E = np.array([sp.E_s, sp.E_p, sp.E_p, sp.E_p])
        table.append((flat, chi, E))
    return table
