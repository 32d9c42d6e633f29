"""Divide-and-conquer partition, restriction and assembly (Sec. 5.A.2 and 5.A.5).

Cores Omega_C^alpha are disjoint index boxes covering the global grid (binary partition of
unity p^alpha).  Each subdomain extends its core by `buf` points on each side.  Reading
(boundary condition not given): the subdomain Hamiltonian is Dirichlet-zero outside
Omega^alpha, except along an axis where Omega^alpha spans the whole period, where it is
periodic; the subdomain is then exactly one period long.  V_eff is restricted from the
periodic global grid.  Projectors of atoms whose sphere meets Omega^alpha are truncated
to Omega^alpha; their normalisation is that of the full sphere on the global grid.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from synth import lanczos_start

from . import chefsi, fermi, pseudo
from .operator import SubdomainHamiltonian


@dataclass
class Subdomain:
    start: np.ndarray       # global index of local point 0 (may be negative), (x, y, z)
    size: np.ndarray        # local points per axis
    periodic: np.ndarray    # bool per axis
    core_lo: np.ndarray     # local index of the first core point
    core_n: np.ndarray
    core_global_lo: np.ndarray

    @property
    def N(self) -> int:
        return int(np.prod(self.size))


def partition(w) -> list:
    n = np.asarray(w.n)
    subs = []
    for a in range(w.n_sub):
        core_lo, core_n, buf = (np.asarray(v[a]) for v in (w.core_lo, w.core_n, w.buf))
        size = core_n + 2 * buf
        periodic = size >= n
        b = np.where(periodic, np.minimum(buf, (n - core_n) // 2), buf)
        size = np.where(periodic, n, size)
        subs.append(Subdomain(start=core_lo - b, size=size, periodic=periodic, core_lo=b,
                              core_n=core_n, core_global_lo=core_lo))
    return subs


def restrict(V: np.ndarray, s: Subdomain) -> np.ndarray:
    """V on Omega^alpha, (nz, ny, nx), from the periodic global grid V (nz, ny, nx)."""
    nz, ny, nx = V.shape
    ix = (s.start[0] + np.arange(s.size[0])) % nx
    iy = (s.start[1] + np.arange(s.size[1])) % ny
    iz = (s.start[2] + np.arange(s.size[2])) % nz
    return V[np.ix_(iz, iy, ix)]


def core_local_indices(s: Subdomain) -> np.ndarray:
    k, j, i = np.meshgrid(*(s.core_lo[d] + np.arange(s.core_n[d]) for d in (2, 1, 0)), indexing="ij")
    return (i + s.size[0] * (j + s.size[1] * k)).ravel()


def core_global_indices(s: Subdomain, n) -> np.ndarray:
    k, j, i = np.meshgrid(*((s.core_global_lo[d] + np.arange(s.core_n[d])) % n[d] for d in (2, 1, 0)),
                          indexing="ij")
    return (i + n[0] * (j + n[1] * k)).ravel()


def interior_weights(Psi: np.ndarray, s: Subdomain) -> np.ndarray:
    """c_n = sum over core points of psi_n^2 (Sec. 5.A.4)."""
    idx = core_local_indices(s)
    return np.sum(Psi[:, idx] ** 2, axis=1)


def subdomain_operator(w, s: Subdomain, V: np.ndarray, norms: np.ndarray) -> SubdomainHamiltonian:
    proj = pseudo.subdomain_projectors(w, s.start, s.size, norms)
    return SubdomainHamiltonian(s.size, w.h, s.periodic, restrict(V, s), proj)


def subdomain_operator_local(w, s: Subdomain, V: np.ndarray) -> SubdomainHamiltonian:
    """subdomain_operator for cells too large to normalise every projector on the whole grid:
    only the atoms within r_cut + 1 bohr of the subdomain box are kept (the others have no
    support in it), and each kept atom's normalisation sum runs over one conventional cell of the
    same spacing carrying the atom at its position modulo the cell -- the grid points within
    r_cut of the atom form the same set of displacements as on the global grid (r_cut is below
    half the cell), so the sum has the same terms."""
    import synth
    near = synth.near_atoms(w, s.start, s.size, max(sp.r_cut for sp in w.species) + 1.0)
    a = synth.SI_LATTICE_BOHR
    cell = synth.Workload("norm_cell", (a, a, a), (synth.POINTS_PER_CELL,) * 3, np.mod(w.pos[near], a),
                          w.species_index[near], w.species, core_lo=np.zeros((1, 3), int),
                          core_n=np.full((1, 3), synth.POINTS_PER_CELL), buf=np.zeros((1, 3), int),
                          n_states=np.array([1]), degree=1, n_passes=1, psi_seed=0)
    norms = pseudo.projector_norms(cell)
    local = synth.Workload("near", w.L, w.n, w.pos[near], w.species_index[near], w.species, w.core_lo, w.core_n,
                           w.buf, w.n_states, w.degree, w.n_passes, w.psi_seed)
    return subdomain_operator(local, s, V, norms)


@dataclass
class DCResult:
    lam: list
    c: list
    Psi: list
    b: list
    mu: float
    rho: np.ndarray
    e_band: float
    e_entropy: float


def assemble(w, subs, lam, c, Psi, kT: float, n_electrons: float):
    """mu from all (lambda, c); rho on every core point from its own subdomain; energies."""
    mu = fermi.fermi_level(np.concatenate(lam), np.concatenate(c), kT, n_electrons)
    n = np.asarray(w.n)
    dV = float(np.prod(w.h))
    rho = np.zeros(int(np.prod(n)))
    for s, la, P in zip(subs, lam, Psi):
        g = fermi.occupations(la, mu, kT)
        rho[core_global_indices(s, n)] = fermi.point_density(P[:, core_local_indices(s)], g, dV)
    lam_all, c_all = np.concatenate(lam), np.concatenate(c)
    return (mu, rho.reshape(n[2], n[1], n[0]), fermi.band_energy(lam_all, c_all, mu, kT),
            fermi.entropy_energy(lam_all, c_all, mu, kT))


def run(w, V: np.ndarray, Psi0: list, n_passes: int | None = None, bounds: list | None = None,
        n_electrons: float | None = None, subdomains=None) -> DCResult:
    """The D&C CheFSI pass over every subdomain (independent for fixed V_eff), then mu, rho, E."""
    subs = partition(w)
    which = range(w.n_sub) if subdomains is None else subdomains
    norms = pseudo.projector_norms(w)
    n_passes = w.n_passes if n_passes is None else n_passes
    lam, c, Psi, bs = [], [], [], []
    for k, a in enumerate(which):
        H = subdomain_operator(w, subs[a], V, norms)
        b = None if bounds is None else bounds[k]
        la, P, b = chefsi.run_chefsi(H, Psi0[k], w.degree, n_passes, b, v0=lanczos_start(H.N))
        lam.append(la)
        Psi.append(P)
        c.append(interior_weights(P, subs[a]))
        bs.append(b)
    if subdomains is not None:
        return DCResult(lam, c, Psi, bs, float("nan"), None, float("nan"), float("nan"))
    ne = w.n_electrons if n_electrons is None else n_electrons
    mu, rho, eb, es = assemble(w, subs, lam, c, Psi, w.kT, ne)
    return DCResult(lam, c, Psi, bs, mu, rho, eb, es)
