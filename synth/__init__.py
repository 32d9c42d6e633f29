"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds input generation only: random numbers, atom geometries, the
subdomain partition descriptors of each workload and a stand-in effective
potential.  It contains none of the CheFSI method's arithmetic (no Hamiltonian,
no filter, no Rayleigh-Ritz, no Fermi level), so that the oracle and the CUDA
path can both consume its outputs without sharing any computation.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), used as
a counter-based generator: output i of seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SI_LATTICE_BOHR = 10.26          # diamond-cubic Si conventional cell edge
POINTS_PER_CELL = 24             # 24 points per cell edge -> h = 0.4275 bohr


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream of `seed` (uint64)."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm_half(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles on [-0.5, 0.5): top 53 bits of each SplitMix64 output."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 0.5


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller on consecutive output pairs."""
    npair = (count + 1) // 2
    z = splitmix64(seed, 2 * npair)
    u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)   # (0, 1]
    u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)           # [0, 1)
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:count]


def seeded_permutation(seed: int, n: int) -> np.ndarray:
    """Fisher-Yates shuffle of range(n) driven by SplitMix64 outputs."""
    z = splitmix64(seed, max(n - 1, 0))
    perm = np.arange(n)
    for k, i in enumerate(range(n - 1, 0, -1)):
        j = int(z[k] % np.uint64(i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return perm


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------

_FCC = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
DIAMOND_FRAC = np.concatenate([_FCC, _FCC + 0.25])   # 8 sites of the conventional cell


def si_diamond(ncell=(1, 1, 1), a: float = SI_LATTICE_BOHR) -> np.ndarray:
    """Cartesian positions (bohr) of an ideal diamond-cubic supercell, x-major cell order."""
    cells = [(i, j, k) for k in range(ncell[2]) for j in range(ncell[1]) for i in range(ncell[0])]
    pos = [(np.array(c) + f) * a for c in cells for f in DIAMOND_FRAC]
    return np.array(pos, dtype=np.float64)


def displace(pos: np.ndarray, sigma: float, seed: int, L) -> np.ndarray:
    """i.i.d. N(0, sigma^2) per Cartesian component (atom-major order), wrapped into the cell."""
    if sigma == 0.0:
        return pos.copy()
    d = normals(seed, pos.size).reshape(pos.shape) * sigma
    return np.mod(pos + d, np.asarray(L, dtype=np.float64))


@dataclass(frozen=True)
class Species:
    """Synthetic pseudopotential of one species (local erf potential + s/p KB projectors)."""
    Zv: float = 4.0          # valence charge
    rc_loc: float = 1.0      # V_loc(r) = -Zv erf(r / rc_loc) / r
    w_proj: float = 0.8      # projector Gaussian width
    r_cut: float = 4.0       # projectors vanish for r >= r_cut
    E_s: float = 2.0         # KB energy of the s projector (Ha)
    E_p: float = 0.5         # KB energy of each p projector (Ha)


SI = Species()
SPECIES_B = Species(Zv=3.0, rc_loc=1.2, w_proj=0.9)


@dataclass
class Workload:
    """One synthetic workload: periodic orthorhombic cell, global grid, atoms, D&C partition."""
    name: str
    L: tuple                      # cell edges (bohr)
    n: tuple                      # global grid points per axis (x, y, z)
    pos: np.ndarray               # (n_atoms, 3) bohr, inside [0, L)
    species_index: np.ndarray     # (n_atoms,) index into `species`
    species: list
    core_lo: np.ndarray           # (n_sub, 3) global index of the first core point
    core_n: np.ndarray            # (n_sub, 3) core points per axis
    buf: np.ndarray               # (n_sub, 3) buffer points on each side
    n_states: np.ndarray          # (n_sub,)
    degree: int
    n_passes: int
    psi_seed: int
    kT: float = 0.01
    meta: dict = field(default_factory=dict)

    @property
    def n_sub(self) -> int:
        return len(self.core_lo)

    @property
    def h(self) -> np.ndarray:
        return np.asarray(self.L, dtype=np.float64) / np.asarray(self.n, dtype=np.float64)

    @property
    def n_electrons(self) -> float:
        return float(sum(self.species[s].Zv for s in self.species_index))

    def sub_size(self, a: int) -> np.ndarray:
        """Subdomain points per axis: core + 2 buffers, capped at the period (then periodic)."""
        return np.minimum(self.core_n[a] + 2 * self.buf[a], np.asarray(self.n))

    def sub_points(self, a: int) -> int:
        return int(np.prod(self.sub_size(a)))


def consistent_states(n_electrons_sub: float, factor: float = 1.2, multiple: int = 16) -> int:
    """State count that can hold a subdomain's electrons with room to spare."""
    k = math.ceil(factor * n_electrons_sub / 2.0)
    return multiple * math.ceil(k / multiple)


def workload(cfg: int, consistent: bool = True, ncell: int | None = None) -> Workload:
    """The synthetic workloads.  cfg 0: 8-atom cell, 24^3, no D&C.  cfg 1: 64 atoms, 8
    subdomains of 48^3 (buffer covers the cell).  cfg 3: 72^3 subdomains (1-cell core and
    1-cell buffer) of a 12^3-cell crystal; `ncell` shrinks the crystal for tests."""
    a = SI_LATTICE_BOHR
    P = POINTS_PER_CELL
    if cfg == 0:
        L = (a, a, a)
        pos = si_diamond((1, 1, 1))
        return Workload("si8_24cube_ns24_m16", L, (P, P, P), pos, np.zeros(len(pos), int), [SI],
                        core_lo=np.zeros((1, 3), int), core_n=np.full((1, 3), P), buf=np.zeros((1, 3), int),
                        n_states=np.array([24]), degree=16, n_passes=4, psi_seed=1000)
    if cfg == 1:
        k = 2
        L = (k * a,) * 3
        pos = displace(si_diamond((k, k, k)), 0.05, 2001, L)
        cores = np.array([(i, j, l) for l in range(k) for j in range(k) for i in range(k)]) * P
        ns = consistent_states(4.0 * 64) if consistent else 80   # 160 / 80
        nsub = len(cores)
        return Workload(f"si64_dc8_48cube_ns{ns}_m20", L, (k * P,) * 3, pos, np.zeros(len(pos), int), [SI],
                        core_lo=cores, core_n=np.full((nsub, 3), P), buf=np.full((nsub, 3), P // 2),
                        n_states=np.full(nsub, ns), degree=20, n_passes=1, psi_seed=1001)
    if cfg == 2:
        # 2 % vacancies (round half up) by a seeded shuffle, displacements sigma = 0.1 bohr; every subdomain
        # a 1-cell core with a buffer of 0.5, 0.75 or 1 cell (12, 18 or 24 points) drawn from the seed
        k = 8 if ncell is None else ncell
        L = (k * a,) * 3
        full = si_diamond((k, k, k))
        n_vac = int(math.floor(0.02 * len(full) + 0.5))
        vac = set(seeded_permutation(2002 ^ 0x5A5A, len(full))[:n_vac].tolist())
        keep = np.array([i for i in range(len(full)) if i not in vac])
        pos = displace(full[keep], 0.1, 2002, L)
        cores = np.array([(i, j, l) for l in range(k) for j in range(k) for i in range(k)]) * P
        nsub = len(cores)
        widths = np.array([P // 2, (3 * P) // 4, P])[(splitmix64(1002 ^ 0x3C3C, nsub) % np.uint64(3)).astype(int)]
        buf = np.repeat(widths[:, None], 3, axis=1)
        w0 = Workload(f"si{len(pos)}_dc{nsub}_uneven", L, (k * P,) * 3, pos, np.zeros(len(pos), int), [SI],
                      core_lo=cores, core_n=np.full((nsub, 3), P), buf=buf, n_states=np.zeros(nsub, int),
                      degree=20, n_passes=1, psi_seed=1002)
        if consistent:   # electrons of the atoms inside each subdomain's box
            ns = []
            for aa in range(nsub):
                start = cores[aa] - buf[aa]
                inside = near_atoms(w0, start, w0.sub_size(aa), 0.0)
                ns.append(consistent_states(4.0 * len(inside)))
            w0.n_states = np.array(ns)
        else:
            w0.n_states = np.array([{P // 2: 80, (3 * P) // 4: 160, P: 240}[int(x)] for x in widths])
        w0.name = f"si{len(pos)}_dc{nsub}_uneven_m20"
        return w0
    if cfg == 3:
        k = 12 if ncell is None else ncell
        L = (k * a,) * 3
        pos = displace(si_diamond((k, k, k)), 0.1, 2003, L)
        cores = np.array([(i, j, l) for l in range(k) for j in range(k) for i in range(k)]) * P
        ns = consistent_states(4.0 * 216) if consistent else 240
        nsub = len(cores)
        return Workload(f"si{8 * k ** 3}_dc{nsub}_72cube_ns{ns}_m20", L, (k * P,) * 3, pos,
                        np.zeros(len(pos), int), [SI], core_lo=cores, core_n=np.full((nsub, 3), P),
                        buf=np.full((nsub, 3), P), n_states=np.full(nsub, ns), degree=20, n_passes=1,
                        psi_seed=1003)
    raise ValueError(f"unknown workload {cfg}")


def near_atoms(w: Workload, start, size, margin: float) -> np.ndarray:
    """Indices (in order) of the atoms within `margin` of the box of grid points start .. start +
    size - 1 (minimum image): the atoms that can meet a subdomain of that box."""
    h = w.h
    L = np.asarray(w.L, dtype=np.float64)
    lo = np.asarray(start) * h
    hi = (np.asarray(start) + np.asarray(size) - 1) * h
    c = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo) + margin
    d = w.pos - c
    d -= L * np.round(d / L)
    return np.nonzero(np.all(np.abs(d) <= half, axis=1))[0]


def psi0_block(seed: int, n_points: int, n_states: int, offset: int = 0) -> np.ndarray:
    """Start block of one subdomain: (n_states, n_points), vector-major, U[-0.5, 0.5)."""
    u = uniform_pm_half(seed, n_points * n_states, offset)
    return u.reshape(n_states, n_points)


LANCZOS_SEED = 0x1A4C705

def lanczos_start(n_points: int) -> np.ndarray:
    """Start vector of the Lanczos spectrum bound: U[-0.5, 0.5) from a fixed seed."""
    return uniform_pm_half(LANCZOS_SEED, n_points)


def psi0_offsets(w: Workload) -> list:
    """Stream offset of each subdomain's start block (blocks follow each other in the stream)."""
    off, out = 0, []
    for a in range(w.n_sub):
        out.append(off)
        off += w.sub_points(a) * int(w.n_states[a])
    return out


def _erf_wells_slab(args):
    """Contribution of every atom to the z-planes [z0, z1) of the stand-in potential (atoms in
    index order, so that each grid value receives its terms in the same order as a serial sum)."""
    n, h, L, pos, zv, rc, r_trunc, z0, z1 = args
    from scipy.special import erf as erf_v
    V = np.zeros((z1 - z0, n[1], n[0]))
    axes = [np.arange(n[d]) * h[d] for d in range(3)]
    axes[2] = axes[2][z0:z1]
    for I, R in enumerate(pos):
        idx, dis = [], []
        for d in range(3):
            dd = axes[d] - R[d]
            dd -= L[d] * np.round(dd / L[d])
            m = np.abs(dd) < r_trunc
            idx.append(np.nonzero(m)[0])
            dis.append(dd[m])
        if idx[2].size == 0:
            continue
        dz, dy, dx = np.meshgrid(dis[2], dis[1], dis[0], indexing="ij")
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        r_safe = np.where(r > 1e-12, r, 1.0)
        v = np.where(r > 1e-12, -zv[I] * erf_v(r_safe / rc[I]) / r_safe, -zv[I] * 2.0 / (math.sqrt(math.pi) * rc[I]))
        v = np.where(r < r_trunc, v, 0.0)
        V[np.ix_(idx[2], idx[1], idx[0])] += v
    return V


def veff_erf_wells(w: Workload, r_trunc: float = 8.0, processes: int | None = None) -> np.ndarray:
    """Stand-in effective potential on the global grid, shape (nz, ny, nx): the sum over atoms
    of -Zv erf(r/rc)/r (minimum image, truncated at r_trunc), shifted to zero mean.  It has
    the shape and scale of a self-consistent local potential of the workload and is used as
    an input wherever the workload's electrostatics are not solved.  Large grids are built in
    z-slabs by a pool of processes (the same values as one process)."""
    n = np.asarray(w.n)
    h = w.h
    L = np.asarray(w.L, dtype=np.float64)
    zv = np.array([w.species[s].Zv for s in w.species_index], dtype=np.float64)
    rc = np.array([w.species[s].rc_loc for s in w.species_index], dtype=np.float64)
    if processes is None:
        import os
        processes = min(16, os.cpu_count() or 1) if int(np.prod(n)) * len(w.pos) > 2 ** 31 else 1
    cuts = np.linspace(0, n[2], max(1, min(processes, n[2])) + 1).astype(int)
    jobs = [(n, h, L, w.pos, zv, rc, r_trunc, int(cuts[k]), int(cuts[k + 1])) for k in range(len(cuts) - 1)]
    if len(jobs) == 1:
        V = _erf_wells_slab(jobs[0])
    else:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(len(jobs), mp_context=mp.get_context("spawn")) as ex:
            V = np.concatenate(list(ex.map(_erf_wells_slab, jobs)), axis=0)
    return V - V.mean()


def mlp_init(seed: int, layers=((32, 64), (64, 64), (64, 64), (64, 1))) -> np.ndarray:
    """Flat parameters of the learned-start MLP (W row = input, then bias, per layer): weights
    uniform in +-sqrt(6 / (fan_in + fan_out)) from the SplitMix64 stream, biases zero."""
    out, off = [], 0
    for i, o in layers:
        a = math.sqrt(6.0 / (i + o))
        out.append(2.0 * a * uniform_pm_half(seed, i * o, off))
        off += i * o
        out.append(np.zeros(o))
    return np.concatenate(out)


def two_species(w: Workload, substitute: list) -> Workload:
    """Copy of w with the atoms `substitute` turned into the second species."""
    idx = np.array(w.species_index).copy()
    idx[list(substitute)] = 1
    return Workload(w.name + "_2sp", w.L, w.n, w.pos, idx, [w.species[0], SPECIES_B], w.core_lo, w.core_n, w.buf,
                    w.n_states, w.degree, w.n_passes, w.psi_seed, w.kT)
