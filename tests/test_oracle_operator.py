"""Pins of the oracle's operator parts (FD Laplacian, electrostatics, projectors, H) against
closed forms, published weights, exact polynomial calculus and invariants."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import dc, fd, pseudo
from oracle.operator import SubdomainHamiltonian

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fd_weights_match_published_table():
    table = {}
    with open(os.path.join(GOLDEN, "fd12_weights.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p, v = line.split(":")
            table[int(p)] = Fraction(v.strip())
    w = fd.fd_weights_exact(6)
    assert [table[p] for p in range(7)] == w


def test_fd_stencil_exact_on_polynomials():
    """A 13-point order-12 second-derivative stencil differentiates x^k exactly for k <= 13."""
    w = fd.fd_weights_exact(6)
    for x0 in (Fraction(0), Fraction(3), Fraction(-7, 2)):
        for k in range(0, 14):
            approx = w[0] * x0 ** k + sum(w[p] * ((x0 + p) ** k + (x0 - p) ** k) for p in range(1, 7))
            exact = k * (k - 1) * x0 ** (k - 2) if k >= 2 else Fraction(0)
            assert approx == exact, (x0, k)
    # and the stencil is not exact one degree higher (order is exactly 12)
    k = 14
    approx = w[0] * 0 + sum(w[p] * (Fraction(p) ** k + Fraction(-p) ** k) for p in range(1, 7))
    assert approx != 0


def test_laplacian_polynomial_interior_dirichlet():
    """On interior points (>= 6 from the walls) the Dirichlet Laplacian is exact for cubic polynomials in each axis."""
    n = (15, 14, 13)
    h = (0.3, 0.4, 0.5)
    z, y, x = np.meshgrid(*(np.arange(n[d]) * h[d] for d in (2, 1, 0)), indexing="ij")
    f = x ** 3 + 2 * y ** 2 * z + z ** 4
    lap = fd.laplacian(f, h, (False, False, False))
    exact = 6 * x + 4 * z + 12 * z ** 2
    sl = (slice(6, -6),) * 3
    np.testing.assert_allclose(lap[sl], exact[sl], rtol=1e-9, atol=1e-9)


def test_periodic_laplacian_plane_waves_match_symbol():
    n = (12, 10, 8)
    h = (0.43, 0.5, 0.61)
    for j in [(1, 0, 0), (3, 2, 1), (6, 5, 4)]:
        z, y, x = np.meshgrid(*(np.arange(n[d]) for d in (2, 1, 0)), indexing="ij")
        th = [2 * math.pi * j[d] / n[d] for d in range(3)]
        f = np.cos(th[0] * x + th[1] * y + th[2] * z)
        got = -fd.laplacian(f, h, (True, True, True))
        lam = sum(fd.symbol_1d(np.array(th[d]), h[d]) for d in range(3))
        np.testing.assert_allclose(got, lam * f, atol=1e-10 * abs(lam))


def test_kinetic_maximum_equals_gershgorin():
    """At theta = pi the 1-D symbol is (-w0 + 2 sum |w_p|)/h^2 (alternating weights)."""
    w = fd.fd_weights(6)
    h = 0.4275
    assert fd.symbol_1d(np.array(math.pi), h) == pytest.approx((-w[0] + 2 * np.abs(w[1:]).sum()) / h ** 2, rel=1e-14)
    assert 1.5 * fd.symbol_1d(np.array(math.pi), h) == pytest.approx(58.05, abs=0.01)


def test_poisson_solution_satisfies_fd_equation():
    w = synth.workload(0)
    b = pseudo.pseudocharge(w)
    assert abs(b.sum()) < 1e-9 * np.abs(b).sum()
    phi = pseudo.solve_poisson_periodic(b, w.h)
    res = -fd.laplacian(phi, w.h, (True, True, True)) - 4 * math.pi * b
    assert np.linalg.norm(res) < 1e-11 * np.linalg.norm(4 * math.pi * b)
    assert abs(phi.mean()) < 1e-12


def test_poisson_on_orthorhombic_grid():
    """The same equation, -Delta_h phi = 4 pi (f - mean f), on a grid with three different point
    counts and spacings (each axis's symbol paired with its own spacing), phi of zero mean."""
    rng = np.random.default_rng(8)
    n, h = (14, 16, 18), (0.41, 0.47, 0.53)
    f = rng.standard_normal((n[2], n[1], n[0]))
    phi = pseudo.solve_poisson_periodic(f, h)
    res = -fd.laplacian(phi, h, (True, True, True)) - 4 * math.pi * (f - f.mean())
    assert np.linalg.norm(res) < 1e-11 * np.linalg.norm(4 * math.pi * f)
    assert abs(phi.mean()) < 1e-12


def test_single_atom_potential_matches_erf_coulomb():
    """One well-resolved pseudocharge in a large periodic cube: phi(r) = -Z erf(r/rc)/r
    - (2 pi Z / 3 Omega) r^2 + const near the atom (neutralising background, cubic images)."""
    L = 16.0
    n = 64
    Z, rc = 4.0, 1.0
    w = synth.Workload("one", (L,) * 3, (n,) * 3, np.array([[8.0, 8.0, 8.0]]), np.zeros(1, int),
                       [synth.Species(Zv=Z, rc_loc=rc)], np.zeros((1, 3), int), np.full((1, 3), n),
                       np.zeros((1, 3), int), np.array([1]), 1, 1, 0)
    phi = pseudo.local_potential(w)
    h = L / n
    pts = [(32, 32, 32 + k) for k in range(0, 12)]
    r = np.array([abs(p[2] - 32) * h for p in pts])
    got = np.array([phi[p] for p in pts])
    erf_part = np.array([-Z * math.erf(x / rc) / x if x > 0 else -Z * 2 / (math.sqrt(math.pi) * rc) for x in r])
    model = erf_part - 2 * math.pi * Z / (3 * L ** 3) * r ** 2
    d_got = got - got[0]
    d_model = model - model[0]
    np.testing.assert_allclose(d_got, d_model, atol=2e-4 * Z / rc)


def test_projector_norms_and_symmetry():
    w = synth.workload(0)
    norms = pseudo.projector_norms(w)
    # continuum value of the s factor: (pi w^2)^(-3/4); the cut at 4 bohr (5 w) is negligible
    np.testing.assert_allclose(norms[:, 0], (math.pi * 0.8 ** 2) ** -0.75, rtol=1e-3)
    # ideal sites on a cubic grid: the three p factors are equal
    np.testing.assert_allclose(norms[:, 1], norms[:, 2], rtol=1e-12)
    np.testing.assert_allclose(norms[:, 1], norms[:, 3], rtol=1e-12)
    subs = dc.partition(w)
    tab = pseudo.subdomain_projectors(w, subs[0].start, subs[0].size, norms)
    dV = float(np.prod(w.h))
    for flat, chi, E in tab:
        G = chi @ chi.T * dV
        np.testing.assert_allclose(np.diag(G), 1.0, rtol=1e-12)   # periodic cell: whole sphere inside
        assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12       # s/p orthogonal at ideal sites


def _toy_operator(periodic, seed=5):
    w = synth.workload(0)
    norms = pseudo.projector_norms(w)
    size = np.array([11, 9, 10])
    start = np.array([3, -2, 7])
    rng = np.random.default_rng(seed)
    V = rng.standard_normal(size[::-1])
    proj = pseudo.subdomain_projectors(w, start, size, norms)
    return SubdomainHamiltonian(size, w.h, periodic, V, proj)


@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True), (True, True, True)])
def test_hamiltonian_is_symmetric(periodic):
    H = _toy_operator(periodic)
    assert len(H.projectors) > 0
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal((2, H.N))
    Hx, Hy = H.apply(x[None])[0], H.apply(y[None])[0]
    scale = np.linalg.norm(x) * np.linalg.norm(y) * 100.0
    assert abs(x @ Hy - y @ Hx) < 1e-13 * scale


def test_dense_matches_matrix_free():
    H = _toy_operator((True, False, False))
    D = H.dense()
    assert np.abs(D - D.T).max() < 1e-12
    rng = np.random.default_rng(2)
    X = rng.standard_normal((3, H.N))
    np.testing.assert_allclose((D @ X.T).T, H.apply(X), atol=1e-11)


def test_restriction_wraps_periodically():
    w = synth.workload(1)
    subs = dc.partition(w)
    n = w.n
    V = np.arange(np.prod(n), dtype=float).reshape(n[2], n[1], n[0])
    s = subs[0]
    assert list(s.start) == [-12, -12, -12] and all(s.periodic)
    Vs = dc.restrict(V, s)
    assert Vs[0, 0, 0] == V[36, 36, 36]
    assert Vs[12, 12, 12] == V[0, 0, 0]
    # the cores tile the global grid exactly once
    seen = np.zeros(np.prod(n), int)
    for s in subs:
        seen[dc.core_global_indices(s, n)] += 1
    assert (seen == 1).all()


def test_local_subdomain_operator_equals_global_one():
    """The operator built from the atoms near a subdomain, with projector norms summed on one
    conventional cell, equals the operator with norms summed on the whole periodic grid."""
    from oracle import dc
    w = synth.workload(1)
    V = synth.veff_erf_wells(w)
    subs = dc.partition(w)
    norms = pseudo.projector_norms(w)
    x = synth.psi0_block(5, subs[3].N, 2)
    H_glob = dc.subdomain_operator(w, subs[3], V, norms)
    H_loc = dc.subdomain_operator_local(w, subs[3], V)
    assert len(H_loc.projectors) == len(H_glob.projectors)
    y0, y1 = H_glob.apply(x), H_loc.apply(x)
    assert np.abs(y1 - y0).max() < 1e-13 * np.abs(y0).max()


def _fd_matrix_1d(n, periodic):
    """The 1-D second-difference matrix built entry by entry: row i takes w_|p| at column i + p
    for |p| <= 6, wrapped modulo n on a periodic axis and dropped outside [0, n) on a Dirichlet one."""
    w = fd.fd_weights(6)
    D = np.zeros((n, n))
    for i in range(n):
        for p in range(-6, 7):
            j = i + p
            if periodic:
                D[i, j % n] += w[abs(p)]
            elif 0 <= j < n:
                D[i, j] += w[abs(p)]
    return D


@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, False), (False, True, True)])
def test_hamiltonian_equals_kronecker_sum_matrix(periodic):
    """H = -1/2 (D_x/h_x^2 (+) D_y/h_y^2 (+) D_z/h_z^2) + diag(V) on a grid with x fastest, from 1-D
    matrices assembled entry by entry: pins the boundary handling of each axis (zero outside a
    Dirichlet box, wrap on a periodic axis), which spacing goes with which axis, the kinetic factor
    and where each value of V sits."""
    size, h = (7, 13, 5), (0.31, 0.42, 0.57)
    rng = np.random.default_rng(17)
    V = rng.standard_normal(size[::-1])
    H = SubdomainHamiltonian(size, h, periodic, V, [])
    Dx, Dy, Dz = (_fd_matrix_1d(size[d], periodic[d]) / h[d] ** 2 for d in range(3))
    Ix, Iy, Iz = (np.eye(s) for s in size)
    lap = np.kron(Iz, np.kron(Iy, Dx)) + np.kron(Iz, np.kron(Dy, Ix)) + np.kron(Dz, np.kron(Iy, Ix))
    ref = -0.5 * lap + np.diag(V.ravel())
    np.testing.assert_allclose(H.dense(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_projectors_are_eigenvectors_of_the_nonlocal_term():
    """One atom on a grid point of a periodic cube: its four projectors are orthonormal (parity
    of the grid about the atom), so V_nl chi_l = E_l chi_l for each channel and V_nl vanishes on a
    vector supported outside the projector sphere.  The spacing (12/28 bohr) puts no grid point
    on the cut-off sphere, where rounding could keep a point on one side of the atom and drop its
    mirror image."""
    L, n = 12.0, 28
    sp = synth.SI
    w = synth.Workload("one_atom", (L,) * 3, (n,) * 3, np.array([[6.0, 6.0, 6.0]]), np.zeros(1, int), [sp],
                       np.zeros((1, 3), int), np.full((1, 3), n), np.zeros((1, 3), int), np.array([4]), 1, 1, 0)
    s = dc.partition(w)[0]
    H = dc.subdomain_operator(w, s, np.zeros((n, n, n)), pseudo.projector_norms(w))
    (flat, chi, E), = H.projectors
    np.testing.assert_allclose(E, [sp.E_s, sp.E_p, sp.E_p, sp.E_p])
    for l in range(4):
        x = np.zeros((1, H.N))
        x[0, flat] = chi[l]
        y = H.apply_nonlocal(x)
        np.testing.assert_allclose(y, E[l] * x, rtol=0, atol=1e-12 * abs(E[l]) * np.abs(x).max())
    far = np.zeros((1, H.N))
    far[0, 0] = 1.0                                       # the corner, 10.4 bohr from the atom
    assert 0 not in set(flat)
    assert np.abs(H.apply_nonlocal(far)).max() == 0.0


def test_local_subdomain_operator_with_random_atoms():
    """Random atom positions on a 3^3-cell box (72^3 grid) cut into Dirichlet subdomains of 48^3, so
    that some atoms sit outside a subdomain within the projector cutoff of its faces: the local
    operator keeps exactly the atoms whose spheres meet the subdomain, and equals the operator with
    whole-grid norms.  (On the 64-atom cell every subdomain spans the period, so every atom meets
    every subdomain and the choice of atoms is not exercised.)"""
    a = synth.workload(0).L[0]
    rng = np.random.default_rng(23)
    n_at = 60
    pos = rng.uniform(0.0, 3 * a, size=(n_at, 3))
    cores = np.array([[0, 0, 0], [24, 36, 12], [48, 12, 36]])
    w = synth.Workload("random_box3", (3 * a,) * 3, (72,) * 3, pos, np.zeros(n_at, int), [synth.SI],
                       core_lo=cores, core_n=np.full((3, 3), 24), buf=np.full((3, 3), 12),
                       n_states=np.full(3, 4), degree=4, n_passes=1, psi_seed=3)
    subs = dc.partition(w)
    assert not any(s.periodic.any() for s in subs)
    norms = pseudo.projector_norms(w)
    V = np.zeros((72, 72, 72))
    for k, s in enumerate(subs):
        H_glob = dc.subdomain_operator(w, s, V, norms)
        H_loc = dc.subdomain_operator_local(w, s, V)
        assert 0 < len(H_loc.projectors) == len(H_glob.projectors) < n_at
        x = synth.psi0_block(9 + k, s.N, 2)
        y0, y1 = H_glob.apply(x), H_loc.apply(x)
        assert np.abs(y1 - y0).max() < 1e-13 * np.abs(y0).max()


def test_partition_mixes_periodic_and_dirichlet_axes():
    """A 2 x 4 x 2-cell box (48 x 96 x 48 points) with 24^3 cores and 12-point buffers: along x and
    z a subdomain spans the period (48 points, periodic, one period long), along y it is a 48-point
    Dirichlet box starting 12 points before its core; the core sits 12 points into the subdomain
    on every axis, and the restriction reads V at the wrapped global indices."""
    a = synth.workload(0).L[0]
    cores = np.array([[0, 0, 0], [24, 72, 24], [0, 48, 24]])
    w = synth.Workload("mixed", (2 * a, 4 * a, 2 * a), (48, 96, 48), np.zeros((0, 3)), np.zeros(0, int), [synth.SI],
                       core_lo=cores, core_n=np.full((3, 3), 24), buf=np.full((3, 3), 12),
                       n_states=np.full(3, 4), degree=4, n_passes=1, psi_seed=3)
    V = np.arange(96 * 48 * 48, dtype=float).reshape(48, 96, 48)      # (nz, ny, nx), distinct values
    for s, c in zip(dc.partition(w), cores):
        assert list(s.periodic) == [True, False, True]
        assert list(s.size) == [48, 48, 48]
        assert list(s.start) == [c[0] - 12, c[1] - 12, c[2] - 12]
        assert list(s.core_lo) == [12, 12, 12] and list(s.core_global_lo) == list(c)
        Vs = dc.restrict(V, s)
        for (i, j, k) in [(0, 0, 0), (47, 5, 30), (12, 12, 12), (3, 47, 47)]:
            gi, gj, gk = (s.start[0] + i) % 48, (s.start[1] + j) % 96, (s.start[2] + k) % 48
            assert Vs[k, j, i] == V[gk, gj, gi]
        # the core box of the subdomain is the core box on the global grid
        loc = dc.core_local_indices(s)
        glob = dc.core_global_indices(s, w.n)
        flatV = V.ravel()
        np.testing.assert_array_equal(Vs.ravel()[loc], flatV[glob])
