"""Degenerate shapes of the pass against the oracle: a cell without atoms (no projector slots
anywhere: local H only, Sec. 5.A.3 with V_nl = 0) and a cell whose only atom meets some
subdomains and misses the others (subdomains with and without projector slots in the same
launches), on TMA-eligible 44^3 Dirichlet subdomains with a ragged last row tile."""
import numpy as np
import pytest

import synth
from oracle import chefsi, dc, pseudo
from paper_2609_13115_gb300 import xls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2609_13115_gb300 import build
    if not os.path.exists(xls.LIB_PATH):
        build.build()
    xls.load()


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def box3(pos):
    """A 3 x 3 x 3 box of Si conventional cells (30.78 bohr, 72^3 grid) cut into 8 subdomains with
    36^3 cores and Dirichlet buffers of 4 points (44^3 each, 8 states): a subdomain spans 18.8 bohr,
    so with the 4-bohr projector cutoff an atom misses the subdomains on the far side."""
    w = synth.workload(0)
    L = tuple(3 * x for x in w.L)
    cores = np.array([(i, j, k) for k in (0, 36) for j in (0, 36) for i in (0, 36)])
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    return synth.Workload("si_box3_dc8", L, (72, 72, 72), pos, np.zeros(len(pos), dtype=int), w.species,
                          core_lo=cores, core_n=np.full((8, 3), 36), buf=np.full((8, 3), 4),
                          n_states=np.full(8, 8), degree=12, n_passes=2, psi_seed=71)


def smooth_potential(w):
    """A smooth periodic stand-in for V_eff when there are no atoms."""
    x = [np.arange(w.n[d]) * w.h[d] * 2 * np.pi / w.L[d] for d in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    return -0.4 * (np.cos(X) * np.cos(Y) + 0.5 * np.cos(Z)) - 0.1 * np.cos(2 * X + Z)


@pytest.mark.parametrize("prec", [xls.XLS_FP64, xls.XLS_MIXED_FP16])
def test_cell_without_atoms(prec):
    w = box3(np.zeros((0, 3)))
    V = smooth_potential(w)
    subs = dc.partition(w)
    norms = pseudo.projector_norms(w)
    ops = [dc.subdomain_operator(w, s, V, norms) for s in subs]
    assert all(len(op.projectors) == 0 for op in ops)
    offs = synth.psi0_offsets(w)
    with xls.Grid(w, prec) as g:
        g.set_hamiltonian(V)
        for a in (0, 5):
            x = synth.psi0_block(13 + a, subs[a].N, 2)
            y = np.zeros_like(x)
            xls.xls_hamiltonian_apply(g.h, a, x, y)
            assert relerr(y, ops[a].apply(x)) < (1e-12 if prec == xls.XLS_FP64 else 2e-6)
        bnd = xls.xls_get_bounds(g.h, w.n_sub)
        xls.xls_orbitals_random(g.h, w.psi_seed)
        xls.xls_chefsi_batch(g.h, w.degree, w.n_passes)
        lam = [xls.xls_get_eigs(g.h, a, 8)[0] for a in range(w.n_sub)]
    for a in (0, 3, 7):
        H = ops[a]
        b = chefsi.lanczos_upper_bound(H, synth.lanczos_start(H.N))
        assert abs(bnd[a][0] - b) < 1e-9 * abs(b)
        psi0 = synth.psi0_block(w.psi_seed, subs[a].N, 8, offs[a])
        lam_o, _, _ = chefsi.run_chefsi(H, psi0, w.degree, w.n_passes, v0=synth.lanczos_start(H.N))
        if prec == xls.XLS_FP64:
            np.testing.assert_allclose(lam[a], lam_o, rtol=0, atol=1e-8 * max(1.0, np.abs(lam_o).max()))
        else:   # the lower half, which two passes have converged (the upper Ritz values still move)
            np.testing.assert_allclose(lam[a][:4], lam_o[:4], rtol=0, atol=1e-4)


@pytest.mark.parametrize("prec", [xls.XLS_FP64, xls.XLS_MIXED_FP16])
def test_subdomains_with_and_without_projectors(prec):
    w = box3([[15.0, 15.0, 7.7]])
    V = pseudo.local_potential(w)
    subs = dc.partition(w)
    norms = pseudo.projector_norms(w)
    ops = [dc.subdomain_operator(w, s, V, norms) for s in subs]
    n_proj = [len(op.projectors) for op in ops]
    assert min(n_proj) == 0 and max(n_proj) > 0, n_proj
    offs = synth.psi0_offsets(w)
    psi0 = [synth.psi0_block(w.psi_seed, subs[a].N, 8, offs[a]) for a in range(w.n_sub)]
    ref = dc.run(w, V, psi0)
    with xls.Grid(w, prec) as g:
        g.set_hamiltonian(V)
        for a in range(w.n_sub):
            x = synth.psi0_block(29 + a, subs[a].N, 2)
            y = np.zeros_like(x)
            xls.xls_hamiltonian_apply(g.h, a, x, y)
            assert relerr(y, ops[a].apply(x)) < (1e-12 if prec == xls.XLS_FP64 else 2e-6), (a, n_proj[a])
        xls.xls_orbitals_random(g.h, w.psi_seed)
        xls.xls_chefsi_batch(g.h, w.degree, w.n_passes)
        lam = [xls.xls_get_eigs(g.h, a, 8)[0] for a in range(w.n_sub)]
        rho = np.zeros(int(np.prod(w.n)))
        mu, eb, es = xls.xls_density(g.h, w.n_electrons, w.kT, rho)
    for a in range(w.n_sub):
        if prec == xls.XLS_FP64:
            np.testing.assert_allclose(lam[a], ref.lam[a], rtol=0, atol=1e-8 * max(1.0, np.abs(ref.lam[a]).max()))
        else:   # the states below mu + 0.1 Ha, as in the other mixed-path parity tests
            occ = ref.lam[a] < ref.mu + 0.1
            np.testing.assert_allclose(lam[a][occ], ref.lam[a][occ], rtol=0, atol=1e-4)
    assert abs(mu - ref.mu) < (1e-8 if prec == xls.XLS_FP64 else 1e-4)
    assert relerr(rho, ref.rho.ravel()) < (1e-7 if prec == xls.XLS_FP64 else 1e-4)
