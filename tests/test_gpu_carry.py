"""Wave carry mode (xls_wave_carry, xls_chefsi_wave) against the oracle.

In carry mode a worker of W subdomain slots is re-targeted to each wave in turn, and each wave's
passes start from the rotated block the previous wave left in the same slot (Sec. 5.A.5,
"Parallel CheFSI": subdomains are independent for a fixed V_eff; the restart from a neighbour's
subspace is this library's).  The oracle follows the same schedule with its own pieces: per wave
and slot, the Lanczos bound of the new subdomain, (a, a0) from the subdomain's own last pass or
else from the slot's last pass (from the Rayleigh-Ritz values of the random start block on the
very first wave), one CheFSI pass; then the Fermi level of all subdomains and each core's
density from its own subdomain.
"""
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


def dirichlet_cell():
    """The 8-atom cell cut into eight 18^3 subdomains (12^3 cores, Dirichlet buffers of 3 points)."""
    w = synth.workload(0)
    cores = np.array([(i, j, k) for k in (0, 12) for j in (0, 12) for i in (0, 12)])
    return synth.Workload("si8_dc8_dirichlet", w.L, w.n, synth.displace(w.pos, 0.05, 77, w.L), w.species_index,
                          w.species, core_lo=cores, core_n=np.full((8, 3), 12), buf=np.full((8, 3), 3),
                          n_states=np.full(8, 16), degree=10, n_passes=3, psi_seed=55)


def oracle_carry(w, V, slots, cycles):
    """The oracle on the carry schedule: (lambda, Psi) of every subdomain after `cycles` sweeps."""
    subs = dc.partition(w)
    norms = pseudo.projector_norms(w)
    ops = [dc.subdomain_operator(w, s, V, norms) for s in subs]
    offs = synth.psi0_offsets(w)
    slot_psi = [synth.psi0_block(w.psi_seed, subs[j].N, int(w.n_states[j]), offs[j]) for j in range(slots)]
    slot_lam = [None] * slots
    own = [None] * w.n_sub
    for _ in range(cycles):
        for first in range(0, w.n_sub, slots):
            for j in range(slots):
                a = first + j
                H = ops[a]
                b = chefsi.lanczos_upper_bound(H, synth.lanczos_start(H.N))
                prev = own[a][0] if own[a] is not None else slot_lam[j]
                if prev is None:
                    prev = chefsi.ritz_values(H, slot_psi[j])
                lam, P = chefsi.chefsi_pass(H, slot_psi[j], w.degree, float(prev.max()), b, float(prev.min()))
                slot_psi[j], slot_lam[j] = P, lam
                own[a] = (lam, P)
    lam = [own[a][0] for a in range(w.n_sub)]
    Psi = [own[a][1] for a in range(w.n_sub)]
    c = [dc.interior_weights(Psi[a], subs[a]) for a in range(w.n_sub)]
    mu, rho, e_band, e_ent = dc.assemble(w, subs, lam, c, Psi, w.kT, w.n_electrons)
    return lam, mu, rho, e_band, e_ent


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [xls.XLS_FP64, xls.XLS_MIXED_FP16])
def test_carry_waves_match_oracle_schedule(prec):
    w = dirichlet_cell()
    V = pseudo.local_potential(w)
    slots, cycles = 2, 3
    lam_o, mu_o, rho_o, eb_o, es_o = oracle_carry(w, V, slots, cycles)
    budget = (1 << 26) + 20 * (1 << 20)          # below the footprint of all eight subdomains
    with xls.Grid(w, prec, hbm_budget_bytes=budget) as g:
        g.set_hamiltonian(V)
        n_waves, _ = xls.xls_get_waves(g.h, w.n_sub)
        assert n_waves > 1
        xls.xls_wave_carry(g.h, slots)
        n_waves, firsts = xls.xls_get_waves(g.h, w.n_sub)
        assert n_waves == w.n_sub // slots and firsts == list(range(0, w.n_sub, slots))
        xls.xls_orbitals_random(g.h, w.psi_seed)
        for c in range(cycles):
            if c == 0:
                for k in range(n_waves):                 # one wave at a time
                    xls.xls_chefsi_wave(g.h, k, w.degree, 1)
            else:
                xls.xls_chefsi_batch(g.h, w.degree, 1)   # every wave in turn
        lam = [xls.xls_get_eigs(g.h, a, int(w.n_states[a]))[0] for a in range(w.n_sub)]
        rho = np.zeros(int(np.prod(w.n)))
        mu, eb, es = xls.xls_density(g.h, w.n_electrons, w.kT, rho)
    n_at = len(w.pos)
    if prec == xls.XLS_FP64:
        for a in range(w.n_sub):
            np.testing.assert_allclose(lam[a], lam_o[a], rtol=0, atol=1e-8)
        assert abs(mu - mu_o) < 1e-8
        assert abs(eb - eb_o) < 1e-8 * n_at and abs(es - es_o) < 1e-8 * n_at
        assert relerr(rho, rho_o.ravel()) < 1e-7
    else:
        for a in range(w.n_sub):
            occ = lam_o[a] < mu_o + 0.1
            np.testing.assert_allclose(lam[a][occ], lam_o[a][occ], rtol=0, atol=1e-4)
        assert abs(eb - eb_o) / n_at < 1e-5 and abs(es - es_o) / n_at < 1e-5
        assert relerr(rho, rho_o.ravel()) < 1e-4


def test_carry_mode_rejects_what_it_cannot_do():
    w = dirichlet_cell()
    V = pseudo.local_potential(w)
    with xls.Grid(w, xls.XLS_FP64, hbm_budget_bytes=(1 << 26) + 20 * (1 << 20)) as g:
        g.set_hamiltonian(V)
        with pytest.raises(xls.XlsError) as e:
            xls.xls_wave_carry(g.h, 3)                   # does not divide 8
        assert e.value.status == xls.XLS_EINVAL
        xls.xls_wave_carry(g.h, 2)
        with pytest.raises(xls.XlsError) as e:
            xls.xls_orbitals_set(g.h, 0, np.zeros((16, 18 ** 3)))
        assert e.value.status == xls.XLS_EINVAL
        xls.xls_orbitals_random(g.h, w.psi_seed)
        with pytest.raises(xls.XlsError):
            xls.xls_chefsi_wave(g.h, 5, w.degree, 1)     # only four waves
    u = dirichlet_cell()
    u.n_states = np.array([16, 16, 16, 16, 16, 16, 16, 24])
    with xls.Grid(u, xls.XLS_FP64, hbm_budget_bytes=(1 << 26) + 20 * (1 << 20)) as g:
        with pytest.raises(xls.XlsError) as e:
            xls.xls_wave_carry(g.h, 2)                   # unequal shapes
        assert e.value.status == xls.XLS_EINVAL
