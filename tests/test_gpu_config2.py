"""The uneven-subdomain workload (vacancies, 1-cell cores with 0.5-, 0.75- or 1-cell buffers, so
48^3, 60^3 and 72^3 subdomains with their own state counts in the same launches; Sec. 5.A.5
"Parallel CheFSI") against the oracle on a sample of its subdomains, on the 512-site crystal of the
same construction (4^3 cells, 64 subdomains, all with Dirichlet buffers)."""
import numpy as np
import pytest

import synth
from oracle import chefsi, dc
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


def sample_by_width(w, per_width=1):
    """The first `per_width` subdomains of each buffer width."""
    out = []
    for width in sorted(set(int(b) for b in w.buf[:, 0])):
        out += [a for a in range(w.n_sub) if int(w.buf[a][0]) == width][:per_width]
    return out


@pytest.mark.parametrize("prec", [xls.XLS_FP64, xls.XLS_MIXED_FP16])
def test_uneven_subdomains_match_oracle(prec):
    """All 64 subdomains (three sizes, 16 states each) in the same launches: H on two vectors of a
    subdomain of each size against the oracle's operator; one pass (Lanczos bound, Rayleigh-Ritz of
    the start block, filter, projection, eigensolve, rotation) from the SplitMix64 start, Ritz values
    of a subdomain of each size against the oracle's pass."""
    w = synth.workload(2, ncell=4)
    w.n_states = np.full(w.n_sub, 16)
    V = synth.veff_erf_wells(w)
    subs = dc.partition(w)
    sample = sample_by_width(w)
    ops = {a: dc.subdomain_operator_local(w, subs[a], V) for a in sample}
    with xls.Grid(w, prec) as g:
        g.set_hamiltonian(V)
        for a in sample:
            x = synth.psi0_block(91 + a, subs[a].N, 2)
            y = np.zeros_like(x)
            xls.xls_hamiltonian_apply(g.h, a, x, y)
            assert relerr(y, ops[a].apply(x)) < (1e-12 if prec == xls.XLS_FP64 else 2e-6), a
        xls.xls_orbitals_random(g.h, w.psi_seed)
        xls.xls_chefsi_batch(g.h, w.degree, 1)
        lam = {a: xls.xls_get_eigs(g.h, a, 16)[0] for a in sample}
    offs = synth.psi0_offsets(w)
    for a in sample:
        H = ops[a]
        psi0 = synth.psi0_block(w.psi_seed, subs[a].N, 16, offs[a])
        lam_o, _, _ = chefsi.run_chefsi(H, psi0, w.degree, 1, v0=synth.lanczos_start(H.N))
        tol = 1e-8 if prec == xls.XLS_FP64 else 1e-4
        np.testing.assert_allclose(lam[a], lam_o, rtol=0, atol=tol * max(1.0, np.abs(lam_o).max()))
