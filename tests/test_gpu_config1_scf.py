"""The 64-atom D&C SCF at its stated size (2 x 2 x 2 Si cells, 48^3 global grid, 8 periodic
subdomains of 48^3 with 160 states, degree 20, LDA, Pulay + Kerker; Sec. 5.A.4 and Sec. 5.A.5) run to
a density residual of 1e-6 on the FP64 path and on the mixed path from the same start, and the two
converged states compared.  The single SCF step of this solver is checked against the oracle on
the smaller Dirichlet cell (test_gpu_bench_size.py); the oracle's own SCF at this size takes hours."""
import numpy as np
import pytest

import synth
from oracle import pseudo
from paper_2609_13115_gb300 import xls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2609_13115_gb300 import build
    if not os.path.exists(xls.LIB_PATH):
        build.build()
    xls.load()


def scf_to(w, prec, tol, max_steps):
    """SCF steps from the neutral start density and the seeded random blocks (four passes in the
    first step, then two; Pulay every step) until the residual is below tol."""
    b = pseudo.pseudocharge(w)
    rho = np.ascontiguousarray((w.n_electrons / (int(np.prod(w.n)) * float(np.prod(w.h))) - b).ravel())
    hist = []
    with xls.Grid(w, prec) as g:
        g.set_hamiltonian(pseudo.local_potential(w))
        xls.xls_orbitals_random(g.h, w.psi_seed)
        xls.xls_scf_setup(g.h, w.n_electrons, w.kT, w.degree, n_passes=4, pulay_period=1)
        for k in range(max_steps):
            hist.append(xls.xls_scf_step(g.h, rho))
            if k == 0:
                xls.xls_scf_setup(g.h, w.n_electrons, w.kT, w.degree, n_passes=2, pulay_period=1)
            if hist[-1][0] < tol:
                break
    return hist, rho


def test_config1_scf_converges_on_both_paths():
    """Measured: FP64 26 steps to 8.3e-7 (34.5 s), mixed 38 steps to 7.4e-7 (3.0 s); the residual
    stalls near 1e-5 for a few steps on both paths before Pulay resumes; converged energies 2.3e-7
    Ha/atom and densities 5e-6 apart."""
    w = synth.workload(1)
    n_at = len(w.pos)
    h64, r64 = scf_to(w, xls.XLS_FP64, 1e-6, 45)
    hm, rm = scf_to(w, xls.XLS_MIXED_FP16, 1e-6, 70)
    assert h64[-1][0] < 1e-6, [f"{h[0]:.1e}" for h in h64]
    assert hm[-1][0] < 1e-6, [f"{h[0]:.1e}" for h in hm]
    assert abs(h64[-1][1] - hm[-1][1]) / n_at < 1e-5
    assert abs(h64[-1][2] - hm[-1][2]) < 1e-4
    assert np.linalg.norm(rm - r64) / np.linalg.norm(r64) < 1e-4
    dV = float(np.prod(w.h))
    assert abs(r64.sum() * dV - w.n_electrons) < 1e-6 * w.n_electrons
