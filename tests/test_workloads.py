"""The synthetic workloads' construction (seeded geometry and partitions; no method arithmetic)."""
import numpy as np

import synth


def test_uneven_workload_construction():
    """4,096 diamond sites of 8^3 cells with 2 % of them vacant (82, rounded half up), every
    subdomain a 1-cell core with a buffer of 12, 18 or 24 points (48^3, 60^3, 72^3 subdomains), state
    counts multiples of 16 that hold 1.2 times the electrons of the atoms inside each subdomain."""
    w = synth.workload(2)
    assert w.n_sub == 512 and len(w.pos) == 4096 - 82
    assert set(int(b) for b in w.buf[:, 0]) == {12, 18, 24}
    assert set(int(w.sub_size(a)[0]) for a in range(w.n_sub)) == {48, 60, 72}
    for a in range(0, w.n_sub, 37):
        start = w.core_lo[a] - w.buf[a]
        n_in = len(synth.near_atoms(w, start, w.sub_size(a), 0.0))
        ns = int(w.n_states[a])
        assert ns % 16 == 0 and 2 * ns >= 1.2 * 4 * n_in > 2 * (ns - 16)
    lit = synth.workload(2, consistent=False)
    assert set(lit.n_states.tolist()) == {80, 160, 240}
    assert np.array_equal([{12: 80, 18: 160, 24: 240}[int(b)] for b in lit.buf[:, 0]], lit.n_states)
