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


def test_64_atom_and_13824_atom_workload_construction():
    """The 64-atom cell: 2^3 cells (48^3 grid), 8 periodic subdomains of 48^3 whose 0.5-cell buffers
    cover the cell, 160 (consistent) or 80 (literal) states.  The 13,824-atom cell: 12^3 cells
    (288^3 grid), 1,728 Dirichlet subdomains of 72^3 (1-cell core and buffer), 528 (consistent) or
    240 (literal) states; its cores tile the grid exactly once."""
    w1 = synth.workload(1)
    assert len(w1.pos) == 64 and tuple(w1.n) == (48, 48, 48) and w1.n_sub == 8
    assert all(tuple(w1.sub_size(a)) == (48, 48, 48) for a in range(w1.n_sub))
    assert set(w1.n_states.tolist()) == {160}
    assert set(synth.workload(1, consistent=False).n_states.tolist()) == {80}
    w3 = synth.workload(3)
    assert len(w3.pos) == 13824 and tuple(w3.n) == (288, 288, 288) and w3.n_sub == 1728
    assert set(int(x) for x in w3.buf.ravel()) == {24} and set(int(x) for x in w3.core_n.ravel()) == {24}
    assert set(w3.n_states.tolist()) == {528}
    assert set(synth.workload(3, consistent=False).n_states.tolist()) == {240}
    cover = np.zeros(w3.n, dtype=np.int32)
    for a in range(w3.n_sub):
        x0, y0, z0 = (int(v) for v in w3.core_lo[a])
        cx, cy, cz = (int(v) for v in w3.core_n[a])
        cover[x0:x0 + cx, y0:y0 + cy, z0:z0 + cz] += 1
    assert cover.min() == 1 and cover.max() == 1
