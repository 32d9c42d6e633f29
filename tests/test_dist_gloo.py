"""Host side of the multi-rank path on CPU ranks (gloo, world sizes 2 and 4): the distributed Fermi level
(histogram + Newton with allreduces, Sec. 5.A.5) against the oracle's bisection on the union of
all states, and the assembly of core-owned grid fields."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import fermi
        from paper_2609_13115_gb300 import dist as xd
        rng = np.random.default_rng(17)
        lam = np.sort(rng.uniform(-0.4, 0.9, 400))
        c = rng.uniform(0.0, 1.0, 400)
        mine = slice(rank * 200, (rank + 1) * 200)
        kT, ne = 0.01, 2.0 * 0.55 * c.sum()
        lam_r, c_r = lam[mine], c[mine]

        def partial(mu):
            g = fermi.occupations(lam_r, mu, kT)
            return np.array([2.0 * np.sum(c_r * g), 2.0 * np.sum(c_r * g * (1 - g)) / kT, lam_r.min(), lam_r.max()])

        def histogram(lo, hi, nb):
            b = np.clip(np.floor((lam_r - lo) / (hi - lo) * nb).astype(int), 0, nb - 1)
            return np.bincount(b, weights=2.0 * c_r, minlength=nb)

        mu, n_red = xd.fermi_level(partial, histogram, ne, kT)
        ref = fermi.fermi_level(lam, c, kT, ne)
        # a core-owned field: rank r owns the points with (index % 2 == r)
        n = 1000
        full = np.sin(np.arange(n) * 0.1)
        local = np.where(np.arange(n) % world == rank, full, 0.0)
        field = xd.assemble_cores(local)
        q.put((rank, mu, ref, n_red, float(np.abs(field - full).max())))
    finally:
        dist.destroy_process_group()


def test_distributed_fermi_level_and_core_assembly():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = [q.get() for _ in range(2)]
    for rank, mu, ref, n_red, ferr in res:
        assert abs(mu - ref) < 1e-12, (rank, mu, ref)
        assert n_red <= 14, n_red            # histogram + a few Newton steps, not 50 bisection steps
        assert ferr == 0.0
    assert res[0][1] == res[1][1]            # every rank ends with the same mu


def _partition_worker(rank, world, port, q):
    """Rank `rank` owns every world-th subdomain of the eight-subdomain Dirichlet cell: it runs the
    oracle's passes on its own subdomains only, takes part in the distributed Fermi level, forms
    the densities of its own cores at that level and the grid field is assembled over ranks."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import dc, fermi, pseudo
        from paper_2609_13115_gb300 import dist as xd
        w = _dirichlet_cell()
        V = pseudo.local_potential(w)
        subs = dc.partition(w)
        mine = [a for a in range(w.n_sub) if a % world == rank]
        psi0 = [_start_block(w, subs, a) for a in mine]
        part = dc.run(w, V, psi0, subdomains=mine)
        lam_r, c_r = np.concatenate(part.lam), np.concatenate(part.c)

        def partial(mu):
            g = fermi.occupations(lam_r, mu, w.kT)
            return np.array([2.0 * np.sum(c_r * g), 2.0 * np.sum(c_r * g * (1 - g)) / w.kT, lam_r.min(), lam_r.max()])

        def histogram(lo, hi, nb):
            b = np.clip(np.floor((lam_r - lo) / (hi - lo) * nb).astype(int), 0, nb - 1)
            return np.bincount(b, weights=2.0 * c_r, minlength=nb)

        mu, _ = xd.fermi_level(partial, histogram, w.n_electrons, w.kT)
        n = np.asarray(w.n)
        dV = float(np.prod(w.h))
        local = np.zeros(int(np.prod(n)))
        for k, a in enumerate(mine):
            P = part.Psi[k]
            local[dc.core_global_indices(subs[a], n)] = fermi.point_density(
                P[:, dc.core_local_indices(subs[a])], fermi.occupations(part.lam[k], mu, w.kT), dV)
        rho = xd.assemble_cores(local)
        e_band = float(xd._allreduce(np.array([fermi.band_energy(lam_r, c_r, mu, w.kT)]), "sum")[0])
        q.put((rank, mu, rho, e_band))
    finally:
        dist.destroy_process_group()


def _dirichlet_cell():
    import synth
    w = synth.workload(0)
    cores = np.array([(i, j, k) for k in (0, 12) for j in (0, 12) for i in (0, 12)])
    return synth.Workload("si8_dc8_dirichlet", w.L, w.n, synth.displace(w.pos, 0.05, 77, w.L), w.species_index,
                          w.species, core_lo=cores, core_n=np.full((8, 3), 12), buf=np.full((8, 3), 3),
                          n_states=np.full(8, 16), degree=10, n_passes=3, psi_seed=55)


def _start_block(w, subs, a):
    import synth
    return synth.psi0_block(w.psi_seed + a, subs[a].N, int(w.n_states[a]))


@pytest.mark.parametrize("world", [2, 4])
def test_partitioned_subdomains_reproduce_single_process_run(world):
    """Two or four ranks, each owning every world-th subdomain, give the single-process oracle
    run's mu, density and band energy (the ranks exchange only the Fermi-level sums and the
    core-owned density field)."""
    import torch.multiprocessing as mp
    from oracle import dc, pseudo
    w = _dirichlet_cell()
    subs = dc.partition(w)
    ref = dc.run(w, pseudo.local_potential(w), [_start_block(w, subs, a) for a in range(w.n_sub)])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]   # read before joining: a full pipe blocks the put
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    for rank, mu, rho, e_band in res:
        assert abs(mu - ref.mu) < 1e-12, (rank, mu, ref.mu)
        assert np.abs(rho - ref.rho.ravel()).max() < 1e-12 * np.abs(ref.rho).max()
        assert abs(e_band - ref.e_band) < 1e-11 * abs(ref.e_band)
