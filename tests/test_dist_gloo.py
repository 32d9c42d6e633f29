"""Host side of the multi-rank path on CPU ranks (gloo, world size 2): the distributed Fermi level
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
