"""Fermi level of states spread over ranks (Sec. 5.A.5, "Chemical potential").

Every rank holds the Ritz values and core weights of its own subdomains on its GPU; the
electron count N_e(mu) = 2 sum c g((lambda - mu)/kT) is a sum over all of them.  The paper
narrows the bracket with a histogram of the eigenvalues and then takes Newton steps on N_e(mu)
using dN_e/dmu, so that each step needs the global sum of two scalars.  This module is the host
side of that scheme: the per-rank sums come from the GPU (`xls_fermi_partial`,
`xls_fermi_histogram`), the combination across ranks is an allreduce of `torch.distributed`
(NCCL between GPUs, gloo on the host), and the bracket / Newton bookkeeping is scalar host logic.

`partial(mu)` returns this rank's [N_e, dN_e/dmu, min lambda, max lambda];
`histogram(lo, hi, n_bins)` this rank's weighted counts per bin.  Without a process group the
functions work on the local sums alone.
"""
from __future__ import annotations

import numpy as np


def _allreduce(x: np.ndarray, op: str, group=None) -> np.ndarray:
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return x
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    rop = {"sum": dist.ReduceOp.SUM, "min": dist.ReduceOp.MIN, "max": dist.ReduceOp.MAX}[op]
    dist.all_reduce(t, op=rop, group=group)
    return t.cpu().numpy()


def fermi_level(partial, histogram, n_electrons: float, kT: float, group=None, n_bins: int = 256,
                tol: float = 1e-14, max_iter: int = 200):
    """mu with sum over all ranks of N_e(mu) = n_electrons, and the number of allreduces used.

    1. bracket: global min / max of lambda, widened by 1 Ha (one allreduce each);
    2. histogram of 2c over n_bins bins of the bracket, summed over ranks (one allreduce): the
       bin whose cumulative count crosses n_electrons, widened by 40 kT on both sides (where the
       Fermi function has reached e^-40), becomes the bracket when it holds the root;
    3. Newton steps mu <- mu - (N_e - n_electrons) / N_e', two scalars summed per step, kept
       inside the bracket (bisection when a step leaves it), until the bracket is below tol.
    """
    loc = partial(0.0)
    lo = float(_allreduce(np.array([loc[2]]), "min", group)[0]) - 1.0
    hi = float(_allreduce(np.array([loc[3]]), "max", group)[0]) + 1.0
    n_red = 2
    hist = _allreduce(np.asarray(histogram(lo, hi, n_bins), dtype=np.float64), "sum", group)
    n_red += 1
    cum = np.cumsum(hist)
    b = int(np.searchsorted(cum, n_electrons))
    w = (hi - lo) / n_bins
    cand_lo, cand_hi = lo + max(b - 1, 0) * w - 40 * kT, lo + min(b + 2, n_bins) * w + 40 * kT

    def count(mu):
        nonlocal n_red
        n_red += 1
        v = _allreduce(np.asarray(partial(mu)[:2], dtype=np.float64), "sum", group)
        return float(v[0]), float(v[1])

    n_lo, _ = count(max(cand_lo, lo))
    n_hi, _ = count(min(cand_hi, hi))
    if n_lo <= n_electrons <= n_hi:
        lo, hi = max(cand_lo, lo), min(cand_hi, hi)
    else:
        n_lo, _ = count(lo)
        n_hi, _ = count(hi)
        if not (n_lo <= n_electrons <= n_hi):
            raise ValueError("Fermi level not bracketed: N_e exceeds the states' capacity")
    mu = 0.5 * (lo + hi)
    for _ in range(max_iter):
        nm, dn = count(mu)
        if nm < n_electrons:
            lo = mu
        else:
            hi = mu
        if nm == n_electrons or hi - lo <= tol:
            break
        nxt = mu - (nm - n_electrons) / dn if dn > 0 else 0.5 * (lo + hi)
        if not (lo < nxt < hi):
            nxt = 0.5 * (lo + hi)
        if abs(nxt - mu) <= 1e-15 * max(1.0, abs(mu)):
            mu = nxt
            break
        mu = nxt
    return mu, n_red


def grid_fermi_level(g, n_electrons: float, kT: float, group=None, n_bins: int = 256):
    """fermi_level over the ranks' grids (`g` a grid handle of the binding on this rank)."""
    from . import xls
    return fermi_level(lambda mu: xls.xls_fermi_partial(g, mu, kT),
                       lambda lo, hi, nb: xls.xls_fermi_histogram(g, lo, hi, nb),
                       n_electrons, kT, group, n_bins)


def assemble_cores(local: np.ndarray, group=None) -> np.ndarray:
    """A global-grid field of which every rank filled the points of its own subdomain cores (the
    cores tile the grid once, Sec. 5.A.2), the other points 0: the sum over ranks is the field.
    Used for the density after xls_density_at and for the effective potential each rank needs
    for the restriction to its subdomains (one allreduce of the grid; at these cell sizes it
    replaces a halo exchange of the buffer regions)."""
    return _allreduce(np.asarray(local, dtype=np.float64), "sum", group)
