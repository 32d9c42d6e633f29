"""The allocation-free Gram entry point (xls_gram_noalloc) against the library's regular Gram
and against the oracle's projection (Sec. 5.A.3 step (2)) of the same block.

Callers that cannot let a library allocate device memory (applications whose device memory
belongs to their own pool allocator, latency-critical loops that cannot take cudaMalloc's
implicit synchronisation) use xls_gram_noalloc; its scratch is a fixed array inside the
library.  This file is collected last on purpose: it must pass on its own in a fresh process
and after every other test, and two calls in a row must not see each other's scratch.
"""
import os

import numpy as np
import pytest

import synth
from oracle import chefsi, dc, pseudo
from paper_2609_13115_gb300 import xls

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_gram_noalloc_matches_regular_gram_twice():
    import torch
    from paper_2609_13115_gb300 import build
    if not os.path.exists(xls.LIB_PATH):
        build.build()
    xls.load()
    w = synth.workload(0)                       # 24^3 periodic cell, 24 states
    V = pseudo.local_potential(w)
    sub = dc.partition(w)[0]
    ns = int(w.n_states[0])
    psi0 = synth.psi0_block(w.psi_seed, sub.N, ns)
    bounds = np.array([[70.0, 9.0, -0.3]])
    with xls.Grid(w, xls.XLS_MIXED_BF16) as g:
        g.set_hamiltonian(V)
        xls.xls_orbitals_set(g.h, 0, psi0)
        xls.xls_chefsi_stage(g.h, 1, w.degree, bounds)       # block becomes Psi_f
        xls.xls_chefsi_stage(g.h, 2, w.degree)               # regular Gram of Psi_f
        Ms_ref, Hs_ref = xls.xls_get_subspace(g.h, 0, ns)
        F = xls.xls_orbitals_get(g.h, 0, np.zeros((ns, sub.N)))
        HF = np.zeros_like(F)
        xls.xls_hamiltonian_apply(g.h, 0, F, HF)             # same FP32 H Psi_f as the pass
    Ft = torch.tensor(F, dtype=torch.float32, device="cuda")
    HFt = torch.tensor(HF, dtype=torch.float32, device="cuda")
    # first call: the whole block
    Ms = torch.zeros((ns, ns), dtype=torch.float64, device="cuda")
    Hs = torch.zeros_like(Ms)
    xls.xls_gram_noalloc(Ft, HFt, Ms, Hs)
    torch.cuda.synchronize()
    assert _relerr(Ms.cpu().numpy(), Ms_ref) < 1e-6
    assert _relerr(Hs.cpu().numpy(), Hs_ref) < 1e-6
    # second call in a row: a smaller block (the first 16 vectors) reuses the same scratch
    k = 16
    Ms2 = torch.full((k, k), float("nan"), dtype=torch.float64, device="cuda")
    Hs2 = torch.full((k, k), float("nan"), dtype=torch.float64, device="cuda")
    xls.xls_gram_noalloc(Ft[:k].contiguous(), HFt[:k].contiguous(), Ms2, Hs2)
    torch.cuda.synchronize()
    assert _relerr(Ms2.cpu().numpy(), Ms_ref[:k, :k]) < 1e-6
    assert _relerr(Hs2.cpu().numpy(), Hs_ref[:k, :k]) < 1e-6


def test_gram_noalloc_rejects_oversized_block():
    import torch
    xls.load()
    F = torch.zeros((300, 64), dtype=torch.float32, device="cuda")
    M = torch.zeros((300, 300), dtype=torch.float64, device="cuda")
    with pytest.raises(xls.XlsError) as e:
        xls.xls_gram_noalloc(F, F, M, M)
    assert e.value.status == xls.XLS_EINVAL


class _DiagonalOperator:
    """H = diag(d): H Psi_f scales every grid value, so F (H F)^T is symmetric like the pass's."""

    def __init__(self, d):
        self.d = d
        self.N = d.size

    def apply(self, X):
        return X * self.d[None, :]


@pytest.mark.parametrize("n_states", [200, 256])
def test_gram_noalloc_two_blocks_ragged_tail_matches_oracle(n_states):
    """Two 128-state blocks (three block pairs, 21 K chunks of uneven length) and a ragged last
    K tile (n_points = 64 m + 8), against the oracle's FP64 projection of the same FP32 block;
    two calls in a row (the second on a shorter block) share the fixed scratch."""
    import torch
    xls.load()
    n_points = 64 * 300 + 8
    F = synth.uniform_pm_half(4242 + n_states, n_states * n_points).reshape(n_states, n_points)
    F = F.astype(np.float32).astype(np.float64)               # the FP32 block both sides see
    d = (1.0 + synth.uniform_pm_half(77, n_points)).astype(np.float32).astype(np.float64)
    H = _DiagonalOperator(d)
    HF = H.apply(F).astype(np.float32).astype(np.float64)
    Ms_o, Hs_o = chefsi.projection(H, F)     # FP64 (the FP32 rounding of HF is far below the bound)
    Ft = torch.tensor(F, dtype=torch.float32, device="cuda")
    HFt = torch.tensor(HF, dtype=torch.float32, device="cuda")
    for rows in (n_states, n_states - 72):                    # second call: one block + a partial one
        Ms = torch.full((rows, rows), float("nan"), dtype=torch.float64, device="cuda")
        Hs = torch.full_like(Ms, float("nan"))
        xls.xls_gram_noalloc(Ft[:rows].contiguous(), HFt[:rows].contiguous(), Ms, Hs)
        torch.cuda.synchronize()
        # split-BF16 products (about 16 significant bits per operand) summed in FP32 partial sums
        assert _relerr(Ms.cpu().numpy(), Ms_o[:rows, :rows]) < 2e-5
        assert _relerr(Hs.cpu().numpy(), Hs_o[:rows, :rows]) < 2e-5


def test_gram_noalloc_checks_tensor_arguments():
    import torch
    xls.load()
    F = torch.zeros((16, 64), dtype=torch.float32, device="cuda")
    M = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        xls.xls_gram_noalloc(F, F, M.float(), M)
    with pytest.raises(ValueError):
        xls.xls_gram_noalloc(F, F[:8].contiguous(), M, M)
    with pytest.raises(ValueError):
        xls.xls_gram_noalloc(F, F, M[:8, :8].contiguous(), M)
