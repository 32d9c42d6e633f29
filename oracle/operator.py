"""The subdomain Kohn-Sham Hamiltonian H^alpha (Eq. ks restricted to Omega^alpha, Sec. 5.A.2):
H = -1/2 Delta_h + diag(V) + sum_I sum_l E_l dV chi_Il chi_Il^T, matrix-free, on a
(nx, ny, nz) grid with Dirichlet-zero or periodic boundaries per axis.

Vectors are rows: a block Y has shape (k, N_d) with N_d = nx*ny*nz, x fastest."""
from __future__ import annotations

import numpy as np

from . import fd


class SubdomainHamiltonian:
    def __init__(self, size, h, periodic, V, projectors, n0: int = fd.N0):
        self.size = tuple(int(s) for s in size)              # (nx, ny, nz)
        self.shape = (self.size[2], self.size[1], self.size[0])
        self.N = int(np.prod(self.size))
        self.h = tuple(float(x) for x in h)
        self.dV = float(np.prod(self.h))
        self.periodic = tuple(bool(p) for p in periodic)
        self.V = np.asarray(V, dtype=np.float64).reshape(self.shape)
        self.projectors = projectors
        self.n0 = n0

    def apply_local(self, Y: np.ndarray) -> np.ndarray:
        k = Y.shape[0]
        Yg = Y.reshape((k,) + self.shape)
        out = -0.5 * fd.laplacian(Yg, self.h, self.periodic, self.n0) + self.V * Yg
        return out.reshape(k, self.N)

    def apply_nonlocal(self, Y: np.ndarray) -> np.ndarray:
        out = np.zeros_like(Y)
        for flat, chi, E in self.projectors:
            P = (Y[:, flat] @ chi.T) * self.dV            # <chi_l|psi> for each row, (k, 4)
            out[:, flat] += (P * E) @ chi
        return out

    def apply(self, Y: np.ndarray) -> np.ndarray:
        Y = np.atleast_2d(Y)
        return self.apply_local(Y) + self.apply_nonlocal(Y)

    def dense(self) -> np.ndarray:
        """H as an (N, N) matrix, column j = H e_j (tiny grids only)."""
        return self.apply(np.eye(self.N)).T
