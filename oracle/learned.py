"""Learned SCF start (Sec. 5.A.4, SCF initialisation: a superposition of atomic densities plus a
material-specific learned correction).

Test infrastructure only: plain numpy.

Readings (the paper names the idea, not the model):
  * SAD: per atom a normalised Gaussian of Z_v electrons with the width of the species' erf
    radius, rho_I(r) = Z_v pi^-3/2 r_c^-3 exp(-r^2 / r_c^2), periodic images summed, the total
    renormalised on the grid to N_e;
  * descriptors: per species s and k = 0..15, d_{s,k}(x) = sum_{I in s} exp(-(r_I - r_k)^2 /
    (2 * 0.25^2)) f_c(r_I), r_k = k * 6/15 bohr, f_c(r) = (cos(pi r / 6) + 1) / 2 for r < 6 bohr,
    else 0; r_I the minimum-image distance (cells wider than 12 bohr);
  * model: 32 -> 64 -> 64 -> 64 -> 1, tanh on the hidden layers, linear output; parameters
    flattened as W1 (32x64, row = input), b1, W2 (64x64), b2, W3 (64x64), b3, w4 (64), b4;
  * training: mean squared error over points, Adam (beta1 0.9, beta2 0.999, eps 1e-8);
  * start density: rho_0 = max(rho_SAD + MLP(d), 0), renormalised to N_e.
"""
from __future__ import annotations

import math

import numpy as np

N_RADIAL = 16
R_CUT = 6.0
SIGMA = 0.25
LAYERS = [(32, 64), (64, 64), (64, 64), (64, 1)]
N_PARAMS = sum(i * o + o for i, o in LAYERS)


def radial_centres() -> np.ndarray:
    return np.arange(N_RADIAL) * (R_CUT / (N_RADIAL - 1))


def cutoff(r: np.ndarray) -> np.ndarray:
    return np.where(r < R_CUT, 0.5 * (np.cos(math.pi * r / R_CUT) + 1.0), 0.0)


def grid_points(w) -> np.ndarray:
    """Cartesian coordinates (N, 3) of the global grid, flat index x fastest."""
    n = np.asarray(w.n)
    h = np.asarray(w.h)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return np.stack([i.ravel() * h[0], j.ravel() * h[1], k.ravel() * h[2]], axis=1)


def descriptors(w, points: np.ndarray | None = None, n_species: int = 2) -> np.ndarray:
    """(N, n_species * 16): species-major, radial index minor."""
    x = grid_points(w) if points is None else np.asarray(points, dtype=np.float64)
    L = np.asarray(w.L, dtype=np.float64)
    rk = radial_centres()
    D = np.zeros((len(x), n_species * N_RADIAL))
    for I, R in enumerate(np.asarray(w.pos)):
        s = w.species_index[I]
        d = x - R
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(axis=1))
        m = r < R_CUT
        fc = cutoff(r[m])
        D[np.ix_(m, range(s * N_RADIAL, (s + 1) * N_RADIAL))] += (
            np.exp(-((r[m, None] - rk[None, :]) ** 2) / (2.0 * SIGMA * SIGMA)) * fc[:, None])
    return D


def sad_density(w) -> np.ndarray:
    """Superposition of atomic Gaussian densities on the grid (nz, ny, nx), sum dV = N_e."""
    n = np.asarray(w.n)
    h = np.asarray(w.h)
    L = np.asarray(w.L, dtype=np.float64)
    rho = np.zeros((n[2], n[1], n[0]))
    for I, R in enumerate(np.asarray(w.pos)):
        sp = w.species[w.species_index[I]]
        rc = sp.rc_loc
        g1 = []
        for d in range(3):
            x = np.arange(n[d]) * h[d]
            kmax = int(math.ceil(12.0 * rc / L[d])) + 1
            g1.append(sum(np.exp(-((x - R[d] - k * L[d]) ** 2) / rc ** 2) for k in range(-kmax, kmax + 1)))
        rho += sp.Zv * math.pi ** -1.5 * rc ** -3 * np.einsum("k,j,i->kji", g1[2], g1[1], g1[0])
    return rho * (w.n_electrons / (rho.sum() * float(np.prod(h))))


def unpack(theta: np.ndarray) -> list:
    """[(W, b)] per layer from the flat parameter vector."""
    out, o = [], 0
    for i, j in LAYERS:
        W = theta[o:o + i * j].reshape(i, j)
        o += i * j
        b = theta[o:o + j]
        o += j
        out.append((W, b))
    return out


def forward(theta: np.ndarray, X: np.ndarray, keep: bool = False):
    """MLP output (N,); with keep, also the hidden activations."""
    acts = [X]
    h = X
    layers = unpack(theta)
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        h = np.tanh(z) if li < len(layers) - 1 else z
        acts.append(h)
    y = h[:, 0]
    return (y, acts) if keep else y


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) and back to float64, through the float32 bits."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def forward_bf16(theta: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Inference with BF16 operands (inputs, weights, hidden activations rounded to BF16), exact
    accumulation; biases and the output layer's accumulation in full precision."""
    h = bf16(X)
    layers = unpack(theta)
    for li, (W, b) in enumerate(layers):
        z = h @ bf16(W) + b
        h = bf16(np.tanh(z)) if li < len(layers) - 1 else z
    return h[:, 0]


def loss_and_grad(theta: np.ndarray, X: np.ndarray, y: np.ndarray):
    """Mean squared error and its gradient by backpropagation."""
    yp, acts = forward(theta, X, keep=True)
    n = len(y)
    loss = float(np.mean((yp - y) ** 2))
    layers = unpack(theta)
    grads = []
    delta = (2.0 / n) * (yp - y)[:, None]                     # dL/dz of the output layer
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        a_in = acts[li]
        grads.append((a_in.T @ delta, delta.sum(axis=0)))
        if li > 0:
            delta = (delta @ W.T) * (1.0 - acts[li] ** 2)      # through tanh of layer li - 1
    grads.reverse()
    return loss, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


class Adam:
    def __init__(self, n: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def learned_start(w, theta: np.ndarray, n_species: int = 2) -> np.ndarray:
    """rho_0 = max(rho_SAD + MLP(d), 0) renormalised to N_e (BF16 inference)."""
    n = np.asarray(w.n)
    sad = sad_density(w)
    corr = forward_bf16(theta, descriptors(w, n_species=n_species)).reshape(n[2], n[1], n[0])
    rho = np.maximum(sad + corr, 0.0)
    return rho * (w.n_electrons / (rho.sum() * float(np.prod(w.h))))
