"""Pins of the learned-start oracle: backpropagation against finite differences, Adam's first
step, descriptors and the atomic density against their closed forms on single atoms, and the
BF16 rounding against known values."""
import math

import numpy as np
import pytest

import synth
from oracle import learned


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    theta = synth.mlp_init(77) + 0.05 * rng.standard_normal(learned.N_PARAMS)
    X = rng.standard_normal((40, 32)) * 0.7
    y = rng.standard_normal(40) * 0.3
    loss, g = learned.loss_and_grad(theta, X, y)
    idx = rng.choice(learned.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [learned.N_PARAMS - 1, 32 * 64, 32 * 64 + 64]])   # b4, b1[0], W2[0,0]
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = 1e-6
        fd = (learned.loss_and_grad(theta + e, X, y)[0] - learned.loss_and_grad(theta - e, X, y)[0]) / 2e-6
        assert abs(fd - g[i]) < 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])
    assert abs(loss - np.mean((learned.forward(theta, X) - y) ** 2)) < 1e-15


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    opt = learned.Adam(50, lr=1e-3)
    new = opt.step(theta, g)
    # up to eps / |g| (eps = 1e-8)
    np.testing.assert_allclose(new - theta, -1e-3 * np.sign(g), rtol=1e-8 / np.abs(g).min() + 1e-12)


def test_descriptors_single_atom_closed_form():
    w = synth.workload(0)
    w2 = synth.Workload("one", w.L, w.n, np.array([[1.0, 2.0, 3.0]]), np.array([1]), [w.species[0], synth.SPECIES_B],
                        w.core_lo, w.core_n, w.buf, w.n_states, w.degree, w.n_passes, w.psi_seed)
    rk = np.arange(16) * 0.4
    pts = np.array([[1.0, 2.0, 3.0], [1.0 + 0.8, 2.0, 3.0], [1.0, 2.0 - 3.3, 3.0], [1.0 + 6.5, 2.0, 3.0],
                    [1.0 + w.L[0], 2.0, 3.0 + 2.0]])
    D = learned.descriptors(w2, pts)
    assert np.all(D[:, :16] == 0.0)
    for p, r in zip(pts, [0.0, 0.8, 3.3, None, 2.0]):
        row = D[list(map(tuple, pts)).index(tuple(p)), 16:]
        if r is None:                     # beyond the cutoff (6.5 bohr; the image is 3.76 away)
            r = w.L[0] - 6.5
        ref = np.exp(-((r - rk) ** 2) / (2 * 0.25 ** 2)) * 0.5 * (math.cos(math.pi * r / 6.0) + 1.0)
        np.testing.assert_allclose(row, ref, rtol=1e-12, atol=1e-300)


def test_descriptor_cutoff_is_smooth_and_zero_outside():
    assert learned.cutoff(np.array([6.0, 7.0]))[0] == 0.0
    r = np.array([5.999999])
    assert learned.cutoff(r)[0] < 1e-10


def test_sad_matches_gaussian_and_normalisation():
    """One atom in a cell much wider than r_c: the grid sum of the Gaussian equals its integral
    (Poisson summation error exp(-pi^2 r_c^2 / h^2)), so no renormalisation is visible and the
    values are Z pi^-3/2 r_c^-3 exp(-r^2/r_c^2)."""
    w = synth.workload(0)
    R = np.array([[w.L[0] / 2, w.L[1] / 2, w.L[2] / 2]])
    w1 = synth.Workload("one", w.L, w.n, R, np.array([0]), [w.species[0]], w.core_lo, w.core_n, w.buf,
                        w.n_states, w.degree, w.n_passes, w.psi_seed)
    rho = learned.sad_density(w1)
    assert abs(rho.sum() * np.prod(w1.h) - 4.0) < 1e-12
    Z, rc = 4.0, w.species[0].rc_loc
    c = np.array(w.n) // 2
    h = w1.h
    for di in [(0, 0, 0), (1, 0, 0), (2, 1, 0), (3, 2, 1)]:
        r2 = sum((di[d] * h[d]) ** 2 for d in range(3))
        val = rho[c[2] + di[2], c[1] + di[1], c[0] + di[0]]
        assert abs(val - Z * math.pi ** -1.5 * rc ** -3 * math.exp(-r2 / rc ** 2)) < 1e-9


def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, math.pi, -2.5, 0.0])
    ref = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 3.140625, -2.5, 0.0])
    np.testing.assert_array_equal(learned.bf16(vals), ref)


def test_learned_start_normalised_and_nonnegative():
    w = synth.two_species(synth.workload(0), [0])
    theta = synth.mlp_init(5) * 0.1
    rho = learned.learned_start(w, theta)
    assert rho.min() >= 0.0
    assert abs(rho.sum() * np.prod(w.h) - w.n_electrons) < 1e-9
    # an output bias that drives the correction below the atomic density in the interstitial:
    # there the start density is clipped to zero, elsewhere it is proportional to SAD + MLP
    theta[-1] = -0.5 * float(learned.sad_density(w).mean())
    rho = learned.learned_start(w, theta).ravel()
    raw = learned.sad_density(w).ravel() + learned.forward_bf16(theta, learned.descriptors(w))
    assert (raw < 0).any() and (raw > 0).any()
    assert np.all(rho[raw <= 0] == 0.0) and rho.min() >= 0.0
    ratio = rho[raw > 0] / raw[raw > 0]
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-12)
    assert abs(rho.sum() * np.prod(w.h) - w.n_electrons) < 1e-9


def test_bf16_inference_within_rounding_of_full_precision():
    """BF16 operands (unit roundoff 2^-9) on the four layers put the inference within a few per
    mille of the FP64 forward pass and not equal to it: no rounding at all, a dropped bias, a
    transposed weight or a missing tanh moves it out of that band."""
    rng = np.random.default_rng(12)
    theta = synth.mlp_init(31) + 0.05 * rng.standard_normal(learned.N_PARAMS)   # biases nonzero too
    X = rng.standard_normal((400, 32))
    y64 = learned.forward(theta, X)
    y16 = learned.forward_bf16(theta, X)
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-4 < rel < 2e-2, rel
