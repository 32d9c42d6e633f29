"""Planted mistakes in the oracle, on the CPU.  Each mutant replaces one oracle function (or one
constant) with a variant carrying a single plausible error: a dropped term or factor, a flipped
sign, a wrong index, axis or spacing, a transposed operand, a missing normalisation.  The test
runs the pin that should notice it and asserts that the pin fails; a mutant no pin caught would
mark a gap in the pins.  The mutants cover the oracle module by module: finite differences, the
subdomain operator, electrostatics and projectors, the CheFSI steps, the Fermi level, density
and energies, the partition, the SCF pieces and the learned start.  Two kinds of change are left
out because they are no mistake: swapping the filter bounds a and b (C_m has the parity of m, so
the scaled filter is unchanged) and the direction of the stencil shifts (the weights are
symmetric).  The mutants live only inside this test (monkeypatch); the pins are the committed
ones of tests/test_oracle_*.py, called as they are."""
import copy
import dataclasses
import math

import numpy as np
import pytest
import scipy.linalg as sla

import test_oracle_chefsi as pc
import test_oracle_learned as pl
import test_oracle_operator as po
import test_oracle_scf as ps
from oracle import chefsi, dc, fd, fermi, learned, pseudo, scf
from oracle.operator import SubdomainHamiltonian

_orig = {}


def original(mod, name):
    key = (mod.__name__, name)
    if key not in _orig:
        _orig[key] = getattr(mod, name)
    return _orig[key]


# ---- finite differences (Sec. 5.B.2) ---------------------------------------------------------
def m_fd_weight_signs(mp):
    f = original(fd, "fd_weights_exact")
    mp.setattr(fd, "fd_weights_exact", lambda n0=fd.N0: [-x for x in f(n0)])


def m_fd_centre_weight(mp):
    f = original(fd, "fd_weights_exact")
    mp.setattr(fd, "fd_weights_exact", lambda n0=fd.N0: [-sum(f(n0)[1:])] + f(n0)[1:])


def m_fd_over_h(mp):
    f = original(fd, "second_derivative")
    mp.setattr(fd, "second_derivative", lambda g, axis, h, periodic, n0=fd.N0: f(g, axis, h, periodic, n0) * h)


def m_fd_x_spacing_everywhere(mp):
    f = original(fd, "laplacian")
    mp.setattr(fd, "laplacian", lambda g, h, periodic, n0=fd.N0: f(g, (h[0],) * 3, periodic, n0))


def m_fd_spacings_reversed(mp):
    f = original(fd, "laplacian")
    mp.setattr(fd, "laplacian", lambda g, h, periodic, n0=fd.N0: f(g, tuple(h)[::-1], periodic, n0))


def m_fd_boundaries_reversed(mp):
    f = original(fd, "laplacian")
    mp.setattr(fd, "laplacian", lambda g, h, periodic, n0=fd.N0: f(g, h, tuple(periodic)[::-1], n0))


def m_fd_dirichlet_wraps(mp):
    f = original(fd, "_shift")
    mp.setattr(fd, "_shift", lambda g, axis, p, periodic: f(g, axis, p, True))


def m_fd_symbol_half_sum(mp):
    def symbol(theta, h, n0=fd.N0):
        w = fd.fd_weights(n0)
        return -(w[0] + sum(w[p] * np.cos(p * theta) for p in range(1, n0 + 1))) / (h * h)
    mp.setattr(fd, "symbol_1d", symbol)


# ---- subdomain Hamiltonian (Sec. 5.A.2, 5.B.2) ------------------------------------------------
def _local(kin, mirror=False):
    def apply_local(self, Y):
        k = Y.shape[0]
        Yg = Y.reshape((k,) + self.shape)
        V = self.V[..., ::-1] if mirror else self.V
        return (kin * fd.laplacian(Yg, self.h, self.periodic, self.n0) + V * Yg).reshape(k, self.N)
    return apply_local


def m_kinetic_factor(mp):
    mp.setattr(SubdomainHamiltonian, "apply_local", _local(-1.0))


def m_potential_mirrored(mp):
    mp.setattr(SubdomainHamiltonian, "apply_local", _local(-0.5, mirror=True))


def _nonlocal(variant):
    def apply_nonlocal(self, Y):
        out = np.zeros_like(Y)
        for flat, chi, E in self.projectors:
            P = Y[:, flat] @ chi.T * (1.0 if variant == "no_dV" else self.dV)
            Ev = np.full(4, E[0]) if variant == "s_energy" else E
            if variant == "assign":
                out[:, flat] = (P * Ev) @ chi
            else:
                out[:, flat] += (P * Ev) @ chi
        return out
    return apply_nonlocal


def m_nonlocal_no_dV(mp):
    mp.setattr(SubdomainHamiltonian, "apply_nonlocal", _nonlocal("no_dV"))


def m_nonlocal_s_energy_everywhere(mp):
    mp.setattr(SubdomainHamiltonian, "apply_nonlocal", _nonlocal("s_energy"))


def m_nonlocal_overwrites(mp):
    mp.setattr(SubdomainHamiltonian, "apply_nonlocal", _nonlocal("assign"))


# ---- electrostatics and projectors (Sec. 5.A.1, 5.B.2) ----------------------------------------
def m_norms_no_dV(mp):
    f = original(pseudo, "projector_norms")
    mp.setattr(pseudo, "projector_norms", lambda w: f(w) * math.sqrt(float(np.prod(w.h))))


def m_px_uses_y(mp):
    def chi(dz, dy, dx, wdt):
        g = np.exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * wdt * wdt))
        return np.stack([g, dy * g, dy * g, dz * g])
    mp.setattr(pseudo, "_chi", chi)


def m_min_image_floor(mp):
    mp.setattr(pseudo, "_min_image", lambda d, L: d - L * np.floor(d / L))


def m_pseudocharge_width(mp):
    f = original(pseudo, "pseudocharge")

    def pseudocharge(w):
        w2 = copy.copy(w)
        w2.species = [dataclasses.replace(s, rc_loc=s.rc_loc * math.sqrt(2.0)) for s in w.species]
        return f(w2)
    mp.setattr(pseudo, "pseudocharge", pseudocharge)


def m_poisson_two_pi(mp):
    f = original(pseudo, "solve_poisson_periodic")
    mp.setattr(pseudo, "solve_poisson_periodic", lambda g, h, n0=fd.N0: 0.5 * f(g, h, n0))


def m_poisson_symbols_swapped(mp):
    def solve(g, h, n0=fd.N0):
        nz, ny, nx = g.shape
        th = [2.0 * math.pi * np.fft.fftfreq(m) for m in (nx, ny, nz)]
        S = (fd.symbol_1d(th[2], h[0], n0)[:, None, None] + fd.symbol_1d(th[1], h[1], n0)[None, :, None]
             + fd.symbol_1d(th[0], h[2], n0)[None, None, :])
        S[0, 0, 0] = 1.0
        P = np.fft.fftn(4.0 * math.pi * g) / S
        P[0, 0, 0] = 0.0
        return np.real(np.fft.ifftn(P))
    mp.setattr(pseudo, "solve_poisson_periodic", solve)


# ---- CheFSI pass (Sec. 5.A.3) -----------------------------------------------------------------
def m_lanczos_no_residual(mp):
    def bound(H, v0, k=10):
        v = np.asarray(v0, dtype=np.float64).reshape(1, H.N)
        v = v / np.linalg.norm(v)
        a, b = np.zeros(k), np.zeros(k)
        f = H.apply(v)
        a[0] = float(np.sum(v * f))
        f = f - a[0] * v
        for j in range(1, k):
            b[j] = float(np.linalg.norm(f))
            vp, v = v, f / b[j]
            f = H.apply(v) - b[j] * vp
            a[j] = float(np.sum(v * f))
            f = f - a[j] * v
        return float(np.linalg.eigvalsh(np.diag(a) + np.diag(b[1:], 1) + np.diag(b[1:], -1))[-1])
    mp.setattr(chefsi, "lanczos_upper_bound", bound)


def m_filter_sigma_sign(mp):
    def coefficients(m, a, b, a0):
        e, c = (b - a) / 2.0, (b + a) / 2.0
        s1 = e / (a0 - c)
        s, out = s1, [(s1 / e, c, 0.0)]
        for _ in range(2, m + 1):
            s2 = 1.0 / (2.0 / s1 + s)
            out.append((2.0 * s2 / e, c, s * s2))
            s = s2
        return out
    mp.setattr(chefsi, "filter_coefficients", coefficients)


def m_filter_centre_and_half_width_swapped(mp):
    # e = (b + a)/2, c = (b - a)/2: the bounds a -> -a give exactly that (swapping a and b instead
    # is no mistake: C_m has the parity of m, so the scaled filter is unchanged)
    f = original(chefsi, "filter_coefficients")
    mp.setattr(chefsi, "filter_coefficients", lambda m, a, b, a0: f(m, -a, b, a0))


def m_filter_shift_on_current(mp):
    def chebyshev_filter(H, X, m, a, b, a0):
        coef = chefsi.filter_coefficients(m, a, b, a0)
        scale, c, _ = coef[0]
        Y = scale * (H.apply(X) - c * X)
        for scale, c, shift in coef[1:]:
            X, Y = Y, scale * (H.apply(Y) - c * Y) - shift * Y
        return Y
    mp.setattr(chefsi, "chebyshev_filter", chebyshev_filter)


def m_projection_ms_from_hpsi(mp):
    def projection(H, Psi_f):
        HPsi = H.apply(Psi_f)
        Hs = Psi_f @ HPsi.T
        Ms = HPsi @ Psi_f.T
        return 0.5 * (Ms + Ms.T), 0.5 * (Hs + Hs.T)
    mp.setattr(chefsi, "projection", projection)


def _geig(variant):
    def generalized_eig(Hs, Ms):
        Lc = np.linalg.cholesky(Ms)
        W = sla.solve_triangular(Lc, Hs, lower=True)
        A = W if variant == "one_sided" else sla.solve_triangular(Lc, W.T, lower=True)
        A = 0.5 * (A + A.T)
        lam, Z = np.linalg.eigh(A)
        if variant == "back_with_L":
            Y = sla.solve_triangular(Lc, Z, lower=True)
        else:
            Y = sla.solve_triangular(Lc.T, Z, lower=False)
        return lam, Y
    return generalized_eig


def m_geig_back_with_L(mp):
    mp.setattr(chefsi, "generalized_eig", _geig("back_with_L"))


def m_geig_one_sided(mp):
    mp.setattr(chefsi, "generalized_eig", _geig("one_sided"))


def m_rotate_untransposed(mp):
    mp.setattr(chefsi, "rotate", lambda Psi_f, Y: Y @ Psi_f)


def m_bounds_a_a0_swapped(mp):
    def run_chefsi(H, Psi0, m, n_passes, b=None, lam_prev=None, v0=None):
        if b is None:
            b = chefsi.lanczos_upper_bound(H, v0)
        lam = chefsi.ritz_values(H, Psi0) if lam_prev is None else lam_prev
        Psi = Psi0
        for _ in range(n_passes):
            lam, Psi = chefsi.chefsi_pass(H, Psi, m, a=float(lam[0]), b=b, a0=float(lam[-1]))
        return lam, Psi, b
    mp.setattr(chefsi, "run_chefsi", run_chefsi)


# ---- Fermi level, density, energies (Sec. 5.A.4-5) --------------------------------------------
def m_fermi_sign(mp):
    f = original(fermi, "fermi")
    mp.setattr(fermi, "fermi", lambda x: f(-np.asarray(x, dtype=np.float64)))


def m_count_no_spin(mp):
    f = original(fermi, "electron_count")
    mp.setattr(fermi, "electron_count", lambda mu, lam, c, kT: 0.5 * f(mu, lam, c, kT))


def m_bisection_wrong_end(mp):
    def fermi_level(lam, c, kT, n_electrons, tol=1e-14, max_iter=200):
        lam, c = np.ravel(lam), np.ravel(c)
        lo, hi = float(lam.min()) - 1.0, float(lam.max()) + 1.0
        for _ in range(max_iter):
            mid = 0.5 * (lo + hi)
            if hi - lo <= tol or mid in (lo, hi):
                break
            if fermi.electron_count(mid, lam, c, kT) < n_electrons:
                hi = mid
            else:
                lo = mid
        return 0.5 * (lo + hi)
    mp.setattr(fermi, "fermi_level", fermi_level)


def m_band_energy_unoccupied(mp):
    mp.setattr(fermi, "band_energy", lambda lam, c, mu, kT: float(2.0 * np.sum(np.asarray(c) * np.asarray(lam))))


def m_entropy_sign(mp):
    f = original(fermi, "entropy_energy")
    mp.setattr(fermi, "entropy_energy", lambda lam, c, mu, kT: -f(lam, c, mu, kT))


def m_density_no_dV(mp):
    f = original(fermi, "point_density")
    mp.setattr(fermi, "point_density", lambda P, g, dV: f(P, g, 1.0))


def m_dos_no_spin(mp):
    f = original(fermi, "dos")
    mp.setattr(fermi, "dos", lambda lam, c, e, width: 0.5 * f(lam, c, e, width))


# ---- divide and conquer (Sec. 5.A.2, 5.A.5) ---------------------------------------------------
def m_weights_whole_subdomain(mp):
    mp.setattr(dc, "interior_weights", lambda Psi, s: np.sum(Psi ** 2, axis=1))


def m_restrict_offset_sign(mp):
    def restrict(V, s):
        nz, ny, nx = V.shape
        ix, iy, iz = ((-s.start[d] + np.arange(s.size[d])) % V.shape[2 - d] for d in range(3))
        return V[np.ix_(iz, iy, ix)]
    mp.setattr(dc, "restrict", restrict)


# ---- SCF pieces (Sec. 5.A.4, 5.B.3) -----------------------------------------------------------
def _exchange(rho):
    rho = np.asarray(rho, dtype=np.float64)
    return np.where(rho > 0, -0.75 * np.cbrt(3.0 * np.maximum(rho, 0.0) / math.pi), 0.0)


def m_exchange_prefactor(mp):
    f = original(scf, "lda_pz81")

    def lda(rho):
        eps, v = f(rho)
        return eps + _exchange(rho) / 3.0, v
    mp.setattr(scf, "lda_pz81", lda)


def m_exchange_potential_factor(mp):
    f = original(scf, "lda_pz81")

    def lda(rho):
        eps, v = f(rho)
        return eps, v - _exchange(rho) / 3.0
    mp.setattr(scf, "lda_pz81", lda)


def m_pz_beta1_digit(mp):
    mp.setattr(scf, "PZ_BETA1", 1.529)


def m_pz_a_digit(mp):
    mp.setattr(scf, "PZ_A", 0.0313)


def m_pz_c_digit(mp):
    mp.setattr(scf, "PZ_C", 0.0200)


def m_self_energy_no_half(mp):
    f = original(scf, "self_energy")
    mp.setattr(scf, "self_energy", lambda w: 2.0 * f(w))


def m_kerker_kappa_not_squared(mp):
    def kerker(R, h, kappa):
        nz, ny, nx = R.shape
        th = [2.0 * math.pi * np.fft.fftfreq(m) for m in (nx, ny, nz)]
        S = (fd.symbol_1d(th[2], h[2])[:, None, None] + fd.symbol_1d(th[1], h[1])[None, :, None]
             + fd.symbol_1d(th[0], h[0])[None, None, :])
        return np.real(np.fft.ifftn(S / (S + kappa) * np.fft.fftn(R)))
    mp.setattr(scf, "kerker", kerker)


def m_pulay_drops_residual_term(mp):
    def step(self, x, g):
        x = x.ravel()
        f = g.ravel() - x
        if self.x_prev is not None:
            self.dX.append(x - self.x_prev)
            self.dF.append(f - self.f_prev)
            if len(self.dX) > self.history:
                self.dX.pop(0)
                self.dF.pop(0)
        self.x_prev, self.f_prev = x.copy(), f.copy()
        nxt = x + self.beta * self.precondition(f)
        if (self.k + 1) % self.period == 0 and self.dF:
            F, X = np.stack(self.dF, axis=1), np.stack(self.dX, axis=1)
            nxt = nxt - X @ np.linalg.solve(F.T @ F, F.T @ f)
        self.k += 1
        return nxt
    mp.setattr(scf.Mixer, "step", step)


def m_pulay_every_step(mp):
    f = original(scf.Mixer, "step")

    def step(self, x, g):
        self.period = 1
        return f(self, x, g)
    mp.setattr(scf.Mixer, "step", step)


# ---- learned start (Sec. 5.A.4, initialisation) -----------------------------------------------
def m_tanh_derivative(mp):
    def loss_and_grad(theta, X, y):
        yp, acts = learned.forward(theta, X, keep=True)
        n = len(y)
        layers = learned.unpack(theta)
        grads, delta = [], (2.0 / n) * (yp - y)[:, None]
        for li in range(len(layers) - 1, -1, -1):
            W, _ = layers[li]
            grads.append((acts[li].T @ delta, delta.sum(axis=0)))
            if li > 0:
                delta = (delta @ W.T) * (1.0 - acts[li])
        grads.reverse()
        return float(np.mean((yp - y) ** 2)), np.concatenate([np.concatenate([a.ravel(), b]) for a, b in grads])
    mp.setattr(learned, "loss_and_grad", loss_and_grad)


def m_adam_no_bias_correction(mp):
    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        return theta - self.lr * self.m / (np.sqrt(self.v) + self.eps)
    mp.setattr(learned.Adam, "step", step)


def m_descriptor_width(mp):
    mp.setattr(learned, "SIGMA", 0.25 * math.sqrt(2.0))


def m_cutoff_no_offset(mp):
    mp.setattr(learned, "cutoff", lambda r: np.where(r < learned.R_CUT, 0.5 * np.cos(math.pi * r / learned.R_CUT), 0.0))


def m_sad_width(mp):
    f = original(learned, "sad_density")

    def sad(w):
        w2 = copy.copy(w)
        w2.species = [dataclasses.replace(s, rc_loc=s.rc_loc * math.sqrt(2.0)) for s in w.species]
        return f(w2)
    mp.setattr(learned, "sad_density", sad)


def m_bf16_truncates(mp):
    def bf16(x):
        u = np.asarray(x, dtype=np.float32).view(np.uint32)
        return ((u >> 16) << 16).astype(np.uint32).view(np.float32).astype(np.float64)
    mp.setattr(learned, "bf16", bf16)


def m_occupations_times_kT(mp):
    mp.setattr(fermi, "occupations", lambda lam, mu, kT: fermi.fermi((np.asarray(lam, dtype=np.float64) - mu) * kT))


def m_assemble_unoccupied_density(mp):
    f = original(fermi, "point_density")

    def assemble(w, subs, lam, c, Psi, kT, n_electrons):
        mu = fermi.fermi_level(np.concatenate(lam), np.concatenate(c), kT, n_electrons)
        n = np.asarray(w.n)
        rho = np.zeros(int(np.prod(n)))
        for s, la, P in zip(subs, lam, Psi):
            rho[dc.core_global_indices(s, n)] = f(P[:, dc.core_local_indices(s)], np.ones(len(la)), float(np.prod(w.h)))
        lam_all, c_all = np.concatenate(lam), np.concatenate(c)
        return (mu, rho.reshape(n[2], n[1], n[0]), fermi.band_energy(lam_all, c_all, mu, kT),
                fermi.entropy_energy(lam_all, c_all, mu, kT))
    mp.setattr(dc, "assemble", assemble)


# ---- further index and convention mistakes --------------------------------------------------
def m_partition_strict_period(mp):
    def partition(w):
        n = np.asarray(w.n)
        subs = []
        for a in range(w.n_sub):
            core_lo, core_n, buf = (np.asarray(v[a]) for v in (w.core_lo, w.core_n, w.buf))
            size = core_n + 2 * buf
            periodic = size > n
            b = np.where(periodic, np.minimum(buf, (n - core_n) // 2), buf)
            size = np.where(periodic, n, size)
            subs.append(dc.Subdomain(start=core_lo - b, size=size, periodic=periodic, core_lo=b, core_n=core_n,
                                     core_global_lo=core_lo))
        return subs
    mp.setattr(dc, "partition", partition)


def m_core_indices_wrong_stride(mp):
    def core_local_indices(s):
        k, j, i = np.meshgrid(*(s.core_lo[d] + np.arange(s.core_n[d]) for d in (2, 1, 0)), indexing="ij")
        return (i + s.size[0] * (j + s.size[2] * k)).ravel()
    mp.setattr(dc, "core_local_indices", core_local_indices)


def m_projector_energies_swapped(mp):
    f = original(pseudo, "subdomain_projectors")
    mp.setattr(pseudo, "subdomain_projectors",
               lambda w, start, size, norms: [(fl, chi, E[::-1].copy()) for fl, chi, E in f(w, start, size, norms)])


def m_entropy_one_sided(mp):
    def entropy_s(g):
        g = np.asarray(g, dtype=np.float64)
        return np.where(g > 0, g * np.log(np.where(g > 0, g, 1.0)), 0.0)
    mp.setattr(fermi, "entropy_s", entropy_s)


def m_last_hidden_layer_linear(mp):
    def forward(theta, X, keep=False):
        acts, h = [X], X
        layers = learned.unpack(theta)
        for li, (W, b) in enumerate(layers):
            z = h @ W + b
            h = np.tanh(z) if li < len(layers) - 2 else z
            acts.append(h)
        return (h[:, 0], acts) if keep else h[:, 0]
    mp.setattr(learned, "forward", forward)


def m_descriptor_species_blocks_swapped(mp):
    f = original(learned, "descriptors")

    def descriptors(w, points=None, n_species=2):
        D = f(w, points, n_species)
        return np.concatenate([D[:, learned.N_RADIAL:], D[:, :learned.N_RADIAL]], axis=1)
    mp.setattr(learned, "descriptors", descriptors)


def m_inference_unrounded(mp):
    mp.setattr(learned, "forward_bf16", lambda theta, X: learned.forward(theta, X))


def m_inference_drops_bias(mp):
    def forward_bf16(theta, X):
        h = learned.bf16(X)
        layers = learned.unpack(theta)
        for li, (W, b) in enumerate(layers):
            z = h @ learned.bf16(W)
            h = learned.bf16(np.tanh(z)) if li < len(layers) - 1 else z
        return h[:, 0]
    mp.setattr(learned, "forward_bf16", forward_bf16)


def m_learned_start_unclipped(mp):
    def learned_start(w, theta, n_species=2):
        n = np.asarray(w.n)
        corr = learned.forward_bf16(theta, learned.descriptors(w, n_species=n_species)).reshape(n[2], n[1], n[0])
        rho = learned.sad_density(w) + corr
        return rho * (w.n_electrons / (rho.sum() * float(np.prod(w.h))))
    mp.setattr(learned, "learned_start", learned_start)


def m_local_operator_near_radius(mp):
    # the local operator keeps the atoms within r_cut - 1 bohr of the box instead of r_cut + 1
    import synth
    f = original(synth, "near_atoms")
    mp.setattr(synth, "near_atoms", lambda w, start, size, margin: f(w, start, size, margin - 2.0))


def m_partition_core_at_origin(mp):
    f = original(dc, "partition")

    def partition(w):
        subs = f(w)
        for sd in subs:
            sd.core_lo = np.zeros(3, dtype=int)
        return subs
    mp.setattr(dc, "partition", partition)


def m_partition_start_after_core(mp):
    f = original(dc, "partition")

    def partition(w):
        subs = f(w)
        for sd in subs:
            sd.start = sd.core_global_lo + sd.core_lo
        return subs
    mp.setattr(dc, "partition", partition)


# ---- SCF energy assembly (Sec. 5.A.4): the Janak pin, three converged SCF runs each -------------
def _scf_step(variant):
    from synth import lanczos_start

    def step(w, st, n_passes=1, n_electrons=None):
        dV = float(np.prod(w.h))
        V, phi, eps, vxc = scf.effective_potential(w, st.rho, st.b)
        subs = dc.partition(w)
        lam, c, Psi = [], [], []
        for a, s in enumerate(subs):
            H = dc.subdomain_operator(w, s, V, st.norms)
            bup = chefsi.lanczos_upper_bound(H, lanczos_start(H.N))
            P = st.Psi[a]
            la = st.lam[a] if st.lam[a] is not None else chefsi.ritz_values(H, P)
            for _ in range(n_passes):
                la, P = chefsi.chefsi_pass(H, P, w.degree, float(la.max()), bup, float(la.min()))
            lam.append(la)
            Psi.append(P)
            c.append(dc.interior_weights(P, s))
        ne = w.n_electrons if n_electrons is None else float(n_electrons)
        mu, rho_out, e_band, e_ent = dc.assemble(w, subs, lam, c, Psi, w.kT, ne)
        rho_in = st.rho
        hartree = 0.5 * float(((st.b - rho_in) * phi).sum() * dV)
        dc_xc = float((vxc * rho_in).sum() * dV)
        energy = (e_band + float((rho_in * eps).sum() * dV) - (0.0 if variant == "no_vxc_rho" else dc_xc)
                  + (-hartree if variant == "hartree_sign" else hartree) - scf.self_energy(w) - e_ent)
        residual = float(np.linalg.norm(rho_out - rho_in) / np.linalg.norm(rho_out))
        st.rho = st.mixer.step(rho_in, rho_out).reshape(rho_in.shape)
        st.Psi, st.lam = Psi, lam
        return residual, energy, mu, rho_out
    return step


def m_veff_minus_vxc(mp):
    def effective_potential(w, rho, b):
        phi = pseudo.solve_poisson_periodic(rho + b, w.h)
        eps, vxc = scf.lda_pz81(rho)
        return phi - vxc, phi, eps, vxc
    mp.setattr(scf, "effective_potential", effective_potential)


def m_energy_hartree_sign(mp):
    mp.setattr(scf, "step", _scf_step("hartree_sign"))


def m_energy_drops_vxc_rho(mp):
    mp.setattr(scf, "step", _scf_step("no_vxc_rho"))


# mutant -> the pin that must fail under it
MUTANTS = [
    (m_fd_weight_signs, po.test_fd_weights_match_published_table),
    (m_fd_centre_weight, po.test_fd_stencil_exact_on_polynomials),
    (m_fd_over_h, po.test_periodic_laplacian_plane_waves_match_symbol),
    (m_fd_x_spacing_everywhere, po.test_periodic_laplacian_plane_waves_match_symbol),
    (m_fd_spacings_reversed, lambda: po.test_hamiltonian_equals_kronecker_sum_matrix((False, False, False))),
    (m_fd_boundaries_reversed, lambda: po.test_hamiltonian_equals_kronecker_sum_matrix((True, False, False))),
    (m_fd_dirichlet_wraps, lambda: po.test_hamiltonian_equals_kronecker_sum_matrix((False, False, False))),
    (m_fd_symbol_half_sum, po.test_periodic_laplacian_plane_waves_match_symbol),
    (m_kinetic_factor, lambda: po.test_hamiltonian_equals_kronecker_sum_matrix((False, False, False))),
    (m_potential_mirrored, lambda: po.test_hamiltonian_equals_kronecker_sum_matrix((False, False, False))),
    (m_nonlocal_no_dV, po.test_projectors_are_eigenvectors_of_the_nonlocal_term),
    (m_nonlocal_s_energy_everywhere, po.test_projectors_are_eigenvectors_of_the_nonlocal_term),
    (m_nonlocal_overwrites, lambda: po.test_hamiltonian_is_symmetric((True, True, True))),
    (m_norms_no_dV, po.test_projector_norms_and_symmetry),
    (m_px_uses_y, po.test_projector_norms_and_symmetry),
    (m_min_image_floor, po.test_projector_norms_and_symmetry),
    (m_pseudocharge_width, po.test_single_atom_potential_matches_erf_coulomb),
    (m_poisson_two_pi, po.test_poisson_solution_satisfies_fd_equation),
    (m_poisson_symbols_swapped, po.test_poisson_on_orthorhombic_grid),
    (m_lanczos_no_residual, pc.test_lanczos_bound_above_spectrum_and_tight),
    (m_filter_sigma_sign, lambda: pc.test_filter_is_scaled_chebyshev_on_diagonal_operator(7)),
    (m_filter_centre_and_half_width_swapped, lambda: pc.test_filter_is_scaled_chebyshev_on_diagonal_operator(7)),
    (m_filter_shift_on_current, lambda: pc.test_filter_is_scaled_chebyshev_on_diagonal_operator(7)),
    (m_projection_ms_from_hpsi, pc.test_chefsi_converges_to_fd_laplacian_spectrum),
    (m_geig_back_with_L, pc.test_generalized_eig_matches_lapack_and_invariants),
    (m_geig_one_sided, pc.test_generalized_eig_matches_lapack_and_invariants),
    (m_rotate_untransposed, pc.test_chefsi_converges_to_fd_laplacian_spectrum),
    (m_bounds_a_a0_swapped, pc.test_chefsi_converges_to_fd_laplacian_spectrum),
    (m_fermi_sign, pc.test_fermi_function_and_entropy),
    (m_count_no_spin, pc.test_fermi_level_bisection_against_brent),
    (m_bisection_wrong_end, pc.test_fermi_level_bisection_against_brent),
    (m_band_energy_unoccupied, pc.test_energies_definitions_on_two_levels),
    (m_entropy_sign, pc.test_energies_definitions_on_two_levels),
    (m_density_no_dV, pc.test_config0_invariants),
    (m_dos_no_spin, pc.test_energies_definitions_on_two_levels),
    (m_weights_whole_subdomain, pc.test_interior_weights_count_core_points_only),
    (m_restrict_offset_sign, po.test_restriction_wraps_periodically),
    (m_exchange_prefactor, ps.test_slater_exchange_high_density_limit),
    (m_exchange_potential_factor, lambda: ps.test_xc_potential_is_derivative_of_energy_density(2.0)),
    (m_pz_beta1_digit, ps.test_pz81_correlation_joins_smoothly_at_rs_one),
    (m_pz_a_digit, ps.test_pz81_high_density_expansion),
    (m_pz_c_digit, ps.test_pz81_correlation_joins_smoothly_at_rs_one),
    (m_self_energy_no_half, ps.test_self_energy_matches_quadrature),
    (m_kerker_kappa_not_squared, ps.test_kerker_matches_real_space_operator),
    (m_pulay_drops_residual_term, ps.test_pulay_exact_on_linear_map),
    (m_pulay_every_step, ps.test_periodic_pulay_alternates_linear_and_extrapolated_steps),
    (m_tanh_derivative, pl.test_gradient_matches_finite_differences),
    (m_adam_no_bias_correction, pl.test_adam_first_step_is_lr_times_sign),
    (m_descriptor_width, pl.test_descriptors_single_atom_closed_form),
    (m_cutoff_no_offset, pl.test_descriptors_single_atom_closed_form),
    (m_sad_width, pl.test_sad_matches_gaussian_and_normalisation),
    (m_bf16_truncates, pl.test_bf16_rounding_known_values),
    (m_partition_strict_period, po.test_restriction_wraps_periodically),
    (m_core_indices_wrong_stride, pc.test_interior_weights_count_core_points_only),
    (m_projector_energies_swapped, po.test_projectors_are_eigenvectors_of_the_nonlocal_term),
    (m_entropy_one_sided, pc.test_fermi_function_and_entropy),
    (m_last_hidden_layer_linear, pl.test_gradient_matches_finite_differences),
    (m_descriptor_species_blocks_swapped, pl.test_descriptors_single_atom_closed_form),
    (m_inference_unrounded, pl.test_bf16_inference_within_rounding_of_full_precision),
    (m_inference_drops_bias, pl.test_bf16_inference_within_rounding_of_full_precision),
    (m_learned_start_unclipped, pl.test_learned_start_normalised_and_nonnegative),
    (m_local_operator_near_radius, po.test_local_subdomain_operator_with_random_atoms),
    (m_partition_core_at_origin, po.test_partition_mixes_periodic_and_dirichlet_axes),
    (m_partition_start_after_core, po.test_partition_mixes_periodic_and_dirichlet_axes),
    (m_occupations_times_kT, pc.test_energies_definitions_on_two_levels),
    (m_assemble_unoccupied_density, pc.test_config0_invariants),
    pytest.param(m_energy_hartree_sign, ps.test_scf_energy_derivative_is_chemical_potential, marks=pytest.mark.slow),
    pytest.param(m_energy_drops_vxc_rho, ps.test_scf_energy_derivative_is_chemical_potential, marks=pytest.mark.slow),
    pytest.param(m_veff_minus_vxc, ps.test_scf_energy_derivative_is_chemical_potential, marks=pytest.mark.slow),
]


def _pair(entry):
    return tuple(entry.values) if hasattr(entry, "values") else entry


@pytest.mark.parametrize("plant,pin", MUTANTS, ids=[_pair(e)[0].__name__[2:] for e in MUTANTS])
def test_pin_fails_on_planted_mistake(plant, pin, monkeypatch):
    plant(monkeypatch)
    with pytest.raises((AssertionError, np.linalg.LinAlgError, fermi.NoBracket)):
        pin()


@pytest.mark.parametrize("pin", [p for p in dict.fromkeys(_pair(e)[1] for e in MUTANTS)
                                 if p is not ps.test_scf_energy_derivative_is_chemical_potential],
                         ids=lambda p: getattr(p, "__name__", "case"))
def test_pins_pass_on_the_oracle(pin):
    """The same pin calls, unpatched, pass: a failure above comes from the planted mistake."""
    pin()
