"""One self-consistent-field step of the D&C Kohn-Sham solver (Sec. 5.A.4 and 5.B.3: SCF with
CheFSI, periodic Pulay density mixing with a Kerker-type elliptic preconditioner).

Test infrastructure only: plain FP64 numpy, FFT Poisson with the FD symbol.

Readings (the paper fixes none of these numbers):
  * exchange-correlation: LDA, Slater exchange + Perdew-Zunger 1981 correlation (unpolarised),
    parameters from that publication; eps_xc = v_xc = 0 where rho <= 0;
  * electrostatics: -Delta_h phi = 4 pi (rho + b), phi(G = 0) = 0 (Eq. poisson); V_eff = phi + v_xc;
  * energy (Harris-Foulkes form at the input density, pseudocharge electrostatics):
        E = E_band + E_xc[rho] - sum v_xc rho dV + 1/2 sum (b - rho) phi dV - E_self - E_entropy
    with E_self = 1/2 sum_I int b_I V_I = 1/2 sum_I Z_I^2 sqrt(2/pi) / r_c,I (continuum value;
    the Gaussian-overlap ion correction is omitted: a geometry constant);
  * mixing: periodic Pulay (Pulay extrapolation every p-th step, preconditioned linear mixing
    otherwise), history m = 7, beta = 0.3, Kerker preconditioner P = S / (S + kappa^2) with S the
    FD symbol of -Delta_h, kappa = 0.5 / bohr;
  * residual: ||rho_out - rho_in||_2 / ||rho_out||_2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from synth import lanczos_start

from . import chefsi, dc, fd, fermi, pseudo

# Perdew-Zunger 1981 (Phys. Rev. B 23, 5048), unpolarised correlation fit to Ceperley-Alder
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334          # r_s >= 1
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116         # r_s < 1


def lda_pz81(rho: np.ndarray):
    """(eps_xc, v_xc) per point: energy per electron and potential d(rho eps)/d rho."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    m = rho > 0.0
    r = rho[m]
    rs = (3.0 / (4.0 * math.pi * r)) ** (1.0 / 3.0)
    # Slater exchange: eps_x = -(3/4)(3 rho/pi)^(1/3), v_x = (4/3) eps_x
    ex = -0.75 * (3.0 * r / math.pi) ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex
    ec = np.empty_like(r)
    vc = np.empty_like(r)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * s + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    # v_c = eps_c - (r_s / 3) d eps_c / d r_s
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_BETA1 * s + 4.0 / 3.0 * PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    x = rs[lo]
    lx = np.log(x)
    ec[lo] = PZ_A * lx + PZ_B + PZ_C * x * lx + PZ_D * x
    vc[lo] = (PZ_A * lx + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * x * lx
              + (2.0 * PZ_D - PZ_C) / 3.0 * x)
    eps[m] = ex + ec
    v[m] = vx + vc
    return eps, v


def self_energy(w) -> float:
    """1/2 sum_I int b_I V_I for Gaussian pseudocharges and V_I = -Z erf(r/r_c)/r."""
    tot = 0.0
    for s in w.species_index:
        sp = w.species[s]
        tot += 0.5 * sp.Zv ** 2 * math.sqrt(2.0 / math.pi) / sp.rc_loc
    return tot


def kerker(R: np.ndarray, h, kappa: float) -> np.ndarray:
    """P R with P = S / (S + kappa^2) in Fourier space, S the FD symbol of -Delta_h."""
    nz, ny, nx = R.shape
    th = [2.0 * math.pi * np.fft.fftfreq(m) for m in (nx, ny, nz)]
    S = (fd.symbol_1d(th[2], h[2])[:, None, None] + fd.symbol_1d(th[1], h[1])[None, :, None]
         + fd.symbol_1d(th[0], h[0])[None, None, :])
    return np.real(np.fft.ifftn(S / (S + kappa * kappa) * np.fft.fftn(R)))


@dataclass
class Mixer:
    """Periodic Pulay mixing of densities (flattened) with Kerker preconditioning."""
    h: tuple
    shape: tuple
    beta: float = 0.3
    kappa: float | None = 0.5
    history: int = 7
    period: int = 2
    k: int = 0
    x_prev: np.ndarray | None = None
    f_prev: np.ndarray | None = None
    dX: list = field(default_factory=list)
    dF: list = field(default_factory=list)

    def precondition(self, f: np.ndarray) -> np.ndarray:
        if self.kappa is None:          # plain (unpreconditioned) mixing
            return f
        return kerker(f.reshape(self.shape), self.h, self.kappa).ravel()

    def step(self, x: np.ndarray, g: np.ndarray) -> np.ndarray:
        """Next input density from the input x and the output g of the current step."""
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
            F = np.stack(self.dF, axis=1)
            X = np.stack(self.dX, axis=1)
            gam = np.linalg.solve(F.T @ F, F.T @ f)
            PF = np.stack([self.precondition(F[:, i]) for i in range(F.shape[1])], axis=1)
            nxt = nxt - (X + self.beta * PF) @ gam
        self.k += 1
        return nxt


@dataclass
class SCFState:
    rho: np.ndarray                     # input density of the next step, (nz, ny, nx)
    Psi: list                           # per subdomain (N_s, N_d)
    lam: list                           # Ritz values of the last pass (bounds a, a0)
    mixer: Mixer
    b: np.ndarray                       # total pseudocharge
    norms: np.ndarray                   # projector normalisation


def start(w, rho0: np.ndarray, Psi0: list) -> SCFState:
    """State before the first step: the start density and blocks; Ritz values of the unfiltered
    blocks give the first filter's (a, a0)."""
    b = pseudo.pseudocharge(w)
    return SCFState(rho=np.array(rho0, dtype=np.float64), Psi=[np.array(P) for P in Psi0], lam=[None] * w.n_sub,
                    mixer=Mixer(h=tuple(w.h), shape=tuple(rho0.shape)), b=b, norms=pseudo.projector_norms(w))


def effective_potential(w, rho: np.ndarray, b: np.ndarray):
    """(V_eff, phi, eps_xc, v_xc) of the density rho."""
    phi = pseudo.solve_poisson_periodic(rho + b, w.h)
    eps, vxc = lda_pz81(rho)
    return phi + vxc, phi, eps, vxc


def step(w, st: SCFState, n_passes: int = 1, n_electrons: float | None = None):
    """One SCF step: V_eff[rho_in]; per subdomain the Lanczos bound b of the new operator and
    n_passes CheFSI passes (a, a0 from the previous Ritz values); mu, rho_out, energies; the
    residual; mixing.  n_electrons defaults to the cell's valence count (another count leaves
    the cell charged against the neutralising background of the G = 0 convention).  Returns
    (residual, energy, mu, rho_out) and advances the state."""
    dV = float(np.prod(w.h))
    V, phi, eps, vxc = effective_potential(w, st.rho, st.b)
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
    e_xc = float((rho_in * eps).sum() * dV)
    energy = (e_band + e_xc - float((vxc * rho_in).sum() * dV) + 0.5 * float(((st.b - rho_in) * phi).sum() * dV)
              - self_energy(w) - e_ent)
    residual = float(np.linalg.norm(rho_out - rho_in) / np.linalg.norm(rho_out))
    st.rho = st.mixer.step(rho_in, rho_out).reshape(rho_in.shape)
    st.Psi, st.lam = Psi, lam
    return residual, energy, mu, rho_out
