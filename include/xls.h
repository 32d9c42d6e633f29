/*
 * xls.h - C ABI of libxls: the per-subdomain CheFSI pass of divide-and-conquer Kohn-Sham DFT
 * (arXiv 2609.13115, "XLSDFT"), on one GB300 GPU.
 *
 * The library owns every device buffer it uses (allocated at xls_grid_create, freed at
 * xls_grid_destroy).  Pointers passed in are only read (or written, for outputs) during the
 * call; "on_device" flags say whether a pointer is device memory of the current CUDA device
 * (else host memory).  All work is queued on the stream given at creation; calls that return
 * host results synchronise that stream.  No call throws or exits: every call returns an
 * xls_status, and xls_last_error() describes the last failure of the calling thread (with the
 * failing subdomain where there is one).  Errors detected by kernels (non-SPD Gram matrix,
 * non-finite values, a Fermi level that cannot be bracketed) are reported by the next call
 * that synchronises.
 *
 * Grid conventions.  A global periodic orthorhombic cell of edges L[3] (bohr) carries n[3]
 * grid points, spacing h = L/n, point (i,j,k) at (i h_x, j h_y, k h_z), flat index
 * i + n_x (j + n_y k) (x fastest).  Subdomain alpha (Sec. 5.A.2, the partition equation) is
 * a core box of core_n points starting at global index core_lo, extended by buf points on
 * each side; along an axis where core_n + 2 buf >= n the subdomain is the whole period and
 * periodic, elsewhere the Hamiltonian is Dirichlet-zero outside it.  A block of vectors of a
 * subdomain is stored vector-major: vector v occupies N_d consecutive values (x fastest).
 */
#ifndef XLS_H
#define XLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xls_grid_s* xls_grid;
typedef struct xls_mlp_s* xls_mlp;   /* learned-start model: owns its device parameters */

typedef enum {
  XLS_OK = 0,
  XLS_EINVAL = 1,     /* bad argument (sizes, pointers, state) */
  XLS_ENOMEM = 2,     /* device allocation failed or exceeds the HBM budget */
  XLS_ECUDA = 3,      /* a CUDA runtime/driver call failed */
  XLS_ENOTSPD = 4,    /* Gram matrix M_s not positive definite (Cholesky pivot <= 0) */
  XLS_ENOCONV = 5,    /* Fermi level not bracketed: N_e outside the capacity of the states */
  XLS_ETIMEOUT = 6,   /* a bounded device wait gave up */
  XLS_ENONFINITE = 7  /* NaN/Inf detected in a result */
} xls_status;

typedef enum {
  XLS_FP64 = 0,        /* every step in FP64 */
  XLS_MIXED_BF16 = 1,  /* FP32 filter, split-BF16 tensor-core Gram/rotation with FP32 accumulation,
                          FP64 Cholesky / eigensolve / Fermi level / energies */
  XLS_MIXED_FP16 = 2   /* as XLS_MIXED_BF16 with split-FP16 products: every vector is scaled by a power
                          of two (its largest entry into (2^13, 2^14]) before the split, undone exactly
                          after the accumulation; about 16x smaller product error than split BF16 */
} xls_precision;

typedef struct {
  double L[3];        /* cell edges, bohr */
  int n[3];           /* global grid points per axis */
} xls_cell;

typedef struct {
  int n_sub;               /* number of subdomains (>= 1) */
  const int* core_lo;      /* [3*n_sub] global index of the first core point per axis */
  const int* core_n;       /* [3*n_sub] core points per axis (cores must tile the grid) */
  const int* buf;          /* [3*n_sub] buffer points on each side per axis */
  const int* n_states;     /* [n_sub] vectors per subdomain, N_s^alpha (1..1024) */
} xls_dc;

typedef struct {
  double Zv;       /* valence charge (enters only through the electron count given by the caller) */
  double rc_loc;   /* local-potential radius (unused by the pass; V_eff is an input) */
  double w_proj;   /* projector Gaussian width w: chi_s = exp(-r^2/2w^2), chi_p = x_a chi_s */
  double r_cut;    /* projectors vanish for r >= r_cut (must be < half of every cell edge) */
  double E_s;      /* Kleinman-Bylander energy of the s projector, Ha */
  double E_p;      /* Kleinman-Bylander energy of each p projector, Ha */
} xls_species;

/* Create a grid handle: validates the partition, allocates the blocks of every subdomain in
 * the requested precision and the subspace workspaces.  hbm_budget_bytes (0 = no limit): when
 * the estimated device footprint of all subdomains exceeds it, the grid runs in waves of
 * consecutive subdomains whose footprint fits (see xls_get_waves); XLS_ENOMEM if one subdomain
 * alone exceeds it.  cuda_stream may be NULL (legacy default stream).  Sec. 5.A.2 (partition),
 * Sec. 5.B (data kept resident in HBM). */
xls_status xls_grid_create(const xls_cell* cell, const xls_dc* dc, int precision,
                           size_t hbm_budget_bytes, void* cuda_stream, xls_grid* out);

xls_status xls_grid_destroy(xls_grid g);

/* Restrict V_eff (global grid, n_x*n_y*n_z doubles) to every subdomain and build the
 * nonlocal projector tables of every atom whose r_cut sphere meets it (minimum periodic
 * image; each chi normalised on the global grid, sum chi^2 dV = 1), then compute each
 * subdomain's spectrum upper bound b by a 10-step Lanczos run from a fixed SplitMix64 start
 * vector (seed 0x1A4C705, stream position = subdomain point index).  pos: [3*n_atoms] bohr;
 * species: [n_atoms] indices into sp[0..n_species).  Sec. 5.A.5 "Restriction of effective
 * potentials", Sec. 5.B.2 (projectors grouped by atom). */
xls_status xls_hamiltonian_set(xls_grid g, const double* veff, int veff_on_device, int n_atoms,
                               const double* pos, const int* species, int n_species,
                               const xls_species* sp);

/* Load the start block of subdomain `sub` (N_s x N_d doubles, vector-major) into the grid's
 * orbital storage (rounded to FP32 on the mixed path). */
xls_status xls_orbitals_set(xls_grid g, int sub, const double* psi, int on_device);

/* FP32 forms of xls_orbitals_set / xls_orbitals_get (N_s x N_d floats, vector-major, host or
 * device): on the mixed paths the block is the grid's own FP32 storage, copied without
 * conversion (half the bytes of the FP64 forms); on the FP64 path it is widened to (set) or
 * rounded from (get) FP64 on the device.  Library-specific: the paper keeps FP64 orbitals.
 * Errors: XLS_EINVAL for bad arguments and in wave mode (whose host store the FP64 forms fill),
 * XLS_ECUDA. */
xls_status xls_orbitals_set_f32(xls_grid g, int sub, const float* psi, int on_device);
xls_status xls_orbitals_get_f32(xls_grid g, int sub, float* psi_out, int on_device);

/* Fill every subdomain's start block with U[-0.5, 0.5) from SplitMix64 (Steele et al. 2014):
 * value k of the concatenated blocks (subdomains in order, each vector-major) is the top 53
 * bits of output k of the stream of `seed`, times 2^-53, minus 0.5. */
xls_status xls_orbitals_random(xls_grid g, uint64_t seed);

/* Copy subdomain `sub`'s current orbital block (N_s x N_d, vector-major) out as doubles. */
xls_status xls_orbitals_get(xls_grid g, int sub, double* psi_out, int on_device);

/* n_passes CheFSI iterations on every subdomain (Sec. 5.A.3 steps (1)-(4)):
 *   (1) scaled Chebyshev filter of degree `degree` on [a, b] (three-term recurrence,
 *       Zhou et al. 2006): Psi_f = C_m((H-c)/e) Psi / C_m((a0-c)/e), e = (b-a)/2, c = (b+a)/2;
 *   (2) M_s = Psi_f^T Psi_f, H_s = Psi_f^T H Psi_f;
 *   (3) H_s y = lambda M_s y by Cholesky reduction and a symmetric eigensolve (FP64);
 *   (4) Psi = Psi_f Y; then the interior weights c_n = sum over core points of psi_n^2.
 * bounds: NULL, or [3*n_sub] (b, a, a0) per subdomain for the first pass; with NULL the
 * first pass of a fresh start block takes b from xls_hamiltonian_set and (a, a0) = the
 * (largest, smallest) Ritz values of the unfiltered block, and later passes take (a, a0)
 * from the previous pass's Ritz values.  Every subdomain runs in the same launches. */
xls_status xls_chefsi_batch(xls_grid g, int degree, int n_passes, const double* bounds);

/* Autotuner of the batched launches (library-specific: the paper tunes its kernels by hand for
 * its CPUs).  On the grid's own data it times the launch configurations of the tunable stages
 * and keeps the fastest of each:
 *   choices_out[0]: CTAs per subdomain cluster of the Cholesky factorisation and the
 *                   tridiagonalisation, 8 or 16 (0: clusters off, not tuned);
 *   choices_out[1]: K split of the tensor-core Gram, in CTAs per SM aimed at, one of 1, 2, 3, 4,
 *                   6, 8 (0: no tensor-core Gram on this grid, not tuned);
 *   choices_out[2]: vectors per CTA of the nonlocal projection, 8, 16 or 32 (0: no projectors).
 * It also times the back-projection with one and with two grid points per thread and, per class
 * of the FP32 TMA stencil whose slot pitch has a compile-time variant
 * (80 or 112 floats), that variant against the runtime-pitch one (the default) and keeps the
 * faster (not reported; XLS_TRACE=1 prints the timings).
 * Every candidate runs `reps` (1..100) times after one warm-up call, timed with CUDA events on
 * the grid's stream.  The input is the last pass's M_s and H_s: they and the split exponents are
 * saved and put back, the eigenpairs recomputed with the chosen configuration, so the next pass
 * differs from an untuned one by rounding only.  Captured pass graphs are dropped (the next
 * graphed pass captures the tuned launches).  In wave carry mode it tunes the worker on the last
 * wave it ran (the choices hold for every wave: all have the same shapes).  choices_out: NULL or
 * room for 3 ints.
 * Errors: XLS_EINVAL (bad arguments, store-mode waves, no pass run yet), XLS_ENOMEM (no room for the
 * saved matrices), XLS_ECUDA, and the status of the eigensolve (XLS_ENOTSPD). */
xls_status xls_autotune(xls_grid g, int reps, int* choices_out);

/* Stage-wise entry points with the same arithmetic as one pass of xls_chefsi_batch, for
 * checking each step on its own.  stage 1: filter only (the orbital block becomes Psi_f);
 * stage 2: projection of the current block into M_s, H_s; stage 3: eigensolve of the current
 * M_s, H_s (lambda, Y); stage 4: rotation of the current block by Y and interior weights. */
xls_status xls_chefsi_stage(xls_grid g, int stage, int degree, const double* bounds);

/* Apply H^alpha to k <= N_s vectors x (k x N_d, vector-major) of subdomain `sub`, giving y.
 * Uses (and overwrites) the subdomain's first k work vectors; in the grid's precision. */
xls_status xls_hamiltonian_apply(xls_grid g, int sub, int k, const double* x, double* y, int on_device);

/* Fermi level, density and energies (Sec. 5.A.4-5): mu solves
 * 2 sum_alpha sum_n g((lambda_n - mu)/kT) c_n = n_electrons by FP64 bisection on
 * [min lambda - 1, max lambda + 1] to a bracket below 1e-14 Ha (XLS_ENOCONV if not bracketed);
 * rho (optional, global grid) = (2/dV) sum_n g_n psi_n^2 on each core point from its own
 * subdomain; E_band = 2 sum sum g c lambda; E_entropy = -2 kT sum sum c s(g). */
xls_status xls_density(xls_grid g, double n_electrons, double kT, double* mu_out, double* rho_out,
                       int rho_on_device, double* e_band_out, double* e_entropy_out);

/* Read back lambda (ascending) and c of subdomain `sub` (N_s doubles each; either may be NULL). */
xls_status xls_get_eigs(xls_grid g, int sub, double* lambda_out, double* c_out);

/* Density of states (Eq. dos, Sec. 5.A.4 "Postprocessing"): D(E) = 2 sum_alpha sum_n c_n
 * delta(E - lambda_n) over the Ritz values and interior weights of every subdomain from the last
 * pass, the delta function broadened to a normalised Gaussian of width `width` (Ha, > 0).
 * energies: n_energies host doubles (Ha); dos_out: n_energies host doubles (states per Ha).
 * Synchronous on the grid's stream.  XLS_EINVAL for a non-positive width or missing arrays. */
xls_status xls_dos(xls_grid g, const double* energies, int n_energies, double width, double* dos_out);

/* Read back M_s and H_s (N_s x N_s, row-major) of subdomain `sub` from the last projection. */
xls_status xls_get_subspace(xls_grid g, int sub, double* Ms_out, double* Hs_out);

/* Read back the N_s x N_s rotation Y of subdomain `sub` from the last generalised eigensolve
 * (row-major; the rotated block is psi_n = sum_k Y[k][n] psi_f,k, Sec. 5.A.3 step (4): Psi = Psi_f Y).
 * Test/readback helper; XLS_EINVAL in wave mode. */
xls_status xls_get_rotation(xls_grid g, int sub, double* Y_out);

/* Read back the work arrays of subdomain `sub`'s last generalised eigensolve (test/readback
 * helper, Sec. 5.A.3 step (3)): L_out the Cholesky factor of M_s (lower, N_s x N_s row-major),
 * A_out the reduced matrix after the tridiagonalisation (the Householder vectors below the
 * subdiagonal), vecs_out [8*N_s]: the tridiagonal's diagonal, off-diagonal, Householder scalars,
 * the FP32 bisection estimates of its eigenvalues, the cluster starts (then the cluster count and
 * the norm estimate).  Any pointer may be NULL.  In wave carry mode: subdomains of the last wave
 * run; XLS_EINVAL otherwise in wave mode. */
xls_status xls_get_eig_work(xls_grid g, int sub, double* L_out, double* A_out, double* vecs_out);

/* Read back the (b, a, a0) filter bounds the next pass will use, [3*n_sub]. */
xls_status xls_get_bounds(xls_grid g, double* bounds_out);

/* Per-stage device time (ms) of the last xls_chefsi_batch pass: [filter, projection, eigensolve,
 * rotation+weights] and the number of kernel launches of that pass. */
xls_status xls_get_timings(xls_grid g, double* ms4_out, int* launches_out);

/* Turn on (1) or off (0) per-kernel timing: CUDA events around every launch of each pass on
 * the grid's stream (a few microseconds of overhead per launch).  In wave carry mode it times the
 * worker's passes (xls_get_kernel_times then reads the last wave's); in store mode XLS_EINVAL.
 * Library-specific: the paper has no counterpart; it feeds roofline measurements. */
xls_status xls_set_profiling(xls_grid g, int on);

/* Parameters of the self-consistent-field iteration (Sec. 5.A.4, Sec. 5.B.3 SCF): electron count
 * n_electrons, smearing kT (Ha), filter degree and CheFSI passes per SCF step, mixing weight beta,
 * Kerker constant kappa (1/bohr), Pulay history (1..8) and Pulay period (a Pulay extrapolation
 * every pulay_period-th step, preconditioned linear mixing otherwise).  Requires
 * xls_hamiltonian_set (the atoms give the pseudocharge; the projectors stay fixed across steps)
 * and resets the mixing history.  Device memory for the global-grid fields and the history
 * (3 * history + 16 arrays of the global grid, FP64) is taken on the first call.
 * Errors: XLS_EINVAL (bad values, no Hamiltonian), XLS_ENOMEM. */
xls_status xls_scf_setup(xls_grid g, double n_electrons, double kT, int degree, int n_passes, double beta,
                         double kappa, int history, int pulay_period);

/* One SCF step (Sec. 5.A.4; Eq. poisson): from the input density rho_inout (global grid,
 * [n_z][n_y][n_x] FP64, host pointer, or device pointer with rho_on_device = 1):
 *   phi:   -Delta_h phi = 4 pi (rho + b) on the periodic grid, zero mean (conjugate gradients to
 *          a relative residual of 1e-13), b the Gaussian pseudocharge of the atoms renormalised to
 *          -sum Z with its mean removed;
 *   V_eff = phi + v_xc[rho] (LDA: Slater exchange, Perdew-Zunger 1981 correlation), restricted to
 *          every subdomain; new Lanczos upper bounds; n_passes CheFSI passes;
 *   mu, rho_out, E_band, E_entropy as xls_density;
 *   energy = E_band + E_xc[rho] - sum v_xc rho dV + 1/2 sum (b - rho) phi dV - E_self - E_entropy
 *          (input density; E_self = 1/2 sum_I Z_I^2 sqrt(2/pi) / r_c,I);
 *   residual = ||rho_out - rho||_2 / ||rho_out||_2;
 *   rho_inout <- periodic Pulay mix of (rho, rho_out) with preconditioner
 *          P = -Delta_h (-Delta_h + kappa^2)^-1 (solved by conjugate gradients).
 * Outputs may be NULL.  Errors: XLS_EINVAL (no setup, no orbitals), XLS_ENOCONV (Fermi level or
 * conjugate gradients), XLS_ENONFINITE, XLS_ENOTSPD, XLS_ECUDA. */
xls_status xls_scf_step(xls_grid g, double* rho_inout, int rho_on_device, double* residual_out, double* energy_out,
                        double* mu_out);

/* Conjugate-gradient iterations spent by the SCF steps so far (Poisson and Kerker solves).  The
 * solves are preconditioned by one FP32 multigrid V-cycle of the 7-point operator per iteration
 * (Sec. 5.B "Poisson solver": FP64 CG, FP32 V-cycle); with the environment variable
 * XLS_SCF_PLAIN_CG=1 set when the SCF state is first set up they are plain CG. */
xls_status xls_scf_cg_iterations(xls_grid g, long long* iterations_out);

/* FP16 warm-start storage of one subdomain's current orbitals (Sec. 5.B.3: orbitals kept in FP16
 * between SCF steps): vector v is stored as half(psi_v * 2^e_v), with the power of two e_v
 * (exp_out[v]) placing max |psi_v| 2^e_v in [2^13, 2^14); half_out holds n_states x N_d
 * IEEE binary16 values (vector-major, x fastest), host memory.  Relative error per element
 * <= 2^-11 of the vector's largest entry.  Loading converts back into the grid's block
 * (FP32 or FP64) and keeps the filter bounds of the last pass (a warm start).  Library-
 * specific layout; not available in wave mode.  Errors: XLS_EINVAL, XLS_ECUDA. */
xls_status xls_orbitals_store_fp16(xls_grid g, int sub, uint16_t* half_out, int* exp_out);
xls_status xls_orbitals_load_fp16(xls_grid g, int sub, const uint16_t* half_in, const int* exp_in);

/* Self-test of the failure path every bounded device wait of the library takes: a kernel waits
 * on a shared-memory barrier that nothing completes, gives up after spin_limit tries
 * (1..2^20; each try returns after a short hardware-defined time) and records XLS_ETIMEOUT, which
 * this call returns.  No fault, no trap; the context stays usable.  Library-specific: the paper
 * has no counterpart.  Errors: XLS_EINVAL, XLS_ECUDA. */
xls_status xls_selftest_wait(int spin_limit, void* cuda_stream);

/* ---- Fermi level across grids (Sec. 5.A.5, "Chemical potential": a histogram of the eigenvalues
 * narrows the bracket, then Newton steps on N_e(mu) with dN_e/dmu, each needing only global sums of
 * two scalars).  These calls give one grid's contribution; the host combines the contributions of
 * the grids of all ranks (for instance by an allreduce) and steers the iteration.  Library-
 * specific split of xls_density, which does the whole solve on one grid. */
/* out4 = [2 sum c g((lambda - mu)/kT), 2 sum c g (1 - g) / kT, min lambda, max lambda] over the
 * grid's states (FP64; g the Fermi-Dirac function). */
xls_status xls_fermi_partial(xls_grid g, double mu, double kT, double* out4);
/* hist_out[b] = 2 sum of the weights c over the states with lambda in bin b of n_bins equal bins
 * of [lo, hi) (states below lo in bin 0, at or above hi in the last bin); n_bins <= 4096. */
xls_status xls_fermi_histogram(xls_grid g, double lo, double hi, int n_bins, double* hist_out);
/* Occupations at the given mu; rho on the grid's core points ([n_z][n_y][n_x] FP64, the other
 * points 0; may be NULL); e3_out = [E_band, E_entropy, N_e] of the grid's states (may be NULL). */
xls_status xls_density_at(xls_grid g, double mu, double kT, double* rho_out, int rho_on_device, double* e3_out);

/* Waves of the grid (Sec. 5.B.3: subdomains processed in batches that fit the node): 1 when every
 * subdomain is resident at once, else the number of waves of consecutive subdomains admitted by
 * the HBM budget given to xls_grid_create; first_sub_out (optional, n_sub entries suffice)
 * receives each wave's first subdomain.  In wave mode the orbitals of all subdomains live in a
 * pinned host store in the device format (FP32 on the mixed path, FP64 otherwise);
 * xls_chefsi_batch runs the waves in turn (per wave: a partial grid, the projector tables and
 * Lanczos bounds of its subdomains, orbitals up, passes, orbitals, Ritz values, weights and
 * bounds back), xls_density finds mu from all Ritz values and weights on the device and forms
 * rho from the core rows of every subdomain's orbitals, gathered on the device after its wave's
 * passes when they take at most an eighth of the HBM budget (else in a second sweep over the
 * stored orbitals, as also after the store's format changed); xls_scf_step solves the global-grid parts as
 * on a resident grid and runs the passes in waves (each wave's partial grid restricts the new
 * V_eff and takes its own Lanczos upper bound).  xls_chefsi_stage, xls_hamiltonian_apply,
 * xls_get_subspace and profiling return XLS_EINVAL in wave mode.
 * Library-specific: the paper batches subdomains per MPI rank instead. */
xls_status xls_get_waves(xls_grid g, int* n_waves_out, int* first_sub_out);

/* Wave mode only: carry mode with `slots` subdomains per wave (slots > 0: that many, a divisor of
 * the subdomain count; slots < 0: the largest divisor whose worker and core store fit the HBM
 * budget given at creation) or store mode (slots == 0, the default).  In carry mode the
 * grid keeps no copy of the orbitals between waves: one worker grid of W subdomain slots is
 * allocated once and re-targeted to each wave in turn (its descriptors moved, V_eff restricted,
 * projector tables rebuilt and the Lanczos bound taken for the wave's subdomains), and every
 * wave's passes start from the rotated block the previous wave left in the worker -- the restart
 * of a crystal's subdomains from a neighbouring subdomain's subspace, for subdomains too many for
 * the host to keep (the 1,728 subdomains of 72^3 points with 528 states of a 13,824-atom cell
 * would need 1.4 TB of FP32 orbitals).  xls_orbitals_random draws the first wave's start block
 * (the first pass then takes (a, a0) from a Rayleigh-Ritz step of it); later waves take a and a0
 * from the subdomain's own last pass, or from the slot's last pass on the first cycle.  After
 * each wave the core rows of every subdomain's orbitals go to a device store (core points x
 * N_s values per subdomain, the compute precision), from which xls_density forms rho after the
 * Fermi level of all subdomains.  Every subdomain must have the shape of subdomain 0 (points,
 * boundaries, core box, states); the waves become equal.  Switching the mode or the slot count
 * drops the orbitals (xls_orbitals_random again).  xls_orbitals_set and xls_orbitals_get return
 * XLS_EINVAL in carry mode.  Errors: XLS_EINVAL (not a wave grid, unequal shapes, a slot count
 * that does not divide the subdomain count), XLS_ENOMEM (the slots and the core store exceed the
 * budget).  Sec. 5.A.5
 * "Parallel CheFSI" (subdomains processed independently); the restart between waves is
 * library-specific. */
xls_status xls_wave_carry(xls_grid g, int slots);

/* Wave mode only: the passes of one wave (waves numbered as xls_get_waves lists them): in store
 * mode the wave's orbitals go up from the host store and come back; in carry mode the worker is
 * re-targeted to the wave and starts from the block the previous call left.  Ritz values,
 * weights and bounds of the wave's subdomains are kept; xls_density needs every wave to have run
 * since the last xls_hamiltonian_set.  bounds: optional [3*n_sub] (b, a, a0) of every subdomain
 * (only the wave's entries are read).  Library-specific (a unit of work sized to the HBM budget). */
xls_status xls_chefsi_wave(xls_grid g, int wave, int degree, int n_passes, const double* bounds);

/* Wave mode only: keep the host store of the orbitals in FP16 (on != 0) or in the compute
 * precision (on == 0).  FP16: every vector v of a subdomain is stored as half(psi_v 2^e_v) with
 * the power of two e_v putting max |psi_v| 2^e_v into [2^13, 2^14) (the FP16 warm-start storage of
 * Sec. 5.B.3), half the FP32 store (the exponents stay in device memory); conversions run on the
 * device when a wave's orbitals go up or come back.  Orbitals already stored are converted.  XLS_EINVAL on a resident grid, XLS_ENOMEM
 * if the new pinned store cannot be allocated. */
xls_status xls_wave_store_fp16(xls_grid g, int on);

/* ---- learned SCF start (Sec. 5.A.4, SCF initialisation: superposed atomic densities plus a
 * learned, material-specific correction).  The paper names the idea, not the model; this library
 * fixes: per grid point 2 species x 16 radial descriptors
 *   d_{s,k}(x) = sum_{I in s} exp(-(r_I - r_k)^2 / (2 * 0.25^2)) f_c(r_I), r_k = k * 6/15 bohr,
 *   f_c(r) = (cos(pi r / 6) + 1) / 2 for r < 6 bohr, minimum-image r_I;
 * a 32 -> 64 -> 64 -> 64 -> 1 MLP with tanh hidden layers and a linear output; parameters as
 * W1 (32 x 64, row = input), b1 (64), W2 (64 x 64), b2, W3 (64 x 64), b3, w4 (64), b4 (1):
 * 10497 values. */

/* Model from host parameters (FP64 in, FP32 master copy on the device; Adam moments zero).
 * cuda_stream may be NULL.  Errors: XLS_EINVAL (n_params != 10497), XLS_ENOMEM. */
xls_status xls_mlp_create(const double* params, int n_params, void* cuda_stream, xls_mlp* out);
xls_status xls_mlp_destroy(xls_mlp m);
/* Current parameters (10497 values, FP32 master copy widened). */
xls_status xls_mlp_get_params(xls_mlp m, double* params_out);
/* Inference with BF16 operands (inputs, weights, hidden activations rounded to BF16) and FP32
 * accumulation: y[p] = MLP(X[p]), X row-major [n][32] FP32.  Host or device arrays
 * (on_device = 1: both X and y on the device).  Work arrays grow to n points. */
xls_status xls_mlp_infer(xls_mlp m, const float* X, long long n, float* y_out, int on_device);
/* FP32 training quantities: loss = mean_p (MLP(X[p]) - y[p])^2 and its gradient (10497 values,
 * host; may be NULL).  Backpropagation per point, weight gradients as fixed-order batch sums. */
xls_status xls_mlp_loss_grad(xls_mlp m, const float* X, const float* y, long long n, double* loss_out,
                             double* grad_out, int on_device);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the loss above; loss_out
 * receives the loss before the step. */
xls_status xls_mlp_train_step(xls_mlp m, const float* X, const float* y, long long n, double lr, double* loss_out,
                              int on_device);
/* Descriptors of the grid's atoms (from xls_hamiltonian_set; species indices 0 and 1) at every
 * global grid point, [n_z n_y n_x][32] FP32 (x fastest), host or device output. */
xls_status xls_descriptors(xls_grid g, float* X_out, int on_device);
/* Start density rho_0 = max(rho_SAD + MLP(d), 0) renormalised to sum rho dV = n_electrons, with
 * rho_SAD the superposed normalised Gaussians of Z_v electrons and width r_c (the species' local
 * radius), itself renormalised to n_electrons; m = NULL gives rho_SAD alone (the fallback).
 * Global grid FP64 [n_z][n_y][n_x], host or device. */
xls_status xls_learned_start(xls_grid g, xls_mlp m, double n_electrons, double* rho_out, int on_device);

/* Turn on (1) or off (0) CUDA-graph replay of the CheFSI pass (Sec. 5.A.3 steps (1)-(4) as one
 * graph: filter, projection, eigensolve, rotation).  With graphs on, xls_chefsi_batch captures a
 * pass the first time it meets a given (orbital block, degree) and replays the graph afterwards;
 * the captured kernels read the filter bounds, coefficients and orbitals from device memory, so
 * replays follow every change of those.  xls_hamiltonian_set and turning graphs off drop the
 * captured graphs (after synchronising the grid's stream).  While profiling is on, passes are
 * launched directly.  A grid created on the legacy default stream captures on a private stream
 * and replays on the legacy stream.  Library-specific: the paper has no counterpart.
 * Errors: XLS_EINVAL (null grid), XLS_ECUDA (capture or instantiation failed). */
xls_status xls_set_graphs(xls_grid g, int on);

/* Device time (ms) and launch count per kernel class in the last profiled pass: [0] stencil,
 * [1] nonlocal projection, [2] nonlocal back-projection, [3] Gram/projection GEMM,
 * [4] eigensolve, [5] rotation GEMM, [6] other, [7] unused.  Either pointer may be NULL. */
xls_status xls_get_kernel_times(xls_grid g, double* ms8_out, int* count8_out);

/* Allocation-free Gram of one block of vectors (the paper has no counterpart: a service for
 * callers that cannot let a library allocate device memory, e.g. applications whose device
 * memory is owned by their own pool allocator, or latency-critical loops that cannot accept
 * the implicit synchronisation of cudaMalloc/cudaFree).
 *   psi_f, hpsi_f: device FP32 blocks F and HF, n_states x n_points, vector-major, 16-byte
 *                  aligned; n_points a positive multiple of 8; 1 <= n_states <= 256.
 *   Ms_out, Hs_out: device FP64 n_states x n_states row-major: F F^T and F HF^T by the split-BF16
 *                  tensor-core kernel (FP32 accumulation, FP64 sum of the partial sums); the
 *                  off-diagonal 128 x 128 blocks are mirrored, so both outputs are symmetric.
 * It allocates nothing: its scratch is a fixed 8 MiB + 256 B device array of the library, which
 * every GPU that loads the library holds until the process exits; larger n_states are rejected
 * with XLS_EINVAL.  The first call on a device looks up that array's device address.  A CUDA
 * error already pending on the calling thread is reported as XLS_ECUDA before any work is
 * queued.  All calls share the array and it keeps the last call's
 * contents: calls that can overlap on the GPU (other host threads, other streams) race and
 * must be serialised by the caller.  The call queues its work on cuda_stream (NULL = legacy
 * default stream) and returns after it has completed. */
xls_status xls_gram_noalloc(const float* psi_f, const float* hpsi_f, long long n_points, int n_states,
                            double* Ms_out, double* Hs_out, void* cuda_stream);

/* Message of the calling thread's last failure ("" if none). */
const char* xls_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* XLS_H */
