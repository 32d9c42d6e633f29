// Internal types and launcher declarations of libxls (shared by the .cu translation units).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/xls.h"

namespace xls {

constexpr int kN0 = 6;           // stencil half-width: 12th-order FD (Sec. 5.B.2, n0 = 6)
constexpr int kMaxStates = 1024;

// Per-subdomain descriptor, resident on the device.  All offsets are in elements.
struct SubDev {
  int n[3];              // local grid points per axis
  int periodic[3];       // 1 = periodic along the axis (subdomain spans the period)
  int start[3];          // global index of local point 0
  int core_lo[3];        // local index of the first core point
  int core_n[3];
  int core_glo[3];       // global index of the first core point
  int ns;                // vectors in this view (N_s, or 1 for single-vector views)
  int off_state;         // offset into per-state arrays (lambda, c)
  long long nd;          // points
  long long off_blk;     // offset of this subdomain's block in a block arena (ns * nd elements)
  long long off_pt;      // offset into per-point arrays (V)
  long long off_ss;      // offset into N_s x N_s arrays
  int slot_lo, slot_n;   // range in the projector-slot array (one slot per atom meeting the subdomain)
  long long off_proj;    // offset into the projection array P (4 * ns per slot)
  double h[3];
  double dV;
};

// One periodic image of an atom whose projector sphere meets a subdomain.
struct AtomImg {
  double R[3];           // position in the subdomain's local frame: x_local(i) = i * h
  int box_lo[3];         // first local index of the bounding box (may be < 0 on periodic axes)
  int box_n[3];          // box points per axis (clipped to the subdomain on Dirichlet axes)
  int slot;              // projector slot (atom) this image belongs to
};

// The projectors of one atom in one subdomain: the periodic function sum_T chi(x - R - T)
// restricted to the subdomain, i.e. every image of the atom that meets it, with one
// projection coefficient per (projector, vector).
struct ProjSlot {
  int sub;               // owning subdomain
  int atom;              // global atom index
  int img_lo, img_n;     // range in the image array
  double w, rcut2;       // projector width and squared cutoff
  double norm[4];        // grid normalisation of chi_s, chi_px, chi_py, chi_pz
  double E[4];           // KB energies E_s, E_p, E_p, E_p
};

// Coefficients of one filter step: Y_out = scale * (H - c) Y_in - shift * Y_prev.
struct StepCoef {
  double scale, c, shift, pad;
};
constexpr int kMaxDegree = 64;

// Launch plan of a block-wise kernel over all subdomains of a view: prefix of CTA counts.
struct Plan {
  int* d_blk_off = nullptr;   // [n_sub + 1]
  int total = 0;
};

// ---- launchers (filter / operator) --------------------------------------------------------
template <typename T>
void launch_stencil(const SubDev* d_subs, int n_sub, const Plan& plan, const T* Yin, const T* Yprev,
                    T* Yout, const T* V, const StepCoef* coef, int step, cudaStream_t st);
template <typename T>
void launch_nl_project(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const AtomImg* d_imgs, int max_ns,
                       const T* Y, double* P, cudaStream_t st);
template <typename T>
void launch_nl_back(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const AtomImg* d_imgs, int max_ns,
                    const double* P, T* Yout, const StepCoef* coef, int step, cudaStream_t st);
int stencil_blocks(const int n[3], int ns);

// ---- dense subspace work -------------------------------------------------------------------
template <typename T>
void launch_gram(const SubDev* d_subs, int n_sub, int max_ns, long long max_nd, const T* F, const T* HF,
                 double* Ms, double* Hs, cudaStream_t st);
template <typename T>
void launch_rotate(const SubDev* d_subs, int n_sub, int max_ns, long long max_nd, const T* F, const double* Y,
                   T* Out, cudaStream_t st);
template <typename T>
void launch_core_weights(const SubDev* d_subs, int n_sub, int max_ns, const T* Psi, double* c, cudaStream_t st);
template <typename T>
void launch_density_occ(const SubDev* d_subs, int n_sub, long long max_core, const T* Psi, const double* occ,
                        const int gn[3], double* rho, cudaStream_t st);
void launch_fermi_occ(const double* lam, const double* c, int n_tot, double n_e, double kT, double* out4, double* occ,
                      int* status, cudaStream_t st);

// ---- eigensolver (FP64) --------------------------------------------------------------------
// L (in: M_s, out: Cholesky factor), A (in: H_s, out: reflectors), W (workspace/Z), Y (out),
// R (cluster workspace), all n x n per subdomain; lam (out); vecs 8n per subdomain.
void launch_eig(const SubDev* d_subs, int n_sub, int max_ns, double* L, double* A, double* Y, double* W, double* lam,
                double* vecs, int* status, double* scratch, double* R, cudaStream_t st);
size_t eig_scratch_doubles(int n_sub, int max_ns);

// ---- small kernels -------------------------------------------------------------------------
void launch_filter_coef(int n_sub, const double* bounds, int degree, StepCoef* coef, cudaStream_t st);
void launch_bounds_from_ritz(const SubDev* d_subs, int n_sub, const double* lam, double* bounds, cudaStream_t st);
void launch_restrict(const SubDev* d_subs, int n_sub, long long max_nd, const double* Vg, const int gn[3],
                     double* V, float* Vf, cudaStream_t st);
void launch_proj_norms(const AtomImg* d_imgs_global, const ProjSlot* d_slots_global, int n_atoms, const int gn[3],
                       const double gh[3], double* norms, cudaStream_t st);
void launch_splitmix_fill_f64(double* out, long long count, uint64_t seed, long long offset, cudaStream_t st);
void launch_splitmix_fill_f32(float* out, long long count, uint64_t seed, long long offset, cudaStream_t st);
void launch_convert_f64_f32(const double* in, float* out, long long count, cudaStream_t st);
void launch_convert_f32_f64(const float* in, double* out, long long count, cudaStream_t st);
// Lanczos helpers on single-vector views (FP64)
void launch_lanczos_step(const SubDev* d_subs, int n_sub, int j, const double* Hv, double* v, double* vprev,
                         double* f, double* alpha, double* beta, cudaStream_t st);
void launch_lanczos_init(const SubDev* d_subs, int n_sub, double* v, cudaStream_t st);
void launch_lanczos_finish(int n_sub, int k, const double* alpha, const double* beta, const SubDev* d_subs,
                           const double* f, double* bounds, cudaStream_t st);

}  // namespace xls
