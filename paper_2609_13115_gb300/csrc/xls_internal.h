// Internal types and launcher declarations of libxls (shared by the .cu translation units).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

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
  int off_nlb;           // first back-projection point block of the subdomain (blocks of kBackPts points)
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
  long long pt_off;      // first entry of this slot's point table
  int pt_n;              // points of the table (grid points of the subdomain inside any image's sphere)
  int pad;
  double w, rcut2;       // projector width and squared cutoff
  double norm[4];        // grid normalisation of chi_s, chi_px, chi_py, chi_pz
  double E[4];           // KB energies E_s, E_p, E_p, E_p
};

// Coefficients of one filter step: Y_out = scale * (H - c) Y_in - shift * Y_prev.
struct StepCoef {
  double scale, c, shift, pad;
};
constexpr int kMaxDegree = 64;

// TMA stencil: subdomains grouped in classes of equal tile shape (one launch per class).
struct TmaJob {
  int sub;        // subdomain
  int n_ytiles;   // row tiles per vector
  int W;          // staged row width (floats)
  int TY;         // rows per tile
};
constexpr int kMapsPerSub = 10;  // TMA stencil tensor maps per subdomain (3 per block + V)
struct TmaClass {
  int nq = 0, TY = 0, W = 0;   // threads per row (x-points / 4), rows per tile, row width
  double h[3] = {0, 0, 0};     // grid spacing shared by the class
  int n_jobs = 0, total = 0;   // subdomains and CTAs of the class
  int rt_pitch = 1;            // 1: the runtime-pitch variant (the default: it measured faster for
                               // 48- and 72-point rows); 0: the compile-time variant where one exists
  TmaJob* d_jobs = nullptr;
  int* d_job_off = nullptr;    // [n_jobs + 1] CTA prefix
};

// Tensor-core Gram: CTA jobs (subdomain, 128x128 block (I <= J), range of 64-point K tiles);
// jobs of one (subdomain, block) are consecutive and form a reduction group.
struct GramJob {
  int sub, I, J, kt0, kt1, pad;
};
struct GramPlan {
  int n_jobs = 0, n_groups = 0;
  int cap_jobs = 0;            // job capacity of the device arrays (the finest K split tried)
  GramJob* d_jobs = nullptr;
  int* d_grp_first = nullptr;
  int* d_grp_n = nullptr;
  float* d_work = nullptr;     // [n_jobs][2][128][128] FP32 partial sums
  int* d_ex_f = nullptr;       // FP16 split: power-of-two exponent of every vector of F and HF
  int* d_ex_hf = nullptr;
};
// Tensor-core rotation: CTA jobs (subdomain, tile of 128 grid points, first of up to 256 output
// states)
struct RotJob {
  int sub, tile, n0;
};
struct RotPlan {
  int n_jobs = 0, kpad_max = 0;
  RotJob* d_jobs = nullptr;
  uint16_t* d_yhi = nullptr;   // Y^T split into bf16 hi / lo, [states][kpad_max]
  uint16_t* d_ylo = nullptr;
  int* d_ex_y = nullptr;       // FP16 split: exponent of every row of Y^T
};
void set_last_error(const std::string& m);
bool tc_setup();
int gram_single_pairs(int n_states);
bool launch_gram_tc_single(const float* F, const float* HF, long long n_points, int n_states, int kc, float* work,
                           double* Ms, double* Hs, int* status, cudaStream_t st);
void launch_gram_tc(const SubDev* d_subs, int n_sub, int max_ns, const GramPlan& gp, bool fp16, const float* F,
                    const float* HF, double* Ms, double* Hs, int* status, cudaStream_t st);
void launch_rotate_tc(const SubDev* d_subs, int n_sub, int max_ns, const RotPlan& rp, const GramPlan& gp, bool fp16,
                      bool need_exponents, const float* F, const double* Y, float* Out, int* status, cudaStream_t st);

// Launch plan of a block-wise kernel over all subdomains of a view: prefix of CTA counts.
struct Plan {
  int* d_blk_off = nullptr;   // [n_sub + 1]
  int total = 0;
};

// ---- launchers (filter / operator) --------------------------------------------------------
template <typename T>
void launch_stencil(const SubDev* d_subs, int n_sub, const Plan& plan, const T* Yin, const T* Yprev,
                    T* Yout, const T* V, const StepCoef* coef, int step, cudaStream_t st);
// Projector tables: for every slot, its grid points (local flat index) and the four chi values
// there, in the precision T of the block (chi of type T4: double4 / float4).
template <typename T> struct Vec4;
template <> struct Vec4<double> { using type = double4; };
template <> struct Vec4<float> { using type = float4; };
template <typename T>
void launch_proj_table_count(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const AtomImg* d_imgs,
                             int* counts, cudaStream_t st);
template <typename T>
void launch_proj_table_fill(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const AtomImg* d_imgs,
                            int* idx, typename Vec4<T>::type* chi, cudaStream_t st);
template <typename T>
void launch_nl_project(const SubDev* d_subs, const ProjSlot* d_slots, int slot_off, int n_slot, const int* idx,
                       const typename Vec4<T>::type* chi, int max_ns, const T* Y, double* P, int kpv, int nw,
                       int chunk_slots, cudaStream_t st);
void launch_rcsr_count(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const int* idx, int* cnt,
                       cudaStream_t st);
template <typename T>
void launch_rcsr_build(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const int* idx,
                       const typename Vec4<T>::type* chi, const long long* row_ptr, int* cursor, int* rslot,
                       typename Vec4<T>::type* rchi, cudaStream_t st);
// back-projection point blocks: the slots each block's reverse-table rows name, and the rows'
// slot entries rewritten to ranks in that list (pass 0 counts, pass 1 ranks and lists)
constexpr int kBackPts = 2048;
// exclusive prefix sum of n counts into rp[0..n] on the device; tmp holds scan_temp_count(n) values
long long scan_temp_count(long long n);
void launch_exclusive_scan(const int* cnt, long long n, long long* tmp, long long* rp, cudaStream_t st);
void launch_rcsr_localize(const SubDev* d_subs, const int* d_blk_sub, int n_blk, const long long* row_ptr,
                          int* rslot, int* blk_cnt, int* blk_list, int list_max, int pass, cudaStream_t st);
template <typename T>
void launch_nl_back_csr(const SubDev* d_subs, int n_sub, long long max_nd, int max_ns, int list_max,
                        const long long* row_ptr, const int* rslot, const typename Vec4<T>::type* rchi,
                        const int* blk_cnt, const int* blk_list, const double* P, T* Yout, const StepCoef* coef,
                        int step, int variant, cudaStream_t st);   // variant: 1 (1 point x 8 vectors), 2 (2 x 8), 16 (1 x 16)
// single-vector views (ns = 1 per subdomain): one warp per slot; one thread per grid point
template <typename T>
void launch_nl_project1(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const int* idx,
                        const typename Vec4<T>::type* chi, const T* Y, double* P, cudaStream_t st);
template <typename T>
void launch_nl_back1(const SubDev* d_subs, int n_sub, long long max_nd, int list_max, const long long* row_ptr,
                     const int* rslot, const typename Vec4<T>::type* rchi, const int* blk_list, const double* P,
                     T* Yout, const StepCoef* coef, int step, cudaStream_t st);
template <typename T>
void launch_nl_back(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const int* idx,
                    const typename Vec4<T>::type* chi, int max_ns, const double* P, T* Yout, const StepCoef* coef,
                    int step, cudaStream_t st);
int stencil_blocks(const int n[3], int ns);
}  // namespace xls
struct CUtensorMap_st;
namespace xls {
bool tma_eligible(const SubDev& S);
int tma_tile_rows(const SubDev& S);
int tma_row_width(const SubDev& S);
bool build_tma_maps(const SubDev& S, const float* Vf, void* const bufs[3], struct CUtensorMap_st* out);
void launch_stencil_tma(const SubDev* d_subs, const TmaClass& cls, const struct CUtensorMap_st* d_maps, int buf_in,
                        int buf_prev, float* Yout, const StepCoef* coef, int step, int* status, cudaStream_t st);

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
void launch_core_gather(const SubDev* d_subs, int n_sub, int max_ns, const T* Psi, T* store, const SubDev* d_dst,
                        cudaStream_t st);
template <typename T>
void launch_density_occ(const SubDev* d_subs, int n_sub, long long max_core, const T* Psi, const double* occ,
                        const int gn[3], double* rho, cudaStream_t st);
void launch_dos(const double* lam, const double* c, int n, const double* energies, int n_e, double w, double* out,
                cudaStream_t st);
void launch_fermi_occ(const double* lam, const double* c, int n_tot, double n_e, double kT, double* out4, double* occ,
                      int* status, cudaStream_t st);

// ---- eigensolver (FP64) --------------------------------------------------------------------
// L (in: M_s, out: Cholesky factor), A (in: H_s, out: reflectors), W (workspace/Z), Y (out),
// R (cluster workspace), all n x n per subdomain; lam (out); vecs 8n per subdomain.
bool launch_cholesky_cluster(const SubDev* d_subs, int n_sub, int max_ns, double* Ms, int* status, int cl_first,
                             cudaStream_t st);
bool launch_tridiag_cluster(const SubDev* d_subs, int n_sub, int max_ns, double* A, double* vecs, int cl_first,
                            cudaStream_t st);
// ---- learned start ---------------------------------------------------------------------------
}  // namespace xls
// model handle: FP32 master parameters, Adam moments and the training work arrays
struct xls_mlp_s {
  cudaStream_t st = nullptr;
  int n_params = 0;
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  int t = 0;                              // Adam steps taken
  long long cap = 0;                      // points the work arrays hold
  float *A = nullptr, *D = nullptr, *e = nullptr, *wpartial = nullptr, *X = nullptr, *y = nullptr, *yp = nullptr;
  double *loss_partial = nullptr, *loss = nullptr;
};
namespace xls {
xls_status mlp_reserve(xls_mlp_s* m, long long n);
int mlp_param_count();
size_t mlp_wpartial_floats();
void launch_descriptors(long long n, const int gn[3], const double gh[3], const double gL[3], const float4* atoms,
                        int n_atoms, int n_species, float* X, cudaStream_t st);
void launch_mlp_infer(long long n, const float* theta, const float* X, float* y, cudaStream_t st);
void launch_mlp_grad(long long n, const float* theta, const float* X, const float* yt, float* A, float* D, float* e,
                     double* loss_partial, float* wpartial, float* grad, double* loss_out, cudaStream_t st);
void launch_adam(int n, float* theta, float* m, float* v, const float* g, float lr, int t, cudaStream_t st);
void launch_add_clamp(long long n, const double* sad, const float* corr, double* rho, cudaStream_t st);

// ---- SCF on the global grid -----------------------------------------------------------------
void launch_dots(long long n, const double* const* x, const double* const* y, int nq, double* partial, double* out,
                 double scale, cudaStream_t st);
void launch_sum(long long n, const double* x, double* partial, double* out, cudaStream_t st);
void launch_axpbypcz(long long n, double a, const double* x, double b, double* y, double c, const double* z,
                     cudaStream_t st);
void launch_sub_mean(long long n, const double* sum, double* y, cudaStream_t st);
void launch_cg_xr(long long n, const double* s, double* x, double* r, const double* p, const double* q,
                  double* partial, cudaStream_t st);
void launch_cg_p(long long n, double* s, const double* r, double* p, cudaStream_t st);
int mg_level_count(const int n[3]);
size_t mg_floats(const int n[3]);
void launch_mg_vcycle(const int n[3], const double h[3], double sigma, const double* r, double* z, float* work,
                      cudaStream_t st);
void launch_pcg_p(long long n, double* s, const double* z, double* p, cudaStream_t st);
void launch_lda(long long n, const double* rho, double* eps, double* vxc, cudaStream_t st);
void launch_pseudocharge(int n_atoms, const double* d_pos, const double* d_rc, const double* d_amp, const int gn[3],
                         const double gh[3], const double gL[3], double* g1, double* b, double z_total, double* partial,
                         double* s4, cudaStream_t st);
size_t pulay_partial_doubles();
void launch_gaussian_density(int n_atoms, const double* d_pos, const double* d_rc, const double* d_amp, const int gn[3],
                             const double gh[3], const double gL[3], double* g1, double* out, double total,
                             double* partial, double* s4, cudaStream_t st);
void launch_rescale(long long n, const double* sum, double target, double* y, cudaStream_t st);
void launch_pulay(long long n, int m, const double* dF, const double* dX, const double* dPF, const double* f, double beta,
                  double* partial, double* gamma, double* x, cudaStream_t st);
constexpr int kRedPartials = 296 * 4;  // doubles of a reduction's partial-sum buffer

void launch_eig(const SubDev* d_subs, int n_sub, int max_ns, double* L, double* A, double* Y, double* W, double* lam,
                double* vecs, int* status, double* scratch, double* R, int cluster, cudaStream_t st);
size_t eig_scratch_doubles(int n_sub, int max_ns);

// ---- small kernels -------------------------------------------------------------------------
void launch_wait_selftest(int spin_limit, int* status, cudaStream_t st);
template <typename T>
void launch_store_half(const T* X, long long nd, int ns, int* ex, void* out, cudaStream_t st);
template <typename T>
void launch_load_half(const void* in, long long nd, int ns, const int* ex, T* X, cudaStream_t st);
void launch_fermi_partial(const double* lam, const double* c, int n, double mu, double kT, double* out,
                          cudaStream_t st);
void launch_fermi_hist(const double* lam, const double* c, int n, double lo, double hi, int nb, double* hist,
                       cudaStream_t st);
void launch_occ_at(const double* lam, const double* c, int n, double mu, double kT, double* occ, double* out,
                   cudaStream_t st);
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
