// libxls C ABI: grid handle, restriction/projector set-up, CheFSI pass orchestration over all
// subdomains (one launch per stage), Fermi level and density.  Host code only orchestrates;
// every arithmetic step of the pass runs in the kernels of k_filter.cu, k_dense.cu, k_eig.cu
// and k_tc.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include <cuda.h>
#include <cstdlib>

#include "xls_internal.h"

using namespace xls;

namespace {

thread_local std::string g_last_error;

xls_status fail(xls_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define XLS_CUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return fail(XLS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));             \
  } while (0)

#define XLS_TRY(expr)                 \
  do {                                \
    xls_status _s = (expr);           \
    if (_s != XLS_OK) return _s;      \
  } while (0)

}  // namespace

namespace xls {
void set_last_error(const std::string& m) { g_last_error = m; }
}  // namespace xls

struct xls_grid_s {
  int prec = XLS_FP64;
  cudaStream_t st = nullptr;
  int gn[3];
  double gL[3], gh[3];
  int n_sub = 0;
  std::vector<SubDev> subs;     // main view (ns = N_s)
  std::vector<SubDev> subs1;    // single-vector view (ns = 1), for the Lanczos bound and tests
  SubDev* d_subs = nullptr;
  SubDev* d_subs1 = nullptr;
  Plan plan, plan1;
  int max_ns = 0, tot_states = 0;
  long long max_nd = 0, tot_pts = 0, tot_blk = 0, tot_ss = 0, max_core = 0;
  size_t elem = 8;              // bytes per block element (8 FP64, 4 mixed)
  void* blk[3] = {nullptr, nullptr, nullptr};
  int cur = 0;                  // block holding the current orbitals
  double* V = nullptr;
  float* Vf = nullptr;
  double *Ms = nullptr, *Hs = nullptr, *Lb = nullptr, *Ab = nullptr, *W = nullptr, *Y = nullptr, *R = nullptr;
  double *lam = nullptr, *cw = nullptr, *occ = nullptr, *vecs = nullptr, *eig_scr = nullptr;
  double* bounds = nullptr;
  StepCoef* coef = nullptr;
  int* status = nullptr;
  double* out4 = nullptr;
  double* rho = nullptr;
  double* Vg = nullptr;
  // wave mode (HBM budget below the whole footprint): waves of consecutive subdomains run on
  // partial grids; the orbitals of every subdomain live in a pinned host store (device format)
  bool wave = false;
  xls_cell cell{};
  std::vector<std::pair<int, int>> waves;   // (first subdomain, count)
  std::vector<int> dc_core_lo, dc_core_n, dc_buf, dc_ns;
  void* store = nullptr;
  // FP16 store (xls_wave_store_fp16): half(psi_v 2^e_v) per value, the exponents per state on the
  // host, converted on the device through a half staging block and an exponent array
  bool store16 = false;
  void* stage16 = nullptr;
  int* d_store_ex = nullptr;   // exponents of every stored state, kept on the device
  std::vector<double> host_bounds;
  double wave_stage_ms[4] = {0, 0, 0, 0};
  // carry mode (xls_wave_carry): no orbital store; one worker grid, re-targeted to every wave in
  // turn, whose rotated block starts the next wave's passes; the core rows of every subdomain's
  // orbitals stay on the device (compact store) for the density after the Fermi level
  bool carry = false, carry_primed = false;
  xls_grid worker = nullptr;
  void* core_store = nullptr;
  SubDev* d_core_subs = nullptr;
  // store mode: the same compact core store when it was reserved in the wave plan (core_reserve
  // bytes), filled after every wave's passes; core_fresh marks the subdomains whose core rows are
  // those of the orbitals held in the host store
  size_t core_reserve = 0;
  std::vector<char> core_fresh;
  std::vector<double> carry_ab;      // (a, a0) of every worker slot after its last pass
  std::vector<char> wave_ran;        // waves that have run since the orbitals were set
  int carry_last = -1;               // the wave the worker holds (its last run)
  // geometry of the last xls_hamiltonian_set (for the pseudocharge of the SCF step)
  std::vector<double> atom_pos;
  std::vector<int> atom_sp;
  std::vector<xls_species> species;
  // projector normalisations of the last geometry (reused while the atoms, their species
  // parameters and the grid stay the same: a carry-mode worker re-targeted to every wave)
  std::vector<double> norm_cache;
  bool norm_valid = false;
  int setup_launches = 0;   // kernels of the last xls_hamiltonian_set
  void* scr_a = nullptr;    // set-up scratch (counts, row cursors, scan partial sums), reserved
  void* scr_b = nullptr;
  void* scr_c = nullptr;
  int proj_vec = 8;         // vectors per CTA of the projection (8, 16 or 32; xls_autotune)
  int proj_warps = 4;       // warps per CTA of the projection (4 or 8; xls_autotune)
  int back_var = 1;         // back-projection variant: 1 (1 point x 8 vectors per CTA), 2 (2 x 8), 16 (1 x 16)
  int proj_chunk = 256;     // slots per chunk of the projection's CTA order (256, 512, 1024)
  // concurrent halves (XLS_CONCURRENT=1): the subdomains split in two views whose passes run on
  // two streams, half 1's filter beside half 0's projection, eigensolve and rotation
  struct View {
    int first = 0, n = 0;
    const SubDev* ds = nullptr;           // descriptors of the view (d_subs + first)
    StepCoef* coef = nullptr;             // per-subdomain arrays offset to the view
    double* bounds = nullptr;
    const CUtensorMap* maps = nullptr;
    Plan plan;                            // generic stencil
    std::vector<TmaClass> tcls;           // TMA stencil classes, jobs relative to `first`
    GramPlan gplan;
    RotPlan rplan;
    int slot_off = 0, n_slot = 0;         // projector slots (global indices)
    long long ss_off = 0, ss_n = 0;       // subspace-matrix range (doubles)
    double* eig_scr = nullptr;
    int max_ns = 0;
    long long max_nd = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
  };
  View full;
  View halves[2];
  bool concurrent = false;
  cudaEvent_t ev_fork = nullptr, ev_mid = nullptr;
  // side stream of the FP32 filter steps: the projection of a step runs beside its stencil
  cudaStream_t side_st = nullptr;
  cudaEvent_t ev_side_in = nullptr, ev_side_out = nullptr;
  // learned start: descriptors, correction, SAD and their atom tables
  float* ls_X = nullptr;
  float* ls_y = nullptr;
  float4* ls_atoms = nullptr;
  double *ls_sad = nullptr, *ls_g1 = nullptr, *ls_pos = nullptr, *ls_rc = nullptr, *ls_amp = nullptr;
  double *ls_partial = nullptr, *ls_s = nullptr;
  int ls_na = -1;
  // SCF (global periodic grid)
  struct Scf {
    bool ready = false, pc_ready = false;
    double ne = 0, kT = 0, beta = 0.3, kappa = 0.5;
    int degree = 20, passes = 1, hist = 7, period = 2, k = 0;
    SubDev gs{};
    SubDev* d_gs = nullptr;
    Plan plan;
    StepCoef* d_coef = nullptr;
    double *b = nullptr, *phi = nullptr, *eps = nullptr, *vxc = nullptr, *rho_in = nullptr, *rho_out = nullptr;
    double *zero = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *tmp = nullptr, *f = nullptr, *pf = nullptr;
    double *x_prev = nullptr, *f_prev = nullptr, *pf_prev = nullptr, *dX = nullptr, *dF = nullptr, *dPF = nullptr;
    double *partial = nullptr, *pulay_partial = nullptr, *scal = nullptr, *gamma = nullptr, *g1 = nullptr;
    double *d_pos = nullptr, *d_rc = nullptr, *d_amp = nullptr;
    double e_self = 0, z_total = 0;
    int cg_iters = 0;
    // multigrid-preconditioned CG (XLS_SCF_PLAIN_CG=1: plain CG)
    bool pcg = true;
    double *z = nullptr, *r_old = nullptr;
    float* mg = nullptr;
  } scf;
  // TMA stencil (mixed path): classes of equal tile shape and the tensor maps of every
  // (subdomain, block buffer, box height)
  bool use_tma = false;
  std::vector<TmaClass> tcls;
  CUtensorMap* d_maps = nullptr;
  // tensor-core GEMMs (mixed path): Gram and rotation can be switched to SIMT independently
  bool use_tc = false, use_tc_gram = false, use_tc_rot = false;
  bool eig_cluster = true;  // Cholesky / tridiagonalisation on CTA clusters (XLS_EIG=single: one CTA)
  int eig_cl = 8;            // cluster size tried first (8 or 16; xls_autotune)
  int gram_cps = 4;          // tensor-core Gram: K split aiming at this many CTAs per SM (xls_autotune)
  GramPlan gplan;
  RotPlan rplan;
  // projectors
  AtomImg* d_imgs = nullptr;
  ProjSlot* d_slots = nullptr;
  int n_slot = 0;
  int* d_pidx = nullptr;          // projector tables: point index, chi (FP64 and, on the mixed path, FP32)
  double4* d_chi64 = nullptr;
  float4* d_chi32 = nullptr;
  long long* d_rptr = nullptr;    // reverse tables (rows = grid points of every subdomain)
  int* d_rslot = nullptr;
  double4* d_rchi64 = nullptr;
  float4* d_rchi32 = nullptr;
  int max_slots = 0;
  // back-projection point blocks: subdomain of each block, slots per block, the blocks' slot lists
  int* d_nlb_sub = nullptr;
  int* d_nlb_cnt = nullptr;
  int* d_nlb_list = nullptr;
  int nlb_max = 0;
  double *P = nullptr, *P1 = nullptr;
  // Lanczos (single-vector view, FP64)
  double *lz_v = nullptr, *lz_vp = nullptr, *lz_f = nullptr, *lz_Hv = nullptr, *lz_a = nullptr, *lz_b = nullptr;
  bool ham_set = false, orb_set = false, have_ritz = false;
  size_t bytes = 0, budget = 0;
  std::vector<std::pair<void*, size_t>> allocs;   // device arrays of the grid and their sizes
  cudaEvent_t ev[6];
  double stage_ms[4] = {0, 0, 0, 0};
  int last_launches = 0;
  int launches = 0;
  // optional per-kernel-class timing: event pairs around every launch of the pass
  bool profiling = false;
  // CUDA graphs of one pass, keyed by (block holding Psi, degree); replayed by xls_chefsi_batch
  struct PassGraph {
    int cur, degree, cur_after, launches;
    cudaGraphExec_t exec;
  };
  bool use_graphs = false;
  std::vector<PassGraph> graphs;
  cudaStream_t cap_st = nullptr;  // capture stream when the caller's stream is the legacy stream
  void drop_graphs() {
    for (auto& pg : graphs) cudaGraphExecDestroy(pg.exec);
    graphs.clear();
  }
  std::vector<cudaEvent_t> pev;
  std::vector<int> pcls;
  size_t pused = 0;
  double kms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int kcnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  // capacity of the arrays made by reserve(): the operator tables rebuilt by every
  // xls_hamiltonian_set keep their device memory while the new tables fit (a carry-mode worker
  // re-targeted to every wave allocates them once)
  std::vector<std::pair<void*, size_t>> caps;
  template <typename P_>
  xls_status reserve(P_** p, size_t bytes_) {
    if (bytes_ == 0) bytes_ = 16;
    for (auto& c : caps)
      if (*p && c.first == (void*)*p) {
        if (c.second >= bytes_) return XLS_OK;
        c.first = nullptr;
      }
    release(p);
    const xls_status s = alloc(p, bytes_);
    if (s == XLS_OK) caps.push_back({(void*)*p, bytes_});
    return s;
  }

  template <typename P_>
  xls_status alloc(P_** p, size_t bytes_) {
    if (bytes_ == 0) bytes_ = 16;
    if (budget && bytes + bytes_ > budget)
      return fail(XLS_ENOMEM, "allocation of " + std::to_string(bytes_) + " B exceeds the HBM budget");
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes_);
    if (e != cudaSuccess) return fail(XLS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back({q, bytes_});
    bytes += bytes_;
    *p = (P_*)q;
    return XLS_OK;
  }
  // frees an array of the grid and returns its bytes to the budget
  template <typename P_>
  void release(P_** p) {
    if (!*p) return;
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i].first == (void*)*p) {
        bytes -= allocs[i].second;
        allocs.erase(allocs.begin() + i);
        break;
      }
    cudaFree(*p);
    *p = nullptr;
  }
};

namespace {

xls_status check_status(xls_grid g) {
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return fail(XLS_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(le));
  int h[2] = {0, 0};
  XLS_CUDA(cudaMemcpyAsync(h, g->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, g->st));
  XLS_CUDA(cudaStreamSynchronize(g->st));
  if (h[0] != 0) {
    XLS_CUDA(cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st));
    if (h[0] == XLS_ENOTSPD)
      return fail(XLS_ENOTSPD, "Gram matrix M_s not positive definite in subdomain " + std::to_string(h[1]));
    if (h[0] == XLS_ENOCONV) return fail(XLS_ENOCONV, "Fermi level not bracketed: N_e exceeds the states' capacity");
    if (h[0] == XLS_ETIMEOUT) return fail(XLS_ETIMEOUT, "a bounded device wait (TMA plane load) gave up");
    return fail((xls_status)h[0], "device error " + std::to_string(h[0]) + " in subdomain " + std::to_string(h[1]));
  }
  return XLS_OK;
}

xls_status make_plan(xls_grid g, const std::vector<SubDev>& v, Plan& plan) {
  std::vector<int> off(v.size() + 1, 0);
  for (size_t a = 0; a < v.size(); ++a) off[a + 1] = off[a] + stencil_blocks(v[a].n, v[a].ns);
  plan.total = off.back();
  XLS_TRY(g->alloc(&plan.d_blk_off, off.size() * sizeof(int)));
  XLS_CUDA(cudaMemcpy(plan.d_blk_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  return XLS_OK;
}

template <typename T>
T* blkp(xls_grid g, int i) { return (T*)g->blk[i]; }

template <typename T> const typename Vec4<T>::type* chi_table(xls_grid g);
template <> const double4* chi_table<double>(xls_grid g) { return g->d_chi64; }
template <> const float4* chi_table<float>(xls_grid g) { return g->d_chi32; }
template <typename T> const typename Vec4<T>::type* rchi_table(xls_grid g);
template <> const double4* rchi_table<double>(xls_grid g) { return g->d_rchi64; }
template <> const float4* rchi_table<float>(xls_grid g) { return g->d_rchi32; }

// kernel classes of the profile
enum { K_STENCIL = 0, K_NLPROJ = 1, K_NLBACK = 2, K_GRAM = 3, K_EIG = 4, K_ROTATE = 5, K_OTHER = 6 };

struct ProfScope {
  xls_grid g;
  int cls;
  bool on;
  ProfScope(xls_grid g_, int cls_) : g(g_), cls(cls_), on(g_->profiling && g_->pused + 2 <= g_->pev.size()) {
    if (on) cudaEventRecord(g->pev[g->pused], g->st);
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(g->pev[g->pused + 1], g->st);
    g->pcls[g->pused / 2] = cls;
    g->pused += 2;
  }
};

void prof_collect(xls_grid g) {
  if (!g->profiling) return;
  for (int c = 0; c < 8; ++c) { g->kms[c] = 0; g->kcnt[c] = 0; }
  for (size_t i = 0; i + 1 < g->pused; i += 2) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->pev[i], g->pev[i + 1]);
    g->kms[g->pcls[i / 2]] += ms;
    g->kcnt[g->pcls[i / 2]] += 1;
  }
}

// y_out = scale_step * (H - c) y_in - shift * y_prev for every subdomain of a view
template <typename T>
void h_step(xls_grid g, bool one, const T* yin, const T* yprev, T* yout, int step) {
  const SubDev* ds = one ? g->d_subs1 : g->d_subs;
  const Plan& pl = one ? g->plan1 : g->plan;
  double* P = one ? g->P1 : g->P;
  const int mns = one ? 1 : g->max_ns;
  const T* V = (sizeof(T) == 8) ? (const T*)g->V : (const T*)g->Vf;
  { ProfScope ps(g, K_NLPROJ);
    if (one) launch_nl_project1<T>(ds, g->d_slots, g->n_slot, g->d_pidx, chi_table<T>(g), yin, P, g->st);
    else launch_nl_project<T>(ds, g->d_slots, 0, g->n_slot, g->d_pidx, chi_table<T>(g), mns, yin, P, g->proj_vec,
                              g->proj_warps, g->proj_chunk, g->st); }
  { ProfScope ps(g, K_STENCIL); launch_stencil<T>(ds, g->n_sub, pl, yin, yprev, yout, V, g->coef, step, g->st); }
  { ProfScope ps(g, K_NLBACK);
    if (one)
      launch_nl_back1<T>(ds, g->n_sub, g->max_nd, g->nlb_max, g->d_rptr, g->d_rslot, rchi_table<T>(g), g->d_nlb_list,
                         P, yout, g->coef, step, g->st);
    else
      launch_nl_back_csr<T>(ds, g->n_sub, g->max_nd, mns, g->nlb_max, g->d_rptr, g->d_rslot, rchi_table<T>(g),
                            g->d_nlb_cnt, g->d_nlb_list, P, yout, g->coef, step, g->back_var, g->st); }
  g->launches += (g->n_slot ? 3 : 1);
}

// the whole grid as a view on the grid's current stream (graph capture may substitute a
// capture stream for the legacy stream)
xls_grid_s::View& fv(xls_grid g) {
  g->full.st = g->st;
  return g->full;
}

// same as h_step on a view of the main blocks, with the blocks given by index (the TMA stencil
// addresses its input through the tensor maps of that block)
template <typename T>
void h_step_main(xls_grid g, const xls_grid_s::View& v, int bin, int bprev, int bout, int step) {
  T* yin = (T*)g->blk[bin];
  T* yprev = bprev >= 0 ? (T*)g->blk[bprev] : nullptr;
  T* yout = (T*)g->blk[bout];
  const T* V = (sizeof(T) == 8) ? (const T*)g->V : (const T*)g->Vf;
  // the projection reads Y_in and writes P, the stencil reads Y_in, Y_prev and writes Y_out: with
  // the side stream (FP32 blocks, one view, no per-launch profiling) the two run side by side and
  // the back-projection waits for both
  const bool side = g->side_st && sizeof(T) == 4 && !g->concurrent && !g->profiling;
  if (side) {
    cudaEventRecord(g->ev_side_in, v.st);
    cudaStreamWaitEvent(g->side_st, g->ev_side_in, 0);
  }
  { ProfScope ps(g, K_NLPROJ);
    launch_nl_project<T>(g->d_subs, g->d_slots, v.slot_off, v.n_slot, g->d_pidx, chi_table<T>(g), v.max_ns, yin, g->P,
                         g->proj_vec, g->proj_warps, g->proj_chunk, side ? g->side_st : v.st); }
  if (side) cudaEventRecord(g->ev_side_out, g->side_st);
  if (sizeof(T) == 4 && g->use_tma) {
    ProfScope ps(g, K_STENCIL);
    for (const TmaClass& c : v.tcls)
      launch_stencil_tma(v.ds, c, v.maps, bin, bprev, (float*)yout, v.coef, step, g->status, v.st);
    g->launches += (int)v.tcls.size();
  } else {
    ProfScope ps(g, K_STENCIL);
    launch_stencil<T>(v.ds, v.n, v.plan, yin, yprev, yout, V, v.coef, step, v.st);
    g->launches++;
  }
  if (side) cudaStreamWaitEvent(v.st, g->ev_side_out, 0);
  { ProfScope ps(g, K_NLBACK);
    launch_nl_back_csr<T>(v.ds, v.n, v.max_nd, v.max_ns, g->nlb_max, g->d_rptr, g->d_rslot, rchi_table<T>(g),
                          g->d_nlb_cnt, g->d_nlb_list, g->P,
                          yout, v.coef, step, g->back_var, v.st); }
  g->launches += (v.n_slot ? 2 : 0);
}

constexpr int kUnitStep = kMaxDegree - 1;

// filter the current block in place of the two spare buffers; returns the index of Psi_f
template <typename T>
int run_filter(xls_grid g, const xls_grid_s::View& v, int m) {
  launch_filter_coef(v.n, v.bounds, m, v.coef, v.st);
  g->launches++;
  int ia = g->cur, ib = (g->cur + 1) % 3;
  h_step_main<T>(g, v, ia, -1, ib, 1);
  int yk = ib, yprev = ia;
  for (int k = 2; k <= m; ++k) {
    h_step_main<T>(g, v, yk, yprev, yprev, k);
    const int t = yk;
    yk = yprev;
    yprev = t;
  }
  return yk;
}

// third buffer index distinct from a and b
int other(int a, int b) {
  for (int i = 0; i < 3; ++i)
    if (i != a && i != b) return i;
  return 0;
}

template <typename T>
void projection(xls_grid g, const xls_grid_s::View& v, int f) {
  const int hf = other(f, f == 0 ? 1 : 0);
  h_step_main<T>(g, v, f, -1, hf, kUnitStep);
  if (sizeof(T) == 4 && g->use_tc_gram) {
    ProfScope ps(g, K_GRAM);
    launch_gram_tc(v.ds, v.n, v.max_ns, v.gplan, g->prec == XLS_MIXED_FP16, (const float*)g->blk[f],
                   (const float*)g->blk[hf], g->Ms, g->Hs, g->status, v.st);
    g->launches += g->prec == XLS_MIXED_FP16 ? 3 : 2;
    return;
  }
  cudaMemsetAsync(g->Ms + v.ss_off, 0, v.ss_n * sizeof(double), v.st);
  cudaMemsetAsync(g->Hs + v.ss_off, 0, v.ss_n * sizeof(double), v.st);
  { ProfScope ps(g, K_GRAM);
    launch_gram<T>(v.ds, v.n, v.max_ns, v.max_nd, blkp<T>(g, f), blkp<T>(g, hf), g->Ms, g->Hs, v.st); }
  g->launches++;
}

void eigensolve(xls_grid g, const xls_grid_s::View& v) {
  cudaMemcpyAsync(g->Lb + v.ss_off, g->Ms + v.ss_off, v.ss_n * sizeof(double), cudaMemcpyDeviceToDevice, v.st);
  cudaMemcpyAsync(g->Ab + v.ss_off, g->Hs + v.ss_off, v.ss_n * sizeof(double), cudaMemcpyDeviceToDevice, v.st);
  { ProfScope ps(g, K_EIG);
    launch_eig(v.ds, v.n, v.max_ns, g->Lb, g->Ab, g->Y, g->W, g->lam, g->vecs, g->status, v.eig_scr, g->R,
               g->eig_cluster ? g->eig_cl : 0, v.st); }
  g->launches += 8;
}

// rotation, interior weights and the next pass's (a, a0); returns the block now holding Psi
template <typename T>
int rotation(xls_grid g, const xls_grid_s::View& v, int f) {
  const int out = other(f, f == 0 ? 1 : 0);
  if (sizeof(T) == 4 && g->use_tc_rot) {
    ProfScope ps(g, K_ROTATE);
    launch_rotate_tc(v.ds, v.n, v.max_ns, v.rplan, v.gplan, g->prec == XLS_MIXED_FP16, !g->use_tc_gram,
                     (const float*)g->blk[f], g->Y, (float*)g->blk[out], g->status, v.st);
    g->launches += 2;
  } else {
    ProfScope ps(g, K_ROTATE);
    launch_rotate<T>(v.ds, v.n, v.max_ns, v.max_nd, blkp<T>(g, f), g->Y, blkp<T>(g, out), v.st);
  }
  { ProfScope ps(g, K_OTHER); launch_core_weights<T>(v.ds, v.n, v.max_ns, blkp<T>(g, out), g->cw, v.st); }
  launch_bounds_from_ritz(v.ds, v.n, g->lam, v.bounds, v.st);
  g->launches += 3;
  return out;
}

template <typename T>
xls_status bootstrap_bounds(xls_grid g) {
  // (a, a0) from the Ritz values of the unfiltered block; b was set by the Lanczos bound
  projection<T>(g, fv(g), g->cur);
  eigensolve(g, fv(g));
  launch_bounds_from_ritz(g->d_subs, g->n_sub, g->lam, g->bounds, g->st);
  g->launches++;
  return check_status(g);
}

xls_status upload_bounds(xls_grid g, const double* bounds) {
  XLS_CUDA(cudaMemcpyAsync(g->bounds, bounds, 3 * g->n_sub * sizeof(double), cudaMemcpyHostToDevice, g->st));
  return XLS_OK;
}

// stage events of a pass: external event-record nodes while a graph is being captured
void stage_event(xls_grid g, int i) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(g->st, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(g->ev[i], g->st, cudaEventRecordExternal);
  else cudaEventRecord(g->ev[i], g->st);
}

// one CheFSI pass (filter, projection, eigensolve, rotation).  Sequential on the grid's stream
// (stage events when timed), or, with concurrent halves and profiling off, the two halves on two
// streams forked from and joined back into the grid's stream: the GPU then overlaps the
// eigensolve (few SMs, FP64 latency) of one half with the filter of the other.
template <typename T>
void one_pass(xls_grid g, int degree, bool timed) {
  g->launches = 0;
  g->pused = 0;
  if (g->concurrent && !g->profiling) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(g->st, &cs);
    const bool cap = cs == cudaStreamCaptureStatusActive;
    if (timed) stage_event(g, 0);
    if (cap) cudaEventRecordWithFlags(g->ev_fork, g->st, cudaEventRecordDefault);
    else cudaEventRecord(g->ev_fork, g->st);
    // half 0: filter, then projection / eigensolve / rotation; half 1 starts its filter when half
    // 0's filter is done, so that half 0's subspace stages run beside half 1's filter
    auto& h0 = g->halves[0];
    auto& h1 = g->halves[1];
    cudaStreamWaitEvent(h0.st, g->ev_fork, 0);
    const int f = run_filter<T>(g, h0, degree);
    cudaEventRecord(g->ev_mid, h0.st);
    projection<T>(g, h0, f);
    eigensolve(g, h0);
    rotation<T>(g, h0, f);
    cudaEventRecord(h0.ev, h0.st);
    cudaStreamWaitEvent(h1.st, g->ev_mid, 0);
    run_filter<T>(g, h1, degree);
    projection<T>(g, h1, f);
    eigensolve(g, h1);
    const int out = rotation<T>(g, h1, f);
    cudaEventRecord(h1.ev, h1.st);
    cudaStreamWaitEvent(g->st, h0.ev, 0);
    cudaStreamWaitEvent(g->st, h1.ev, 0);
    g->cur = out;
    if (timed) {   // stages overlap: the whole pass is reported as the filter stage
      stage_event(g, 1);
      stage_event(g, 2);
      stage_event(g, 3);
      stage_event(g, 4);
    }
    return;
  }
  if (timed) stage_event(g, 0);
  const int f = run_filter<T>(g, fv(g), degree);
  if (timed) stage_event(g, 1);
  projection<T>(g, fv(g), f);
  if (timed) stage_event(g, 2);
  eigensolve(g, fv(g));
  if (timed) stage_event(g, 3);
  g->cur = rotation<T>(g, fv(g), f);
  if (timed) stage_event(g, 4);
}

// the pass as a CUDA graph: captured on first use for this (block, degree), replayed after
template <typename T>
xls_status graph_pass(xls_grid g, int degree) {
  for (auto& pg : g->graphs)
    if (pg.cur == g->cur && pg.degree == degree) {
      XLS_CUDA(cudaGraphLaunch(pg.exec, g->st));
      g->cur = pg.cur_after;
      g->launches = pg.launches;
      return XLS_OK;
    }
  const int cur0 = g->cur;
  cudaStream_t user = g->st;
  if (!user) {  // the legacy stream cannot be captured: capture on a private stream
    if (!g->cap_st) XLS_CUDA(cudaStreamCreateWithFlags(&g->cap_st, cudaStreamNonBlocking));
    g->st = g->cap_st;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(g->st, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    one_pass<T>(g, degree, true);
    e = cudaStreamEndCapture(g->st, &graph);
  }
  g->st = user;
  if (e != cudaSuccess) {
    g->cur = cur0;
    return fail(XLS_ECUDA, std::string("pass graph capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->cur = cur0;
    return fail(XLS_ECUDA, std::string("pass graph instantiation: ") + cudaGetErrorString(e));
  }
  g->graphs.push_back({cur0, degree, g->cur, g->launches, exec});
  XLS_CUDA(cudaGraphLaunch(exec, g->st));
  return XLS_OK;
}

template <typename T>
xls_status chefsi(xls_grid g, int degree, int n_passes, const double* bounds) {
  if (bounds) {
    XLS_TRY(upload_bounds(g, bounds));
  } else if (!g->have_ritz) {
    XLS_TRY(bootstrap_bounds<T>(g));
  }
  for (int p = 0; p < n_passes; ++p) {
    if (g->use_graphs && !g->profiling) XLS_TRY(graph_pass<T>(g, degree));
    else one_pass<T>(g, degree, p == n_passes - 1);
  }
  g->have_ritz = true;
  g->last_launches = g->launches;
  XLS_TRY(check_status(g));
  prof_collect(g);
  if (n_passes > 0) {
    for (int i = 0; i < 4; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, g->ev[i], g->ev[i + 1]);
      g->stage_ms[i] = ms;
    }
  }
  return XLS_OK;
}

template <typename T>
xls_status stage(xls_grid g, int which, int degree, const double* bounds) {
  switch (which) {
    case 1: {
      if (bounds) XLS_TRY(upload_bounds(g, bounds));
      else if (!g->have_ritz) XLS_TRY(bootstrap_bounds<T>(g));
      g->cur = run_filter<T>(g, fv(g), degree);
      break;
    }
    case 2: projection<T>(g, fv(g), g->cur); break;
    case 3: eigensolve(g, fv(g)); break;
    case 4: g->cur = rotation<T>(g, fv(g), g->cur); g->have_ritz = true; break;
    default: return fail(XLS_EINVAL, "stage must be 1..4");
  }
  return check_status(g);
}

// Lanczos upper bound of every subdomain (10 steps, FP64, single-vector view)
xls_status lanczos_bounds(xls_grid g) {
  const int k = 10;
  launch_lanczos_init(g->d_subs1, g->n_sub, g->lz_v, g->st);
  for (int j = 0; j < k; ++j) {
    h_step<double>(g, true, g->lz_v, nullptr, g->lz_Hv, kUnitStep);
    launch_lanczos_step(g->d_subs1, g->n_sub, j, g->lz_Hv, g->lz_v, g->lz_vp, g->lz_f, g->lz_a, g->lz_b, g->st);
  }
  launch_lanczos_finish(g->n_sub, k, g->lz_a, g->lz_b, g->d_subs1, g->lz_f, g->bounds, g->st);
  return check_status(g);
}

// periodic images of one atom that touch a subdomain (local frame of the subdomain)
void atom_images(xls_grid g, int a, const double R[3], const xls_species& sp, int slot, std::vector<AtomImg>& out) {
  const SubDev& S = g->subs[a];
  // candidate positions per axis in the subdomain's frame (one on a periodic axis, the five
  // nearest periodic images on a Dirichlet axis) whose r_cut interval meets the subdomain;
  // fixed-size arrays: this runs for every atom and subdomain of a set-up
  double cand[3][5];
  int lo[3][5], cnt[3][5], nc[3];
  for (int d = 0; d < 3; ++d) {
    const double h = g->gh[d], L = g->gL[d];
    const double Rl = R[d] - S.start[d] * h;
    nc[d] = 0;
    if (S.periodic[d]) {
      double r = std::fmod(Rl, L);
      if (r < 0) r += L;
      cand[d][nc[d]] = r;
      lo[d][nc[d]] = (int)std::floor((r - sp.r_cut) / h);
      cnt[d][nc[d]] = (int)std::ceil((r + sp.r_cut) / h) - lo[d][nc[d]] + 1;
      ++nc[d];
    } else {
      for (int sh = -2; sh <= 2; ++sh) {
        const double r = Rl + sh * L;
        int b0 = (int)std::floor((r - sp.r_cut) / h), b1 = (int)std::ceil((r + sp.r_cut) / h);
        b0 = std::max(b0, 0);
        b1 = std::min(b1, S.n[d] - 1);
        if (b1 < b0) continue;
        cand[d][nc[d]] = r;
        lo[d][nc[d]] = b0;
        cnt[d][nc[d]] = b1 - b0 + 1;
        ++nc[d];
      }
    }
    if (nc[d] == 0) return;   // no image meets the subdomain along this axis
  }
  for (int ix = 0; ix < nc[0]; ++ix)
    for (int iy = 0; iy < nc[1]; ++iy)
      for (int iz = 0; iz < nc[2]; ++iz) {
        AtomImg A{};
        const int ii[3] = {ix, iy, iz};
        double dist2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          A.R[d] = cand[d][ii[d]];
          A.box_lo[d] = lo[d][ii[d]];
          A.box_n[d] = cnt[d][ii[d]];
          // distance from the sphere centre to the box (clamped), for the intersection test
          const double h = g->gh[d];
          const double bl = A.box_lo[d] * h, bh = (A.box_lo[d] + A.box_n[d] - 1) * h;
          const double c = std::min(std::max(A.R[d], bl), bh);
          dist2 += (A.R[d] - c) * (A.R[d] - c);
        }
        if (dist2 >= sp.r_cut * sp.r_cut) continue;
        A.slot = slot;
        out.push_back(A);
      }
}

}  // namespace

// ---- views --------------------------------------------------------------------------------------

void set_view_slots(xls_grid g, xls_grid_s::View& v) {
  v.slot_off = v.n ? g->subs[v.first].slot_lo : 0;
  v.n_slot = 0;
  for (int a = v.first; a < v.first + v.n; ++a) v.n_slot += g->subs[a].slot_n;
}

// TMA stencil classes of subdomains [first, first + n): equal (x-points / 4, rows per tile, row
// width, spacing); jobs index the subdomains relative to `first`
xls_status build_tma_classes(xls_grid g, int first, int n, std::vector<TmaClass>& out) {
  std::vector<std::vector<int>> members;
  std::vector<TmaClass> cls;
  for (int a = first; a < first + n; ++a) {
    const SubDev& S = g->subs[a];
    const int nq = S.n[0] / 4, ty = tma_tile_rows(S), W = tma_row_width(S);
    size_t k = 0;
    for (; k < cls.size(); ++k)
      if (cls[k].nq == nq && cls[k].TY == ty && cls[k].W == W && cls[k].h[0] == S.h[0] && cls[k].h[1] == S.h[1] &&
          cls[k].h[2] == S.h[2])
        break;
    if (k == cls.size()) {
      TmaClass c;
      c.nq = nq; c.TY = ty; c.W = W;
      c.h[0] = S.h[0]; c.h[1] = S.h[1]; c.h[2] = S.h[2];
      cls.push_back(c);
      members.emplace_back();
    }
    members[k].push_back(a);
  }
  for (size_t k = 0; k < cls.size(); ++k) {
    std::vector<TmaJob> jobs;
    std::vector<int> off(1, 0);
    for (int a : members[k]) {
      const SubDev& S = g->subs[a];
      const int nyt = (S.n[1] + cls[k].TY - 1) / cls[k].TY;
      jobs.push_back(TmaJob{a - first, nyt, cls[k].W, cls[k].TY});
      off.push_back(off.back() + nyt * S.ns);
    }
    cls[k].n_jobs = (int)jobs.size();
    cls[k].total = off.back();
    XLS_TRY(g->alloc(&cls[k].d_jobs, jobs.size() * sizeof(TmaJob)));
    XLS_TRY(g->alloc(&cls[k].d_job_off, off.size() * sizeof(int)));
    XLS_CUDA(cudaMemcpy(cls[k].d_jobs, jobs.data(), jobs.size() * sizeof(TmaJob), cudaMemcpyHostToDevice));
    XLS_CUDA(cudaMemcpy(cls[k].d_job_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  out = cls;
  return XLS_OK;
}

// Tensor-core Gram jobs of subdomains [first, first + n) (indices relative to `first`): the upper
// block triangle of every subdomain, each block's K range split so that the grid aims at `cps`
// CTAs per SM (152 SMs); jobs of one block are consecutive (a reduction group).
constexpr int kMaxGramCps = 8;   // finest K split xls_autotune tries (sizes the job arrays)
void gram_jobs(xls_grid g, int first, int n, int cps, std::vector<GramJob>& jobs, std::vector<int>& gfirst,
               std::vector<int>& gn) {
  int groups = 0;
  for (int a = first; a < first + n; ++a) {
    const int nt = (g->subs[a].ns + 127) / 128;
    groups += nt * (nt + 1) / 2;
  }
  const int kchunks = std::max(1, (cps * 152 + groups - 1) / groups);
  jobs.clear();
  gfirst.clear();
  gn.clear();
  for (int a = first; a < first + n; ++a) {
    const SubDev& S = g->subs[a];
    const int nt = (S.ns + 127) / 128;
    const int nkt = (int)((S.nd + 63) / 64);
    const int kc = std::min(kchunks, nkt);
    for (int I = 0; I < nt; ++I)
      for (int J = I; J < nt; ++J) {
        gfirst.push_back((int)jobs.size());
        for (int c = 0; c < kc; ++c)
          jobs.push_back(GramJob{a - first, I, J, (int)((long long)nkt * c / kc), (int)((long long)nkt * (c + 1) / kc), 0});
        gn.push_back(kc);
      }
  }
}

// device arrays of a Gram plan sized for the finest split, then the jobs of the grid's split
xls_status alloc_gram_plan(xls_grid g, int first, int n, GramPlan& gp) {
  std::vector<GramJob> jobs;
  std::vector<int> gfirst, gn;
  gram_jobs(g, first, n, kMaxGramCps, jobs, gfirst, gn);
  gp.cap_jobs = (int)jobs.size();
  gp.n_groups = (int)gfirst.size();
  XLS_TRY(g->alloc(&gp.d_jobs, jobs.size() * sizeof(GramJob)));
  XLS_TRY(g->alloc(&gp.d_grp_first, gfirst.size() * sizeof(int)));
  XLS_TRY(g->alloc(&gp.d_grp_n, gn.size() * sizeof(int)));
  XLS_TRY(g->alloc(&gp.d_work, jobs.size() * 2 * 128 * 128 * sizeof(float)));
  gram_jobs(g, first, n, g->gram_cps, jobs, gfirst, gn);
  gp.n_jobs = (int)jobs.size();
  XLS_CUDA(cudaMemcpy(gp.d_jobs, jobs.data(), jobs.size() * sizeof(GramJob), cudaMemcpyHostToDevice));
  XLS_CUDA(cudaMemcpy(gp.d_grp_first, gfirst.data(), gfirst.size() * sizeof(int), cudaMemcpyHostToDevice));
  XLS_CUDA(cudaMemcpy(gp.d_grp_n, gn.data(), gn.size() * sizeof(int), cudaMemcpyHostToDevice));
  return XLS_OK;
}

// rewrite a plan's jobs for the grid's current split (stream-ordered on st)
xls_status replan_gram(xls_grid g, int first, int n, GramPlan& gp, cudaStream_t st) {
  std::vector<GramJob> jobs;
  std::vector<int> gfirst, gn;
  gram_jobs(g, first, n, g->gram_cps, jobs, gfirst, gn);
  if ((int)jobs.size() > gp.cap_jobs || (int)gfirst.size() != gp.n_groups)
    return fail(XLS_EINVAL, "Gram plan: split beyond the planned capacity");
  gp.n_jobs = (int)jobs.size();
  XLS_CUDA(cudaMemcpyAsync(gp.d_jobs, jobs.data(), jobs.size() * sizeof(GramJob), cudaMemcpyHostToDevice, st));
  XLS_CUDA(cudaMemcpyAsync(gp.d_grp_first, gfirst.data(), gfirst.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  XLS_CUDA(cudaMemcpyAsync(gp.d_grp_n, gn.data(), gn.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  XLS_CUDA(cudaStreamSynchronize(st));   // the host vectors go out of scope
  return XLS_OK;
}

// tensor-core Gram and rotation jobs of subdomains [first, first + n) (indices relative to
// `first`); the exponent and split-Y arrays are indexed by state and shared with `shared`
xls_status build_tc_plans(xls_grid g, int first, int n, GramPlan& gp, RotPlan& rp, const GramPlan* gshared,
                          const RotPlan* rshared) {
  XLS_TRY(alloc_gram_plan(g, first, n, gp));
  if (gshared) {
    gp.d_ex_f = gshared->d_ex_f;
    gp.d_ex_hf = gshared->d_ex_hf;
  } else {
    XLS_TRY(g->alloc(&gp.d_ex_f, g->tot_states * sizeof(int)));
    XLS_TRY(g->alloc(&gp.d_ex_hf, g->tot_states * sizeof(int)));
  }
  std::vector<RotJob> rj;
  for (int a = first; a < first + n; ++a)
    for (int t = 0; t < (int)((g->subs[a].nd + 127) / 128); ++t)
      for (int n0 = 0; n0 < g->subs[a].ns; n0 += 256) rj.push_back(RotJob{a - first, t, n0});
  rp.n_jobs = (int)rj.size();
  rp.kpad_max = ((g->max_ns + 63) / 64) * 64;
  XLS_TRY(g->alloc(&rp.d_jobs, rj.size() * sizeof(RotJob)));
  if (rshared) {
    rp.d_yhi = rshared->d_yhi;
    rp.d_ylo = rshared->d_ylo;
    rp.d_ex_y = rshared->d_ex_y;
  } else {
    XLS_TRY(g->alloc(&rp.d_yhi, (size_t)g->tot_states * rp.kpad_max * sizeof(uint16_t)));
    XLS_TRY(g->alloc(&rp.d_ylo, (size_t)g->tot_states * rp.kpad_max * sizeof(uint16_t)));
    XLS_TRY(g->alloc(&rp.d_ex_y, g->tot_states * sizeof(int)));
  }
  XLS_CUDA(cudaMemcpy(rp.d_jobs, rj.data(), rj.size() * sizeof(RotJob), cudaMemcpyHostToDevice));
  return XLS_OK;
}

// the descriptors, offsets and plans of subdomains [first, first + n) on stream st
xls_status make_view(xls_grid g, int first, int n, cudaStream_t st, bool own_plans, xls_grid_s::View& v) {
  v.first = first;
  v.n = n;
  v.ds = g->d_subs + first;
  v.coef = g->coef + (size_t)first * kMaxDegree;
  v.bounds = g->bounds + 3 * (size_t)first;
  v.maps = g->d_maps ? g->d_maps + (size_t)first * kMapsPerSub : nullptr;
  v.ss_off = g->subs[first].off_ss;
  const SubDev& L = g->subs[first + n - 1];
  v.ss_n = L.off_ss + (long long)L.ns * L.ns - v.ss_off;
  v.max_ns = 0;
  v.max_nd = 0;
  for (int a = first; a < first + n; ++a) {
    v.max_ns = std::max(v.max_ns, g->subs[a].ns);
    v.max_nd = std::max(v.max_nd, g->subs[a].nd);
  }
  v.eig_scr = g->eig_scr + (size_t)first * (eig_scratch_doubles(g->n_sub, g->max_ns) / g->n_sub);
  v.st = st;
  if (own_plans) {
    std::vector<SubDev> sub(g->subs.begin() + first, g->subs.begin() + first + n);
    XLS_TRY(make_plan(g, sub, v.plan));
    if (g->use_tma) XLS_TRY(build_tma_classes(g, first, n, v.tcls));
    if (g->use_tc) XLS_TRY(build_tc_plans(g, first, n, v.gplan, v.rplan, &g->gplan, &g->rplan));
  } else {
    v.plan = g->plan;
    v.tcls = g->tcls;
    v.gplan = g->gplan;
    v.rplan = g->rplan;
  }
  set_view_slots(g, v);
  return XLS_OK;
}

// ---- SCF step on the global periodic grid ------------------------------------------------------
xls_status scf_alloc(xls_grid g) {
  auto& S = g->scf;
  const long long n = (long long)g->gn[0] * g->gn[1] * g->gn[2];
  SubDev& G = S.gs;
  G = SubDev{};
  for (int d = 0; d < 3; ++d) {
    G.n[d] = g->gn[d];
    G.periodic[d] = 1;
    G.core_n[d] = g->gn[d];
    G.h[d] = g->gh[d];
  }
  G.ns = 1;
  G.nd = n;
  G.dV = g->gh[0] * g->gh[1] * g->gh[2];
  XLS_TRY(g->alloc(&S.d_gs, sizeof(SubDev)));
  XLS_CUDA(cudaMemcpy(S.d_gs, &G, sizeof(SubDev), cudaMemcpyHostToDevice));
  XLS_TRY(make_plan(g, std::vector<SubDev>{G}, S.plan));
  XLS_TRY(g->alloc(&S.d_coef, kMaxDegree * sizeof(StepCoef)));
  double** bufs[] = {&S.b, &S.phi, &S.eps, &S.vxc, &S.rho_in, &S.rho_out, &S.zero, &S.r, &S.p,
                     &S.q, &S.tmp, &S.f, &S.pf, &S.x_prev, &S.f_prev, &S.pf_prev};
  for (double** b : bufs) XLS_TRY(g->alloc(b, n * sizeof(double)));
  XLS_CUDA(cudaMemsetAsync(S.zero, 0, n * sizeof(double), g->st));
  XLS_CUDA(cudaMemsetAsync(S.phi, 0, n * sizeof(double), g->st));
  XLS_TRY(g->alloc(&S.dX, (size_t)S.hist * n * sizeof(double)));
  XLS_TRY(g->alloc(&S.dF, (size_t)S.hist * n * sizeof(double)));
  XLS_TRY(g->alloc(&S.dPF, (size_t)S.hist * n * sizeof(double)));
  XLS_TRY(g->alloc(&S.partial, kRedPartials * sizeof(double)));
  XLS_TRY(g->alloc(&S.pulay_partial, pulay_partial_doubles() * sizeof(double)));
  XLS_TRY(g->alloc(&S.scal, 16 * sizeof(double)));
  XLS_TRY(g->alloc(&S.gamma, 16 * sizeof(double)));
  const char* env = std::getenv("XLS_SCF_PLAIN_CG");
  S.pcg = !(env && env[0] == '1');
  if (S.pcg) {
    XLS_TRY(g->alloc(&S.z, n * sizeof(double)));
    XLS_TRY(g->alloc(&S.r_old, n * sizeof(double)));
    XLS_TRY(g->alloc(&S.mg, mg_floats(g->gn) * sizeof(float)));
  }
  return XLS_OK;
}

// z = M r: one FP32 V-cycle of the 7-point operator (+ kappa^2 for which 1); the Poisson case
// keeps z at zero mean (the periodic operator's null space)
void scf_precondition(xls_grid g, int which, const double* r, double* z) {
  auto& S = g->scf;
  const long long n = S.gs.nd;
  launch_mg_vcycle(g->gn, g->gh, which == 1 ? S.kappa * S.kappa : 0.0, r, z, S.mg, g->st);
  if (which == 0) {
    launch_sum(n, z, S.partial, S.scal + 6, g->st);
    launch_sub_mean(n, S.scal + 6, z, g->st);
  }
}

// the stencil's step coefficients on the global grid: step 0: -Delta_h, step 1: -Delta_h + kappa^2
xls_status scf_coefficients(xls_grid g) {
  std::vector<StepCoef> c(kMaxDegree, StepCoef{0, 0, 0, 0});
  c[0] = StepCoef{2.0, 0.0, 0.0, 0.0};
  c[1] = StepCoef{2.0, -0.5 * g->scf.kappa * g->scf.kappa, 0.0, 0.0};
  XLS_CUDA(cudaMemcpy(g->scf.d_coef, c.data(), c.size() * sizeof(StepCoef), cudaMemcpyHostToDevice));
  return XLS_OK;
}

void scf_apply(xls_grid g, int which, const double* x, double* y) {
  launch_stencil<double>(g->scf.d_gs, 1, g->scf.plan, x, nullptr, y, g->scf.zero, g->scf.d_coef, which, g->st);
}

// conjugate gradients for A x = rhs (A = -Delta_h (which 0, rhs of zero mean) or -Delta_h + kappa^2
// (which 1)), x holds the start and receives the solution; stops at
// ||r||^2 <= tol^2 max(||rhs||^2, ref_sq) (ref_sq: the scale of the terms that formed rhs, for
// right-hand sides that cancel to rounding)
xls_status scf_pcg(xls_grid g, int which, const double* rhs, double* x, double tol, int max_iter, double ref_sq);

xls_status scf_cg(xls_grid g, int which, const double* rhs, double* x, double tol, int max_iter, double ref_sq = 0.0) {
  if (g->scf.pcg) return scf_pcg(g, which, rhs, x, tol, max_iter, ref_sq);
  auto& S = g->scf;
  const long long n = S.gs.nd;
  double* s = S.scal;  // s[0] r.r, s[1] p.Ap, s[2] new r.r, s[3] rhs.rhs
  scf_apply(g, which, x, S.q);
  launch_axpbypcz(n, 1.0, rhs, 0.0, S.r, -1.0, S.q, g->st);
  XLS_CUDA(cudaMemcpyAsync(S.p, S.r, n * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
  {
    const double* xs[2] = {S.r, rhs};
    const double* ys[2] = {S.r, rhs};
    launch_dots(n, xs, ys, 2, S.partial, s + 4, 1.0, g->st);   // s[4] = r.r, s[5] = rhs.rhs
    XLS_CUDA(cudaMemcpyAsync(s, s + 4, sizeof(double), cudaMemcpyDeviceToDevice, g->st));
    XLS_CUDA(cudaMemcpyAsync(s + 3, s + 5, sizeof(double), cudaMemcpyDeviceToDevice, g->st));
  }
  double h[4];
  XLS_CUDA(cudaMemcpyAsync(h, s, 4 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
  XLS_CUDA(cudaStreamSynchronize(g->st));
  const double stop = tol * tol * std::max(h[3], ref_sq);
  if (h[0] <= stop) return XLS_OK;
  for (int it = 1; it <= max_iter; ++it) {
    scf_apply(g, which, S.p, S.q);
    const double* xs[1] = {S.p};
    const double* ys[1] = {S.q};
    launch_dots(n, xs, ys, 1, S.partial, s + 1, 1.0, g->st);
    launch_cg_xr(n, s, x, S.r, S.p, S.q, S.partial, g->st);
    launch_cg_p(n, s, S.r, S.p, g->st);
    S.cg_iters++;
    if (it % 16 == 0 || it == max_iter) {
      XLS_CUDA(cudaMemcpyAsync(h, s, sizeof(double), cudaMemcpyDeviceToHost, g->st));
      XLS_CUDA(cudaStreamSynchronize(g->st));
      if (!std::isfinite(h[0])) return fail(XLS_ENONFINITE, "SCF: conjugate gradients produced a non-finite residual");
      if (h[0] <= stop) return XLS_OK;
    }
  }
  return fail(XLS_ENOCONV, "SCF: conjugate gradients did not reach the tolerance");
}

// The same solve by flexible preconditioned CG (Polak-Ribiere beta, robust to the FP32 rounding of
// the preconditioner), the preconditioner one multigrid V-cycle; same stopping rule on ||r||^2.
// s[0] r.z, s[1] p.Ap, s[2] r.r, s[3] rhs.rhs, s[4] new r.z, s[5] r_old.z, s[6] scratch sum
xls_status scf_pcg(xls_grid g, int which, const double* rhs, double* x, double tol, int max_iter, double ref_sq) {
  auto& S = g->scf;
  const long long n = S.gs.nd;
  double* s = S.scal;
  scf_apply(g, which, x, S.q);
  launch_axpbypcz(n, 1.0, rhs, 0.0, S.r, -1.0, S.q, g->st);
  scf_precondition(g, which, S.r, S.z);
  XLS_CUDA(cudaMemcpyAsync(S.p, S.z, n * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
  {
    const double* xs[3] = {S.r, S.r, rhs};
    const double* ys[3] = {S.z, S.r, rhs};
    launch_dots(n, xs, ys, 3, S.partial, s + 8, 1.0, g->st);   // s[8] r.z, s[9] r.r, s[10] rhs.rhs
    XLS_CUDA(cudaMemcpyAsync(s, s + 8, sizeof(double), cudaMemcpyDeviceToDevice, g->st));
    XLS_CUDA(cudaMemcpyAsync(s + 2, s + 9, 2 * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
  }
  double h[4];
  XLS_CUDA(cudaMemcpyAsync(h, s, 4 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
  XLS_CUDA(cudaStreamSynchronize(g->st));
  const double stop = tol * tol * std::max(h[3], ref_sq);
  if (h[2] <= stop) return XLS_OK;
  for (int it = 1; it <= max_iter; ++it) {
    scf_apply(g, which, S.p, S.q);
    const double* xs[1] = {S.p};
    const double* ys[1] = {S.q};
    launch_dots(n, xs, ys, 1, S.partial, s + 1, 1.0, g->st);
    XLS_CUDA(cudaMemcpyAsync(S.r_old, S.r, n * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
    launch_cg_xr(n, s, x, S.r, S.p, S.q, S.partial, g->st);   // x += a p, r -= a q, s[2] = r.r
    scf_precondition(g, which, S.r, S.z);
    {
      const double* xz[2] = {S.r, S.r_old};
      const double* yz[2] = {S.z, S.z};
      launch_dots(n, xz, yz, 2, S.partial, s + 4, 1.0, g->st);
    }
    launch_pcg_p(n, s, S.z, S.p, g->st);
    S.cg_iters++;
    if (it % 4 == 0 || it == max_iter) {
      XLS_CUDA(cudaMemcpyAsync(h, s, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
      XLS_CUDA(cudaStreamSynchronize(g->st));
      if (!std::isfinite(h[2])) return fail(XLS_ENONFINITE, "SCF: conjugate gradients produced a non-finite residual");
      if (h[2] <= stop) return XLS_OK;
    }
  }
  return fail(XLS_ENOCONV, "SCF: conjugate gradients did not reach the tolerance");
}

// P f = -Delta_h (-Delta_h + kappa^2)^-1 f
xls_status scf_kerker(xls_grid g, const double* f, double* out) {
  auto& S = g->scf;
  XLS_CUDA(cudaMemsetAsync(S.tmp, 0, S.gs.nd * sizeof(double), g->st));
  XLS_TRY(scf_cg(g, 1, f, S.tmp, 1e-13, 4000));
  scf_apply(g, 0, S.tmp, out);
  return XLS_OK;
}

xls_status scf_pseudocharge(xls_grid g) {
  auto& S = g->scf;
  const int na = (int)g->atom_sp.size();
  if (na == 0) return fail(XLS_EINVAL, "SCF: the Hamiltonian has no atoms");
  std::vector<double> rc(na), amp(na);
  S.z_total = 0.0;
  S.e_self = 0.0;
  for (int i = 0; i < na; ++i) {
    const xls_species& q = g->species[g->atom_sp[i]];
    rc[i] = q.rc_loc;
    amp[i] = -q.Zv * std::pow(M_PI, -1.5) / (q.rc_loc * q.rc_loc * q.rc_loc);
    S.z_total += q.Zv;
    S.e_self += 0.5 * q.Zv * q.Zv * std::sqrt(2.0 / M_PI) / q.rc_loc;   // 1/2 int b_I V_I
  }
  if (!S.d_pos) {
    XLS_TRY(g->alloc(&S.d_pos, 3 * (size_t)na * sizeof(double)));
    XLS_TRY(g->alloc(&S.d_rc, (size_t)na * sizeof(double)));
    XLS_TRY(g->alloc(&S.d_amp, (size_t)na * sizeof(double)));
    XLS_TRY(g->alloc(&S.g1, (size_t)na * (g->gn[0] + g->gn[1] + g->gn[2]) * sizeof(double)));
  }
  XLS_CUDA(cudaMemcpy(S.d_pos, g->atom_pos.data(), 3 * (size_t)na * sizeof(double), cudaMemcpyHostToDevice));
  XLS_CUDA(cudaMemcpy(S.d_rc, rc.data(), na * sizeof(double), cudaMemcpyHostToDevice));
  XLS_CUDA(cudaMemcpy(S.d_amp, amp.data(), na * sizeof(double), cudaMemcpyHostToDevice));
  launch_pseudocharge(na, S.d_pos, S.d_rc, S.d_amp, g->gn, g->gh, g->gL, S.g1, S.b, S.z_total, S.partial, S.scal,
                      g->st);
  S.pc_ready = true;
  return XLS_OK;
}

extern "C" {

const char* xls_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// The grid of a set of subdomains.  `partial` grids (one wave of a wave-mode grid) need not tile
// the global grid; `wave` grids keep only the per-state arrays on the device (the orbitals stay
// in a host store and the waves run on partial grids).
xls_status create_grid(const xls_cell* cell, const xls_dc* dc, int precision, size_t hbm_budget_bytes,
                       void* cuda_stream, xls_grid* out, bool partial, bool wave, bool dry = false) {
  xls_grid g = new xls_grid_s();
  g->prec = precision;
  g->st = (cudaStream_t)cuda_stream;
  g->budget = hbm_budget_bytes;
  g->elem = precision == XLS_FP64 ? 8 : 4;
  for (int d = 0; d < 3; ++d) {
    g->gn[d] = cell->n[d];
    g->gL[d] = cell->L[d];
    g->gh[d] = cell->L[d] / cell->n[d];
  }
  g->n_sub = dc->n_sub;
  long long covered = 0;
  for (int a = 0; a < dc->n_sub; ++a) {
    SubDev S{};
    const int ns = dc->n_states[a];
    if (ns < 1 || ns > kMaxStates) {
      delete g;
      return fail(XLS_EINVAL, "n_states out of range in subdomain " + std::to_string(a));
    }
    long long nd = 1;
    for (int d = 0; d < 3; ++d) {
      const int cl = dc->core_lo[3 * a + d], cn = dc->core_n[3 * a + d], b = dc->buf[3 * a + d];
      if (cn < 1 || cn > cell->n[d] || b < 0 || cl < 0 || cl >= cell->n[d]) {
        delete g;
        return fail(XLS_EINVAL, "bad core/buffer in subdomain " + std::to_string(a));
      }
      int size = cn + 2 * b;
      const bool per = size >= cell->n[d];
      const int be = per ? std::min(b, (cell->n[d] - cn) / 2) : b;
      if (per) size = cell->n[d];
      S.n[d] = size;
      S.periodic[d] = per ? 1 : 0;
      S.start[d] = cl - be;
      S.core_lo[d] = be;
      S.core_n[d] = cn;
      S.core_glo[d] = cl;
      S.h[d] = g->gh[d];
      nd *= size;
    }
    for (int d = 0; d < 3; ++d)
      if (S.n[d] < 2 * kN0 + 1) {
        delete g;
        return fail(XLS_EINVAL, "subdomain shorter than 13 points along an axis");
      }
    S.ns = ns;
    S.nd = nd;
    S.dV = g->gh[0] * g->gh[1] * g->gh[2];
    S.off_blk = g->tot_blk;
    S.off_pt = g->tot_pts;
    S.off_ss = g->tot_ss;
    S.off_state = g->tot_states;
    g->tot_blk += nd * ns;
    g->tot_pts += nd;
    g->tot_ss += (long long)ns * ns;
    g->tot_states += ns;
    g->max_ns = std::max(g->max_ns, ns);
    g->max_nd = std::max(g->max_nd, nd);
    g->max_core = std::max(g->max_core, (long long)S.core_n[0] * S.core_n[1] * S.core_n[2]);
    covered += (long long)S.core_n[0] * S.core_n[1] * S.core_n[2];
    g->subs.push_back(S);
    SubDev S1 = S;
    S1.ns = 1;
    S1.off_blk = S.off_pt;
    g->subs1.push_back(S1);
  }
  if (!partial && covered != (long long)cell->n[0] * cell->n[1] * cell->n[2]) {
    delete g;
    return fail(XLS_EINVAL, "cores do not tile the global grid exactly once");
  }
  g->cell = *cell;
  if (dry) {  // descriptors only
    *out = g;
    return XLS_OK;
  }
  xls_status s = XLS_OK;
#define ALLOC(p, n)                         \
  if ((s = g->alloc(&(p), (n))) != XLS_OK) { \
    xls_grid_destroy(g);                    \
    return s;                               \
  }
  if (wave) {
    g->wave = true;
    ALLOC(g->lam, g->tot_states * sizeof(double));
    ALLOC(g->cw, g->tot_states * sizeof(double));
    ALLOC(g->occ, g->tot_states * sizeof(double));
    ALLOC(g->status, 2 * sizeof(int));
    ALLOC(g->out4, 4 * sizeof(double));
    ALLOC(g->d_subs, g->n_sub * sizeof(SubDev));
    {  // descriptors of a subdomain staged alone in blk[0] (the density sweep)
      std::vector<SubDev> staged = g->subs;
      for (SubDev& S : staged) S.off_blk = 0;
      cudaMemcpy(g->d_subs, staged.data(), staged.size() * sizeof(SubDev), cudaMemcpyHostToDevice);
    }
    cudaMemset(g->status, 0, 2 * sizeof(int));
    cudaMemset(g->lam, 0, g->tot_states * sizeof(double));
    cudaMemset(g->cw, 0, g->tot_states * sizeof(double));
    for (int i = 0; i < 6; ++i) cudaEventCreate(&g->ev[i]);
    // the pinned orbital store and the device staging block are allocated at first use (carry
    // mode needs neither)
    g->host_bounds.assign(3 * (size_t)g->n_sub, 0.0);
    *out = g;
    return XLS_OK;
  }
  for (int i = 0; i < 3; ++i) ALLOC(g->blk[i], g->tot_blk * g->elem);
  ALLOC(g->V, g->tot_pts * sizeof(double));
  ALLOC(g->Vf, g->tot_pts * sizeof(float));
  ALLOC(g->Ms, g->tot_ss * sizeof(double));
  ALLOC(g->Hs, g->tot_ss * sizeof(double));
  ALLOC(g->Lb, g->tot_ss * sizeof(double));
  ALLOC(g->Ab, g->tot_ss * sizeof(double));
  ALLOC(g->W, g->tot_ss * sizeof(double));
  ALLOC(g->Y, g->tot_ss * sizeof(double));
  ALLOC(g->R, g->tot_ss * sizeof(double));
  ALLOC(g->lam, g->tot_states * sizeof(double));
  ALLOC(g->cw, g->tot_states * sizeof(double));
  ALLOC(g->occ, g->tot_states * sizeof(double));
  ALLOC(g->vecs, 8LL * g->tot_states * sizeof(double));
  ALLOC(g->eig_scr, eig_scratch_doubles(g->n_sub, g->max_ns) * sizeof(double));
  ALLOC(g->bounds, 3 * g->n_sub * sizeof(double));
  ALLOC(g->coef, (size_t)g->n_sub * kMaxDegree * sizeof(StepCoef));
  ALLOC(g->status, 2 * sizeof(int));
  ALLOC(g->out4, 4 * sizeof(double));
  ALLOC(g->lz_v, g->tot_pts * sizeof(double));
  ALLOC(g->lz_vp, g->tot_pts * sizeof(double));
  ALLOC(g->lz_f, g->tot_pts * sizeof(double));
  ALLOC(g->lz_Hv, g->tot_pts * sizeof(double));
  ALLOC(g->lz_a, 16 * g->n_sub * sizeof(double));
  ALLOC(g->lz_b, 16 * g->n_sub * sizeof(double));
  ALLOC(g->d_subs, g->n_sub * sizeof(SubDev));
  ALLOC(g->d_subs1, g->n_sub * sizeof(SubDev));
#undef ALLOC
  if ((s = make_plan(g, g->subs, g->plan)) != XLS_OK || (s = make_plan(g, g->subs1, g->plan1)) != XLS_OK) {
    xls_grid_destroy(g);
    return s;
  }
  if (precision != XLS_FP64) {
    const char* env = std::getenv("XLS_STENCIL");
    bool ok = !(env && std::string(env) == "generic");
    for (const SubDev& S : g->subs) ok = ok && tma_eligible(S);
    if (ok) {
      std::vector<CUtensorMap> maps((size_t)g->n_sub * kMapsPerSub);
      for (int a = 0; a < g->n_sub && ok; ++a)
        ok = build_tma_maps(g->subs[a], g->Vf, g->blk, (CUtensorMap_st*)&maps[(size_t)a * kMapsPerSub]);
      if (ok) {
        // classes of equal (x-points/4, rows per tile, row width)
        std::vector<std::vector<int>> members;
        std::vector<TmaClass> cls;
        for (int a = 0; a < g->n_sub; ++a) {
          const SubDev& S = g->subs[a];
          const int nq = S.n[0] / 4, ty = tma_tile_rows(S), W = tma_row_width(S);
          size_t k = 0;
          for (; k < cls.size(); ++k)
            if (cls[k].nq == nq && cls[k].TY == ty && cls[k].W == W && cls[k].h[0] == S.h[0] && cls[k].h[1] == S.h[1] &&
                cls[k].h[2] == S.h[2])
              break;
          if (k == cls.size()) {
            TmaClass c;
            c.nq = nq; c.TY = ty; c.W = W;
            c.h[0] = S.h[0]; c.h[1] = S.h[1]; c.h[2] = S.h[2];
            cls.push_back(c);
            members.emplace_back();
          }
          members[k].push_back(a);
        }
        for (size_t k = 0; k < cls.size() && s == XLS_OK; ++k) {
          std::vector<TmaJob> jobs;
          std::vector<int> off(1, 0);
          for (int a : members[k]) {
            const SubDev& S = g->subs[a];
            const int nyt = (S.n[1] + cls[k].TY - 1) / cls[k].TY;
            jobs.push_back(TmaJob{a, nyt, cls[k].W, cls[k].TY});
            off.push_back(off.back() + nyt * S.ns);
          }
          cls[k].n_jobs = (int)jobs.size();
          cls[k].total = off.back();
          if ((s = g->alloc(&cls[k].d_jobs, jobs.size() * sizeof(TmaJob))) != XLS_OK) break;
          if ((s = g->alloc(&cls[k].d_job_off, off.size() * sizeof(int))) != XLS_OK) break;
          cudaMemcpy(cls[k].d_jobs, jobs.data(), jobs.size() * sizeof(TmaJob), cudaMemcpyHostToDevice);
          cudaMemcpy(cls[k].d_job_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
        }
        if (s == XLS_OK) s = g->alloc(&g->d_maps, maps.size() * sizeof(CUtensorMap));
        if (s != XLS_OK) {
          xls_grid_destroy(g);
          return s;
        }
        cudaMemcpy(g->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
        g->tcls = cls;
        g->use_tma = true;
      }
    }
  }
  {
    const char* env = std::getenv("XLS_EIG");
    g->eig_cluster = !(env && std::string(env) == "single");
    const char* ecl = std::getenv("XLS_EIG_CL");   // cluster size tried first (xls_autotune changes it)
    if (ecl && std::atoi(ecl) == 16) g->eig_cl = 16;
    const char* pv = std::getenv("XLS_PROJ_VEC");  // projection vectors per CTA (xls_autotune changes it)
    if (pv && (std::atoi(pv) == 16 || std::atoi(pv) == 32)) g->proj_vec = std::atoi(pv);
  }
  if (precision != XLS_FP64) {
    const char* env = std::getenv("XLS_GEMM");
    bool ok = !(env && std::string(env) == "simt") && tc_setup();
    for (const SubDev& S : g->subs) ok = ok && S.ns <= 2048 && S.nd % 8 == 0;
    if (ok) {
      // Gram jobs: upper block triangle of every subdomain, K split so that the grid fills the GPU
      GramPlan& gp = g->gplan;
      s = alloc_gram_plan(g, 0, g->n_sub, gp);
      if (s == XLS_OK) s = g->alloc(&gp.d_ex_f, g->tot_states * sizeof(int));
      if (s == XLS_OK) s = g->alloc(&gp.d_ex_hf, g->tot_states * sizeof(int));
      std::vector<RotJob> rj;
      for (int a = 0; a < g->n_sub; ++a)
        for (int t = 0; t < (int)((g->subs[a].nd + 127) / 128); ++t)
          for (int n0 = 0; n0 < g->subs[a].ns; n0 += 256) rj.push_back(RotJob{a, t, n0});
      RotPlan& rp = g->rplan;
      rp.n_jobs = (int)rj.size();
      rp.kpad_max = ((g->max_ns + 63) / 64) * 64;
      if (s == XLS_OK && (s = g->alloc(&rp.d_jobs, rj.size() * sizeof(RotJob))) == XLS_OK &&
          (s = g->alloc(&rp.d_yhi, (size_t)g->tot_states * rp.kpad_max * sizeof(uint16_t))) == XLS_OK)
        s = g->alloc(&rp.d_ylo, (size_t)g->tot_states * rp.kpad_max * sizeof(uint16_t));
      if (s == XLS_OK) s = g->alloc(&rp.d_ex_y, g->tot_states * sizeof(int));
      if (s != XLS_OK) {
        xls_grid_destroy(g);
        return s;
      }
      cudaMemcpy(rp.d_jobs, rj.data(), rj.size() * sizeof(RotJob), cudaMemcpyHostToDevice);
      g->use_tc = true;
      const char* eg = std::getenv("XLS_GEMM_GRAM");
      const char* er = std::getenv("XLS_GEMM_ROT");
      g->use_tc_gram = !(eg && std::string(eg) == "simt");
      g->use_tc_rot = !(er && std::string(er) == "simt");
    }
  }
  // views: the whole grid, and two halves of about equal work on streams of their own
  if ((s = make_view(g, 0, g->n_sub, g->st, false, g->full)) != XLS_OK) {
    xls_grid_destroy(g);
    return s;
  }
  {
    const char* env = std::getenv("XLS_CONCURRENT");
    const bool want = env && std::string(env) == "1";
    if (want && g->n_sub >= 2) {
      double tot = 0.0, run = 0.0;
      for (const SubDev& S : g->subs) tot += (double)S.nd * S.ns;
      int split = 1;
      double best = 1e300;
      for (int k = 1; k < g->n_sub; ++k) {
        run += (double)g->subs[k - 1].nd * g->subs[k - 1].ns;
        if (std::fabs(2 * run - tot) < best) {
          best = std::fabs(2 * run - tot);
          split = k;
        }
      }
      bool ok = true;
      for (int h = 0; h < 2 && ok; ++h) {
        ok = cudaStreamCreateWithFlags(&g->halves[h].st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&g->halves[h].ev, cudaEventDisableTiming) == cudaSuccess;
        if (ok) ok = make_view(g, h ? split : 0, h ? g->n_sub - split : split, g->halves[h].st, true, g->halves[h]) ==
                     XLS_OK;
      }
      ok = ok && cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&g->ev_mid, cudaEventDisableTiming) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        xls_grid_destroy(g);
        return fail(XLS_ECUDA, "concurrent halves could not be set up");
      }
      g->concurrent = true;
    }
  }
  {
    // the projection of a filter step on a side stream beside the stencil (XLS_PROJ_SIDE=1): off by
    // default -- on 72^3 subdomains the two kernels contend for L2 and DRAM and the step is slower
    const char* env = std::getenv("XLS_PROJ_SIDE");
    if (env && env[0] == '1' && !dry) {
      const bool ok = cudaStreamCreateWithFlags(&g->side_st, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaEventCreateWithFlags(&g->ev_side_in, cudaEventDisableTiming) == cudaSuccess &&
                      cudaEventCreateWithFlags(&g->ev_side_out, cudaEventDisableTiming) == cudaSuccess;
      if (!ok) {   // without the side stream the steps stay sequential
        cudaGetLastError();
        if (g->side_st) cudaStreamDestroy(g->side_st);
        g->side_st = nullptr;
      }
    }
  }
  cudaMemset(g->status, 0, 2 * sizeof(int));
  cudaMemset(g->lz_b, 0, 16 * g->n_sub * sizeof(double));
  cudaMemset(g->cw, 0, g->tot_states * sizeof(double));
  cudaMemset(g->lam, 0, g->tot_states * sizeof(double));
  for (int i = 0; i < 6; ++i) cudaEventCreate(&g->ev[i]);
  cudaError_t e = cudaMemcpy(g->d_subs, g->subs.data(), g->n_sub * sizeof(SubDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_subs1, g->subs1.data(), g->n_sub * sizeof(SubDev), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    xls_grid_destroy(g);
    return fail(XLS_ECUDA, cudaGetErrorString(e));
  }
  *out = g;
  return XLS_OK;
}

// device bytes of one subdomain on a grid (blocks, potential, subspace matrices, per-state
// arrays, Lanczos vectors, projector tables estimated at four supports per point)
size_t sub_footprint(const SubDev& S, size_t elem) {
  const size_t nd = (size_t)S.nd, ns = (size_t)S.ns;
  return 3 * nd * ns * elem + nd * 12 + 7 * ns * ns * 8 + 11 * ns * 8 + 4 * nd * 8 + nd * 4 * 104 + nd * 8;
}


// ---- wave mode ---------------------------------------------------------------------------------
size_t store_elem(xls_grid g) { return g->store16 ? 2 : g->elem; }
char* store_ptr(xls_grid g, int sub) { return (char*)g->store + (size_t)g->subs[sub].off_blk * store_elem(g); }

// the pinned host store of every subdomain's orbitals (compute precision), allocated at first use
xls_status ensure_store(xls_grid g) {
  if (g->store) return XLS_OK;
  if (g->carry) return fail(XLS_EINVAL, "wave carry mode keeps no orbital store");
  if (cudaMallocHost(&g->store, g->tot_blk * g->elem) != cudaSuccess) {
    cudaGetLastError();
    g->store = nullptr;
    return fail(XLS_ENOMEM, "wave mode: pinned host store for the orbitals could not be allocated");
  }
  std::memset(g->store, 0, g->tot_blk * g->elem);
  return XLS_OK;
}

// device staging block of one subdomain (wave mode), allocated at first use
xls_status ensure_stage(xls_grid g) {
  if (g->blk[0]) return XLS_OK;
  long long max_blk = 0;
  for (const SubDev& S : g->subs) max_blk = std::max(max_blk, S.nd * S.ns);
  return g->alloc(&g->blk[0], max_blk * std::max<size_t>(g->elem, 8));
}

// the stored block of subdomain `sub` into device memory `dev` in the compute precision of the
// wave grid g (the store's format: a plain copy, or halves + exponents converted on the device)
xls_status store_to_device(xls_grid g, int sub, void* dev, cudaStream_t st) {
  const SubDev& S = g->subs[sub];
  const size_t n = (size_t)S.nd * S.ns;
  if (!g->store16) {
    XLS_CUDA(cudaMemcpyAsync(dev, store_ptr(g, sub), n * g->elem, cudaMemcpyHostToDevice, st));
    return XLS_OK;
  }
  XLS_CUDA(cudaMemcpyAsync(g->stage16, store_ptr(g, sub), n * 2, cudaMemcpyHostToDevice, st));
  const int* ex = g->d_store_ex + S.off_state;
  if (g->prec == XLS_FP64) launch_load_half<double>(g->stage16, S.nd, S.ns, ex, (double*)dev, st);
  else launch_load_half<float>(g->stage16, S.nd, S.ns, ex, (float*)dev, st);
  XLS_CUDA(cudaGetLastError());
  return XLS_OK;
}

// device block `dev` (compute precision) of subdomain `sub` into the store, queued on st (the
// FP16 store's exponents stay on the device; the halves go through the one staging buffer, whose
// reuse the stream orders)
xls_status device_to_store(xls_grid g, int sub, const void* dev, cudaStream_t st) {
  const SubDev& S = g->subs[sub];
  const size_t n = (size_t)S.nd * S.ns;
  if (!g->store16) {
    XLS_CUDA(cudaMemcpyAsync(store_ptr(g, sub), dev, n * g->elem, cudaMemcpyDeviceToHost, st));
    return XLS_OK;
  }
  int* ex = g->d_store_ex + S.off_state;
  if (g->prec == XLS_FP64) launch_store_half<double>((const double*)dev, S.nd, S.ns, ex, g->stage16, st);
  else launch_store_half<float>((const float*)dev, S.nd, S.ns, ex, g->stage16, st);
  XLS_CUDA(cudaGetLastError());
  XLS_CUDA(cudaMemcpyAsync(store_ptr(g, sub), g->stage16, n * 2, cudaMemcpyDeviceToHost, st));
  return XLS_OK;
}

// the partial grid of wave w with the Hamiltonian of the wave-mode grid
xls_status wave_worker(xls_grid g, int w, xls_grid* out) {
  const int first = g->waves[w].first, cnt = g->waves[w].second;
  xls_dc dc{cnt, &g->dc_core_lo[3 * (size_t)first], &g->dc_core_n[3 * (size_t)first], &g->dc_buf[3 * (size_t)first],
            &g->dc_ns[first]};
  XLS_TRY(create_grid(&g->cell, &dc, g->prec, 0, g->st, out, true, false));
  const int na = (int)g->atom_sp.size();
  const xls_status s = xls_hamiltonian_set(*out, g->Vg, 1, na, na ? g->atom_pos.data() : nullptr,
                                           na ? g->atom_sp.data() : nullptr, (int)g->species.size(),
                                           g->species.empty() ? nullptr : g->species.data());
  if (s != XLS_OK) {
    xls_grid_destroy(*out);
    *out = nullptr;
  }
  return s;
}

xls_status wave_hamiltonian_set(xls_grid g, const double* veff, int veff_on_device, int n_atoms, const double* pos,
                                const int* species, int n_species, const xls_species* sp) {
  const long long ng = (long long)g->gn[0] * g->gn[1] * g->gn[2];
  if (!g->Vg) XLS_TRY(g->alloc(&g->Vg, ng * sizeof(double)));
  XLS_CUDA(cudaMemcpyAsync(g->Vg, veff, ng * sizeof(double),
                           veff_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->st));
  XLS_CUDA(cudaStreamSynchronize(g->st));
  g->atom_pos.assign(pos, pos + 3 * (size_t)n_atoms);
  g->atom_sp.assign(species, species + n_atoms);
  g->species.assign(sp, sp + n_species);
  g->ham_set = true;
  g->have_ritz = false;
  std::fill(g->wave_ran.begin(), g->wave_ran.end(), 0);   // Ritz values of the old potential
  return XLS_OK;
}

xls_status wave_orbitals_set(xls_grid g, int sub, const double* psi, int on_device) {
  if (g->carry) return fail(XLS_EINVAL, "xls_orbitals_set: wave carry mode draws its start block with xls_orbitals_random");
  XLS_TRY(ensure_store(g));
  XLS_TRY(ensure_stage(g));
  const SubDev& S = g->subs[sub];
  const size_t n = (size_t)S.nd * S.ns;
  std::vector<double> tmp;
  const double* src = psi;
  if (on_device) {
    tmp.resize(n);
    XLS_CUDA(cudaMemcpy(tmp.data(), psi, n * sizeof(double), cudaMemcpyDeviceToHost));
    src = tmp.data();
  }
  if (g->store16) {   // FP64 up, halves + exponents back
    XLS_CUDA(cudaMemcpyAsync(g->blk[0], src, n * sizeof(double), cudaMemcpyHostToDevice, g->st));
    launch_store_half<double>((const double*)g->blk[0], S.nd, S.ns, g->d_store_ex + S.off_state, g->stage16, g->st);
    XLS_CUDA(cudaGetLastError());
    XLS_CUDA(cudaMemcpyAsync(store_ptr(g, sub), g->stage16, n * 2, cudaMemcpyDeviceToHost, g->st));
    XLS_CUDA(cudaStreamSynchronize(g->st));
  } else if (g->prec == XLS_FP64) {
    std::memcpy(store_ptr(g, sub), src, n * sizeof(double));
  } else {
    float* dst = (float*)store_ptr(g, sub);
    for (size_t i = 0; i < n; ++i) dst[i] = (float)src[i];   // the rounding of the FP32 block
  }
  if (!g->core_fresh.empty()) g->core_fresh[sub] = 0;   // the device core rows are those of the old block
  g->orb_set = true;
  g->have_ritz = false;
  return XLS_OK;
}

int carry_slot(xls_grid g, int sub);

xls_status wave_orbitals_get(xls_grid g, int sub, double* out, int on_device) {
  if (g->carry) {
    const int j = carry_slot(g, sub);
    if (j < 0) return fail(XLS_EINVAL, "xls_orbitals_get: in wave carry mode only the subdomains of the last wave run");
    return xls_orbitals_get(g->worker, j, out, on_device);
  }
  XLS_TRY(ensure_store(g));
  XLS_TRY(ensure_stage(g));
  const SubDev& S = g->subs[sub];
  const size_t n = (size_t)S.nd * S.ns;
  std::vector<double> tmp;
  if (on_device) tmp.resize(n);
  double* dst = on_device ? tmp.data() : out;
  if (g->store16) {   // halves + exponents up, FP64 back
    XLS_CUDA(cudaMemcpyAsync(g->stage16, store_ptr(g, sub), n * 2, cudaMemcpyHostToDevice, g->st));
    launch_load_half<double>(g->stage16, S.nd, S.ns, g->d_store_ex + S.off_state, (double*)g->blk[0], g->st);
    XLS_CUDA(cudaGetLastError());
    XLS_CUDA(cudaMemcpyAsync(dst, g->blk[0], n * sizeof(double), cudaMemcpyDeviceToHost, g->st));
    XLS_CUDA(cudaStreamSynchronize(g->st));
  } else if (g->prec == XLS_FP64) {
    std::memcpy(dst, store_ptr(g, sub), n * sizeof(double));
  } else {
    const float* src = (const float*)store_ptr(g, sub);
    for (size_t i = 0; i < n; ++i) dst[i] = src[i];
  }
  if (on_device) XLS_CUDA(cudaMemcpy(out, tmp.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  return XLS_OK;
}

xls_status carry_orbitals_random(xls_grid g, uint64_t seed);

xls_status wave_orbitals_random(xls_grid g, uint64_t seed) {
  if (g->carry) return carry_orbitals_random(g, seed);
  XLS_TRY(ensure_store(g));
  XLS_TRY(ensure_stage(g));
  for (int a = 0; a < g->n_sub; ++a) {
    const SubDev& S = g->subs[a];
    const long long n = S.nd * S.ns;
    if (g->prec == XLS_FP64) launch_splitmix_fill_f64((double*)g->blk[0], n, seed, S.off_blk, g->st);
    else launch_splitmix_fill_f32((float*)g->blk[0], n, seed, S.off_blk, g->st);
    XLS_TRY(device_to_store(g, a, g->blk[0], g->st));
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  std::fill(g->core_fresh.begin(), g->core_fresh.end(), (char)0);
  g->orb_set = true;
  g->have_ritz = false;
  return XLS_OK;
}

// one wave of a wave-mode grid with an orbital store: partial grid, orbitals up, passes,
// orbitals / Ritz values / weights / bounds back, partial grid released
// fresh_b: the potential changed since the last pass (an SCF step): the upper bound b of every
// subdomain is the worker's new Lanczos bound, a and a0 stay those of the last pass's Ritz values
// (what the resident grid's SCF step does with its Lanczos bounds)
// the compact core store and its density descriptors (subdomain a's core box is a block of its
// own, at the prefix of the core points x states before it)
xls_status alloc_core_store(xls_grid g) {
  std::vector<SubDev> cs(g->subs);
  long long off = 0;
  for (SubDev& S : cs) {
    const long long core_pts = (long long)S.core_n[0] * S.core_n[1] * S.core_n[2];
    for (int d = 0; d < 3; ++d) {
      S.n[d] = S.core_n[d];
      S.periodic[d] = 0;
      S.start[d] = S.core_glo[d];
      S.core_lo[d] = 0;
    }
    S.nd = core_pts;
    S.off_blk = off;
    off += core_pts * S.ns;
  }
  XLS_TRY(g->alloc(&g->core_store, (size_t)off * g->elem));
  const xls_status s = g->alloc(&g->d_core_subs, g->n_sub * sizeof(SubDev));
  if (s != XLS_OK) {
    g->release(&g->core_store);
    return s;
  }
  XLS_CUDA(cudaMemcpy(g->d_core_subs, cs.data(), cs.size() * sizeof(SubDev), cudaMemcpyHostToDevice));
  std::fill(g->core_fresh.begin(), g->core_fresh.end(), (char)0);
  return XLS_OK;
}

// core rows of the worker k's blocks (subdomains first .. first + k->n_sub - 1) into the store
void gather_cores(xls_grid g, xls_grid k, int first) {
  if (g->prec == XLS_FP64)
    launch_core_gather<double>(k->d_subs, k->n_sub, k->max_ns, (const double*)k->blk[k->cur], (double*)g->core_store,
                               g->d_core_subs + first, g->st);
  else
    launch_core_gather<float>(k->d_subs, k->n_sub, k->max_ns, (const float*)k->blk[k->cur], (float*)g->core_store,
                              g->d_core_subs + first, g->st);
}

xls_status wave_run(xls_grid g, int w, int degree, int n_passes, const double* bounds, bool fresh_b, int& launches) {
  XLS_TRY(ensure_store(g));
  // XLS_TRACE=1: host wall times of the wave's phases on stderr (diagnostics)
  static const bool trace = std::getenv("XLS_TRACE") != nullptr;
  auto tnow = []() { return std::chrono::steady_clock::now(); };
  auto tms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  const auto t0 = tnow();
  const int first = g->waves[w].first, cnt = g->waves[w].second;
  xls_grid k = nullptr;
  XLS_TRY(wave_worker(g, w, &k));
  const auto t1 = tnow();
  xls_status s = XLS_OK;
  for (int j = 0; j < cnt && s == XLS_OK; ++j)
    s = store_to_device(g, first + j, (char*)k->blk[k->cur] + (size_t)k->subs[j].off_blk * k->elem, g->st);
  if (trace) cudaStreamSynchronize(g->st);
  const auto t2 = tnow();
  k->orb_set = true;
  const double* bw = bounds ? bounds + 3 * (size_t)first
                            : (g->have_ritz ? g->host_bounds.data() + 3 * (size_t)first : nullptr);
  std::vector<double> mixed;
  if (s == XLS_OK && fresh_b && bw) {
    mixed.assign(bw, bw + 3 * (size_t)cnt);
    std::vector<double> wb(3 * (size_t)cnt);
    s = xls_get_bounds(k, wb.data());
    for (int j = 0; j < cnt; ++j) mixed[3 * (size_t)j] = wb[3 * (size_t)j];
    bw = mixed.data();
  }
  if (s == XLS_OK) s = xls_chefsi_batch(k, degree, n_passes, bw);
  if (s == XLS_OK && g->core_reserve && !g->core_store) s = alloc_core_store(g);
  if (s == XLS_OK && g->core_store) {
    gather_cores(g, k, first);
    if (cudaGetLastError() != cudaSuccess) s = fail(XLS_ECUDA, "wave: core-row gather failed");
    std::fill(g->core_fresh.begin() + first, g->core_fresh.begin() + first + cnt, (char)1);
  }
  if (trace) cudaStreamSynchronize(g->st);
  const auto t3 = tnow();
  if (s == XLS_OK) {
    const SubDev& S0 = g->subs[first];
    cudaMemcpyAsync(g->lam + S0.off_state, k->lam, k->tot_states * sizeof(double), cudaMemcpyDeviceToDevice, g->st);
    cudaMemcpyAsync(g->cw + S0.off_state, k->cw, k->tot_states * sizeof(double), cudaMemcpyDeviceToDevice, g->st);
    s = xls_get_bounds(k, g->host_bounds.data() + 3 * (size_t)first);
  }
  for (int j = 0; j < cnt && s == XLS_OK; ++j)
    s = device_to_store(g, first + j, (const char*)k->blk[k->cur] + (size_t)k->subs[j].off_blk * k->elem, g->st);
  if (s == XLS_OK && cudaStreamSynchronize(g->st) != cudaSuccess) s = fail(XLS_ECUDA, "wave: synchronisation failed");
  const auto t4 = tnow();
  if (s == XLS_OK) {
    for (int i = 0; i < 4; ++i) g->wave_stage_ms[i] += k->stage_ms[i];
    launches += k->last_launches + (g->core_store ? 1 : 0);
  }
  xls_grid_destroy(k);
  if (trace) {
    const auto t5 = tnow();
    std::fprintf(stderr, "[xls] store wave %d (%d subdomains): worker + Hamiltonian %.1f ms, load %.1f ms, passes %.1f ms, "
                 "store %.1f ms, destroy %.1f ms\n", w, cnt, tms(t0, t1), tms(t1, t2), tms(t2, t3), tms(t3, t4),
                 tms(t4, t5));
  }
  return s;
}

// ---- carry mode -----------------------------------------------------------------------------
// every subdomain of the grid has the shape of subdomain 0 (grid points, boundary conditions,
// core box position inside the subdomain, states)
bool uniform_shapes(xls_grid g) {
  const SubDev& A = g->subs[0];
  for (const SubDev& S : g->subs)
    for (int d = 0; d < 3; ++d)
      if (S.n[d] != A.n[d] || S.periodic[d] != A.periodic[d] || S.core_lo[d] != A.core_lo[d] ||
          S.core_n[d] != A.core_n[d] || S.ns != A.ns)
        return false;
  return true;
}

// the worker's slots take the subdomains first .. first + W - 1 of the grid: descriptors moved
// (same shapes, new positions), then V_eff restricted, projector tables rebuilt and the Lanczos
// bound of every slot taken (xls_hamiltonian_set of the worker)
xls_status carry_retarget(xls_grid g, int first) {
  xls_grid k = g->worker;
  for (int j = 0; j < k->n_sub; ++j) {
    const SubDev& S = g->subs[first + j];
    for (int d = 0; d < 3; ++d) {
      k->subs[j].start[d] = k->subs1[j].start[d] = S.start[d];
      k->subs[j].core_glo[d] = k->subs1[j].core_glo[d] = S.core_glo[d];
    }
  }
  XLS_CUDA(cudaMemcpyAsync(k->d_subs, k->subs.data(), k->n_sub * sizeof(SubDev), cudaMemcpyHostToDevice, g->st));
  XLS_CUDA(cudaMemcpyAsync(k->d_subs1, k->subs1.data(), k->n_sub * sizeof(SubDev), cudaMemcpyHostToDevice, g->st));
  const int na = (int)g->atom_sp.size();
  return xls_hamiltonian_set(k, g->Vg, 1, na, na ? g->atom_pos.data() : nullptr, na ? g->atom_sp.data() : nullptr,
                             (int)g->species.size(), g->species.empty() ? nullptr : g->species.data());
}

// the worker slot holding subdomain `sub` (carry mode: only the subdomains of the wave it ran last)
int carry_slot(xls_grid g, int sub) {
  if (!g->carry || !g->worker || g->carry_last < 0) return -1;
  const int first = g->waves[g->carry_last].first, cnt = g->waves[g->carry_last].second;
  return (sub >= first && sub < first + cnt) ? sub - first : -1;
}

xls_status carry_orbitals_random(xls_grid g, uint64_t seed) {
  xls_grid k = g->worker;
  // the stream values of the first wave's subdomains (blocks concatenated in subdomain order)
  if (k->prec == XLS_FP64) launch_splitmix_fill_f64((double*)k->blk[k->cur], k->tot_blk, seed, 0, k->st);
  else launch_splitmix_fill_f32((float*)k->blk[k->cur], k->tot_blk, seed, 0, k->st);
  XLS_CUDA(cudaGetLastError());
  k->orb_set = true;
  k->have_ritz = false;
  g->orb_set = true;
  g->have_ritz = false;
  g->carry_primed = false;
  std::fill(g->wave_ran.begin(), g->wave_ran.end(), 0);
  return XLS_OK;
}

// one wave in carry mode: the worker re-targeted to the wave, its passes from the block the
// previous wave left (bounds: b from the new Lanczos run; a, a0 from the subdomain's own last pass
// when it has one, else from the slot's last pass; the first wave after xls_orbitals_random
// takes them from a Rayleigh-Ritz step of the random block), then the Ritz values, weights,
// bounds and core rows of the orbitals copied out
xls_status carry_run(xls_grid g, int w, int degree, int n_passes, const double* bounds, int& launches) {
  xls_grid k = g->worker;
  const int first = g->waves[w].first, cnt = g->waves[w].second;
  // XLS_TRACE=1: host wall times of the wave's phases on stderr (diagnostics)
  static const bool trace = std::getenv("XLS_TRACE") != nullptr;
  const auto t0 = std::chrono::steady_clock::now();
  XLS_TRY(carry_retarget(g, first));
  if (trace) cudaStreamSynchronize(g->st);
  const auto t1 = std::chrono::steady_clock::now();
  g->carry_last = w;   // the worker's slots now hold this wave's subdomains
  k->orb_set = true;
  std::vector<double> bw;
  const double* bp = nullptr;
  if (bounds) {
    bp = bounds + 3 * (size_t)first;
  } else if (g->carry_primed) {
    bw.assign(3 * (size_t)cnt, 0.0);
    XLS_TRY(xls_get_bounds(k, bw.data()));   // b of the new Lanczos run
    for (int j = 0; j < cnt; ++j) {
      const bool own = g->wave_ran[w] != 0;
      const double* src = own ? g->host_bounds.data() + 3 * (size_t)(first + j) : g->carry_ab.data() + 3 * (size_t)j;
      bw[3 * (size_t)j + 1] = src[1];
      bw[3 * (size_t)j + 2] = src[2];
    }
    bp = bw.data();
  }
  XLS_TRY(xls_chefsi_batch(k, degree, n_passes, bp));
  const auto t2 = std::chrono::steady_clock::now();
  const SubDev& S0 = g->subs[first];
  XLS_CUDA(cudaMemcpyAsync(g->lam + S0.off_state, k->lam, k->tot_states * sizeof(double), cudaMemcpyDeviceToDevice,
                           g->st));
  XLS_CUDA(cudaMemcpyAsync(g->cw + S0.off_state, k->cw, k->tot_states * sizeof(double), cudaMemcpyDeviceToDevice,
                           g->st));
  gather_cores(g, k, first);
  XLS_CUDA(cudaGetLastError());
  XLS_TRY(xls_get_bounds(k, g->host_bounds.data() + 3 * (size_t)first));
  g->carry_ab.assign(g->host_bounds.begin() + 3 * (size_t)first, g->host_bounds.begin() + 3 * (size_t)(first + cnt));
  for (int i = 0; i < 4; ++i) g->wave_stage_ms[i] += k->stage_ms[i];
  // kernels of the re-targeting (restriction, projector norms and tables, reverse tables, unit
  // coefficients; 10 Lanczos steps of one H application each) and of the core-row gather
  launches += k->last_launches + k->setup_launches + 1;
  if (trace) {
    cudaStreamSynchronize(g->st);
    const auto t3 = std::chrono::steady_clock::now();
    auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
      return std::chrono::duration<double, std::milli>(b - a).count();
    };
    std::fprintf(stderr, "[xls] wave %d: set-up %.1f ms, passes %.1f ms, copies %.1f ms\n", w, ms(t0, t1), ms(t1, t2),
                 ms(t2, t3));
  }
  g->carry_primed = true;
  g->wave_ran[w] = 1;
  g->have_ritz = std::all_of(g->wave_ran.begin(), g->wave_ran.end(), [](char c) { return c != 0; });
  return XLS_OK;
}

// every wave in turn
xls_status wave_chefsi(xls_grid g, int degree, int n_passes, const double* bounds, bool fresh_b = false) {
  for (double& t : g->wave_stage_ms) t = 0.0;
  int launches = 0;
  for (size_t w = 0; w < g->waves.size(); ++w) {
    if (g->carry) XLS_TRY(carry_run(g, (int)w, degree, n_passes, bounds, launches));
    else XLS_TRY(wave_run(g, (int)w, degree, n_passes, bounds, fresh_b, launches));
  }
  g->last_launches = launches;
  g->have_ritz = true;
  return XLS_OK;
}

xls_status wave_density(xls_grid g, double n_electrons, double kT, double* mu_out, double* rho_out, int rho_on_device,
                        double* e_band_out, double* e_entropy_out) {
  if (!g->carry) {
    XLS_TRY(ensure_store(g));
    XLS_TRY(ensure_stage(g));
  }
  launch_fermi_occ(g->lam, g->cw, g->tot_states, n_electrons, kT, g->out4, g->occ, g->status, g->st);
  XLS_TRY(check_status(g));
  double h4[4];
  XLS_CUDA(cudaMemcpy(h4, g->out4, sizeof(h4), cudaMemcpyDeviceToHost));
  if (mu_out) *mu_out = h4[0];
  if (e_band_out) *e_band_out = h4[1];
  if (e_entropy_out) *e_entropy_out = h4[2];
  if (!rho_out) return XLS_OK;
  const long long ng = (long long)g->gn[0] * g->gn[1] * g->gn[2];
  if (!g->rho) XLS_TRY(g->alloc(&g->rho, ng * sizeof(double)));
  const bool from_cores =
      g->carry || (g->core_store && std::all_of(g->core_fresh.begin(), g->core_fresh.end(), [](char c) { return c != 0; }));
  if (from_cores) {   // the compact device store of the core rows
    if (g->prec == XLS_FP64)
      launch_density_occ<double>(g->d_core_subs, g->n_sub, g->max_core, (const double*)g->core_store, g->occ, g->gn,
                                 g->rho, g->st);
    else
      launch_density_occ<float>(g->d_core_subs, g->n_sub, g->max_core, (const float*)g->core_store, g->occ, g->gn,
                                g->rho, g->st);
    XLS_CUDA(cudaGetLastError());
  }
  // second sweep: every subdomain's block staged alone; its core points of rho written
  static const bool trace = std::getenv("XLS_TRACE") != nullptr;
  const auto ts0 = std::chrono::steady_clock::now();
  for (int a = 0; a < g->n_sub && !from_cores; ++a) {
    const SubDev& S = g->subs[a];
    const long long core = (long long)S.core_n[0] * S.core_n[1] * S.core_n[2];
    XLS_TRY(store_to_device(g, a, g->blk[0], g->st));
    if (g->prec == XLS_FP64)
      launch_density_occ<double>(g->d_subs + a, 1, core, (const double*)g->blk[0], g->occ, g->gn, g->rho, g->st);
    else
      launch_density_occ<float>(g->d_subs + a, 1, core, (const float*)g->blk[0], g->occ, g->gn, g->rho, g->st);
  }
  XLS_CUDA(cudaMemcpyAsync(rho_out, g->rho, ng * sizeof(double),
                           rho_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->st));
  XLS_CUDA(cudaStreamSynchronize(g->st));
  if (trace)
    std::fprintf(stderr, "[xls] density: %s %.1f ms\n", from_cores ? "device core store" : "second sweep over the store",
                 std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts0).count());
  return XLS_OK;
}

xls_status not_in_wave_mode(const char* what) {
  return fail(XLS_EINVAL, std::string(what) + ": not available on a grid running in waves (HBM budget below its footprint)");
}

}  // namespace

extern "C" {

xls_status xls_grid_create(const xls_cell* cell, const xls_dc* dc, int precision, size_t hbm_budget_bytes,
                           void* cuda_stream, xls_grid* out) {
  if (!cell || !dc || !out || dc->n_sub < 1 || !dc->core_lo || !dc->core_n || !dc->buf || !dc->n_states)
    return fail(XLS_EINVAL, "xls_grid_create: null argument or n_sub < 1");
  if (precision != XLS_FP64 && precision != XLS_MIXED_BF16 && precision != XLS_MIXED_FP16)
    return fail(XLS_EINVAL, "unknown precision");
  for (int d = 0; d < 3; ++d)
    if (cell->n[d] < 2 * kN0 + 1 || !(cell->L[d] > 0)) return fail(XLS_EINVAL, "cell: n >= 13 and L > 0 per axis");
  if (hbm_budget_bytes == 0) return create_grid(cell, dc, precision, 0, cuda_stream, out, false, false);
  // HBM budget: everything at once if it fits, else waves of consecutive subdomains
  xls_grid probe = nullptr;
  XLS_TRY(create_grid(cell, dc, precision, 0, cuda_stream, &probe, false, false, true));
  const size_t elem = precision == XLS_FP64 ? 8 : 4;
  size_t total = 1 << 26, run = 0;
  std::vector<std::pair<int, int>> waves;
  int first = 0;
  // the compact store of the core rows (density without a second sweep over the host store) is
  // reserved when it takes at most an eighth of the budget
  size_t core_bytes = 0;
  for (const SubDev& S : probe->subs) core_bytes += (size_t)S.core_n[0] * S.core_n[1] * S.core_n[2] * S.ns * elem;
  const size_t core_reserve = core_bytes <= hbm_budget_bytes / 8 ? core_bytes : 0;
  const size_t fixed = ((size_t)1 << 26) + core_reserve;  // per-grid plans, events and small tables
  for (int a = 0; a < probe->n_sub; ++a) {
    const size_t f = sub_footprint(probe->subs[a], elem);
    total += f;
    if (f + fixed > hbm_budget_bytes) {
      delete probe;
      return fail(XLS_ENOMEM, "HBM budget below the footprint of subdomain " + std::to_string(a));
    }
    if (run + f + fixed > hbm_budget_bytes) {
      waves.push_back({first, a - first});
      first = a;
      run = 0;
    }
    run += f;
  }
  waves.push_back({first, probe->n_sub - first});
  delete probe;   // descriptors only: nothing allocated
  if (total <= hbm_budget_bytes) return create_grid(cell, dc, precision, hbm_budget_bytes, cuda_stream, out, false, false);
  xls_grid g = nullptr;
  XLS_TRY(create_grid(cell, dc, precision, hbm_budget_bytes, cuda_stream, &g, false, true));
  g->waves = waves;
  g->core_reserve = core_reserve;
  g->core_fresh.assign(g->n_sub, 0);
  g->dc_core_lo.assign(dc->core_lo, dc->core_lo + 3 * (size_t)dc->n_sub);
  g->dc_core_n.assign(dc->core_n, dc->core_n + 3 * (size_t)dc->n_sub);
  g->dc_buf.assign(dc->buf, dc->buf + 3 * (size_t)dc->n_sub);
  g->dc_ns.assign(dc->n_states, dc->n_states + dc->n_sub);
  *out = g;
  return XLS_OK;
}

xls_status xls_grid_destroy(xls_grid g) {
  if (!g) return XLS_OK;
  if (g->st) cudaStreamSynchronize(g->st);
  else cudaDeviceSynchronize();
  for (const auto& a : g->allocs) cudaFree(a.first);
  for (int i = 0; i < 6; ++i)
    if (g->ev[i]) cudaEventDestroy(g->ev[i]);
  for (auto& e : g->pev) cudaEventDestroy(e);
  g->drop_graphs();
  if (g->cap_st) cudaStreamDestroy(g->cap_st);
  for (auto& v : g->halves) {
    if (v.st) cudaStreamDestroy(v.st);
    if (v.ev) cudaEventDestroy(v.ev);
  }
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_mid) cudaEventDestroy(g->ev_mid);
  if (g->side_st) cudaStreamDestroy(g->side_st);
  if (g->ev_side_in) cudaEventDestroy(g->ev_side_in);
  if (g->ev_side_out) cudaEventDestroy(g->ev_side_out);
  if (g->worker) xls_grid_destroy(g->worker);
  if (g->store) cudaFreeHost(g->store);
  if (g->stage16) cudaFree(g->stage16);
  if (g->d_store_ex) cudaFree(g->d_store_ex);
  delete g;
  return XLS_OK;
}

xls_status xls_hamiltonian_set(xls_grid g, const double* veff, int veff_on_device, int n_atoms, const double* pos,
                               const int* species, int n_species, const xls_species* sp) {
  if (!g || !veff || n_atoms < 0 || (n_atoms > 0 && (!pos || !species || !sp || n_species < 1)))
    return fail(XLS_EINVAL, "xls_hamiltonian_set: bad arguments");
  for (int i = 0; i < n_atoms; ++i)
    if (species[i] < 0 || species[i] >= n_species) return fail(XLS_EINVAL, "species index out of range");
  if (!g->graphs.empty()) {  // captured passes hold the previous operator's tables
    XLS_CUDA(cudaStreamSynchronize(g->st));
    g->drop_graphs();
  }
  for (int s = 0; s < n_species; ++s)
    for (int d = 0; d < 3; ++d)
      if (!(sp[s].r_cut > 0) || !(sp[s].w_proj > 0) || 2 * sp[s].r_cut >= g->gL[d])
        return fail(XLS_EINVAL, "projector cutoff must be positive and below half of every cell edge");
  if (g->wave) return wave_hamiltonian_set(g, veff, veff_on_device, n_atoms, pos, species, n_species, sp);
  static const bool trace = std::getenv("XLS_TRACE") != nullptr;
  auto tnow = []() { return std::chrono::steady_clock::now(); };
  auto tms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  const auto h0 = tnow();
  int nl = 0;   // kernels launched by the set-up (for the caller's launch count)
  const long long ng = (long long)g->gn[0] * g->gn[1] * g->gn[2];
  if (!g->Vg) {
    xls_status s = g->alloc(&g->Vg, ng * sizeof(double));
    if (s != XLS_OK) return s;
  }
  const bool same_geometry =
      g->norm_valid && g->atom_pos.size() == 3 * (size_t)n_atoms && g->atom_sp.size() == (size_t)n_atoms &&
      g->species.size() == (size_t)n_species &&
      (n_atoms == 0 || (std::memcmp(g->atom_pos.data(), pos, 3 * (size_t)n_atoms * sizeof(double)) == 0 &&
                        std::memcmp(g->atom_sp.data(), species, (size_t)n_atoms * sizeof(int)) == 0 &&
                        std::memcmp(g->species.data(), sp, (size_t)n_species * sizeof(xls_species)) == 0));
  g->atom_pos.assign(pos, pos + 3 * (size_t)n_atoms);
  g->atom_sp.assign(species, species + n_atoms);
  g->species.assign(sp, sp + n_species);
  g->scf.pc_ready = false;
  XLS_CUDA(cudaMemcpyAsync(g->Vg, veff, ng * sizeof(double),
                           veff_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->st));
  launch_restrict(g->d_subs, g->n_sub, g->max_nd, g->Vg, g->gn, g->V, g->Vf, g->st); ++nl;
  // projector normalisation on the global grid (one image per atom, wrapped box)
  std::vector<double> norms(4 * (size_t)n_atoms, 1.0);
  if (same_geometry) norms = g->norm_cache;
  if (n_atoms > 0 && !same_geometry) {
    std::vector<AtomImg> glob(n_atoms);
    std::vector<ProjSlot> gslot(n_atoms);
    for (int i = 0; i < n_atoms; ++i) {
      const xls_species& q = sp[species[i]];
      AtomImg& A = glob[i];
      for (int d = 0; d < 3; ++d) {
        double r = std::fmod(pos[3 * i + d], g->gL[d]);
        if (r < 0) r += g->gL[d];
        A.R[d] = r;
        A.box_lo[d] = (int)std::floor((r - q.r_cut) / g->gh[d]);
        A.box_n[d] = (int)std::ceil((r + q.r_cut) / g->gh[d]) - A.box_lo[d] + 1;
      }
      A.slot = i;
      gslot[i] = ProjSlot{};
      gslot[i].w = q.w_proj;
      gslot[i].rcut2 = q.r_cut * q.r_cut;
    }
    AtomImg* dglob = nullptr;
    ProjSlot* dgs = nullptr;
    double* dn = nullptr;
    XLS_CUDA(cudaMalloc(&dglob, n_atoms * sizeof(AtomImg)));
    XLS_CUDA(cudaMalloc(&dgs, n_atoms * sizeof(ProjSlot)));
    XLS_CUDA(cudaMalloc(&dn, 4 * (size_t)n_atoms * sizeof(double)));
    XLS_CUDA(cudaMemcpyAsync(dglob, glob.data(), n_atoms * sizeof(AtomImg), cudaMemcpyHostToDevice, g->st));
    XLS_CUDA(cudaMemcpyAsync(dgs, gslot.data(), n_atoms * sizeof(ProjSlot), cudaMemcpyHostToDevice, g->st));
    launch_proj_norms(dglob, dgs, n_atoms, g->gn, g->gh, dn, g->st); ++nl;
    XLS_CUDA(cudaMemcpyAsync(norms.data(), dn, 4 * (size_t)n_atoms * sizeof(double), cudaMemcpyDeviceToHost, g->st));
    XLS_CUDA(cudaStreamSynchronize(g->st));
    cudaFree(dglob);
    cudaFree(dgs);
    cudaFree(dn);
  }
  g->norm_cache = norms;
  g->norm_valid = true;
  const auto h1 = tnow();
  // projector slots (atom x subdomain) and their periodic images; the atoms are visited in the
  // Z-order (Morton order) of their grid cells of 8 points, so that consecutive slots of a
  // subdomain are spatial neighbours (the projection walks slots in chunks that then share points)
  std::vector<int> aorder(n_atoms);
  {
    std::vector<std::pair<unsigned long long, int>> key(n_atoms);
    for (int i = 0; i < n_atoms; ++i) {
      unsigned long long m = 0;
      unsigned c[3];
      for (int d = 0; d < 3; ++d) {
        double r = std::fmod(pos[3 * i + d], g->gL[d]);
        if (r < 0) r += g->gL[d];
        c[d] = (unsigned)(r / (8.0 * g->gh[d]));
      }
      for (int bit = 0; bit < 20; ++bit)
        for (int d = 0; d < 3; ++d) m |= (unsigned long long)((c[d] >> bit) & 1u) << (3 * bit + d);
      key[i] = {m, i};
    }
    std::stable_sort(key.begin(), key.end());
    for (int i = 0; i < n_atoms; ++i) aorder[i] = key[i].second;
  }
  std::vector<AtomImg> imgs;
  std::vector<ProjSlot> slots;
  long long poff = 0;
  for (int a = 0; a < g->n_sub; ++a) {
    const size_t first = slots.size();
    for (int ii = 0; ii < n_atoms; ++ii) {
      const int i = aorder[ii];
      const xls_species& q = sp[species[i]];
      const size_t before = imgs.size();
      atom_images(g, a, pos + 3 * i, q, (int)slots.size(), imgs);
      if (imgs.size() == before) continue;
      ProjSlot Q{};
      Q.sub = a;
      Q.atom = i;
      Q.img_lo = (int)before;
      Q.img_n = (int)(imgs.size() - before);
      Q.w = q.w_proj;
      Q.rcut2 = q.r_cut * q.r_cut;
      for (int l = 0; l < 4; ++l) Q.norm[l] = norms[4 * i + l];
      Q.E[0] = q.E_s;
      Q.E[1] = Q.E[2] = Q.E[3] = q.E_p;
      slots.push_back(Q);
    }
    g->subs[a].slot_lo = g->subs1[a].slot_lo = (int)first;
    g->subs[a].slot_n = g->subs1[a].slot_n = (int)(slots.size() - first);
    g->subs[a].off_proj = poff;
    poff += 4LL * g->subs[a].ns * g->subs[a].slot_n;
    g->subs1[a].off_proj = 4LL * (long long)first;
  }
  std::vector<int> nlb_sub;   // subdomain of every back-projection point block
  for (int a = 0; a < g->n_sub; ++a) {
    g->subs[a].off_nlb = g->subs1[a].off_nlb = (int)nlb_sub.size();
    for (long long p = 0; p < g->subs[a].nd; p += kBackPts) nlb_sub.push_back(a);
    if (g->subs[a].slot_n > 32768) return fail(XLS_EINVAL, "more than 32768 projector slots in one subdomain");
  }
  g->n_slot = (int)slots.size();
  xls_status s;
  if ((s = g->reserve(&g->d_imgs, imgs.size() * sizeof(AtomImg))) != XLS_OK) return s;
  if ((s = g->reserve(&g->d_slots, slots.size() * sizeof(ProjSlot))) != XLS_OK) return s;
  if ((s = g->reserve(&g->P, std::max<long long>(poff, 1) * sizeof(double))) != XLS_OK) return s;
  if ((s = g->reserve(&g->P1, std::max<size_t>(4 * slots.size(), 1) * sizeof(double))) != XLS_OK) return s;
  if (!imgs.empty())
    XLS_CUDA(cudaMemcpyAsync(g->d_imgs, imgs.data(), imgs.size() * sizeof(AtomImg), cudaMemcpyHostToDevice, g->st));
  if (!slots.empty())
    XLS_CUDA(cudaMemcpyAsync(g->d_slots, slots.data(), slots.size() * sizeof(ProjSlot), cudaMemcpyHostToDevice, g->st));
  XLS_CUDA(cudaMemcpyAsync(g->d_subs, g->subs.data(), g->n_sub * sizeof(SubDev), cudaMemcpyHostToDevice, g->st));
  XLS_CUDA(cudaMemcpyAsync(g->d_subs1, g->subs1.data(), g->n_sub * sizeof(SubDev), cudaMemcpyHostToDevice, g->st));
  // projector tables: count the points of every slot, lay the tables out, fill them
  if (!slots.empty()) {
    int* dcnt = nullptr;
    if ((s = g->reserve(&g->scr_a, slots.size() * sizeof(int))) != XLS_OK) return s;
    dcnt = (int*)g->scr_a;
    launch_proj_table_count<double>(g->d_subs, g->d_slots, g->n_slot, g->d_imgs, dcnt, g->st); ++nl;
    std::vector<int> cnt(slots.size());
    XLS_CUDA(cudaMemcpyAsync(cnt.data(), dcnt, cnt.size() * sizeof(int), cudaMemcpyDeviceToHost, g->st));
    XLS_CUDA(cudaStreamSynchronize(g->st));
    long long tot = 0;
    for (size_t k = 0; k < slots.size(); ++k) {
      slots[k].pt_off = tot;
      slots[k].pt_n = cnt[k];
      tot += cnt[k];
    }
    XLS_CUDA(cudaMemcpyAsync(g->d_slots, slots.data(), slots.size() * sizeof(ProjSlot), cudaMemcpyHostToDevice, g->st));
    if ((s = g->reserve(&g->d_pidx, std::max<long long>(tot, 1) * sizeof(int))) != XLS_OK) return s;
    if ((s = g->reserve(&g->d_chi64, std::max<long long>(tot, 1) * sizeof(double4))) != XLS_OK) return s;
    launch_proj_table_fill<double>(g->d_subs, g->d_slots, g->n_slot, g->d_imgs, g->d_pidx, g->d_chi64, g->st); ++nl;
    if (g->prec != XLS_FP64) {
      if ((s = g->reserve(&g->d_chi32, std::max<long long>(tot, 1) * sizeof(float4))) != XLS_OK) return s;
      launch_proj_table_fill<float>(g->d_subs, g->d_slots, g->n_slot, g->d_imgs, g->d_pidx, g->d_chi32, g->st); ++nl;
    }
    // reverse tables: count per grid point, exclusive prefix (device), fill
    int* dc = nullptr;
    int* dcur = nullptr;
    if ((s = g->reserve(&g->scr_a, g->tot_pts * sizeof(int))) != XLS_OK) return s;
    if ((s = g->reserve(&g->scr_b, g->tot_pts * sizeof(int))) != XLS_OK) return s;
    dc = (int*)g->scr_a;
    dcur = (int*)g->scr_b;
    XLS_CUDA(cudaMemsetAsync(dc, 0, g->tot_pts * sizeof(int), g->st));
    launch_rcsr_count(g->d_subs, g->d_slots, g->n_slot, g->d_pidx, dc, g->st); ++nl;
    // row pointers by a device prefix sum; only the total comes back to size the tables
    if ((s = g->reserve(&g->d_rptr, (g->tot_pts + 1) * sizeof(long long))) != XLS_OK) return s;
    long long* dtmp = nullptr;
    if ((s = g->reserve(&g->scr_c, scan_temp_count(g->tot_pts) * sizeof(long long))) != XLS_OK) return s;
    dtmp = (long long*)g->scr_c;
    launch_exclusive_scan(dc, g->tot_pts, dtmp, g->d_rptr, g->st); nl += 3;
    long long n_entries = 0;
    XLS_CUDA(cudaMemcpyAsync(&n_entries, g->d_rptr + g->tot_pts, sizeof(long long), cudaMemcpyDeviceToHost, g->st));
    XLS_CUDA(cudaStreamSynchronize(g->st));
    const std::vector<long long> rp{0, n_entries};   // rp.back(): the number of table entries
    if ((s = g->reserve(&g->d_rslot, std::max<long long>(rp.back(), 1) * sizeof(int))) != XLS_OK) return s;
    if ((s = g->reserve(&g->d_rchi64, std::max<long long>(rp.back(), 1) * sizeof(double4))) != XLS_OK) return s;
    XLS_CUDA(cudaMemsetAsync(dcur, 0, g->tot_pts * sizeof(int), g->st));
    launch_rcsr_build<double>(g->d_subs, g->d_slots, g->n_slot, g->d_pidx, g->d_chi64, g->d_rptr, dcur, g->d_rslot,
                              g->d_rchi64, g->st); ++nl;
    if (g->prec != XLS_FP64) {
      if ((s = g->reserve(&g->d_rchi32, std::max<long long>(rp.back(), 1) * sizeof(float4))) != XLS_OK) return s;
      // same entry order as the FP64 table (the fill order of the atomics is not reproducible)
      launch_convert_f64_f32((const double*)g->d_rchi64, (float*)g->d_rchi32, 4 * rp.back(), g->st); ++nl;
    }
    XLS_CUDA(cudaStreamSynchronize(g->st));
    g->max_slots = 0;
    for (const SubDev& S : g->subs) g->max_slots = std::max(g->max_slots, S.slot_n);
    // per point block of the back-projection: the slots its rows name (rows' entries as ranks)
          const int n_nlb = (int)nlb_sub.size();
    if ((s = g->reserve(&g->d_nlb_sub, n_nlb * sizeof(int))) != XLS_OK) return s;
    if ((s = g->reserve(&g->d_nlb_cnt, n_nlb * sizeof(int))) != XLS_OK) return s;
    XLS_CUDA(cudaMemcpyAsync(g->d_nlb_sub, nlb_sub.data(), n_nlb * sizeof(int), cudaMemcpyHostToDevice, g->st));
    launch_rcsr_localize(g->d_subs, g->d_nlb_sub, n_nlb, g->d_rptr, g->d_rslot, g->d_nlb_cnt, nullptr, 0, 0, g->st);
    ++nl;
    std::vector<int> cnt_b(n_nlb);
    XLS_CUDA(cudaMemcpyAsync(cnt_b.data(), g->d_nlb_cnt, n_nlb * sizeof(int), cudaMemcpyDeviceToHost, g->st));
    XLS_CUDA(cudaStreamSynchronize(g->st));
    g->nlb_max = 0;
    for (int c : cnt_b) g->nlb_max = std::max(g->nlb_max, c);
    if ((s = g->reserve(&g->d_nlb_list, std::max<size_t>((size_t)n_nlb * g->nlb_max, 1) * sizeof(int))) != XLS_OK)
      return s;
    launch_rcsr_localize(g->d_subs, g->d_nlb_sub, n_nlb, g->d_rptr, g->d_rslot, g->d_nlb_cnt, g->d_nlb_list,
                         g->nlb_max, 1, g->st); ++nl;
    XLS_CUDA(cudaGetLastError());
  }
  const auto h2 = tnow();
  set_view_slots(g, g->full);
  if (g->concurrent)
    for (auto& v : g->halves) set_view_slots(g, v);
  // unit coefficients (plain H) for every subdomain, then the Lanczos bound b
  std::vector<double> bz(3 * g->n_sub, 1.0);
  for (int a = 0; a < g->n_sub; ++a) { bz[3 * a] = 2.0; bz[3 * a + 1] = 1.0; bz[3 * a + 2] = 0.0; }
  XLS_CUDA(cudaMemcpyAsync(g->bounds, bz.data(), bz.size() * sizeof(double), cudaMemcpyHostToDevice, g->st));
  launch_filter_coef(g->n_sub, g->bounds, 1, g->coef, g->st); ++nl;
  XLS_TRY(lanczos_bounds(g));
  g->setup_launches = nl + 2 + 10 * ((g->n_slot ? 3 : 1) + 1);   // with the Lanczos steps
  if (trace) {
    cudaStreamSynchronize(g->st);
    std::fprintf(stderr, "[xls] hamiltonian_set: potential + norms %.1f ms, slots + tables %.1f ms, Lanczos %.1f ms\n",
                 tms(h0, h1), tms(h1, h2), tms(h2, tnow()));
  }
  g->ham_set = true;
  g->have_ritz = false;
  return XLS_OK;
}

xls_status xls_orbitals_set(xls_grid g, int sub, const double* psi, int on_device) {
  if (!g || !psi || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_orbitals_set: bad arguments");
  if (g->wave) return wave_orbitals_set(g, sub, psi, on_device);
  const SubDev& S = g->subs[sub];
  const long long n = S.nd * S.ns;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (g->prec == XLS_FP64) {
    XLS_CUDA(cudaMemcpyAsync((double*)g->blk[g->cur] + S.off_blk, psi, n * sizeof(double), kind, g->st));
  } else {
    // stage through the free block (as doubles) and round to FP32
    double* tmp = (double*)g->blk[(g->cur + 1) % 3];
    const long long cap = g->tot_blk / 2;  // doubles that fit in a float block
    for (long long o = 0; o < n; o += cap) {
      const long long c = std::min(cap, n - o);
      XLS_CUDA(cudaMemcpyAsync(tmp, psi + o, c * sizeof(double), kind, g->st));
      launch_convert_f64_f32(tmp, (float*)g->blk[g->cur] + S.off_blk + o, c, g->st);
    }
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  g->orb_set = true;
  g->have_ritz = false;
  return XLS_OK;
}

xls_status xls_orbitals_random(xls_grid g, uint64_t seed) {
  if (!g) return fail(XLS_EINVAL, "null grid");
  if (g->wave) return wave_orbitals_random(g, seed);
  if (g->prec == XLS_FP64) launch_splitmix_fill_f64((double*)g->blk[g->cur], g->tot_blk, seed, 0, g->st);
  else launch_splitmix_fill_f32((float*)g->blk[g->cur], g->tot_blk, seed, 0, g->st);
  XLS_CUDA(cudaGetLastError());
  g->orb_set = true;
  g->have_ritz = false;
  return XLS_OK;
}

xls_status xls_orbitals_get(xls_grid g, int sub, double* psi_out, int on_device) {
  if (!g || !psi_out || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_orbitals_get: bad arguments");
  if (g->wave) return wave_orbitals_get(g, sub, psi_out, on_device);
  const SubDev& S = g->subs[sub];
  const long long n = S.nd * S.ns;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (g->prec == XLS_FP64) {
    XLS_CUDA(cudaMemcpyAsync(psi_out, (double*)g->blk[g->cur] + S.off_blk, n * sizeof(double), kind, g->st));
  } else {
    double* tmp = (double*)g->blk[(g->cur + 1) % 3];
    const long long cap = g->tot_blk / 2;
    for (long long o = 0; o < n; o += cap) {
      const long long c = std::min(cap, n - o);
      launch_convert_f32_f64((float*)g->blk[g->cur] + S.off_blk + o, tmp, c, g->st);
      XLS_CUDA(cudaMemcpyAsync(psi_out + o, tmp, c * sizeof(double), kind, g->st));
    }
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  return XLS_OK;
}

xls_status xls_orbitals_set_f32(xls_grid g, int sub, const float* psi, int on_device) {
  if (!g || !psi || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_orbitals_set_f32: bad arguments");
  if (g->wave) return fail(XLS_EINVAL, "xls_orbitals_set_f32: not in wave mode (xls_orbitals_set takes doubles)");
  const SubDev& S = g->subs[sub];
  const long long n = S.nd * S.ns;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (g->prec != XLS_FP64) {
    XLS_CUDA(cudaMemcpyAsync((float*)g->blk[g->cur] + S.off_blk, psi, n * sizeof(float), kind, g->st));
  } else {
    // stage through the free block (n floats fit in a block of doubles) and widen to FP64
    float* tmp = (float*)g->blk[(g->cur + 1) % 3];
    XLS_CUDA(cudaMemcpyAsync(tmp, psi, n * sizeof(float), kind, g->st));
    launch_convert_f32_f64(tmp, (double*)g->blk[g->cur] + S.off_blk, n, g->st);
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  g->orb_set = true;
  g->have_ritz = false;
  return XLS_OK;
}

xls_status xls_orbitals_get_f32(xls_grid g, int sub, float* psi_out, int on_device) {
  if (!g || !psi_out || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_orbitals_get_f32: bad arguments");
  if (g->wave) return fail(XLS_EINVAL, "xls_orbitals_get_f32: not in wave mode (xls_orbitals_get gives doubles)");
  const SubDev& S = g->subs[sub];
  const long long n = S.nd * S.ns;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (g->prec != XLS_FP64) {
    XLS_CUDA(cudaMemcpyAsync(psi_out, (float*)g->blk[g->cur] + S.off_blk, n * sizeof(float), kind, g->st));
  } else {
    float* tmp = (float*)g->blk[(g->cur + 1) % 3];
    launch_convert_f64_f32((double*)g->blk[g->cur] + S.off_blk, tmp, n, g->st);
    XLS_CUDA(cudaMemcpyAsync(psi_out, tmp, n * sizeof(float), kind, g->st));
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  return XLS_OK;
}

xls_status xls_chefsi_batch(xls_grid g, int degree, int n_passes, const double* bounds) {
  if (!g || degree < 1 || degree >= kMaxDegree - 1 || n_passes < 0) return fail(XLS_EINVAL, "xls_chefsi_batch: bad arguments");
  if (!g->ham_set || !g->orb_set) return fail(XLS_EINVAL, "xls_chefsi_batch: Hamiltonian or orbitals not set");
  if (g->wave) return wave_chefsi(g, degree, n_passes, bounds);
  return g->prec == XLS_FP64 ? chefsi<double>(g, degree, n_passes, bounds) : chefsi<float>(g, degree, n_passes, bounds);
}

xls_status xls_autotune(xls_grid g, int reps, int* choices_out) {
  if (!g || reps < 1 || reps > 100) return fail(XLS_EINVAL, "xls_autotune: bad arguments");
  if (g->wave && g->carry && g->worker) return xls_autotune(g->worker, reps, choices_out);   // the worker's last wave
  if (g->wave) return fail(XLS_EINVAL, "xls_autotune: not in wave mode");
  if (!g->have_ritz) return fail(XLS_EINVAL, "xls_autotune: run a pass first (its subspace matrices are the input)");
  XLS_TRY(check_status(g));
  cudaStream_t st = g->st;
  // the last projection's M_s, H_s and split exponents are saved and put back afterwards
  const size_t ss = (size_t)g->tot_ss * sizeof(double);
  const bool tc_gram = g->prec != XLS_FP64 && g->use_tc && g->use_tc_gram;
  const size_t ex = tc_gram ? (size_t)g->tot_states * sizeof(int) : 0;
  unsigned char* save = nullptr;
  if (cudaMalloc((void**)&save, 2 * ss + 2 * ex) != cudaSuccess) {
    cudaGetLastError();
    return fail(XLS_ENOMEM, "xls_autotune: no room to save the subspace matrices");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  xls_status rc = XLS_OK;
  auto cuda_ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == XLS_OK) rc = fail(XLS_ECUDA, std::string("xls_autotune: ") + cudaGetErrorString(e));
    return rc == XLS_OK;
  };
  cuda_ok(cudaMemcpyAsync(save, g->Ms, ss, cudaMemcpyDeviceToDevice, st));
  cuda_ok(cudaMemcpyAsync(save + ss, g->Hs, ss, cudaMemcpyDeviceToDevice, st));
  if (tc_gram) {
    cuda_ok(cudaMemcpyAsync(save + 2 * ss, g->gplan.d_ex_f, ex, cudaMemcpyDeviceToDevice, st));
    cuda_ok(cudaMemcpyAsync(save + 2 * ss + ex, g->gplan.d_ex_hf, ex, cudaMemcpyDeviceToDevice, st));
  }
  cuda_ok(cudaEventCreate(&e0));
  cuda_ok(cudaEventCreate(&e1));
  // mean time of `reps` calls after one warm-up call, CUDA events on the grid's stream
  auto time_it = [&](const std::function<void()>& fn) -> float {
    fn();
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) fn();
    cudaEventRecord(e1, st);
    float ms = -1.f;
    if (!cuda_ok(cudaEventSynchronize(e1)) || !cuda_ok(cudaEventElapsedTime(&ms, e0, e1))) return -1.f;
    const xls_status k = check_status(g);
    if (k != XLS_OK && rc == XLS_OK) rc = k;
    return rc == XLS_OK ? ms / reps : -1.f;
  };
  auto replan_all = [&]() {
    if (rc == XLS_OK) rc = replan_gram(g, 0, g->n_sub, g->gplan, st);
    g->full.gplan = g->gplan;
    if (g->concurrent)
      for (auto& h : g->halves)
        if (rc == XLS_OK) rc = replan_gram(g, h.first, h.n, h.gplan, st);
  };
  // (1) cluster size of the Cholesky and the tridiagonalisation
  if (rc == XLS_OK && g->eig_cluster) {
    int best = g->eig_cl;
    float bt = -1.f;
    for (int cl : {8, 16}) {
      g->eig_cl = cl;
      const float t = time_it([&] { eigensolve(g, fv(g)); });
      if (rc != XLS_OK) break;
      if (bt < 0.f || t < bt) {
        bt = t;
        best = cl;
      }
    }
    g->eig_cl = best;
  }
  // (2) K split of the tensor-core Gram
  if (rc == XLS_OK && tc_gram) {
    const int f = g->cur, hf = (g->cur + 1) % 3;
    int best = g->gram_cps;
    float bt = -1.f;
    for (int cps : {1, 2, 3, 4, 6, 8}) {
      g->gram_cps = cps;
      replan_all();
      if (rc != XLS_OK) break;
      xls_grid_s::View& v = fv(g);
      const float t = time_it([&] {
        launch_gram_tc(v.ds, v.n, v.max_ns, v.gplan, g->prec == XLS_MIXED_FP16, (const float*)g->blk[f],
                       (const float*)g->blk[hf], g->Ms, g->Hs, g->status, st);
      });
      if (rc != XLS_OK) break;
      if (bt < 0.f || t < bt) {
        bt = t;
        best = cps;
      }
    }
    g->gram_cps = best;
    replan_all();
  }
  // (3) vectors per CTA, warps per CTA and slots per chunk of the nonlocal projection, timed on
  // the current block (the projection coefficients it overwrites are recomputed at the start of
  // every filter step)
  if (rc == XLS_OK && g->n_slot > 0) {
    int best_v = g->proj_vec, best_w = g->proj_warps, best_c = g->proj_chunk;
    float bt = -1.f;
    const int shapes[5][2] = {{8, 8}, {16, 8}, {32, 8}, {8, 4}, {16, 4}};   // (vectors, warps)
    for (const auto& sh : shapes)
      for (int chunk : {256, 512, 1024}) {
        const int kpv = sh[0], nw = sh[1];
        const float t = time_it([&] {
          if (g->prec == XLS_FP64)
            launch_nl_project<double>(g->d_subs, g->d_slots, 0, g->n_slot, g->d_pidx, g->d_chi64, g->max_ns,
                                      (const double*)g->blk[g->cur], g->P, kpv, nw, chunk, st);
          else
            launch_nl_project<float>(g->d_subs, g->d_slots, 0, g->n_slot, g->d_pidx, g->d_chi32, g->max_ns,
                                     (const float*)g->blk[g->cur], g->P, kpv, nw, chunk, st);
        });
        if (rc != XLS_OK) break;
        if (std::getenv("XLS_TRACE"))
          std::fprintf(stderr, "[xls] autotune: projection %d vectors per CTA of %d warps, chunks of %d slots %.3f ms\n",
                       kpv, nw, chunk, t);
        if (bt < 0.f || t < bt) {
          bt = t;
          best_v = kpv;
          best_w = nw;
          best_c = chunk;
        }
      }
    g->proj_vec = best_v;
    g->proj_warps = best_w;
    g->proj_chunk = best_c;
  }
  // (3b) back-projection variant (points per thread x vectors per CTA), adding into a free arena
  // (scratch between passes) with the coefficients the projection timing left in P
  if (rc == XLS_OK && g->n_slot > 0 && g->nlb_max > 0) {
    int best = g->back_var;
    float bt = -1.f;
    const int bout = (g->cur + 1) % 3;
    xls_grid_s::View& v = fv(g);
    for (int var : {1, 2, 16}) {
      const float t = time_it([&] {
        if (g->prec == XLS_FP64)
          launch_nl_back_csr<double>(v.ds, v.n, v.max_nd, v.max_ns, g->nlb_max, g->d_rptr, g->d_rslot, g->d_rchi64,
                                     g->d_nlb_cnt, g->d_nlb_list, g->P, (double*)g->blk[bout], v.coef, 0, var, st);
        else
          launch_nl_back_csr<float>(v.ds, v.n, v.max_nd, v.max_ns, g->nlb_max, g->d_rptr, g->d_rslot, g->d_rchi32,
                                    g->d_nlb_cnt, g->d_nlb_list, g->P, (float*)g->blk[bout], v.coef, 0, var, st);
      });
      if (rc != XLS_OK) break;
      if (std::getenv("XLS_TRACE"))
        std::fprintf(stderr, "[xls] autotune: back-projection variant %d (%s) %.3f ms\n", var,
                     var == 16 ? "1 point x 16 vectors" : (var == 2 ? "2 points x 8 vectors" : "1 point x 8 vectors"), t);
      if (bt < 0.f || t < bt) {
        bt = t;
        best = var;
      }
    }
    g->back_var = best;
  }
  // (4) slot pitch of the TMA stencil per class: compile-time (where one exists: 80, 112 floats)
  // or runtime, timed on the current block into a free arena (its contents are scratch between
  // passes); the choice goes to every view's class of the same pitch
  if (rc == XLS_OK && g->prec != XLS_FP64 && g->use_tma) {
    const int bin = g->cur, bprev = (g->cur + 2) % 3, bout = (g->cur + 1) % 3;
    xls_grid_s::View& v = fv(g);
    for (size_t i = 0; i < v.tcls.size(); ++i) {
      if (v.tcls[i].W != 80 && v.tcls[i].W != 112) continue;
      int best = v.tcls[i].rt_pitch;
      float bt = -1.f;
      for (int rt : {0, 1}) {
        v.tcls[i].rt_pitch = rt;
        const float t = time_it([&] {
          launch_stencil_tma(v.ds, v.tcls[i], v.maps, bin, bprev, (float*)g->blk[bout], v.coef, 0, g->status, st);
        });
        if (rc != XLS_OK) break;
        if (std::getenv("XLS_TRACE"))
          std::fprintf(stderr, "[xls] autotune: stencil pitch %d (%s) %.3f ms\n", v.tcls[i].W, rt ? "runtime" : "compile-time", t);
        if (bt < 0.f || t < bt) {
          bt = t;
          best = rt;
        }
      }
      v.tcls[i].rt_pitch = best;
      auto apply = [&](std::vector<TmaClass>& cl) {
        for (TmaClass& c : cl)
          if (c.W == v.tcls[i].W) c.rt_pitch = best;
      };
      apply(g->tcls);
      if (g->concurrent)
        for (auto& h : g->halves) apply(h.tcls);
    }
  }
  // the saved matrices and exponents back; eigenpairs of the last pass recomputed with the
  // chosen configuration; passes captured with the old launch shapes dropped
  cuda_ok(cudaMemcpyAsync(g->Ms, save, ss, cudaMemcpyDeviceToDevice, st));
  cuda_ok(cudaMemcpyAsync(g->Hs, save + ss, ss, cudaMemcpyDeviceToDevice, st));
  if (tc_gram) {
    cuda_ok(cudaMemcpyAsync(g->gplan.d_ex_f, save + 2 * ss, ex, cudaMemcpyDeviceToDevice, st));
    cuda_ok(cudaMemcpyAsync(g->gplan.d_ex_hf, save + 2 * ss + ex, ex, cudaMemcpyDeviceToDevice, st));
  }
  if (rc == XLS_OK) {
    eigensolve(g, fv(g));
    rc = check_status(g);
  }
  cudaStreamSynchronize(st);
  g->drop_graphs();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(save);
  if (choices_out) {
    choices_out[0] = g->eig_cluster ? g->eig_cl : 0;
    choices_out[1] = tc_gram ? g->gram_cps : 0;
    choices_out[2] = g->n_slot > 0 ? g->proj_vec : 0;
  }
  return rc;
}

xls_status xls_chefsi_stage(xls_grid g, int which, int degree, const double* bounds) {
  if (!g || degree < 1 || degree >= kMaxDegree - 1) return fail(XLS_EINVAL, "xls_chefsi_stage: bad arguments");
  if (g->wave) return not_in_wave_mode("xls_chefsi_stage");
  if (!g->ham_set || !g->orb_set) return fail(XLS_EINVAL, "xls_chefsi_stage: Hamiltonian or orbitals not set");
  return g->prec == XLS_FP64 ? stage<double>(g, which, degree, bounds) : stage<float>(g, which, degree, bounds);
}

xls_status xls_hamiltonian_apply(xls_grid g, int sub, int k, const double* x, double* y, int on_device) {
  if (!g || !x || !y || sub < 0 || sub >= g->n_sub || k < 1 || k > g->subs[sub].ns)
    return fail(XLS_EINVAL, "xls_hamiltonian_apply: bad arguments");
  if (g->wave) return not_in_wave_mode("xls_hamiltonian_apply");
  if (!g->ham_set) return fail(XLS_EINVAL, "xls_hamiltonian_apply: Hamiltonian not set");
  const SubDev& S = g->subs[sub];
  const long long n = S.nd * k;
  const int in = (g->cur + 1) % 3, outb = (g->cur + 2) % 3;
  XLS_CUDA(cudaMemsetAsync(g->blk[in], 0, g->tot_blk * g->elem, g->st));
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (g->prec == XLS_FP64) {
    XLS_CUDA(cudaMemcpyAsync((double*)g->blk[in] + S.off_blk, x, n * sizeof(double), kin, g->st));
    h_step<double>(g, false, (double*)g->blk[in], nullptr, (double*)g->blk[outb], kUnitStep);
    XLS_CUDA(cudaMemcpyAsync(y, (double*)g->blk[outb] + S.off_blk, n * sizeof(double), kout, g->st));
  } else {
    double* tmp = (double*)g->blk[g->cur];  // orbitals are clobbered on the mixed path's staging
    (void)tmp;
    double* dtmp = nullptr;
    XLS_CUDA(cudaMalloc(&dtmp, n * sizeof(double)));
    XLS_CUDA(cudaMemcpyAsync(dtmp, x, n * sizeof(double), kin, g->st));
    launch_convert_f64_f32(dtmp, (float*)g->blk[in] + S.off_blk, n, g->st);
    h_step_main<float>(g, fv(g), in, -1, outb, kUnitStep);
    launch_convert_f32_f64((float*)g->blk[outb] + S.off_blk, dtmp, n, g->st);
    XLS_CUDA(cudaMemcpyAsync(y, dtmp, n * sizeof(double), kout, g->st));
    XLS_CUDA(cudaStreamSynchronize(g->st));
    cudaFree(dtmp);
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  return XLS_OK;
}

xls_status xls_density(xls_grid g, double n_electrons, double kT, double* mu_out, double* rho_out, int rho_on_device,
                       double* e_band_out, double* e_entropy_out) {
  if (!g || !(kT > 0) || !g->have_ritz) return fail(XLS_EINVAL, "xls_density: bad arguments or no pass run yet");
  if (g->wave) return wave_density(g, n_electrons, kT, mu_out, rho_out, rho_on_device, e_band_out, e_entropy_out);
  launch_fermi_occ(g->lam, g->cw, g->tot_states, n_electrons, kT, g->out4, g->occ, g->status, g->st);
  XLS_TRY(check_status(g));
  double h4[4];
  XLS_CUDA(cudaMemcpy(h4, g->out4, sizeof(h4), cudaMemcpyDeviceToHost));
  if (mu_out) *mu_out = h4[0];
  if (e_band_out) *e_band_out = h4[1];
  if (e_entropy_out) *e_entropy_out = h4[2];
  if (rho_out) {
    const long long ng = (long long)g->gn[0] * g->gn[1] * g->gn[2];
    if (!g->rho) XLS_TRY(g->alloc(&g->rho, ng * sizeof(double)));
    if (g->prec == XLS_FP64)
      launch_density_occ<double>(g->d_subs, g->n_sub, g->max_core, (const double*)g->blk[g->cur], g->occ, g->gn, g->rho, g->st);
    else
      launch_density_occ<float>(g->d_subs, g->n_sub, g->max_core, (const float*)g->blk[g->cur], g->occ, g->gn, g->rho, g->st);
    XLS_CUDA(cudaMemcpyAsync(rho_out, g->rho, ng * sizeof(double),
                             rho_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->st));
    XLS_CUDA(cudaStreamSynchronize(g->st));
  }
  return XLS_OK;
}

xls_status xls_get_eigs(xls_grid g, int sub, double* lambda_out, double* c_out) {
  if (!g || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_get_eigs: bad arguments");
  const SubDev& S = g->subs[sub];
  XLS_CUDA(cudaStreamSynchronize(g->st));
  if (lambda_out) XLS_CUDA(cudaMemcpy(lambda_out, g->lam + S.off_state, S.ns * sizeof(double), cudaMemcpyDeviceToHost));
  if (c_out) XLS_CUDA(cudaMemcpy(c_out, g->cw + S.off_state, S.ns * sizeof(double), cudaMemcpyDeviceToHost));
  return XLS_OK;
}

xls_status xls_wave_store_fp16(xls_grid g, int on) {
  if (!g) return fail(XLS_EINVAL, "xls_wave_store_fp16: bad arguments");
  if (!g->wave) return fail(XLS_EINVAL, "xls_wave_store_fp16: the grid is not running in waves");
  if ((on != 0) == g->store16) return XLS_OK;
  long long max_blk = 0;
  for (const SubDev& S : g->subs) max_blk = std::max(max_blk, S.nd * S.ns);
  if (!g->stage16) {
    if (cudaMalloc(&g->stage16, (size_t)max_blk * 2) != cudaSuccess ||
        cudaMalloc((void**)&g->d_store_ex, (size_t)g->tot_states * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(XLS_ENOMEM, "xls_wave_store_fp16: device staging could not be allocated");
    }
    XLS_CUDA(cudaMemsetAsync(g->d_store_ex, 0, (size_t)g->tot_states * sizeof(int), g->st));
  }
  // new store; the orbitals held so far move over through the device
  const bool to16 = on != 0;
  const size_t new_elem = to16 ? 2 : g->elem;
  void* ns_ = nullptr;
  if (cudaMallocHost(&ns_, (size_t)g->tot_blk * new_elem) != cudaSuccess) {
    cudaGetLastError();
    return fail(XLS_ENOMEM, "xls_wave_store_fp16: pinned host store could not be allocated");
  }
  std::memset(ns_, 0, (size_t)g->tot_blk * new_elem);
  void* old = g->store;
  const bool was16 = g->store16;
  for (int a = 0; a < g->n_sub && g->orb_set; ++a) {
    g->store = old;
    g->store16 = was16;
    XLS_TRY(store_to_device(g, a, g->blk[0], g->st));
    g->store = ns_;
    g->store16 = to16;
    XLS_TRY(device_to_store(g, a, g->blk[0], g->st));
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  g->store = ns_;
  g->store16 = to16;
  cudaFreeHost(old);
  // the stored orbitals are now rounded to the new format; the device core rows are not
  std::fill(g->core_fresh.begin(), g->core_fresh.end(), (char)0);
  return XLS_OK;
}

xls_status xls_wave_carry(xls_grid g, int slots) {
  if (!g) return fail(XLS_EINVAL, "xls_wave_carry: bad arguments");
  if (!g->wave) return fail(XLS_EINVAL, "xls_wave_carry: the grid is not running in waves");
  if (slots > 0 && (slots > g->n_sub || g->n_sub % slots != 0))
    return fail(XLS_EINVAL, "xls_wave_carry: the slot count must divide the subdomain count");
  if (g->carry && slots != 0) {   // already in carry mode: only a change of the slot count matters
    if (slots < 0 || slots == g->worker->n_sub) return XLS_OK;
    XLS_TRY(xls_wave_carry(g, 0));
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  if (slots == 0) {
    if (!g->carry) return XLS_OK;
    if (g->worker) xls_grid_destroy(g->worker);
    g->worker = nullptr;
    g->release(&g->core_store);
    g->release(&g->d_core_subs);
    std::fill(g->core_fresh.begin(), g->core_fresh.end(), (char)0);
    g->carry = false;
    g->orb_set = false;
    g->have_ritz = false;
    return XLS_OK;
  }
  if (!uniform_shapes(g))
    return fail(XLS_EINVAL, "xls_wave_carry: every subdomain must have the shape of subdomain 0 (points, boundaries, "
                            "core box, states)");
  const SubDev& A = g->subs[0];
  const size_t core_pts = (size_t)A.core_n[0] * A.core_n[1] * A.core_n[2];
  const size_t store_bytes = core_pts * A.ns * g->elem * (size_t)g->n_sub;
  // a core store of store-mode waves (if one was made) is replaced by carry mode's own
  g->release(&g->core_store);
  g->release(&g->d_core_subs);
  std::fill(g->core_fresh.begin(), g->core_fresh.end(), (char)0);
  const size_t f = sub_footprint(A, g->elem);
  const size_t fixed = ((size_t)1 << 26) + g->bytes + store_bytes;
  int W = 0;
  for (int w = slots > 0 ? slots : g->n_sub; w >= 1; --w)
    if (g->n_sub % w == 0 && (!g->budget || fixed + (size_t)w * f <= g->budget)) {
      W = w;
      break;
    }
  if (W == 0) return fail(XLS_ENOMEM, "xls_wave_carry: the core store and one subdomain exceed the HBM budget");
  if (slots > 0 && W != slots)
    return fail(XLS_ENOMEM, "xls_wave_carry: " + std::to_string(slots) + " slots and the core store exceed the HBM budget");
  // the host store (if one was made) is no longer used
  if (g->store) cudaFreeHost(g->store);
  g->store = nullptr;
  g->store16 = false;
  XLS_TRY(alloc_core_store(g));   // store_bytes of core rows and their density descriptors
  g->waves.clear();
  for (int first = 0; first < g->n_sub; first += W) g->waves.push_back({first, W});
  xls_dc dc{W, g->dc_core_lo.data(), g->dc_core_n.data(), g->dc_buf.data(), g->dc_ns.data()};
  xls_grid k = nullptr;
  const xls_status s = create_grid(&g->cell, &dc, g->prec, 0, g->st, &k, true, false);
  if (s != XLS_OK) {
    g->release(&g->core_store);
    g->release(&g->d_core_subs);
    return s;
  }
  g->worker = k;
  g->carry = true;
  g->carry_primed = false;
  g->wave_ran.assign(g->waves.size(), 0);
  g->orb_set = false;
  g->have_ritz = false;
  return XLS_OK;
}

xls_status xls_chefsi_wave(xls_grid g, int wave, int degree, int n_passes, const double* bounds) {
  if (!g || degree < 1 || degree >= kMaxDegree - 1 || n_passes < 0) return fail(XLS_EINVAL, "xls_chefsi_wave: bad arguments");
  if (!g->wave) return fail(XLS_EINVAL, "xls_chefsi_wave: the grid is not running in waves");
  if (wave < 0 || wave >= (int)g->waves.size()) return fail(XLS_EINVAL, "xls_chefsi_wave: wave index out of range");
  if (!g->ham_set || !g->orb_set) return fail(XLS_EINVAL, "xls_chefsi_wave: Hamiltonian or orbitals not set");
  for (double& t : g->wave_stage_ms) t = 0.0;
  int launches = 0;
  if (g->carry) XLS_TRY(carry_run(g, wave, degree, n_passes, bounds, launches));
  else XLS_TRY(wave_run(g, wave, degree, n_passes, bounds, false, launches));
  g->last_launches = launches;
  return XLS_OK;
}

xls_status xls_scf_cg_iterations(xls_grid g, long long* iterations_out) {
  if (!g || !iterations_out) return fail(XLS_EINVAL, "xls_scf_cg_iterations: bad arguments");
  *iterations_out = g->scf.cg_iters;
  return XLS_OK;
}

xls_status xls_dos(xls_grid g, const double* energies, int n_energies, double width, double* dos_out) {
  if (!g || n_energies < 0 || (n_energies > 0 && (!energies || !dos_out)) || !(width > 0))
    return fail(XLS_EINVAL, "xls_dos: bad arguments");
  if (n_energies == 0) return XLS_OK;
  double* d = nullptr;
  if (cudaMalloc(&d, 2 * (size_t)n_energies * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(XLS_ENOMEM, "xls_dos: device allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(d, energies, (size_t)n_energies * sizeof(double), cudaMemcpyHostToDevice, g->st);
  if (e == cudaSuccess) {
    launch_dos(g->lam, g->cw, (int)g->tot_states, d, n_energies, width, d + n_energies, g->st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dos_out, d + n_energies, (size_t)n_energies * sizeof(double), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  cudaFree(d);
  if (e != cudaSuccess) return fail(XLS_ECUDA, std::string("xls_dos: ") + cudaGetErrorString(e));
  return XLS_OK;
}

xls_status xls_get_subspace(xls_grid g, int sub, double* Ms_out, double* Hs_out) {
  if (!g || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_get_subspace: bad arguments");
  if (g->wave && carry_slot(g, sub) >= 0) return xls_get_subspace(g->worker, carry_slot(g, sub), Ms_out, Hs_out);
  if (g->wave) return not_in_wave_mode("xls_get_subspace");
  const SubDev& S = g->subs[sub];
  XLS_CUDA(cudaStreamSynchronize(g->st));
  const size_t b = (size_t)S.ns * S.ns * sizeof(double);
  if (Ms_out) XLS_CUDA(cudaMemcpy(Ms_out, g->Ms + S.off_ss, b, cudaMemcpyDeviceToHost));
  if (Hs_out) XLS_CUDA(cudaMemcpy(Hs_out, g->Hs + S.off_ss, b, cudaMemcpyDeviceToHost));
  return XLS_OK;
}

xls_status xls_get_rotation(xls_grid g, int sub, double* Y_out) {
  if (!g || !Y_out || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_get_rotation: bad arguments");
  if (g->wave && carry_slot(g, sub) >= 0) return xls_get_rotation(g->worker, carry_slot(g, sub), Y_out);
  if (g->wave) return not_in_wave_mode("xls_get_rotation");
  const SubDev& S = g->subs[sub];
  XLS_CUDA(cudaStreamSynchronize(g->st));
  XLS_CUDA(cudaMemcpy(Y_out, g->Y + S.off_ss, (size_t)S.ns * S.ns * sizeof(double), cudaMemcpyDeviceToHost));
  return XLS_OK;
}

xls_status xls_get_eig_work(xls_grid g, int sub, double* L_out, double* A_out, double* vecs_out) {
  if (!g || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_get_eig_work: bad arguments");
  if (g->wave && carry_slot(g, sub) >= 0) return xls_get_eig_work(g->worker, carry_slot(g, sub), L_out, A_out, vecs_out);
  if (g->wave) return not_in_wave_mode("xls_get_eig_work");
  const SubDev& S = g->subs[sub];
  XLS_CUDA(cudaStreamSynchronize(g->st));
  const size_t b = (size_t)S.ns * S.ns * sizeof(double);
  if (L_out) XLS_CUDA(cudaMemcpy(L_out, g->Lb + S.off_ss, b, cudaMemcpyDeviceToHost));
  if (A_out) XLS_CUDA(cudaMemcpy(A_out, g->Ab + S.off_ss, b, cudaMemcpyDeviceToHost));
  if (vecs_out) XLS_CUDA(cudaMemcpy(vecs_out, g->vecs + 8LL * S.off_state, 8 * (size_t)S.ns * sizeof(double),
                                    cudaMemcpyDeviceToHost));
  return XLS_OK;
}

xls_status xls_get_bounds(xls_grid g, double* bounds_out) {
  if (!g || !bounds_out) return fail(XLS_EINVAL, "xls_get_bounds: bad arguments");
  if (g->wave) {
    std::memcpy(bounds_out, g->host_bounds.data(), 3 * (size_t)g->n_sub * sizeof(double));
    return XLS_OK;
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  XLS_CUDA(cudaMemcpy(bounds_out, g->bounds, 3 * g->n_sub * sizeof(double), cudaMemcpyDeviceToHost));
  return XLS_OK;
}

xls_status xls_set_profiling(xls_grid g, int on) {
  if (!g) return fail(XLS_EINVAL, "null grid");
  if (g->wave && g->carry && g->worker) return xls_set_profiling(g->worker, on);   // the worker's passes
  if (g->wave && on) return not_in_wave_mode("xls_set_profiling");
  g->profiling = on != 0;
  if (g->profiling && g->pev.empty()) {
    g->pev.resize(4096);
    g->pcls.resize(2048);
    for (auto& e : g->pev) XLS_CUDA(cudaEventCreate(&e));
  }
  return XLS_OK;
}

xls_status xls_scf_setup(xls_grid g, double n_electrons, double kT, int degree, int n_passes, double beta,
                         double kappa, int history, int pulay_period) {
  if (!g || !(n_electrons > 0) || !(kT > 0) || degree < 1 || degree >= kMaxDegree || n_passes < 1 || !(beta > 0) ||
      !(kappa > 0) || history < 1 || history > 8 || pulay_period < 1)
    return fail(XLS_EINVAL, "xls_scf_setup: bad arguments");
  if (!g->ham_set) return fail(XLS_EINVAL, "xls_scf_setup: call xls_hamiltonian_set first (atoms and projectors)");
  auto& S = g->scf;
  const bool need_alloc = !S.d_gs || history > S.hist;
  S.ne = n_electrons;
  S.kT = kT;
  S.degree = degree;
  S.passes = n_passes;
  S.beta = beta;
  S.kappa = kappa;
  S.period = pulay_period;
  S.k = 0;
  if (need_alloc) {
    if (S.d_gs && history > S.hist) return fail(XLS_EINVAL, "xls_scf_setup: history cannot grow after the first setup");
    S.hist = history;
    XLS_TRY(scf_alloc(g));
  }
  S.hist = history;
  XLS_TRY(scf_coefficients(g));
  S.ready = true;
  return XLS_OK;
}

xls_status xls_scf_step(xls_grid g, double* rho_inout, int rho_on_device, double* residual_out, double* energy_out,
                        double* mu_out) {
  if (!g || !rho_inout) return fail(XLS_EINVAL, "xls_scf_step: bad arguments");
  auto& S = g->scf;
  if (!S.ready) return fail(XLS_EINVAL, "xls_scf_step: call xls_scf_setup first");
  if (!g->orb_set) return fail(XLS_EINVAL, "xls_scf_step: orbitals not set");
  const long long n = S.gs.nd;
  const double dV = S.gs.dV;
  cudaStream_t st = g->st;
  if (!S.pc_ready) XLS_TRY(scf_pseudocharge(g));
  XLS_CUDA(cudaMemcpyAsync(S.rho_in, rho_inout, n * sizeof(double),
                           rho_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  // 1. electrostatics: -Delta_h phi = 4 pi (rho + b), zero mean (warm start from the last phi)
  launch_axpbypcz(n, 4.0 * M_PI, S.rho_in, 0.0, S.f, 4.0 * M_PI, S.b, st);
  launch_sum(n, S.f, S.partial, S.scal + 8, st);
  launch_sub_mean(n, S.scal + 8, S.f, st);
  double ref_sq = 0.0;   // ||4 pi rho||^2: the scale of the cancelling terms
  {
    const double* xs[1] = {S.rho_in};
    launch_dots(n, xs, xs, 1, S.partial, S.scal + 8, 16.0 * M_PI * M_PI, st);
    XLS_CUDA(cudaMemcpyAsync(&ref_sq, S.scal + 8, sizeof(double), cudaMemcpyDeviceToHost, st));
    XLS_CUDA(cudaStreamSynchronize(st));
  }
  XLS_TRY(scf_cg(g, 0, S.f, S.phi, 1e-13, 6000, ref_sq));
  launch_sum(n, S.phi, S.partial, S.scal + 8, st);
  launch_sub_mean(n, S.scal + 8, S.phi, st);
  // 2. exchange-correlation and V_eff = phi + v_xc, restricted to the subdomains
  launch_lda(n, S.rho_in, S.eps, S.vxc, st);
  if (!g->Vg) XLS_TRY(g->alloc(&g->Vg, n * sizeof(double)));
  launch_axpbypcz(n, 1.0, S.phi, 0.0, g->Vg, 1.0, S.vxc, st);
  if (g->wave) {
    // 3'. in waves: every wave's worker grid restricts V_eff from the global grid, takes its new
    // Lanczos bounds and runs the passes with its orbitals staged from the host store
    XLS_CUDA(cudaStreamSynchronize(st));
    XLS_TRY(wave_chefsi(g, S.degree, S.passes, nullptr, true));
  } else {
    launch_restrict(g->d_subs, g->n_sub, g->max_nd, g->Vg, g->gn, g->V, g->Vf, st);
    // 3. new upper bounds (Lanczos) and the CheFSI passes
    XLS_TRY(lanczos_bounds(g));
    if (g->prec == XLS_FP64) XLS_TRY(chefsi<double>(g, S.degree, S.passes, nullptr));
    else XLS_TRY(chefsi<float>(g, S.degree, S.passes, nullptr));
  }
  // 4. Fermi level, output density, band and entropy energies
  double mu = 0, e_band = 0, e_ent = 0;
  XLS_TRY(xls_density(g, S.ne, S.kT, &mu, S.rho_out, 1, &e_band, &e_ent));
  // 5. energy at the input density and the residual
  double sums[4], rr[2];
  {
    const double* xs[4] = {S.rho_in, S.vxc, S.b, S.rho_in};
    const double* ys[4] = {S.eps, S.rho_in, S.phi, S.phi};
    launch_dots(n, xs, ys, 4, S.partial, S.scal + 8, 1.0, st);
    XLS_CUDA(cudaMemcpyAsync(sums, S.scal + 8, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  launch_axpbypcz(n, 1.0, S.rho_out, 0.0, S.f, -1.0, S.rho_in, st);   // f = rho_out - rho_in
  {
    const double* xs[2] = {S.f, S.rho_out};
    const double* ys[2] = {S.f, S.rho_out};
    launch_dots(n, xs, ys, 2, S.partial, S.scal + 12, 1.0, st);
    XLS_CUDA(cudaMemcpyAsync(rr, S.scal + 12, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  XLS_CUDA(cudaStreamSynchronize(st));
  const double energy = e_band + dV * (sums[0] - sums[1] + 0.5 * (sums[2] - sums[3])) - S.e_self - e_ent;
  const double residual = std::sqrt(rr[0] / rr[1]);
  // 6. periodic Pulay mixing with the Kerker preconditioner: x_next = x + beta P f
  //    [- sum_i gamma_i (dX_i + beta dPF_i) on every period-th step]
  XLS_TRY(scf_kerker(g, S.f, S.pf));
  if (S.k > 0) {
    const int slot = (S.k - 1) % S.hist;
    launch_axpbypcz(n, 1.0, S.rho_in, 0.0, S.dX + (size_t)slot * n, -1.0, S.x_prev, st);
    launch_axpbypcz(n, 1.0, S.f, 0.0, S.dF + (size_t)slot * n, -1.0, S.f_prev, st);
    launch_axpbypcz(n, 1.0, S.pf, 0.0, S.dPF + (size_t)slot * n, -1.0, S.pf_prev, st);
  }
  XLS_CUDA(cudaMemcpyAsync(S.x_prev, S.rho_in, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  XLS_CUDA(cudaMemcpyAsync(S.f_prev, S.f, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  XLS_CUDA(cudaMemcpyAsync(S.pf_prev, S.pf, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_axpbypcz(n, 1.0, S.rho_in, 0.0, S.tmp, S.beta, S.pf, st);     // tmp = x + beta P f
  const int nh = std::min(S.k, S.hist);
  if ((S.k + 1) % S.period == 0 && nh > 0)
    launch_pulay(n, nh, S.dF, S.dX, S.dPF, S.f, S.beta, S.pulay_partial, S.gamma, S.tmp, st);
  S.k++;
  XLS_CUDA(cudaMemcpyAsync(rho_inout, S.tmp, n * sizeof(double),
                           rho_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  XLS_CUDA(cudaStreamSynchronize(st));
  if (residual_out) *residual_out = residual;
  if (energy_out) *energy_out = energy;
  if (mu_out) *mu_out = mu;
  return XLS_OK;
}

// atom tables of the learned start for the grid's current atoms
xls_status ls_tables(xls_grid g) {
  const int na = (int)g->atom_sp.size();
  if (na == 0) return fail(XLS_EINVAL, "learned start: the Hamiltonian has no atoms");
  for (int s : g->atom_sp)
    if (s > 1) return fail(XLS_EINVAL, "learned start: the descriptors cover two species (indices 0 and 1)");
  if (g->ls_na != na) {
    if (g->ls_na >= 0) return fail(XLS_EINVAL, "learned start: the atom count changed since the first call");
    const long long ng = (long long)g->gn[0] * g->gn[1] * g->gn[2];
    XLS_TRY(g->alloc(&g->ls_atoms, na * sizeof(float4)));
    XLS_TRY(g->alloc(&g->ls_pos, 3 * (size_t)na * sizeof(double)));
    XLS_TRY(g->alloc(&g->ls_rc, na * sizeof(double)));
    XLS_TRY(g->alloc(&g->ls_amp, na * sizeof(double)));
    XLS_TRY(g->alloc(&g->ls_g1, (size_t)na * (g->gn[0] + g->gn[1] + g->gn[2]) * sizeof(double)));
    XLS_TRY(g->alloc(&g->ls_sad, ng * sizeof(double)));
    XLS_TRY(g->alloc(&g->ls_partial, kRedPartials * sizeof(double)));
    XLS_TRY(g->alloc(&g->ls_s, 4 * sizeof(double)));
    g->ls_na = na;
  }
  std::vector<float4> at(na);
  std::vector<double> rc(na), amp(na);
  for (int i = 0; i < na; ++i) {
    const xls_species& q = g->species[g->atom_sp[i]];
    double r[3];
    for (int d = 0; d < 3; ++d) {
      r[d] = std::fmod(g->atom_pos[3 * i + d], g->gL[d]);
      if (r[d] < 0) r[d] += g->gL[d];
    }
    at[i] = make_float4((float)r[0], (float)r[1], (float)r[2], (float)g->atom_sp[i]);
    rc[i] = q.rc_loc;
    amp[i] = q.Zv * std::pow(M_PI, -1.5) / (q.rc_loc * q.rc_loc * q.rc_loc);
  }
  XLS_CUDA(cudaMemcpy(g->ls_atoms, at.data(), na * sizeof(float4), cudaMemcpyHostToDevice));
  XLS_CUDA(cudaMemcpy(g->ls_pos, g->atom_pos.data(), 3 * (size_t)na * sizeof(double), cudaMemcpyHostToDevice));
  XLS_CUDA(cudaMemcpy(g->ls_rc, rc.data(), na * sizeof(double), cudaMemcpyHostToDevice));
  XLS_CUDA(cudaMemcpy(g->ls_amp, amp.data(), na * sizeof(double), cudaMemcpyHostToDevice));
  return XLS_OK;
}

xls_status xls_descriptors(xls_grid g, float* X_out, int on_device) {
  if (!g || !X_out) return fail(XLS_EINVAL, "xls_descriptors: bad arguments");
  if (!g->ham_set) return fail(XLS_EINVAL, "xls_descriptors: call xls_hamiltonian_set first (atoms)");
  XLS_TRY(ls_tables(g));
  const long long ng = (long long)g->gn[0] * g->gn[1] * g->gn[2];
  if (!g->ls_X) XLS_TRY(g->alloc(&g->ls_X, (size_t)ng * 32 * sizeof(float)));
  launch_descriptors(ng, g->gn, g->gh, g->gL, g->ls_atoms, g->ls_na, 2, g->ls_X, g->st);
  XLS_CUDA(cudaGetLastError());
  XLS_CUDA(cudaMemcpyAsync(X_out, g->ls_X, (size_t)ng * 32 * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->st));
  XLS_CUDA(cudaStreamSynchronize(g->st));
  return XLS_OK;
}

xls_status xls_learned_start(xls_grid g, xls_mlp m, double n_electrons, double* rho_out, int on_device) {
  if (!g || !rho_out || !(n_electrons > 0)) return fail(XLS_EINVAL, "xls_learned_start: bad arguments");
  if (!g->ham_set) return fail(XLS_EINVAL, "xls_learned_start: call xls_hamiltonian_set first (atoms)");
  XLS_TRY(ls_tables(g));
  const long long ng = (long long)g->gn[0] * g->gn[1] * g->gn[2];
  cudaStream_t st = g->st;
  launch_gaussian_density(g->ls_na, g->ls_pos, g->ls_rc, g->ls_amp, g->gn, g->gh, g->gL, g->ls_g1, g->ls_sad,
                          n_electrons, g->ls_partial, g->ls_s, st);
  double* out = g->ls_sad;
  if (m) {
    if (!g->ls_X) XLS_TRY(g->alloc(&g->ls_X, (size_t)ng * 32 * sizeof(float)));
    if (!g->ls_y) XLS_TRY(g->alloc(&g->ls_y, (size_t)ng * sizeof(float)));
    if (!g->rho) XLS_TRY(g->alloc(&g->rho, ng * sizeof(double)));
    launch_descriptors(ng, g->gn, g->gh, g->gL, g->ls_atoms, g->ls_na, 2, g->ls_X, st);
    if (m->st != st) XLS_CUDA(cudaStreamSynchronize(m->st));   // the model's pending updates
    launch_mlp_infer(ng, m->theta, g->ls_X, g->ls_y, st);
    launch_add_clamp(ng, g->ls_sad, g->ls_y, g->rho, st);
    launch_sum(ng, g->rho, g->ls_partial, g->ls_s, st);
    launch_rescale(ng, g->ls_s, n_electrons / (g->gh[0] * g->gh[1] * g->gh[2]), g->rho, st);
    out = g->rho;
  }
  XLS_CUDA(cudaGetLastError());
  XLS_CUDA(cudaMemcpyAsync(rho_out, out, ng * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           st));
  XLS_CUDA(cudaStreamSynchronize(st));
  return XLS_OK;
}

xls_status xls_orbitals_store_fp16(xls_grid g, int sub, uint16_t* half_out, int* exp_out) {
  if (!g || !half_out || !exp_out || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_orbitals_store_fp16: bad arguments");
  if (g->wave) return not_in_wave_mode("xls_orbitals_store_fp16");
  const SubDev& S = g->subs[sub];
  const size_t n = (size_t)S.nd * S.ns;
  void* dh = nullptr;
  int* de = nullptr;
  XLS_CUDA(cudaMallocAsync(&dh, n * 2, g->st));
  XLS_CUDA(cudaMallocAsync((void**)&de, S.ns * sizeof(int), g->st));
  if (g->prec == XLS_FP64) launch_store_half<double>((const double*)g->blk[g->cur] + S.off_blk, S.nd, S.ns, de, dh, g->st);
  else launch_store_half<float>((const float*)g->blk[g->cur] + S.off_blk, S.nd, S.ns, de, dh, g->st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(half_out, dh, n * 2, cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(exp_out, de, S.ns * sizeof(int), cudaMemcpyDeviceToHost, g->st);
  cudaFreeAsync(dh, g->st);
  cudaFreeAsync(de, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return fail(XLS_ECUDA, cudaGetErrorString(e));
  return XLS_OK;
}

xls_status xls_orbitals_load_fp16(xls_grid g, int sub, const uint16_t* half_in, const int* exp_in) {
  if (!g || !half_in || !exp_in || sub < 0 || sub >= g->n_sub) return fail(XLS_EINVAL, "xls_orbitals_load_fp16: bad arguments");
  if (g->wave) return not_in_wave_mode("xls_orbitals_load_fp16");
  const SubDev& S = g->subs[sub];
  const size_t n = (size_t)S.nd * S.ns;
  void* dh = nullptr;
  int* de = nullptr;
  XLS_CUDA(cudaMallocAsync(&dh, n * 2, g->st));
  XLS_CUDA(cudaMallocAsync((void**)&de, S.ns * sizeof(int), g->st));
  cudaError_t e = cudaMemcpyAsync(dh, half_in, n * 2, cudaMemcpyHostToDevice, g->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(de, exp_in, S.ns * sizeof(int), cudaMemcpyHostToDevice, g->st);
  if (e == cudaSuccess) {
    if (g->prec == XLS_FP64) launch_load_half<double>(dh, S.nd, S.ns, de, (double*)g->blk[g->cur] + S.off_blk, g->st);
    else launch_load_half<float>(dh, S.nd, S.ns, de, (float*)g->blk[g->cur] + S.off_blk, g->st);
    e = cudaGetLastError();
  }
  cudaFreeAsync(dh, g->st);
  cudaFreeAsync(de, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  if (e != cudaSuccess) return fail(XLS_ECUDA, cudaGetErrorString(e));
  g->orb_set = true;
  return XLS_OK;
}

xls_status xls_selftest_wait(int spin_limit, void* cuda_stream) {
  if (spin_limit < 1 || spin_limit > (1 << 20)) return fail(XLS_EINVAL, "xls_selftest_wait: spin_limit in 1..2^20");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int* d = nullptr;
  XLS_CUDA(cudaMalloc(&d, sizeof(int)));
  XLS_CUDA(cudaMemsetAsync(d, 0, sizeof(int), st));
  launch_wait_selftest(spin_limit, d, st);
  int h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return fail(XLS_ECUDA, cudaGetErrorString(e));
  if (h == XLS_ETIMEOUT) return fail(XLS_ETIMEOUT, "bounded device wait gave up (self-test)");
  return XLS_OK;
}

xls_status xls_fermi_partial(xls_grid g, double mu, double kT, double* out4) {
  if (!g || !out4 || !(kT > 0) || !g->have_ritz) return fail(XLS_EINVAL, "xls_fermi_partial: bad arguments or no pass run yet");
  launch_fermi_partial(g->lam, g->cw, g->tot_states, mu, kT, g->out4, g->st);
  XLS_CUDA(cudaGetLastError());
  XLS_CUDA(cudaMemcpyAsync(out4, g->out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
  XLS_CUDA(cudaStreamSynchronize(g->st));
  return XLS_OK;
}

xls_status xls_fermi_histogram(xls_grid g, double lo, double hi, int n_bins, double* hist_out) {
  if (!g || !hist_out || !(hi > lo) || n_bins < 1 || n_bins > 4096 || !g->have_ritz)
    return fail(XLS_EINVAL, "xls_fermi_histogram: bad arguments or no pass run yet");
  double* d = nullptr;
  XLS_CUDA(cudaMallocAsync(&d, n_bins * sizeof(double), g->st));
  launch_fermi_hist(g->lam, g->cw, g->tot_states, lo, hi, n_bins, d, g->st);
  XLS_CUDA(cudaGetLastError());
  XLS_CUDA(cudaMemcpyAsync(hist_out, d, n_bins * sizeof(double), cudaMemcpyDeviceToHost, g->st));
  XLS_CUDA(cudaFreeAsync(d, g->st));
  XLS_CUDA(cudaStreamSynchronize(g->st));
  return XLS_OK;
}

xls_status xls_density_at(xls_grid g, double mu, double kT, double* rho_out, int rho_on_device, double* e3_out) {
  if (!g || !(kT > 0) || !g->have_ritz) return fail(XLS_EINVAL, "xls_density_at: bad arguments or no pass run yet");
  if (g->wave) return not_in_wave_mode("xls_density_at");
  launch_occ_at(g->lam, g->cw, g->tot_states, mu, kT, g->occ, g->out4, g->st);
  double h[3];
  XLS_CUDA(cudaMemcpyAsync(h, g->out4, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
  if (rho_out) {
    const long long ng = (long long)g->gn[0] * g->gn[1] * g->gn[2];
    if (!g->rho) XLS_TRY(g->alloc(&g->rho, ng * sizeof(double)));
    XLS_CUDA(cudaMemsetAsync(g->rho, 0, ng * sizeof(double), g->st));
    if (g->prec == XLS_FP64)
      launch_density_occ<double>(g->d_subs, g->n_sub, g->max_core, (const double*)g->blk[g->cur], g->occ, g->gn, g->rho, g->st);
    else
      launch_density_occ<float>(g->d_subs, g->n_sub, g->max_core, (const float*)g->blk[g->cur], g->occ, g->gn, g->rho, g->st);
    XLS_CUDA(cudaMemcpyAsync(rho_out, g->rho, ng * sizeof(double),
                             rho_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->st));
  }
  XLS_CUDA(cudaStreamSynchronize(g->st));
  if (e3_out) {
    e3_out[0] = h[0];
    e3_out[1] = h[1];
    e3_out[2] = h[2];
  }
  return XLS_OK;
}

xls_status xls_get_waves(xls_grid g, int* n_waves_out, int* first_sub_out) {
  if (!g || !n_waves_out) return fail(XLS_EINVAL, "xls_get_waves: bad arguments");
  *n_waves_out = g->wave ? (int)g->waves.size() : 1;
  if (first_sub_out) {
    if (g->wave)
      for (size_t w = 0; w < g->waves.size(); ++w) first_sub_out[w] = g->waves[w].first;
    else
      first_sub_out[0] = 0;
  }
  return XLS_OK;
}

xls_status xls_set_graphs(xls_grid g, int on) {
  if (!g) return fail(XLS_EINVAL, "null grid");
  if (!on && !g->graphs.empty()) {
    XLS_CUDA(cudaStreamSynchronize(g->st));
    g->drop_graphs();
  }
  g->use_graphs = on != 0;
  return XLS_OK;
}

xls_status xls_get_kernel_times(xls_grid g, double* ms8_out, int* count8_out) {
  if (!g) return fail(XLS_EINVAL, "null grid");
  if (g->wave && g->carry && g->worker) return xls_get_kernel_times(g->worker, ms8_out, count8_out);
  for (int c = 0; c < 8; ++c) {
    if (ms8_out) ms8_out[c] = g->kms[c];
    if (count8_out) count8_out[c] = g->kcnt[c];
  }
  return XLS_OK;
}

xls_status xls_get_timings(xls_grid g, double* ms4_out, int* launches_out) {
  if (!g) return fail(XLS_EINVAL, "null grid");
  if (g->wave) {
    if (ms4_out)
      for (int i = 0; i < 4; ++i) ms4_out[i] = g->wave_stage_ms[i];
    if (launches_out) *launches_out = g->last_launches;
    return XLS_OK;
  }
  if (ms4_out)
    for (int i = 0; i < 4; ++i) ms4_out[i] = g->stage_ms[i];
  if (launches_out) *launches_out = g->last_launches;
  return XLS_OK;
}

}  // extern "C"
