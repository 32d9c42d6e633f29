// Subspace contractions on SIMT cores (FP64 path), interior weights, Fermi level, density,
// and the small set-up kernels (restriction, projector norms, Lanczos bound, random start).
#include <cooperative_groups.h>
#include <cstdlib>
#include <cuda_fp16.h>

#include "xls_internal.h"

namespace xls {

__device__ __forceinline__ int wrapd(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = (T)0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double block_sum_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = -1e300;
  for (int i = 0; i < nw; ++i) s = fmax(s, red[i]);
  __syncthreads();
  return s;
}

// ---- projection: M_s = F F^T, H_s = F HF^T over the grid (Sec. 5.A.3 step (2)) -------------
// Blocks: (subdomain, 32x32 output tile, K-chunk of the grid); FP64 atomics combine K-chunks.
constexpr int kGT = 32, kGK = 32, kGChunk = 4096;

template <typename T>
__global__ void __launch_bounds__(256)
k_gram(const SubDev* __restrict__ subs, const T* __restrict__ F, const T* __restrict__ HF, double* Ms, double* Hs) {
  const SubDev& S = subs[blockIdx.z];
  const int ns = S.ns;
  const int nt = (ns + kGT - 1) / kGT;
  const int ti = blockIdx.y % nt, tj = blockIdx.y / nt;
  if (tj >= nt) return;
  const long long g0 = (long long)blockIdx.x * kGChunk;
  if (g0 >= S.nd) return;
  const long long g1 = min(S.nd, g0 + kGChunk);
  __shared__ T A[kGK][kGT + 1], B[kGK][kGT + 1], C[kGK][kGT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 x 32
  const T* f = F + S.off_blk;
  const T* hf = HF + S.off_blk;
  T m[4] = {0, 0, 0, 0}, h[4] = {0, 0, 0, 0};
  for (long long k0 = g0; k0 < g1; k0 += kGK) {
    // load rows (i0 + r) and (j0 + r), points k0 + tx
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = ty * 4 + rr;
      const long long g = k0 + tx;
      const int i = ti * kGT + r, j = tj * kGT + r;
      const bool okg = g < g1;
      A[tx][r] = (okg && i < ns) ? f[(long long)i * S.nd + g] : (T)0;
      B[tx][r] = (okg && j < ns) ? f[(long long)j * S.nd + g] : (T)0;
      C[tx][r] = (okg && j < ns) ? hf[(long long)j * S.nd + g] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kGK; ++k) {
      const T b = B[k][tx], c = C[k][tx];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const T a = A[k][ty * 4 + rr];
        m[rr] += a * b;
        h[rr] += a * c;
      }
    }
    __syncthreads();
  }
  const int j = tj * kGT + tx;
  if (j >= ns) return;
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int i = ti * kGT + ty * 4 + rr;
    if (i < ns) {
      atomicAdd(Ms + S.off_ss + (long long)i * ns + j, (double)m[rr]);
      atomicAdd(Hs + S.off_ss + (long long)i * ns + j, (double)h[rr]);
    }
  }
}

template <typename T>
void launch_gram(const SubDev* d_subs, int n_sub, int max_ns, long long max_nd, const T* F, const T* HF, double* Ms,
                 double* Hs, cudaStream_t st) {
  const int nt = (max_ns + kGT - 1) / kGT;
  dim3 grid((unsigned)((max_nd + kGChunk - 1) / kGChunk), nt * nt, n_sub);
  k_gram<T><<<grid, 256, 0, st>>>(d_subs, F, HF, Ms, Hs);
}

// ---- rotation: Out[n][g] = sum_k Y[k][n] F[k][g] (Sec. 5.A.3 step (4)) ----------------------
constexpr int kRG = 64, kRN = 64, kRK = 16;

template <typename T>
__global__ void __launch_bounds__(256)
k_rotate(const SubDev* __restrict__ subs, const T* __restrict__ F, const double* __restrict__ Y, T* Out) {
  const SubDev& S = subs[blockIdx.z];
  const int ns = S.ns;
  const long long g0 = (long long)blockIdx.x * kRG;
  const int n0 = blockIdx.y * kRN;
  if (g0 >= S.nd || n0 >= ns) return;
  __shared__ T Fs[kRK][kRG];
  __shared__ T Ys[kRK][kRN];
  const int tg = threadIdx.x & 15, tn = threadIdx.x >> 4;  // 16 x 16
  const T* f = F + S.off_blk;
  const double* y = Y + S.off_ss;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
  for (int k0 = 0; k0 < ns; k0 += kRK) {
    for (int s = threadIdx.x; s < kRK * kRG; s += 256) {
      const int kk = s / kRG, gg = s % kRG;
      const int k = k0 + kk;
      const long long g = g0 + gg;
      Fs[kk][gg] = (k < ns && g < S.nd) ? f[(long long)k * S.nd + g] : (T)0;
    }
    for (int s = threadIdx.x; s < kRK * kRN; s += 256) {
      const int kk = s / kRN, nn = s % kRN;
      const int k = k0 + kk, n = n0 + nn;
      Ys[kk][nn] = (k < ns && n < ns) ? (T)y[(long long)k * ns + n] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kRK; ++kk) {
      T fv[4], yv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) fv[a] = Fs[kk][tg + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) yv[b] = Ys[kk][tn * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += fv[a] * yv[b];
    }
    __syncthreads();
  }
  T* o = Out + S.off_blk;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int n = n0 + tn * 4 + b;
    if (n >= ns) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const long long g = g0 + tg + 16 * a;
      if (g < S.nd) o[(long long)n * S.nd + g] = acc[a][b];
    }
  }
}

template <typename T>
void launch_rotate(const SubDev* d_subs, int n_sub, int max_ns, long long max_nd, const T* F, const double* Y, T* Out,
                   cudaStream_t st) {
  dim3 grid((unsigned)((max_nd + kRG - 1) / kRG), (max_ns + kRN - 1) / kRN, n_sub);
  k_rotate<T><<<grid, 256, 0, st>>>(d_subs, F, Y, Out);
}

// ---- interior weights c_n = sum over core points of psi_n^2 (Sec. 5.A.4) ------------------
template <typename T>
__global__ void __launch_bounds__(256) k_core_weights(const SubDev* __restrict__ subs, const T* __restrict__ Psi, double* c) {
  const SubDev& S = subs[blockIdx.y];
  const int v = blockIdx.x;
  if (v >= S.ns) return;
  const T* p = Psi + S.off_blk + (long long)v * S.nd;
  const int cx = S.core_n[0], cy = S.core_n[1], cz = S.core_n[2];
  // core rows (j, k) by warps, points of a row by lanes; each thread's partial sum in the block's
  // precision (a few dozen terms), the block sum in FP64
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  T part = (T)0;
  for (int r = warp; r < cy * cz; r += nw) {
    const int j = r % cy, k = r / cy;
    const T* row = p + ((long long)(S.core_lo[2] + k) * S.n[1] + (S.core_lo[1] + j)) * S.n[0] + S.core_lo[0];
    for (int i = lane; i < cx; i += 32) {
      const T x = row[i];
      part += x * x;
    }
  }
  __shared__ double red[32];
  const double acc = block_sum((double)part, red);
  if (threadIdx.x == 0) c[S.off_state + v] = acc;
}

template <typename T>
void launch_core_weights(const SubDev* d_subs, int n_sub, int max_ns, const T* Psi, double* c, cudaStream_t st) {
  dim3 grid(max_ns, n_sub);
  k_core_weights<T><<<grid, 256, 0, st>>>(d_subs, Psi, c);
}

// ---- core rows of every vector into a compact store (waves): subdomain j of the launch, vector
// v at store + dst[j].off_blk + v * core_points, x fastest (dst: the store's descriptors of the
// launch's subdomains); the density is formed from it after the Fermi level of all subdomains
// is known ----------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_core_gather(const SubDev* __restrict__ subs, const T* __restrict__ Psi, T* __restrict__ store,
              const SubDev* __restrict__ dst) {
  const SubDev& S = subs[blockIdx.y];
  const int v = blockIdx.x;
  if (v >= S.ns) return;
  const int cx = S.core_n[0], cy = S.core_n[1], cz = S.core_n[2];
  const T* p = Psi + S.off_blk + (long long)v * S.nd;
  T* q = store + dst[blockIdx.y].off_blk + (long long)v * cx * cy * cz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = warp; r < cy * cz; r += nw) {
    const int j = r % cy, k = r / cy;
    const T* row = p + ((long long)(S.core_lo[2] + k) * S.n[1] + (S.core_lo[1] + j)) * S.n[0] + S.core_lo[0];
    T* out = q + (long long)r * cx;
    for (int i = lane; i < cx; i += 32) out[i] = row[i];
  }
}

template <typename T>
void launch_core_gather(const SubDev* d_subs, int n_sub, int max_ns, const T* Psi, T* store, const SubDev* d_dst,
                        cudaStream_t st) {
  dim3 grid(max_ns, n_sub);
  k_core_gather<T><<<grid, 256, 0, st>>>(d_subs, Psi, store, d_dst);
}

// ---- density on the core points: rho = (2/dV) sum_n occ_n psi_n^2 (Eq. density) ----------
template <typename T>
__global__ void __launch_bounds__(256)
k_density(const SubDev* __restrict__ subs, const T* __restrict__ Psi, const double* __restrict__ occ, int gnx, int gny,
          double* rho) {
  const SubDev& S = subs[blockIdx.y];
  const int cx = S.core_n[0], cy = S.core_n[1], cz = S.core_n[2];
  const long long ncore = (long long)cx * cy * cz;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ncore) return;
  const int qi = (int)q;   // a subdomain core has fewer than 2^31 points
  const int i = qi % cx, j = (qi / cx) % cy, k = qi / (cx * cy);
  const long long g = ((long long)(S.core_lo[2] + k) * S.n[1] + (S.core_lo[1] + j)) * S.n[0] + (S.core_lo[0] + i);
  const T* p = Psi + S.off_blk + g;
  const double* o = occ + S.off_state;
  // sum over the states in the block's precision (FP32 blocks: FP32 FMAs, relative error ~1e-7)
  T acc_t = (T)0;
  for (int v = 0; v < S.ns; ++v) {
    const T x = p[(long long)v * S.nd];
    acc_t += (T)o[v] * x * x;
  }
  const double acc = (double)acc_t;
  const long long G = ((long long)(S.core_glo[2] + k) * gny + (S.core_glo[1] + j)) * gnx + (S.core_glo[0] + i);
  rho[G] = 2.0 * acc / S.dV;
}

template <typename T>
void launch_density_occ(const SubDev* d_subs, int n_sub, long long max_core, const T* Psi, const double* occ,
                        const int gn[3], double* rho, cudaStream_t st) {
  dim3 grid((unsigned)((max_core + 255) / 256), n_sub);
  k_density<T><<<grid, 256, 0, st>>>(d_subs, Psi, occ, gn[0], gn[1], rho);
}

// ---- Fermi level by FP64 bisection, occupations and energies (Sec. 5.A.4-5) ----------------
__device__ __forceinline__ double fermi_fn(double x) {
  if (x > 0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

// out: [0] mu, [1] E_band, [2] E_entropy, [3] N_e(mu); occ[n] = g_n.
__global__ void __launch_bounds__(1024)
k_fermi(const double* __restrict__ lam, const double* __restrict__ c, int n, double ne, double kT, double* out,
        double* occ, int* status) {
  __shared__ double red[32];
  __shared__ double s_lo, s_hi;
  double lmin = 1e300, lmax = -1e300;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    lmin = fmin(lmin, lam[i]);
    lmax = fmax(lmax, lam[i]);
  }
  // block min/max via shuffles + shared
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lmin = fmin(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  }
  __shared__ double smin[32], smax[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) { smin[w] = lmin; smax[w] = lmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 1e300, b = -1e300;
    for (int i = 0; i < nw; ++i) { a = fmin(a, smin[i]); b = fmax(b, smax[i]); }
    s_lo = a - 1.0;
    s_hi = b + 1.0;
  }
  __syncthreads();
  // N_e(mu) and dN_e/dmu in one sweep (the paper's Newton refinement, Sec. 5.A.5), safeguarded by
  // the bracket: a Newton step outside (lo, hi) is replaced by bisection.
  auto count2 = [&](double mu, double& dn) -> double {
    double acc = 0.0, dacc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double g = fermi_fn((lam[i] - mu) / kT);
      acc += g * c[i];
      dacc += g * (1.0 - g) * c[i];
    }
    dn = 2.0 * block_sum(dacc, red) / kT;
    return 2.0 * block_sum(acc, red);
  };
  double lo = s_lo, hi = s_hi, dn;
  const double nlo = count2(lo, dn), nhi = count2(hi, dn);
  if (!(nlo <= ne && ne <= nhi)) {
    if (threadIdx.x == 0) { *status = XLS_ENOCONV; out[0] = out[1] = out[2] = out[3] = 0.0; }
    return;
  }
  double mu_k = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    const double nm = count2(mu_k, dn);
    if (nm < ne) lo = mu_k; else hi = mu_k;
    if (nm == ne || hi - lo <= 1e-14) break;
    double next = (dn > 0.0) ? mu_k - (nm - ne) / dn : 0.5 * (lo + hi);
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    if (fabs(next - mu_k) <= 1e-15 * fmax(1.0, fabs(mu_k))) { mu_k = next; break; }
    mu_k = next;
  }
  const double mu = mu_k;
  double eb = 0.0, es = 0.0, nn = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double g = fermi_fn((lam[i] - mu) / kT);
    occ[i] = g;
    eb += g * c[i] * lam[i];
    const double q = 1.0 - g;
    const double s = (g > 0 ? g * log(g) : 0.0) + (q > 0 ? q * log(q) : 0.0);
    es += c[i] * s;
    nn += g * c[i];
  }
  eb = block_sum(eb, red);
  es = block_sum(es, red);
  nn = block_sum(nn, red);
  if (threadIdx.x == 0) {
    out[0] = mu;
    out[1] = 2.0 * eb;
    out[2] = -2.0 * kT * es;
    out[3] = 2.0 * nn;
  }
}

// The same Fermi level on a cluster of kFermiCL CTAs, so that the FP64 Fermi-function sums of
// every iteration run on kFermiCL SMs.  Every CTA sums its share of the states and pushes its
// partial sums into a slot of every CTA's shared memory (distributed shared memory); after one
// cluster barrier every CTA adds the slots in the same order and takes the same decision.  The
// bracket comes from a histogram of 2 c_n over the eigenvalue range (no exponentials): the bin
// where the cumulative count crosses N_e, widened by 40 kT on both sides (where the Fermi
// function has reached e^-40), holds the root whenever N_e changes inside it; Newton steps on
// N_e(mu), kept inside the bracket, then take a few iterations instead of dozens of bisections.
namespace cg = cooperative_groups;
constexpr int kFermiCL = 8, kFermiBins = 256;

__global__ void __launch_bounds__(256)
k_fermi_cl(const double* __restrict__ lam, const double* __restrict__ c, int n, double ne, double kT, double* out,
           double* occ, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  __shared__ double red[32];
  __shared__ double part[2][kFermiCL][4];         // partial sums of every CTA, alternate buffers
  __shared__ double hist[kFermiCL][kFermiBins];   // histogram of every CTA
  __shared__ double hloc[kFermiBins];
  __shared__ double s_cum[kFermiBins];
  const int t = threadIdx.x;
  const int i0 = rank * blockDim.x + t, stride = CL * blockDim.x;
  int buf = 0;
  // all-gather of four scalars; returns after the cluster barrier
  auto gather = [&](double a0, double a1, double a2, double a3) {
    if (t < CL) {
      double* dst = cl.map_shared_rank(&part[buf][rank][0], t);
      dst[0] = a0; dst[1] = a1; dst[2] = a2; dst[3] = a3;
    }
    cl.sync();
  };
  auto total = [&](int k) {
    double s = 0.0;
    for (int q = 0; q < CL; ++q) s += part[buf][q][k];
    return s;
  };
  double lmin = 1e300, lmax = -1e300;
  for (int i = i0; i < n; i += stride) {
    lmin = fmin(lmin, lam[i]);
    lmax = fmax(lmax, lam[i]);
  }
  lmax = block_sum_max(lmax, red);
  lmin = -block_sum_max(-lmin, red);
  gather(lmin, lmax, 0.0, 0.0);
  double lo = 1e300, hi = -1e300;
  for (int q = 0; q < CL; ++q) {
    lo = fmin(lo, part[buf][q][0]);
    hi = fmax(hi, part[buf][q][1]);
  }
  lo -= 1.0;
  hi += 1.0;
  buf ^= 1;
  // histogram bracket
  const double w = (hi - lo) / kFermiBins;
  for (int b = t; b < kFermiBins; b += blockDim.x) hloc[b] = 0.0;
  __syncthreads();
  for (int i = i0; i < n; i += stride) {
    const int b = min(kFermiBins - 1, max(0, (int)((lam[i] - lo) / w)));
    atomicAdd(&hloc[b], 2.0 * c[i]);
  }
  __syncthreads();
  for (int b = t; b < kFermiBins; b += blockDim.x)
    for (int q = 0; q < CL; ++q) cl.map_shared_rank(&hist[rank][0], q)[b] = hloc[b];
  cl.sync();
  // cumulative counts by a block-wide scan (one bin per thread; blockDim == kFermiBins), then the
  // first bin whose cumulative count reaches N_e
  __shared__ double s_wsum[kFermiBins / 32];
  __shared__ int s_bstar;
  {
    double tb = 0.0;
    for (int q = 0; q < CL; ++q) tb += hist[q][t];
    const int l = t & 31, w = t >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, tb, o);
      if (l >= o) tb += y;
    }
    if (l == 31) s_wsum[w] = tb;
    if (t == 0) s_bstar = kFermiBins - 1;
    __syncthreads();
    double base = 0.0;
    for (int q = 0; q < w; ++q) base += s_wsum[q];
    s_cum[t] = base + tb;
    __syncthreads();
    if (s_cum[t] >= ne && (t == 0 || s_cum[t - 1] < ne)) s_bstar = t;
    __syncthreads();
  }
  const int bstar = s_bstar;
  auto count2 = [&](double mu, double& dn) -> double {
    double acc = 0.0, dacc = 0.0;
    for (int i = i0; i < n; i += stride) {
      const double g = fermi_fn((lam[i] - mu) / kT);
      acc += g * c[i];
      dacc += g * (1.0 - g) * c[i];
    }
    acc = block_sum(acc, red);
    dacc = block_sum(dacc, red);
    gather(acc, dacc, 0.0, 0.0);
    const double nm = 2.0 * total(0);
    dn = 2.0 * total(1) / kT;
    buf ^= 1;
    return nm;
  };
  double dn;
  double blo = fmax(lo, lo + fmax(bstar - 1, 0) * w - 40.0 * kT);
  double bhi = fmin(hi, lo + fmin(bstar + 2, kFermiBins) * w + 40.0 * kT);
  double nlo = count2(blo, dn), nhi = count2(bhi, dn);
  if (!(nlo <= ne && ne <= nhi)) {
    blo = lo;
    bhi = hi;
    nlo = count2(blo, dn);
    nhi = count2(bhi, dn);
    if (!(nlo <= ne && ne <= nhi)) {
      if (rank == 0 && t == 0) { *status = XLS_ENOCONV; out[0] = out[1] = out[2] = out[3] = 0.0; }
      return;
    }
  }
  lo = blo;
  hi = bhi;
  double mu_k = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    const double nm = count2(mu_k, dn);
    if (nm < ne) lo = mu_k; else hi = mu_k;
    if (nm == ne || hi - lo <= 1e-14) break;
    double next = (dn > 0.0) ? mu_k - (nm - ne) / dn : 0.5 * (lo + hi);
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    if (fabs(next - mu_k) <= 1e-15 * fmax(1.0, fabs(mu_k))) { mu_k = next; break; }
    mu_k = next;
  }
  const double mu = mu_k;
  double eb = 0.0, es = 0.0, nn = 0.0;
  for (int i = i0; i < n; i += stride) {
    const double g = fermi_fn((lam[i] - mu) / kT);
    occ[i] = g;
    eb += g * c[i] * lam[i];
    const double q = 1.0 - g;
    const double sl = (g > 0 ? g * log(g) : 0.0) + (q > 0 ? q * log(q) : 0.0);
    es += c[i] * sl;
    nn += g * c[i];
  }
  eb = block_sum(eb, red);
  es = block_sum(es, red);
  nn = block_sum(nn, red);
  gather(eb, es, nn, 0.0);
  if (rank == 0 && t == 0) {
    out[0] = mu;
    out[1] = 2.0 * total(0);
    out[2] = -2.0 * kT * total(1);
    out[3] = 2.0 * total(2);
  }
}

void launch_fermi_occ(const double* lam, const double* c, int n_tot, double n_e, double kT, double* out4, double* occ,
                      int* status, cudaStream_t st) {
  if (!std::getenv("XLS_FERMI_SINGLE")) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kFermiCL);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kFermiCL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_fermi_cl, lam, c, n_tot, n_e, kT, out4, occ, status) == cudaSuccess) return;
    cudaGetLastError();
  }
  k_fermi<<<1, 1024, 0, st>>>(lam, c, n_tot, n_e, kT, out4, occ, status);
}

// ---- density of states, Eq. dos: D(E) = 2 sum_alpha sum_n c_n delta(E - lambda_n), the delta
// function broadened to a normalised Gaussian of width w.  One thread per energy point; the
// Ritz values and weights are staged through shared memory in chunks.
__global__ void __launch_bounds__(256)
k_dos(const double* __restrict__ lam, const double* __restrict__ c, int n, const double* __restrict__ energies,
      int n_e, double w, double* out) {
  __shared__ double sl[256], sc[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double e = i < n_e ? energies[i] : 0.0;
  const double inv2w2 = 0.5 / (w * w), norm = 1.0 / (w * sqrt(2.0 * 3.14159265358979323846));
  double acc = 0.0;
  for (int q0 = 0; q0 < n; q0 += 256) {
    const int q = q0 + threadIdx.x;
    sl[threadIdx.x] = q < n ? lam[q] : 0.0;
    sc[threadIdx.x] = q < n ? c[q] : 0.0;
    __syncthreads();
    const int m = min(256, n - q0);
    for (int k = 0; k < m; ++k) {
      const double d = e - sl[k];
      acc += sc[k] * exp(-d * d * inv2w2);
    }
    __syncthreads();
  }
  if (i < n_e) out[i] = 2.0 * norm * acc;
}

void launch_dos(const double* lam, const double* c, int n, const double* energies, int n_e, double w, double* out,
                cudaStream_t st) {
  if (n_e <= 0) return;
  k_dos<<<(n_e + 255) / 256, 256, 0, st>>>(lam, c, n, energies, n_e, w, out);
}

// ---- FP16 orbital storage (warm start between SCF steps): vector v stored as
// half(psi_v * 2^e_v) with e_v such that max |psi_v| 2^e_v lies in [2^13, 2^14) -------------------
template <typename T>
__global__ void __launch_bounds__(256) k_vec_exp14(const T* __restrict__ X, long long nd, int* ex) {
  __shared__ float red[8];
  const T* x = X + (long long)blockIdx.x * nd;
  float m = 0.f;
  for (long long i = threadIdx.x; i < nd; i += blockDim.x) m = fmaxf(m, fabsf((float)x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmaxf(t, red[i]);
    int k = 0;
    frexpf(t, &k);                       // 2^(k-1) <= t < 2^k
    ex[blockIdx.x] = t > 0.f ? 14 - k : 0;
  }
}

template <typename T>
__global__ void k_to_half(const T* __restrict__ X, long long nd, int ns, const int* __restrict__ ex, __half* out) {
  const long long n = nd * ns;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = __float2half_rn((float)ldexp((double)X[q], ex[q / nd]));
}

template <typename T>
__global__ void k_from_half(const __half* __restrict__ in, long long nd, int ns, const int* __restrict__ ex, T* X) {
  const long long n = nd * ns;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    X[q] = (T)ldexp((double)__half2float(in[q]), -ex[q / nd]);
}

template <typename T>
void launch_store_half(const T* X, long long nd, int ns, int* ex, void* out, cudaStream_t st) {
  k_vec_exp14<T><<<ns, 256, 0, st>>>(X, nd, ex);
  k_to_half<T><<<592, 256, 0, st>>>(X, nd, ns, ex, (__half*)out);
}
template <typename T>
void launch_load_half(const void* in, long long nd, int ns, const int* ex, T* X, cudaStream_t st) {
  k_from_half<T><<<592, 256, 0, st>>>((const __half*)in, nd, ns, ex, X);
}
template void launch_store_half<float>(const float*, long long, int, int*, void*, cudaStream_t);
template void launch_store_half<double>(const double*, long long, int, int*, void*, cudaStream_t);
template void launch_load_half<float>(const void*, long long, int, const int*, float*, cudaStream_t);
template void launch_load_half<double>(const void*, long long, int, const int*, double*, cudaStream_t);

// ---- bounded-wait self-test: an mbarrier that nothing completes, waited on with an iteration
// limit; the wait gives up and records XLS_ETIMEOUT (the path every bounded wait of the library
// takes when its copy or peer never arrives) ------------------------------------------------------
__global__ void k_wait_selftest(int spin_limit, int* status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1) : "memory");
  __syncthreads();
  bool done = false;
  for (int i = 0; i < spin_limit && !done; ++i) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(a), "r"(0u)
                 : "memory");
    done = ok != 0;
  }
  if (!done && threadIdx.x == 0) atomicCAS(status, 0, XLS_ETIMEOUT);
}

void launch_wait_selftest(int spin_limit, int* status, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(spin_limit, status);
}

// ---- partial sums of this grid's states for a Fermi level found across ranks (Sec. 5.A.5:
// histogram of the eigenvalues, then Newton on N_e(mu) with dN_e/dmu) -------------------------
// out: [0] 2 sum c g, [1] 2 sum c g (1 - g) / kT, [2] min lambda, [3] max lambda
__global__ void __launch_bounds__(1024)
k_fermi_partial(const double* __restrict__ lam, const double* __restrict__ c, int n, double mu, double kT, double* out) {
  __shared__ double red[32];
  double acc = 0.0, dacc = 0.0, lmin = 1e300, lmax = -1e300;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double g = fermi_fn((lam[i] - mu) / kT);
    acc += g * c[i];
    dacc += g * (1.0 - g) * c[i];
    lmin = fmin(lmin, lam[i]);
    lmax = fmax(lmax, lam[i]);
  }
  acc = block_sum(acc, red);
  dacc = block_sum(dacc, red);
  lmin = -block_sum_max(-lmin, red);
  lmax = block_sum_max(lmax, red);
  if (threadIdx.x == 0) {
    out[0] = 2.0 * acc;
    out[1] = 2.0 * dacc / kT;
    out[2] = lmin;
    out[3] = lmax;
  }
}

// hist[b] = 2 sum of c over the states with lambda in bin b of [lo, hi) (nb bins; below lo
// counted in bin 0, at or above hi in bin nb - 1)
__global__ void __launch_bounds__(1024)
k_fermi_hist(const double* __restrict__ lam, const double* __restrict__ c, int n, double lo, double hi, int nb,
             double* hist) {
  extern __shared__ double sh[];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int b = (int)floor((lam[i] - lo) / (hi - lo) * nb);
    b = b < 0 ? 0 : (b >= nb ? nb - 1 : b);
    atomicAdd(&sh[b], 2.0 * c[i]);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = sh[b];
}

// occupations at a given mu and the partial energies: out [0] E_band, [1] E_entropy, [2] N_e
__global__ void __launch_bounds__(1024)
k_occ_at(const double* __restrict__ lam, const double* __restrict__ c, int n, double mu, double kT, double* occ,
         double* out) {
  __shared__ double red[32];
  double eb = 0.0, es = 0.0, nn = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double g = fermi_fn((lam[i] - mu) / kT);
    occ[i] = g;
    eb += g * c[i] * lam[i];
    const double q = 1.0 - g;
    es += c[i] * ((g > 0 ? g * log(g) : 0.0) + (q > 0 ? q * log(q) : 0.0));
    nn += g * c[i];
  }
  eb = block_sum(eb, red);
  es = block_sum(es, red);
  nn = block_sum(nn, red);
  if (threadIdx.x == 0) {
    out[0] = 2.0 * eb;
    out[1] = -2.0 * kT * es;
    out[2] = 2.0 * nn;
  }
}

void launch_fermi_partial(const double* lam, const double* c, int n, double mu, double kT, double* out,
                          cudaStream_t st) {
  k_fermi_partial<<<1, 1024, 0, st>>>(lam, c, n, mu, kT, out);
}
void launch_fermi_hist(const double* lam, const double* c, int n, double lo, double hi, int nb, double* hist,
                       cudaStream_t st) {
  k_fermi_hist<<<1, 1024, nb * sizeof(double), st>>>(lam, c, n, lo, hi, nb, hist);
}
void launch_occ_at(const double* lam, const double* c, int n, double mu, double kT, double* occ, double* out,
                   cudaStream_t st) {
  k_occ_at<<<1, 1024, 0, st>>>(lam, c, n, mu, kT, occ, out);
}

// ---- filter coefficients of the scaled recurrence (Zhou et al. 2006) ----------------------
// bounds[3a..3a+2] = (b, a, a0); coef[a][1..m]; coef[a][kMaxDegree-1] = (1, 0, 0) = plain H.
__global__ void k_filter_coef(int n_sub, const double* bounds, int m, StepCoef* coef) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_sub) return;
  const double b = bounds[3 * a], lo = bounds[3 * a + 1], a0 = bounds[3 * a + 2];
  const double e = (b - lo) / 2.0, c = (b + lo) / 2.0;
  const double sigma1 = e / (a0 - c);
  double sigma = sigma1;
  StepCoef* cf = coef + (long long)a * kMaxDegree;
  cf[0] = StepCoef{0.0, 0.0, 0.0, 0.0};
  cf[1] = StepCoef{sigma1 / e, c, 0.0, 0.0};
  for (int k = 2; k <= m && k < kMaxDegree - 1; ++k) {
    const double sigma2 = 1.0 / (2.0 / sigma1 - sigma);
    cf[k] = StepCoef{2.0 * sigma2 / e, c, sigma * sigma2, 0.0};
    sigma = sigma2;
  }
  cf[kMaxDegree - 1] = StepCoef{1.0, 0.0, 0.0, 0.0};
}

void launch_filter_coef(int n_sub, const double* bounds, int degree, StepCoef* coef, cudaStream_t st) {
  k_filter_coef<<<(n_sub + 127) / 128, 128, 0, st>>>(n_sub, bounds, degree, coef);
}

// next pass: a = largest, a0 = smallest Ritz value (ascending lambda); b unchanged
__global__ void k_bounds_from_ritz(const SubDev* subs, int n_sub, const double* lam, double* bounds) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_sub) return;
  const SubDev& S = subs[a];
  bounds[3 * a + 1] = lam[S.off_state + S.ns - 1];
  bounds[3 * a + 2] = lam[S.off_state];
}

void launch_bounds_from_ritz(const SubDev* d_subs, int n_sub, const double* lam, double* bounds, cudaStream_t st) {
  k_bounds_from_ritz<<<(n_sub + 127) / 128, 128, 0, st>>>(d_subs, n_sub, lam, bounds);
}

// ---- restriction of V_eff to the subdomains (Sec. 5.A.5) ----------------------------------
__global__ void k_restrict(const SubDev* __restrict__ subs, const double* __restrict__ Vg, int gx, int gy, int gz,
                           double* V, float* Vf) {
  const SubDev& S = subs[blockIdx.y];
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < S.nd; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % S.n[0]), j = (int)((q / S.n[0]) % S.n[1]), k = (int)(q / ((long long)S.n[0] * S.n[1]));
    const int I = wrapd(S.start[0] + i, gx), J = wrapd(S.start[1] + j, gy), K = wrapd(S.start[2] + k, gz);
    const double v = Vg[((long long)K * gy + J) * gx + I];
    V[S.off_pt + q] = v;
    Vf[S.off_pt + q] = (float)v;
  }
}

void launch_restrict(const SubDev* d_subs, int n_sub, long long max_nd, const double* Vg, const int gn[3], double* V,
                     float* Vf, cudaStream_t st) {
  dim3 grid((unsigned)min((max_nd + 255) / 256, 1024LL), n_sub);
  k_restrict<<<grid, 256, 0, st>>>(d_subs, Vg, gn[0], gn[1], gn[2], V, Vf);
}

// ---- projector normalisation on the global periodic grid ----------------------------------
__global__ void k_proj_norms(const AtomImg* __restrict__ imgs, const ProjSlot* __restrict__ slots, double hx,
                             double hy, double hz, double* norms) {
  const AtomImg& A = imgs[blockIdx.x];
  const ProjSlot& Q = slots[blockIdx.x];
  const int bx = A.box_n[0], by = A.box_n[1];
  const int npts = bx * by * A.box_n[2];
  double s[4] = {0, 0, 0, 0};
  for (int p = threadIdx.x; p < npts; p += blockDim.x) {
    const int i = A.box_lo[0] + p % bx, j = A.box_lo[1] + (p / bx) % by, k = A.box_lo[2] + p / (bx * by);
    const double dx = i * hx - A.R[0], dy = j * hy - A.R[1], dz = k * hz - A.R[2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= Q.rcut2) continue;
    const double e = exp(-r2 / (2.0 * Q.w * Q.w));
    s[0] += e * e;
    s[1] += dx * dx * e * e;
    s[2] += dy * dy * e * e;
    s[3] += dz * dz * e * e;
  }
  __shared__ double red[32];
  const double dV = hx * hy * hz;
  for (int l = 0; l < 4; ++l) {
    const double t = block_sum(s[l], red);
    if (threadIdx.x == 0) norms[4 * blockIdx.x + l] = 1.0 / sqrt(t * dV);
  }
}

void launch_proj_norms(const AtomImg* d_imgs_global, const ProjSlot* d_slots_global, int n_atoms, const int gn[3],
                       const double gh[3], double* norms, cudaStream_t st) {
  if (n_atoms == 0) return;
  (void)gn;
  k_proj_norms<<<n_atoms, 256, 0, st>>>(d_imgs_global, d_slots_global, gh[0], gh[1], gh[2], norms);
}

// ---- SplitMix64 (Steele, Lea & Flood 2014), counter form: output i = mix(seed + (i+1) gamma)
__device__ __forceinline__ double splitmix_u(uint64_t seed, unsigned long long i) {
  uint64_t z = seed + (uint64_t)(i + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53 - 0.5;
}

template <typename T>
__global__ void k_splitmix_fill(T* out, long long count, uint64_t seed, long long offset) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (long long)gridDim.x * blockDim.x)
    out[q] = (T)splitmix_u(seed, (unsigned long long)(offset + q));
}

void launch_splitmix_fill_f64(double* out, long long count, uint64_t seed, long long offset, cudaStream_t st) {
  k_splitmix_fill<double><<<4 * 152, 256, 0, st>>>(out, count, seed, offset);
}
void launch_splitmix_fill_f32(float* out, long long count, uint64_t seed, long long offset, cudaStream_t st) {
  k_splitmix_fill<float><<<4 * 152, 256, 0, st>>>(out, count, seed, offset);
}

__global__ void k_f64_to_f32(const double* in, float* out, long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = (float)in[q];
}
__global__ void k_f32_to_f64(const float* in, double* out, long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = (double)in[q];
}
void launch_convert_f64_f32(const double* in, float* out, long long count, cudaStream_t st) {
  k_f64_to_f32<<<4 * 152, 256, 0, st>>>(in, out, count);
}
void launch_convert_f32_f64(const float* in, double* out, long long count, cudaStream_t st) {
  k_f32_to_f64<<<4 * 152, 256, 0, st>>>(in, out, count);
}

// ---- Lanczos upper bound (k steps, per subdomain, FP64) ------------------------------------
// Single-vector views: v, vprev, f hold one vector per subdomain at S.off_blk (ns = 1).
__global__ void __launch_bounds__(1024) k_lz_init(const SubDev* __restrict__ subs, double* v) {
  const SubDev& S = subs[blockIdx.x];
  double* p = v + S.off_blk;
  double acc = 0.0;
  for (long long q = threadIdx.x; q < S.nd; q += blockDim.x) {
    const double x = splitmix_u(0x1A4C705ULL, (unsigned long long)q);
    p[q] = x;
    acc += x * x;
  }
  __shared__ double red[32];
  const double inv = 1.0 / sqrt(block_sum(acc, red));
  for (long long q = threadIdx.x; q < S.nd; q += blockDim.x) p[q] *= inv;
}

void launch_lanczos_init(const SubDev* d_subs, int n_sub, double* v, cudaStream_t st) {
  k_lz_init<<<n_sub, 1024, 0, st>>>(d_subs, v);
}

// Step j (given Hv = H v): f = Hv - beta_j vprev (j > 0); alpha_j = v.f; f -= alpha_j v;
// beta_{j+1} = |f|; then vprev <- v, v <- f / beta_{j+1} for the next step.
__global__ void __launch_bounds__(1024)
k_lz_step(const SubDev* __restrict__ subs, int j, const double* __restrict__ Hv, double* v, double* vprev, double* f,
          double* alpha, double* beta) {
  const int a = blockIdx.x;
  const SubDev& S = subs[a];
  const long long o = S.off_blk;
  const double bj = (j > 0) ? beta[a * 16 + j] : 0.0;
  double acc = 0.0;
  for (long long q = threadIdx.x; q < S.nd; q += blockDim.x) {
    double x = Hv[o + q];
    if (j > 0) x -= bj * vprev[o + q];
    f[o + q] = x;
    acc += v[o + q] * x;
  }
  __shared__ double red[32];
  const double al = block_sum(acc, red);
  acc = 0.0;
  for (long long q = threadIdx.x; q < S.nd; q += blockDim.x) {
    const double x = f[o + q] - al * v[o + q];
    f[o + q] = x;
    acc += x * x;
  }
  const double nb = sqrt(block_sum(acc, red));
  if (threadIdx.x == 0) {
    alpha[a * 16 + j] = al;
    beta[a * 16 + j + 1] = nb;
  }
  const double inv = nb > 0 ? 1.0 / nb : 0.0;
  for (long long q = threadIdx.x; q < S.nd; q += blockDim.x) {
    const double vv = v[o + q];
    vprev[o + q] = vv;
    v[o + q] = f[o + q] * inv;
  }
}

void launch_lanczos_step(const SubDev* d_subs, int n_sub, int j, const double* Hv, double* v, double* vprev, double* f,
                         double* alpha, double* beta, cudaStream_t st) {
  k_lz_step<<<n_sub, 1024, 0, st>>>(d_subs, j, Hv, v, vprev, f, alpha, beta);
}

// b = max eigenvalue of the k x k Lanczos matrix (bisection on Sturm counts) + |f_k|
__global__ void k_lz_finish(int n_sub, int k, const double* alpha, const double* beta, double* bounds) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_sub) return;
  const double* al = alpha + a * 16;
  const double* be = beta + a * 16;  // be[1..k-1] off-diagonals, be[k] = |f_k|
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(be[i]) : 0.0) + (i + 1 < k ? fabs(be[i + 1]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  // largest eigenvalue: smallest x with count(eigs < x) == k
  for (int it = 0; it < 200 && hi - lo > 1e-13 * fmax(1.0, fabs(hi)); ++it) {
    const double x = 0.5 * (lo + hi);
    int cnt = 0;
    double d = al[0] - x;
    if (d < 0) ++cnt;
    for (int i = 1; i < k; ++i) {
      if (d == 0.0) d = 1e-300;
      d = al[i] - x - be[i] * be[i] / d;
      if (d < 0) ++cnt;
    }
    if (cnt >= k) hi = x; else lo = x;
  }
  bounds[3 * a] = hi + be[k];
}

void launch_lanczos_finish(int n_sub, int k, const double* alpha, const double* beta, const SubDev*, const double*,
                           double* bounds, cudaStream_t st) {
  k_lz_finish<<<(n_sub + 127) / 128, 128, 0, st>>>(n_sub, k, alpha, beta, bounds);
}

template void launch_gram<double>(const SubDev*, int, int, long long, const double*, const double*, double*, double*,
                                  cudaStream_t);
template void launch_gram<float>(const SubDev*, int, int, long long, const float*, const float*, double*, double*,
                                 cudaStream_t);
template void launch_rotate<double>(const SubDev*, int, int, long long, const double*, const double*, double*,
                                    cudaStream_t);
template void launch_rotate<float>(const SubDev*, int, int, long long, const float*, const double*, float*,
                                   cudaStream_t);
template void launch_core_gather<double>(const SubDev*, int, int, const double*, double*, const SubDev*,
                                         cudaStream_t);
template void launch_core_gather<float>(const SubDev*, int, int, const float*, float*, const SubDev*,
                                        cudaStream_t);
template void launch_core_weights<double>(const SubDev*, int, int, const double*, double*, cudaStream_t);
template void launch_core_weights<float>(const SubDev*, int, int, const float*, double*, cudaStream_t);
template void launch_density_occ<double>(const SubDev*, int, long long, const double*, const double*, const int*,
                                         double*, cudaStream_t);
template void launch_density_occ<float>(const SubDev*, int, long long, const float*, const double*, const int*,
                                        double*, cudaStream_t);

}  // namespace xls
