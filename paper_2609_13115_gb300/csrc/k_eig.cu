// Generalised symmetric eigensolve H_s y = lambda M_s y of every subdomain, FP64 (Sec. 5.A.3
// step (3); the paper's "dense generalized eigensolver", specialised DSYGVD in Sec. 5.B.3).
//
//   1. M_s = L L^T                   k_cholesky      one CTA per subdomain
//   2. W = L^-1 H_s, A = L^-1 W^T    k_trsm_lower x2 column-parallel CTAs
//   3. A = Q T Q^T (Householder)     k_tridiag       one CTA per subdomain
//   4. T = Z_T diag(lambda) Z_T^T    k_tri_eig       FP32 Sturm bisection for shifts, inverse
//                                                    iteration + Gram-Schmidt per cluster (two
//                                                    FP32 iterations, a final FP64 one), FP64
//                                                    Rayleigh-Ritz (Jacobi) inside each cluster
//                                                    of close eigenvalues
//   5. Z = Q Z_T                     k_backtransform column-parallel CTAs
//   6. Y = L^-T Z                    k_trsm_upper    column-parallel CTAs
//
// Matrices are n x n row-major at S.off_ss; per-subdomain vectors at 8 * S.off_state.
#include "xls_internal.h"

namespace xls {


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_d(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

__device__ void set_status(int* status, int code, int sub) {
  if (atomicCAS(status, 0, code) == 0) status[1] = sub;
}

// ---- 1. Cholesky, left-looking by columns; warp per row for the column update -------------
template <bool kSmem>
__global__ void __launch_bounds__(512) k_cholesky(const SubDev* __restrict__ subs, double* Ms, int* status) {
  const SubDev& S = subs[blockIdx.x];
  const int n = S.ns;
  double* Lg = Ms + S.off_ss;
  extern __shared__ double smat[];
  double* L = kSmem ? smat : Lg;
  if (kSmem) {
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) L[q] = Lg[q];
    __syncthreads();
  }
  __shared__ double red[32];
  __shared__ double s_piv;
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      double acc = 0.0;
      for (int k = lane; k < j; k += 32) acc += L[(long long)j * n + k] * L[(long long)j * n + k];
      acc = warp_sum(acc);
      if (lane == 0) {
      const double dj = L[(long long)j * n + j] - acc;
      if (!(dj > 0.0) || !isfinite(dj)) {
        s_fail = 1;
        set_status(status, XLS_ENOTSPD, blockIdx.x);
        s_piv = 1.0;
      } else {
        s_piv = sqrt(dj);
      }
      L[(long long)j * n + j] = s_piv;
      }
    }
    __syncthreads();
    if (s_fail) return;
    const double piv = s_piv;
    for (int i = j + 1 + warp; i < n; i += nwarp) {
      double a = 0.0;
      for (int k = lane; k < j; k += 32) a += L[(long long)i * n + k] * L[(long long)j * n + k];
      a = warp_sum(a);
      if (lane == 0) L[(long long)i * n + j] = (L[(long long)i * n + j] - a) / piv;
    }
    __syncthreads();
  }
  // clear the strict upper triangle
  for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) {
    const int i = (int)(q / n), k = (int)(q % n);
    Lg[q] = (k > i) ? 0.0 : L[q];
  }
}

// ---- 2./6. triangular solves, one warp per right-hand-side column --------------------------
// lower:  X = L^-1 B  (B[i][c] = trans ? Bm[c][i] : Bm[i][c]);  upper: X = L^-T B.
// Lane l keeps the solution entries x_k with k = l (mod 32) in registers; entry i is finished by
// its owner lane after a warp-wide dot product over the already known entries.
template <bool kUpper, int kTrsmRegs>
__global__ void __launch_bounds__(256)
k_trsm(const SubDev* __restrict__ subs, const double* __restrict__ Lm, const double* Bm, int trans, double* Xm) {
  const SubDev& S = subs[blockIdx.y];
  const int n = S.ns;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= n) return;
  const double* L = Lm + S.off_ss;
  const double* B = Bm + S.off_ss;
  double* X = Xm + S.off_ss;
  double xr[kTrsmRegs];
#pragma unroll
  for (int q = 0; q < kTrsmRegs; ++q) xr[q] = 0.0;
  if (!kUpper) {
    for (int i = 0; i < n; ++i) {
      const double* Li = L + (long long)i * n;
      double part = 0.0;
#pragma unroll
      for (int q = 0; q < kTrsmRegs; ++q) {
        const int k = q * 32 + lane;
        if (q * 32 < i && k < i) part += Li[k] * xr[q];
      }
      part = warp_sum(part);
      double x = 0.0;
      if (lane == (i & 31)) {
        const double b = trans ? B[(long long)c * n + i] : B[(long long)i * n + c];
        x = (b - part) / Li[i];
        X[(long long)i * n + c] = x;
      }
      x = __shfl_sync(0xffffffffu, x, i & 31);
      const bool own = (lane == (i & 31));
#pragma unroll
      for (int q = 0; q < kTrsmRegs; ++q) xr[q] = (own && q == (i >> 5)) ? x : xr[q];
    }
  } else {
    for (int i = n - 1; i >= 0; --i) {
      double part = 0.0;
#pragma unroll
      for (int q = 0; q < kTrsmRegs; ++q) {
        const int k = q * 32 + lane;
        if (q * 32 + 31 > i && k > i && k < n) part += L[(long long)k * n + i] * xr[q];
      }
      part = warp_sum(part);
      double x = 0.0;
      if (lane == (i & 31)) {
        x = (B[(long long)i * n + c] - part) / L[(long long)i * n + i];
        X[(long long)i * n + c] = x;
      }
      x = __shfl_sync(0xffffffffu, x, i & 31);
      const bool own = (lane == (i & 31));
#pragma unroll
      for (int q = 0; q < kTrsmRegs; ++q) xr[q] = (own && q == (i >> 5)) ? x : xr[q];
    }
  }
}

// ---- 3. Householder tridiagonalisation of A (lower, reflectors kept below the subdiagonal) -
// vec layout (8n per subdomain): d[0..n), e[n..2n), tau[2n..3n), lam32[3n..4n), cluster[4n..5n)
template <bool kSmem>
__global__ void __launch_bounds__(512) k_tridiag(const SubDev* __restrict__ subs, double* Am, double* vecs, int max_ns) {
  const SubDev& S = subs[blockIdx.x];
  const int n = S.ns;
  double* Ag = Am + S.off_ss;
  double* d = vecs + 8LL * S.off_state;
  double* e = d + n;
  double* tau = d + 2 * n;
  extern __shared__ double sm[];
  double* sv = sm;          // reflector v (length <= n)
  double* sw = sm + max_ns; // p, then w
  double* A = kSmem ? sm + 2 * max_ns : Ag;
  if (kSmem) {
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) A[q] = Ag[q];
    __syncthreads();
  }
  __shared__ double red[32];
  __shared__ double s_tau, s_K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  // symmetrise
  for (int i = warp; i < n; i += nwarp)
    for (int k = i + 1 + lane; k < n; k += 32) {
      const double m = 0.5 * (A[(long long)i * n + k] + A[(long long)k * n + i]);
      A[(long long)i * n + k] = m;
      A[(long long)k * n + i] = m;
    }
  __syncthreads();
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;
    double acc = 0.0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) {
      const double x = A[(long long)(k + 1 + i) * n + k];
      acc += x * x;
    }
    const double xn2 = block_sum_d(acc, red);
    const double alpha = A[(long long)(k + 1) * n + k];
    double beta, t, scal;
    if (xn2 == 0.0) {
      t = 0.0;
      beta = alpha;
      scal = 0.0;
    } else {
      beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
      t = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double v = (i == 0) ? 1.0 : A[(long long)(k + 1 + i) * n + k] * scal;
      sv[i] = v;
      if (i > 0) A[(long long)(k + 1 + i) * n + k] = v;
    }
    if (threadIdx.x == 0) {
      e[k] = beta;
      tau[k] = t;
      d[k] = A[(long long)k * n + k];
      s_tau = t;
    }
    __syncthreads();
    if (s_tau != 0.0) {
      // p = tau A22 v
      for (int i = warp; i < m; i += nwarp) {
        const double* row = A + (long long)(k + 1 + i) * n + (k + 1);
        double a = 0.0;
        for (int j = lane; j < m; j += 32) a += row[j] * sv[j];
        a = warp_sum(a);
        if (lane == 0) sw[i] = s_tau * a;
      }
      __syncthreads();
      double pv = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) pv += sw[i] * sv[i];
      pv = block_sum_d(pv, red);
      if (threadIdx.x == 0) s_K = 0.5 * s_tau * pv;
      __syncthreads();
      const double K = s_K;
      for (int i = threadIdx.x; i < m; i += blockDim.x) sw[i] -= K * sv[i];
      __syncthreads();
      for (int i = warp; i < m; i += nwarp) {
        double* row = A + (long long)(k + 1 + i) * n + (k + 1);
        const double vi = sv[i], wi = sw[i];
        for (int j = lane; j < m; j += 32) row[j] -= vi * sw[j] + wi * sv[j];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    d[n - 1] = A[(long long)(n - 1) * n + (n - 1)];
    e[n - 1] = 0.0;
    tau[n - 1] = 0.0;
  }
  if (kSmem) {  // reflectors (below the subdiagonal) back to global memory for the back-transformation
    __syncthreads();
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) {
      const int i = (int)(q / n), k = (int)(q % n);
      if (i > k + 1) Ag[q] = A[q];
    }
  }
}

// ---- 4. eigenpairs of the tridiagonal T ----------------------------------------------------
__device__ __forceinline__ int sturm_count_f(const float* d, const float* e2, int n, float x, float pivmin) {
  int cnt = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  if (q < 0.f) ++cnt;
  for (int j = 1; j < n; ++j) {
    q = d[j] - x - e2[j - 1] / q;
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++cnt;
  }
  return cnt;
}

__device__ __forceinline__ double hash_unit(unsigned a, unsigned b) {
  unsigned h = a * 2654435761u ^ (b * 40503u + 0x9E3779B9u);
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (double)(h & 0xFFFFFFu) * (1.0 / 16777216.0) - 0.5;
}

// Eigenpairs of T.  Shifts: FP32 Sturm bisection per index.  Vectors: FP64 inverse iteration
// with an LDL^T factorisation of T - sigma I (tiny pivots replaced by +-1e-15 |T|), one
// thread per cluster of close eigenvalues; members of a cluster are Gram-Schmidt-orthogonalised
// against the earlier ones at every iteration and finally Rayleigh-Ritz-rotated inside the
// cluster (Jacobi on the k x k projected T).  Per-thread work arrays are interleaved across the
// threads of the block (element j of thread t at [j * blockDim + t]) so that the warps' accesses
// coalesce.
constexpr int kTriThreads = 128;

// (a) shifts: FP32 Sturm bisection for every eigenvalue index; clusters of close eigenvalues.
// vecs per subdomain: d [0,n), e [n,2n), tau [2n,3n), lam32 [3n,4n), cluster starts [4n,5n] (as doubles),
// [5n+1] cluster count, [5n+2] |T| estimate.
__global__ void __launch_bounds__(1024)
k_tri_bisect(const SubDev* __restrict__ subs, double* vecs) {
  const SubDev& S = subs[blockIdx.x];
  const int n = S.ns;
  double* d = vecs + 8LL * S.off_state;
  double* e = d + n;
  double* lam32 = d + 3 * n;
  extern __shared__ float smf[];
  float* df = smf;
  float* e2f = smf + n;
  __shared__ float s_gl, s_gu, s_pivmin;
  __shared__ double s_tnorm;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    df[i] = (float)d[i];
    e2f[i] = (float)(e[i] * e[i]);
  }
  __syncthreads();
  // Gershgorin bounds: per-thread extrema over a strided share of the rows, then warp shuffles
  // and one pass over the warps' results (no serial loop over n on one thread)
  __shared__ double s_ext[3][32];
  {
    double gl = 1e300, gu = -1e300, emax2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
      gl = fmin(gl, d[i] - r);
      gu = fmax(gu, d[i] + r);
      if (i + 1 < n) emax2 = fmax(emax2, e[i] * e[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
      gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
      emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
    }
    if ((threadIdx.x & 31) == 0) {
      s_ext[0][threadIdx.x >> 5] = gl;
      s_ext[1][threadIdx.x >> 5] = gu;
      s_ext[2][threadIdx.x >> 5] = emax2;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double gl = 1e300, gu = -1e300, emax2 = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) {
      gl = fmin(gl, s_ext[0][w]);
      gu = fmax(gu, s_ext[1][w]);
      emax2 = fmax(emax2, s_ext[2][w]);
    }
    const double tn = fmax(fabs(gl), fabs(gu));
    s_tnorm = tn > 0 ? tn : 1.0;
    s_gl = (float)(gl - 1e-5 * s_tnorm - 1e-30);
    s_gu = (float)(gu + 1e-5 * s_tnorm + 1e-30);
    s_pivmin = (float)fmax(1e-30, 1e-30 * emax2);
  }
  __syncthreads();
  // multisection: four threads per eigenvalue index evaluate the counts at the three quarter
  // points of its interval (and one spare), the interval shrinks to the quarter where the count
  // passes the index (two bits per round)
  const int sub = threadIdx.x & 3;
  const unsigned gmask = 0xFu << (threadIdx.x & 28);   // the four lanes of this group
  const int groups = blockDim.x >> 2;
  for (int i = blockIdx.y * groups + (threadIdx.x >> 2); i < n; i += groups * gridDim.y) {  // uniform inside a group
    float lo = s_gl, hi = s_gu;
    for (int it = 0; it < 26; ++it) {
      const float w = hi - lo;
      const float pt = lo + 0.25f * (float)(sub + 1) * w;      // sub = 3: the upper end (count known)
      const int cnt = sub < 3 ? sturm_count_f(df, e2f, n, pt, s_pivmin) : 0x7fffffff;
      // first quarter point whose count exceeds i
      const int c1 = __shfl_sync(gmask, cnt, 0, 4), c2 = __shfl_sync(gmask, cnt, 1, 4),
                c3 = __shfl_sync(gmask, cnt, 2, 4);
      const int q = c1 > i ? 0 : (c2 > i ? 1 : (c3 > i ? 2 : 3));
      const float nlo = q == 0 ? lo : lo + 0.25f * (float)q * w;
      const float nhi = q == 3 ? hi : lo + 0.25f * (float)(q + 1) * w;
      if (!(nlo > lo || nhi < hi) || nlo >= nhi) break;   // no longer divisible in FP32 (uniform per group)
      lo = nlo;
      hi = nhi;
    }
    if (sub == 0) lam32[i] = 0.5 * ((double)lo + (double)hi);
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) d[5 * n + 2] = s_tnorm;
}

// clusters of the bisection estimates (after all of them are in): runs of eigenvalues closer than
// 1e-4 ||T|| are one cluster, solved together by one thread of the vector stage
__global__ void k_tri_clusters(const SubDev* __restrict__ subs, double* vecs) {
  const SubDev& S = subs[blockIdx.x];
  const int n = S.ns;
  double* d = vecs + 8LL * S.off_state;
  const double* lam32 = d + 3 * n;
  double* cst = d + 4 * n;
  // one warp: 32 indices at a time, the cluster starts compacted by ballot and prefix count
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double ctol = 1e-4 * d[5 * n + 2];
    int c = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int i = i0 + lane;
      const bool start = i < n && (i == 0 || lam32[i] - lam32[i - 1] > ctol);
      const unsigned m = __ballot_sync(0xffffffffu, start);
      if (start) cst[c + __popc(m & ((1u << lane) - 1u))] = (double)i;
      c += __popc(m);
    }
    if (lane == 0) {
      cst[c] = (double)n;
      d[5 * n + 1] = (double)c;
    }
  }
}

// (b) vectors: CTA (subdomain, group) handles the clusters c = group * blockDim + t (stride
// gridDim.y * blockDim).  kSmemWork: per-thread work arrays in shared memory, else in the
// interleaved global scratch.
//
// Attempt 0 (fast): two FP32 inverse iterations with an unpivoted LDL^T of T - sigma I, then FP64
// iterations from that vector (singletons with Rayleigh-quotient shifts).  Every cluster is then
// checked: each member's Ritz value must lie within 1e-5 |T| of the cluster's bisection range and
// its residual |T z - lambda z| stay below 1e-9 |T|.  An unpivoted factorisation can lose the
// iterate when a tiny pivot falls inside the recurrence (the iterate then drifts to another
// eigenpair, or is noise); a cluster that fails the check is recomputed (attempt 1) in FP64 with
// Gaussian elimination with partial pivoting of T - sigma I (backward stable for tridiagonal
// matrices), the bisection shifts held fixed for two iterations before a guarded
// Rayleigh-quotient step.
template <bool kSmemWork>
__global__ void __launch_bounds__(kTriThreads)
k_tri_eig(const SubDev* __restrict__ subs, double* vecs, double* Zm, double* scratch_all, long long scr_stride,
          double* Rm, double* lam_out, int max_ns) {
  const SubDev& S = subs[blockIdx.x];
  const int n = S.ns;
  double* d = vecs + 8LL * S.off_state;
  double* e = d + n;
  double* lam32 = d + 3 * n;
  const double* cst = d + 4 * n;
  double* Z = Zm + S.off_ss;
  double* Rb = Rm + S.off_ss;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ncl = (int)d[5 * n + 1];
  const double tnorm = d[5 * n + 2];
  const int T = blockDim.x, t = threadIdx.x;
  double* scr;
  if (kSmemWork) {
    scr = reinterpret_cast<double*>(smraw);
  } else {
    scr = scratch_all + ((long long)blockIdx.x * gridDim.y + blockIdx.y) * scr_stride;
  }
  // interleaved arrays: lm (n), dinv (n), x (n), u2 (n); the pivoted solve keeps U's diagonal
  // in dinv, its first and second superdiagonals in lm and u2
  auto LM = [&](int j) -> double& { return scr[(long long)j * T + t]; };
  auto DI = [&](int j) -> double& { return scr[(long long)(n + j) * T + t]; };
  auto X = [&](int j) -> double& { return scr[(long long)(2 * n + j) * T + t]; };
  auto U2 = [&](int j) -> double& { return scr[(long long)(3 * n + j) * T + t]; };
  const double tiny = 1e-15 * tnorm;
  // Rayleigh quotient x^T T x / x^T x of the work vector
  auto rayleigh = [&]() -> double {
    double rq = 0.0, xx = 0.0, xm = 0.0, x0 = X(0);
    for (int j = 0; j < n; ++j) {
      const double xp = (j + 1 < n) ? X(j + 1) : 0.0;
      double tx = d[j] * x0 + (j + 1 < n ? e[j] * xp : 0.0);
      if (j > 0) tx += e[j - 1] * xm;
      rq += x0 * tx;
      xx += x0 * x0;
      xm = x0;
      x0 = xp;
    }
    return rq / xx;
  };
  // scale by the largest entry (the solves grow entries far beyond the square root of the
  // range), orthogonalise against the cluster's earlier members, normalise
  auto finish_iterate = [&](int s, int mbr) {
    double amax = 0.0;
    for (int j = 0; j < n; ++j) amax = fmax(amax, fabs(X(j)));
    if (!(amax > 0.0) || !isfinite(amax)) {   // restart from a fresh vector
      for (int j = 0; j < n; ++j) X(j) = hash_unit((unsigned)mbr + 7u, (unsigned)j + 1u);
      amax = 1.0;
    }
    const double asc = 1.0 / amax;
    for (int j = 0; j < n; ++j) X(j) *= asc;
    for (int pass = 0; pass < 2; ++pass)
      for (int q = s; q < mbr; ++q) {
        double dot = 0.0;
        for (int j = 0; j < n; ++j) dot += Z[(long long)j * n + q] * X(j);
        for (int j = 0; j < n; ++j) X(j) -= dot * Z[(long long)j * n + q];
      }
    double nrm = 0.0;
    for (int j = 0; j < n; ++j) nrm += X(j) * X(j);
    nrm = 1.0 / sqrt(nrm);
    for (int j = 0; j < n; ++j) X(j) *= nrm;
  };
  for (int c = blockIdx.y * T + t; c < ncl; c += gridDim.y * T) {
    const int s = (int)cst[c], tt = (int)cst[c + 1];
    const int k = tt - s;
    for (int attempt = 0; attempt < 2; ++attempt) {
      for (int mbr = s; mbr < tt; ++mbr) {
        double sigma = lam32[mbr];
        if (attempt == 0) {
          // ---- fast path: two FP32 iterations (FP32 latency on the dependent chains), then FP64
          bool ok32 = true;
          {
            // FP32 arrays: element jj of this thread in the low half of the thread's own FP64 slot
            // of the same array (an FP32 view indexed like the FP64 one would give each float an
            // address inside another thread's FP64 slots, and the threads run their FP32 and FP64
            // phases at different times)
            float* fs = reinterpret_cast<float*>(scr);
            auto LMf = [&](int jj) -> float& { return fs[2 * ((long long)jj * T + t)]; };
            auto DIf = [&](int jj) -> float& { return fs[2 * ((long long)(n + jj) * T + t)]; };
            auto Xf = [&](int jj) -> float& { return fs[2 * ((long long)(2 * n + jj) * T + t)]; };
            const float tiny_f = (float)fmax(1e-7 * tnorm, 1e-30);   // FP32 rounding level of the shift
            float sig_f = (float)sigma;
            for (int jj = 0; jj < n; ++jj) Xf(jj) = (float)hash_unit((unsigned)mbr + 1u, (unsigned)jj);
            for (int iter = 0; iter < 2; ++iter) {
              if (iter == 0 || k == 1) {
                float dp = (float)d[0] - sig_f;
                if (fabsf(dp) < tiny_f) dp = dp < 0.f ? -tiny_f : tiny_f;
                DIf(0) = 1.f / dp;
                for (int jj = 1; jj < n; ++jj) {
                  const float ej = (float)e[jj - 1];
                  const float l = ej * DIf(jj - 1);
                  LMf(jj - 1) = l;
                  dp = ((float)d[jj] - sig_f) - l * ej;
                  if (fabsf(dp) < tiny_f) dp = dp < 0.f ? -tiny_f : tiny_f;
                  DIf(jj) = 1.f / dp;
                }
              }
              float yv = Xf(0);
              Xf(0) = yv * DIf(0);
              for (int jj = 1; jj < n; ++jj) {
                yv = Xf(jj) - LMf(jj - 1) * yv;
                Xf(jj) = yv * DIf(jj);
              }
              float xn = Xf(n - 1);
              for (int jj = n - 2; jj >= 0; --jj) {
                xn = Xf(jj) - LMf(jj) * xn;
                Xf(jj) = xn;
              }
              float amax = 0.f;
              for (int jj = 0; jj < n; ++jj) amax = fmaxf(amax, fabsf(Xf(jj)));
              if (!(amax > 0.f) || isinf(amax) || isnan(amax)) {   // FP32 range exceeded
                ok32 = false;
                break;
              }
              const float asc = 1.f / amax;
              for (int jj = 0; jj < n; ++jj) Xf(jj) *= asc;
              for (int pass = 0; pass < 2; ++pass)
                for (int q = s; q < mbr; ++q) {
                  float dot = 0.f;
                  for (int jj = 0; jj < n; ++jj) dot += (float)Z[(long long)jj * n + q] * Xf(jj);
                  for (int jj = 0; jj < n; ++jj) Xf(jj) -= dot * (float)Z[(long long)jj * n + q];
                }
              float nrm = 0.f;
              for (int jj = 0; jj < n; ++jj) nrm += Xf(jj) * Xf(jj);
              if (!(nrm > 0.f) || isinf(nrm)) {
                ok32 = false;
                break;
              }
              nrm = rsqrtf(nrm);
              for (int jj = 0; jj < n; ++jj) Xf(jj) *= nrm;
              if (k == 1) {
                float rq = 0.f, xm = 0.f, x0 = Xf(0);
                for (int jj = 0; jj < n; ++jj) {
                  const float xp = (jj + 1 < n) ? Xf(jj + 1) : 0.f;
                  float tx = (float)d[jj] * x0 + (jj + 1 < n ? (float)e[jj] * xp : 0.f);
                  if (jj > 0) tx += (float)e[jj - 1] * xm;
                  rq += x0 * tx;
                  xm = x0;
                  x0 = xp;
                }
                sig_f = rq;
              }
            }
            for (int jj = 0; jj < n; ++jj) X(jj) = (double)Xf(jj);   // Xf(jj) is read before its slot is written
          }
          int it0 = 2;
          if (!ok32) {
            for (int j = 0; j < n; ++j) X(j) = hash_unit((unsigned)mbr + 1u, (unsigned)j);
            it0 = 0;
          } else if (k == 1) {
            sigma = rayleigh();   // FP64 Rayleigh quotient of the FP32 vector
          }
          // members of a cluster take a second FP64 iteration: their shifts are the FP32
          // bisection values
          const int iters = k == 1 ? 3 : 4;
          for (int iter = it0; iter < iters; ++iter) {
            if (iter == it0 || k == 1) {
              double dp = d[0] - sigma;  // LDL^T of T - sigma I
              if (fabs(dp) < tiny) dp = dp < 0 ? -tiny : tiny;
              DI(0) = 1.0 / dp;
              for (int j = 1; j < n; ++j) {
                const double l = e[j - 1] * DI(j - 1);   // e / dp through the reciprocal already formed
                LM(j - 1) = l;
                dp = (d[j] - sigma) - l * e[j - 1];
                if (fabs(dp) < tiny) dp = dp < 0 ? -tiny : tiny;
                DI(j) = 1.0 / dp;
              }
            }
            double y = X(0);                      // forward: L y = b (in place), then z = D^-1 y
            X(0) = y * DI(0);
            for (int j = 1; j < n; ++j) {
              y = X(j) - LM(j - 1) * y;
              X(j) = y * DI(j);
            }
            double xn = X(n - 1);                 // back: L^T x = z
            for (int j = n - 2; j >= 0; --j) {
              xn = X(j) - LM(j) * xn;
              X(j) = xn;
            }
            finish_iterate(s, mbr);
            if (k == 1 && iter < 2) sigma = rayleigh();
          }
        } else {
          // ---- robust path: FP64 Gaussian elimination with partial pivoting of T - sigma I,
          // the factorisation and the forward substitution in one sweep (U: diagonal in DI, first
          // and second superdiagonals in LM and U2), then back substitution
          for (int j = 0; j < n; ++j) X(j) = hash_unit((unsigned)mbr + 3u, (unsigned)j);
          for (int iter = 0; iter < 3; ++iter) {
            if (k == 1 && iter == 2) {   // guarded Rayleigh-quotient shift of a singleton
              const double rq = rayleigh();
              if (fabs(rq - lam32[mbr]) <= 1e-5 * tnorm) sigma = rq;
            }
            double ak = d[0] - sigma, bk = (n > 1) ? e[0] : 0.0, yk = X(0);
            for (int j = 0; j + 1 < n; ++j) {
              const double cj = e[j];
              const double ak1 = d[j + 1] - sigma, bk1 = (j + 2 < n) ? e[j + 1] : 0.0, yk1 = X(j + 1);
              if (fabs(ak) >= fabs(cj)) {   // no interchange
                const double m = ak != 0.0 ? cj / ak : 0.0;
                DI(j) = ak;
                LM(j) = bk;
                U2(j) = 0.0;
                X(j) = yk;
                ak = ak1 - m * bk;
                bk = bk1;
                yk = yk1 - m * yk;
              } else {                      // rows j and j + 1 interchanged
                const double m = ak / cj;
                DI(j) = cj;
                LM(j) = ak1;
                U2(j) = bk1;
                X(j) = yk1;
                ak = bk - m * ak1;
                bk = -m * bk1;
                yk = yk - m * yk1;
              }
            }
            DI(n - 1) = ak;
            X(n - 1) = yk;
            for (int j = n - 1; j >= 0; --j) {
              double u = DI(j);
              if (fabs(u) < tiny) u = u < 0.0 ? -tiny : tiny;
              double r = X(j);
              if (j + 1 < n) r -= LM(j) * X(j + 1);
              if (j + 2 < n) r -= U2(j) * X(j + 2);
              X(j) = r / u;
            }
            finish_iterate(s, mbr);
          }
        }
        for (int j = 0; j < n; ++j) Z[(long long)j * n + mbr] = X(j);
      }
      // Rayleigh-Ritz inside the cluster, in pieces of at most 64 members (a longer run of close
      // eigenvalues is cut at its largest gaps; its vectors are orthogonal across the whole run)
      for (int ps = s; ps < tt;) {
        int pt = tt;
        if (tt - ps > 64) {
          double best = -1.0;
          for (int p = ps + 16; p <= ps + 64; ++p)
            if (lam32[p] - lam32[p - 1] > best) {
              best = lam32[p] - lam32[p - 1];
              pt = p;
            }
        }
        const int kp = pt - ps, sp = ps;
        ps = pt;
        double* Sm = Rb + (long long)sp * n;
        double* Rr = Sm + (long long)kp * kp;
        const bool fits = (2LL * kp * kp <= (long long)kp * n) && kp <= 64;
        if (kp == 1 || !fits) {
          for (int mbr = sp; mbr < pt; ++mbr) {
            double rq = 0.0;
            for (int j = 0; j < n; ++j) {
              double tx = d[j] * Z[(long long)j * n + mbr];
              if (j > 0) tx += e[j - 1] * Z[(long long)(j - 1) * n + mbr];
              if (j + 1 < n) tx += e[j] * Z[(long long)(j + 1) * n + mbr];
              rq += Z[(long long)j * n + mbr] * tx;
            }
            lam_out[S.off_state + mbr] = rq;
          }
          continue;
        }
        for (int a = 0; a < kp; ++a)
          for (int b = a; b < kp; ++b) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) {
              double tx = d[j] * Z[(long long)j * n + sp + b];
              if (j > 0) tx += e[j - 1] * Z[(long long)(j - 1) * n + sp + b];
              if (j + 1 < n) tx += e[j] * Z[(long long)(j + 1) * n + sp + b];
              acc += Z[(long long)j * n + sp + a] * tx;
            }
            Sm[a * kp + b] = acc;
            Sm[b * kp + a] = acc;
          }
        for (int a = 0; a < kp; ++a)
          for (int b = 0; b < kp; ++b) Rr[a * kp + b] = (a == b) ? 1.0 : 0.0;
        for (int sweep = 0; sweep < 30; ++sweep) {
          double off = 0.0, tot = 0.0;
          for (int a = 0; a < kp; ++a)
            for (int b = 0; b < kp; ++b) {
              tot += Sm[a * kp + b] * Sm[a * kp + b];
              if (a != b) off += Sm[a * kp + b] * Sm[a * kp + b];
            }
          if (off <= 1e-30 * tot || off == 0.0) break;
          for (int p = 0; p < kp - 1; ++p)
            for (int q = p + 1; q < kp; ++q) {
              const double apq = Sm[p * kp + q];
              if (apq == 0.0) continue;
              const double theta = (Sm[q * kp + q] - Sm[p * kp + p]) / (2.0 * apq);
              const double tq = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
              const double cs = 1.0 / sqrt(tq * tq + 1.0), sn = tq * cs;
              for (int r = 0; r < kp; ++r) {
                const double a1 = Sm[r * kp + p], a2 = Sm[r * kp + q];
                Sm[r * kp + p] = cs * a1 - sn * a2;
                Sm[r * kp + q] = sn * a1 + cs * a2;
              }
              for (int r = 0; r < kp; ++r) {
                const double a1 = Sm[p * kp + r], a2 = Sm[q * kp + r];
                Sm[p * kp + r] = cs * a1 - sn * a2;
                Sm[q * kp + r] = sn * a1 + cs * a2;
              }
              for (int r = 0; r < kp; ++r) {
                const double rp = Rr[r * kp + p], rq = Rr[r * kp + q];
                Rr[r * kp + p] = cs * rp - sn * rq;
                Rr[r * kp + q] = sn * rp + cs * rq;
              }
            }
        }
        int order[64];
        for (int a = 0; a < kp; ++a) order[a] = a;
        for (int a = 0; a < kp; ++a)
          for (int b = a + 1; b < kp; ++b)
            if (Sm[order[b] * kp + order[b]] < Sm[order[a] * kp + order[a]]) {
              const int tmp = order[a];
              order[a] = order[b];
              order[b] = tmp;
            }
        for (int j = 0; j < n; ++j) {
          double row[64];
          for (int b = 0; b < kp; ++b) {
            double acc = 0.0;
            for (int a = 0; a < kp; ++a) acc += Z[(long long)j * n + sp + a] * Rr[a * kp + order[b]];
            row[b] = acc;
          }
          for (int b = 0; b < kp; ++b) Z[(long long)j * n + sp + b] = row[b];
        }
        for (int b = 0; b < kp; ++b) lam_out[S.off_state + sp + b] = Sm[order[b] * kp + order[b]];
      }
      // check of the cluster: Ritz values within the bisection range, small residuals
      bool ok = true;
      const double lo = lam32[s] - 1e-5 * tnorm, hi = lam32[tt - 1] + 1e-5 * tnorm;
      for (int mbr = s; mbr < tt && ok; ++mbr) {
        const double lm = lam_out[S.off_state + mbr];
        if (!(lm >= lo && lm <= hi)) {
          ok = false;
          break;
        }
        double r2 = 0.0;
        for (int j = 0; j < n; ++j) {
          double tx = (d[j] - lm) * Z[(long long)j * n + mbr];
          if (j > 0) tx += e[j - 1] * Z[(long long)(j - 1) * n + mbr];
          if (j + 1 < n) tx += e[j] * Z[(long long)(j + 1) * n + mbr];
          r2 += tx * tx;
        }
        if (!(sqrt(r2) <= 1e-9 * tnorm)) ok = false;
      }
      if (ok) break;
    }
  }
}

// ---- 5. back-transformation Z = Q Z_T, Q = H_0 H_1 ... H_{n-2} --------------------------
__global__ void __launch_bounds__(256)
k_backtransform(const SubDev* __restrict__ subs, const double* __restrict__ Am, const double* __restrict__ vecs,
                double* Zm) {
  const SubDev& S = subs[blockIdx.y];
  const int n = S.ns;
  const int c0 = blockIdx.x * 32;
  if (c0 >= n) return;
  const double* A = Am + S.off_ss;
  const double* tau = vecs + 8LL * S.off_state + 2 * n;
  double* Z = Zm + S.off_ss;
  extern __shared__ double sm[];
  double* v = sm;              // n
  double* part = sm + n;       // 8 x 32
  const int col = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int c = c0 + col;
  for (int k = n - 2; k >= 0; --k) {
    const double t = tau[k];
    if (t == 0.0) continue;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) v[i] = (i == k + 1) ? 1.0 : A[(long long)i * n + k];
    __syncthreads();
    double acc = 0.0;
    if (c < n)
      for (int i = k + 1 + rg; i < n; i += 8) acc += v[i] * Z[(long long)i * n + c];
    part[rg * 32 + col] = acc;
    __syncthreads();
    double dot = 0.0;
#pragma unroll
    for (int r = 0; r < 8; ++r) dot += part[r * 32 + col];
    if (c < n)
      for (int i = k + 1 + rg; i < n; i += 8) Z[(long long)i * n + c] -= t * v[i] * dot;
    __syncthreads();
  }
}

// Same back-transformation with everything it touches in shared memory and one warp per column:
// a CTA takes 8 columns of Z (8 warps), stages all n - 1 reflectors (the strict lower triangle
// of the reduced matrix, packed by columns) and tau, and each warp applies the reflectors to its
// column with lane-strided rows and a shuffle reduction, without block barriers.  Global memory
// is read once at the start and Z written once at the end; the n / 8 CTAs per subdomain spread
// the FP64 work over the SMs.
constexpr int kBtCols = 8;

__host__ __device__ inline long long bt_col_off(int k, int n) { return (long long)k * (n - 1) - (long long)k * (k - 1) / 2; }

size_t backtransform_sm_bytes(int n) {
  return ((size_t)kBtCols * n + (size_t)n * (n - 1) / 2 + (size_t)n) * sizeof(double);
}

__global__ void __launch_bounds__(kBtCols * 32)
k_backtransform_sm(const SubDev* __restrict__ subs, const double* __restrict__ Am, const double* __restrict__ vecs,
                   double* Zm) {
  const SubDev& S = subs[blockIdx.y];
  const int n = S.ns;
  const int c0 = blockIdx.x * kBtCols;
  if (c0 >= n) return;
  const double* A = Am + S.off_ss;
  const double* tau = vecs + 8LL * S.off_state + 2 * n;
  double* Z = Zm + S.off_ss;
  extern __shared__ double sm[];
  double* Zs = sm;                                        // [kBtCols][n]
  double* Vs = Zs + (size_t)kBtCols * n;                  // reflector k: entries i = k+1 .. n-1
  double* ts = Vs + (long long)n * (n - 1) / 2;           // tau
  for (int q = threadIdx.x; q < n * kBtCols; q += blockDim.x) {
    const int i = q / kBtCols, cc = q % kBtCols;
    Zs[cc * n + i] = (c0 + cc < n) ? Z[(long long)i * n + c0 + cc] : 0.0;
  }
  for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) {
    const int i = (int)(q / n), k = (int)(q - (long long)i * n);
    if (i > k) Vs[bt_col_off(k, n) + (i - k - 1)] = (i == k + 1) ? 1.0 : A[q];
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) ts[k] = tau[k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* z = Zs + warp * n;
  for (int k = n - 2; k >= 0; --k) {
    const double t = ts[k];
    if (t == 0.0) continue;
    const long long vo = bt_col_off(k, n) - (k + 1);   // entry i > k of reflector k at Vs[vo + i]
    double acc = 0.0;
    for (int i = k + 1 + lane; i < n; i += 32) acc += Vs[vo + i] * z[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const double td = t * acc;
    for (int i = k + 1 + lane; i < n; i += 32) z[i] -= td * Vs[vo + i];
    __syncwarp();
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n * kBtCols; q += blockDim.x) {
    const int i = q / kBtCols, cc = q % kBtCols;
    if (c0 + cc < n) Z[(long long)i * n + c0 + cc] = Zs[cc * n + i];
  }
}

// ---- 2./6. blocked triangular solves: CTA = (8 right-hand-side columns, subdomain) ----------
// lower: X = L^-1 B (B[i][c] = trans ? Bm[c][i] : Bm[i][c]); upper: X = L^-T B.  The 8 columns
// live in shared memory; rows are taken in blocks of 32: the block's diagonal part of L is staged
// in shared memory with the reciprocals of its diagonal, one warp per column solves it
// right-looking (lane = row: per unknown one multiply, one broadcast and one FMA, from shared
// memory only), and all warps subtract the block's contribution from the remaining rows.  The per-column kernel above (warp
// per column) remains for reference runs with XLS_EIG=single.
constexpr int kTrsmCols = 8, kTrsmRB = 32;

template <bool kUpper>
__global__ void __launch_bounds__(256)
k_trsm_blk(const SubDev* __restrict__ subs, const double* __restrict__ Lm, const double* Bm, int trans, double* Xm) {
  const SubDev& S = subs[blockIdx.y];
  const int n = S.ns;
  const int c0 = blockIdx.x * kTrsmCols;
  if (c0 >= n) return;
  const int nc = min(kTrsmCols, n - c0);
  const double* L = Lm + S.off_ss;
  const double* B = Bm + S.off_ss;
  double* X = Xm + S.off_ss;
  extern __shared__ double xs[];   // [n][kTrsmCols], then the diagonal block of L
  double* Ld = xs + (size_t)n * kTrsmCols;        // [kTrsmRB][kTrsmRB + 1]: (row, col) of the block
  double* dinv = Ld + kTrsmRB * (kTrsmRB + 1);    // reciprocals of its diagonal
  for (int q = threadIdx.x; q < n * kTrsmCols; q += blockDim.x) {
    const int i = q / kTrsmCols, c = q % kTrsmCols;
    xs[q] = c < nc ? (trans ? B[(long long)(c0 + c) * n + i] : B[(long long)i * n + c0 + c]) : 0.0;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (n + kTrsmRB - 1) / kTrsmRB;
  for (int bb = 0; bb < nblk; ++bb) {
    // rows of this block: lower from the top, upper from the bottom
    const int r0 = kUpper ? max(0, n - (bb + 1) * kTrsmRB) : bb * kTrsmRB;
    const int r1 = kUpper ? n - bb * kTrsmRB : min(n, r0 + kTrsmRB);
    const int m = r1 - r0;
    // the block's part of L in shared memory (all threads, coalesced), so that the sequential
    // diagonal solve below waits on shared memory only
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
      const int a = q / m, b = q % m;
      Ld[a * (kTrsmRB + 1) + b] = L[(long long)(r0 + a) * n + r0 + b];
    }
    __syncthreads();
    if (threadIdx.x < m) dinv[threadIdx.x] = 1.0 / Ld[threadIdx.x * (kTrsmRB + 2)];
    __syncthreads();
    {
      // warp c solves column c; lane l holds row l of the block and is updated as soon as each
      // unknown is known (right-looking), so every step is one multiply, one broadcast and one FMA
      const int c = warp;
      double xl = lane < m ? xs[(r0 + lane) * kTrsmCols + c] : 0.0;
      for (int t = 0; t < m; ++t) {
        const int il = kUpper ? m - 1 - t : t;    // row within the block
        const double xi = __shfl_sync(0xffffffffu, xl * dinv[il], il);
        if (lane == il) xl = xi;
        const bool pending = kUpper ? lane < il : (lane > il && lane < m);
        if (pending) xl -= (kUpper ? Ld[il * (kTrsmRB + 1) + lane] : Ld[lane * (kTrsmRB + 1) + il]) * xi;
      }
      if (lane < m) xs[(r0 + lane) * kTrsmCols + c] = xl;
    }
    __syncthreads();
    // remaining rows: lower r1..n-1, upper 0..r0-1
    const int u0 = kUpper ? 0 : r1, u1 = kUpper ? r0 : n;
    for (int q = threadIdx.x; q < (u1 - u0) * kTrsmCols; q += blockDim.x) {
      const int i = u0 + q / kTrsmCols, c = q % kTrsmCols;
      double acc = 0.0;
      if (!kUpper) {
        const double* Li = L + (long long)i * n;
        for (int k = r0; k < r1; ++k) acc += Li[k] * xs[k * kTrsmCols + c];
      } else {
        for (int k = r0; k < r1; ++k) acc += L[(long long)k * n + i] * xs[k * kTrsmCols + c];
      }
      xs[i * kTrsmCols + c] -= acc;
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < n * kTrsmCols; q += blockDim.x) {
    const int i = q / kTrsmCols, c = q % kTrsmCols;
    if (c < nc) X[(long long)i * n + c0 + c] = xs[q];
  }
}

template <int RC>
static void trsm_rc(bool upper, dim3 gt, const SubDev* d_subs, const double* L, const double* B, int trans, double* X,
                    cudaStream_t st) {
  if (upper) k_trsm<true, RC><<<gt, 256, 0, st>>>(d_subs, L, B, trans, X);
  else k_trsm<false, RC><<<gt, 256, 0, st>>>(d_subs, L, B, trans, X);
}
static void trsm(bool upper, int max_ns, dim3 gt, const SubDev* d_subs, const double* L, const double* B, int trans,
                 double* X, cudaStream_t st, bool blocked = true) {
  if (blocked) {
    dim3 g((max_ns + kTrsmCols - 1) / kTrsmCols, gt.y);
    const size_t smem = ((size_t)max_ns * kTrsmCols + kTrsmRB * (kTrsmRB + 1) + kTrsmRB) * sizeof(double);
    if (smem > 48 * 1024) {
      cudaFuncSetAttribute(k_trsm_blk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_trsm_blk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (upper) k_trsm_blk<true><<<g, 256, smem, st>>>(d_subs, L, B, trans, X);
    else k_trsm_blk<false><<<g, 256, smem, st>>>(d_subs, L, B, trans, X);
    return;
  }
  const int rc = (max_ns + 31) / 32;
  if (rc <= 2) trsm_rc<2>(upper, gt, d_subs, L, B, trans, X, st);
  else if (rc <= 4) trsm_rc<4>(upper, gt, d_subs, L, B, trans, X, st);
  else if (rc <= 8) trsm_rc<8>(upper, gt, d_subs, L, B, trans, X, st);
  else if (rc <= 16) trsm_rc<16>(upper, gt, d_subs, L, B, trans, X, st);
  else trsm_rc<32>(upper, gt, d_subs, L, B, trans, X, st);
}

// Dynamic shared memory for the matrix-resident variants: request exactly what a launch needs;
// if the device refuses (static + dynamic above its opt-in limit), use the global-memory variant.
template <typename K>
static bool smem_ok(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return true;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return false;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (bytes + fa.sharedSizeBytes > (size_t)optin) return false;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

void launch_eig(const SubDev* d_subs, int n_sub, int max_ns, double* Ms, double* Hs, double* Y, double* W, double* lam,
                double* vecs, int* status, double* scratch, double* R, int cluster, cudaStream_t st) {
  const size_t mat = (size_t)max_ns * max_ns * sizeof(double);
  const size_t vbytes = 2 * (size_t)max_ns * sizeof(double);
  // Cholesky and tridiagonalisation on a cluster of CTAs per subdomain; one CTA per subdomain
  // where the cluster variant cannot be launched, or when the caller asks for it (cluster = 0;
  // else the cluster size tried first, 8 or 16)
  if (cluster && launch_cholesky_cluster(d_subs, n_sub, max_ns, Ms, status, cluster, st)) {
  } else if (smem_ok(k_cholesky<true>, mat)) k_cholesky<true><<<n_sub, 512, mat, st>>>(d_subs, Ms, status);
  else k_cholesky<false><<<n_sub, 512, 0, st>>>(d_subs, Ms, status);
  dim3 gt((max_ns + 7) / 8, n_sub);   // 8 warps (columns) per CTA
  trsm(false, max_ns, gt, d_subs, Ms, Hs, 0, W, st, cluster != 0);   // W = L^-1 H_s
  trsm(false, max_ns, gt, d_subs, Ms, W, 1, Hs, st, cluster != 0);   // A = L^-1 W^T
  if (cluster && launch_tridiag_cluster(d_subs, n_sub, max_ns, Hs, vecs, cluster, st)) {
  } else if (smem_ok(k_tridiag<true>, mat + vbytes)) k_tridiag<true><<<n_sub, 512, mat + vbytes, st>>>(d_subs, Hs, vecs, max_ns);
  else k_tridiag<false><<<n_sub, 512, vbytes, st>>>(d_subs, Hs, vecs, max_ns);
  // 32 eigenvalue indices (128 threads) per CTA, spread over the SMs
  k_tri_bisect<<<dim3(n_sub, (max_ns + 31) / 32), 128, 2 * max_ns * sizeof(float), st>>>(d_subs, vecs);
  k_tri_clusters<<<n_sub, 32, 0, st>>>(d_subs, vecs);
  {
    // vector stage: 32 threads per CTA with shared-memory work arrays where they fit, one CTA per
    // 32 clusters of a subdomain; else 128 threads per CTA on the global scratch (8 threads per
    // CTA, spreading the clusters over more SMs, measured no faster: the longest cluster's
    // dependent FP64 chain sets the time)
    constexpr int kVecThreads = 32;
    const size_t per_thread = 4 * (size_t)max_ns * sizeof(double);
    const int groups = (max_ns + kVecThreads - 1) / kVecThreads;
    if (per_thread * kVecThreads <= 200 * 1024 && smem_ok(k_tri_eig<true>, per_thread * kVecThreads)) {
      dim3 gv(n_sub, groups);
      k_tri_eig<true><<<gv, kVecThreads, per_thread * kVecThreads, st>>>(d_subs, vecs, W, scratch, 0, R, lam, max_ns);
    } else {
      dim3 gv(n_sub, 1);
      k_tri_eig<false><<<gv, kTriThreads, 0, st>>>(d_subs, vecs, W, scratch, 4LL * max_ns * kTriThreads, R, lam,
                                                   max_ns);
    }
  }
  dim3 gb((max_ns + 31) / 32, n_sub);
  const size_t bt_smem = backtransform_sm_bytes(max_ns);
  if (bt_smem <= 200 * 1024 && smem_ok(k_backtransform_sm, bt_smem))
    k_backtransform_sm<<<dim3((max_ns + kBtCols - 1) / kBtCols, n_sub), kBtCols * 32, bt_smem, st>>>(d_subs, Hs, vecs,
                                                                                                   W);
  else
    k_backtransform<<<gb, 256, (max_ns + 256) * sizeof(double), st>>>(d_subs, Hs, vecs, W);
  trsm(true, max_ns, gt, d_subs, Ms, W, 0, Y, st, cluster != 0);     // Y = L^-T Z
}

size_t eig_scratch_doubles(int n_sub, int max_ns) { return (size_t)n_sub * kTriThreads * 4 * max_ns; }

}  // namespace xls
