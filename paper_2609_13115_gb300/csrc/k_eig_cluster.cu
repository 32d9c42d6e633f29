// Cholesky factorisation and Householder tridiagonalisation of one subdomain's N_s x N_s
// matrices on a thread-block cluster (Sec. 5.A.3 step (3)): the rows are distributed cyclically
// over the CL CTAs of the cluster (row i in CTA i % CL, local row i / CL) and kept in shared
// memory; vectors that every CTA needs are pushed into each CTA's copy through distributed shared
// memory, and the CTAs meet at cluster barriers.  Same arithmetic as k_cholesky / k_tridiag
// (k_eig.cu), which remain for blocks too large for the cluster's shared memory.
#include <cooperative_groups.h>

#include <cstdlib>

#include "xls_internal.h"

namespace cg = cooperative_groups;

namespace xls {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum with the result in every thread
__device__ double bsum(double v, double* red) {
  v = wsum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// ---- Cholesky M_s = L L^T, left-looking by columns ----------------------------------------
// shared memory: local rows [ceil(n / CL)][n], then the broadcast row j in two buffers [2][n]
__global__ void __launch_bounds__(256)
k_cholesky_cl(const SubDev* __restrict__ subs, double* Ms, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int a = blockIdx.x / CL;
  const SubDev& S = subs[a];
  const int n = S.ns;
  const int nloc = (n + CL - 1) / CL;
  double* G = Ms + S.off_ss;
  extern __shared__ __align__(16) double csm[];
  double* Lr = csm;                      // local rows
  double* rowb = csm + (size_t)nloc * n; // [2][n + 1]: row j of L, then a failure flag
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j < n; j += blockDim.x) Lr[(size_t)r * n + j] = G[(size_t)i * n + j];
  }
  cl.sync();
  for (int j = 0; j < n; ++j) {
    double* rb = rowb + (size_t)(j & 1) * (n + 1);
    if (j % CL == rank && warp == 0) {   // owner of row j: diagonal, then push row j to every CTA
      double* row = Lr + (size_t)(j / CL) * n;
      double acc = 0.0;
      for (int k = lane; k < j; k += 32) acc += row[k] * row[k];
      acc = wsum(acc);
      const double dj = row[j] - acc;
      const bool bad = !(dj > 0.0) || !isfinite(dj);
      if (lane == 0) {
        row[j] = bad ? 1.0 : sqrt(dj);
        if (bad && atomicCAS(status, 0, XLS_ENOTSPD) == 0) status[1] = a;
      }
      __syncwarp();
      for (int q = 0; q < CL; ++q) {
        double* dst = cl.map_shared_rank(rb, q);
        for (int k = lane; k <= j; k += 32) dst[k] = row[k];
        if (lane == 0) dst[n] = bad ? 1.0 : 0.0;
      }
    }
    cl.sync();
    if (rb[n] != 0.0) return;  // not positive definite: every CTA leaves after the same barrier
    const double piv = rb[j];
    for (int r = warp; r < nloc; r += nw) {
      const int i = r * CL + rank;
      if (i <= j || i >= n) continue;
      double* row = Lr + (size_t)r * n;
      double acc = 0.0;
      for (int k = lane; k < j; k += 32) acc += row[k] * rb[k];
      acc = wsum(acc);
      if (lane == 0) row[j] = (row[j] - acc) / piv;
    }
    __syncthreads();
  }
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j < n; j += blockDim.x) G[(size_t)i * n + j] = (j > i) ? 0.0 : Lr[(size_t)r * n + j];
  }
  cl.sync();
}

// Right-looking Cholesky on the same row distribution: per column j every CTA pushes the current
// entries A_ij of its own rows i >= j into every CTA; after the one cluster barrier every CTA forms
// the pivot sqrt(A_jj) and the scaled column L_kj = A_kj / L_jj (k > j) itself and applies the
// rank-1 update A_ik -= L_ij L_kj (j < k <= i) to its own rows -- element-parallel FP64 FMAs and
// no dot-product reductions on the critical path.  Buffers alternate with the column parity.
// shared memory: local rows [nloc][n], column buffers [2][n]
__global__ void __launch_bounds__(256)
k_cholesky_cl2(const SubDev* __restrict__ subs, double* Ms, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int a = blockIdx.x / CL;
  const SubDev& S = subs[a];
  const int n = S.ns;
  const int nloc = (n + CL - 1) / CL;
  double* G = Ms + S.off_ss;
  extern __shared__ __align__(16) double csm[];
  double* Lr = csm;                      // local rows
  double* colb = csm + (size_t)nloc * n; // [2][n]: column j of the working matrix, rows j..n-1
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j < n; j += blockDim.x) Lr[(size_t)r * n + j] = G[(size_t)i * n + j];
  }
  __syncthreads();
  bool failed = false;
  for (int j = 0; j < n; ++j) {
    double* cb = colb + (size_t)(j & 1) * n;
    // push column j of the own rows i >= j
    for (int r = threadIdx.x; r < nloc; r += blockDim.x) {
      const int i = r * CL + rank;
      if (i < j || i >= n) continue;
      const double x = Lr[(size_t)r * n + j];
      for (int q = 0; q < CL; ++q) cl.map_shared_rank(cb, q)[i] = x;
    }
    cl.sync();
    const double dj = cb[j];
    if (!(dj > 0.0) || !isfinite(dj)) {   // not positive definite: every CTA sees the same value
      if (rank == 0 && threadIdx.x == 0 && atomicCAS(status, 0, XLS_ENOTSPD) == 0) status[1] = a;
      failed = true;
      break;
    }
    const double piv = sqrt(dj), rinv = 1.0 / piv;
    // own rows: L_ij = A_ij / L_jj, then A_ik -= L_ij L_kj for j < k <= i (L_kj = cb[k] / L_jj)
    for (int r = warp; r < nloc; r += nw) {
      const int i = r * CL + rank;
      if (i < j || i >= n) continue;
      double* row = Lr + (size_t)r * n;
      if (i == j) {
        if (lane == 0) row[j] = piv;
        continue;
      }
      const double lij = cb[i] * rinv;
      const double f = lij * rinv;
      for (int k = j + 1 + lane; k <= i; k += 32) row[k] -= f * cb[k];
      if (lane == 0) row[j] = lij;
    }
    __syncthreads();
  }
  if (!failed)
    for (int r = 0; r < nloc; ++r) {
      const int i = r * CL + rank;
      if (i >= n) break;
      for (int j = threadIdx.x; j < n; j += blockDim.x) G[(size_t)i * n + j] = (j > i) ? 0.0 : Lr[(size_t)r * n + j];
    }
  cl.sync();
}

// ---- Householder tridiagonalisation (lower, reflectors below the subdiagonal) --------------
// shared memory: local rows [nloc][n], full v [n], full w [n], partial sums [4]
__global__ void __launch_bounds__(256)
k_tridiag_cl(const SubDev* __restrict__ subs, double* Am, double* vecs) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int a = blockIdx.x / CL;
  const SubDev& S = subs[a];
  const int n = S.ns;
  const int nloc = (n + CL - 1) / CL;
  double* Ag = Am + S.off_ss;
  double* d = vecs + 8LL * S.off_state;
  double* e = d + n;
  double* tau = d + 2 * n;
  extern __shared__ __align__(16) double tsm[];
  double* Ar = tsm;
  double* vf = Ar + (size_t)nloc * n;
  double* wf = vf + n;
  double* part = wf + n;                  // [0] |x|^2 partial, [1] alpha, [2] p.v partial
  __shared__ double red[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // local rows of the symmetrised matrix
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      Ar[(size_t)r * n + j] = 0.5 * (Ag[(size_t)i * n + j] + Ag[(size_t)j * n + i]);
  }
  cl.sync();
  for (int k = 0; k + 1 < n; ++k) {
    // (1) norm of the column below the subdiagonal and its first entry
    double acc = 0.0;
    for (int r = threadIdx.x; r < nloc; r += blockDim.x) {
      const int i = r * CL + rank;
      if (i >= k + 2 && i < n) {
        const double x = Ar[(size_t)r * n + k];
        acc += x * x;
      }
    }
    acc = bsum(acc, red);
    if (threadIdx.x == 0) {
      part[0] = acc;
      part[1] = ((k + 1) % CL == rank) ? Ar[(size_t)((k + 1) / CL) * n + k] : 0.0;
      if (k % CL == rank) d[k] = Ar[(size_t)(k / CL) * n + k];
    }
    cl.sync();                                                     // S1
    double xn2 = 0.0;
    for (int q = 0; q < CL; ++q) xn2 += cl.map_shared_rank(part, q)[0];
    const double alpha = cl.map_shared_rank(part, (k + 1) % CL)[1];
    double beta, t, scal;
    if (xn2 == 0.0) {
      t = 0.0; beta = alpha; scal = 0.0;
    } else {
      beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
      t = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    if (rank == 0 && threadIdx.x == 0) {
      e[k] = beta;
      tau[k] = t;
    }
    // (2) reflector v on the owned rows, stored below the subdiagonal and pushed to every CTA
    for (int r = threadIdx.x; r < nloc; r += blockDim.x) {
      const int i = r * CL + rank;
      if (i < k + 1 || i >= n) continue;
      double v = 1.0;
      if (i >= k + 2) {
        v = Ar[(size_t)r * n + k] * scal;
        Ar[(size_t)r * n + k] = v;
      }
      for (int q = 0; q < CL; ++q) cl.map_shared_rank(vf, q)[i] = v;
    }
    cl.sync();                                                     // S2
    if (t != 0.0) {
      // (3) p = tau A22 v on the owned rows (warp per row), and p.v
      double pv = 0.0;
      for (int r = warp; r < nloc; r += nw) {
        const int i = r * CL + rank;
        if (i < k + 1 || i >= n) continue;
        const double* row = Ar + (size_t)r * n;
        double s = 0.0;
        for (int j = k + 1 + lane; j < n; j += 32) s += row[j] * vf[j];
        s = wsum(s) * t;
        if (lane == 0) {
          wf[i] = s;               // p_i, kept locally until w is formed
          pv += s * vf[i];
        }
      }
      pv = bsum(lane == 0 ? pv : 0.0, red);
      if (threadIdx.x == 0) part[2] = pv;
      cl.sync();                                                   // S3
      double tot = 0.0;
      for (int q = 0; q < CL; ++q) tot += cl.map_shared_rank(part, q)[2];
      const double K = 0.5 * t * tot;
      // (4) w = p - K v on the owned rows, pushed to every CTA
      for (int r = threadIdx.x; r < nloc; r += blockDim.x) {
        const int i = r * CL + rank;
        if (i < k + 1 || i >= n) continue;
        const double w = wf[i] - K * vf[i];
        for (int q = 0; q < CL; ++q) cl.map_shared_rank(wf, q)[i] = w;
      }
      cl.sync();                                                   // S4
      // (5) rank-2 update of the owned rows
      for (int r = warp; r < nloc; r += nw) {
        const int i = r * CL + rank;
        if (i < k + 1 || i >= n) continue;
        double* row = Ar + (size_t)r * n;
        const double vi = vf[i], wi = wf[i];
        for (int j = k + 1 + lane; j < n; j += 32) row[j] -= vi * wf[j] + wi * vf[j];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if ((n - 1) % CL == rank) d[n - 1] = Ar[(size_t)((n - 1) / CL) * n + (n - 1)];
    if (rank == 0) {
      e[n - 1] = 0.0;
      tau[n - 1] = 0.0;
    }
  }
  // reflectors back to global memory for the back-transformation
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j + 1 < i; j += blockDim.x) Ag[(size_t)i * n + j] = Ar[(size_t)r * n + j];
  }
  cl.sync();
}

// ---- Householder tridiagonalisation with one cluster barrier per column ----------------------
// Every CTA keeps the full reflector v, the full update vector w and the pivot row, and updates
// only its own rows.  Per column k: each CTA forms the partial column sums q_r = A_own^T v of its
// rows (A symmetric, so these are the rows' contributions to p = tau A v) and pushes them, with
// the owner also pushing row k+1 (still before this column's update), into every CTA; after the
// single barrier every CTA adds the partials (p), forms K and w, updates its own rows, applies the
// same update to the pushed row k+1 -- which is column k+1 below the diagonal, by symmetry -- and
// derives the next reflector from it redundantly, so no further exchange is needed.  Buffers
// alternate with the column parity: a CTA can be at most one column ahead of another.
// shared memory: own rows [nloc][n], partials [2][CL][n], pivot rows [2][n], v, w, p [3][n]
__global__ void __launch_bounds__(256)
k_tridiag_cl1(const SubDev* __restrict__ subs, double* Am, double* vecs) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int a = blockIdx.x / CL;
  const SubDev& S = subs[a];
  const int n = S.ns;
  const int nloc = (n + CL - 1) / CL;
  double* Ag = Am + S.off_ss;
  double* d = vecs + 8LL * S.off_state;
  double* e = d + n;
  double* tau = d + 2 * n;
  extern __shared__ __align__(16) double tsm[];
  double* Ar = tsm;
  double* qb = Ar + (size_t)nloc * n;          // [2][CL][n]
  double* rb = qb + 2 * (size_t)CL * n;        // [2][n]
  double* vf = rb + 2 * (size_t)n;
  double* wf = vf + n;
  double* pf = wf + n;
  __shared__ double red[8];
  __shared__ double s_sc[4];                   // tau, K, scale of the reflector
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      Ar[(size_t)r * n + j] = 0.5 * (Ag[(size_t)i * n + j] + Ag[(size_t)j * n + i]);
  }
  __syncthreads();
  // row 0 to every CTA, then the first reflector (from column 0 = row 0)
  if (rank == 0)
    for (int q = 0; q < CL; ++q) {
      double* dst = cl.map_shared_rank(rb, q);
      for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = Ar[j];
    }
  cl.sync();
  // reflector of column k from the pivot row buffer `row` (entries j > k): v, tau; d[k], e[k]
  auto reflector = [&](int k, const double* row) {
    double acc = 0.0;
    for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) acc += row[j] * row[j];
    const double xn2 = bsum(acc, red);
    const double alpha = row[k + 1];
    double beta, t, scal;
    if (xn2 == 0.0) {
      t = 0.0; beta = alpha; scal = 0.0;
    } else {
      beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
      t = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) vf[j] = j <= k ? 0.0 : (j == k + 1 ? 1.0 : row[j] * scal);
    if (threadIdx.x == 0) {
      s_sc[0] = t;
      if (rank == 0) {
        d[k] = row[k];
        e[k] = beta;
        tau[k] = t;
      }
    }
    __syncthreads();
  };
  if (n >= 2) reflector(0, rb);
  for (int k = 0; k + 1 < n; ++k) {
    const int par = k & 1;
    const double t = s_sc[0];
    // own reflector entries into the owned rows (column k, below the subdiagonal)
    for (int r = threadIdx.x; r < nloc; r += blockDim.x) {
      const int i = r * CL + rank;
      if (i >= k + 2 && i < n) Ar[(size_t)r * n + k] = vf[i];
    }
    // partial column sums of the own rows: q_j = sum_{i own, i > k} A_ij v_i, j > k
    double* qmine = qb + ((size_t)par * CL + rank) * n;
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
      double acc = 0.0;
      for (int r = 0; r < nloc; ++r) {
        const int i = r * CL + rank;
        if (i > k && i < n) acc += Ar[(size_t)r * n + j] * vf[i];
      }
      for (int q = 0; q < CL; ++q) cl.map_shared_rank(qmine, q)[j] = acc;
    }
    // the owner of row k+1 pushes it (before this column's update) for the next reflector
    if ((k + 1) % CL == rank) {
      const double* src = Ar + (size_t)((k + 1) / CL) * n;
      for (int q = 0; q < CL; ++q) {
        double* dst = cl.map_shared_rank(rb + (size_t)(1 - par) * n, q);
        for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) dst[j] = src[j];
      }
    }
    cl.sync();
    // p = tau sum_r q_r, K = tau p.v / 2, w = p - K v (all j > k, in every CTA)
    double pv = 0.0;
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < CL; ++q) s += qb[((size_t)par * CL + q) * n + j];
      s *= t;
      pf[j] = s;
      pv += s * vf[j];
    }
    pv = bsum(pv, red);
    const double K = 0.5 * t * pv;
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) wf[j] = pf[j] - K * vf[j];
    __syncthreads();
    if (t != 0.0) {
      // own rows: A_ij -= v_i w_j + w_i v_j (i, j > k)
      for (int r = warp; r < nloc; r += nw) {
        const int i = r * CL + rank;
        if (i <= k || i >= n) continue;
        double* row = Ar + (size_t)r * n;
        const double vi = vf[i], wi = wf[i];
        for (int j = k + 1 + lane; j < n; j += 32) row[j] -= vi * wf[j] + wi * vf[j];
      }
      // the pushed row k+1, updated the same way (every CTA)
      double* row1 = rb + (size_t)(1 - par) * n;
      const double v1 = vf[k + 1], w1 = wf[k + 1];
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) row1[j] -= v1 * wf[j] + w1 * vf[j];
    }
    __syncthreads();
    if (k + 2 < n) {
      reflector(k + 1, rb + (size_t)(1 - par) * n);
    } else if (threadIdx.x == 0 && rank == 0) {   // last diagonal entries
      const double* row1 = rb + (size_t)(1 - par) * n;
      d[k + 1] = row1[k + 1];
      e[k + 1] = 0.0;
      tau[k + 1] = 0.0;
    }
  }
  if (n == 1 && threadIdx.x == 0 && rank == 0) {
    d[0] = Ar[0];
    e[0] = 0.0;
    tau[0] = 0.0;
  }
  // reflectors back to global memory for the back-transformation
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j + 1 < i; j += blockDim.x) Ag[(size_t)i * n + j] = Ar[(size_t)r * n + j];
  }
  cl.sync();
}

// Same reduction with the redundant vector work of each column on four warps (one per SM
// sub-partition, so that their FP64 instructions -- each of which holds a sub-partition's FP64
// pipe for tens of cycles on GB300 -- spread over all four pipes): after the cluster barrier
// warps 0-3 form p.v, K and w, update the pushed row k+1 and derive the next reflector from it
// (into the other half of a double-buffered v), synchronising among themselves with a named
// barrier, while the other warps wait at the one block barrier before the row update; a second
// block barrier separates the update from the next column's products.  p = A v is formed row by
// row (the stored rows are full rows of the symmetric matrix): each CTA takes the entries of its
// own rows, one warp per row, and pushes each into every CTA's copy of p, so a CTA receives n
// values per column instead of CL partial vectors and no sum over the cluster is left on the
// vector warps' path.  Per column: one cluster barrier and two block barriers (the block-wide
// reductions of k_tridiag_cl1 take nine).
// shared memory: own rows [nloc][n], p [2][n], pivot rows [2][n], v [2][n], w [n]
__global__ void __launch_bounds__(256)
k_tridiag_cl2(const SubDev* __restrict__ subs, double* Am, double* vecs) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int a = blockIdx.x / CL;
  const SubDev& S = subs[a];
  const int n = S.ns;
  const int nloc = (n + CL - 1) / CL;
  double* Ag = Am + S.off_ss;
  double* d = vecs + 8LL * S.off_state;
  double* e = d + n;
  double* tau = d + 2 * n;
  extern __shared__ __align__(16) double tsm[];
  double* Ar = tsm;
  double* pb = Ar + (size_t)nloc * n;          // [2][n]
  double* rb = pb + 2 * (size_t)n;             // [2][n]
  double* vb = rb + 2 * (size_t)n;             // [2][n]
  double* wf = vb + 2 * (size_t)n;             // [n]
  __shared__ double s_t[2];                    // tau of the reflector in vb[0], vb[1]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      Ar[(size_t)r * n + j] = 0.5 * (Ag[(size_t)i * n + j] + Ag[(size_t)j * n + i]);
  }
  __syncthreads();
  if (rank == 0)
    for (int q = 0; q < CL; ++q) {
      double* dst = cl.map_shared_rank(rb, q);
      for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = Ar[j];
    }
  cl.sync();
  // the four vector warps: thread tv of 128, their own barrier and reduction slots
  const int tv = threadIdx.x;
  __shared__ double s_red[4];
  auto vbar = []() { asm volatile("bar.sync 1, 128;" ::: "memory"); };
  auto vsum = [&](double x) {   // sum over the 128 vector threads (all of them get it)
    x = wsum(x);
    if (lane == 0) s_red[warp] = x;
    vbar();
    const double r = (s_red[0] + s_red[1]) + (s_red[2] + s_red[3]);
    vbar();
    return r;
  };
  // reflector of column k from `row` (entries j > k) into vout / tout; d[k], e[k], tau[k]
  auto reflector_w = [&](int k, const double* row, double* vout, double* tout) {
    double acc = 0.0;
    for (int j = k + 2 + tv; j < n; j += 128) acc += row[j] * row[j];
    const double xn2 = vsum(acc);
    const double alpha = row[k + 1];
    double beta, t, scal;
    if (xn2 == 0.0) {
      t = 0.0; beta = alpha; scal = 0.0;
    } else {
      beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
      t = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    for (int j = tv; j < n; j += 128) vout[j] = j <= k ? 0.0 : (j == k + 1 ? 1.0 : row[j] * scal);
    if (tv == 0) {
      *tout = t;
      if (rank == 0) {
        d[k] = row[k];
        e[k] = beta;
        tau[k] = t;
      }
    }
  };
  if (n >= 2 && warp < 4) reflector_w(0, rb, vb, &s_t[0]);
  __syncthreads();
  for (int k = 0; k + 1 < n; ++k) {
    const int par = k & 1;
    const double* vf = vb + (size_t)par * n;
    const double t = s_t[par];
    // own reflector entries into the owned rows (column k, below the subdiagonal)
    for (int r = threadIdx.x; r < nloc; r += blockDim.x) {
      const int i = r * CL + rank;
      if (i >= k + 2 && i < n) Ar[(size_t)r * n + k] = vf[i];
    }
    // p_i = (A v)_i for the own rows i > k (one warp per row), pushed into every CTA's p
    double* pcur = pb + (size_t)par * n;
    for (int r = warp; r < nloc; r += nw) {
      const int i = r * CL + rank;
      if (i <= k || i >= n) continue;   // uniform in the warp
      const double* row = Ar + (size_t)r * n;
      double acc = 0.0;
      for (int j = k + 1 + lane; j < n; j += 32) acc += row[j] * vf[j];
      acc = wsum(acc);
      if (lane < CL) cl.map_shared_rank(pcur, lane)[i] = acc;
    }
    // the owner of row k+1 pushes it (before this column's update) for the next reflector
    if ((k + 1) % CL == rank) {
      const double* src = Ar + (size_t)((k + 1) / CL) * n;
      for (int q = 0; q < CL; ++q) {
        double* dst = cl.map_shared_rank(rb + (size_t)(1 - par) * n, q);
        for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) dst[j] = src[j];
      }
    }
    cl.sync();
    if (warp < 4) {
      // p = tau A v, K = tau p.v / 2, w = p - K v (j > k); then row k+1 and the next reflector
      double pv = 0.0;
      for (int j = k + 1 + tv; j < n; j += 128) {
        const double sacc = t * pcur[j];
        wf[j] = sacc;
        pv += sacc * vf[j];
      }
      pv = vsum(pv);
      const double K = 0.5 * t * pv;
      for (int j = k + 1 + tv; j < n; j += 128) wf[j] -= K * vf[j];
      vbar();
      double* row1 = rb + (size_t)(1 - par) * n;
      if (t != 0.0) {
        const double v1 = vf[k + 1], w1 = wf[k + 1];
        for (int j = k + 1 + tv; j < n; j += 128) row1[j] -= v1 * wf[j] + w1 * vf[j];
      }
      vbar();
      if (k + 2 < n) {
        reflector_w(k + 1, row1, vb + (size_t)(1 - par) * n, &s_t[1 - par]);
      } else if (tv == 0 && rank == 0) {   // last diagonal entries
        d[k + 1] = row1[k + 1];
        e[k + 1] = 0.0;
        tau[k + 1] = 0.0;
      }
    }
    __syncthreads();
    if (t != 0.0) {
      // own rows: A_ij -= v_i w_j + w_i v_j (i, j > k)
      for (int r = warp; r < nloc; r += nw) {
        const int i = r * CL + rank;
        if (i <= k || i >= n) continue;
        double* row = Ar + (size_t)r * n;
        const double vi = vf[i], wi = wf[i];
        for (int j = k + 1 + lane; j < n; j += 32) row[j] -= vi * wf[j] + wi * vf[j];
      }
    }
    __syncthreads();
  }
  if (n == 1 && threadIdx.x == 0 && rank == 0) {
    d[0] = Ar[0];
    e[0] = 0.0;
    tau[0] = 0.0;
  }
  // reflectors back to global memory for the back-transformation
  for (int r = 0; r < nloc; ++r) {
    const int i = r * CL + rank;
    if (i >= n) break;
    for (int j = threadIdx.x; j + 1 < i; j += blockDim.x) Ag[(size_t)i * n + j] = Ar[(size_t)r * n + j];
  }
  cl.sync();
}

// cluster size and shared memory per CTA for an n x n matrix (0: not possible)
static int pick_cluster(int n, size_t extra_per_cta, size_t& smem) {
  for (int CL : {8, 16}) {
    const size_t nloc = (size_t)(n + CL - 1) / CL;
    smem = nloc * n * sizeof(double) + extra_per_cta;
    if (smem <= 200 * 1024) return CL;
  }
  return 0;
}

template <typename K>
static bool launch_cluster(K kernel, int n_sub, int CL, size_t smem, cudaStream_t st, const SubDev* subs, double* m,
                           void* third, bool tridiag) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (CL > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_sub * CL);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // ask the occupancy calculator before launching: a refused launch inside a stream capture would
  // end the capture
  int active = 0;
  if (cudaOccupancyMaxActiveClusters(&active, (const void*)kernel, &cfg) != cudaSuccess || active < 1) {
    cudaGetLastError();
    return false;
  }
  cudaError_t err;
  if (tridiag)
    err = cudaLaunchKernelEx(&cfg, (void (*)(const SubDev*, double*, double*))kernel, subs, m, (double*)third);
  else
    err = cudaLaunchKernelEx(&cfg, (void (*)(const SubDev*, double*, int*))kernel, subs, m, (int*)third);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Both factorisations run on clusters of cl_first CTAs (8 by default; 16, a non-portable size,
// where the autotuner finds it faster, and as the fallback where 8 do not fit: measured at
// N_s = 160, the extra barrier latency of 16 CTAs outweighs their extra FP64 pipes).
bool launch_cholesky_cluster(const SubDev* d_subs, int n_sub, int max_ns, double* Ms, int* status, int cl_first,
                             cudaStream_t st) {
  for (int CL : {cl_first == 16 ? 16 : 8, cl_first == 16 ? 8 : 16}) {
    const size_t smem = ((size_t)(max_ns + CL - 1) / CL * max_ns + 2 * (size_t)(max_ns + 1)) * sizeof(double);
    if (smem <= 200 * 1024 &&
        launch_cluster(std::getenv("XLS_CHOL_LEFT") ? k_cholesky_cl : k_cholesky_cl2, n_sub, CL, smem, st, d_subs, Ms,
                       status, false))
      return true;
  }
  return false;
}

bool launch_tridiag_cluster(const SubDev* d_subs, int n_sub, int max_ns, double* A, double* vecs, int cl_first,
                            cudaStream_t st) {
  size_t smem = 0;
  // one barrier per column: own rows, p [2][n], pivot rows [2][n], v [2][n], w [n] (k_tridiag_cl2;
  // the two-barrier k_tridiag_cl1 with XLS_TRIDIAG_CL1=1 keeps CL partial vectors: [2][CL][n])
  for (int CL : {cl_first == 16 ? 16 : 8, cl_first == 16 ? 8 : 16}) {
    const bool cl2 = !std::getenv("XLS_TRIDIAG_CL1");
    const size_t rows = (size_t)(max_ns + CL - 1) / CL * max_ns;
    const size_t exact = (rows + (cl2 ? 7 : 2 * (size_t)CL + 5) * max_ns) * sizeof(double);
    if (exact <= 200 * 1024 && launch_cluster(cl2 ? k_tridiag_cl2 : k_tridiag_cl1, n_sub, CL, exact, st, d_subs, A, vecs,
                                              true))
      return true;
  }
  const int CL4 = pick_cluster(max_ns, (2 * (size_t)max_ns + 4) * sizeof(double), smem);
  if (!CL4) return false;
  return launch_cluster(k_tridiag_cl, n_sub, CL4, smem, st, d_subs, A, vecs, true);
}

}  // namespace xls
