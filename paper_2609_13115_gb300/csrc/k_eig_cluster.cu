// Cholesky factorisation and Householder tridiagonalisation of one subdomain's N_s x N_s
// matrices on a thread-block cluster (Sec. 5.A.3 step (3)): the rows are distributed cyclically
// over the CL CTAs of the cluster (row i in CTA i % CL, local row i / CL) and kept in shared
// memory; vectors that every CTA needs are pushed into each CTA's copy through distributed shared
// memory, and the CTAs meet at cluster barriers.  Same arithmetic as k_cholesky / k_tridiag
// (k_eig.cu), which remain for blocks too large for the cluster's shared memory.
#include <cooperative_groups.h>

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

bool launch_cholesky_cluster(const SubDev* d_subs, int n_sub, int max_ns, double* Ms, int* status, cudaStream_t st) {
  size_t smem = 0;
  const int CL = pick_cluster(max_ns, 2 * (size_t)(max_ns + 1) * sizeof(double), smem);
  if (!CL) return false;
  return launch_cluster(k_cholesky_cl, n_sub, CL, smem, st, d_subs, Ms, status, false);
}

bool launch_tridiag_cluster(const SubDev* d_subs, int n_sub, int max_ns, double* A, double* vecs, cudaStream_t st) {
  size_t smem = 0;
  const int CL = pick_cluster(max_ns, (2 * (size_t)max_ns + 4) * sizeof(double), smem);
  if (!CL) return false;
  return launch_cluster(k_tridiag_cl, n_sub, CL, smem, st, d_subs, A, vecs, true);
}

}  // namespace xls
