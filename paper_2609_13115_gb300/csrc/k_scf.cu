// Self-consistent-field step on the global periodic grid (Sec. 5.A.4): pseudocharge
// electrostatics (Eq. poisson) by conjugate gradients on the FD Laplacian, LDA exchange-
// correlation (Slater + Perdew-Zunger 1981, unpolarised), the energy sums, and periodic Pulay
// mixing with a Kerker-type preconditioner solved in real space.
//
// Reductions are deterministic: fixed grids of kRedBlocks CTAs write partial sums, one CTA adds
// them in a fixed order.
#include <cmath>

#include "xls_internal.h"

namespace xls {

constexpr int kRedBlocks = 296;   // 2 x 148: partial sums per reduction
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_reduce(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;  // valid in thread 0
}

// ---- pseudocharge: b = sum_I -Z pi^-3/2 rc^-3 prod_d sum_k exp(-(x_d - R_d - k L_d)^2 / rc^2) --
// per atom and axis the periodic image sum of the one-dimensional Gaussian (separable)
__global__ void k_pc_axis(int n_atoms, const double* __restrict__ pos, const double* __restrict__ rc, int nx, int ny,
                          int nz, double hx, double hy, double hz, double Lx, double Ly, double Lz, double* g1) {
  const int I = blockIdx.x;
  const int ntot = nx + ny + nz;
  const double r = rc[I];
  for (int q = threadIdx.x; q < ntot; q += blockDim.x) {
    int d, i;
    if (q < nx) { d = 0; i = q; } else if (q < nx + ny) { d = 1; i = q - nx; } else { d = 2; i = q - nx - ny; }
    const double h = d == 0 ? hx : (d == 1 ? hy : hz), L = d == 0 ? Lx : (d == 1 ? Ly : Lz);
    const double x = i * h - pos[3 * I + d];
    const int kmax = (int)ceil(12.0 * r / L) + 1;
    double acc = 0.0;
    for (int k = -kmax; k <= kmax; ++k) {
      const double u = (x - k * L) / r;
      acc += exp(-u * u);
    }
    g1[(size_t)I * ntot + q] = acc;
  }
}

__global__ void k_pc_sum(int n_atoms, const double* __restrict__ g1, const double* __restrict__ amp, int nx, int ny,
                         int nz, double* b) {
  const long long n = (long long)nx * ny * nz;
  const int ntot = nx + ny + nz;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long long)nx * ny));
    double s = 0.0;
    for (int I = 0; I < n_atoms; ++I) {
      const double* g = g1 + (size_t)I * ntot;
      s += amp[I] * g[i] * g[nx + j] * g[nx + ny + k];
    }
    b[q] = s;
  }
}

// ---- reductions ------------------------------------------------------------------------------
// up to four dot products x[t] . y[t] in one pass; partial[blk * 4 + t]
struct DotSpec {
  const double* x[4];
  const double* y[4];
  int nq;
};

__global__ void __launch_bounds__(kRedThreads) k_dots(long long n, DotSpec sp, double* partial) {
  __shared__ double red[32];
  double acc[4] = {0, 0, 0, 0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    for (int t = 0; t < sp.nq; ++t) acc[t] += sp.x[t][q] * sp.y[t][q];
  for (int t = 0; t < sp.nq; ++t) {
    const double s = block_reduce(acc[t], red);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * 4 + t] = s;
  }
}

// out[t] = sum over blocks of partial[. * 4 + t], t < nq (one CTA, fixed order)
__global__ void k_sum_partials(const double* __restrict__ partial, int nblk, int nq, double scale, double* out) {
  __shared__ double red[32];
  for (int t = 0; t < nq; ++t) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(size_t)b * 4 + t];
    s = block_reduce(s, red);
    if (threadIdx.x == 0) out[t] = s * scale;
  }
}

void launch_dots(long long n, const double* const* x, const double* const* y, int nq, double* partial, double* out,
                 double scale, cudaStream_t st) {
  DotSpec sp{};
  sp.nq = nq;
  for (int t = 0; t < nq; ++t) {
    sp.x[t] = x[t];
    sp.y[t] = y[t];
  }
  k_dots<<<kRedBlocks, kRedThreads, 0, st>>>(n, sp, partial);
  k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, nq, scale, out);
}

// ---- elementwise ------------------------------------------------------------------------------
// y = a x + b y + c z  (pointers may alias y)
__global__ void k_axpbypcz(long long n, double a, const double* x, double b, double* y, double c, const double* z) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    double v = b != 0.0 ? b * y[q] : 0.0;   // y may be uninitialised when b == 0
    if (x) v += a * x[q];
    if (z) v += c * z[q];
    y[q] = v;
  }
}
void launch_axpbypcz(long long n, double a, const double* x, double b, double* y, double c, const double* z,
                     cudaStream_t st) {
  k_axpbypcz<<<kRedBlocks * 2, 256, 0, st>>>(n, a, x, b, y, c, z);
}

// y -= mean, mean = *sum / n
__global__ void k_sub_mean(long long n, const double* sum, double* y) {
  const double m = *sum / (double)n;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] -= m;
}
void launch_sub_mean(long long n, const double* sum, double* y, cudaStream_t st) {
  k_sub_mean<<<kRedBlocks * 2, 256, 0, st>>>(n, sum, y);
}

// y *= target / *sum
__global__ void k_rescale(long long n, const double* sum, double target, double* y) {
  const double f = target / *sum;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] *= f;
}

// ---- conjugate gradients (scalars on the device) --------------------------------------------
// s[0] = r.r, s[1] = p.q, s[2] = new r.r
__global__ void k_cg_xr(long long n, const double* __restrict__ s, double* x, double* r, const double* __restrict__ p,
                        const double* __restrict__ q, double* partial) {
  __shared__ double red[32];
  const double alpha = s[1] != 0.0 ? s[0] / s[1] : 0.0;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc += ri * ri;
  }
  const double t = block_reduce(acc, red);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * 4] = t;
}

__global__ void k_cg_p(long long n, double* s, const double* __restrict__ r, double* p) {
  const double beta = s[0] != 0.0 ? s[2] / s[0] : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * p[i];
}

__global__ void k_cg_roll(double* s) {
  s[0] = s[2];
}

void launch_cg_xr(long long n, const double* s, double* x, double* r, const double* p, const double* q,
                  double* partial, cudaStream_t st) {
  k_cg_xr<<<kRedBlocks, kRedThreads, 0, st>>>(n, s, x, r, p, q, partial);
  k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, 1, 1.0, const_cast<double*>(s) + 2);
}
void launch_cg_p(long long n, double* s, const double* r, double* p, cudaStream_t st) {
  k_cg_p<<<kRedBlocks * 2, 256, 0, st>>>(n, s, r, p);
  k_cg_roll<<<1, 1, 0, st>>>(s);
}

// ---- LDA: Slater exchange + Perdew-Zunger 1981 correlation ---------------------------------
__global__ void k_lda(long long n, const double* __restrict__ rho, double* eps, double* vxc) {
  const double PI = 3.14159265358979323846;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const double r = rho[q];
    if (!(r > 0.0)) {
      eps[q] = 0.0;
      vxc[q] = 0.0;
      continue;
    }
    const double rs = cbrt(3.0 / (4.0 * PI * r));
    const double ex = -0.75 * cbrt(3.0 * r / PI);
    const double vx = 4.0 / 3.0 * ex;
    double ec, vc;
    if (rs >= 1.0) {
      const double s = sqrt(rs);
      const double den = 1.0 + 1.0529 * s + 0.3334 * rs;
      ec = -0.1423 / den;
      vc = ec * (1.0 + 7.0 / 6.0 * 1.0529 * s + 4.0 / 3.0 * 0.3334 * rs) / den;
    } else {
      const double lx = log(rs);
      ec = 0.0311 * lx - 0.048 + 0.0020 * rs * lx - 0.0116 * rs;
      vc = 0.0311 * lx + (-0.048 - 0.0311 / 3.0) + 2.0 / 3.0 * 0.0020 * rs * lx + (2.0 * -0.0116 - 0.0020) / 3.0 * rs;
    }
    eps[q] = ex + ec;
    vxc[q] = vx + vc;
  }
}
void launch_lda(long long n, const double* rho, double* eps, double* vxc, cudaStream_t st) {
  k_lda<<<kRedBlocks * 2, 256, 0, st>>>(n, rho, eps, vxc);
}

// ---- plain sum ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kRedThreads) k_sum(long long n, const double* __restrict__ x, double* partial) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    acc += x[q];
  const double s = block_reduce(acc, red);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * 4] = s;
}
void launch_sum(long long n, const double* x, double* partial, double* out, cudaStream_t st) {
  k_sum<<<kRedBlocks, kRedThreads, 0, st>>>(n, x, partial);
  k_sum_partials<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, 1, 1.0, out);
}

// ---- pseudocharge: b, renormalised to sum b dV = -sum Z, mean removed -----------------------
void launch_pseudocharge(int n_atoms, const double* d_pos, const double* d_rc, const double* d_amp, const int gn[3],
                         const double gh[3], const double gL[3], double* g1, double* b, double z_total, double* partial,
                         double* s4, cudaStream_t st) {
  const long long n = (long long)gn[0] * gn[1] * gn[2];
  k_pc_axis<<<n_atoms, 128, 0, st>>>(n_atoms, d_pos, d_rc, gn[0], gn[1], gn[2], gh[0], gh[1], gh[2], gL[0], gL[1],
                                     gL[2], g1);
  k_pc_sum<<<kRedBlocks * 4, 256, 0, st>>>(n_atoms, g1, d_amp, gn[0], gn[1], gn[2], b);
  launch_sum(n, b, partial, s4, st);
  const double dV = gh[0] * gh[1] * gh[2];
  k_rescale<<<kRedBlocks * 2, 256, 0, st>>>(n, s4, -z_total / dV, b);
  launch_sum(n, b, partial, s4, st);
  launch_sub_mean(n, s4, b, st);
}

// ---- superposed atomic Gaussians renormalised to sum x dV = total (no mean removal) ----------
void launch_gaussian_density(int n_atoms, const double* d_pos, const double* d_rc, const double* d_amp, const int gn[3],
                             const double gh[3], const double gL[3], double* g1, double* out, double total,
                             double* partial, double* s4, cudaStream_t st) {
  const long long n = (long long)gn[0] * gn[1] * gn[2];
  k_pc_axis<<<n_atoms, 128, 0, st>>>(n_atoms, d_pos, d_rc, gn[0], gn[1], gn[2], gh[0], gh[1], gh[2], gL[0], gL[1],
                                     gL[2], g1);
  k_pc_sum<<<kRedBlocks * 4, 256, 0, st>>>(n_atoms, g1, d_amp, gn[0], gn[1], gn[2], out);
  launch_sum(n, out, partial, s4, st);
  k_rescale<<<kRedBlocks * 2, 256, 0, st>>>(n, s4, total / (gh[0] * gh[1] * gh[2]), out);
}

void launch_rescale(long long n, const double* sum, double target, double* y, cudaStream_t st) {
  k_rescale<<<kRedBlocks * 2, 256, 0, st>>>(n, sum, target, y);
}

// ---- Pulay: Gram matrix of the residual history and its solve --------------------------------
// partial[blk * kPulayQ + t]: t < m*m: dF_i . dF_j (i, j < m), then m entries dF_i . f
constexpr int kPulayMax = 8;
constexpr int kPulayQ = kPulayMax * kPulayMax + kPulayMax;

__global__ void __launch_bounds__(kRedThreads)
k_pulay_gram(long long n, int m, const double* __restrict__ dF, const double* __restrict__ f, double* partial) {
  __shared__ double red[32];
  for (int i = 0; i < m; ++i)
    for (int j = i; j <= m; ++j) {   // j == m: the right-hand side dF_i . f
      const double* a = dF + (size_t)i * n;
      const double* b = j < m ? dF + (size_t)j * n : f;
      double acc = 0.0;
      for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        acc += a[q] * b[q];
      const double s = block_reduce(acc, red);
      if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kPulayQ + (j < m ? i * m + j : m * m + i)] = s;
    }
}

// sums the partials, mirrors the Gram matrix and solves G gamma = rhs by Gaussian elimination
// with partial pivoting (one thread; m <= 8)
__global__ void k_pulay_solve(const double* __restrict__ partial, int nblk, int m, double* gamma) {
  __shared__ double G[kPulayMax][kPulayMax + 1];
  for (int t = threadIdx.x; t < m * m + m; t += blockDim.x) {
    const int i = t < m * m ? t / m : t - m * m, j = t < m * m ? t % m : m;
    if (t < m * m && j < i) continue;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * kPulayQ + t];
    G[i][j] = s;
    if (t < m * m) G[j][i] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(G[r][c]) > fabs(G[piv][c])) piv = r;
    if (piv != c)
      for (int k = 0; k <= m; ++k) {
        const double t = G[c][k];
        G[c][k] = G[piv][k];
        G[piv][k] = t;
      }
    const double d = G[c][c];
    for (int r = c + 1; r < m; ++r) {
      const double f = d != 0.0 ? G[r][c] / d : 0.0;
      for (int k = c; k <= m; ++k) G[r][k] -= f * G[c][k];
    }
  }
  for (int c = m - 1; c >= 0; --c) {
    double s = G[c][m];
    for (int k = c + 1; k < m; ++k) s -= G[c][k] * gamma[k];
    gamma[c] = G[c][c] != 0.0 ? s / G[c][c] : 0.0;
  }
}

// x_next -= sum_i gamma_i (dX_i + beta dPF_i)
__global__ void k_pulay_update(long long n, int m, const double* __restrict__ gamma, double beta,
                               const double* __restrict__ dX, const double* __restrict__ dPF, double* x) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    double v = x[q];
    for (int i = 0; i < m; ++i) v -= gamma[i] * (dX[(size_t)i * n + q] + beta * dPF[(size_t)i * n + q]);
    x[q] = v;
  }
}

size_t pulay_partial_doubles() { return (size_t)kRedBlocks * kPulayQ; }

void launch_pulay(long long n, int m, const double* dF, const double* dX, const double* dPF, const double* f, double beta,
                  double* partial, double* gamma, double* x, cudaStream_t st) {
  k_pulay_gram<<<kRedBlocks, kRedThreads, 0, st>>>(n, m, dF, f, partial);
  k_pulay_solve<<<1, 128, 0, st>>>(partial, kRedBlocks, m, gamma);
  k_pulay_update<<<kRedBlocks * 2, 256, 0, st>>>(n, m, gamma, beta, dX, dPF, x);
}

}  // namespace xls
