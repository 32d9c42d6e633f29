// Geometric multigrid preconditioner for the periodic Poisson and screened-Poisson solves of the
// SCF step (-Delta_h x = f and (-Delta_h + kappa^2) x = f on the global grid, Eq. poisson), after
// the paper's PCG scheme: an FP64 conjugate-gradient iteration on the 12th-order operator whose
// preconditioner is one FP32 V-cycle of the 7-point (second-order) Laplacian (Sec. 5.B,
// "Poisson solver").  The 7-point operator has the same low-frequency behaviour as the 12th-order
// one (their symbols agree to O(h^2 k^4) and stay within a bounded ratio up to the Nyquist
// frequency), so the V-cycle is a spectrally equivalent preconditioner.
//
// Levels: the grid halves along every axis while all three extents are even and at least 6;
// weighted Jacobi smoothing (two sweeps before and after, the same weight, so the V-cycle is a
// symmetric operator), full-weighting restriction (27 points, weights 1/8 (1/2)^|d|), trilinear
// prolongation (its adjoint times 8), and sweeps of Jacobi on the coarsest grid.  All grids are
// periodic; a zero-mean right-hand side keeps every level's iterate at zero mean.
#include "xls_internal.h"

namespace xls {

__device__ __forceinline__ int mg_wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

struct MgOp {
  int n[3];
  float cx, cy, cz;   // 1 / h^2 per axis
  float sigma;        // kappa^2 (0 for Poisson)
};

__device__ __forceinline__ float mg_apply_at(const MgOp& o, const float* __restrict__ u, int i, int j, int k) {
  const int nx = o.n[0], ny = o.n[1], nz = o.n[2];
  const long long c = ((long long)k * ny + j) * nx + i;
  const float uc = u[c];
  const float ux = u[((long long)k * ny + j) * nx + mg_wrap(i - 1, nx)] + u[((long long)k * ny + j) * nx + mg_wrap(i + 1, nx)];
  const float uy = u[((long long)k * ny + mg_wrap(j - 1, ny)) * nx + i] + u[((long long)k * ny + mg_wrap(j + 1, ny)) * nx + i];
  const float uz = u[((long long)mg_wrap(k - 1, nz) * ny + j) * nx + i] + u[((long long)mg_wrap(k + 1, nz) * ny + j) * nx + i];
  return (2.f * (o.cx + o.cy + o.cz) + o.sigma) * uc - o.cx * ux - o.cy * uy - o.cz * uz;
}

// u_out = u_in + w D^-1 (f - A u_in); u_in == nullptr means u_in = 0
__global__ void k_mg_jacobi(MgOp o, float w, const float* __restrict__ f, const float* __restrict__ u_in, float* u_out) {
  const long long n = (long long)o.n[0] * o.n[1] * o.n[2];
  const float dinv = 1.f / (2.f * (o.cx + o.cy + o.cz) + o.sigma);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % o.n[0]), j = (int)((q / o.n[0]) % o.n[1]), k = (int)(q / ((long long)o.n[0] * o.n[1]));
    if (u_in) u_out[q] = u_in[q] + w * dinv * (f[q] - mg_apply_at(o, u_in, i, j, k));
    else u_out[q] = w * dinv * f[q];
  }
}

// r = f - A u
__global__ void k_mg_residual(MgOp o, const float* __restrict__ f, const float* __restrict__ u, float* r) {
  const long long n = (long long)o.n[0] * o.n[1] * o.n[2];
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % o.n[0]), j = (int)((q / o.n[0]) % o.n[1]), k = (int)(q / ((long long)o.n[0] * o.n[1]));
    r[q] = f[q] - mg_apply_at(o, u, i, j, k);
  }
}

// coarse point I sits on fine point 2I; f_c(I) = sum_d 1/8 (1/2)^(|dx|+|dy|+|dz|) r_f(2I + d)
__global__ void k_mg_restrict(int cx, int cy, int cz, const float* __restrict__ rf, float* fc) {
  const int fx = 2 * cx, fy = 2 * cy, fz = 2 * cz;
  const long long n = (long long)cx * cy * cz;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(q % cx), J = (int)((q / cx) % cy), K = (int)(q / ((long long)cx * cy));
    float s = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const float wgt = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f);
          s += wgt * rf[((long long)mg_wrap(2 * K + dz, fz) * fy + mg_wrap(2 * J + dy, fy)) * fx + mg_wrap(2 * I + dx, fx)];
        }
    fc[q] = 0.125f * s;
  }
}

// u_f += trilinear interpolation of u_c (fine point i: coarse i/2 if even, the mean of its two
// coarse neighbours if odd, per axis)
__global__ void k_mg_prolong_add(int cx, int cy, int cz, const float* __restrict__ uc, float* uf) {
  const int fx = 2 * cx, fy = 2 * cy, fz = 2 * cz;
  const long long n = (long long)fx * fy * fz;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % fx), j = (int)((q / fx) % fy), k = (int)(q / ((long long)fx * fy));
    const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    const int i1 = (i & 1) ? mg_wrap(i0 + 1, cx) : i0, j1 = (j & 1) ? mg_wrap(j0 + 1, cy) : j0,
              k1 = (k & 1) ? mg_wrap(k0 + 1, cz) : k0;
    auto at = [&](int a, int b, int c) { return uc[((long long)c * cy + b) * cx + a]; };
    const float v = 0.125f * (at(i0, j0, k0) + at(i1, j0, k0) + at(i0, j1, k0) + at(i1, j1, k0) + at(i0, j0, k1) +
                              at(i1, j0, k1) + at(i0, j1, k1) + at(i1, j1, k1));
    uf[q] += v;
  }
}

__global__ void k_mg_to_f32(long long n, const double* __restrict__ x, float* y) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = (float)x[q];
}
__global__ void k_mg_to_f64(long long n, const float* __restrict__ x, double* y) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = (double)x[q];
}

// flexible (Polak-Ribiere) PCG direction: beta = (z.r - z.r_old) / s_old, p = z + beta p
// s[0] = r.z of the previous iteration, s[4] = r.z, s[5] = r_old.z
__global__ void k_pcg_p(long long n, double* s, const double* __restrict__ z, double* p) {
  const double beta = s[0] != 0.0 ? (s[4] - s[5]) / s[0] : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}
__global__ void k_pcg_roll(double* s) { s[0] = s[4]; }

static int mg_blocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 1184); }

int mg_level_count(const int n[3]) {
  int L = 1, a = n[0], b = n[1], c = n[2];
  while (a % 2 == 0 && b % 2 == 0 && c % 2 == 0 && a >= 6 && b >= 6 && c >= 6 && L < 8) {
    a /= 2;
    b /= 2;
    c /= 2;
    ++L;
  }
  return L;
}

size_t mg_floats(const int n[3]) {
  size_t tot = 0;
  int a = n[0], b = n[1], c = n[2];
  for (int l = 0; l < mg_level_count(n); ++l) {
    tot += 4 * (size_t)a * b * c;   // u, u2, f, r
    a /= 2;
    b /= 2;
    c /= 2;
  }
  return tot;
}

// z = M r: one V-cycle from a zero start; work: mg_floats(n) floats
void launch_mg_vcycle(const int n[3], const double h[3], double sigma, const double* r, double* z, float* work,
                      cudaStream_t st) {
  const int L = mg_level_count(n);
  struct Lev {
    MgOp o;
    long long np;
    float *u, *u2, *f, *r;
  } lev[8];
  float* w = work;
  int a = n[0], b = n[1], c = n[2];
  double hx = h[0], hy = h[1], hz = h[2];
  for (int l = 0; l < L; ++l) {
    Lev& v = lev[l];
    v.o.n[0] = a;
    v.o.n[1] = b;
    v.o.n[2] = c;
    v.o.cx = (float)(1.0 / (hx * hx));
    v.o.cy = (float)(1.0 / (hy * hy));
    v.o.cz = (float)(1.0 / (hz * hz));
    v.o.sigma = (float)sigma;
    v.np = (long long)a * b * c;
    v.u = w;
    v.u2 = w + v.np;
    v.f = w + 2 * v.np;
    v.r = w + 3 * v.np;
    w += 4 * v.np;
    a /= 2;
    b /= 2;
    c /= 2;
    hx *= 2;
    hy *= 2;
    hz *= 2;
  }
  constexpr float kW = 0.8f;   // Jacobi weight (smoothing factor of the 7-point operator near its optimum)
  constexpr int kNu = 2, kCoarse = 12;
  k_mg_to_f32<<<mg_blocks(lev[0].np), 256, 0, st>>>(lev[0].np, r, lev[0].f);
  // descent: smooth from zero, restrict the residual
  for (int l = 0; l < L; ++l) {
    Lev& v = lev[l];
    const int sweeps = (l == L - 1) ? kCoarse : kNu;
    k_mg_jacobi<<<mg_blocks(v.np), 256, 0, st>>>(v.o, kW, v.f, nullptr, v.u);
    for (int s = 1; s < sweeps; ++s) {
      k_mg_jacobi<<<mg_blocks(v.np), 256, 0, st>>>(v.o, kW, v.f, v.u, v.u2);
      std::swap(v.u, v.u2);
    }
    if (l + 1 < L) {
      k_mg_residual<<<mg_blocks(v.np), 256, 0, st>>>(v.o, v.f, v.u, v.r);
      const Lev& cl = lev[l + 1];
      k_mg_restrict<<<mg_blocks(cl.np), 256, 0, st>>>(cl.o.n[0], cl.o.n[1], cl.o.n[2], v.r, cl.f);
    }
  }
  // ascent: add the coarse correction, smooth again
  for (int l = L - 2; l >= 0; --l) {
    Lev& v = lev[l];
    const Lev& cl = lev[l + 1];
    k_mg_prolong_add<<<mg_blocks(v.np), 256, 0, st>>>(cl.o.n[0], cl.o.n[1], cl.o.n[2], cl.u, v.u);
    for (int s = 0; s < kNu; ++s) {
      k_mg_jacobi<<<mg_blocks(v.np), 256, 0, st>>>(v.o, kW, v.f, v.u, v.u2);
      std::swap(v.u, v.u2);
    }
  }
  k_mg_to_f64<<<mg_blocks(lev[0].np), 256, 0, st>>>(lev[0].np, lev[0].u, z);
}

void launch_pcg_p(long long n, double* s, const double* z, double* p, cudaStream_t st) {
  k_pcg_p<<<mg_blocks(n), 256, 0, st>>>(n, s, z, p);
  k_pcg_roll<<<1, 1, 0, st>>>(s);
}

}  // namespace xls
