// Learned SCF start (Sec. 5.A.4, SCF initialisation: atomic densities plus a learned correction):
// radial descriptors of the atoms around every grid point, a 32-64-64-64-1 tanh MLP (inference
// with BF16 operands and FP32 accumulation; training in FP32: forward, backpropagation, weight
// gradients as batch reductions, Adam), and the start density SAD + correction.
//
// Parameter layout (floats): W1 (32 x 64, row = input), b1 (64), W2 (64 x 64), b2, W3 (64 x 64),
// b3, w4 (64), b4 (1).
#include <cuda_bf16.h>

#include "xls_internal.h"

namespace xls {

constexpr int kIn = 32, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kIn * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH;
constexpr int kMlpParams = kOffB4 + 1;
static_assert(kMlpParams == 10497, "parameter count");
constexpr int kNRad = 16;
constexpr float kRcut = 6.0f, kSigma = 0.25f;

int mlp_param_count() { return kMlpParams; }

// ---- descriptors -------------------------------------------------------------------------------
// X[p][s * 16 + k] = sum over atoms I of species s of exp(-(r - r_k)^2 / (2 sigma^2)) f_c(r),
// r the minimum-image distance, r_k = k * 6/15, f_c(r) = (cos(pi r / 6) + 1) / 2 for r < 6.
// atoms: float4 (x, y, z, species) staged through shared memory in chunks.
__global__ void __launch_bounds__(256) k_descriptors(long long n, int nx, int ny, float hx, float hy, float hz,
                                                      float Lx, float Ly, float Lz, const float4* __restrict__ atoms,
                                                      int n_atoms, int n_species, float* X) {
  constexpr int kChunk = 1024;
  __shared__ float4 sa[kChunk];
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = p < n;
  float px = 0.f, py = 0.f, pz = 0.f;
  if (on) {
    px = (float)(p % nx) * hx;
    py = (float)((p / nx) % ny) * hy;
    pz = (float)(p / ((long long)nx * ny)) * hz;
  }
  float acc[2 * kNRad];
#pragma unroll
  for (int k = 0; k < 2 * kNRad; ++k) acc[k] = 0.f;
  const float inv2s2 = 1.0f / (2.0f * kSigma * kSigma), dr = kRcut / (kNRad - 1);
  for (int c0 = 0; c0 < n_atoms; c0 += kChunk) {
    const int cn = min(kChunk, n_atoms - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) sa[i] = atoms[c0 + i];
    __syncthreads();
    if (!on) continue;
    for (int i = 0; i < cn; ++i) {
      const float4 A = sa[i];
      float dx = px - A.x, dy = py - A.y, dz = pz - A.z;
      dx -= Lx * rintf(dx / Lx);
      dy -= Ly * rintf(dy / Ly);
      dz -= Lz * rintf(dz / Lz);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 >= kRcut * kRcut) continue;
      const float r = sqrtf(r2);
      const float fc = 0.5f * (cospif(r / kRcut) + 1.0f);
      const int s = (int)A.w;
#pragma unroll
      for (int k = 0; k < kNRad; ++k) {
        const float u = r - k * dr;
        const float e = expf(-u * u * inv2s2) * fc;
        if (s == 0) acc[k] += e; else acc[kNRad + k] += e;
      }
    }
  }
  if (!on) return;
  float* out = X + p * (long long)(n_species * kNRad);
#pragma unroll
  for (int k = 0; k < 2 * kNRad; ++k)
    if (k < n_species * kNRad) out[k] = acc[k];
}

void launch_descriptors(long long n, const int gn[3], const double gh[3], const double gL[3], const float4* atoms,
                        int n_atoms, int n_species, float* X, cudaStream_t st) {
  k_descriptors<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, gn[0], gn[1], (float)gh[0], (float)gh[1], (float)gh[2],
                                                             (float)gL[0], (float)gL[1], (float)gL[2], atoms, n_atoms,
                                                             n_species, X);
}

// ---- inference: BF16 operands, FP32 accumulation ---------------------------------------------
__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// weights rounded to BF16 once per launch into shared memory (as floats); one thread per point
__global__ void __launch_bounds__(128) k_mlp_infer(long long n, const float* __restrict__ theta,
                                                   const float* __restrict__ X, float* y) {
  extern __shared__ float w[];   // kMlpParams floats: BF16-rounded weights, biases as they are
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    const bool bias = (i >= kOffB1 && i < kOffW2) || (i >= kOffB2 && i < kOffW3) || (i >= kOffB3 && i < kOffW4) ||
                      i == kOffB4;
    w[i] = bias ? theta[i] : bf(theta[i]);
  }
  __syncthreads();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float x[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = bf(X[p * kIn + i]);
  float h[kH], g[kH];
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float z = w[kOffB1 + o];
#pragma unroll
    for (int i = 0; i < kIn; ++i) z = fmaf(x[i], w[kOffW1 + i * kH + o], z);
    h[o] = bf(tanhf(z));
  }
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float z = w[kOffB2 + o];
#pragma unroll
    for (int i = 0; i < kH; ++i) z = fmaf(h[i], w[kOffW2 + i * kH + o], z);
    g[o] = bf(tanhf(z));
  }
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float z = w[kOffB3 + o];
#pragma unroll
    for (int i = 0; i < kH; ++i) z = fmaf(g[i], w[kOffW3 + i * kH + o], z);
    h[o] = bf(tanhf(z));
  }
  float z = w[kOffB4];
#pragma unroll
  for (int i = 0; i < kH; ++i) z = fmaf(h[i], w[kOffW4 + i], z);
  y[p] = z;
}

void launch_mlp_infer(long long n, const float* theta, const float* X, float* y, cudaStream_t st) {
  cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kMlpParams * 4);   // per device
  if (n > 0) k_mlp_infer<<<(unsigned)((n + 127) / 128), 128, kMlpParams * 4, st>>>(n, theta, X, y);
}

// ---- training (FP32) -----------------------------------------------------------------------------
// forward keeping the activations A[p] = (a1, a2, a3) and the output error e[p] = 2 (y_p - y) / n;
// deltas D[p] = (d1, d2, d3) of the hidden layers by backpropagation; loss partial sums
__global__ void __launch_bounds__(128) k_mlp_fwd_bwd(long long n, const float* __restrict__ theta,
                                                     const float* __restrict__ X, const float* __restrict__ yt,
                                                     float* A, float* D, float* e, double* loss_partial) {
  extern __shared__ float w[];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = theta[i];
  __syncthreads();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (p < n) {
    float a1[kH], a2[kH], a3[kH];
    const float* x = X + p * kIn;
    for (int o = 0; o < kH; ++o) {
      float z = w[kOffB1 + o];
      for (int i = 0; i < kIn; ++i) z = fmaf(x[i], w[kOffW1 + i * kH + o], z);
      a1[o] = tanhf(z);
    }
    for (int o = 0; o < kH; ++o) {
      float z = w[kOffB2 + o];
#pragma unroll 16
      for (int i = 0; i < kH; ++i) z = fmaf(a1[i], w[kOffW2 + i * kH + o], z);
      a2[o] = tanhf(z);
    }
    for (int o = 0; o < kH; ++o) {
      float z = w[kOffB3 + o];
#pragma unroll 16
      for (int i = 0; i < kH; ++i) z = fmaf(a2[i], w[kOffW3 + i * kH + o], z);
      a3[o] = tanhf(z);
    }
    float z = w[kOffB4];
    for (int i = 0; i < kH; ++i) z = fmaf(a3[i], w[kOffW4 + i], z);
    const float err = z - yt[p];
    l = (double)err * err;
    const float d4 = 2.0f * err / (float)n;
    e[p] = d4;
    float* Ap = A + p * (3 * kH);
    for (int i = 0; i < kH; ++i) {
      Ap[i] = a1[i];
      Ap[kH + i] = a2[i];
      Ap[2 * kH + i] = a3[i];
    }
    // backpropagation: d3 = d4 w4 (1 - a3^2); d2 = (W3 d3)(1 - a2^2); d1 = (W2 d2)(1 - a1^2)
    float d3[kH], d2[kH];
    for (int i = 0; i < kH; ++i) d3[i] = d4 * w[kOffW4 + i] * (1.0f - a3[i] * a3[i]);
    for (int i = 0; i < kH; ++i) {
      float s = 0.f;
#pragma unroll 16
      for (int o = 0; o < kH; ++o) s = fmaf(w[kOffW3 + i * kH + o], d3[o], s);
      d2[i] = s * (1.0f - a2[i] * a2[i]);
    }
    float* Dp = D + p * (3 * kH);
    for (int i = 0; i < kH; ++i) {
      float s = 0.f;
#pragma unroll 16
      for (int o = 0; o < kH; ++o) s = fmaf(w[kOffW2 + i * kH + o], d2[o], s);
      Dp[i] = s * (1.0f - a1[i] * a1[i]);
      Dp[kH + i] = d2[i];
      Dp[2 * kH + i] = d3[i];
    }
  }
  // block partial of the squared error
  __shared__ double red[4];
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) loss_partial[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

// weight gradients of one layer as a batch reduction: G[i][o] = sum_p In[p][i] Dl[p][o] and
// Gb[o] = sum_p Dl[p][o]; fixed slices of points per block (partials, then a fixed-order sum).
// In rows have stride sin, Dl rows stride sd (element offsets ioff / doff inside the row).
constexpr int kGradBlocks = 148;

__global__ void __launch_bounds__(256) k_mlp_wgrad(long long n, int ni, int no, const float* __restrict__ In, int sin,
                                                   int ioff, const float* __restrict__ Dl, int sd, int doff,
                                                   float* partial) {
  constexpr int kP = 32;
  __shared__ float si[kP][kH + 1];
  __shared__ float sdl[kP][kH + 1];
  const int nio = ni * no;
  const int per = (nio + no + blockDim.x - 1) / blockDim.x;   // entries per thread (<= 17)
  float acc[17];
#pragma unroll
  for (int k = 0; k < 17; ++k) acc[k] = 0.f;
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long p0 = (long long)blockIdx.x * chunk, p1 = min(n, p0 + chunk);
  for (long long q0 = p0; q0 < p1; q0 += kP) {
    const int m = (int)min((long long)kP, p1 - q0);
    __syncthreads();
    for (int t = threadIdx.x; t < kP * kH; t += blockDim.x) {
      const int r = t / kH, c = t % kH;
      si[r][c] = (r < m && c < ni) ? In[(q0 + r) * sin + ioff + c] : 0.f;
      sdl[r][c] = (r < m && c < no) ? Dl[(q0 + r) * sd + doff + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 17; ++k) {
      const int idx = threadIdx.x + k * blockDim.x;
      if (k >= per || idx >= nio + no) continue;
      float s = acc[k];
      if (idx < nio) {
        const int i = idx / no, o = idx % no;
        for (int r = 0; r < m; ++r) s = fmaf(si[r][i], sdl[r][o], s);
      } else {
        const int o = idx - nio;
        for (int r = 0; r < m; ++r) s += sdl[r][o];
      }
      acc[k] = s;
    }
  }
#pragma unroll
  for (int k = 0; k < 17; ++k) {
    const int idx = threadIdx.x + k * blockDim.x;
    if (k < per && idx < nio + no) partial[(size_t)blockIdx.x * (nio + no) + idx] = acc[k];
  }
}

// grad[off_w + idx] (weights, then biases at off_b) = sum over blocks of the partials (fixed order)
__global__ void k_mlp_wgrad_sum(int nblk, int nio, int no, const float* __restrict__ partial, float* grad, int off_w,
                                int off_b) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nio + no) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * (nio + no) + idx];
  if (idx < nio) grad[off_w + idx] = (float)s;
  else grad[off_b + idx - nio] = (float)s;
}

__global__ void k_sum_d(int n, const double* __restrict__ x, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *out = t;
  }
}

// work: A, D (3 * 64 floats per point), e (1 per point), partials; loss_out: device double
void launch_mlp_grad(long long n, const float* theta, const float* X, const float* yt, float* A, float* D, float* e,
                     double* loss_partial, float* wpartial, float* grad, double* loss_out, cudaStream_t st) {
  cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kMlpParams * 4);   // per device
  const unsigned nb = (unsigned)((n + 127) / 128);
  k_mlp_fwd_bwd<<<nb, 128, kMlpParams * 4, st>>>(n, theta, X, yt, A, D, e, loss_partial);
  k_sum_d<<<1, 256, 0, st>>>((int)nb, loss_partial, loss_out);
  struct L {
    int ni, no;
    const float* in;
    int sin, ioff;
    const float* dl;
    int sd, doff;
    int off_w, off_b;
  };
  const L layers[4] = {
      {kIn, kH, X, kIn, 0, D, 3 * kH, 0, kOffW1, kOffB1},
      {kH, kH, A, 3 * kH, 0, D, 3 * kH, kH, kOffW2, kOffB2},
      {kH, kH, A, 3 * kH, kH, D, 3 * kH, 2 * kH, kOffW3, kOffB3},
      {kH, 1, A, 3 * kH, 2 * kH, e, 1, 0, kOffW4, kOffB4},
  };
  for (const L& l : layers) {
    k_mlp_wgrad<<<kGradBlocks, 256, 0, st>>>(n, l.ni, l.no, l.in, l.sin, l.ioff, l.dl, l.sd, l.doff, wpartial);
    const int tot = l.ni * l.no + l.no;
    k_mlp_wgrad_sum<<<(tot + 255) / 256, 256, 0, st>>>(kGradBlocks, l.ni * l.no, l.no, wpartial, grad, l.off_w,
                                                        l.off_b);
  }
}

size_t mlp_wpartial_floats() { return (size_t)kGradBlocks * (kH * kH + kH); }

// Adam (beta1 0.9, beta2 0.999, eps 1e-8), step t >= 1
__global__ void k_adam(int n, float* theta, float* m, float* v, const float* __restrict__ g, float lr, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f;
  const float mi = b1 * m[i] + (1.0f - b1) * g[i];
  const float vi = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.0f - powf(b1, (float)t)), vh = vi / (1.0f - powf(b2, (float)t));
  theta[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

void launch_adam(int n, float* theta, float* m, float* v, const float* g, float lr, int t, cudaStream_t st) {
  k_adam<<<(n + 255) / 256, 256, 0, st>>>(n, theta, m, v, g, lr, t);
}

// ---- start density: rho = max(sad + corr, 0), then renormalised by the caller ---------------
__global__ void k_add_clamp(long long n, const double* __restrict__ sad, const float* __restrict__ corr, double* rho) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    rho[q] = fmax(sad[q] + (double)corr[q], 0.0);
}
void launch_add_clamp(long long n, const double* sad, const float* corr, double* rho, cudaStream_t st) {
  k_add_clamp<<<592, 256, 0, st>>>(n, sad, corr, rho);
}

}  // namespace xls
