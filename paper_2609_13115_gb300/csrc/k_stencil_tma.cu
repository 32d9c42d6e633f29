// TMA-staged FP32 filter step: 12th-order FD Laplacian + local potential + scaled Chebyshev
// recurrence (Sec. 5.A.3 step (1); Sec. 5.B.2 stencil, cache blocking, axis-neighbour reuse).
//
//   Y_out = scale * (-1/2 Delta_h Y_in + V Y_in - c Y_in) - shift * Y_prev
//
// A CTA owns a tile of TY full-width rows of one vector of one subdomain and marches along z.
// Each xy-plane of the tile, with 6 halo rows above and below and 8 halo columns left and right,
// is brought into a ring of shared-memory slots by TMA (cp.async.bulk.tensor, three boxes: top
// halo rows, interior rows, bottom halo rows; out-of-range boxes are zero-filled, which is the
// Dirichlet boundary; periodic axes wrap the box coordinates instead).  A thread computes four
// consecutive x-points of one row: the x- and y-neighbours come from the plane slot with 128-bit
// shared loads, the z-neighbours from a register queue of 13 planes fed from the same slots.
// The nonlocal projector terms are added by the projection / back-projection launches around
// this one.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "xls_internal.h"

namespace xls {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ int wrapt(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Bounded wait on a TMA landing: on expiry the status word gets XLS_ETIMEOUT (never a trap).
__device__ __forceinline__ bool wait_slot(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < (1LL << 28); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

constexpr int kSlots = 10;       // ring depth: 7 resident planes + 3 in flight
constexpr int kHaloX = 8;        // halo columns on each side (16-byte aligned TMA x coordinate)

// Stencil weights of one launch (all subdomains of a launch share the grid spacing): passed by
// value so that the FMAs read them from the constant bank instead of registers.
struct StencilW {
  float wx[kN0 + 1], wy[kN0 + 1], wz[kN0 + 1];
  float wc;
};

__global__ void __launch_bounds__(288, 2)
k_stencil_tma(const SubDev* __restrict__ subs, const TmaJob* __restrict__ jobs, const int* __restrict__ job_off,
              int n_jobs, const CUtensorMap* __restrict__ maps, int buf_in, const float* Yprev, float* Yout,
              const float* __restrict__ Vall, const StepCoef* __restrict__ coef, int step, int* status,
              const StencilW sw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kSlots];
  __shared__ int s_abort;
  // locate the job (class-uniform launch: all jobs share W and TY)
  const int b = blockIdx.x;
  int lo = 0, hi = n_jobs;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (job_off[mid] <= b) lo = mid; else hi = mid;
  }
  const TmaJob J = jobs[lo];
  const SubDev& S = subs[J.sub];
  const int local = b - job_off[lo];
  const int nyt = J.n_ytiles;
  const int vec = local / nyt, yt = local % nyt;
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const int TY = blockDim.y, W = J.W;
  const int y0 = yt * TY;
  const int rows = TY + 2 * kN0;
  float* ring = reinterpret_cast<float*>(smem_raw);
  const int slot_floats = rows * W;
  const CUtensorMap* map_tb = maps + (size_t)(J.sub * 3 + buf_in) * 2;   // 6-row boxes
  const CUtensorMap* map_in = map_tb + 1;                                // TY-row boxes
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * blockDim.x + tx;
  const int x4 = 4 * tx;                 // first of this thread's four x-points
  const int y = y0 + ty;
  const bool row_ok = (y < ny);
  const bool px = S.periodic[0], py = S.periodic[1], pz = S.periodic[2];
  const int nplanes = nz + 2 * kN0;      // planes -6 .. nz+5
  const uint32_t slot_bytes = (uint32_t)slot_floats * 4u;
  const int ytop = py ? wrapt(y0 - kN0, ny) : y0 - kN0;
  const int ybot = py ? wrapt(y0 + TY, ny) : y0 + TY;

  auto issue = [&](int pi) {  // plane index pi (z = pi - 6) into slot pi % kSlots
    const int z = pi - kN0;
    uint64_t* bar = &bars[pi % kSlots];
    const bool in_range = pz || (z >= 0 && z < nz);
    if (!in_range) {
      mbar_arrive(bar);
      return;
    }
    const int zz = pz ? wrapt(z, nz) : z;
    float* dst = ring + (size_t)(pi % kSlots) * slot_floats;
    mbar_expect_tx(bar, slot_bytes);
    tma_load_4d(dst, map_tb, bar, -kHaloX, ytop, zz, vec);
    tma_load_4d(dst + kN0 * W, map_in, bar, -kHaloX, y0, zz, vec);
    tma_load_4d(dst + (kN0 + TY) * W, map_tb, bar, -kHaloX, ybot, zz, vec);
  };

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < kSlots; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int pi = 0; pi < kSlots && pi < nplanes; ++pi) issue(pi);

  // step coefficients
  const float wc = sw.wc;
  const StepCoef cf = coef[J.sub * kMaxDegree + step];
  const float scale = (float)cf.scale, cshift = (float)cf.c, pshift = (float)cf.shift;
  const long long plane_sz = (long long)nx * ny;
  const long long base = S.off_blk + (long long)vec * S.nd;
  const float* V = Vall + S.off_pt;
  const bool active = (x4 < nx);

  float4 q[2 * kN0 + 1];
#pragma unroll
  for (int k = 0; k < 2 * kN0 + 1; ++k) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  // V and Y_prev of the next output plane are loaded one iteration ahead (their HBM latency
  // then overlaps a plane of work)
  const bool io = active && row_ok;
  auto ld_v = [&](int zo_) -> float4 {
    return (io && zo_ < nz) ? *reinterpret_cast<const float4*>(V + (long long)zo_ * plane_sz + (long long)y * nx + x4)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto ld_p = [&](int zo_) -> float4 {
    return (io && Yprev && zo_ < nz)
               ? *reinterpret_cast<const float4*>(Yprev + base + (long long)zo_ * plane_sz + (long long)y * nx + x4)
               : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  float4 v_next = ld_v(0), p_next = ld_p(0);

  for (int pi = 0; pi < nplanes; ++pi) {
    const int slot = pi % kSlots;
    const uint32_t parity = (uint32_t)((pi / kSlots) & 1);
    const bool ok = wait_slot(&bars[slot], parity);
    if (!ok) s_abort = 1;
    const float* P = ring + (size_t)slot * slot_floats;
    const int z = pi - kN0;
    const bool plane_loaded = pz || (z >= 0 && z < nz);
    // push this plane's values of the thread's four columns into the z-queue
#pragma unroll
    for (int k = 0; k < 2 * kN0; ++k) q[k] = q[k + 1];
    q[2 * kN0] = (ok && plane_loaded && active) ? *reinterpret_cast<const float4*>(P + (ty + kN0) * W + kHaloX + x4)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
    const int zo = pi - 2 * kN0;  // output plane whose z-window is now complete
    if (ok && zo >= 0 && active && row_ok) {
      const float* C = ring + (size_t)((pi - kN0) % kSlots) * slot_floats;  // slot of plane zo
      const float* rowp = C + (ty + kN0) * W;
      // x-neighbours: columns x4-6 .. x4+9 of the halo-shifted row (aligned float4 window);
      // along a periodic x axis the edge threads read the wrapped columns of the same row
      float xr[20];
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        // chunk j covers x = x4 - 8 + 4j .. +3: wholly inside [0, nx) or wholly outside
        // (n_x and x4 are multiples of 4); outside chunks of a periodic axis wrap
        int xs = x4 - kHaloX + 4 * j;
        if (px) xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        const int col = xs + kHaloX;
        const float4 v4 = *reinterpret_cast<const float4*>(rowp + col);
        xr[4 * j] = v4.x; xr[4 * j + 1] = v4.y; xr[4 * j + 2] = v4.z; xr[4 * j + 3] = v4.w;
      }
      // element r of the thread's points sits at xr[kHaloX + r]
      float acc[4];
      const float4 c4 = q[kN0];
      const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = wc * cv[r];
#pragma unroll
      for (int p = 1; p <= kN0; ++p) {
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] += sw.wx[p] * (xr[kHaloX + r + p] + xr[kHaloX + r - p]);
        const float4 up = *reinterpret_cast<const float4*>(C + (ty + kN0 + p) * W + kHaloX + x4);
        const float4 dn = *reinterpret_cast<const float4*>(C + (ty + kN0 - p) * W + kHaloX + x4);
        acc[0] += sw.wy[p] * (up.x + dn.x);
        acc[1] += sw.wy[p] * (up.y + dn.y);
        acc[2] += sw.wy[p] * (up.z + dn.z);
        acc[3] += sw.wy[p] * (up.w + dn.w);
        const float4 zu = q[kN0 + p], zd = q[kN0 - p];
        acc[0] += sw.wz[p] * (zu.x + zd.x);
        acc[1] += sw.wz[p] * (zu.y + zd.y);
        acc[2] += sw.wz[p] * (zu.z + zd.z);
        acc[3] += sw.wz[p] * (zu.w + zd.w);
      }
      const long long g = (long long)zo * plane_sz + (long long)y * nx + x4;
      const float4 v4 = v_next, pv = p_next;
      v_next = ld_v(zo + 1);
      p_next = ld_p(zo + 1);
      const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
      float o[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) o[r] = scale * (acc[r] + vv[r] * cv[r] - cshift * cv[r]);
      o[0] -= pshift * pv.x;
      o[1] -= pshift * pv.y;
      o[2] -= pshift * pv.z;
      o[3] -= pshift * pv.w;
      *reinterpret_cast<float4*>(Yout + base + g) = make_float4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();  // every thread is done with plane index pi - 6 (x/y of output zo)
    if (s_abort) {    // a plane never landed: record it and leave (uniform: read after the barrier)
      if (tid == 0) atomicCAS(status, 0, XLS_ETIMEOUT);
      return;
    }
    const int rel = pi - kN0;
    if (tid == 0 && rel >= 0) {
      const int nxt = rel + kSlots;  // reuses the slot of plane index rel
      if (nxt < nplanes) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(nxt);
      }
    }
  }
}

// ---- host side: tensor maps and launch ----------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int tma_tile_rows(const SubDev& S) {
  // rows per tile: 16, or a divisor of n_y along a periodic y axis (the wrapped halo boxes
  // then start exactly at the tile edges)
  if (!S.periodic[1]) return 16;
  for (int ty : {16, 12, 8, 24, 6})
    if (S.n[1] % ty == 0) return ty;
  return 0;
}

bool tma_eligible(const SubDev& S) {
  const int W = ((S.n[0] + 2 * kHaloX + 31) / 32) * 32;
  const int ty = tma_tile_rows(S);
  if (S.n[0] % 4 != 0 || W > 256 || ty == 0 || S.n[0] / 4 * ty > 1024) return false;
  const size_t smem = (size_t)kSlots * (ty + 2 * kN0) * W * 4;
  return smem <= 200 * 1024;
}

int tma_row_width(const SubDev& S) { return ((S.n[0] + 2 * kHaloX + 31) / 32) * 32; }

// out[buf * 2 + {0: 6-row box, 1: TY-row box}] for one subdomain; the device array holds the
// maps of subdomain `sub` at [(sub * 3 + buf) * 2 + k]
bool build_tma_maps(const SubDev& S, int sub, void* const bufs[3], CUtensorMap* out) {
  (void)sub;
  auto enc = get_encode();
  if (!enc) return false;
  const int W = tma_row_width(S), TY = tma_tile_rows(S);
  for (int bi = 0; bi < 3; ++bi) {
    const float* basep = (const float*)bufs[bi] + S.off_blk;
    cuuint64_t dims[4] = {(cuuint64_t)S.n[0], (cuuint64_t)S.n[1], (cuuint64_t)S.n[2], (cuuint64_t)S.ns};
    cuuint64_t strides[3] = {(cuuint64_t)S.n[0] * 4, (cuuint64_t)S.n[0] * S.n[1] * 4, (cuuint64_t)S.nd * 4};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int k = 0; k < 2; ++k) {
      cuuint32_t box[4] = {(cuuint32_t)W, (cuuint32_t)(k == 0 ? kN0 : TY), 1, 1};
      CUresult r = enc(&out[(size_t)bi * 2 + k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)basep, dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
  }
  return true;
}

void launch_stencil_tma(const SubDev* d_subs, const TmaClass& cls, const CUtensorMap* d_maps, int buf_in,
                        const float* Yprev, float* Yout, const float* V, const StepCoef* coef, int step, int* status,
                        cudaStream_t st) {
  if (cls.total == 0) return;
  const size_t smem = (size_t)kSlots * (cls.TY + 2 * kN0) * cls.W * 4;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_stencil_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_stencil_tma, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = true;
  }
  StencilW sw;
  const float ihx = (float)(-0.5 / (cls.h[0] * cls.h[0])), ihy = (float)(-0.5 / (cls.h[1] * cls.h[1])),
              ihz = (float)(-0.5 / (cls.h[2] * cls.h[2]));
  static const double fdw[kN0 + 1] = {-5369.0 / 1800.0, 12.0 / 7.0, -15.0 / 56.0, 10.0 / 189.0,
                                      -1.0 / 112.0,     2.0 / 1925.0, -1.0 / 16632.0};
  for (int p = 0; p <= kN0; ++p) {
    sw.wx[p] = (float)fdw[p] * ihx;
    sw.wy[p] = (float)fdw[p] * ihy;
    sw.wz[p] = (float)fdw[p] * ihz;
  }
  sw.wc = sw.wx[0] + sw.wy[0] + sw.wz[0];
  dim3 block(cls.nq, cls.TY);
  k_stencil_tma<<<cls.total, block, smem, st>>>(d_subs, cls.d_jobs, cls.d_job_off, cls.n_jobs, d_maps, buf_in, Yprev,
                                                Yout, V, coef, step, status, sw);
}

}  // namespace xls
