// TMA-staged FP32 filter step: 12th-order FD Laplacian + local potential + scaled Chebyshev
// recurrence (Sec. 5.A.3 step (1); Sec. 5.B.2 stencil, cache blocking, axis-neighbour reuse).
//
//   Y_out = scale * (-1/2 Delta_h Y_in + V Y_in - c Y_in) - shift * Y_prev
//
// Every operand reaches shared memory by TMA (cp.async.bulk.tensor): the Y_in planes with their
// halo, and the rows of V and Y_prev.  A producer warp keeps a ring of plane slots filled; the
// consumer warps never meet at a block-wide barrier.  The z-direction is a register-resident
// scatter into thirteen plane accumulators, so a plane leaves shared memory as soon as it has
// been read once.  The nonlocal projector terms are added by the projection / back-projection
// launches around this one.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>

#include "xls_internal.h"

namespace xls {

constexpr uint32_t kSuspendNs = 100000;   // suspend-time hint of the barrier waits (100 us)

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

// try_wait with a suspend-time hint: the thread sleeps until the phase completes or the hint
// (in ns) elapses, instead of spinning on the barrier word
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
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

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ int wrapt(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

constexpr int kNS = 5;              // ring slots: planes in flight + the one being read
constexpr int kHaloX = 8;           // halo columns on each side (16-byte aligned TMA x coordinate)
constexpr int kQ = 2 * kN0 + 1;     // output planes accumulating at any time
constexpr int kMaxThreads = 320;    // consumer threads (<= 288) + one producer warp

// Two FP32 values in one 64-bit register (low half = first value), the operand type of the
// packed f32x2 instructions of sm_100 and later: one instruction does the arithmetic of two
// x-points.
using f2 = unsigned long long;
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 pack2(float lo, float hi) {
  f2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void unpack2(f2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}

// Stencil weights of one launch (all subdomains of a launch share the grid spacing), passed by
// value so that the FMAs read them from the constant bank: each packed weight holds the same
// value in both halves; wxs are the scalar x-weights of the odd offsets.
struct StencilW {
  f2 wx[kN0 + 1], wy[kN0 + 1], wz[kN0 + 1];
  f2 wc;
  float wxs[kN0 + 1];
};

// Bounded waits (iteration limit; on expiry the caller records XLS_ETIMEOUT, never a trap).
constexpr int kSpin = 20000;   // x kSuspendNs: a wait gives up after about two seconds
__device__ __forceinline__ bool wait_full(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < kSpin; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// One CTA: TY full-width rows of one vector of one subdomain, marching along z.  A producer
// warp streams, for every plane z_t, three boxes of Y_in (6 halo rows above, TY rows, 6 halo
// rows below, 8 halo columns each side; out-of-range boxes zero-filled = Dirichlet, periodic
// axes wrap the coordinates) plus the TY rows of V at z_t and of Y_prev at z_t - 6 into a ring
// of kNS slots (full/empty mbarriers, no block-wide barrier).  A consumer thread owns four
// consecutive x-points of one row: when plane z_t lands it adds the plane's x/y-stencil, centre
// and potential terms into the accumulator of z_t and scatters w_z[p] * Y(z_t) into the
// accumulators of z_t +- p; the output plane z_t - 6 is then complete and is written out.
// Thirteen accumulators live in registers (the loop is unrolled by 13 so their indices are
// static), two x-points per 64-bit register, and the arithmetic runs on packed f32x2
// instructions (the odd x-offsets, whose partner pairs straddle register pairs, on scalars).
// Along a periodic z axis the six wrapped planes at either end contribute only their
// z-neighbour terms: of those planes only the TY centre rows are loaded.
template <int kW>
__global__ void __launch_bounds__(kMaxThreads, 2)
k_stencil_tma(const SubDev* __restrict__ subs, const TmaJob* __restrict__ jobs, const int* __restrict__ job_off,
              int n_jobs, const CUtensorMap* __restrict__ maps, int buf_in, int buf_prev, float* Yout,
              const StepCoef* __restrict__ coef, int step, int* status, const StencilW sw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kNS], empty[kNS];
  __shared__ volatile int s_abort;
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
  const int TY = J.TY, W = J.W, nq = nx >> 2;
  const int n_cons = blockDim.x - 32;
  const int y0 = yt * TY;
  const int rows = TY + 2 * kN0;
  const int off_yp = rows * W;
  const int aux = ((TY * nx + 31) / 32) * 32;
  const int off_v = off_yp + aux;
  const int slot_floats = off_v + aux;
  float* ring = reinterpret_cast<float*>(smem_raw);
  const bool px = S.periodic[0], py = S.periodic[1], pz = S.periodic[2];
  const int zbase = pz ? -kN0 : 0;
  const int n_iter = nz + kN0 - zbase;  // arrivals z_t = zbase .. nz + 5
  const bool has_prev = buf_prev >= 0;
  const int tid = threadIdx.x;
  const int n_cons_warps = n_cons >> 5;

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < kNS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], n_cons_warps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid >= n_cons) {
    // ---- producer warp ------------------------------------------------------------------
    if (tid != n_cons) return;
    const CUtensorMap* mb = maps + (size_t)J.sub * kMapsPerSub;
    const CUtensorMap* m_halo = mb + buf_in * 3;
    const CUtensorMap* m_in = m_halo + 1;
    const CUtensorMap* m_prev = has_prev ? mb + buf_prev * 3 + 2 : nullptr;
    const CUtensorMap* m_v = mb + 9;
    const int ytop = py ? wrapt(y0 - kN0, ny) : y0 - kN0;
    const int ybot = py ? wrapt(y0 + TY, ny) : y0 + TY;
    const uint32_t in_bytes = (uint32_t)(rows * W) * 4u, aux_bytes = (uint32_t)(TY * nx) * 4u;
    const uint32_t ctr_bytes = (uint32_t)(TY * W) * 4u;
    int issued = 0;
    for (int it = 0; it < n_iter; ++it) {
      const int slot = it % kNS;
      if (it >= kNS) {
        const uint32_t par = (uint32_t)(((it / kNS) - 1) & 1);
        bool ok = false;
        for (int k = 0; k < kSpin && !ok; ++k) {
          ok = mbar_try_wait(&empty[slot], par);
          if (!ok && s_abort) break;
        }
        if (!ok) {
          if (atomicCAS(status, 0, XLS_ETIMEOUT) == 0) status[1] = J.sub;
          s_abort = 1;
          break;
        }
      }
      const int zt = zbase + it;
      const bool real = pz || zt < nz;
      // planes outside [0, n_z) (periodic z only) feed the z-neighbours of the edge planes: their
      // centre rows are all that is read of them
      const bool interior = zt >= 0 && zt < nz;
      const int zo = zt - kN0;
      const bool yp = has_prev && zo >= 0;
      const uint32_t bytes =
          (real ? (interior ? in_bytes + aux_bytes : ctr_bytes) : 0u) + (yp ? aux_bytes : 0u);
      uint64_t* bar = &full[slot];
      float* dst = ring + (size_t)slot * slot_floats;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // every box destination must be 128-byte aligned (the host sizes the slots so); a slot that
      // is not is recorded and left unloaded instead of issuing the copy
      const uint32_t a0 = smem_u32(dst);
      const bool aligned = ((a0 | (a0 + kN0 * W * 4) | (a0 + (kN0 + TY) * W * 4) | (a0 + off_yp * 4) |
                             (a0 + off_v * 4)) & 127u) == 0;
      if (!aligned && atomicCAS(status, 0, XLS_EINVAL) == 0) status[1] = J.sub;
      if (bytes == 0 || !aligned) {
        mbar_arrive(bar);
      } else {
        mbar_expect_tx(bar, bytes);
        if (real) {
          const int zz = pz ? wrapt(zt, nz) : zt;
          tma_load_4d(dst + kN0 * W, m_in, bar, -kHaloX, y0, zz, vec);
          if (interior) {
            tma_load_4d(dst, m_halo, bar, -kHaloX, ytop, zz, vec);
            tma_load_4d(dst + (kN0 + TY) * W, m_halo, bar, -kHaloX, ybot, zz, vec);
            tma_load_3d(dst + off_v, m_v, bar, 0, y0, zz);
          }
        }
        if (yp) tma_load_4d(dst + off_yp, m_prev, bar, 0, y0, zo, vec);
      }
      ++issued;
    }
    // no copy may still be landing when the CTA exits
    for (int it = issued - kNS < 0 ? 0 : issued - kNS; it < issued; ++it)
      wait_full(&full[it % kNS], (uint32_t)((it / kNS) & 1));
    return;
  }

  // ---- consumers ----------------------------------------------------------------------------
  const int lane = tid & 31;
  const bool active = tid < nq * TY;
  const int tx = active ? tid % nq : 0, ty = active ? tid / nq : 0;
  const int x4 = 4 * tx;
  const int y = y0 + ty;
  const bool store_ok = active && y < ny;
  const StepCoef cf = coef[J.sub * kMaxDegree + step];
  const float scale = (float)cf.scale, cshift = (float)cf.c, pshift = (float)cf.shift;
  const f2 scale2 = pack2(scale, scale), ncs2 = pack2(-cshift, -cshift), nps2 = pack2(-pshift, -pshift);
  const int plane_sz = nx * ny;
  float* outp = Yout + S.off_blk + (long long)vec * S.nd + (long long)y * nx + x4;   // advances one plane per output
  const int rc = (ty + kN0) * W + kHaloX + x4;   // this thread's centre in an input slot
  const int ra = ty * nx + x4;                    // ... and in the V / Y_prev boxes
  // x-neighbour chunks of four columns x4 - 8 + 4q .. +3 (wholly inside [0, n_x) or wholly
  // outside, as n_x and x4 are multiples of 4); along a periodic x axis the outside chunks read
  // the wrapped columns of the same row: offsets of chunks 0, 1 (left) and 3, 4 (right).  Of
  // chunks 0 and 4 only the pair next to the centre is within reach of the 6-point stencil.
  const int wl0 = (px && x4 < 8) ? nx : 0, wl1 = (px && x4 < 4) ? nx : 0;
  const int wr3 = (px && x4 + 4 >= nx) ? -nx : 0, wr4 = (px && x4 + 8 >= nx) ? -nx : 0;
  const int Wr = kW ? kW : W;   // row pitch of a slot (compile-time where specialised)

  // accumulators of the 13 output planes in flight, x-points (x4, x4+1) and (x4+2, x4+3)
  f2 acc[kQ][2];
#pragma unroll
  for (int k = 0; k < kQ; ++k) acc[k][0] = acc[k][1] = 0ull;

  int slot = 0;
  uint32_t par = 0;
  const float* P = ring;
  for (int k0 = 0; k0 < n_iter; k0 += kQ) {
#pragma unroll
    for (int j = 0; j < kQ; ++j) {
      const int it = k0 + j;
      if (it >= n_iter) break;
      if (!wait_full(&full[slot], par)) {
        if (atomicCAS(status, 0, XLS_ETIMEOUT) == 0) status[1] = J.sub;
        s_abort = 1;
        return;
      }
      const int zt = zbase + it;
      const int zo = zt - kN0;
      ulonglong2 yp = make_ulonglong2(0ull, 0ull);
      if ((pz || zt < nz) && active) {
        const float* C = P + rc;
        f2 c01, c23;
        if (zt >= 0 && zt < nz) {
          // row of the plane: packed pairs x[k], k = 2..17 relative to x4 - 8 (centre at 8..11)
          const f2 x2 = *reinterpret_cast<const f2*>(C - 6 + wl0);
          const ulonglong2 x4v = *reinterpret_cast<const ulonglong2*>(C - 4 + wl1);
          const ulonglong2 x8v = *reinterpret_cast<const ulonglong2*>(C);
          const ulonglong2 x12v = *reinterpret_cast<const ulonglong2*>(C + 4 + wr3);
          const f2 x16 = *reinterpret_cast<const f2*>(C + 8 + wr4);
          const ulonglong2 vp = *reinterpret_cast<const ulonglong2*>(P + off_v + ra);
          c01 = x8v.x;
          c23 = x8v.y;
          // centre and potential: (V - c) y + w_c y
          f2 t01 = fma2(add2(vp.x, ncs2), c01, mul2(sw.wc, c01));
          f2 t23 = fma2(add2(vp.y, ncs2), c23, mul2(sw.wc, c23));
          // even x-offsets: both partners of a pair are aligned pairs
          t01 = fma2(sw.wx[2], add2(x8v.y, x4v.y), t01);
          t23 = fma2(sw.wx[2], add2(x12v.x, x8v.x), t23);
          t01 = fma2(sw.wx[4], add2(x12v.x, x4v.x), t01);
          t23 = fma2(sw.wx[4], add2(x12v.y, x4v.y), t23);
          t01 = fma2(sw.wx[6], add2(x12v.y, x2), t01);
          t23 = fma2(sw.wx[6], add2(x16, x4v.x), t23);
          // odd x-offsets on scalars
          float x[20];
          unpack2(x2, x[2], x[3]);
          unpack2(x4v.x, x[4], x[5]);
          unpack2(x4v.y, x[6], x[7]);
          unpack2(x8v.x, x[8], x[9]);
          unpack2(x8v.y, x[10], x[11]);
          unpack2(x12v.x, x[12], x[13]);
          unpack2(x12v.y, x[14], x[15]);
          unpack2(x16, x[16], x[17]);
          float o[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) o[r] = sw.wxs[1] * (x[9 + r] + x[7 + r]);
#pragma unroll
          for (int p = 3; p <= kN0; p += 2)
#pragma unroll
            for (int r = 0; r < 4; ++r) o[r] = fmaf(sw.wxs[p], x[8 + r + p] + x[8 + r - p], o[r]);
          // y-neighbours
#pragma unroll
          for (int p = 1; p <= kN0; ++p) {
            const ulonglong2 up = *reinterpret_cast<const ulonglong2*>(C + p * Wr);
            const ulonglong2 dn = *reinterpret_cast<const ulonglong2*>(C - p * Wr);
            t01 = fma2(sw.wy[p], add2(up.x, dn.x), t01);
            t23 = fma2(sw.wy[p], add2(up.y, dn.y), t23);
          }
          acc[j][0] = add2(acc[j][0], add2(t01, pack2(o[0], o[1])));
          acc[j][1] = add2(acc[j][1], add2(t23, pack2(o[2], o[3])));
        } else {
          // a plane beyond the z-ends (periodic z): only its z-neighbour contributions count
          const ulonglong2 cv = *reinterpret_cast<const ulonglong2*>(C);
          c01 = cv.x;
          c23 = cv.y;
        }
#pragma unroll
        for (int p = 1; p <= kN0; ++p) {
          const int u = (j + p) % kQ, d = (j + kQ - p) % kQ;
          acc[u][0] = fma2(sw.wz[p], c01, acc[u][0]);
          acc[u][1] = fma2(sw.wz[p], c23, acc[u][1]);
          acc[d][0] = fma2(sw.wz[p], c01, acc[d][0]);
          acc[d][1] = fma2(sw.wz[p], c23, acc[d][1]);
        }
      }
      if (has_prev && zo >= 0 && active) yp = *reinterpret_cast<const ulonglong2*>(P + off_yp + ra);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
      if (++slot == kNS) {
        slot = 0;
        par ^= 1u;
        P = ring;
      } else {
        P += slot_floats;
      }
      // output plane z_t - 6 is complete
      const int f = (j + kQ - kN0) % kQ;
      if (zo >= 0 && store_ok)
        *reinterpret_cast<ulonglong2*>(outp) =
            make_ulonglong2(fma2(nps2, yp.x, mul2(scale2, acc[f][0])), fma2(nps2, yp.y, mul2(scale2, acc[f][1])));
      if (zo >= 0) outp += plane_sz;
      acc[f][0] = acc[f][1] = 0ull;
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

// rows per tile: the largest candidate with at most 288 consumer threads (x-points / 4 per row)
// that, along a periodic y axis, divides n_y (the wrapped halo boxes then start exactly at the
// tile edges); XLS_STENCIL_TY (24, 16, 12, 8 or 6) asks for a smaller eligible candidate
static bool ty_ok(const SubDev& S, int ty) {
  return (S.n[0] / 4) * ty <= kMaxThreads - 32 && (!S.periodic[1] || S.n[1] % ty == 0);
}
int tma_tile_rows(const SubDev& S) {
  static const int want = std::getenv("XLS_STENCIL_TY") ? std::atoi(std::getenv("XLS_STENCIL_TY")) : 0;
  int first = 0;
  for (int ty : {24, 16, 12, 8, 6})
    if (ty_ok(S, ty)) {
      if (!first) first = ty;
      if (ty == want) return ty;
    }
  return first;
}

// Shared-memory wavefronts of one plane's y-neighbour loads (16-byte loads of consecutive rows
// at pitch W, nq threads per row, TY rows) by the four 8-lane phases of every warp: a phase
// needs as many wavefronts as the most 16-byte chunks it puts into one bank group.
static long long smem_wavefronts(int W, int nq, int TY) {
  const int n = nq * TY;
  long long waves = 0;
  for (int w0 = 0; w0 < n; w0 += 32)
    for (int ph = 0; ph < 4; ++ph) {
      int per_bank[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // 16-byte bank groups of a 128-byte line
      int addr[8];
      int k = 0;
      for (int l = 0; l < 8; ++l) {
        const int t = w0 + ph * 8 + l;
        if (t >= n) break;
        const int word = (t / nq) * W + kHaloX + 4 * (t % nq);
        bool dup = false;
        for (int j = 0; j < k; ++j) dup = dup || addr[j] == word;
        if (dup) continue;
        addr[k++] = word;
        per_bank[(word / 4) % 8]++;
      }
      int m = 0;
      for (int b = 0; b < 8; ++b) m = per_bank[b] > m ? per_bank[b] : m;
      waves += m;
    }
  return waves;
}

// Row pitch of a plane slot: at least n_x + 16 (8 halo columns each side) and a multiple of 16
// floats, so that with an even tile height every TMA box lands on a 128-byte aligned shared-memory
// address (6 W, (6 + TY) W and (12 + TY) W floats are multiples of 32); among the pitches up to
// 32 floats wider, the one whose y-loads need the fewest shared-memory wavefronts (columns beyond
// the halo are out of range for the TMA box and cost no memory traffic).
int tma_row_width(const SubDev& S) {
  const int nq = S.n[0] / 4;
  const int ty = tma_tile_rows(S);
  const int w0 = ((S.n[0] + 2 * kHaloX + 15) / 16) * 16;
  // XLS_STENCIL_W asks for one of the candidate pitches (w0, w0 + 16, w0 + 32)
  static const int want_w = std::getenv("XLS_STENCIL_W") ? std::atoi(std::getenv("XLS_STENCIL_W")) : 0;
  if (want_w >= w0 && want_w <= w0 + 32 && want_w <= 256 && (want_w - w0) % 16 == 0) return want_w;
  int best = w0;
  long long best_w = -1;
  for (int W = w0; W <= w0 + 32 && W <= 256; W += 16) {
    const long long f = ty ? smem_wavefronts(W, nq, ty) : 0;
    if (best_w < 0 || f < best_w) {
      best_w = f;
      best = W;
    }
  }
  return best;
}

size_t tma_smem_bytes(int TY, int W, int nx) {
  const size_t aux = ((size_t)(TY * nx) + 31) / 32 * 32;
  return (size_t)kNS * ((size_t)(TY + 2 * kN0) * W + 2 * aux) * 4;
}

bool tma_eligible(const SubDev& S) {
  const int W = tma_row_width(S);
  const int ty = tma_tile_rows(S);
  if (S.n[0] % 4 != 0 || W > 256 || ty == 0) return false;
  // every box destination 128-byte aligned: 6 W, (6 + TY) W, (12 + TY) W floats multiples of 32
  if ((6 * W) % 32 || ((6 + ty) * W) % 32 || ((12 + ty) * W) % 32) return false;
  return tma_smem_bytes(ty, W, S.n[0]) <= 200 * 1024;
}

// Maps of one subdomain, kMapsPerSub of them: for each of the three blocks, [halo box (6 rows x
// W), interior box (TY rows x W), auxiliary box (TY rows x n_x)], then the potential's box
// (TY rows x n_x of the FP32 V).
bool build_tma_maps(const SubDev& S, const float* Vf, void* const bufs[3], CUtensorMap* out) {
  auto enc = get_encode();
  if (!enc) return false;
  const int W = tma_row_width(S), TY = tma_tile_rows(S);
  cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int bi = 0; bi < 3; ++bi) {
    const float* basep = (const float*)bufs[bi] + S.off_blk;
    cuuint64_t dims[4] = {(cuuint64_t)S.n[0], (cuuint64_t)S.n[1], (cuuint64_t)S.n[2], (cuuint64_t)S.ns};
    cuuint64_t strides[3] = {(cuuint64_t)S.n[0] * 4, (cuuint64_t)S.n[0] * S.n[1] * 4, (cuuint64_t)S.nd * 4};
    for (int k = 0; k < 3; ++k) {
      cuuint32_t box[4] = {(cuuint32_t)(k == 2 ? S.n[0] : W), (cuuint32_t)(k == 0 ? kN0 : TY), 1, 1};
      CUresult r = enc(&out[(size_t)bi * 3 + k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)basep, dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
  }
  cuuint64_t dims[3] = {(cuuint64_t)S.n[0], (cuuint64_t)S.n[1], (cuuint64_t)S.n[2]};
  cuuint64_t strides[2] = {(cuuint64_t)S.n[0] * 4, (cuuint64_t)S.n[0] * S.n[1] * 4};
  cuuint32_t box[3] = {(cuuint32_t)S.n[0], (cuuint32_t)TY, 1};
  CUresult r = enc(&out[9], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)(Vf + S.off_pt), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int kW>
static void launch_variant(const TmaClass& cls, size_t smem, const SubDev* d_subs, const CUtensorMap* d_maps,
                           int buf_in, int buf_prev, float* Yout, const StepCoef* coef, int step, int* status,
                           const StencilW& sw, cudaStream_t st) {
  // function attributes are per device: set at every launch (a host call of a few microseconds)
  cudaFuncSetAttribute(k_stencil_tma<kW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_stencil_tma<kW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  const int threads = ((cls.nq * cls.TY + 31) / 32) * 32 + 32;
  k_stencil_tma<kW><<<cls.total, threads, smem, st>>>(d_subs, cls.d_jobs, cls.d_job_off, cls.n_jobs, d_maps, buf_in,
                                                      buf_prev, Yout, coef, step, status, sw);
}

void launch_stencil_tma(const SubDev* d_subs, const TmaClass& cls, const CUtensorMap* d_maps, int buf_in,
                        int buf_prev, float* Yout, const StepCoef* coef, int step, int* status, cudaStream_t st) {
  if (cls.total == 0) return;
  const size_t smem = tma_smem_bytes(cls.TY, cls.W, cls.nq * 4);
  StencilW sw;
  const float ihx = (float)(-0.5 / (cls.h[0] * cls.h[0])), ihy = (float)(-0.5 / (cls.h[1] * cls.h[1])),
              ihz = (float)(-0.5 / (cls.h[2] * cls.h[2]));
  static const double fdw[kN0 + 1] = {-5369.0 / 1800.0, 12.0 / 7.0, -15.0 / 56.0, 10.0 / 189.0,
                                      -1.0 / 112.0,     2.0 / 1925.0, -1.0 / 16632.0};
  auto both = [](float v) {
    uint32_t u;
    memcpy(&u, &v, 4);
    return ((f2)u << 32) | u;
  };
  for (int p = 0; p <= kN0; ++p) {
    sw.wxs[p] = (float)fdw[p] * ihx;
    sw.wx[p] = both(sw.wxs[p]);
    sw.wy[p] = both((float)fdw[p] * ihy);
    sw.wz[p] = both((float)fdw[p] * ihz);
  }
  sw.wc = both((float)fdw[0] * ihx + (float)fdw[0] * ihy + (float)fdw[0] * ihz);
  // row pitches of the common subdomain widths as compile-time constants (immediate offsets),
  // unless the class asks for the runtime pitch (xls_autotune times both)
  switch (cls.rt_pitch ? 0 : cls.W) {
    case 80: launch_variant<80>(cls, smem, d_subs, d_maps, buf_in, buf_prev, Yout, coef, step, status, sw, st); break;
    case 112: launch_variant<112>(cls, smem, d_subs, d_maps, buf_in, buf_prev, Yout, coef, step, status, sw, st); break;
    default: launch_variant<0>(cls, smem, d_subs, d_maps, buf_in, buf_prev, Yout, coef, step, status, sw, st);
  }
}

}  // namespace xls
