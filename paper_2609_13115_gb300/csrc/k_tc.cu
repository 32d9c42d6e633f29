// Tensor-core subspace contractions of the mixed path (Sec. 5.A.3 steps (2) and (4); the
// paper's projection DGEMM/DSYRK and rotation DGEMM of Sec. 5.B.3), on 5th-generation tensor
// cores: tcgen05.mma kind::f16 with BF16 operands and FP32 accumulators in tensor memory.
//
// Split-BF16 products: every FP32 operand x is written as hi + lo with hi = bf16(x) and
// lo = bf16(x - hi); a product a b is taken as a_hi b_hi + a_hi b_lo + a_lo b_hi (the lo*lo term,
// below 2^-16 relative, is dropped), all three accumulated in the same FP32 TMEM accumulator.
//
// Data flow of both kernels: eight producer warps read FP32 tiles from HBM with 16-byte loads,
// split them and store hi and lo tiles in shared memory in the UMMA canonical 128-byte-swizzled
// layout; after a proxy fence they arrive on the stage's "full" mbarrier.  One thread of a ninth
// warp issues the MMAs of a stage and commits them to the stage's "empty" mbarrier, which the
// producers wait on before refilling it (two stages).  A final commit releases the epilogue,
// in which the producer warps read the accumulators with tcgen05.ld.
//
//   Gram:     D1 = Psi_f[I]^T Psi_f[J], D2 = Psi_f[I]^T (H Psi_f)[J] over a chunk of grid points,
//             for the upper block triangle (I <= J) of 128 x 128 blocks; FP32 partial sums of the
//             chunks go to a workspace that k_gram_reduce sums (FP64) into M_s, H_s, mirroring
//             the off-diagonal blocks.
//   Rotation: Psi[n][g] = sum_k Psi_f[k][g] Y[k][n] for a tile of 128 grid points, A = Psi_f
//             (MN-major: grid points contiguous), B = Y^T (K-major, pre-split hi/lo in HBM).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "xls_internal.h"

namespace xls {
namespace tc {

constexpr int kThreads = 288;      // 8 producer/epilogue warps + 1 MMA warp
constexpr int kProducers = 256;
constexpr int kKT = 64;            // K elements per tile (128-byte bf16 rows)
constexpr int kStages = 2;
constexpr long long kSpin = 1LL << 26;  // bounded mbarrier waits
// Tensor-core FP32 accumulation does not round to nearest; its error grows with the number of
// MMAs added into one accumulator.  The Gram kernels therefore read their accumulators out every
// kFlush K tiles (12 * kFlush MMAs) into FP32 partial sums with round-to-nearest adds.
constexpr int kFlush = 4;
constexpr int kFlushGram = 8;   // flush period of the batched Gram (k_gram_tc): 96 MMAs per accumulator

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(su32(b)), "r"(parity)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
  for (long long i = 0; i < kSpin; ++i)
    if (bar_try(b, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst_smem)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, M = 128, N from idesc, K = 16
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// 32 lanes x 32 bit, 16 consecutive columns per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 32 bit, 32 consecutive columns per thread (no wait: the caller issues
// tcgen05.wait::ld after overlapping other loads)
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t r[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
// A major (bit 15), B K-major (bit 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
// (A = B = F16: type code 0 in bits 7-9 and 10-12)
__host__ __device__ constexpr uint32_t idesc_16(int M, int N, bool a_mn_major, bool fp16) {
  return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) | ((a_mn_major ? 1u : 0u) << 15) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor, 128-byte swizzle: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), version 1 (46-47), layout 2 (61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (2ull << 61);
}

// K-major 128B-swizzled tile: row r (128 bytes = 64 bf16 of K), 16-byte chunk c
__device__ __forceinline__ uint32_t kmaj_off(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }
// MN-major 128B-swizzled tile of 128 MN x 64 K: MN group m (64 elements), K row k, chunk c of 8 MN
// elements; K groups of 8 rows 1024 bytes apart (SBO), MN groups 8192 bytes apart (LBO)
__device__ __forceinline__ uint32_t mnmaj_off(int m, int k, int c) {
  return (uint32_t)(m * 8192 + (k >> 3) * 1024 + (k & 7) * 128 + ((c ^ (k & 7)) << 4));
}

// hi = r(s x), lo = r(s x - hi) with r = round-to-nearest bf16 (kFp16 = false) or fp16 (true);
// s is a power of two (exact), 1 on the BF16 path
template <bool kFp16>
__device__ __forceinline__ void split1(float x, uint16_t& h, uint16_t& l) {
  if (kFp16) {
    const __half hh = __float2half_rn(x);
    h = __half_as_ushort(hh);
    l = __half_as_ushort(__float2half_rn(x - __half2float(hh)));
  } else {
    const __nv_bfloat16 hh = __float2bfloat16_rn(x);
    h = __bfloat16_as_ushort(hh);
    l = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hh)));
  }
}

template <bool kFp16>
__device__ __forceinline__ void split8(const float4 a, const float4 b, float s, uint4& hi, uint4& lo) {
  const float x[8] = {a.x * s, a.y * s, a.z * s, a.w * s, b.x * s, b.y * s, b.z * s, b.w * s};
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint16_t h0, h1, l0, l1;
    split1<kFp16>(x[2 * i], h0, l0);
    split1<kFp16>(x[2 * i + 1], h1, l1);
    h[i] = (uint32_t)h0 | ((uint32_t)h1 << 16);
    l[i] = (uint32_t)l0 | ((uint32_t)l1 << 16);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void sts128(uint32_t saddr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(saddr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// ---------------------------------------------------------------------------------------------
// Gram: one CTA = (subdomain, block (I, J), chunk of K tiles)
// stage layout (bytes): A_hi 16K, A_lo 16K, B1_hi 16K, B1_lo 16K, B2_hi 16K, B2_lo 16K
constexpr uint32_t kTile = 128 * 128;        // one 128-row x 128-byte tile
constexpr uint32_t kGramStage = 6 * kTile;

template <bool kFp16>
__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc(const SubDev* __restrict__ subs, const GramJob* __restrict__ jobs, const float* __restrict__ F,
          const float* __restrict__ HF, const int* __restrict__ ex_f, const int* __restrict__ ex_hf,
          float* __restrict__ work, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const GramJob J = jobs[blockIdx.x];
  const SubDev& S = subs[J.sub];
  const int ns = S.ns;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = 128 * J.I, j0 = 128 * J.J;
  const int nj = min(128, ns - j0);
  const int nj16 = (nj + 15) & ~15;
  const bool diag = (J.I == J.J);
  const int nkt = J.kt1 - J.kt0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&full[s], kProducers / 2);   // one producer group per stage
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&acc_full[b], 1);
      bar_init(&acc_empty[b], kProducers);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) tmem_alloc(&s_tmem, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = su32(smem);
  const float* f = F + S.off_blk;
  const float* hf = HF + S.off_blk;

  // Read the accumulators of flush period p (buffer p % 2, D1 at +0, D2 at +128 columns) and add
  // them to the CTA's FP32 partial sums with round-to-nearest adds (the first period stores).
  const int lg = warp & 3, out_m = warp >> 2, prow = lg * 32 + lane;
  float* wrow = work + (long long)blockIdx.x * 2 * 128 * 128 + (long long)out_m * 128 * 128 + (long long)prow * 128;
  // The first period stores, later periods add with fire-and-forget vector reductions in L2
  // (round-to-nearest FP32 adds, in program order per address: one thread owns each row).
  auto flush = [&](int p) {
    const int b = p & 1;
    const bool ok = bar_wait(&acc_full[b], (p >> 1) & 1);
    tc_fence_after();
    if (!ok) atomicExch(&s_fail, 1);
    for (int c0 = 0; c0 < nj16; c0 += 32) {
      uint32_t r[32];
      tmem_ld32_nowait(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * 256 + out_m * 128 + c0), r);
      tmem_wait_ld();
      if (ok) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (c0 + 4 * u >= nj16) break;
          const float4 o = make_float4(__uint_as_float(r[4 * u]), __uint_as_float(r[4 * u + 1]),
                                       __uint_as_float(r[4 * u + 2]), __uint_as_float(r[4 * u + 3]));
          float4* dst = reinterpret_cast<float4*>(wrow + c0 + 4 * u);
          if (p == 0) *dst = o;
          else atomicAdd(dst, o);
        }
      }
    }
    tc_fence_before();
    bar_arrive(&acc_empty[b]);
  };
  if (warp < 8) {
    // ---------------- producers: two groups of four warps, group g fills stage g with the K tiles
    // it = g (mod 2), so that two tiles are in flight; both groups flush every period (group 0 the
    // D1 accumulator rows, group 1 the D2 rows)
    const int grp = warp >> 2, gt = threadIdx.x & 127;
    const int rowsB1 = diag ? 0 : nj16;
    const int nrows = 128 + rowsB1 + nj16;     // A rows, B1 rows, B2 rows
    bool go = true;
    for (int p = 0; p * kFlushGram < nkt; ++p) {
      const int t_end = min((p + 1) * kFlushGram, nkt);
      for (int it = p * kFlushGram + grp; go && it < t_end; it += 2) {
        const long long k0 = (long long)(J.kt0 + it) * kKT;
        const uint32_t stage = sbase + grp * kGramStage;
        // rounds of 8 items (row, 8-element chunk) per thread: the global loads of a round (and the
        // rows' scale exponents) are issued before any item is split and stored, so that their
        // latencies overlap; the wait for the stage to be free comes after the first round's loads
        constexpr int kItems = 8;
        for (int q0 = 0; q0 < nrows * 8; q0 += 128 * kItems) {
          float4 a[kItems], b[kItems];
          int ex[kItems];
#pragma unroll
          for (int u = 0; u < kItems; ++u) {
            const int q = q0 + gt + u * 128;
            a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            b[u] = a[u];
            ex[u] = 0;
            if (q >= nrows * 8) continue;
            const int row = q >> 3, c = q & 7;
            const bool isA = row < 128, isB1 = !isA && row < 128 + rowsB1;
            const int r = isA ? row : (isB1 ? row - 128 : row - 128 - rowsB1);
            const int grow = isA ? i0 + r : j0 + r;
            const bool valid = isA ? (grow < ns) : (r < nj);
            const long long kk = k0 + c * 8;
            if (valid && kk < S.nd) {
              const float4* src = reinterpret_cast<const float4*>((isA || isB1 ? f : hf) + (long long)grow * S.nd + kk);
              a[u] = src[0];
              b[u] = src[1];
            }
            if (kFp16 && valid) ex[u] = (isA || isB1 ? ex_f : ex_hf)[S.off_state + grow];
          }
          if (q0 == 0 && it >= 2 && !bar_wait(&empty[grp], ((it >> 1) - 1) & 1)) {
            atomicExch(&s_fail, 1);
            go = false;
            break;
          }
#pragma unroll
          for (int u = 0; u < kItems; ++u) {
            const int q = q0 + gt + u * 128;
            if (q >= nrows * 8) continue;
            const int row = q >> 3, c = q & 7;
            const bool isA = row < 128, isB1 = !isA && row < 128 + rowsB1;
            const int r = isA ? row : (isB1 ? row - 128 : row - 128 - rowsB1);
            const uint32_t thi = isA ? stage : (isB1 ? stage + 2 * kTile : stage + 4 * kTile);
            const float sc = kFp16 ? ldexpf(1.f, ex[u]) : 1.f;
            uint4 hi, lo;
            split8<kFp16>(a[u], b[u], sc, hi, lo);
            const uint32_t off = kmaj_off(r, c);
            sts128(thi + off, hi);
            sts128(thi + kTile + off, lo);
          }
        }
        if (!go) break;
        fence_async_smem();
        bar_arrive(&full[grp]);
      }
      if (!go) break;
      flush(p);
    }
  } else if (lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_16(128, nj16, false, kFp16);
    bool ok = true;
    for (int it = 0; it < nkt; ++it) {
      const int st = it % kStages;
      if (!bar_wait(&full[st], (it / kStages) & 1)) { ok = false; break; }
      const int per = it / kFlushGram, buf = per & 1;
      if (it % kFlushGram == 0 && per >= 2 && !bar_wait(&acc_empty[buf], ((per >> 1) - 1) & 1)) { ok = false; break; }
      tc_fence_after();
      const uint32_t acc_base = tmem + (uint32_t)(buf * 256);
      const uint32_t stage = sbase + st * kGramStage;
      const uint32_t a_hi = stage, a_lo = stage + kTile;
      const uint32_t b1_hi = diag ? a_hi : stage + 2 * kTile, b1_lo = diag ? a_lo : stage + 3 * kTile;
      const uint32_t b2_hi = stage + 4 * kTile, b2_lo = stage + 5 * kTile;
#pragma unroll
      for (int ks = 0; ks < kKT / 16; ++ks) {
        const uint32_t ko = ks * 32;           // 16 bf16 = 32 bytes along K inside the swizzle row
        const int acc = (it % kFlushGram > 0 || ks > 0) ? 1 : 0;
        const uint64_t ah = sdesc(a_hi + ko, 16, 1024), al = sdesc(a_lo + ko, 16, 1024);
        mma_bf16(acc_base + 0, ah, sdesc(b1_hi + ko, 16, 1024), idesc, acc);
        mma_bf16(acc_base + 0, ah, sdesc(b1_lo + ko, 16, 1024), idesc, 1);
        mma_bf16(acc_base + 0, al, sdesc(b1_hi + ko, 16, 1024), idesc, 1);
        mma_bf16(acc_base + 128, ah, sdesc(b2_hi + ko, 16, 1024), idesc, acc);
        mma_bf16(acc_base + 128, ah, sdesc(b2_lo + ko, 16, 1024), idesc, 1);
        mma_bf16(acc_base + 128, al, sdesc(b2_hi + ko, 16, 1024), idesc, 1);
      }
      mma_commit(&empty[st]);
      if (it % kFlushGram == kFlushGram - 1 || it == nkt - 1) mma_commit(&acc_full[buf]);
    }
    if (!ok) atomicExch(&s_fail, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 8) tmem_dealloc(tmem, 512);
  if (threadIdx.x == 0 && s_fail) atomicCAS(status, 0, XLS_ETIMEOUT);
}

// Sum the K-chunk partials of every block into M_s, H_s (FP64) and mirror off-diagonal blocks.
__global__ void __launch_bounds__(256)
k_gram_reduce(const SubDev* __restrict__ subs, const GramJob* __restrict__ jobs, const int* __restrict__ grp_first,
              const int* __restrict__ grp_n, const float* __restrict__ work, const int* __restrict__ ex_f,
              const int* __restrict__ ex_hf, double* Ms, double* Hs) {
  const int gi = blockIdx.y;  // group = (subdomain, block)
  const int first = grp_first[gi], cnt = grp_n[gi];
  const GramJob J = jobs[first];
  const SubDev& S = subs[J.sub];
  const int ns = S.ns;
  const int i0 = 128 * J.I, j0 = 128 * J.J;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128 * 128; e += gridDim.x * blockDim.x) {
    const int r = e / 128, c = e % 128;
    const int i = i0 + r, j = j0 + c;
    if (i >= ns || j >= ns) continue;
    // compensated FP32 sums of the K-chunk partials (FP32 adds: the FP64 pipe is a few percent of
    // the FP32 one); the sum and its running error are combined in FP64
    float ms = 0.f, mc = 0.f, hs = 0.f, hc = 0.f;
    for (int q = 0; q < cnt; ++q) {
      const float* w = work + (long long)(first + q) * 2 * 128 * 128;
      const float ym = w[e] - mc, yh = w[128 * 128 + e] - hc;
      const float tm = ms + ym, th = hs + yh;
      mc = (tm - ms) - ym;
      hc = (th - hs) - yh;
      ms = tm;
      hs = th;
    }
    double m = (double)ms - (double)mc, h = (double)hs - (double)hc;
    if (ex_f) {  // undo the power-of-two row scales of the FP16 split
      const int ei = ex_f[S.off_state + i];
      m = ldexp(m, -(ei + ex_f[S.off_state + j]));
      h = ldexp(h, -(ei + ex_hf[S.off_state + j]));
    }
    Ms[S.off_ss + (long long)i * ns + j] = m;
    Hs[S.off_ss + (long long)i * ns + j] = h;
    if (J.I != J.J) {
      Ms[S.off_ss + (long long)j * ns + i] = m;
      Hs[S.off_ss + (long long)j * ns + i] = h;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Gram of one block of vectors with caller-provided scratch (the allocation-free entry point):
// the same split-BF16 computation as k_gram_tc for a single block F, HF (n_states x n_points,
// vector-major); CTA b handles block pair b / kc and K chunk b % kc; the FP32 partial sums go to
// `work` ([jobs][2][128][128]), which k_gram_reduce_single sums into M_s, H_s.
__device__ __forceinline__ void single_job(int b, int ns, long long nd, int kc, int& I, int& J, int& kt0, int& kt1) {
  const int pair = b / kc, chunk = b % kc;
  const int nt = (ns + 127) / 128;
  I = 0;
  J = pair;
  if (nt == 2) {
    I = pair == 2 ? 1 : 0;
    J = pair == 0 ? 0 : 1;
  }
  const long long nkt = (nd + kKT - 1) / kKT;
  kt0 = (int)(nkt * chunk / kc);
  kt1 = (int)(nkt * (chunk + 1) / kc);
}

__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc_single(const float* __restrict__ f, const float* __restrict__ hf, long long nd, int ns, int kc,
                 float* __restrict__ work, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  int JI, JJ, kt0, kt1;
  single_job(blockIdx.x, ns, nd, kc, JI, JJ, kt0, kt1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = 128 * JI, j0 = 128 * JJ;
  const int nj = min(128, ns - j0);
  const int nj16 = (nj + 15) & ~15;
  const bool diag = (JI == JJ);
  const int nkt = kt1 - kt0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&full[s], kProducers);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&acc_full[b], 1);
      bar_init(&acc_empty[b], kProducers);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) tmem_alloc(&s_tmem, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = su32(smem);
  // Read the accumulators of flush period p (buffer p % 2, D1 at +0, D2 at +128 columns) and add
  // them to the CTA's FP32 partial sums with round-to-nearest adds (the first period stores).
  const int lg = warp & 3, out_m = warp >> 2, prow = lg * 32 + lane;
  float* wrow = work + (long long)blockIdx.x * 2 * 128 * 128 + (long long)out_m * 128 * 128 + (long long)prow * 128;
  auto flush = [&](int p) {
    const int b = p & 1;
    const bool ok = bar_wait(&acc_full[b], (p >> 1) & 1);
    tc_fence_after();
    if (!ok) atomicExch(&s_fail, 1);
    for (int c0 = 0; c0 < nj16; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * 256 + out_m * 128 + c0), v);
      if (ok) {
#pragma unroll
        for (int u = 0; u < 16; u += 4) {
          float4* dst = reinterpret_cast<float4*>(wrow + c0 + u);
          float4 o = make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
          if (p > 0) {
            const float4 q = *dst;
            o.x += q.x; o.y += q.y; o.z += q.z; o.w += q.w;
          }
          *dst = o;
        }
      }
    }
    tc_fence_before();
    bar_arrive(&acc_empty[b]);
  };
  if (warp < 8) {
    const int rowsB1 = diag ? 0 : nj16;
    const int nrows = 128 + rowsB1 + nj16;
    for (int it = 0; it < nkt; ++it) {
      const int st = it % kStages;
      if (it >= kStages && !bar_wait(&empty[st], ((it / kStages) - 1) & 1)) { atomicExch(&s_fail, 1); break; }
      const long long k0 = (long long)(kt0 + it) * kKT;
      const uint32_t stage = sbase + st * kGramStage;
      for (int q = threadIdx.x; q < nrows * 8; q += kProducers) {
        const int row = q >> 3, c = q & 7;
        const float* src;
        int grow, r;
        uint32_t thi, tlo;
        if (row < 128) {
          r = row; grow = i0 + r; src = f; thi = stage; tlo = stage + kTile;
        } else if (row < 128 + rowsB1) {
          r = row - 128; grow = j0 + r; src = f; thi = stage + 2 * kTile; tlo = stage + 3 * kTile;
        } else {
          r = row - 128 - rowsB1; grow = j0 + r; src = hf; thi = stage + 4 * kTile; tlo = stage + 5 * kTile;
        }
        const bool valid = (row < 128) ? (grow < ns) : (r < nj);
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        const long long kk = k0 + c * 8;
        if (valid && kk < nd) {
          const float4* p = reinterpret_cast<const float4*>(src + (long long)grow * nd + kk);
          a = p[0];
          b = p[1];
        }
        uint4 hi, lo;
        split8<false>(a, b, 1.f, hi, lo);
        const uint32_t off = kmaj_off(r, c);
        sts128(thi + off, hi);
        sts128(tlo + off, lo);
      }
      fence_async_smem();
      bar_arrive(&full[st]);
      if (it % kFlush == kFlush - 1 || it == nkt - 1) flush(it / kFlush);
    }
  } else if (lane == 0) {
    const uint32_t idesc = idesc_16(128, nj16, false, false);
    bool ok = true;
    for (int it = 0; it < nkt; ++it) {
      const int st = it % kStages;
      if (!bar_wait(&full[st], (it / kStages) & 1)) { ok = false; break; }
      const int per = it / kFlush, buf = per & 1;
      if (it % kFlush == 0 && per >= 2 && !bar_wait(&acc_empty[buf], ((per >> 1) - 1) & 1)) { ok = false; break; }
      tc_fence_after();
      const uint32_t acc_base = tmem + (uint32_t)(buf * 256);
      const uint32_t stage = sbase + st * kGramStage;
      const uint32_t a_hi = stage, a_lo = stage + kTile;
      const uint32_t b1_hi = diag ? a_hi : stage + 2 * kTile, b1_lo = diag ? a_lo : stage + 3 * kTile;
      const uint32_t b2_hi = stage + 4 * kTile, b2_lo = stage + 5 * kTile;
#pragma unroll
      for (int ks = 0; ks < kKT / 16; ++ks) {
        const uint32_t ko = ks * 32;
        const int acc = (it % kFlush > 0 || ks > 0) ? 1 : 0;
        const uint64_t ah = sdesc(a_hi + ko, 16, 1024), al = sdesc(a_lo + ko, 16, 1024);
        mma_bf16(acc_base + 0, ah, sdesc(b1_hi + ko, 16, 1024), idesc, acc);
        mma_bf16(acc_base + 0, ah, sdesc(b1_lo + ko, 16, 1024), idesc, 1);
        mma_bf16(acc_base + 0, al, sdesc(b1_hi + ko, 16, 1024), idesc, 1);
        mma_bf16(acc_base + 128, ah, sdesc(b2_hi + ko, 16, 1024), idesc, acc);
        mma_bf16(acc_base + 128, ah, sdesc(b2_lo + ko, 16, 1024), idesc, 1);
        mma_bf16(acc_base + 128, al, sdesc(b2_hi + ko, 16, 1024), idesc, 1);
      }
      mma_commit(&empty[st]);
      if (it % kFlush == kFlush - 1 || it == nkt - 1) mma_commit(&acc_full[buf]);
    }
    if (!ok) atomicExch(&s_fail, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 8) tmem_dealloc(tmem, 512);
  if (threadIdx.x == 0 && s_fail) atomicCAS(status, 0, XLS_ETIMEOUT);
}

// M_s, H_s (n_states x n_states, FP64, row-major) from the partial sums of k_gram_tc_single
__global__ void __launch_bounds__(256)
k_gram_reduce_single(const float* __restrict__ work, int ns, long long nd, int kc, double* Ms, double* Hs) {
  const int pair = blockIdx.y;
  int I, J, kt0, kt1;
  single_job(pair * kc, ns, nd, kc, I, J, kt0, kt1);
  const int i0 = 128 * I, j0 = 128 * J;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128 * 128; e += gridDim.x * blockDim.x) {
    const int i = i0 + e / 128, j = j0 + e % 128;
    if (i >= ns || j >= ns) continue;
    double m = 0.0, h = 0.0;
    for (int q = 0; q < kc; ++q) {
      const float* w = work + (long long)(pair * kc + q) * 2 * 128 * 128;
      m += (double)w[e];
      h += (double)w[128 * 128 + e];
    }
    Ms[(long long)i * ns + j] = m;
    Hs[(long long)i * ns + j] = h;
    if (I != J) {
      Ms[(long long)j * ns + i] = m;
      Hs[(long long)j * ns + i] = h;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Rotation: one CTA = (subdomain, tile of 128 grid points, up to 256 output states from n0); K = N_s
// in tiles of 64 (more than 256 states: one CTA per 256-state slice of the output, each reading the
// tile of Psi_f again)
// stage layout: A_hi 16K, A_lo 16K (MN-major), B_hi, B_lo (N rows x 128 bytes each, <= 32K each)
constexpr uint32_t kRotStage = 2 * kTile + 2 * 256 * 128;

template <bool kFp16>
__global__ void __launch_bounds__(kThreads, 1)
k_rotate_tc(const SubDev* __restrict__ subs, const RotJob* __restrict__ jobs, const float* __restrict__ F,
            const uint16_t* __restrict__ Yhi, const uint16_t* __restrict__ Ylo, int kpad_max,
            const int* __restrict__ ex_f, const int* __restrict__ ex_y, float* __restrict__ Out, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const RotJob J = jobs[blockIdx.x];
  const SubDev& S = subs[J.sub];
  const int ns = S.ns;
  const int n0 = J.n0, nloc = min(256, ns - n0);   // output states n0 .. n0 + nloc - 1
  const int n16 = (nloc + 15) & ~15;
  const int nkt = (ns + kKT - 1) / kKT;
  const long long g0 = (long long)J.tile * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&full[s], kProducers);
      bar_init(&empty[s], 1);
    }
    bar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) tmem_alloc(&s_tmem, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = su32(smem);
  const float* f = F + S.off_blk;
  const long long yoff = (long long)S.off_state * kpad_max;   // Y^T hi/lo of this subdomain: [n][kpad_max]

  if (warp < 8) {
    for (int it = 0; it < nkt; ++it) {
      const int st = it % kStages;
      const int k0 = it * kKT;
      const uint32_t stage = sbase + st * kRotStage;
      // A: 64 k-rows x 128 grid points, chunks of 8 points (MN-major), 4 items per thread; B:
      // n16 rows x 64 k of Y^T hi / lo (already split), K-major, up to 8 items per thread.  All
      // global loads of the tile (and the rows' scale exponents) are issued before the stores, so
      // that their latencies overlap, and before the wait for the stage to be free.
      float4 a[4], b[4];
      int ex[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = threadIdx.x + u * kProducers;
        const int k = q >> 4, c16 = q & 15;     // c16: chunk of 8 points within 128
        const int kk = k0 + k;
        const long long g = g0 + c16 * 8;
        a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        b[u] = a[u];
        ex[u] = 0;
        if (kk < ns && g < S.nd) {
          const float4* p = reinterpret_cast<const float4*>(f + (long long)kk * S.nd + g);
          a[u] = p[0];
          b[u] = p[1];
        }
        if (kFp16 && kk < ns) ex[u] = ex_f[S.off_state + kk];
      }
      uint4 yh[8], yl[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = threadIdx.x + u * kProducers;
        const int n = q >> 3, c = q & 7;
        yh[u] = make_uint4(0, 0, 0, 0);
        yl[u] = yh[u];
        if (q < n16 * 8 && n < nloc) {
          const long long e = yoff + (long long)(n0 + n) * kpad_max + k0 + c * 8;
          yh[u] = *reinterpret_cast<const uint4*>(Yhi + e);
          yl[u] = *reinterpret_cast<const uint4*>(Ylo + e);
        }
      }
      if (it >= kStages && !bar_wait(&empty[st], ((it / kStages) - 1) & 1)) { atomicExch(&s_fail, 1); break; }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = threadIdx.x + u * kProducers;
        const int k = q >> 4, c16 = q & 15;
        const float sc = kFp16 ? ldexpf(1.f, ex[u]) : 1.f;
        uint4 hi, lo;
        split8<kFp16>(a[u], b[u], sc, hi, lo);
        const uint32_t off = mnmaj_off(c16 >> 3, k, c16 & 7);
        sts128(stage + off, hi);
        sts128(stage + kTile + off, lo);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = threadIdx.x + u * kProducers;
        if (q >= n16 * 8) continue;
        const int n = q >> 3, c = q & 7;
        const uint32_t off = kmaj_off(n, c);
        sts128(stage + 2 * kTile + off, yh[u]);
        sts128(stage + 2 * kTile + 256 * 128 + off, yl[u]);
      }
      fence_async_smem();
      bar_arrive(&full[st]);
    }
    const bool ok = bar_wait(&done, 0);
    tc_fence_after();
    if (!ok) atomicExch(&s_fail, 1);
    // epilogue: warp w reads lanes 32 (w & 3).., column half (w >> 2)
    const int lg = warp & 3, half = warp >> 2;
    const long long g = g0 + lg * 32 + lane;
    const int nhalf = ((n16 / 16 + 1) / 2) * 16;
    const int c_lo = half * nhalf, c_hi = min(n16, c_lo + nhalf);
    float* o = Out + S.off_blk;
    for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0, v);
      if (ok && g < S.nd) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (c0 + u < nloc)
            o[(long long)(n0 + c0 + u) * S.nd + g] = kFp16 ? ldexpf(v[u], -ex_y[S.off_state + n0 + c0 + u]) : v[u];
      }
    }
  } else if (lane == 0) {
    const uint32_t idesc = idesc_16(128, n16, true, kFp16);
    bool ok = true;
    for (int it = 0; it < nkt; ++it) {
      const int st = it % kStages;
      if (!bar_wait(&full[st], (it / kStages) & 1)) { ok = false; break; }
      tc_fence_after();
      const uint32_t stage = sbase + st * kRotStage;
      const uint32_t a_hi = stage, a_lo = stage + kTile;
      const uint32_t b_hi = stage + 2 * kTile, b_lo = b_hi + 256 * 128;
#pragma unroll
      for (int ks = 0; ks < kKT / 16; ++ks) {
        const int acc = (it > 0 || ks > 0) ? 1 : 0;
        // A (MN-major): K step of 16 = two 8-row K groups = 2048 bytes; B (K-major): 32 bytes
        const uint64_t ah = sdesc(a_hi + ks * 2048, 8192, 1024), al = sdesc(a_lo + ks * 2048, 8192, 1024);
        const uint64_t bh = sdesc(b_hi + ks * 32, 16, 1024), bl = sdesc(b_lo + ks * 32, 16, 1024);
        mma_bf16(tmem, ah, bh, idesc, acc);
        mma_bf16(tmem, ah, bl, idesc, 1);
        mma_bf16(tmem, al, bh, idesc, 1);
      }
      mma_commit(&empty[st]);
    }
    if (!ok) atomicExch(&s_fail, 1);
    mma_commit(&done);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 8) tmem_dealloc(tmem, 256);
  if (threadIdx.x == 0 && s_fail) atomicCAS(status, 0, XLS_ETIMEOUT);
}

// Y (FP64, row-major [k][n]) -> Y^T hi/lo [n][kpad_max], zero padded.  FP16 path: row k of Y is
// divided by 2^ex_f[k] (it multiplies column k of the A operand) and row n of Y^T is scaled by
// 2^ex_y[n] so that its largest entry lies in (2^13, 2^14]; the epilogue divides column n by it.
// One CTA per column n of one subdomain: the column's scaled maximum (FP16 path) by a block
// reduction, then one element per thread, so that no thread runs a loop over the whole column.
template <bool kFp16>
__global__ void __launch_bounds__(128)
k_split_yt(const SubDev* __restrict__ subs, const double* __restrict__ Y, int kpad_max,
           const int* __restrict__ ex_f, int* ex_y, uint16_t* Yhi, uint16_t* Ylo) {
  const SubDev& S = subs[blockIdx.y];
  const int ns = S.ns;
  const int n = blockIdx.x;
  if (n >= ns) return;
  const long long yoff = (long long)S.off_state * kpad_max;
  __shared__ double red[4];
  int ey = 0;
  if (kFp16) {
    double mx = 0.0;
    for (int k = threadIdx.x; k < ns; k += blockDim.x)
      mx = fmax(mx, fabs(ldexp(Y[S.off_ss + (long long)k * ns + n], -ex_f[S.off_state + k])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
    ey = (mx > 0.0) ? 14 - ilogb(mx) - 1 : 0;
    if (threadIdx.x == 0) ex_y[S.off_state + n] = ey;
  }
  for (int k = threadIdx.x; k < kpad_max; k += blockDim.x) {
    double yv = 0.0;
    if (k < ns) {
      yv = Y[S.off_ss + (long long)k * ns + n];
      if (kFp16) yv = ldexp(yv, ey - ex_f[S.off_state + k]);
    }
    uint16_t h, l;
    split1<kFp16>((float)yv, h, l);
    Yhi[yoff + (long long)n * kpad_max + k] = h;
    Ylo[yoff + (long long)n * kpad_max + k] = l;
  }
}

// per-vector exponent e with max |2^e x| in (2^13, 2^14] (0 for an all-zero vector), for the
// two blocks F and HF; one CTA per (vector, block)
__global__ void __launch_bounds__(512)
k_vec_exponent(const SubDev* __restrict__ subs, int n_sub, const float* __restrict__ F, const float* __restrict__ HF,
               int* ex_f, int* ex_hf) {
  const int v = blockIdx.x, a = blockIdx.y;
  const SubDev& S = subs[a];
  if (v >= S.ns) return;
  const float* src = (blockIdx.z == 0 ? F : HF) + S.off_blk + (long long)v * S.nd;
  float mx = 0.f;
  for (long long q = threadIdx.x * 4LL; q < S.nd; q += 4LL * blockDim.x) {
    const float4 x = *reinterpret_cast<const float4*>(src + q);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float red[16];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    const int e = (mx > 0.f) ? 14 - ilogbf(mx) - 1 : 0;
    (blockIdx.z == 0 ? ex_f : ex_hf)[S.off_state + v] = e;
  }
}

}  // namespace tc

size_t gram_tc_smem() { return tc::kStages * tc::kGramStage + 1024; }
size_t rotate_tc_smem() { return tc::kStages * tc::kRotStage + 1024; }

// the large dynamic shared memory of the tensor-core kernels, set on the current device at every
// grid creation (function attributes are per device)
bool tc_setup() {
  bool ok = true;
  ok &= cudaFuncSetAttribute(tc::k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(tc::k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(tc::k_rotate_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rotate_tc_smem()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(tc::k_rotate_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rotate_tc_smem()) == cudaSuccess;
  cudaGetLastError();
  return ok;
}

void launch_gram_tc(const SubDev* d_subs, int n_sub, int max_ns, const GramPlan& gp, bool fp16, const float* F,
                    const float* HF, double* Ms, double* Hs, int* status, cudaStream_t st) {
  if (gp.n_jobs == 0) return;
  if (fp16) {
    dim3 ge(max_ns, n_sub, 2);
    tc::k_vec_exponent<<<ge, 512, 0, st>>>(d_subs, n_sub, F, HF, gp.d_ex_f, gp.d_ex_hf);
    tc::k_gram_tc<true><<<gp.n_jobs, tc::kThreads, gram_tc_smem(), st>>>(d_subs, gp.d_jobs, F, HF, gp.d_ex_f,
                                                                          gp.d_ex_hf, gp.d_work, status);
  } else {
    tc::k_gram_tc<false><<<gp.n_jobs, tc::kThreads, gram_tc_smem(), st>>>(d_subs, gp.d_jobs, F, HF, nullptr, nullptr,
                                                                           gp.d_work, status);
  }
  dim3 grid(16, gp.n_groups);
  tc::k_gram_reduce<<<grid, 256, 0, st>>>(d_subs, gp.d_jobs, gp.d_grp_first, gp.d_grp_n, gp.d_work,
                                          fp16 ? gp.d_ex_f : nullptr, fp16 ? gp.d_ex_hf : nullptr, Ms, Hs);
}

// Gram of one block with caller-provided scratch; `work` holds at least
// gram_single_jobs(n_states, kc) * 2 * 128 * 128 floats.  Returns false if the shared-memory
// attribute cannot be set (launches nothing then).
int gram_single_pairs(int n_states) {
  const int nt = (n_states + 127) / 128;
  return nt * (nt + 1) / 2;
}

bool launch_gram_tc_single(const float* F, const float* HF, long long n_points, int n_states, int kc, float* work,
                           double* Ms, double* Hs, int* status, cudaStream_t st) {
  // the attribute belongs to the current device: set it on every call (cheap, and no shared
  // state between threads or devices)
  if (cudaFuncSetAttribute(tc::k_gram_tc_single, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem()) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int pairs = gram_single_pairs(n_states);
  tc::k_gram_tc_single<<<pairs * kc, tc::kThreads, gram_tc_smem(), st>>>(F, HF, n_points, n_states, kc, work, status);
  dim3 grid(16, pairs);
  tc::k_gram_reduce_single<<<grid, 256, 0, st>>>(work, n_states, n_points, kc, Ms, Hs);
  return true;
}

// the FP16 path uses the exponents of F computed by the Gram launch of the same pass
void launch_rotate_tc(const SubDev* d_subs, int n_sub, int max_ns, const RotPlan& rp, const GramPlan& gp, bool fp16,
                      bool need_exponents, const float* F, const double* Y, float* Out, int* status, cudaStream_t st) {
  if (rp.n_jobs == 0) return;
  dim3 gs(max_ns, n_sub);
  if (fp16 && need_exponents) {   // the Gram of this pass did not run on tensor cores
    dim3 ge(max_ns, n_sub, 1);
    tc::k_vec_exponent<<<ge, 512, 0, st>>>(d_subs, n_sub, F, F, gp.d_ex_f, gp.d_ex_hf);
  }
  if (fp16) {
    tc::k_split_yt<true><<<gs, 128, 0, st>>>(d_subs, Y, rp.kpad_max, gp.d_ex_f, rp.d_ex_y, rp.d_yhi, rp.d_ylo);
    tc::k_rotate_tc<true><<<rp.n_jobs, tc::kThreads, rotate_tc_smem(), st>>>(
        d_subs, rp.d_jobs, F, rp.d_yhi, rp.d_ylo, rp.kpad_max, gp.d_ex_f, rp.d_ex_y, Out, status);
  } else {
    tc::k_split_yt<false><<<gs, 128, 0, st>>>(d_subs, Y, rp.kpad_max, nullptr, nullptr, rp.d_yhi, rp.d_ylo);
    tc::k_rotate_tc<false><<<rp.n_jobs, tc::kThreads, rotate_tc_smem(), st>>>(
        d_subs, rp.d_jobs, F, rp.d_yhi, rp.d_ylo, rp.kpad_max, nullptr, nullptr, Out, status);
  }
}

}  // namespace xls
