// Chebyshev-filter step kernels: 12th-order FD stencil + local potential + recurrence, and the
// Kleinman-Bylander nonlocal projection / back-projection (Sec. 5.A.3 step (1); Sec. 5.B.2).
//
// One filter step computes, for every subdomain alpha and every vector of its block,
//   Y_out = scale * (H Y_in - c Y_in) - shift * Y_prev,
//   H Y = -1/2 Delta_h Y + V Y + sum_I sum_l chi_Il P_Il,   P_Il = E_l dV <chi_Il, Y>.
// The local part is one launch (k_stencil); the nonlocal part is a projection launch before it
// (k_nl_project, P from Y_in) and a back-projection launch after it (k_nl_back_csr, adds
// scale * chi P into Y_out).  All subdomains of a step share each launch.
#include "xls_internal.h"

namespace xls {

__constant__ double c_fdw[kN0 + 1] = {-5369.0 / 1800.0, 12.0 / 7.0, -15.0 / 56.0, 10.0 / 189.0,
                                      -1.0 / 112.0,     2.0 / 1925.0, -1.0 / 16632.0};

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ int find_sub(const int* blk_off, int n_sub, int b) {
  int lo = 0, hi = n_sub;  // blk_off[lo] <= b < blk_off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (blk_off[mid] <= b) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr int kTX = 32, kTY = 8;

int stencil_blocks(const int n[3], int ns) {
  return ((n[0] + kTX - 1) / kTX) * ((n[1] + kTY - 1) / kTY) * ns;
}

// 2.5-D blocking: a CTA owns a kTX x kTY column tile of one vector and marches along z.  The
// 13 z-values of each column live in a register queue; each xy-plane (with its 6-point halo)
// is staged in shared memory for the x/y neighbours.  Out-of-box points are zero (Dirichlet)
// or wrapped (periodic).
template <typename T>
__global__ void __launch_bounds__(kTX * kTY)
k_stencil(const SubDev* __restrict__ subs, int n_sub, const int* __restrict__ blk_off,
          const T* __restrict__ Yin, const T* Yprev, T* Yout, const T* __restrict__ Vall,
          const StepCoef* __restrict__ coef, int step) {
  __shared__ T tile[kTY + 2 * kN0][kTX + 2 * kN0];
  const int b = blockIdx.x;
  const int a = find_sub(blk_off, n_sub, b);
  const SubDev& S = subs[a];
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const int px = S.periodic[0], py = S.periodic[1], pz = S.periodic[2];
  const int ntx = (nx + kTX - 1) / kTX, nty = (ny + kTY - 1) / kTY;
  const int local = b - blk_off[a];
  const int t = local % (ntx * nty);
  const long long vec = local / (ntx * nty);
  const int x0 = (t % ntx) * kTX, y0 = (t / ntx) * kTY;
  const long long base = S.off_blk + vec * S.nd;
  const T* __restrict__ yin = Yin + base;
  const T* yprev = Yprev ? Yprev + base : nullptr;
  T* yout = Yout + base;
  const T* __restrict__ V = Vall + S.off_pt;
  const StepCoef cf = coef[a * kMaxDegree + step];
  const T scale = (T)cf.scale, cshift = (T)cf.c, pshift = (T)cf.shift;

  T wx[kN0 + 1], wy[kN0 + 1], wz[kN0 + 1];
  {
    const double ix = -0.5 / (S.h[0] * S.h[0]), iy = -0.5 / (S.h[1] * S.h[1]), iz = -0.5 / (S.h[2] * S.h[2]);
#pragma unroll
    for (int p = 0; p <= kN0; ++p) {
      wx[p] = (T)(c_fdw[p] * ix);
      wy[p] = (T)(c_fdw[p] * iy);
      wz[p] = (T)(c_fdw[p] * iz);
    }
  }
  const T wc = (T)(c_fdw[0] * (-0.5 / (S.h[0] * S.h[0]) - 0.5 / (S.h[1] * S.h[1]) - 0.5 / (S.h[2] * S.h[2])));

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < nx) && (y < ny);
  // this thread's column in the (boundary-mapped) grid; -1 = zero column
  int cx = x, cy = y;
  if (cx >= nx) cx = px ? wrapi(cx, nx) : -1;
  if (cy >= ny) cy = py ? wrapi(cy, ny) : -1;
  const bool has_col = (cx >= 0) && (cy >= 0);
  const long long plane = (long long)nx * ny;
  auto load_col = [&](int z) -> T {
    if (!has_col) return (T)0;
    if (z < 0 || z >= nz) {
      if (!pz) return (T)0;
      z = wrapi(z, nz);
    }
    return yin[z * plane + (long long)cy * nx + cx];
  };

  T q[2 * kN0 + 1];
#pragma unroll
  for (int k = 0; k < 2 * kN0 + 1; ++k) q[k] = load_col(k - kN0);

  const int tid = ty * kTX + tx;
  constexpr int RW = kTX + 2 * kN0, RH = kTY + 2 * kN0;
  for (int z = 0; z < nz; ++z) {
    tile[ty + kN0][tx + kN0] = q[kN0];
    // halo ring of the plane
    for (int s = tid; s < RW * RH; s += kTX * kTY) {
      const int sy = s / RW, sx = s - sy * RW;
      if (sy >= kN0 && sy < kN0 + kTY && sx >= kN0 && sx < kN0 + kTX) continue;
      int gx = x0 + sx - kN0, gy = y0 + sy - kN0;
      T val = (T)0;
      bool ok = true;
      if (gx < 0 || gx >= nx) { if (px) gx = wrapi(gx, nx); else ok = false; }
      if (gy < 0 || gy >= ny) { if (py) gy = wrapi(gy, ny); else ok = false; }
      if (ok) val = yin[z * plane + (long long)gy * nx + gx];
      tile[sy][sx] = val;
    }
    __syncthreads();
    if (active) {
      const T c0 = q[kN0];
      T acc = wc * c0;
#pragma unroll
      for (int p = 1; p <= kN0; ++p) {
        acc += wx[p] * (tile[ty + kN0][tx + kN0 + p] + tile[ty + kN0][tx + kN0 - p]);
        acc += wy[p] * (tile[ty + kN0 + p][tx + kN0] + tile[ty + kN0 - p][tx + kN0]);
        acc += wz[p] * (q[kN0 + p] + q[kN0 - p]);
      }
      const long long g = z * plane + (long long)y * nx + x;
      acc += V[g] * c0;
      T out = scale * (acc - cshift * c0);
      if (yprev) out -= pshift * yprev[g];
      yout[g] = out;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2 * kN0; ++k) q[k] = q[k + 1];
    q[2 * kN0] = load_col(z + kN0 + 1);
  }
}

template <typename T>
void launch_stencil(const SubDev* d_subs, int n_sub, const Plan& plan, const T* Yin, const T* Yprev, T* Yout,
                    const T* V, const StepCoef* coef, int step, cudaStream_t st) {
  if (plan.total == 0) return;
  dim3 block(kTX, kTY);
  k_stencil<T><<<plan.total, block, 0, st>>>(d_subs, n_sub, plan.d_blk_off, Yin, Yprev, Yout, V, coef, step);
}

// ---- nonlocal projectors -------------------------------------------------------------------
// Set-up: for every projector slot (one atom in one subdomain, all of its periodic images) a
// table of its grid points and the four chi values there, built once per Hamiltonian in FP64
// and stored in the block's precision.  Per filter step: the projection launch
// P[slot][l][v] = E_l dV sum_g chi_l(g) Y_v(g) (k_nl_project) and the back-projection launch
// Y_out[v][g] += scale sum_l chi_l(g) P[slot][l][v] over the reverse table rows (k_nl_back_csr:
// each element receives one reduction, the sum of its row; k_nl_back is the per-slot variant with
// one atomic per table entry, kept for reference runs).
constexpr int kNlWarps = 8, kNlVec = 8;

template <typename T>
__device__ __forceinline__ bool chi_at(const ProjSlot& A, const AtomImg& I, const SubDev& S, int p, double chi[4],
                                       int& g) {
  const int bx = I.box_n[0], by = I.box_n[1];
  const int i = I.box_lo[0] + p % bx;
  const int j = I.box_lo[1] + (p / bx) % by;
  const int k = I.box_lo[2] + p / (bx * by);
  const double dx = i * S.h[0] - I.R[0], dy = j * S.h[1] - I.R[1], dz = k * S.h[2] - I.R[2];
  const double r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 < A.rcut2)) return false;
  const double e = exp(-r2 / (2.0 * A.w * A.w));
  chi[0] = A.norm[0] * e;
  chi[1] = A.norm[1] * dx * e;
  chi[2] = A.norm[2] * dy * e;
  chi[3] = A.norm[3] * dz * e;
  const int gi = S.periodic[0] ? wrapi(i, S.n[0]) : i;
  const int gj = S.periodic[1] ? wrapi(j, S.n[1]) : j;
  const int gk = S.periodic[2] ? wrapi(k, S.n[2]) : k;
  g = (gk * S.n[1] + gj) * S.n[0] + gi;
  return true;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_proj_count(const SubDev* __restrict__ subs, const ProjSlot* __restrict__ slots, const AtomImg* __restrict__ imgs,
             int* counts) {
  const ProjSlot& A = slots[blockIdx.x];
  const SubDev& S = subs[A.sub];
  int c = 0;
  for (int im = A.img_lo; im < A.img_lo + A.img_n; ++im) {
    const AtomImg& I = imgs[im];
    const int npts = I.box_n[0] * I.box_n[1] * I.box_n[2];
    for (int p = threadIdx.x; p < npts; p += blockDim.x) {
      double chi[4];
      int g;
      if (chi_at<T>(A, I, S, p, chi, g)) ++c;
    }
  }
  __shared__ int red[8];
  c += __shfl_xor_sync(0xffffffffu, c, 16);
  c += __shfl_xor_sync(0xffffffffu, c, 8);
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    counts[blockIdx.x] = t;
  }
}

// ordered compaction: chunk by chunk of blockDim points, ballot + warp prefix + block prefix
template <typename T>
__global__ void __launch_bounds__(256)
k_proj_fill(const SubDev* __restrict__ subs, const ProjSlot* __restrict__ slots, const AtomImg* __restrict__ imgs,
            int* idx, typename Vec4<T>::type* chi_out) {
  const ProjSlot& A = slots[blockIdx.x];
  const SubDev& S = subs[A.sub];
  __shared__ int wsum[8];
  __shared__ int s_base;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int im = A.img_lo; im < A.img_lo + A.img_n; ++im) {
    const AtomImg& I = imgs[im];
    const int npts = I.box_n[0] * I.box_n[1] * I.box_n[2];
    for (int p0 = 0; p0 < npts; p0 += blockDim.x) {
      const int p = p0 + threadIdx.x;
      double chi[4];
      int g = 0;
      const bool in = (p < npts) && chi_at<T>(A, I, S, p, chi, g);
      const unsigned m = __ballot_sync(0xffffffffu, in);
      const int before = __popc(m & ((1u << lane) - 1u));
      if (lane == 0) wsum[warp] = __popc(m);
      __syncthreads();
      int off = s_base;
      for (int w = 0; w < warp; ++w) off += wsum[w];
      if (in) {
        const long long e = A.pt_off + off + before;
        idx[e] = g;
        typename Vec4<T>::type c4;
        c4.x = (T)chi[0]; c4.y = (T)chi[1]; c4.z = (T)chi[2]; c4.w = (T)chi[3];
        chi_out[e] = c4;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < nw; ++w) t += wsum[w];
        s_base += t;
      }
      __syncthreads();
    }
  }
}

// Projection P[slot][l][v] = E_l dV sum_g chi_l(g) Y_v(g).  A CTA takes one slot and a group of
// KPV = 8, 16 or 32 vectors (the autotuner's choice); the grid runs group-major, so that the CTAs
// resident at any time read the same KPV-vector slice of every subdomain's block (tens of MB: it
// stays in L2 and each Y element, shared by the about two spheres that contain its point, comes
// from DRAM about once).  Warp w takes vectors 8 (w % kVH) .. +7 and every kPH-th 32-point chunk
// of the table from chunk w / kVH; a lane two points at a time (16 loads in flight); lanes
// (transpose reduction) and warps are reduced at the end.  Wider groups read each table entry
// once for more vectors (the warps of a CTA share it through L1) and split the slot's points
// over fewer warps.
// slots per chunk of the projection's CTA order (256, 512 or 1024, xls_autotune; 256 by default,
// with 8 vectors on CTAs of 4 warps: measured fastest on 72^3 subdomains with 528 states; a
// 72^3 subdomain has about 430 slots, whose tables (~30 MB) and one vector group's Y slice
// (~12 MB per 8 vectors) stay in L2 while a chunk is walked)

template <typename T, int KPV, int NW>
__global__ void __launch_bounds__(NW * 32)
k_nl_project(const SubDev* __restrict__ subs, const ProjSlot* __restrict__ slots, int slot_off, int n_slot,
             int n_groups, int chunk_slots, const int* __restrict__ idx, const typename Vec4<T>::type* __restrict__ chi,
             const T* __restrict__ Y, double* __restrict__ P) {
  using T4 = typename Vec4<T>::type;
  constexpr int kVH = KPV / 8, kPH = NW / kVH;   // vector eighths and point phases of the NW warps
  static_assert(kPH >= 1, "at least one point phase");
  __shared__ T red[kPH][KPV * 4];
  // CTAs walk the slots in chunks of chunk_slots: every vector group runs over the chunk before
  // the next chunk starts, so the chunk's tables stay in L2 for all groups, and within a group the
  // points that neighbouring slots share are read from DRAM once
  const int chunk = (int)(blockIdx.x / (chunk_slots * n_groups)), rem = (int)(blockIdx.x % (chunk_slots * n_groups));
  const int grp = rem / chunk_slots, sic = chunk * chunk_slots + rem % chunk_slots;
  if (sic >= n_slot) return;
  const int slot = slot_off + sic;
  const ProjSlot& A = slots[slot];
  const SubDev& S = subs[A.sub];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vh = warp % kVH, ph = warp / kVH;
  const int v0 = grp * KPV + vh * 8;
  const int nv = max(0, min(8, S.ns - v0));
  if (grp * KPV >= S.ns) return;   // uniform per CTA
  T acc[4][8];
#pragma unroll
  for (int l = 0; l < 4; ++l)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[l][v] = (T)0;
  const T* yb = Y + S.off_blk + (long long)v0 * S.nd;
  const int* ib = idx + A.pt_off;
  const T4* cb = chi + A.pt_off;
  // the point indices of the next iteration are fetched one iteration ahead, so that only the Y
  // gathers (not the table loads before them) wait on memory
  const int pfirst = ph * 32 + lane;
  int ng0 = pfirst < A.pt_n ? ib[pfirst] : 0;
  int ng1 = pfirst + 32 * kPH < A.pt_n ? ib[pfirst + 32 * kPH] : 0;
  if (nv > 0)
    for (int p = pfirst; p < A.pt_n; p += 64 * kPH) {
      const bool two = p + 32 * kPH < A.pt_n;
      const int g0 = ng0, g1 = two ? ng1 : g0;
      const int pn = p + 64 * kPH;
      if (pn < A.pt_n) {
        ng0 = ib[pn];
        ng1 = pn + 32 * kPH < A.pt_n ? ib[pn + 32 * kPH] : 0;
      }
      const T4 c = cb[p];
      T4 d = cb[two ? p + 32 * kPH : p];
      if (!two) { d.x = (T)0; d.y = (T)0; d.z = (T)0; d.w = (T)0; }
      T y0[8], y1[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        y0[v] = (v < nv) ? yb[(long long)v * S.nd + g0] : (T)0;
        y1[v] = (v < nv) ? yb[(long long)v * S.nd + g1] : (T)0;
      }
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        acc[0][v] += c.x * y0[v] + d.x * y1[v];
        acc[1][v] += c.y * y0[v] + d.y * y1[v];
        acc[2][v] += c.z * y0[v] + d.z * y1[v];
        acc[3][v] += c.w * y0[v] + d.w * y1[v];
      }
    }
  // transpose reduction over the lanes: after five halving steps lane q = l * 8 + v holds the
  // warp's sum of acc[l][v] (31 exchanges instead of 32 x 5)
  T* a = &acc[0][0];
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int q = 0; q < h; ++q) {
      const T send = up ? a[q] : a[q + h];
      const T keep = up ? a[q + h] : a[q];
      a[q] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  red[ph][vh * 32 + lane] = a[0];
  __syncthreads();
  if (threadIdx.x < KPV * 4) {
    const int h = threadIdx.x / 32, l = (threadIdx.x / 8) % 4, v = threadIdx.x % 8;
    const int vg = grp * KPV + h * 8 + v;
    if (vg < S.ns) {
      T s = (T)0;
#pragma unroll
      for (int q = 0; q < kPH; ++q) s += red[q][threadIdx.x];
      double* pa = P + S.off_proj + (long long)(slot - S.slot_lo) * 4 * S.ns;
      pa[l * S.ns + vg] = (double)s * A.E[l] * S.dV;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kNlWarps * 32)
k_nl_back(const SubDev* __restrict__ subs, const ProjSlot* __restrict__ slots, const int* __restrict__ idx,
          const typename Vec4<T>::type* __restrict__ chi, const double* __restrict__ P, T* Yout,
          const StepCoef* __restrict__ coef, int step) {
  const ProjSlot& A = slots[blockIdx.x];
  const SubDev& S = subs[A.sub];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v0 = (blockIdx.y * kNlWarps + warp) * kNlVec;
  if (v0 >= S.ns) return;
  const int nv = min(kNlVec, S.ns - v0);
  const double scale = coef[A.sub * kMaxDegree + step].scale;
  const double* pa = P + S.off_proj + (long long)(blockIdx.x - S.slot_lo) * 4 * S.ns;
  T q[4][kNlVec];
#pragma unroll
  for (int v = 0; v < kNlVec; ++v)
#pragma unroll
    for (int l = 0; l < 4; ++l) q[l][v] = (v < nv) ? (T)(scale * pa[l * S.ns + v0 + v]) : (T)0;
  T* yb = Yout + S.off_blk + (long long)v0 * S.nd;
  const int* ix = idx + A.pt_off;
  const typename Vec4<T>::type* cx = chi + A.pt_off;
  for (int p = lane; p < A.pt_n; p += 32) {
    const int g = ix[p];
    const typename Vec4<T>::type c = cx[p];
#pragma unroll
    for (int v = 0; v < kNlVec; ++v) {
      if (v < nv) atomicAdd(yb + (long long)v * S.nd + g, c.x * q[0][v] + c.y * q[1][v] + c.z * q[2][v] + c.w * q[3][v]);
    }
  }
}

// ---- reverse tables for the back-projection (the paper's reverse CSR over grid points) -----
// row g of subdomain a (global point index S.off_pt + g) lists (slot - S.slot_lo, chi) of every
// slot whose sphere contains the point
__global__ void k_rcsr_count(const SubDev* __restrict__ subs, const ProjSlot* __restrict__ slots,
                             const int* __restrict__ idx, int* cnt) {
  const ProjSlot& A = slots[blockIdx.x];
  const SubDev& S = subs[A.sub];
  for (int p = threadIdx.x; p < A.pt_n; p += blockDim.x) atomicAdd(cnt + S.off_pt + idx[A.pt_off + p], 1);
}

template <typename T>
__global__ void k_rcsr_fill(const SubDev* __restrict__ subs, const ProjSlot* __restrict__ slots,
                            const int* __restrict__ idx, const typename Vec4<T>::type* __restrict__ chi,
                            const long long* __restrict__ row_ptr, int* cursor, int* rslot,
                            typename Vec4<T>::type* rchi) {
  const ProjSlot& A = slots[blockIdx.x];
  const SubDev& S = subs[A.sub];
  for (int p = threadIdx.x; p < A.pt_n; p += blockDim.x) {
    const long long row = S.off_pt + idx[A.pt_off + p];
    const long long e = row_ptr[row] + atomicAdd(cursor + row, 1);
    rslot[e] = (int)blockIdx.x - S.slot_lo;
    rchi[e] = chi[A.pt_off + p];
  }
}

constexpr int kLocBits = 32768;          // slots per subdomain the localisation handles (bitmap in shared memory)

// One CTA per point block: mark the slots named by the block's reverse-table rows in a bitmap;
// pass 0 stores their number, pass 1 replaces every entry's slot by its rank among the marked
// slots (ascending slot order, so the ranks do not depend on the order of the entries) and lists
// the marked slots in that order.
__global__ void __launch_bounds__(256)
k_rcsr_localize(const SubDev* __restrict__ subs, const int* __restrict__ blk_sub, const long long* __restrict__ row_ptr,
                int* rslot, int* blk_cnt, int* blk_list, int list_max, int pass) {
  __shared__ unsigned bits[kLocBits / 32];
  __shared__ int wpre[kLocBits / 32];
  const int b = blockIdx.x;
  const SubDev& S = subs[blk_sub[b]];
  const int nw = (S.slot_n + 31) / 32;
  const long long p0 = (long long)(b - S.off_nlb) * kBackPts;
  const long long p1 = min(S.nd, p0 + kBackPts);
  const long long e0 = row_ptr[S.off_pt + p0], e1 = row_ptr[S.off_pt + p1];
  for (int w = threadIdx.x; w < nw; w += blockDim.x) bits[w] = 0u;
  __syncthreads();
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int sl = rslot[e];
    atomicOr(&bits[sl >> 5], 1u << (sl & 31));
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // exclusive prefix of the words' populations (at most 1024 words)
    int acc = 0;
    for (int w = 0; w < nw; ++w) {
      wpre[w] = acc;
      acc += __popc(bits[w]);
    }
    if (pass == 0) blk_cnt[b] = acc;
  }
  __syncthreads();
  if (pass == 0) return;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int sl = rslot[e];
    rslot[e] = wpre[sl >> 5] + __popc(bits[sl >> 5] & ((1u << (sl & 31)) - 1u));
  }
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    unsigned m = bits[w];
    int r = wpre[w];
    while (m) {
      const int bit = __ffs(m) - 1;
      if (r < list_max) blk_list[(long long)b * list_max + r] = w * 32 + bit;
      ++r;
      m &= m - 1u;
    }
  }
}

// ---- exclusive prefix sum of the reverse-table row counts on the device: rp[i] = sum_{j<i} cnt[j],
// rp[n] = the total (three launches: block sums, one-block scan of the block sums, block scans) ----
constexpr int kScanT = 256, kScanPer = 8, kScanBlk = kScanT * kScanPer;

__global__ void __launch_bounds__(kScanT) k_scan_blocksum(const int* __restrict__ cnt, long long n, long long* bsum) {
  __shared__ long long red[kScanT / 32];
  const long long base = (long long)blockIdx.x * kScanBlk;
  long long acc = 0;
  for (int k = 0; k < kScanPer; ++k) {
    const long long i = base + (long long)k * kScanT + threadIdx.x;
    if (i < n) acc += cnt[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kScanT / 32; ++w) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

// one CTA: exclusive scan of the nb block sums in place, the total in bsum[nb]
__global__ void __launch_bounds__(1024) k_scan_blocks(long long* bsum, int nb) {
  __shared__ long long wsum[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nb; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const long long x = i < nb ? bsum[i] : 0;
    long long v = x;   // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) >= o) v += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      long long w = wsum[threadIdx.x];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (threadIdx.x >= o) w += y;
      }
      wsum[threadIdx.x] = w;   // inclusive over warps
    }
    __syncthreads();
    const long long before = carry + ((threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0) + v - x;
    __syncthreads();
    if (i < nb) bsum[i] = before;
    if (threadIdx.x == 1023) carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kScanT)
k_scan_apply(const int* __restrict__ cnt, long long n, const long long* __restrict__ boff, long long* rp) {
  __shared__ long long wsum[kScanT / 32];
  const long long base = (long long)blockIdx.x * kScanBlk + (long long)threadIdx.x * kScanPer;
  long long loc[kScanPer];
  long long acc = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    loc[k] = acc;
    acc += (base + k < n) ? cnt[base + k] : 0;
  }
  long long v = acc;   // inclusive scan of the threads' totals
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += y;
  }
  if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  long long wbefore = 0;
  for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wbefore += wsum[w];
  const long long start = boff[blockIdx.x] + wbefore + v - acc;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < n) rp[base + k] = start + loc[k];
  if (base + kScanPer >= n && base < n) rp[n] = start + acc;   // the thread holding the last element
}

long long scan_temp_count(long long n) { return (n + kScanBlk - 1) / kScanBlk + 1; }

void launch_exclusive_scan(const int* cnt, long long n, long long* tmp, long long* rp, cudaStream_t st) {
  const int nb = (int)((n + kScanBlk - 1) / kScanBlk);
  if (nb == 0) return;
  k_scan_blocksum<<<nb, kScanT, 0, st>>>(cnt, n, tmp);
  k_scan_blocks<<<1, 1024, 0, st>>>(tmp, nb);
  k_scan_apply<<<nb, kScanT, 0, st>>>(cnt, n, tmp, rp);
}

void launch_rcsr_localize(const SubDev* d_subs, const int* d_blk_sub, int n_blk, const long long* row_ptr, int* rslot,
                          int* blk_cnt, int* blk_list, int list_max, int pass, cudaStream_t st) {
  if (n_blk > 0) k_rcsr_localize<<<n_blk, 256, 0, st>>>(d_subs, d_blk_sub, row_ptr, rslot, blk_cnt, blk_list, list_max, pass);
}

// Y_out[v][g] += scale * sum over the slots s of point g of sum_l chi_l(g) P[s][l][v]; PPT
// points per thread per iteration and KV vectors per CTA (1 x 8, 2 x 8 or 1 x 16, timed by
// xls_autotune: two points give each thread more loads in flight, one point fewer registers and
// so more resident warps, 16 vectors read every table row once for twice the vectors; 1 x 8
// measured 9 % faster than 2 x 8 on 72^3 subdomains with 528 states and is the default)
template <typename T, int PPT, int KV>
__global__ void __launch_bounds__(256)
k_nl_back_csr(const SubDev* __restrict__ subs, const long long* __restrict__ row_ptr, const int* __restrict__ rslot,
              const typename Vec4<T>::type* __restrict__ rchi, const int* __restrict__ blk_cnt,
              const int* __restrict__ blk_list, int list_max, const double* __restrict__ P, T* Yout,
              const StepCoef* __restrict__ coef, int step) {
  using T4 = typename Vec4<T>::type;
  extern __shared__ __align__(16) unsigned char qsm[];
  T4* Qs = reinterpret_cast<T4*>(qsm);   // [slot][KV + 1]: rows padded so consecutive slots use other bank groups
  // the vector groups of one point block are consecutive CTAs: the block's reverse-table rows
  // are read once from DRAM and then from L2
  const SubDev& S = subs[blockIdx.z];
  const int v0 = blockIdx.x * KV;
  const long long p0 = (long long)blockIdx.y * kBackPts;
  if (v0 >= S.ns || p0 >= S.nd || S.slot_n == 0) return;
  const int nv = min(KV, S.ns - v0);
  const double scale = coef[blockIdx.z * kMaxDegree + step].scale;
  // the projector coefficients of the slots this point block meets (its rows name them by rank
  // in the block's list)
  const int nb = S.off_nlb + (int)blockIdx.y;
  const int nloc = blk_cnt[nb];
  const int* list = blk_list + (long long)nb * list_max;
  for (int q = threadIdx.x; q < nloc * KV; q += blockDim.x) {
    const int sl = q / KV, v = q % KV;
    T4 x;
    if (v < nv) {
      const double* pa = P + S.off_proj + (long long)list[sl] * 4 * S.ns + v0 + v;
      x.x = (T)(scale * pa[0]); x.y = (T)(scale * pa[S.ns]); x.z = (T)(scale * pa[2 * S.ns]); x.w = (T)(scale * pa[3 * S.ns]);
    } else {
      x.x = x.y = x.z = x.w = (T)0;
    }
    Qs[sl * (KV + 1) + v] = x;
  }
  __syncthreads();
  T* yb = Yout + S.off_blk + (long long)v0 * S.nd;
  const long long end = min(S.nd, p0 + kBackPts);
  // PPT points per thread per iteration; the sum over the table rows is formed in registers and
  // added to Y_out with fire-and-forget reductions (red.global.add): the read-modify-write happens
  // in L2, no load of Y sits on the thread's critical path, and each element receives exactly one
  // addition (deterministic)
  // the row bounds of the next iteration's points are fetched one iteration ahead, so that only
  // the table entries (not the row pointers before them) wait on memory
  const long long* rp = row_ptr + S.off_pt;
  const long long stride = (long long)PPT * blockDim.x;
  long long g = p0 + threadIdx.x;
  long long nr0[PPT], nr1[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const long long gu = g + (long long)u * blockDim.x;
    nr0[u] = gu < end ? rp[gu] : 0;
    nr1[u] = gu < end ? rp[gu + 1] : 0;
  }
  for (; g < end; g += stride) {
    long long r0[PPT], r1[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      r0[u] = nr0[u];
      r1[u] = nr1[u];
      const long long gn = g + stride + (long long)u * blockDim.x;
      nr0[u] = gn < end ? rp[gn] : 0;
      nr1[u] = gn < end ? rp[gn + 1] : 0;
    }
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      const long long gu = g + (long long)u * blockDim.x;
      if (gu >= end || r1[u] == r0[u]) continue;
      T y[KV];
#pragma unroll
      for (int v = 0; v < KV; ++v) y[v] = (T)0;
      for (long long e = r0[u]; e < r1[u]; ++e) {
        const int sl = rslot[e];
        const T4 c = rchi[e];
        const T4* qq = Qs + sl * (KV + 1);
#pragma unroll
        for (int v = 0; v < KV; ++v) {
          const T4 q = qq[v];
          y[v] += c.x * q.x + c.y * q.y + c.z * q.z + c.w * q.w;
        }
      }
#pragma unroll
      for (int v = 0; v < KV; ++v)
        if (v < nv) atomicAdd(yb + (long long)v * S.nd + gu, y[v]);
    }
  }
}

// ---- single-vector views (one vector per subdomain: the Lanczos bound) -----------------------
// Projection: one warp per slot walks all the slot's points, four per lane at a time.
template <typename T>
__global__ void __launch_bounds__(256)
k_nl_project1(const SubDev* __restrict__ subs, const ProjSlot* __restrict__ slots, int n_slot,
              const int* __restrict__ idx, const typename Vec4<T>::type* __restrict__ chi, const T* __restrict__ Y,
              double* __restrict__ P) {
  using T4 = typename Vec4<T>::type;
  const int slot = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (slot >= n_slot) return;   // warp-uniform
  const ProjSlot& A = slots[slot];
  const SubDev& S = subs[A.sub];
  const T* yb = Y + S.off_blk;
  const int* ib = idx + A.pt_off;
  const T4* cb = chi + A.pt_off;
  T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
  for (int p = lane; p < A.pt_n; p += 128) {
    int g[4];
    T4 c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = p + 32 * u;
      g[u] = q < A.pt_n ? ib[q] : -1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = p + 32 * u;
      if (q < A.pt_n) c[u] = cb[q];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (g[u] >= 0) {
        const T y = yb[g[u]];
        a0 += c[u].x * y;
        a1 += c[u].y * y;
        a2 += c[u].z * y;
        a3 += c[u].w * y;
      }
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    a3 += __shfl_xor_sync(0xffffffffu, a3, o);
  }
  if (lane == 0) {
    double* pa = P + S.off_proj + (long long)(slot - S.slot_lo) * 4;
    pa[0] = (double)a0 * A.E[0] * S.dV;
    pa[1] = (double)a1 * A.E[1] * S.dV;
    pa[2] = (double)a2 * A.E[2] * S.dV;
    pa[3] = (double)a3 * A.E[3] * S.dV;
  }
}

// Back-projection: one thread per grid point adds the sum over its reverse-table row (entries name
// slots by rank in the list of the point's block) to its element; no two threads share an element.
template <typename T>
__global__ void __launch_bounds__(256)
k_nl_back1(const SubDev* __restrict__ subs, const long long* __restrict__ row_ptr, const int* __restrict__ rslot,
           const typename Vec4<T>::type* __restrict__ rchi, const int* __restrict__ blk_list, int list_max,
           const double* __restrict__ P, T* Yout, const StepCoef* __restrict__ coef, int step) {
  using T4 = typename Vec4<T>::type;
  const SubDev& S = subs[blockIdx.y];
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S.nd || S.slot_n == 0) return;
  const long long* rp = row_ptr + S.off_pt;
  const long long e0 = rp[g], e1 = rp[g + 1];
  if (e1 == e0) return;
  const int* list = blk_list + (long long)(S.off_nlb + (int)(g / kBackPts)) * list_max;
  const double* pb = P + S.off_proj;
  double sum = 0.0;
  for (long long e = e0; e < e1; ++e) {
    const int sl = list[rslot[e]];
    const T4 c = rchi[e];
    const double* pa = pb + (long long)sl * 4;
    sum += (double)c.x * pa[0] + (double)c.y * pa[1] + (double)c.z * pa[2] + (double)c.w * pa[3];
  }
  T* y = Yout + S.off_blk + g;
  *y += (T)(coef[blockIdx.y * kMaxDegree + step].scale * sum);
}

template <typename T>
void launch_nl_project1(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const int* idx,
                        const typename Vec4<T>::type* chi, const T* Y, double* P, cudaStream_t st) {
  if (n_slot == 0) return;
  const long long threads = (long long)n_slot * 32;
  k_nl_project1<T><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(d_subs, d_slots, n_slot, idx, chi, Y, P);
}

template <typename T>
void launch_nl_back1(const SubDev* d_subs, int n_sub, long long max_nd, int list_max, const long long* row_ptr,
                     const int* rslot, const typename Vec4<T>::type* rchi, const int* blk_list, const double* P,
                     T* Yout, const StepCoef* coef, int step, cudaStream_t st) {
  if (list_max == 0) return;
  dim3 grid((unsigned)((max_nd + 255) / 256), n_sub);
  k_nl_back1<T><<<grid, 256, 0, st>>>(d_subs, row_ptr, rslot, rchi, blk_list, list_max, P, Yout, coef, step);
}

template <typename T>
void launch_rcsr_build(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const int* idx,
                       const typename Vec4<T>::type* chi, const long long* row_ptr, int* cursor, int* rslot,
                       typename Vec4<T>::type* rchi, cudaStream_t st) {
  if (n_slot) k_rcsr_fill<T><<<n_slot, 256, 0, st>>>(d_subs, d_slots, idx, chi, row_ptr, cursor, rslot, rchi);
}
void launch_rcsr_count(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const int* idx, int* cnt,
                       cudaStream_t st) {
  if (n_slot) k_rcsr_count<<<n_slot, 256, 0, st>>>(d_subs, d_slots, idx, cnt);
}

template <typename T>
void launch_nl_back_csr(const SubDev* d_subs, int n_sub, long long max_nd, int max_ns, int list_max,
                        const long long* row_ptr, const int* rslot, const typename Vec4<T>::type* rchi,
                        const int* blk_cnt, const int* blk_list, const double* P, T* Yout, const StepCoef* coef,
                        int step, int ppt, cudaStream_t st) {
  if (list_max == 0) return;
  const int kv = ppt == 16 ? 16 : 8;   // ppt 16: one point per thread, 16 vectors per CTA
  const size_t smem = (size_t)list_max * (kv + 1) * sizeof(typename Vec4<T>::type);
  auto kern = ppt == 16 ? k_nl_back_csr<T, 1, 16> : (ppt == 2 ? k_nl_back_csr<T, 2, 8> : k_nl_back_csr<T, 1, 8>);
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((max_ns + kv - 1) / kv, (unsigned)((max_nd + kBackPts - 1) / kBackPts), n_sub);
  kern<<<grid, 256, smem, st>>>(d_subs, row_ptr, rslot, rchi, blk_cnt, blk_list, list_max, P, Yout, coef, step);
}

template <typename T>
void launch_proj_table_count(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const AtomImg* d_imgs,
                             int* counts, cudaStream_t st) {
  if (n_slot) k_proj_count<T><<<n_slot, 256, 0, st>>>(d_subs, d_slots, d_imgs, counts);
}
template <typename T>
void launch_proj_table_fill(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const AtomImg* d_imgs, int* idx,
                            typename Vec4<T>::type* chi, cudaStream_t st) {
  if (n_slot) k_proj_fill<T><<<n_slot, 256, 0, st>>>(d_subs, d_slots, d_imgs, idx, chi);
}

template <typename T, int KPV, int NW>
void launch_nl_project_w(const SubDev* d_subs, const ProjSlot* d_slots, int slot_off, int n_slot, const int* idx,
                         const typename Vec4<T>::type* chi, int max_ns, const T* Y, double* P, int chunk_slots,
                         cudaStream_t st) {
  const int groups = (max_ns + KPV - 1) / KPV;
  const int chunks = (n_slot + chunk_slots - 1) / chunk_slots;
  k_nl_project<T, KPV, NW><<<chunks * chunk_slots * groups, NW * 32, 0, st>>>(d_subs, d_slots, slot_off, n_slot, groups,
                                                                              chunk_slots, idx, chi, Y, P);
}

// kpv vectors per CTA of nw warps: (8, 8), (16, 8), (32, 8), (8, 4) or (16, 4) (anything else runs
// (8, 8)); chunk_slots: 256, 512 or 1024
template <typename T>
void launch_nl_project(const SubDev* d_subs, const ProjSlot* d_slots, int slot_off, int n_slot, const int* idx,
                       const typename Vec4<T>::type* chi, int max_ns, const T* Y, double* P, int kpv, int nw,
                       int chunk_slots, cudaStream_t st) {
  if (n_slot == 0) return;
  if (chunk_slots != 256 && chunk_slots != 1024) chunk_slots = 512;
  if (nw == 4 && kpv == 8) launch_nl_project_w<T, 8, 4>(d_subs, d_slots, slot_off, n_slot, idx, chi, max_ns, Y, P, chunk_slots, st);
  else if (nw == 4 && kpv == 16) launch_nl_project_w<T, 16, 4>(d_subs, d_slots, slot_off, n_slot, idx, chi, max_ns, Y, P, chunk_slots, st);
  else if (kpv == 32) launch_nl_project_w<T, 32, 8>(d_subs, d_slots, slot_off, n_slot, idx, chi, max_ns, Y, P, chunk_slots, st);
  else if (kpv == 16) launch_nl_project_w<T, 16, 8>(d_subs, d_slots, slot_off, n_slot, idx, chi, max_ns, Y, P, chunk_slots, st);
  else launch_nl_project_w<T, 8, 8>(d_subs, d_slots, slot_off, n_slot, idx, chi, max_ns, Y, P, chunk_slots, st);
}

template <typename T>
void launch_nl_back(const SubDev* d_subs, const ProjSlot* d_slots, int n_slot, const int* idx,
                    const typename Vec4<T>::type* chi, int max_ns, const double* P, T* Yout, const StepCoef* coef,
                    int step, cudaStream_t st) {
  if (n_slot == 0) return;
  dim3 grid(n_slot, (max_ns + kNlWarps * kNlVec - 1) / (kNlWarps * kNlVec));
  k_nl_back<T><<<grid, kNlWarps * 32, 0, st>>>(d_subs, d_slots, idx, chi, P, Yout, coef, step);
}

#define XLS_INST_NL(T)                                                                                              \
  template void launch_proj_table_count<T>(const SubDev*, const ProjSlot*, int, const AtomImg*, int*, cudaStream_t); \
  template void launch_proj_table_fill<T>(const SubDev*, const ProjSlot*, int, const AtomImg*, int*,                 \
                                          Vec4<T>::type*, cudaStream_t);                                             \
  template void launch_nl_project<T>(const SubDev*, const ProjSlot*, int, int, const int*, const Vec4<T>::type*,     \
                                     int, const T*, double*, int, int, int, cudaStream_t);                           \
  template void launch_nl_back<T>(const SubDev*, const ProjSlot*, int, const int*, const Vec4<T>::type*, int,        \
                                  const double*, T*, const StepCoef*, int, cudaStream_t);                            \
  template void launch_rcsr_build<T>(const SubDev*, const ProjSlot*, int, const int*, const Vec4<T>::type*,         \
                                     const long long*, int*, int*, Vec4<T>::type*, cudaStream_t);                    \
  template void launch_nl_back_csr<T>(const SubDev*, int, long long, int, int, const long long*, const int*,        \
                                      const Vec4<T>::type*, const int*, const int*, const double*, T*,                \
                                      const StepCoef*, int, int, cudaStream_t);                                       \
  template void launch_nl_project1<T>(const SubDev*, const ProjSlot*, int, const int*, const Vec4<T>::type*,         \
                                      const T*, double*, cudaStream_t);                                               \
  template void launch_nl_back1<T>(const SubDev*, int, long long, int, const long long*, const int*,                \
                                   const Vec4<T>::type*, const int*, const double*, T*, const StepCoef*, int,          \
                                   cudaStream_t);
XLS_INST_NL(double)
XLS_INST_NL(float)

template void launch_stencil<double>(const SubDev*, int, const Plan&, const double*, const double*, double*,
                                     const double*, const StepCoef*, int, cudaStream_t);
template void launch_stencil<float>(const SubDev*, int, const Plan&, const float*, const float*, float*,
                                    const float*, const StepCoef*, int, cudaStream_t);
}  // namespace xls
