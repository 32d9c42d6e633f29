// Allocation-free Gram entry point.
//
// Some callers cannot let a library allocate device memory: an application whose device memory
// is owned by its own pool allocator (memory obtained any other way escapes its accounting and
// limits), or a latency-critical loop in which the implicit device-wide synchronisation of
// cudaMalloc / cudaFree is not acceptable.  xls_gram_noalloc serves them: it computes the
// projected matrices of one block of vectors with the split-BF16 tensor-core Gram kernel, and
// its only scratch (the per-CTA FP32 partial sums and a status word) is the file-scope array
// below, which every GPU that loads the library holds until the process exits.
#include <algorithm>
#include <mutex>
#include <string>

#include "xls_internal.h"

namespace {

constexpr int kMaxJobs = 64;  // CTAs of one call: block pairs x K chunks
constexpr size_t kStatusFloats = 64;                                  // 256 bytes: status word
constexpr size_t kScratchFloats = kStatusFloats + (size_t)kMaxJobs * 2 * 128 * 128;  // 8 MiB + 256 B
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_gram_scratch[kScratchFloats];

std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

xls_status err(xls_status s, const std::string& m) {
  xls::set_last_error(m);
  return s;
}

}  // namespace

extern "C" xls_status xls_gram_noalloc(const float* psi_f, const float* hpsi_f, long long n_points, int n_states,
                                       double* Ms_out, double* Hs_out, void* cuda_stream) {
  if (!psi_f || !hpsi_f || !Ms_out || !Hs_out) return err(XLS_EINVAL, "xls_gram_noalloc: null pointer");
  if (n_states < 1 || n_states > 256)
    return err(XLS_EINVAL, "xls_gram_noalloc: n_states must be in 1..256 (the fixed scratch holds two 128-row blocks)");
  if (n_points < 8 || n_points % 8 != 0)
    return err(XLS_EINVAL, "xls_gram_noalloc: n_points must be a positive multiple of 8");
  if (((uintptr_t)psi_f | (uintptr_t)hpsi_f) & 15) return err(XLS_EINVAL, "xls_gram_noalloc: inputs must be 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(XLS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return err(XLS_EINVAL, "xls_gram_noalloc: device index beyond the supported range");
  float* base = nullptr;
  {
    // set-up, once per device with that device current: the device address of the scratch array
    // (in host code the array's name is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_gram_scratch);
      if (e != cudaSuccess) return err(XLS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    base = g_scratch_ptr[dev];
  }
  // an error left pending by earlier, unrelated work would otherwise be reported as this call's
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return err(XLS_ECUDA, std::string("xls_gram_noalloc: a CUDA error was pending before the call: ") +
                              cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* status = reinterpret_cast<int*>(base);
  float* work = base + kStatusFloats;
  const int pairs = xls::gram_single_pairs(n_states);
  const long long nkt = (n_points + 63) / 64;
  const int kc = (int)std::max(1LL, std::min<long long>(kMaxJobs / pairs, nkt));
  // the status word must start at zero; every partial sum the reduction reads is written first
  e = cudaMemsetAsync(status, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return err(XLS_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  if (!xls::launch_gram_tc_single(psi_f, hpsi_f, n_points, n_states, kc, work, Ms_out, Hs_out, status, st))
    return err(XLS_ECUDA, "xls_gram_noalloc: the tensor-core kernel's shared memory could not be configured");
  e = cudaGetLastError();
  if (e != cudaSuccess) return err(XLS_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  int h = 0;
  e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return err(XLS_ECUDA, std::string("xls_gram_noalloc: ") + cudaGetErrorString(e));
  if (h != 0) return err(XLS_ETIMEOUT, "xls_gram_noalloc: a bounded device wait gave up");
  return XLS_OK;
}
