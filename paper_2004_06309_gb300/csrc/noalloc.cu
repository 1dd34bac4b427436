// hz_cgs2_noalloc: the CGS2 orthogonalisation step of hz_cgs2 for callers that
// cannot allocate device memory -- code running where cudaMalloc is forbidden or
// unavailable (inside a memory-pool-managed runtime that owns every byte of the
// device, a real-time loop that must not synchronise on an allocation, or a
// caller without an hz context).  The caller passes every input and output; the
// only other memory the step needs, its per-block partial sums, lives in a
// file-scope device array of fixed size that every GPU loading this library
// holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/hz.h"
#include "dev.h"

namespace {

constexpr int kBlocks = 152 * 4;        // partial-sum blocks of the CGS kernels (hz::cgs_blocks())
constexpr int kSlots = 65;              // per block: 64 dot products + the squared norm
constexpr int kMaxCols = 64;
// partial sums (kBlocks x kSlots), then the reduced h1, h2 and norm (3 x kSlots): 635,440 bytes
constexpr size_t kScratchElems = size_t(kBlocks) * kSlots + 3 * kSlots;

static __device__ __align__(256) double2 g_cgs2_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_scratch[kMaxDevices] = {};

// The device address of g_cgs2_scratch for the current device.  The name of the
// array in host code is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached for the life of the
// process; a device reset in between would leave the cached address stale.
hz_status scratch_address(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "hz_cgs2_noalloc: cudaGetDevice: %s\n", cudaGetErrorString(e));
    return HZ_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    std::fprintf(stderr, "hz_cgs2_noalloc: device %d beyond the %d supported\n", dev, kMaxDevices);
    return HZ_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cgs2_scratch);
    if (e != cudaSuccess || !p) {
      std::fprintf(stderr, "hz_cgs2_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
      return HZ_ERR_CUDA;
    }
    g_scratch[dev] = static_cast<double2*>(p);
  }
  *out = g_scratch[dev];
  return HZ_OK;
}

__global__ void k_sqrt_norm(const double2* nrm, double* out) {
  if (threadIdx.x == 0) *out = sqrt(nrm[kMaxCols].x);
}

}  // namespace

extern "C" hz_status hz_cgs2_noalloc(const void* V, int64_t n, int64_t ldv, int32_t ncols, void* w, void* h,
                                     void* wnorm, uintptr_t stream) {
  if (!V || !w || !h || !wnorm || n < 1 || ldv < n) {
    std::fprintf(stderr, "hz_cgs2_noalloc: null pointer, n < 1 or ldv < n\n");
    return HZ_ERR_ARG;
  }
  if (ncols < 1 || ncols > kMaxCols) {
    std::fprintf(stderr,
                 "hz_cgs2_noalloc: ncols = %d; the static scratch holds partial sums for at most %d columns\n",
                 ncols, kMaxCols);
    return HZ_ERR_ARG;
  }
  if (hz::cgs_blocks() != kBlocks) {
    std::fprintf(stderr, "hz_cgs2_noalloc: scratch sized for %d blocks, kernels use %d\n", kBlocks,
                 hz::cgs_blocks());
    return HZ_ERR_ARG;
  }
  double2* s = nullptr;
  hz_status st = scratch_address(&s);
  if (st != HZ_OK) return st;
  double2* partial = s;
  double2* h1 = s + size_t(kBlocks) * kSlots;
  double2* h2 = h1 + kSlots;
  double2* nrm = h2 + kSlots;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const double2* Vd = static_cast<const double2*>(V);
  double2* wd = static_cast<double2*>(w);
  // Every slot read below is written earlier in the same call, so nothing from a
  // previous call (which leaves its values in the array) leaks into this one.
  hz::launch_cgs(n, ncols, Vd, ldv, nullptr, wd, ncols, partial, cs);
  hz::launch_reduce(partial, kBlocks, ncols, h1, cs);
  hz::launch_cgs(n, ncols, Vd, ldv, h1, wd, ncols, partial, cs);
  hz::launch_reduce(partial, kBlocks, ncols, h2, cs);
  hz::launch_cgs(n, ncols, Vd, ldv, h2, wd, 0, partial, cs);
  hz::launch_reduce(partial, kBlocks, 0, nrm, cs);
  hz::launch_add2(ncols, h1, h2, static_cast<double2*>(h), cs);
  k_sqrt_norm<<<1, 32, 0, cs>>>(nrm, static_cast<double*>(wnorm));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "hz_cgs2_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return HZ_ERR_CUDA;
  }
  return HZ_OK;
}
