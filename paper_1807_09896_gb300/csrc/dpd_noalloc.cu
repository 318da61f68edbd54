// dpd_noalloc.cu -- velocity-profile sums over caller-owned device arrays that
// allocate no memory at all.
//
// Some callers cannot call cudaMalloc: a framework that owns every byte of
// device memory through its own pool and forbids side allocations, a
// memory-capped process that must not grow its footprint, or a latency-bound
// loop where cudaMalloc/cudaFree would synchronise the device.  This entry point
// serves them: the caller passes the particle arrays and the output, and the
// FP64 bin accumulators live in a fixed, file-scope device array that every GPU
// loading the library holds until the process exits (kNoAllocMaxBins x 5
// doubles = 160 KiB).
#include <cuda.h>

#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/dpd.h"
#include "dpd_common.cuh"
#include "dpd_launch.h"

namespace {

constexpr int kNoAllocMaxBins = DPD_NOALLOC_MAX_BINS;

// Accumulators shared by every call on a device.  Each call clears the part it
// uses before accumulating; calls that overlap on the GPU (different streams)
// race on this array.
static __device__ __align__(256) double g_profile_scratch[5 * kNoAllocMaxBins];

// Device address of g_profile_scratch in each CUDA context this process used,
// keyed by the context's unique id: a context created after a cudaDeviceReset (or
// any new context on the same device) reloads the module, so its array has a new
// address, and a key by device ordinal alone would hand out a stale one.  In host
// code the symbol itself is only a host-side stand-in; a kernel given it would
// fault or touch the wrong memory, so only these addresses are passed.
struct ScratchEntry {
  unsigned long long ctx_id;
  void* addr;
};
std::mutex g_mu;
std::vector<ScratchEntry> g_scratch;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
std::once_flag g_entry_once;

// Driver entry points through the runtime (no link against the driver library).
void find_entry_points() {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
          cudaSuccess && q == cudaDriverEntryPointSuccess)
    g_ctx_current = (CtxGetCurrentFn)f;
  f = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
          cudaSuccess && q == cudaDriverEntryPointSuccess)
    g_ctx_id = (CtxGetIdFn)f;
}

// Address of the scratch array in the current context: looked up with
// cudaGetSymbolAddress once per context (the runtime makes the device's primary
// context current on that first lookup), then taken from the table.
cudaError_t scratch_address(void** out) {
  std::call_once(g_entry_once, find_entry_points);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ctx_current || !g_ctx_id) return cudaGetSymbolAddress(out, g_profile_scratch);
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) {
    // no context yet on this thread: the lookup creates the primary one
    const cudaError_t e = cudaGetSymbolAddress(out, g_profile_scratch);
    if (e != cudaSuccess) return e;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return cudaSuccess;
  }
  unsigned long long id = 0;
  if (g_ctx_id(ctx, &id) != CUDA_SUCCESS) return cudaGetSymbolAddress(out, g_profile_scratch);
  for (const ScratchEntry& en : g_scratch)
    if (en.ctx_id == id) {
      *out = en.addr;
      return cudaSuccess;
    }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_profile_scratch);
  if (e != cudaSuccess) return e;
  g_scratch.push_back({id, p});
  *out = p;
  return cudaSuccess;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Same sums as the handle's profile kernel, for arrays in any order with the
// particle type in its own byte array.  Lanes that share a bin add their values
// with a butterfly; one lane per warp and bin issues the FP64 atomics.
__global__ void __launch_bounds__(256)
k_profile_noalloc(const float4* __restrict__ pos, const float4* __restrict__ vel,
                  const uint8_t* __restrict__ type, int n, int axis, int nbins, float lo,
                  float inv_w, double* acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool pending = false;
  int bin = 0;
  double vx = 0, vy = 0, vz = 0;
  if (i < n && type[i] == 0) {
    const float4 p = pos[i];
    const float x = axis == 0 ? p.x : (axis == 1 ? p.y : p.z);
    const float fb = floorf(__fmul_rn(__fsub_rn(x, lo), inv_w));
    if (fb >= 0.0f && fb < (float)nbins) {
      bin = (int)fb;
      pending = true;
      const float4 v = vel[i];
      vx = v.x; vy = v.y; vz = v.z;
    }
  }
  unsigned mask = __ballot_sync(0xffffffffu, pending);
  while (mask) {
    const int leader = __ffs(mask) - 1;
    const int b0 = __shfl_sync(0xffffffffu, bin, leader);
    const bool mine = pending && bin == b0;
    const double c = warp_sum_d(mine ? 1.0 : 0.0);
    const double sx = warp_sum_d(mine ? vx : 0.0);
    const double sy = warp_sum_d(mine ? vy : 0.0);
    const double sz = warp_sum_d(mine ? vz : 0.0);
    const double s2 = warp_sum_d(mine ? vx * vx + vy * vy + vz * vz : 0.0);
    if (lane == leader) {
      double* a = acc + 5 * b0;
      atomicAdd(a + 0, c);
      atomicAdd(a + 1, sx);
      atomicAdd(a + 2, sy);
      atomicAdd(a + 3, sz);
      atomicAdd(a + 4, s2);
    }
    if (mine) pending = false;
    mask = __ballot_sync(0xffffffffu, pending);
  }
}

int nofail(const char* fmt, int code, long a = 0, long b = 0) {
  char buf[256];
  snprintf(buf, sizeof buf, fmt, a, b);
  dpd::set_global_error(buf);
  return code;
}

}  // namespace

extern "C" int dpd_velocity_profile_noalloc(const float* pos4, const float* vel4,
                                            const uint8_t* type, int n, int axis, int nbins,
                                            double lo, double hi, double* out, int where,
                                            void* stream) {
  if (n < 0 || (n > 0 && (!pos4 || !vel4 || !type)) || !out)
    return nofail("dpd_velocity_profile_noalloc: null array or negative n (%ld)", DPD_EINVAL, n);
  if (axis < 0 || axis > 2 || !(hi > lo))
    return nofail("dpd_velocity_profile_noalloc: bad axis %ld or empty range", DPD_EINVAL, axis);
  if (nbins < 1 || nbins > kNoAllocMaxBins)
    return nofail("dpd_velocity_profile_noalloc: nbins = %ld outside 1..%ld (the fixed scratch holds "
                  "DPD_NOALLOC_MAX_BINS bins)", DPD_EINVAL, nbins, kNoAllocMaxBins);
  if (where != DPD_HOST && where != DPD_DEVICE)
    return nofail("dpd_velocity_profile_noalloc: bad `where` (%ld)", DPD_EINVAL, where);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nofail("dpd_velocity_profile_noalloc: no CUDA device", DPD_ECUDA);
  void* scratch = nullptr;
  e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return nofail("dpd_velocity_profile_noalloc: cudaGetSymbolAddress failed", DPD_ECUDA);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * 5 * (size_t)nbins;
  double* acc = (double*)scratch;
  e = cudaMemsetAsync(acc, 0, bytes, s);
  if (e == cudaSuccess && n > 0) {
    const float lo_f = (float)lo;
    const float inv_w = (float)((double)nbins / (hi - lo));
    k_profile_noalloc<<<(n + 255) / 256, 256, 0, s>>>((const float4*)pos4, (const float4*)vel4, type,
                                                       n, axis, nbins, lo_f, inv_w, acc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, acc, bytes,
                        where == DPD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && where == DPD_HOST) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof buf, "dpd_velocity_profile_noalloc: %s", cudaGetErrorString(e));
    dpd::set_global_error(buf);
    return DPD_ECUDA;
  }
  return DPD_OK;
}
