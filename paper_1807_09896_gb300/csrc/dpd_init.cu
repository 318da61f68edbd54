// dpd_init.cu -- particle set-up from the phase field (Xu & Meakin, arXiv:1807.09896,
// Sec. II.C): a dense random fluid fills the whole box, then the interpolated phase
// field classifies every particle -- phi >= 0 fluid, phi_min < phi < 0 frozen solid
// (the layer that carries the wall), phi <= phi_min removed (deep solid, not needed).
//
// Site k of N0 = round(rho V) draws its position from Philox4x32-10 of the counter
// (k, 0xFFFFFFFF, 0xFFFFFFFE, system) and its velocity from (k, 0xFFFFFFFF, 0xFFFFFFFD,
// system), both under the key (seed_lo, seed_hi); pair noise never uses a counter word
// 1 of 0xFFFFFFFF (ids stay below 2^31), so the streams are disjoint.  Uniforms are
// u = ((w >> 9) + 1/2) 2^-23; position r = (u0 Lx, u1 Ly, u2 Lz); velocity
// sqrt(kBT) (n0, n1, n2) with n0, n1 = sqrt(-2 ln u0) (cos, sin)(2 pi u1) and
// n2 = sqrt(-2 ln u2) cos(2 pi u3) (Box-Muller).  The mean fluid velocity is removed;
// kept sites get ids 0..n-1 in order of k.  Everything is deterministic: block sums
// use fixed reduction trees and the block offsets are summed in order.
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/dpd.h"
#include "dpd_common.cuh"
#include "dpd_system.h"

namespace {

constexpr int kInitThreads = 256;
constexpr uint32_t kKeepNone = 2u;  // type code of a removed site

struct SiteOut {
  float4* pos;
  float4* vel;
  uint8_t* type;
  uint32_t* block_keep;   // kept sites per block
  uint32_t* block_fluid;  // fluid sites per block
  double* block_vsum;     // per block: sum vx, vy, vz of fluid sites
};

__global__ void __launch_bounds__(kInitThreads) k_init_sites(dpd::StepParams P, long n0, uint32_t k0,
                                                             uint32_t k1, float sqrt_kbt, float phi_min,
                                                             SiteOut o) {
  __shared__ uint32_t s_keep[kInitThreads], s_fluid[kInitThreads];
  __shared__ double s_v[3][kInitThreads];
  const long k = (long)blockIdx.x * kInitThreads + threadIdx.x;
  uint32_t keep = 0, fluid = 0;
  double vx = 0.0, vy = 0.0, vz = 0.0;
  if (k < n0) {
    uint32_t a0 = (uint32_t)k, a1 = 0xFFFFFFFFu, a2 = 0xFFFFFFFEu, a3 = P.sys;
    dpd::philox4x32_10(a0, a1, a2, a3, k0, k1);
    const float x = dpd::philox_u01(a0) * P.L[0];
    const float y = dpd::philox_u01(a1) * P.L[1];
    const float z = dpd::philox_u01(a2) * P.L[2];
    uint32_t b0 = (uint32_t)k, b1 = 0xFFFFFFFFu, b2 = 0xFFFFFFFDu, b3 = P.sys;
    dpd::philox4x32_10(b0, b1, b2, b3, k0, k1);
    const float u0 = dpd::philox_u01(b0), u1 = dpd::philox_u01(b1);
    const float u2 = dpd::philox_u01(b2), u3 = dpd::philox_u01(b3);
    const float ra = sqrtf(-2.0f * logf(u0)), rb = sqrtf(-2.0f * logf(u2));
    const float v0 = sqrt_kbt * ra * cospif(2.0f * u1);
    const float v1 = sqrt_kbt * ra * sinpif(2.0f * u1);
    const float v2 = sqrt_kbt * rb * cospif(2.0f * u3);
    const float phi = P.phi ? dpd::phi_at(P, x, y, z, 0.f, 0.f, 0.f) : 1.0f;
    const uint32_t type = phi >= 0.0f ? 0u : (phi > phi_min ? 1u : kKeepNone);
    keep = type != kKeepNone;
    o.pos[k] = make_float4(x, y, z, 0.0f);
    o.vel[k] = type == 0u ? make_float4(v0, v1, v2, 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
    o.type[k] = (uint8_t)type;
    if (type == 0u) {
      fluid = 1;
      vx = v0;
      vy = v1;
      vz = v2;
    }
  }
  s_keep[threadIdx.x] = keep;
  s_fluid[threadIdx.x] = fluid;
  s_v[0][threadIdx.x] = vx;
  s_v[1][threadIdx.x] = vy;
  s_v[2][threadIdx.x] = vz;
  __syncthreads();
  for (int w = kInitThreads / 2; w > 0; w >>= 1) {  // fixed tree: same sums every run
    if (threadIdx.x < w) {
      s_keep[threadIdx.x] += s_keep[threadIdx.x + w];
      s_fluid[threadIdx.x] += s_fluid[threadIdx.x + w];
      for (int c = 0; c < 3; ++c) s_v[c][threadIdx.x] += s_v[c][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    o.block_keep[blockIdx.x] = s_keep[0];
    o.block_fluid[blockIdx.x] = s_fluid[0];
    for (int c = 0; c < 3; ++c) o.block_vsum[3 * (size_t)blockIdx.x + c] = s_v[c][0];
  }
}

// One thread: block offsets (exclusive prefix, in order) and the mean fluid velocity.
__global__ void k_init_offsets(int nblocks, const uint32_t* block_keep, const uint32_t* block_fluid,
                               const double* block_vsum, uint32_t* block_off, uint32_t* totals,
                               double* mean) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t acc = 0, nf = 0;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < nblocks; ++b) {
    block_off[b] = acc;
    acc += block_keep[b];
    nf += block_fluid[b];
    for (int c = 0; c < 3; ++c) s[c] += block_vsum[3 * (size_t)b + c];
  }
  totals[0] = acc;
  totals[1] = nf;
  for (int c = 0; c < 3; ++c) mean[c] = nf > 0 ? s[c] / (double)nf : 0.0;
}

__global__ void __launch_bounds__(kInitThreads) k_init_compact(long n0, const float4* pos, const float4* vel,
                                                               const uint8_t* type, const uint32_t* block_off,
                                                               const double* mean, float4* out_pos,
                                                               float4* out_vel, int* out_id, uint8_t* out_type) {
  __shared__ uint32_t s_scan[kInitThreads];
  const long k = (long)blockIdx.x * kInitThreads + threadIdx.x;
  const uint32_t t = k < n0 ? type[k] : kKeepNone;
  const uint32_t keep = t != kKeepNone;
  s_scan[threadIdx.x] = keep;
  __syncthreads();
  for (int w = 1; w < kInitThreads; w <<= 1) {  // inclusive scan (Hillis-Steele)
    const uint32_t v = threadIdx.x >= w ? s_scan[threadIdx.x - w] : 0u;
    __syncthreads();
    s_scan[threadIdx.x] += v;
    __syncthreads();
  }
  if (!keep) return;
  const uint32_t d = block_off[blockIdx.x] + s_scan[threadIdx.x] - 1u;
  float4 v = vel[k];
  if (t == 0u) {
    v.x = (float)((double)v.x - mean[0]);
    v.y = (float)((double)v.y - mean[1]);
    v.z = (float)((double)v.z - mean[2]);
  }
  out_pos[d] = pos[k];
  out_vel[d] = v;
  out_id[d] = (int)d;
  out_type[d] = (uint8_t)t;
}

}  // namespace

extern "C" int dpd_init_particles(dpd_t* h, uint64_t seed, double solid_layer) {
  if (!h) return DPD_EINVAL;
  char msg[256];
  auto fail = [&](int code, const char* m) {
    h->err = m;
    return code;
  };
  if (!(solid_layer >= 0.0) || !std::isfinite(solid_layer)) return fail(DPD_EINVAL, "solid_layer must be >= 0");
  const double volume = h->box[0] * h->box[1] * h->box[2];
  const double n0d = std::floor(h->rho * volume + 0.5);
  if (n0d >= (double)(1 << 30)) return fail(DPD_EOVERFLOW, "too many sites (rho x volume >= 2^30)");
  const long n0 = (long)n0d;
  // phi_min: the phase field of Eq. 14 at signed distance -solid_layer
  const double phi_min = std::tanh(-solid_layer / (std::sqrt(2.0) * h->phase_eps));
  const int nb = (int)((n0 + kInitThreads - 1) / kInitThreads);
  dpd::StepParams P = dpd::make_params(h);
  cudaStream_t st = h->E.stream;
  float4 *pos = nullptr, *vel = nullptr, *opos = nullptr, *ovel = nullptr;
  uint8_t *type = nullptr, *otype = nullptr;
  int* oid = nullptr;
  uint32_t *bk = nullptr, *bf = nullptr, *boff = nullptr, *tot = nullptr;
  double *bv = nullptr, *mean = nullptr;
  const size_t m = n0 > 0 ? (size_t)n0 : 1, b = nb > 0 ? (size_t)nb : 1;
  cudaError_t e = cudaMalloc((void**)&pos, sizeof(float4) * m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&vel, sizeof(float4) * m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&type, m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&opos, sizeof(float4) * m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ovel, sizeof(float4) * m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&otype, m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&oid, sizeof(int) * m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&bk, sizeof(uint32_t) * b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&bf, sizeof(uint32_t) * b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&boff, sizeof(uint32_t) * b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&tot, sizeof(uint32_t) * 2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&bv, sizeof(double) * 3 * b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&mean, sizeof(double) * 3);
  uint32_t totals[2] = {0, 0};
  if (e == cudaSuccess && nb > 0) {
    SiteOut o{pos, vel, type, bk, bf, bv};
    k_init_sites<<<nb, kInitThreads, 0, st>>>(P, n0, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                             (float)std::sqrt(h->kBT), (float)phi_min, o);
    k_init_offsets<<<1, 32, 0, st>>>(nb, bk, bf, bv, boff, tot, mean);
    k_init_compact<<<nb, kInitThreads, 0, st>>>(n0, pos, vel, type, boff, mean, opos, ovel, oid, otype);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(totals, tot, sizeof totals, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  int rc = DPD_OK;
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "dpd_init_particles: %s", cudaGetErrorString(e));
    rc = fail(e == cudaErrorMemoryAllocation ? DPD_ENOMEM : DPD_ECUDA, msg);
  } else {
    rc = dpd_set_particles(h, (int)totals[0], (const float*)opos, (const float*)ovel, oid, otype,
                           DPD_DEVICE);
  }
  cudaFree(pos);
  cudaFree(vel);
  cudaFree(type);
  cudaFree(opos);
  cudaFree(ovel);
  cudaFree(otype);
  cudaFree(oid);
  cudaFree(bk);
  cudaFree(bf);
  cudaFree(boff);
  cudaFree(tot);
  cudaFree(bv);
  cudaFree(mean);
  return rc;
}
