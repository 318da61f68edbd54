// dpd_force.cu -- the pair-force kernel of the DPD step (Eqs. 2-10 of Xu &
// Meakin, arXiv:1807.09896) fused with the closing half-kick of the modified
// velocity-Verlet scheme.
//
// One thread per particle in cell order.  Each fluid particle i scans the 27
// cells around its own (the three x-neighbour cells of a row are one
// contiguous range of the cell-sorted arrays, so a scan is 9 ranges away from
// the periodic x seam), keeps the indices j with r_ij < r_c in a per-thread list
// in shared memory, and then evaluates
//   f_ij = [a_ij (1 - r) - gamma (1 - r)^2 (rhat . vt_ij) + sigma (1 - r) xi_ij / sqrt(dt)] rhat
// for each of them.  Splitting the cheap candidate test from the expensive pair
// work (a Philox4x32-10 block, a logarithm, a square root, a cosine) keeps the
// lanes of a warp busy together in the expensive part: roughly 1 candidate in 6
// is inside the cutoff.
// Every pair is evaluated from both sides (no atomics, no scatter): the noise key
// is symmetric and the minimum-image separation is exactly antisymmetric, so
// f_ji = -f_ij bit for bit.  The sum runs in a fixed order (cells in index
// order, particles by id), which makes the result independent of scheduling.
#include "dpd_common.cuh"
#include "dpd_launch.h"

namespace dpd {

constexpr int kForceThreads = 128;
constexpr int kListCap = 24;

__global__ void __launch_bounds__(kForceThreads)
k_force(StepParams P, Arrays A, const uint32_t* __restrict__ start, int n, DevCounters* ctr,
        int kick) {
  __shared__ int list[kListCap][kForceThreads];
  const int i = blockIdx.x * kForceThreads + threadIdx.x;
  if (i >= n) return;
  const float4 pi = A.pos[i];
  if (is_solid(pi.w)) return;
  const float4 vti = A.vt[i];
  const uint32_t idi = id_of(pi.w);
  const uint32_t step = ctr->step;
  const float4* __restrict__ pos = A.pos;
  const float4* __restrict__ vt = A.vt;

  float fx = 0.f, fy = 0.f, fz = 0.f;
  int cnt = 0;

  auto flush = [&]() {
    for (int k = 0; k < cnt; ++k) {
      const int j = list[k][threadIdx.x];
      const float4 pj = __ldg(&pos[j]);
      const float dx = min_image(pi.x, pj.x, P.L[0], P.halfL[0]);
      const float dy = min_image(pi.y, pj.y, P.L[1], P.halfL[1]);
      const float dz = min_image(pi.z, pj.z, P.L[2], P.halfL[2]);
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float inv_r = rsqrtf(r2);
      const float r = r2 * inv_r;
      const float w = 1.0f - r;
      const float ex = dx * inv_r, ey = dy * inv_r, ez = dz * inv_r;
      float vjx, vjy, vjz, a;
      if (is_solid(pj.w)) {
        vjx = P.vw[0]; vjy = P.vw[1]; vjz = P.vw[2];
        a = P.a_fs;
      } else {
        const float4 vtj = __ldg(&vt[j]);
        vjx = vtj.x; vjy = vtj.y; vjz = vtj.z;
        a = P.a_ff;
      }
      const float ev = ex * (vti.x - vjx) + ey * (vti.y - vjy) + ez * (vti.z - vjz);
      const float xi = pair_noise(idi, id_of(pj.w), step, P.sys, P.seed_lo, P.seed_hi);
      const float mag = w * (a - P.gamma * w * ev + P.sigma_rsqdt * xi);
      fx = fmaf(mag, ex, fx);
      fy = fmaf(mag, ey, fy);
      fz = fmaf(mag, ez, fz);
    }
    cnt = 0;
  };

  auto scan = [&](uint32_t b, uint32_t e) {
    for (uint32_t j = b; j < e; ++j) {
      const float4 pj = __ldg(&pos[j]);
      const float dx = min_image(pi.x, pj.x, P.L[0], P.halfL[0]);
      const float dy = min_image(pi.y, pj.y, P.L[1], P.halfL[1]);
      const float dz = min_image(pi.z, pj.z, P.L[2], P.halfL[2]);
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < 1.0f && r2 > 0.0f) {
        list[cnt][threadIdx.x] = (int)j;
        if (++cnt == kListCap) flush();
      }
    }
  };

  const int cx = cell_coord(pi.x, P.inv_edge[0], P.nc[0]);
  const int cy = cell_coord(pi.y, P.inv_edge[1], P.nc[1]);
  const int cz = cell_coord(pi.z, P.inv_edge[2], P.nc[2]);
  const int ncx = P.nc[0], ncy = P.nc[1], ncz = P.nc[2];
  for (int dz = -1; dz <= 1; ++dz) {
    int z = cz + dz;
    z = z < 0 ? z + ncz : (z >= ncz ? z - ncz : z);
    for (int dy = -1; dy <= 1; ++dy) {
      int y = cy + dy;
      y = y < 0 ? y + ncy : (y >= ncy ? y - ncy : y);
      const int row = (z * ncy + y) * ncx;
      if (cx > 0 && cx < ncx - 1) {
        scan(__ldg(&start[row + cx - 1]), __ldg(&start[row + cx + 2]));
      } else {
        for (int dx = -1; dx <= 1; ++dx) {
          int x = cx + dx;
          x = x < 0 ? x + ncx : (x >= ncx ? x - ncx : x);
          scan(__ldg(&start[row + x]), __ldg(&start[row + x + 1]));
        }
      }
    }
  }
  flush();

  const float4 f_old = A.frc[i];
  A.frc[i] = make_float4(fx, fy, fz, 0.0f);
  if (kick && vti.w == 0.0f) {
    // Closing half-kick: v(t+dt) = v(t) + dt/2 (F(t) + F(t+dt)), F = f + g.
    float4 v = A.vel[i];
    v.x = fmaf(P.half_dt, (f_old.x + fx) + 2.0f * P.g[0], v.x);
    v.y = fmaf(P.half_dt, (f_old.y + fy) + 2.0f * P.g[1], v.y);
    v.z = fmaf(P.half_dt, (f_old.z + fz) + 2.0f * P.g[2], v.z);
    A.vel[i] = v;
  }
  if (!(isfinite(fx) && isfinite(fy) && isfinite(fz)))
    atomicOr(&ctr->status, ST_NAN);
}

void launch_force(const StepParams& P, const Arrays& A, const uint32_t* start, int n,
                  DevCounters* ctr, int kick, cudaStream_t s) {
  if (n <= 0) return;
  const int nb = (n + kForceThreads - 1) / kForceThreads;
  k_force<<<nb, kForceThreads, 0, s>>>(P, A, start, n, ctr, kick);
}

}  // namespace dpd
