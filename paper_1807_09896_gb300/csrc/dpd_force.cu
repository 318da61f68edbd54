// dpd_force.cu -- the pair-force kernel of the DPD step (Eqs. 2-10 of Xu &
// Meakin, arXiv:1807.09896) fused with the second half of the closing kick of the
// modified velocity-Verlet scheme (the drift kernel applies the first half).
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
// order, each cell in the fixed order the reorder gives it), which makes the
// result independent of scheduling.
#include <type_traits>

#include "dpd_common.cuh"
#include "dpd_launch.h"

namespace dpd {

// Launch shapes (threads per block, pair-list slots per thread, minimum resident
// blocks per SM, unroll of the pair loop) of two algorithms: the full shell (every
// pair from both sides, binary32 sums in a fixed order) and Newton's third law
// (every pair once, fixed-point sums; further below).  Within an algorithm every
// shape sums the same pairs in the same order, so its shapes give bit-identical
// forces; dpd_autotune picks the fastest on the device at hand.

// Slope -dw/dv of the cubic spline of Eq. 23 (w = 1 - 3/2 v^2 + 3/4 v^3 below 1,
// (2 - v)^3 / 4 below 2, 0 beyond).
__device__ __forceinline__ float spline_slope(float v) {
  const float u = 2.0f - v;
  return v < 1.0f ? v * fmaf(-2.25f, v, 3.0f) : (v < 2.0f ? 0.75f * u * u : 0.0f);
}

// One pair term of Eq. 2 (Eqs. 3-10) for the separation d = r_i - r_j (|d| < r_c):
// returns (m, e_x, e_y, e_z) with f_ij = m e, e = d / r, w = 1 - r (solid_pair: one
// of the two is solid, which selects the fluid-solid coefficients) and
//   m = C(r) - gamma w^2 (e . (vt_i - vt_j)) + sigma w xi_ij / sqrt(dt),
// C(r) = a_ij w for force law 0 (Eq. 4) and C(r) = -dE/dr of Eq. 22 for law 1
// (Eq. 24).  Every force kernel evaluates pairs through this function, so they agree
// bit for bit.  kKeyTable: the noise's Philox round keys come from P.rkey (free in the
// kernel-parameter bank of the single-system kernels) rather than being formed per
// round (the batch kernels, whose parameters are in global memory); same keys.
template <int kLaw, bool kKeyTable>
__device__ __forceinline__ float4 pair_term(const StepParams& P, float dx, float dy, float dz,
                                            float4 vti, const float4* __restrict__ vt, int jj,
                                            float tagj, bool solid_pair, uint32_t idi, uint32_t step) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float inv_r = rsqrtf(r2);
  const float r = r2 * inv_r;
  const float w = 1.0f - r;
  const float ex = dx * inv_r, ey = dy * inv_r, ez = dz * inv_r;
  // a solid neighbour's vt is the wall velocity at its position
  const float4 vtj = __ldg(&vt[jj]);
  if constexpr (kLaw == 0) {
    const float a = solid_pair ? P.a_fs : P.a_ff;
    const float ev = ex * (vti.x - vtj.x) + ey * (vti.y - vtj.y) + ez * (vti.z - vtj.z);
    const float xi = kKeyTable ? pair_noise(idi, id_of(tagj), step, P.sys, P.rkey)
                               : pair_noise(idi, id_of(tagj), step, P.sys, P.seed_lo, P.seed_hi);
    return make_float4(w * (a - P.gamma * w * ev + P.sigma_rsqdt * xi), ex, ey, ez);
  } else {
    const float kr = solid_pair ? P.sph_kr_fs : P.sph_kr_ff;
    const float ka = solid_pair ? P.sph_ka_fs : P.sph_ka_ff;
    const float c = kr * spline_slope(r * P.sph_ihr) - ka * spline_slope(r * P.sph_iha);
    const float ev = ex * (vti.x - vtj.x) + ey * (vti.y - vtj.y) + ez * (vti.z - vtj.z);
    const float xi = kKeyTable ? pair_noise(idi, id_of(tagj), step, P.sys, P.rkey)
                               : pair_noise(idi, id_of(tagj), step, P.sys, P.seed_lo, P.seed_hi);
    return make_float4(fmaf(w, P.sigma_rsqdt * xi - P.gamma * w * ev, c), ex, ey, ez);
  }
}

// Store the new pair force of target i and complete the closing kick
// v(t+dt) = v(t) + dt/2 (F(t) + F(t+dt)), F = f + g: the drift kernel left
// v(t) + dt/2 F(t) in vel, this adds dt/2 F(t+dt) (not for reflected particles).
__device__ __forceinline__ void finish_target(const StepParams& P, const Arrays& A, int i, float4 vti,
                                              float fx, float fy, float fz, DevCounters* ctr,
                                              int kick) {
  const bool kicked = kick && vti.w == 0.0f;
  float4 v;
  if (kicked) v = A.vel[i];  // before the store below: the arrays could alias
  A.frc[i] = make_float4(fx, fy, fz, 0.0f);
  if (kicked) {
    v.x = fmaf(P.half_dt, fx + P.g[0], v.x);
    v.y = fmaf(P.half_dt, fy + P.g[1], v.y);
    v.z = fmaf(P.half_dt, fz + P.g[2], v.z);
    A.vel[i] = v;
  }
  if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(&ctr->status, ST_NAN);
}

template <int kForceThreads, int kListCap, int kUnroll, int kLaw, bool kKeyTable>
__device__ __forceinline__ void force_body(const StepParams& P, const uint32_t* __restrict__ start,
                                           DevCounters* ctr, const Arrays& A, int i, float4 pi,
                                           int (*list)[kForceThreads],
                                           uint32_t (*seg_b)[kForceThreads],
                                           uint32_t (*seg_e)[kForceThreads], int kick) {
  const float4 vti = A.vt[i];
  const uint32_t idi = id_of(pi.w);
  const uint32_t step = ctr->step;
  const float4* __restrict__ pos = A.pos;
  const float4* __restrict__ vt = A.vt;
  // the closing kick reads this particle's velocity after the whole pair loop: start
  // bringing it into L2 now, so that the thread does not end on a DRAM round trip
  asm volatile("prefetch.global.L2 [%0];" ::"l"(A.vel + i));
  // Candidates are tested against the target shifted once per segment, u = t + s (one
  // rounding at a periodic seam), with a cut of 1 + 8 ulp(L) on r^2 that covers that
  // rounding; the pair loop then keeps exactly the pairs whose minimum-image separation
  // has 0 < r^2 < 1.  For every pair inside r_c
  // that separation equals the segment's bit for bit, so the pairs and their order are
  // those of an exact test.
  const float r2cut = fmaf(8.0f * 0x1p-23f, fmaxf(P.L[0], fmaxf(P.L[1], P.L[2])), 1.0f);

  float fx = 0.f, fy = 0.f, fz = 0.f;
  int cnt = 0;

  // Neighbour cells are visited as segments: for a particle away from the x seam
  // one segment per (dy, dz) row covers the three x-neighbour cells, which are
  // contiguous in cell order; on the seam every cell is its own segment.  Within
  // a segment the periodic image is fixed: d = t - (x_j - c), with t the target
  // coordinate shifted by -L when the cells lie across the upper seam and c = L
  // when they lie across the lower seam.  Both shifts are exact (the shifted
  // coordinate lies in [L/2, L)), and for every pair inside r_c the result equals
  // the minimum-image separation bit for bit.
  const int cx = cell_coord(pi.x, P.inv_edge[0], P.nc[0]);
  const int cy = cell_coord(pi.y, P.inv_edge[1], P.nc[1]);
  const int cz = cell_coord(pi.z, P.inv_edge[2], P.nc[2]);
  const int ncx = P.nc[0], ncy = P.nc[1], ncz = P.nc[2];
  const bool inner = cx > 0 && cx < ncx - 1;
  // Axes on which some lane of the warp has a row or cell across the periodic seam.
  // Elsewhere a listed pair's minimum-image separation is the plain difference (the
  // pair is within 1.00005 r_c < L / 2), so the pair loop skips the image test there.
  const unsigned wm = __activemask();
  const bool wrap_x = __any_sync(wm, !inner);
  const bool wrap_y = __any_sync(wm, cy == 0 || cy == ncy - 1);
  const bool wrap_z = __any_sync(wm, cz == 0 || cz == ncz - 1);
  const int nseg = inner ? 9 : 27;
  if (inner) {
    // the nine row ranges' cell starts, loaded together up front
#pragma unroll
    for (int rowi = 0; rowi < 9; ++rowi) {
      int y = cy + rowi % 3 - 1, z = cz + rowi / 3 - 1;
      y = y < 0 ? y + ncy : (y >= ncy ? y - ncy : y);
      z = z < 0 ? z + ncz : (z >= ncz ? z - ncz : z);
      const int row = (z * ncy + y) * ncx;
      seg_b[rowi][threadIdx.x] = __ldg(&start[row + cx - 1]);
      seg_e[rowi][threadIdx.x] = __ldg(&start[row + cx + 2]);
    }
  }
  int seg = 0;
  uint32_t j = 0, e = 0;
  float tx = pi.x, ty = pi.y, tz = pi.z, sx = 0.f, sy = 0.f, sz = 0.f;
  float ux = tx, uy = ty, uz = tz;
  bool more = true;
  for (;;) {
    // fill the list with candidates in rounds of up to four while it has room for four
    while (cnt <= kListCap - 4) {
      if (j == e) {
        if (seg == nseg) {
          more = false;
          break;
        }
        if (inner) {
          // the row's bounds from the table; a shift only where the row wraps in y or z
          // (the same sums the general path forms: t - L, or t + L)
          const int y = cy + seg % 3 - 1, z = cz + seg / 3 - 1;
          j = seg_b[seg][threadIdx.x];
          e = seg_e[seg][threadIdx.x];
          ux = pi.x;
          uy = y < 0 ? pi.y + P.L[1] : (y >= ncy ? pi.y - P.L[1] : pi.y);
          uz = z < 0 ? pi.z + P.L[2] : (z >= ncz ? pi.z - P.L[2] : pi.z);
        } else {
          const int part = seg % 3, rowi = seg / 3;
          const int dy = rowi % 3 - 1, dz = rowi / 3 - 1;
          int z = cz + dz, y = cy + dy;
          tz = pi.z; sz = 0.f; ty = pi.y; sy = 0.f;
          if (z < 0) { z += ncz; sz = P.L[2]; } else if (z >= ncz) { z -= ncz; tz = pi.z - P.L[2]; }
          if (y < 0) { y += ncy; sy = P.L[1]; } else if (y >= ncy) { y -= ncy; ty = pi.y - P.L[1]; }
          const int row = (z * ncy + y) * ncx;
          int x = cx + part - 1;
          tx = pi.x; sx = 0.f;
          if (x < 0) { x += ncx; sx = P.L[0]; } else if (x >= ncx) { x -= ncx; tx = pi.x - P.L[0]; }
          j = __ldg(&start[row + x]);
          e = __ldg(&start[row + x + 1]);
          ux = tx + sx;
          uy = ty + sy;
          uz = tz + sz;
        }
        ++seg;
        // the round below takes the new segment's first candidates in the same pass
      }
      // up to four candidates per round, their loads issued together
      const uint32_t m = min(e - j, 4u);
      if (m == 0u) continue;  // an empty segment: on to the next
      // four consecutive slots from one address (the arrays carry kPosPad readable slots
      // past the last particle); those past the segment's end never count
      float4 q[4];
      const float4* __restrict__ pj0 = pos + j;
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = __ldg(pj0 + u);
      // branch-free append: every slot is written, the count moves only on a hit (the
      // round starts with room for four, so the writes stay inside the list)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float dx = ux - q[u].x;
        const float dy = uy - q[u].y;
        const float dz = uz - q[u].z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        list[cnt][threadIdx.x] = (int)(j + u);
        cnt += (u < (int)m) & (r2 < r2cut) & (r2 > 0.0f);  // r2 = 0: the particle itself
      }
      j += m;
    }
    // evaluate the listed pairs
#pragma unroll kUnroll
    for (int k = 0; k < cnt; ++k) {
      const int jj = list[k][threadIdx.x];
      const float4 pj = __ldg(&pos[jj]);
      const float dx = wrap_x ? min_image(pi.x, pj.x, P.L[0], P.halfL[0]) : pi.x - pj.x;
      const float dy = wrap_y ? min_image(pi.y, pj.y, P.L[1], P.halfL[1]) : pi.y - pj.y;
      const float dz = wrap_z ? min_image(pi.z, pj.z, P.L[2], P.halfL[2]) : pi.z - pj.z;
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (!(r2 < 1.0f && r2 > 0.0f)) continue;
      const float4 t = pair_term<kLaw, kKeyTable>(P, dx, dy, dz, vti, vt, jj, pj.w, is_solid(pj.w), idi, step);
      fx = fmaf(t.x, t.y, fx);
      fy = fmaf(t.x, t.z, fy);
      fz = fmaf(t.x, t.w, fz);
    }
    if (!more) break;  // the cells ran out
    cnt = 0;
  }

  finish_target(P, A, i, vti, fx, fy, fz, ctr, kick);
}

// ---------------------------------------------------------------------------
// Newton's-third-law shapes.  Each unordered pair is evaluated once, by the
// particle that has the other in its forward half shell: the rest of its own cell
// (later in cell order), the next cell in x, and the rows (dy, dz) = (+1, 0),
// (-1, +1), (0, +1), (+1, +1) of three cells each (13 of the 26 neighbour cells; at
// least three cells per axis make every pair of cells meet once).  The pair force
// f_ij goes to i and -f_ij (what j computes, bit for bit) to j.  The partners' shares
// are summed in 64-bit fixed point, 2^32 units per force unit, one array per component
// (the three atomics of a pair then land in different L2 sectors); i's own share, the
// binary32 sum of the pairs it evaluated, goes to frc without an atomic and joins the
// sums as one more integer term.  Integer additions commute, so the result does not
// depend on the order in which the atomics land and stays bitwise reproducible.  Solid
// particles take part as the first particle of a pair (their pairs with fluid
// particles in their half shell) but receive nothing.  The next drift (or a finish
// pass, where the state is read between steps) converts the sums, completes the
// closing kick and clears them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fix_add(unsigned long long* a, float v) {
  atomicAdd(a, (unsigned long long)to_fixed(v));
}

// forward rows of the half shell, r = 0..3: (dy, dz) = (+1, 0), (-1, +1), (0, +1), (+1, +1)
__device__ __forceinline__ void half_row(int r, int* dy, int* dz) {
  *dy = r == 0 ? 1 : r - 2;
  *dz = r == 0 ? 0 : 1;
}

template <int kForceThreads, int kListCap, int kUnroll, int kLaw, bool kKeyTable>
__device__ __forceinline__ void force_body_n3(const StepParams& P, const uint32_t* __restrict__ start,
                                              const Arrays& A, unsigned long long* __restrict__ facc,
                                              size_t stride, int i, float4 pi, DevCounters* ctr,
                                              int (*list)[kForceThreads],
                                              uint32_t (*seg_b)[kForceThreads],
                                              uint32_t (*seg_e)[kForceThreads]) {
  const uint32_t step = ctr->step;
  const float4 vti = A.vt[i];
  const bool solid_i = is_solid(pi.w);
  const uint32_t idi = id_of(pi.w);
  const float4* __restrict__ pos = A.pos;
  const float4* __restrict__ vt = A.vt;
  // Candidates are tested against the target shifted once per segment, u = t + s (one
  // rounding at a periodic seam), with a cut of 1 + 8 ulp(L) on r^2 that covers that
  // rounding; the pair loop then keeps exactly the pairs whose minimum-image separation
  // has 0 < r^2 < 1.  For every pair inside r_c that separation equals the segment's
  // (shift and subtraction are both exact, or one rounding of the exact difference), so
  // the pairs and their order are those of an exact test.
  const float r2cut = fmaf(8.0f * 0x1p-23f, fmaxf(P.L[0], fmaxf(P.L[1], P.L[2])), 1.0f);
  const uint32_t smask = solid_i ? kSolidBit : 0u;  // solid-solid pairs are never listed
  const int cx = cell_coord(pi.x, P.inv_edge[0], P.nc[0]);
  const int cy = cell_coord(pi.y, P.inv_edge[1], P.nc[1]);
  const int cz = cell_coord(pi.z, P.inv_edge[2], P.nc[2]);
  const int ncx = P.nc[0], ncy = P.nc[1], ncz = P.nc[2];
  const bool inner = cx < ncx - 1 && cx > 0;
  // Axes on which some lane of the warp has a range across the periodic seam (the half
  // shell looks at z + 1 only).  Elsewhere a listed pair's minimum-image separation is
  // the plain difference (the pair is within 1.00005 r_c < L / 2), so the pair loop
  // skips the image test there.
  const unsigned wm = __activemask();
  const bool wrap_x = __any_sync(wm, !inner);
  const bool wrap_y = __any_sync(wm, cy == 0 || cy == ncy - 1);
  const bool wrap_z = __any_sync(wm, cz == ncz - 1);
  // inner: own tail + next cell (contiguous), then 4 rows of 3 cells; on the x seam:
  // own tail, next cell, then the 12 row cells one by one
  const int nseg = inner ? 5 : 14;
  const int own_row = (cz * ncy + cy) * ncx;
  if (inner) {
    // the five ranges' bounds, loaded together up front
    seg_b[0][threadIdx.x] = (uint32_t)i + 1u;
    seg_e[0][threadIdx.x] = __ldg(&start[own_row + cx + 2]);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int dy, dz;
      half_row(r, &dy, &dz);
      int z = cz + dz, y = cy + dy;
      z = z >= ncz ? z - ncz : z;
      y = y < 0 ? y + ncy : (y >= ncy ? y - ncy : y);
      const int row = (z * ncy + y) * ncx;
      seg_b[r + 1][threadIdx.x] = __ldg(&start[row + cx - 1]);
      seg_e[r + 1][threadIdx.x] = __ldg(&start[row + cx + 2]);
    }
  }
  float fx = 0.f, fy = 0.f, fz = 0.f;
  // The walk, specialised on whether any lane of the warp is a solid particle (whose
  // candidates must skip other solid particles: warps of fluid particles, nearly all,
  // test no tags) and on where the warp meets the periodic seams: nowhere (plain: each
  // range comes from the table and needs no shift, and the pair loop takes plain
  // differences), only in x (the lanes away from the x seam take their ranges from the
  // table unshifted, and only x needs the minimum image), or also in y or z (general).
  // Every form lists and evaluates the same pairs in the same order.
  auto walk = [&](auto check_tag, auto seams) {
    constexpr int kSeams = decltype(seams)::value;  // 0 none, 1 x only, 2 any
    int cnt = 0, seg = 0;
    uint32_t j = 0, e = 0;
    float ux = pi.x, uy = pi.y, uz = pi.z;
    bool more = true;
    for (;;) {
      // rounds of up to four candidates while the list has room for four
      while (cnt <= kListCap - 4) {
        if (j == e) {
          if (seg == nseg) {
            more = false;
            break;
          }
          if (kSeams == 0 || (kSeams == 1 && inner)) {
            j = seg_b[seg][threadIdx.x];
            e = seg_e[seg][threadIdx.x];
          } else {
            float tx = pi.x, ty = pi.y, tz = pi.z, sx = 0.f, sy = 0.f, sz = 0.f;
            if (inner) {
              // the range's bounds from the table; a shift only where a row wraps in y or
              // z (the same sums the general path forms: t - L, or t + L)
              j = seg_b[seg][threadIdx.x];
              e = seg_e[seg][threadIdx.x];
              if (seg > 0) {
                int dy, dz;
                half_row(seg - 1, &dy, &dz);
                const int y = cy + dy;
                ty = y < 0 ? pi.y : (y >= ncy ? pi.y - P.L[1] : pi.y);
                sy = y < 0 ? P.L[1] : 0.f;
                tz = cz + dz >= ncz ? pi.z - P.L[2] : pi.z;
              }
            } else if (seg == 0) {
              j = (uint32_t)i + 1u;
              e = __ldg(&start[own_row + cx + 1]);
            } else if (seg == 1) {
              int x = cx + 1;
              if (x >= ncx) { x -= ncx; tx = pi.x - P.L[0]; }
              j = __ldg(&start[own_row + x]);
              e = __ldg(&start[own_row + x + 1]);
            } else {
              int dy, dz;
              half_row((seg - 2) / 3, &dy, &dz);
              int z = cz + dz, y = cy + dy;
              if (z >= ncz) { z -= ncz; tz = pi.z - P.L[2]; }
              if (y < 0) { y += ncy; sy = P.L[1]; } else if (y >= ncy) { y -= ncy; ty = pi.y - P.L[1]; }
              const int row = (z * ncy + y) * ncx;
              int x = cx + (seg - 2) % 3 - 1;
              if (x < 0) { x += ncx; sx = P.L[0]; } else if (x >= ncx) { x -= ncx; tx = pi.x - P.L[0]; }
              j = __ldg(&start[row + x]);
              e = __ldg(&start[row + x + 1]);
            }
            ux = tx + sx;
            uy = ty + sy;
            uz = tz + sz;
          }
          ++seg;
          // the round below takes the new segment's first candidates in the same pass
          // (none if it is empty): lanes that change segments then cost the warp the
          // switch, not a whole extra pass of rounds for the others
        }
        const uint32_t m = min(e - j, 4u);
        if (m == 0u) continue;  // an empty segment: on to the next
        // four consecutive slots from one address (the arrays carry kPosPad readable slots
        // past the last particle); those past the segment's end never count
        float4 q[4];
        const float4* __restrict__ pj0 = pos + j;
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldg(pj0 + u);
        // branch-free append: every slot is written, the count moves only on a hit (the
        // round starts with room for four, so the writes stay inside the list)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float dx = ux - q[u].x;
          const float dy = uy - q[u].y;
          const float dz = uz - q[u].z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          list[cnt][threadIdx.x] = (int)(j + u);
          if constexpr (decltype(check_tag)::value)
            cnt += (u < (int)m) & (r2 < r2cut) & ((tag_of(q[u].w) & smask) == 0u);
          else
            cnt += (u < (int)m) & (r2 < r2cut);
        }
        j += m;
      }
#pragma unroll kUnroll
      for (int k = 0; k < cnt; ++k) {
        const int jj = list[k][threadIdx.x];
        const float4 pj = __ldg(&pos[jj]);
        float dx, dy, dz;
        if constexpr (kSeams == 0) {
          dx = pi.x - pj.x;
          dy = pi.y - pj.y;
          dz = pi.z - pj.z;
        } else if constexpr (kSeams == 1) {
          dx = min_image(pi.x, pj.x, P.L[0], P.halfL[0]);
          dy = pi.y - pj.y;
          dz = pi.z - pj.z;
        } else {
          dx = wrap_x ? min_image(pi.x, pj.x, P.L[0], P.halfL[0]) : pi.x - pj.x;
          dy = wrap_y ? min_image(pi.y, pj.y, P.L[1], P.halfL[1]) : pi.y - pj.y;
          dz = wrap_z ? min_image(pi.z, pj.z, P.L[2], P.halfL[2]) : pi.z - pj.z;
        }
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(r2 < 1.0f && r2 > 0.0f)) continue;
        const bool solid_j = is_solid(pj.w);
        const float4 t = pair_term<kLaw, kKeyTable>(P, dx, dy, dz, vti, vt, jj, pj.w, solid_i || solid_j, idi, step);
        const float gx = t.x * t.y, gy = t.x * t.z, gz = t.x * t.w;
        fx += gx;
        fy += gy;
        fz += gz;
        if (!solid_j) {
          fix_add(&facc[jj], -gx);
          fix_add(&facc[stride + jj], -gy);
          fix_add(&facc[2 * stride + jj], -gz);
        }
      }
      if (!more) break;  // the cells ran out
      cnt = 0;
    }
  };
  using NoSeam = std::integral_constant<int, 0>;
  using XSeam = std::integral_constant<int, 1>;
  using AnySeam = std::integral_constant<int, 2>;
  const bool any_solid = __any_sync(wm, solid_i);
  if (wrap_y || wrap_z) {
    if (any_solid)
      walk(std::true_type{}, AnySeam{});
    else
      walk(std::false_type{}, AnySeam{});
  } else if (wrap_x) {
    if (any_solid)
      walk(std::true_type{}, XSeam{});
    else
      walk(std::false_type{}, XSeam{});
  } else {
    if (any_solid)
      walk(std::true_type{}, NoSeam{});
    else
      walk(std::false_type{}, NoSeam{});
  }
  // the own share goes to frc without an atomic (nothing else writes it): whoever reads
  // the sums adds it as one more integer term
  A.frc[i] = solid_i ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(fx, fy, fz, 0.f);
  // fixed point cannot carry a NaN or a force beyond its range: flag them here (every
  // pair this thread evaluated is in its own float sum)
  const float fmax = fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz)));
  if (!(fmax < 1.0e9f)) atomicOr(&ctr->status, ST_NAN);
}

template <int kForceThreads, int kListCap, int kMinBlocks, int kUnroll, bool kBatch, int kLaw>
__global__ void __launch_bounds__(kForceThreads, kMinBlocks)
k_force_n3(StepParams P0, const SysDesc* __restrict__ S, int nsys, Arrays A,
           const uint32_t* __restrict__ start_all, unsigned long long* __restrict__ facc, int n,
           DevCounters* ctrs) {
  __shared__ int list[kListCap][kForceThreads];
  __shared__ uint32_t seg_b[5][kForceThreads], seg_e[5][kForceThreads];
  const int i = blockIdx.x * kForceThreads + threadIdx.x;
  int sk = 0;
  if constexpr (kBatch) sk = sys_of_block(S, nsys, (uint32_t)i, blockIdx.x * kForceThreads);
  if (i >= n) return;
  const float4 pi = A.pos[i];
  if constexpr (kBatch) {
    force_body_n3<kForceThreads, kListCap, kUnroll, kLaw, false>(S[sk].P, start_all + S[sk].cell_off, A,
                                                          facc, (size_t)n, i, pi, ctrs + sk, list,
                                                          seg_b, seg_e);
  } else {
    force_body_n3<kForceThreads, kListCap, kUnroll, kLaw, true>(P0, start_all, A, facc, (size_t)n, i, pi,
                                                          ctrs, list, seg_b, seg_e);
  }
}

// Finish pass: the fixed-point sums become the force, the closing kick is completed
// and the sums cleared.  A time step leaves this to the next drift; the pass runs
// when the state is read (or handed on) between steps, and after the initial force.
template <bool kBatch>
__global__ void __launch_bounds__(256) k_force_finish(StepParams P0, const SysDesc* __restrict__ S,
                                                      int nsys, Arrays A,
                                                      unsigned long long* __restrict__ facc, int n,
                                                      DevCounters* ctrs, int kick) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (is_solid(A.pos[i].w)) {  // nothing accumulates for solid particles
    A.frc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const size_t ns = (size_t)n;
  const float3 f = fixed_sum_force(facc[i], facc[ns + i], facc[2 * ns + i], A.frc[i]);
  const float fx = f.x, fy = f.y, fz = f.z;
  facc[i] = 0ull;
  facc[(size_t)n + i] = 0ull;
  facc[2 * (size_t)n + i] = 0ull;
  const float4 vti = A.vt[i];
  if constexpr (kBatch) {
    const int sk = sys_of(S, nsys, (uint32_t)i);
    finish_target(S[sk].P, A, i, vti, fx, fy, fz, ctrs + sk, kick);
  } else {
    finish_target(P0, A, i, vti, fx, fy, fz, ctrs, kick);
  }
}

// A single system takes its parameters by value (they stay in the kernel-parameter
// bank); a batch reads each particle's system from the table.  Both run the same
// body, so a system computes the same bits alone and in a batch.
template <int kForceThreads, int kListCap, int kMinBlocks, int kUnroll, bool kBatch, int kLaw>
__global__ void __launch_bounds__(kForceThreads, kMinBlocks)
k_force(StepParams P0, const SysDesc* __restrict__ S, int nsys, Arrays A,
        const uint32_t* __restrict__ start_all, int n, DevCounters* ctrs, int kick) {
  __shared__ int list[kListCap][kForceThreads];
  __shared__ uint32_t seg_b[9][kForceThreads], seg_e[9][kForceThreads];
  const int i = blockIdx.x * kForceThreads + threadIdx.x;
  int sk = 0;
  if constexpr (kBatch) sk = sys_of_block(S, nsys, (uint32_t)i, blockIdx.x * kForceThreads);
  if (i >= n) return;
  const float4 pi = A.pos[i];
  if (is_solid(pi.w)) {  // solid particles feel no force (the reorder does not carry it)
    A.frc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  if constexpr (kBatch) {
    force_body<kForceThreads, kListCap, kUnroll, kLaw, false>(S[sk].P, start_all + S[sk].cell_off, ctrs + sk,
                                                       A, i, pi, list, seg_b, seg_e, kick);
  } else {
    force_body<kForceThreads, kListCap, kUnroll, kLaw, true>(P0, start_all, ctrs, A, i, pi, list, seg_b,
                                                       seg_e, kick);
  }
}

using ForceKernel = void (*)(StepParams, const SysDesc*, int, Arrays, const uint32_t*, int,
                             DevCounters*, int);

using ForceKernelN3 = void (*)(StepParams, const SysDesc*, int, Arrays, const uint32_t*,
                               unsigned long long*, int, DevCounters*);

struct ForceVariant {
  ForceKernel single[2], batch[2];  // by force law (full-shell shapes)
  ForceKernelN3 single3[2], batch3[2];  // Newton's-third-law shapes
  int threads;
  bool n3;
};

#define DPD_FORCE_VARIANT(T, C, M, U)                                            \
  {                                                                              \
    {k_force<T, C, M, U, false, 0>, k_force<T, C, M, U, false, 1>},              \
        {k_force<T, C, M, U, true, 0>, k_force<T, C, M, U, true, 1>},            \
        {nullptr, nullptr}, {nullptr, nullptr}, T, false                         \
  }
#define DPD_FORCE_VARIANT_N3(T, C, M, U)                                          \
  {                                                                              \
    {nullptr, nullptr}, {nullptr, nullptr},                                      \
        {k_force_n3<T, C, M, U, false, 0>, k_force_n3<T, C, M, U, false, 1>},    \
        {k_force_n3<T, C, M, U, true, 0>, k_force_n3<T, C, M, U, true, 1>}, T,   \
        true                                                                     \
  }

static const ForceVariant kForceVariants[] = {
    DPD_FORCE_VARIANT(128, 24, 1, 1), DPD_FORCE_VARIANT(128, 16, 1, 1),
    DPD_FORCE_VARIANT(256, 16, 1, 1), DPD_FORCE_VARIANT(64, 24, 1, 1),
    DPD_FORCE_VARIANT(128, 16, 12, 1), DPD_FORCE_VARIANT(256, 12, 6, 1),
    DPD_FORCE_VARIANT(128, 32, 1, 1), DPD_FORCE_VARIANT(128, 24, 1, 2),
    DPD_FORCE_VARIANT(128, 16, 12, 2),
    DPD_FORCE_VARIANT_N3(128, 12, 1, 1), DPD_FORCE_VARIANT_N3(128, 8, 1, 1),
    DPD_FORCE_VARIANT_N3(64, 12, 1, 1), DPD_FORCE_VARIANT_N3(256, 8, 1, 1),
    DPD_FORCE_VARIANT_N3(128, 16, 1, 1),
    // capped at 64 registers or fewer: eight 128-thread (sixteen 64-thread) blocks per SM
    DPD_FORCE_VARIANT_N3(128, 16, 8, 1), DPD_FORCE_VARIANT_N3(128, 12, 8, 1),
    DPD_FORCE_VARIANT_N3(64, 16, 14, 1), DPD_FORCE_VARIANT_N3(128, 24, 8, 1),
    DPD_FORCE_VARIANT_N3(64, 16, 16, 1), DPD_FORCE_VARIANT_N3(64, 24, 16, 1),
    DPD_FORCE_VARIANT_N3(64, 12, 16, 1),
};

int force_variants() { return (int)(sizeof(kForceVariants) / sizeof(kForceVariants[0])); }

const char* force_variant_name(int v) {
  static const char* names[] = {"128x24", "128x16", "256x16", "64x24", "128x16/min12",
                                "256x12/min6", "128x32", "128x24/unroll2", "128x16/min12/unroll2",
                                "n3 128x12", "n3 128x8", "n3 64x12", "n3 256x8", "n3 128x16",
                                "n3 128x16/min8", "n3 128x12/min8", "n3 64x16/min14",
                                "n3 128x24/min8", "n3 64x16/min16", "n3 64x24/min16",
                                "n3 64x12/min16"};
  return (v >= 0 && v < force_variants()) ? names[v] : "?";
}

void launch_force_pairs(const StepParams& P0, const SysDesc* S, int nsys, const Arrays& A,
                        const uint32_t* start, unsigned long long* facc, int n, DevCounters* ctr,
                        int kick, int variant, cudaStream_t s) {
  if (n <= 0) return;
  if (variant < 0 || variant >= force_variants()) variant = 0;
  const ForceVariant& fv = kForceVariants[variant];
  const int nb = (n + fv.threads - 1) / fv.threads;
  const int law = P0.law == 1 ? 1 : 0;  // a batch holds systems of one law
  if (!fv.n3) {
    (nsys == 1 ? fv.single[law] : fv.batch[law])<<<nb, fv.threads, 0, s>>>(P0, S, nsys, A, start, n,
                                                                            ctr, kick);
    return;
  }
  (nsys == 1 ? fv.single3[law] : fv.batch3[law])<<<nb, fv.threads, 0, s>>>(P0, S, nsys, A, start, facc,
                                                                            n, ctr);
}

bool force_variant_newton3(int variant) {
  if (variant < 0 || variant >= force_variants()) variant = 0;
  return kForceVariants[variant].n3;
}

void launch_force_finish(const StepParams& P0, const SysDesc* S, int nsys, const Arrays& A,
                         unsigned long long* facc, int n, DevCounters* ctr, int kick,
                         cudaStream_t s) {
  if (n <= 0) return;
  const int nb2 = (n + 255) / 256;
  if (nsys == 1)
    k_force_finish<false><<<nb2, 256, 0, s>>>(P0, S, nsys, A, facc, n, ctr, kick);
  else
    k_force_finish<true><<<nb2, 256, 0, s>>>(P0, S, nsys, A, facc, n, ctr, kick);
}

void launch_force(const StepParams& P0, const SysDesc* S, int nsys, const Arrays& A,
                  const uint32_t* start, unsigned long long* facc, int n, DevCounters* ctr, int kick,
                  int variant, cudaStream_t s) {
  launch_force_pairs(P0, S, nsys, A, start, facc, n, ctr, kick, variant, s);
  if (force_variant_newton3(variant)) launch_force_finish(P0, S, nsys, A, facc, n, ctr, kick, s);
}

}  // namespace dpd
