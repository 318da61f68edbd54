// dpd_common.cuh -- device-side types and helpers shared by the kernels of the
// GB300 DPD library (phase-field no-slip walls, Xu & Meakin, arXiv:1807.09896).
//
// Particle data live as structure-of-arrays of float4 in cell order:
//   pos  {x, y, z, tag}   tag = bit pattern of (id | solid << 31)
//   vt   {vtx, vty, vtz, reflected flag}   predicted velocity of the step
//   vel  {vx, vy, vz, reflected flag}  velocity v(t)
//   frc  {fx, fy, fz, 0}  pair force f(t) (body force not included)
// Between the steps of a Newton's-third-law force shape the force is not in frc but
// in 64-bit fixed-point sums, and vel still lacks the second half of the closing
// kick; the host knows which state it left and launches the drift kernel that
// completes it (see the drift kernel).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpd {

constexpr uint32_t kSolidBit = 0x80000000u;
constexpr uint32_t kIdMask = 0x7fffffffu;

// Device status bits (read by dpd_step once per call).
enum : uint32_t {
  ST_BAND = 1u,      // a drift exceeded the band margin
  ST_NAN = 2u,       // non-finite value
  ST_LOST = 4u,      // fluid particle at phi < 0
  ST_OVERFLOW = 8u,  // a cell exceeded the per-cell sort capacity
  ST_BADID = 16u,    // ids are not a permutation of 0..n-1
};

struct DevCounters {
  uint32_t status;
  uint32_t step;                 // noise counter of the most recent force evaluation
  unsigned long long reflections;
  unsigned long long fallbacks;
};

// Fixed-point pair sums of the Newton's-third-law force shapes: 2^32 units per
// force unit, one array of n per component, holding the shares -f_ij handed to
// each particle by its partners.  The particle's own share (the binary32 sum of the
// pairs it evaluated) is stored in frc and added as one more integer term when the
// sums are read.
constexpr float kFixScale = 4294967296.0f;        // 2^32
constexpr float kFixInvF = 1.0f / 4294967296.0f;  // 2^-32

__device__ __forceinline__ long long to_fixed(float v) { return __float2ll_rn(v * kFixScale); }

// The force of particle i: its partners' fixed-point sums plus its own share, one
// rounding from the exact integer (the power-of-two scale is exact).  Integer sums
// do not depend on the order of their terms, so neither does the result.
__device__ __forceinline__ float3 fixed_sum_force(unsigned long long sx, unsigned long long sy,
                                                  unsigned long long sz, float4 own) {
  const long long x = (long long)sx + to_fixed(own.x);
  const long long y = (long long)sy + to_fixed(own.y);
  const long long z = (long long)sz + to_fixed(own.z);
  return make_float3(__ll2float_rn(x) * kFixInvF, __ll2float_rn(y) * kFixInvF,
                     __ll2float_rn(z) * kFixInvF);
}


// Everything a step kernel needs, passed by value.
struct StepParams {
  float L[3], invL[3], halfL[3];
  int nc[3];
  float inv_edge[3];
  int ncells;
  float dt, half_dt, half_dt2, lam_dt;
  float g[3], vw[3];
  float sh[3];   // wall velocity field v_w(r) = vw + d sh, d = r[sh_axis] - sh_ref wrapped
  int sh_axis;   //   into [-L/2, L/2); sh has no component along sh_axis
  float sh_ref;
  int moving;    // vw or sh nonzero: the solid moves
  float a_ff, a_fs, gamma, sigma_rsqdt;
  uint32_t seed_lo, seed_hi, sys;
  // Philox4x32-10 round keys of the pair noise, (seed_lo + r 0x9E3779B9, seed_hi +
  // r 0xBB67AE85) for round r = 0..9: the key schedule depends on the seed alone, so it
  // is formed once on the host (single-system kernels read it from the parameter bank)
  uint32_t rkey[20];
  int reflect_variant;
  float margin;
  const float* phi;   // phase-field nodes, x fastest (nullptr: phi = +1)
  int pd[3];
  float inv_h;
  const uint8_t* band;  // per cell: 1 if a particle starting there may reach phi < 0
  // force law 1 (Eqs. 22-24): C(r) = K_r g(r / h_r) - K_a g(r / h_a), g = -dw/dv of
  // the cubic spline, K = S alpha_D / h^(D+1); ff and fs strengths
  int law;
  float sph_kr_ff, sph_ka_ff, sph_kr_fs, sph_ka_fs, sph_ihr, sph_iha;
};

// Wall velocity at a point whose coordinate along the shear axis is xa: the field
// v_w(r) = v_wall + d S of plane Couette walls, d = xa - ref wrapped into
// [-L/2, L/2) (the walls' own planes, Sec. II.C moving walls).
__device__ __forceinline__ float3 wall_velocity(const StepParams& P, float xa) {
  const float L = P.L[P.sh_axis];
  float d = xa - P.sh_ref;
  if (d >= 0.5f * L) d -= L;
  else if (d < -0.5f * L) d += L;
  return make_float3(fmaf(d, P.sh[0], P.vw[0]), fmaf(d, P.sh[1], P.vw[1]), fmaf(d, P.sh[2], P.vw[2]));
}

__device__ __forceinline__ float axis_coord(const float4& p, int a) {
  return a == 0 ? p.x : (a == 1 ? p.y : p.z);
}

// One system of a batch: its parameters and where its cells and particles sit
// in the concatenated arrays (a single system is a batch of one).  Systems
// occupy contiguous, increasing ranges of cells, hence of particles in cell
// order, and keep their particle counts, so the ranges never move.
struct SysDesc {
  StepParams P;
  uint32_t cell_off;
  uint32_t part_off;
  uint32_t n;
  uint32_t pad;
};

// System of particle i: the last system whose particle range starts at or below i.
__device__ __forceinline__ int sys_of(const SysDesc* __restrict__ S, int nsys, uint32_t i) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (S[mid].part_off <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The same for every thread of a block whose particles start at block_first: thread 0
// searches once, the others step on from there (systems hold contiguous increasing
// ranges, so a block usually meets one or two).  Every thread of the block must call
// it: it synchronises the block, which pays in the long force kernels (-6% on a
// 64-system batch) and not in the short drift.
__device__ __forceinline__ int sys_of_block(const SysDesc* __restrict__ S, int nsys, uint32_t i,
                                            uint32_t block_first) {
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = sys_of(S, nsys, block_first);
  __syncthreads();
  int sk = s_sys;
  while (sk + 1 < nsys && S[sk + 1].part_off <= i) ++sk;
  return sk;
}

// Readable slots past the last particle in the position arrays: a candidate round of
// the force kernels loads four consecutive positions from one address, and the slots
// past a range's end (at most three) never count.
constexpr int kPosPad = 4;

struct Arrays {
  float4* pos;  // n + kPosPad slots in the step's buffers
  float4* vt;
  float4* vel;  // .w: 1 if the particle was reflected in the step that produced it
  float4* frc;
};

struct CellList {
  uint32_t* key;    // cell of each particle (current order)
  uint32_t* count;  // particles per cell; after the scan the cell's next free slot (the
                    // scatter's cursor); zeroed by the per-cell sort
  uint32_t* start;  // exclusive prefix of count, ncells + 1 entries
  uint32_t* perm;   // new position -> old position
  // the scan's tiles of kScanTileCells cells: the particles each tile's cells hold,
  // added by the kernels that fill count, read by the scan, cleared by the scatter
  uint32_t* tile_total;
};

// Cells per tile of the cell scan (one block of the scan per tile).  Each tile's total
// is kept in kTileShards counters (by warp), each on its own 128-byte line, so that the
// producers' atomics spread over the L2 instead of queueing on a few lines.
constexpr int kScanTileCells = 2048;
constexpr int kTileShards = 4;
constexpr int kTileStride = 32;  // uint32 words between counters (128 bytes)
__host__ __device__ constexpr size_t tile_total_words(int ntiles) {
  return (size_t)ntiles * kTileShards * kTileStride;
}
__device__ __forceinline__ uint32_t* tile_counter(uint32_t* tt, uint32_t tile, int warp) {
  return tt + ((size_t)tile * kTileShards + (uint32_t)(warp & (kTileShards - 1))) * kTileStride;
}

__device__ __forceinline__ uint32_t tag_of(float w) { return __float_as_uint(w); }
__device__ __forceinline__ bool is_solid(float w) { return (tag_of(w) & kSolidBit) != 0u; }
__device__ __forceinline__ uint32_t id_of(float w) { return tag_of(w) & kIdMask; }

__device__ __forceinline__ int cell_coord(float x, float inv_edge, int nc) {
  int c = __float2int_rd(x * inv_edge);
  return min(max(c, 0), nc - 1);
}

__device__ __forceinline__ int cell_of(const StepParams& P, float x, float y, float z) {
  int cx = cell_coord(x, P.inv_edge[0], P.nc[0]);
  int cy = cell_coord(y, P.inv_edge[1], P.nc[1]);
  int cz = cell_coord(z, P.inv_edge[2], P.nc[2]);
  return (cz * P.nc[1] + cy) * P.nc[0] + cx;
}

__device__ __forceinline__ int wrap_node(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Particle phase field: trilinear interpolation of the periodic node grid at an
// arbitrary (possibly unwrapped) point (Sec. II.C, 3-D form of the paper's
// linear interpolation).  The point may be given as an unevaluated sum x + lx
// (a binary32 value and its rounding error); the fractional offsets inside the
// grid cell are then formed from the exact sum, so a point a few ulp(L) from a
// node plane keeps its full relative accuracy.
__device__ __forceinline__ float phi_at(const StepParams& P, float x, float y, float z,
                                        float lx = 0.0f, float ly = 0.0f, float lz = 0.0f) {
  if (P.phi == nullptr) return 1.0f;
  const float fx = floorf(x * P.inv_h), fy = floorf(y * P.inv_h), fz = floorf(z * P.inv_h);
  const float tx = fmaf(x, P.inv_h, -fx) + lx * P.inv_h;
  const float ty = fmaf(y, P.inv_h, -fy) + ly * P.inv_h;
  const float tz = fmaf(z, P.inv_h, -fz) + lz * P.inv_h;
  const int ix0 = wrap_node(__float2int_rd(fx), P.pd[0]), ix1 = wrap_node(__float2int_rd(fx) + 1, P.pd[0]);
  const int iy0 = wrap_node(__float2int_rd(fy), P.pd[1]), iy1 = wrap_node(__float2int_rd(fy) + 1, P.pd[1]);
  const int iz0 = wrap_node(__float2int_rd(fz), P.pd[2]), iz1 = wrap_node(__float2int_rd(fz) + 1, P.pd[2]);
  const int sy_ = P.pd[0];
  const long sz_ = (long)P.pd[0] * P.pd[1];
  const float* g = P.phi;
  const float c000 = __ldg(g + iz0 * sz_ + iy0 * sy_ + ix0), c100 = __ldg(g + iz0 * sz_ + iy0 * sy_ + ix1);
  const float c010 = __ldg(g + iz0 * sz_ + iy1 * sy_ + ix0), c110 = __ldg(g + iz0 * sz_ + iy1 * sy_ + ix1);
  const float c001 = __ldg(g + iz1 * sz_ + iy0 * sy_ + ix0), c101 = __ldg(g + iz1 * sz_ + iy0 * sy_ + ix1);
  const float c011 = __ldg(g + iz1 * sz_ + iy1 * sy_ + ix0), c111 = __ldg(g + iz1 * sz_ + iy1 * sy_ + ix1);
  const float ux = 1.0f - tx, uy = 1.0f - ty, uz = 1.0f - tz;
  const float c00 = c000 * ux + c100 * tx, c10 = c010 * ux + c110 * tx;
  const float c01 = c001 * ux + c101 * tx, c11 = c011 * ux + c111 * tx;
  const float c0 = c00 * uy + c10 * ty, c1 = c01 * uy + c11 * ty;
  return c0 * uz + c1 * tz;
}

// s + err = a + b exactly (Knuth's TwoSum; no multiplications, so no contraction).
__device__ __forceinline__ float two_sum(float a, float b, float* err) {
  const float s = a + b;
  const float bb = s - a;
  *err = (a - (s - bb)) + (b - bb);
  return s;
}

// Pair noise xi_ij of Eq. 7.  Philox4x32-10 (Salmon et al., SC'11) of the
// counter (min id, max id, step, system) under the key (seed_lo, seed_hi); the
// first two output words become two uniforms u = ((w >> 9) + 1/2) 2^-23, exact in
// binary32, and the Box-Muller transform gives xi = sqrt(-2 ln u0) cos(2 pi u1).
// Philox4x32-10 (Salmon et al., SC'11): ten rounds on the counter (c0..c3) under the
// key (k0, k1); the result replaces the counter.
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Uniform in (0, 1) from one output word: ((w >> 9) + 1/2) 2^-23, exact in binary32.
__device__ __forceinline__ float philox_u01(uint32_t w) {
  return (__uint2float_rn(w >> 9) + 0.5f) * 0x1p-23f;
}

__device__ __forceinline__ float pair_noise(uint32_t ida, uint32_t idb, uint32_t step, uint32_t sys,
                                            const uint32_t (&rkey)[20]) {
  uint32_t c0 = min(ida, idb), c1 = max(ida, idb), c2 = step, c3 = sys;
  // Philox4x32-10 rounds with the precomputed keys (the same rounds as philox4x32_10)
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ rkey[2 * round];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rkey[2 * round + 1];
    c3 = lo0;
  }
  const float u0 = (__uint2float_rn(c0 >> 9) + 0.5f) * 0x1p-23f;
  const float u1 = (__uint2float_rn(c1 >> 9) + 0.5f) * 0x1p-23f;
  // cos(2 pi u1) = -cos(2 pi u1 - pi), evaluated by the hardware cosine on an
  // argument in (-pi, pi), where its absolute error is below 4e-7; the square root
  // as x * rsqrt(x) (x = -2 ln u0 >= 2.4e-7 > 0).  The logarithm stays the
  // accurate one: near u0 = 1 its value is tiny and needs full relative accuracy.
  const float x = -2.0f * logf(u0);
  const float c = __cosf(fmaf(6.28318530717958648f, u1, -3.14159265358979324f));
  return -(x * rsqrtf(x)) * c;
}

// The same with the round keys formed on the fly (kernels that read their parameters
// from global memory, where loading the table costs more than two adds per round).
__device__ __forceinline__ float pair_noise(uint32_t ida, uint32_t idb, uint32_t step, uint32_t sys,
                                            uint32_t k0, uint32_t k1) {
  uint32_t c0 = min(ida, idb), c1 = max(ida, idb), c2 = step, c3 = sys;
  philox4x32_10(c0, c1, c2, c3, k0, k1);
  const float u0 = (__uint2float_rn(c0 >> 9) + 0.5f) * 0x1p-23f;
  const float u1 = (__uint2float_rn(c1 >> 9) + 0.5f) * 0x1p-23f;
  // cos(2 pi u1) = -cos(2 pi u1 - pi), evaluated by the hardware cosine on an
  // argument in (-pi, pi), where its absolute error is below 4e-7; the square root
  // as x * rsqrt(x) (x = -2 ln u0 >= 2.4e-7 > 0).  The logarithm stays the
  // accurate one: near u0 = 1 its value is tiny and needs full relative accuracy.
  const float x = -2.0f * logf(u0);
  const float c = __cosf(fmaf(6.28318530717958648f, u1, -3.14159265358979324f));
  return -(x * rsqrtf(x)) * c;
}

// Minimum-image separation xi - xj of two coordinates in [0, L).  When the pair
// straddles the periodic seam the operand near L is shifted by -L first; that
// shift is exact (Sterbenz: the operand lies in [L/2, L)), so the separation is
// rounded once, at its own magnitude (below r_c), instead of at the magnitude of
// L.  Swapping i and j negates the result exactly.
__device__ __forceinline__ float min_image(float xi, float xj, float L, float halfL) {
  const float d = xi - xj;
  if (d > halfL) return (xi - L) - xj;
  if (d < -halfL) return xi - (xj - L);
  return d;
}

}  // namespace dpd
