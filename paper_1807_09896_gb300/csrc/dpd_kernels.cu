// dpd_kernels.cu -- the streaming kernels of one DPD time step: drift and
// bounce-back reflection, cell-list counting sort, profile and diagnostic
// reductions, and set-up helpers (Xu & Meakin, arXiv:1807.09896).
//
// All of these are bound by HBM bandwidth: each touches every particle once
// with coalesced float4 loads and stores in cell order.
#include "dpd_common.cuh"
#include "dpd_launch.h"

namespace dpd {

// ---------------------------------------------------------------------------
// Step kernel 1: drift, predicted velocity, reflection, cell key.
//
// Groot-Warren modified velocity-Verlet (Sec. II.A, ref. 35), F = f + g:
//   dr = dt v + dt^2/2 F,  r' = r + dr,  vt = v + lambda dt F,
// and vel <- v + dt/2 F, the first half of the closing kick (the force kernel adds
// dt/2 F(t+dt)), so the old force is not needed after this kernel.
// Bounce-back (Sec. II.C, Eq. 17, Fig. 4): if phi(r') < 0 the particle is put
// at r' - 2 s dr with s = atanh(-phi(r')) / (atanh(-phi(r')) + atanh(phi(r))),
// its velocity becomes 2 v_wall - v(t) (also used as vt), and it is flagged so
// that the closing kick is skipped.  If the reflected point still has
// phi < 0 the particle stays at r(t).  The test runs only for particles whose
// starting cell is flagged in the band mask (Sec. II.C: bulk particles far from
// phi = 0 need no test); the band is conservative for drifts up to `margin`,
// which is checked.  Frozen (solid) particles translate with the wall velocity.
// Then the position is wrapped into the box, its cell found, and the particle
// counted into that cell with one atomic that also gives its arrival slot.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float clamp_phi(float p) {
  return fminf(fmaxf(p, -0.999999f), 0.999999f);
}

__device__ __forceinline__ float wrap_coord(float x, float L) {
  if (x < 0.0f) {
    x += L;
    if (x >= L) x = 0.0f;
  } else if (x >= L) {
    x -= L;
    if (x >= L) x = 0.0f;
  }
  return x;
}

template <bool kPending>
__device__ __forceinline__ void integrate_body(const StepParams& P, uint32_t cell_off,
                                               DevCounters* ctr, const Arrays& A,
                                               const CellList& C,
                                               unsigned long long* __restrict__ facc, int n, int i) {
  // every load of the particle up front, before any branch on them: the kernel is
  // bound by memory latency, and a load behind a branch on another load would wait
  // for two round trips (solid particles read a little they do not need)
  float4 p = A.pos[i];
  float4 v = A.vel[i];
  const float4 f4 = A.frc[i];
  unsigned long long sx = 0ull, sy = 0ull, sz = 0ull;
  if constexpr (kPending) {
    sx = facc[i];
    sy = facc[(size_t)n + i];
    sz = facc[2 * (size_t)n + i];
  }
  if (!is_solid(p.w)) {
    float3 f;
    if constexpr (kPending) {
      // The last force kernel left the force in the fixed-point sums (f4 holds the
      // particle's own share) and v without the second half of its closing kick:
      // convert the sums (and clear them for the next force), then complete the kick
      // unless the particle was reflected (vel.w = 1).  Same arithmetic as the finish
      // pass, so the bits do not depend on which ran.
      f = fixed_sum_force(sx, sy, sz, f4);
      facc[i] = 0ull;
      facc[(size_t)n + i] = 0ull;
      facc[2 * (size_t)n + i] = 0ull;
      if (v.w == 0.0f) {
        v.x = fmaf(P.half_dt, f.x + P.g[0], v.x);
        v.y = fmaf(P.half_dt, f.y + P.g[1], v.y);
        v.z = fmaf(P.half_dt, f.z + P.g[2], v.z);
      }
    } else {
      f = make_float3(f4.x, f4.y, f4.z);
    }
    const float Fx = f.x + P.g[0], Fy = f.y + P.g[1], Fz = f.z + P.g[2];
    const float dx = fmaf(P.half_dt2, Fx, P.dt * v.x);
    const float dy = fmaf(P.half_dt2, Fy, P.dt * v.y);
    const float dz = fmaf(P.half_dt2, Fz, P.dt * v.z);
    // r' = r + dr, kept as the unevaluated sum x + lx for the phase-field lookup
    float lx, ly, lz;
    float x = two_sum(p.x, dx, &lx), y = two_sum(p.y, dy, &ly), z = two_sum(p.z, dz, &lz);
    float4 vt = make_float4(fmaf(P.lam_dt, Fx, v.x), fmaf(P.lam_dt, Fy, v.y),
                            fmaf(P.lam_dt, Fz, v.z), 0.0f);
    // first half of the closing kick, v + dt/2 F(t): the force kernel adds dt/2 F(t+dt),
    // so F(t) is not needed after this kernel (the reorder does not carry it)
    float4 vh = make_float4(fmaf(P.half_dt, Fx, v.x), fmaf(P.half_dt, Fy, v.y),
                            fmaf(P.half_dt, Fz, v.z), 0.0f);
    if (fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))) > P.margin) atomicOr(&ctr->status, ST_BAND);
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) atomicOr(&ctr->status, ST_NAN);
    if (P.band != nullptr && P.band[cell_of(P, p.x, p.y, p.z)]) {
      const float phi_new = phi_at(P, x, y, z, lx, ly, lz);
      if (phi_new < 0.0f) {
        const float phi_old = fmaxf(phi_at(P, p.x, p.y, p.z), 0.0f);
        const float Ad = atanhf(-clamp_phi(phi_new));
        const float Bd = atanhf(clamp_phi(phi_old));
        const float s = Ad / (Ad + Bd);
        const float s2 = 2.0f * s;
        // wall velocity at the crossing point r + (1 - s) dr
        const int ax = P.sh_axis;
        const float dra = ax == 0 ? dx : (ax == 1 ? dy : dz);
        const float3 vw = wall_velocity(P, fmaf(1.0f - s, dra, axis_coord(p, ax)));
        float ex = dx, ey = dy, ez = dz;
        if (P.reflect_variant == 1) {
          ex = (v.x - vw.x) * P.dt;
          ey = (v.y - vw.y) * P.dt;
          ez = (v.z - vw.z) * P.dt;
        }
        // r_bb = r' - 2 s e = r + (dr - 2 s e): one rounding, from the exact r
        const float qx = fmaf(-s2, ex, dx), qy = fmaf(-s2, ey, dy), qz = fmaf(-s2, ez, dz);
        float mx, my, mz;
        float bx = two_sum(p.x, qx, &mx), by = two_sum(p.y, qy, &my), bz = two_sum(p.z, qz, &mz);
        if (phi_at(P, bx, by, bz, mx, my, mz) < 0.0f) {
          bx = p.x; by = p.y; bz = p.z;
          atomicAdd(&ctr->fallbacks, 1ull);
        }
        x = bx; y = by; z = bz;
        const float4 vb = make_float4(2.0f * vw.x - v.x, 2.0f * vw.y - v.y, 2.0f * vw.z - v.z, 1.0f);
        vh = vb;  // a reflected particle keeps its new velocity (no kick); .w flags it
        vt = vb;
        atomicAdd(&ctr->reflections, 1ull);
      }
    }
    p.x = wrap_coord(x, P.L[0]);
    p.y = wrap_coord(y, P.L[1]);
    p.z = wrap_coord(z, P.L[2]);
    A.pos[i] = p;
    A.vel[i] = vh;
    A.vt[i] = vt;
  } else if (P.moving) {
    // frozen particles are part of the solid, which moves with the wall velocity at
    // their position (constant along the motion: the shear has no component along
    // its axis); it is also their velocity in the dissipative force
    const float3 vw = wall_velocity(P, axis_coord(p, P.sh_axis));
    p.x = wrap_coord(p.x + P.dt * vw.x, P.L[0]);
    p.y = wrap_coord(p.y + P.dt * vw.y, P.L[1]);
    p.z = wrap_coord(p.z + P.dt * vw.z, P.L[2]);
    A.pos[i] = p;
    A.vt[i] = make_float4(vw.x, vw.y, vw.z, 0.0f);
  }
  const uint32_t c = cell_off + (uint32_t)cell_of(P, p.x, p.y, p.z);
  C.key[i] = c;
  // The cell's count.  Neighbouring threads mostly hold particles of the same cell (the
  // arrays are in cell order from the previous step), so the lanes of a warp that share
  // a cell add to it with one atomic, whose result nobody waits for; the scatter takes
  // the slots (the per-cell order of the sort fixes the final order).
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, c);
  const int lane = threadIdx.x & 31;
  if (lane == __ffs(peers) - 1) atomicAdd(&C.count[c], (uint32_t)__popc(peers));
  // the scan's tile totals, one atomic per tile the warp touches (usually one)
  const uint32_t tl = c / (uint32_t)kScanTileCells;
  const int first = __ffs(active) - 1;
  const uint32_t tl0 = __shfl_sync(active, tl, first);
  if (__all_sync(active, tl == tl0)) {
    if (lane == first) atomicAdd(tile_counter(C.tile_total, tl0, i >> 5), (uint32_t)__popc(active));
  } else {
    const unsigned tpeers = __match_any_sync(active, tl);
    if (lane == __ffs(tpeers) - 1)
      atomicAdd(tile_counter(C.tile_total, tl, i >> 5), (uint32_t)__popc(tpeers));
  }
}

// A single system takes its parameters by value (kernel-parameter bank); a batch
// reads each particle's system from the table.  Same body, same bits.
// Latency-bound (three particle loads, then mostly arithmetic): the register cap lets 8
// blocks (6 for the batch form) share an SM, which hides more load latency.  The values
// it spills belong to the rare reflection branch; measured with the same bits 13%
// faster on the 1M channel and 25% faster on a 64-system batch.  The pending form holds
// three more loads in flight and gets the 6-block cap (40 registers).
// kPending: the state was left by a Newton's-third-law force kernel (its force in the
// fixed-point sums, its closing kick half done); the host knows which and chooses.
template <bool kBatch, bool kPending>
__global__ void __launch_bounds__(256, kBatch || kPending ? 6 : 8) k_integrate(StepParams P0, const SysDesc* __restrict__ S,
                                                   int nsys, Arrays A, CellList C,
                                                   unsigned long long* __restrict__ facc, int n,
                                                   DevCounters* ctrs, int bump) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // Thread k < nsys advances system k's noise counter for the force of this step;
  // nothing in this launch reads it (the host folds the bump in only when nsys <= n).
  if (bump && i < nsys) ctrs[i].step += 1u;
  if (i >= n) return;
  if constexpr (kBatch) {
    // each thread searches for itself: a block-wide lookup would put a barrier in front
    // of this short, latency-bound kernel (measured 75 -> 99 us on a 64-system batch)
    const int sk = sys_of(S, nsys, (uint32_t)i);
    integrate_body<kPending>(S[sk].P, S[sk].cell_off, ctrs + sk, A, C, facc, n, i);
  } else {
    integrate_body<kPending>(P0, 0u, ctrs, A, C, facc, n, i);
  }
}

// Cell key only (set-up: particles loaded, nothing moves).
__global__ void k_key(const SysDesc* __restrict__ S, int nsys, Arrays A, CellList C, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sk = sys_of(S, nsys, (uint32_t)i);
  const float4 p = A.pos[i];
  const uint32_t c = S[sk].cell_off + (uint32_t)cell_of(S[sk].P, p.x, p.y, p.z);
  C.key[i] = (uint32_t)c;
  atomicAdd(&C.count[c], 1u);
  atomicAdd(tile_counter(C.tile_total, c / (uint32_t)kScanTileCells, i >> 5), 1u);
}

// ---------------------------------------------------------------------------
// Exclusive scan of the per-cell counts in one launch, with no block waiting on
// another.  One block per tile of kScanTileCells cells.  The kernels that fill the
// counts also add each particle to its tile's total (one warp-aggregated atomic per
// tile a warp touches), so a block finds the prefix before its tile by summing the
// totals of the tiles before it: independent loads, all in flight at once.  A
// decoupled look-back (Merrill and Garland 2016) has to learn the same sum from its
// predecessors' published words while they run; on GB300 its chain of release
// stores and acquire polls took 11-13 us for the 340k cells of the 1M-particle
// channel whatever the tile shape.  The scan leaves each cell's start in its count,
// where the scatter takes the cell's slots; the per-cell sort zeroes the counts for the
// next step, and the scatter, which follows every scan, zeroes the tile totals.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;
constexpr int kScanChunk = kScanThreads * kScanPerThread;
static_assert(kScanChunk == kScanTileCells, "one scan block per tile");

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread, plus the block sum of a second
// value; returns the scan, the block total in *total and the second sum in *sum2.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t v2, uint32_t* total,
                                                    uint32_t* sum2) {
  __shared__ uint32_t warp_tot[kScanThreads / 32], warp_tot2[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
  if (lane == 31) warp_tot[warp] = inc;
  if (lane == 0) warp_tot2[warp] = v2;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
    uint32_t t2 = lane < kScanThreads / 32 ? warp_tot2[lane] : 0u;
    t = warp_incl_scan(t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
    if (lane < kScanThreads / 32) warp_tot[lane] = t;
    if (lane == 0) warp_tot2[0] = t2;
  }
  __syncthreads();
  const uint32_t base = warp > 0 ? warp_tot[warp - 1] : 0u;
  *total = warp_tot[kScanThreads / 32 - 1];
  *sum2 = warp_tot2[0];
  return base + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan(uint32_t* count, int m, uint32_t* start,
                                                       uint32_t n_total,
                                                       const uint32_t* __restrict__ tile_total,
                                                       int ntiles) {
  const int t = blockIdx.x;
  const int base = t * kScanChunk + threadIdx.x * kScanPerThread;
  static_assert(kScanPerThread % 4 == 0, "counts move as uint4");
  uint32_t v[kScanPerThread];
  const bool full = base + kScanPerThread <= m;  // base is a multiple of 4: 16-byte aligned
  if (full) {
#pragma unroll
    for (int k = 0; k < kScanPerThread; k += 4) {
      const uint4 q = *reinterpret_cast<const uint4*>(count + base + k);
      v[k] = q.x;
      v[k + 1] = q.y;
      v[k + 2] = q.z;
      v[k + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) v[k] = (base + k < m) ? count[base + k] : 0u;
  }
  // the particles of the tiles before this one
  uint32_t pre = 0;
  for (int j = threadIdx.x; j < t * kTileShards; j += kScanThreads) pre += tile_total[(size_t)j * kTileStride];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) sum += v[k];
  uint32_t total, excl;
  const uint32_t local = block_excl_scan(sum, pre, &total, &excl);
  uint32_t run = excl + local;
  if (full) {
#pragma unroll
    for (int k = 0; k < kScanPerThread; k += 4) {
      uint4 q;
      q.x = run;
      q.y = q.x + v[k];
      q.z = q.y + v[k + 1];
      q.w = q.z + v[k + 2];
      run = q.w + v[k + 3];
      *reinterpret_cast<uint4*>(start + base + k) = q;
      *reinterpret_cast<uint4*>(count + base + k) = q;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
      if (base + k < m) {
        start[base + k] = run;
        count[base + k] = run;
      }
      run += v[k];
    }
  }
  if (t == ntiles - 1 && threadIdx.x == 0) start[m] = n_total;
}

// ---------------------------------------------------------------------------
// Counting-sort scatter, per-cell order, and the gather that reorders the
// particle arrays into cell order.
// ---------------------------------------------------------------------------
// It also clears the scan's tile totals (ntw counters) for the next step's producers:
// the scan, the only reader, has finished.
__global__ void k_scatter(CellList C, int n, int ntw, DevCounters* ctr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int q = i; q < ntw; q += gridDim.x * blockDim.x) C.tile_total[(size_t)q * kTileStride] = 0u;
  if (i >= n) return;
  const uint32_t d = atomicAdd(&C.count[C.key[i]], 1u);  // the cell's next slot
  if (d < (uint32_t)n)
    C.perm[d] = (uint32_t)i;
  else
    atomicOr(&ctr->status, ST_OVERFLOW);  // inconsistent counts: never write out of range
}

// One thread per cell: put the cell's entries of perm in ascending order (insertion
// sort; cells hold a handful of particles, and up to 8 are sorted in registers, the
// rest through a local array).  perm holds each particle's index in the previous cell
// order, itself fixed (particles are loaded in id order), so every cell ends up in an
// order that does not depend on atomic timing, and so does every later floating-point
// sum.  Sorting the indices themselves needs no other load.
constexpr int kCellSortCap = 48;

__global__ void k_cell_sort(CellList C, int ncells, int n, DevCounters* ctr) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  C.count[c] = 0u;  // the scatter's slot cursor: zero for the next step's counts
  const uint32_t b = C.start[c], e = C.start[c + 1];
  if (b > e || e > (uint32_t)n) {  // starts not a valid prefix (only after a failed scan)
    atomicOr(&ctr->status, ST_OVERFLOW);
    return;
  }
  const int m = (int)(e - b);
  if (m <= 1) return;
  if (m > kCellSortCap) {
    atomicOr(&ctr->status, ST_OVERFLOW);
    return;
  }
  if (m <= 8) {
    // small cell (nearly all): sort in registers, fully unrolled
    uint32_t ri[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) ri[k] = k < m ? C.perm[b + k] : 0xFFFFFFFFu;
#pragma unroll
    for (int a = 1; a < 8; ++a)
#pragma unroll
      for (int q = a; q > 0; --q)
        if (ri[q - 1] > ri[q]) {
          const uint32_t t = ri[q - 1];
          ri[q - 1] = ri[q];
          ri[q] = t;
        }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < m) C.perm[b + k] = ri[k];
    return;
  }
  uint32_t idx[kCellSortCap];
  for (int k = 0; k < m; ++k) {
    const uint32_t j = C.perm[b + k];
    int q = k;
    while (q > 0 && idx[q - 1] > j) {
      idx[q] = idx[q - 1];
      --q;
    }
    idx[q] = j;
  }
  for (int k = 0; k < m; ++k) C.perm[b + k] = idx[k];
}

__global__ void __launch_bounds__(256) k_gather(Arrays src, Arrays dst, const uint32_t* perm, int n) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  const uint32_t s = min(perm[d], (uint32_t)(n - 1));
  dst.pos[d] = src.pos[s];
  dst.vt[d] = src.vt[s];
  dst.vel[d] = src.vel[s];
  // the force is not carried: the drift has used it, and the force kernel rewrites it
}

// ---------------------------------------------------------------------------
// Profile sums (Sec. III.A) and whole-system diagnostics, FP64.
// Warps reduce with shuffles: lanes that share a bin add their values with a
// butterfly, and one lane per warp and bin issues the FP64 atomics.  The bin
// index is decided in binary32: b = floor((x - lo) * (nbins / (hi - lo))).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) k_profile(const float4* pos, const float4* vel, int n, int axis,
                                                 int nbins, float lo, float inv_w, double* acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool pending = false;
  int bin = 0;
  double vx = 0, vy = 0, vz = 0;
  if (i < n) {
    const float4 p = pos[i];
    if (!is_solid(p.w)) {
      const float x = axis == 0 ? p.x : (axis == 1 ? p.y : p.z);
      const float u = __fmul_rn(__fsub_rn(x, lo), inv_w);
      const float fb = floorf(u);
      if (fb >= 0.0f && fb < (float)nbins) {
        bin = (int)fb;
        pending = true;
        const float4 v = vel[i];
        vx = v.x; vy = v.y; vz = v.z;
      }
    }
  }
  unsigned mask = __ballot_sync(0xffffffffu, pending);
  while (mask) {
    const int leader = __ffs(mask) - 1;
    const int b0 = __shfl_sync(0xffffffffu, bin, leader);
    const bool mine = pending && bin == b0;
    const double c = warp_sum(mine ? 1.0 : 0.0);
    const double sx = warp_sum(mine ? vx : 0.0);
    const double sy = warp_sum(mine ? vy : 0.0);
    const double sz = warp_sum(mine ? vz : 0.0);
    const double s2 = warp_sum(mine ? vx * vx + vy * vy + vz * vz : 0.0);
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

__global__ void __launch_bounds__(256) k_stats(const float4* pos, const float4* vel, int n, double* acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double vx = 0, vy = 0, vz = 0, c = 0;
  if (i < n) {
    const float4 p = pos[i];
    if (!is_solid(p.w)) {
      const float4 v = vel[i];
      vx = v.x; vy = v.y; vz = v.z; c = 1.0;
    }
  }
  const double s2 = warp_sum(vx * vx + vy * vy + vz * vz);
  vx = warp_sum(vx); vy = warp_sum(vy); vz = warp_sum(vz); c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc + 0, vx);
    atomicAdd(acc + 1, vy);
    atomicAdd(acc + 2, vz);
    atomicAdd(acc + 3, s2);
    atomicAdd(acc + 4, c);
  }
}

// ---------------------------------------------------------------------------
// Set-up kernels.
// ---------------------------------------------------------------------------
// Band mask: a cell is flagged when some point within `margin` of it may have
// phi < 0.  Trilinear interpolation is a convex combination of its eight corner
// nodes, so a point can have phi < 0 only if one of the nodes around it is
// negative; the cell is flagged iff a node in the range covering the cell grown
// by the margin is negative.
__global__ void k_band(StepParams P, uint8_t* band) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.ncells) return;
  const int cx = c % P.nc[0];
  const int cy = (c / P.nc[0]) % P.nc[1];
  const int cz = c / (P.nc[0] * P.nc[1]);
  const int cc[3] = {cx, cy, cz};
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    const float edge = P.L[a] / P.nc[a];
    lo[a] = (int)floorf((cc[a] * edge - P.margin) * P.inv_h) - 1;
    hi[a] = (int)floorf(((cc[a] + 1) * edge + P.margin) * P.inv_h) + 2;
  }
  bool neg = false;
  for (int k = lo[2]; k <= hi[2] && !neg; ++k) {
    const int kz = wrap_node(k, P.pd[2]);
    for (int j = lo[1]; j <= hi[1] && !neg; ++j) {
      const int jy = wrap_node(j, P.pd[1]);
      const float* row = P.phi + ((long)kz * P.pd[1] + jy) * P.pd[0];
      for (int ii = lo[0]; ii <= hi[0]; ++ii) {
        if (row[wrap_node(ii, P.pd[0])] < 0.0f) {
          neg = true;
          break;
        }
      }
    }
  }
  band[c] = neg ? 1 : 0;
}

// Phase field below which a loaded fluid particle counts as inside the solid.
constexpr float kLostPhi = 1e-4f;

// Build the internal arrays from caller input (any order, id a permutation).
__global__ void k_load(StepParams P, const float4* in_pos, const float4* in_vel, const int* in_id,
                       const uint8_t* in_type, Arrays A, uint32_t* seen, int n, DevCounters* ctr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int id = in_id[i];
  if (id < 0 || id >= n || atomicExch(&seen[id], 1u) != 0u) {
    atomicOr(&ctr->status, ST_BADID);
    return;
  }
  const bool solid = in_type[i] != 0;
  const float4 q = in_pos[i];
  float4 p;
  p.x = wrap_coord(q.x - P.L[0] * floorf(q.x * P.invL[0]), P.L[0]);
  p.y = wrap_coord(q.y - P.L[1] * floorf(q.y * P.invL[1]), P.L[1]);
  p.z = wrap_coord(q.z - P.L[2] * floorf(q.z * P.invL[2]), P.L[2]);
  p.w = __uint_as_float((uint32_t)id | (solid ? kSolidBit : 0u));
  if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) atomicOr(&ctr->status, ST_NAN);
  float4 v = in_vel[i];
  v.w = 0.0f;
  if (solid) {
    const float3 vw = wall_velocity(P, axis_coord(p, P.sh_axis));
    v = make_float4(vw.x, vw.y, vw.z, 0.0f);
  }
  // A step decides reflections on the exact drifted position and then stores it
  // rounded to binary32, so a particle that ended just outside the wall can read a
  // phase field a few 1e-6 below zero; only a particle clearly inside the solid is lost.
  if (!solid && phi_at(P, p.x, p.y, p.z) < -kLostPhi) atomicOr(&ctr->status, ST_LOST);
  // stored at index id: the first cell order, and every later one, then does not
  // depend on the order of the input
  A.pos[id] = p;
  A.vel[id] = solid ? make_float4(0.f, 0.f, 0.f, 0.f) : v;
  A.vt[id] = v;
  A.frc[id] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Unsort into id order (outputs may be null).
__global__ void k_unsort(Arrays A, int n, float4* out_pos, float4* out_vel, float4* out_frc,
                         int* out_id, uint8_t* out_type) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = A.pos[i];
  const uint32_t id = id_of(p.w);
  if (id >= (uint32_t)n) return;
  if (out_pos) out_pos[id] = make_float4(p.x, p.y, p.z, 0.0f);
  if (out_vel) {
    float4 v = A.vel[i];
    v.w = A.vt[i].w;  // 1: reflected in the last step
    out_vel[id] = v;
  }
  if (out_frc) {
    float4 f = A.frc[i];
    f.w = 0.0f;
    out_frc[id] = f;
  }
  if (out_id) out_id[id] = (int)id;
  if (out_type) out_type[id] = is_solid(p.w) ? 1 : 0;
}

__global__ void k_bump_step(DevCounters* ctr, int nsys) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nsys) ctr[k].step += 1u;
}

// ---------------------------------------------------------------------------
// Host launch wrappers.
// ---------------------------------------------------------------------------
static inline int blocks(long n, int t) { return (int)((n + t - 1) / t); }

static bool bump_folded(int n, int nsys) { return n > 0 && nsys <= n; }

int integrate_kernels(int n, int nsys) { return (n > 0 ? 1 : 0) + (bump_folded(n, nsys) ? 0 : 1); }

void launch_integrate(const StepParams& P0, const SysDesc* S, int nsys, const Arrays& A,
                      const CellList& C, unsigned long long* facc, bool pending, int n,
                      DevCounters* ctr, cudaStream_t s) {
  const int bump = bump_folded(n, nsys) ? 1 : 0;
  if (!bump) k_bump_step<<<blocks(nsys, 128), 128, 0, s>>>(ctr, nsys);
  if (n <= 0) return;
  const int nb = blocks(n, 256);
  if (nsys == 1) {
    if (pending)
      k_integrate<false, true><<<nb, 256, 0, s>>>(P0, S, nsys, A, C, facc, n, ctr, bump);
    else
      k_integrate<false, false><<<nb, 256, 0, s>>>(P0, S, nsys, A, C, facc, n, ctr, bump);
  } else {
    if (pending)
      k_integrate<true, true><<<nb, 256, 0, s>>>(P0, S, nsys, A, C, facc, n, ctr, bump);
    else
      k_integrate<true, false><<<nb, 256, 0, s>>>(P0, S, nsys, A, C, facc, n, ctr, bump);
  }
}

void launch_key(const SysDesc* S, int nsys, const Arrays& A, const CellList& C, int n,
                cudaStream_t s) {
  if (n > 0) k_key<<<blocks(n, 256), 256, 0, s>>>(S, nsys, A, C, n);
}

int scan_blocks(int ncells) { return ncells > 0 ? blocks(ncells, kScanChunk) : 1; }

int scan_kernels(int) { return 1; }

void launch_scan(const CellList& C, int ncells, int n, cudaStream_t s) {
  const int nt = scan_blocks(ncells);
  k_scan<<<nt, kScanThreads, 0, s>>>(C.count, ncells, C.start, (uint32_t)n, C.tile_total, nt);
}

// With no particles nothing fills the counts, so the tile totals stay zero.
void launch_scatter(const CellList& C, int n, int ncells, DevCounters* ctr, cudaStream_t s) {
  if (n > 0) k_scatter<<<blocks(n, 256), 256, 0, s>>>(C, n, scan_blocks(ncells) * kTileShards, ctr);
}

void launch_cell_sort(const CellList& C, int n, int ncells, DevCounters* ctr, cudaStream_t s) {
  if (n > 0) k_cell_sort<<<blocks(ncells, 128), 128, 0, s>>>(C, ncells, n, ctr);
}

void launch_gather(const CellList& C, const Arrays& src, const Arrays& dst, int n, cudaStream_t s) {
  if (n > 0) k_gather<<<blocks(n, 256), 256, 0, s>>>(src, dst, C.perm, n);
}

void launch_sort(const CellList& C, const Arrays& src, const Arrays& dst, int n, int ncells,
                 DevCounters* ctr, cudaStream_t s) {
  launch_scatter(C, n, ncells, ctr, s);
  launch_cell_sort(C, n, ncells, ctr, s);
  launch_gather(C, src, dst, n, s);
}

void launch_profile(const float4* pos, const float4* vel, int n, int axis, int nbins, float lo,
                    float inv_w, double* acc, cudaStream_t s) {
  if (n > 0) k_profile<<<blocks(n, 256), 256, 0, s>>>(pos, vel, n, axis, nbins, lo, inv_w, acc);
}

void launch_stats(const float4* pos, const float4* vel, int n, double* acc, cudaStream_t s) {
  if (n > 0) k_stats<<<blocks(n, 256), 256, 0, s>>>(pos, vel, n, acc);
}

void launch_band(const StepParams& P, uint8_t* band, cudaStream_t s) {
  k_band<<<blocks(P.ncells, 128), 128, 0, s>>>(P, band);
}

void launch_load(const StepParams& P, const float4* in_pos, const float4* in_vel, const int* in_id,
                 const uint8_t* in_type, const Arrays& A, uint32_t* seen, int n, DevCounters* ctr,
                 cudaStream_t s) {
  if (n > 0)
    k_load<<<blocks(n, 256), 256, 0, s>>>(P, in_pos, in_vel, in_id, in_type, A, seen, n, ctr);
}

void launch_unsort(const Arrays& A, int n, float4* out_pos, float4* out_vel, float4* out_frc,
                   int* out_id, uint8_t* out_type, cudaStream_t s) {
  if (n > 0)
    k_unsort<<<blocks(n, 256), 256, 0, s>>>(A, n, out_pos, out_vel, out_frc, out_id, out_type);
}


}  // namespace dpd
