// dpd_phasefield.cu -- relaxation of a phase field from a step function on a
// periodic grid (Xu & Meakin, arXiv:1807.09896, Sec. II.B, Eqs. 13-15).
//
// In the scaled coordinates x' = x / eps the field evolves in pseudo time by
//   d phi / dt' = lap' phi + phi (1 - phi^2) - kappa |grad' phi|,
//   kappa = div'(grad' phi / |grad' phi|)                               (Eq. 15).
// Since kappa |grad phi| = lap phi - phi_nn (phi_nn: the second derivative along the
// unit normal), the right-hand side is phi_nn + phi (1 - phi^2): the 1-D Allen-Cahn
// equation along the normal, whose steady profile is tanh(d / (sqrt(2) eps)) (Eq. 14),
// with no curvature-driven motion of the interface.  Where grad phi -> 0 the normal is
// undefined; there phi_nn is blended into the Laplacian (see kDelta).  One launch is one explicit
// Euler step over every node: a 19-point stencil (second-order central
// differences), bound by memory traffic: 4 B read and 4 B written per node.
//
// The field lives on the device in a padded layout: one ghost node on each side in x
// and y (x padded to a row of a multiple of 4 floats, so that every row starts on a
// 16-byte boundary).  A launch reads halo'd planes of its tile with bulk tensor
// copies (TMA) and writes every node together with its periodic ghost copies, so the
// next launch's copies never need to wrap in x or y (z wraps by plane index).
#include <cuda.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/dpd.h"
#include "dpd_launch.h"

namespace {

constexpr float kDelta = 1e-4f;  // blend of the normal second derivative into the Laplacian

// Tile of one thread block: (2 TX) x TY nodes of a z plane (two x neighbours per
// thread), marching through KZ planes.
constexpr int TX = 32, TY = 8, KZ = 16;
constexpr int NXT = 2 * TX;  // nodes of a tile row
// One halo'd plane of the tile as one tensor-copy box: SX x SY nodes from padded
// (i0, j0), i.e. x from i0 - 1 (the halo) to i0 + 66 and y from j0 - 1 to j0 + TY; SX
// is a multiple of 4 (16-byte rows, the copy's rule) and even (paired shared loads).
constexpr int SX = NXT + 4, SY = TY + 2;
constexpr int kSlot = ((SX * SY * 4 + 127) / 128) * 128 / 4;  // slot pitch, 128-byte aligned
constexpr int kAhead = 4;                                      // planes in flight
constexpr int kRing = 8;  // slots (>= kAhead + 2, a power of 2)
constexpr unsigned kBoxBytes = SX * SY * 4;
static_assert(SX % 4 == 0, "a tensor-copy row must be a multiple of 16 bytes");
static_assert(kRing >= kAhead + 2 && (kRing & (kRing - 1)) == 0, "ring too small");
// Bounded waits: polls of a plane's barrier before the block gives up (a copy that
// never lands); the launch then reports the failure through an error word.
constexpr int kWaitPolls = 1 << 20;

// Elementwise arithmetic on a thread's two nodes, rounded to nearest with no
// contraction, so the result does not depend on how the compiler fuses it.
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// A shared-memory barrier that counts the bytes of one tensor copy.
__device__ __forceinline__ void bar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// Copy the box at (x, y, z) of the tensor map into dst; bar completes when it landed.
__device__ __forceinline__ void copy_plane(float* dst, const CUtensorMap* map, int x, int y, int z,
                                           unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(kBoxBytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Wait until the barrier's phase `parity` completed; false if it did not within the
// poll limit.
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned parity) {
  for (int k = 0; k < kWaitPolls; ++k) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// What one plane contributes at the thread's two nodes (x = node i, y = node i + 1),
// as raw differences (no 1/h' factors): value, x and y central differences, x and
// y neighbour sums and the 4-point mixed xy difference.
struct PlaneTerms {
  float2 p, dx, dy, xs, ys, sxy;
};

__device__ __forceinline__ PlaneTerms plane_terms(const float* slot, int row, int col) {
  // rows j-1, j, j+1 of columns i-1 .. i+2, read as pairs (col is even)
  const float2 d0 = *reinterpret_cast<const float2*>(slot + (row - 1) * SX + col);
  const float2 d1 = *reinterpret_cast<const float2*>(slot + (row - 1) * SX + col + 2);
  const float2 r0 = *reinterpret_cast<const float2*>(slot + row * SX + col);
  const float2 r1 = *reinterpret_cast<const float2*>(slot + row * SX + col + 2);
  const float2 u0 = *reinterpret_cast<const float2*>(slot + (row + 1) * SX + col);
  const float2 u1 = *reinterpret_cast<const float2*>(slot + (row + 1) * SX + col + 2);
  PlaneTerms t;
  t.p = make_float2(r0.y, r1.x);
  t.dx = sub2(r1, r0);
  t.xs = add2(r1, r0);
  const float2 yp = make_float2(u0.y, u1.x), ym = make_float2(d0.y, d1.x);
  t.dy = sub2(yp, ym);
  t.ys = add2(yp, ym);
  t.sxy = sub2(sub2(u1, d1), sub2(u0, d0));  // (i+1,j+1) - (i+1,j-1) - (i-1,j+1) + (i-1,j-1)
  return t;
}

// New value of the thread's two nodes of plane k from the terms of planes k-1, k, k+1
// (the right-hand side written out in raw differences, see k_relax).
template <bool kCurvature>
__device__ __forceinline__ float2 node_update(const PlaneTerms& prev, const PlaneTerms& cur,
                                              const PlaneTerms& nxt, float inv2, float dprime,
                                              float dtau) {
  const float2 p = cur.p;
  const float2 dz = sub2(nxt.p, prev.p);
  const float2 sxx = fma2(splat(-2.0f), p, cur.xs);
  const float2 syy = fma2(splat(-2.0f), p, cur.ys);
  const float2 szz = fma2(splat(-2.0f), p, add2(nxt.p, prev.p));
  const float2 lap = add2(add2(sxx, syy), szz);
  const float2 reaction = fma2(mul2(p, p), make_float2(-p.x, -p.y), p);
  float2 q = lap;
  if (kCurvature) {
    const float2 dx = cur.dx, dy = cur.dy;
    const float2 sxz = sub2(nxt.dx, prev.dx), syz = sub2(nxt.dy, prev.dy);
    const float2 G = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, splat(dprime))));
    float2 N = mul2(mul2(dz, szz), dz);
    N = fma2(mul2(dy, syy), dy, N);
    N = fma2(mul2(dx, sxx), dx, N);
    const float2 m1 = fma2(dz, sxz, mul2(dy, cur.sxy));
    const float2 M = fma2(dx, m1, mul2(dy, mul2(dz, syz)));
    N = fma2(splat(0.5f), M, N);
    const float2 num = fma2(splat(dprime), lap, N);
    q = make_float2(__fdividef(num.x, G.x), __fdividef(num.y, G.y));  // G >= d' > 0
  }
  const float2 rhs = fma2(splat(inv2), q, reaction);
  return fma2(splat(dtau), rhs, p);
}

// Padded layout: node (x, y, z) at z * pz + (y + 1) * px + (x + 1); ghosts at x = -1,
// nx and y = -1, ny hold the periodic images.
struct Padded {
  int nx, ny, nz, px;  // px: row pitch in floats (multiple of 4, >= nx + 2)
  long pz;             // plane pitch: px (ny + 2)
};

// The ghost images of node (x, y) of a plane (pl: the plane's padded base), for a node
// on the edge of the grid (x or y at 0 or at its last index).
__device__ __noinline__ void store_ghosts(float* pl, const Padded& G, int x, int y, float v) {
  const int xs[2] = {x + 1, x == 0 ? G.nx + 1 : (x == G.nx - 1 ? 0 : -1)};
  const int ys[2] = {y + 1, y == 0 ? G.ny + 1 : (y == G.ny - 1 ? 0 : -1)};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      if ((a || b) && xs[a] >= 0 && ys[b] >= 0) pl[(long)ys[b] * G.px + xs[a]] = v;
}

// 2.5-D blocked stencil.  Each block streams planes k0-1 .. k0+KZ (periodic in z)
// through a ring of halo'd shared-memory slots, each filled by one tensor copy issued
// kAhead planes ahead by one thread and completed through the slot's barrier, and
// carries the per-plane terms of planes k-1, k, k+1 in registers; the plane loop has a
// constant trip count and is unrolled, so those roles rotate without copies.  Each node
// is read from global memory SX SY / (NXT TY) (KZ + 2) / KZ = 1.5 times (the halo share
// hits L2) and written once (plus its ghost images at the edges).  Planes past nz (last
// block row) are read wrapped and not stored.  A copy that does not land within the
// poll limit makes the block set *err, wait (bounded) for its other copies and return.
//
// In raw differences (D_a = 2 h' g_a, S_aa = h'^2 phi_aa, S_ab = 4 h'^2 phi_ab) the
// right-hand side is  (1/h'^2) (N + d' L) / (G + d') + phi (1 - phi^2)  with
// G = sum D_a^2, L = sum S_aa, N = sum D_a^2 S_aa + (1/2) sum_{a<b} D_a D_b S_ab and
// d' = 4 delta h'^2: the same expression as (n.H.n |g|^2 + delta lap)/(|g|^2 + delta).
template <bool kCurvature>
__global__ void __launch_bounds__(TX * TY) k_relax(const __grid_constant__ CUtensorMap map,
                                                   float* __restrict__ out, Padded G, float inv,
                                                   float dtau, int* err) {
  __shared__ __align__(128) float ring[kRing][kSlot];
  __shared__ __align__(8) unsigned long long bar[kRing];
  __shared__ int failed;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int i0 = blockIdx.x * NXT, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * KZ;
  if (tid == 0) {
    for (int q = 0; q < kRing; ++q) bar_init(&bar[q]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    failed = 0;
  }
  __syncthreads();
  int kk = k0 == 0 ? G.nz - 1 : k0 - 1;  // next plane to copy
  auto issue = [&](int s) {  // copy the plane of step s into slot s (thread 0)
    copy_plane(ring[s & (kRing - 1)], &map, i0, j0, kk, &bar[s & (kRing - 1)]);
    kk = kk + 1 == G.nz ? 0 : kk + 1;
  };
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < kAhead; ++s) issue(s);
  }
  const int i = i0 + 2 * threadIdx.x, j = j0 + threadIdx.y;
  const bool active = i < G.nx && j < G.ny;
  const int row = threadIdx.y + 1, col = 2 * threadIdx.x;
  const float inv2 = inv * inv;
  const float dprime = 4.0f * kDelta / inv2;
  PlaneTerms prev{}, cur{};
  int issued = kAhead, stopped = KZ + 2;
#pragma unroll
  for (int s = 0; s < KZ + 2; ++s) {  // step s consumes plane k0 - 1 + s
    if (tid == 0 && s + kAhead < KZ + 2) {
      issue(s + kAhead);  // its slot was last read at step s + kAhead - kRing < s - 1
      ++issued;
    }
    // slot s & (kRing - 1) is used for the (s / kRing)-th time: that phase's parity.
    // One warp waits for it; the block barrier holds the others (and makes sure every
    // thread is past reading slot s - 1).
    if (tid < 32 && !bar_wait(&bar[s & (kRing - 1)], (unsigned)((s / kRing) & 1))) failed = 1;
    __syncthreads();
    if (failed) {
      stopped = s;
      break;
    }
    const PlaneTerms nxt = plane_terms(ring[s & (kRing - 1)], row, col);
    if (s >= 2) {
      const int k = k0 + s - 2;
      if (active && k < G.nz) {
        const float2 o = node_update<kCurvature>(prev, cur, nxt, inv2, dprime, dtau);
        float* pl = out + (long)k * G.pz;
        float* row_out = pl + (long)(j + 1) * G.px + (i + 1);
        row_out[0] = o.x;
        const bool second = i + 1 < G.nx;
        if (second) row_out[1] = o.y;
        if (i == 0 || i + 2 >= G.nx || j == 0 || j == G.ny - 1) {  // a node on the grid's edge
          store_ghosts(pl, G, i, j, o.x);
          if (second) store_ghosts(pl, G, i + 1, j, o.y);
        }
      }
    }
    prev = cur;
    cur = nxt;
  }
  if (failed && tid == 0) {
    atomicExch(err, 1);
    // let the copies issued but not consumed land before the block's shared memory is
    // released (each slot is at most kRing - kAhead uses ahead, so the parities are exact)
    for (int s = stopped; s < issued; ++s) bar_wait(&bar[s & (kRing - 1)], (unsigned)((s / kRing) & 1));
  }
}

// Plain layout (x fastest, nx ny nz) <-> padded layout with ghost images.
__global__ void k_pad(const float* __restrict__ src, float* __restrict__ dst, Padded G) {
  const long n = (long)G.px * (G.ny + 2) * G.nz;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int px = (int)(q % G.px);
    const int py = (int)((q / G.px) % (G.ny + 2));
    const int z = (int)(q / ((long)G.px * (G.ny + 2)));
    if (px > G.nx + 1) {
      dst[q] = 0.0f;  // beyond the row's ghost: never read
      continue;
    }
    const int x = px == 0 ? G.nx - 1 : (px == G.nx + 1 ? 0 : px - 1);
    const int y = py == 0 ? G.ny - 1 : (py == G.ny + 1 ? 0 : py - 1);
    dst[q] = src[((long)z * G.ny + y) * G.nx + x];
  }
}

__global__ void k_unpad(const float* __restrict__ src, float* __restrict__ dst, Padded G) {
  const long n = (long)G.nx * G.ny * G.nz;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int x = (int)(q % G.nx);
    const int y = (int)((q / G.nx) % G.ny);
    const int z = (int)(q / ((long)G.nx * G.ny));
    dst[q] = src[(long)z * G.pz + (long)(y + 1) * G.px + (x + 1)];
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the
// driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;

bool encode_map(CUtensorMap* map, float* base, const Padded& G) {
  std::call_once(g_encode_once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_encode = (EncodeTiledFn)f;
  });
  if (!g_encode) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)G.px, (cuuint64_t)(G.ny + 2), (cuuint64_t)G.nz};
  const cuuint64_t stride[2] = {(cuuint64_t)G.px * 4, (cuuint64_t)G.pz * 4};
  const cuuint32_t box[3] = {SX, SY, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dim, stride, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" int dpd_relax_phase_field(float* phi, const int dims[3], double spacing, double eps,
                                     int iters, double dtau, int curvature, double* ms_per_iter) {
  char msg[256];
  if (!phi || !dims || !(spacing > 0) || !(eps > 0) || iters < 0 || !(dtau > 0)) {
    dpd::set_global_error("dpd_relax_phase_field: bad argument");
    return DPD_EINVAL;
  }
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 3) {
      dpd::set_global_error("dpd_relax_phase_field: every dimension needs at least 3 nodes");
      return DPD_EINVAL;
    }
  if (dims[1] > 65535 * TY || dims[2] > 65535) {
    dpd::set_global_error("dpd_relax_phase_field: at most 524280 nodes along y and 65535 along z");
    return DPD_EINVAL;
  }
  const double hp = spacing / eps;
  if (dtau > hp * hp / 6.0) {
    snprintf(msg, sizeof msg,
             "dpd_relax_phase_field: dtau %g exceeds the explicit stability limit (h/eps)^2/6 = %g",
             dtau, hp * hp / 6.0);
    dpd::set_global_error(msg);
    return DPD_EINVAL;
  }
  const long n = (long)dims[0] * dims[1] * dims[2];
  Padded G;
  G.nx = dims[0];
  G.ny = dims[1];
  G.nz = dims[2];
  G.px = ((dims[0] + 2 + 3) / 4) * 4;
  G.pz = (long)G.px * (dims[1] + 2);
  const long np = G.pz * dims[2];
  const dim3 grid((unsigned)((dims[0] + NXT - 1) / NXT), (unsigned)((dims[1] + TY - 1) / TY),
                  (unsigned)((dims[2] + KZ - 1) / KZ));
  float *a = nullptr, *b = nullptr;
  int* d_err = nullptr;
  int h_err = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUtensorMap map_a, map_b;
  cudaError_t e = cudaMalloc((void**)&a, sizeof(float) * np);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b, sizeof(float) * np);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(int));
  // the plain field goes to b (np >= n), then into a's padded layout with its ghosts
  if (e == cudaSuccess) e = cudaMemcpy(b, phi, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_pad<<<1024, 256>>>(b, a, G);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !(encode_map(&map_a, a, G) && encode_map(&map_b, b, G))) {
    dpd::set_global_error("dpd_relax_phase_field: cuTensorMapEncodeTiled unavailable or failed");
    cudaFree(a);
    cudaFree(b);
    cudaFree(d_err);
    return DPD_ECUDA;
  }
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    const CUtensorMap& src = (it & 1) ? map_b : map_a;
    float* dst = (it & 1) ? a : b;
    if (curvature)
      k_relax<true><<<grid, dim3(TX, TY)>>>(src, dst, G, (float)(1.0 / hp), (float)dtau, d_err);
    else
      k_relax<false><<<grid, dim3(TX, TY)>>>(src, dst, G, (float)(1.0 / hp), (float)dtau, d_err);
    e = cudaGetLastError();
  }
  float* result = (iters & 1) ? b : a;
  float* plain = (iters & 1) ? a : b;
  if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
  if (e == cudaSuccess) {
    k_unpad<<<1024, 256>>>(result, plain, G);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(phi, plain, sizeof(float) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ms_per_iter) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_per_iter = iters > 0 ? ms / iters : 0.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(a);
  cudaFree(b);
  cudaFree(d_err);
  if (e == cudaSuccess && h_err) {
    dpd::set_global_error("dpd_relax_phase_field: a plane copy did not complete (bounded wait gave up)");
    return DPD_ETIMEOUT;
  }
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "dpd_relax_phase_field: %s", cudaGetErrorString(e));
    dpd::set_global_error(msg);
    return DPD_ECUDA;
  }
  return DPD_OK;
}
