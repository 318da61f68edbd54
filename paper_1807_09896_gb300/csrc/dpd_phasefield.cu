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
#include <cmath>
#include <cstdio>

#include "../../include/dpd.h"
#include "dpd_launch.h"

namespace {

constexpr float kDelta = 1e-4f;  // blend of the normal second derivative into the Laplacian

// Tile of one thread block: (2 TX) x TY nodes of a z plane (two x neighbours per
// thread), marching through KZ planes.
constexpr int TX = 32, TY = 8, KZ = 16;
constexpr int NXT = 2 * TX;                             // nodes of a tile row
constexpr int SX = NXT + 2, SY = TY + 2, SN = SX * SY;  // one halo'd plane of the tile
constexpr int kLoads = (SN + TX * TY - 1) / (TX * TY);  // tile nodes each thread copies
constexpr int kAhead = 4;                               // planes in flight
constexpr int kRing = 8;                                // slots (>= kAhead + 2, a power of 2)
static_assert(SX % 2 == 0 && SN % 2 == 0, "paired shared loads need even row and plane pitch");
static_assert(kRing >= kAhead + 2 && (kRing & (kRing - 1)) == 0, "ring too small");
static_assert((kLoads - 1) * TX * TY < SN, "every thread copies kLoads - 1 nodes unconditionally");

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

__device__ __forceinline__ void copy4_async(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void commit_async() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_async() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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

__device__ __forceinline__ void store_pair(float* dst, float2 o, int i, int nx, int pair_store) {
  if (pair_store) {
    *reinterpret_cast<float2*>(dst) = o;  // i even and nx even: 8-byte aligned, i + 1 < nx
  } else {
    dst[0] = o.x;
    if (i + 1 < nx) dst[1] = o.y;
  }
}

// 2.5-D blocked stencil.  Each block streams planes k0-1 .. k0+KZ (periodic) through
// a ring of halo'd shared-memory slots filled kAhead planes ahead by cp.async, and
// carries the per-plane terms of planes k-1, k, k+1 in registers; the plane loop has
// a constant trip count and is unrolled, so those roles rotate without copies.  Each
// node is read from global memory (SX SY / NXT TY) (KZ + 2) / KZ = 1.45 times (the
// halo share hits L2) and written once.  Planes past nz (last block row) are read
// wrapped and not stored.
//
// In raw differences (D_a = 2 h' g_a, S_aa = h'^2 phi_aa, S_ab = 4 h'^2 phi_ab) the
// right-hand side is  (1/h'^2) (N + d' L) / (G + d') + phi (1 - phi^2)  with
// G = sum D_a^2, L = sum S_aa, N = sum D_a^2 S_aa + (1/2) sum_{a<b} D_a D_b S_ab and
// d' = 4 delta h'^2: the same expression as (n.H.n |g|^2 + delta lap)/(|g|^2 + delta).
template <bool kCurvature>
__global__ void __launch_bounds__(TX * TY) k_relax(const float* __restrict__ phi, float* __restrict__ out,
                                                   int nx, int ny, int nz, float inv, float dtau,
                                                   int pair_store) {
  __shared__ __align__(16) float ring[kRing][SN];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int i0 = blockIdx.x * NXT, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * KZ;
  const long plane = (long)nx * ny;
  long off[kLoads];  // offsets within a plane of the tile nodes this thread copies
#pragma unroll
  for (int e = 0; e < kLoads; ++e) {
    const int t = min(tid + e * TX * TY, SN - 1);
    const int gi = ((i0 - 1 + t % SX) % nx + nx) % nx;
    const int gj = ((j0 - 1 + t / SX) % ny + ny) % ny;
    off[e] = (long)gj * nx + gi;
  }
  int kk = k0 == 0 ? nz - 1 : k0 - 1;  // next plane to copy, and its start
  const float* src = phi + (long)kk * plane;
  auto issue = [&](int s) {  // copy the plane of step s into slot s
    float* dst = ring[s & (kRing - 1)];
#pragma unroll
    for (int e = 0; e < kLoads; ++e)
      if (e < kLoads - 1 || tid + e * TX * TY < SN) copy4_async(dst + tid + e * TX * TY, src + off[e]);
    commit_async();
    if (++kk == nz) {
      kk = 0;
      src = phi;
    } else {
      src += plane;
    }
  };
#pragma unroll
  for (int s = 0; s < kAhead; ++s) issue(s);

  const int i = i0 + 2 * threadIdx.x, j = j0 + threadIdx.y;
  const bool active = i < nx && j < ny;
  const int row = threadIdx.y + 1, col = 2 * threadIdx.x;
  const float inv2 = inv * inv;
  const float dprime = 4.0f * kDelta / inv2;
  float* dst = out + (long)k0 * plane + (long)j * nx + i;
  PlaneTerms prev{}, cur{};
#pragma unroll
  for (int s = 0; s < KZ + 2; ++s) {  // step s consumes plane k0 - 1 + s
    if (s + kAhead < KZ + 2)
      issue(s + kAhead);
    else
      commit_async();      // empty group: the count below stays uniform
    wait_async<kAhead>();  // plane of step s has landed (at most kAhead younger groups pending)
    __syncthreads();       // ... for every thread's copies
    const PlaneTerms nxt = plane_terms(ring[s & (kRing - 1)], row, col);
    if (s >= 2) {
      if (active && k0 + s - 2 < nz)  // node plane k = k0 + s - 2
        store_pair(dst, node_update<kCurvature>(prev, cur, nxt, inv2, dprime, dtau), i, nx, pair_store);
      dst += plane;
    }
    prev = cur;
    cur = nxt;
  }
  wait_async<0>();
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
  const dim3 grid((unsigned)((dims[0] + NXT - 1) / NXT), (unsigned)((dims[1] + TY - 1) / TY),
                  (unsigned)((dims[2] + KZ - 1) / KZ));
  float *a = nullptr, *b = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&a, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMemcpy(a, phi, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    if (curvature)
      k_relax<true><<<grid, dim3(TX, TY)>>>(a, b, dims[0], dims[1], dims[2], (float)(1.0 / hp),
                                            (float)dtau, dims[0] % 2 == 0);
    else
      k_relax<false><<<grid, dim3(TX, TY)>>>(a, b, dims[0], dims[1], dims[2], (float)(1.0 / hp),
                                             (float)dtau, dims[0] % 2 == 0);
    e = cudaGetLastError();
    float* t = a;
    a = b;
    b = t;
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
  if (e == cudaSuccess) e = cudaMemcpy(phi, a, sizeof(float) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ms_per_iter) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_per_iter = iters > 0 ? ms / iters : 0.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(a);
  cudaFree(b);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "dpd_relax_phase_field: %s", cudaGetErrorString(e));
    dpd::set_global_error(msg);
    return DPD_ECUDA;
  }
  return DPD_OK;
}
