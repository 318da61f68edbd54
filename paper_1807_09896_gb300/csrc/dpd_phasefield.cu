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

// Tile of one thread block: TX x TY nodes of a z plane, marching through KZ planes.
constexpr int TX = 32, TY = 8, KZ = 16;
constexpr int SX = TX + 2, SY = TY + 2, SN = SX * SY;  // one plane of the tile with its halo
constexpr int kRing = 4;  // planes k-1, k, k+1 in use and k+2 being filled: one barrier per plane
static_assert(SN <= 2 * TX * TY, "each thread loads at most two halo'd tile nodes per plane");

// 2.5-D blocked stencil: each block keeps a ring of halo'd planes in shared memory,
// so every node is read from global memory about (SX SY / TX TY) (KZ + 2) / KZ = 1.5
// times (the halo share hits L2) and written once.  Periodic in every direction.
__global__ void __launch_bounds__(TX * TY) k_relax(const float* __restrict__ phi, float* __restrict__ out,
                                                   int nx, int ny, int nz, float inv, float dtau,
                                                   int curvature) {
  __shared__ float tile[kRing][SN];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * KZ;
  const int k1 = min(k0 + KZ, nz);
  const long plane = (long)nx * ny;
  // offsets within a plane of the (at most two) tile nodes this thread loads; fixed along z
  long off[2];
  bool has[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int t = tid + e * TX * TY;
    has[e] = t < SN;
    const int gi = ((i0 - 1 + t % SX) % nx + nx) % nx;
    const int gj = ((j0 - 1 + t / SX) % ny + ny) % ny;
    off[e] = (long)gj * nx + gi;
  }
  auto load = [&](int slot, int kk) {
    kk = kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk);
    const float* src = phi + (long)kk * plane;
#pragma unroll
    for (int e = 0; e < 2; ++e)
      if (has[e]) tile[slot][tid + e * TX * TY] = __ldg(src + off[e]);
  };
  load((k0 - 1 + kRing) % kRing, k0 - 1);
  load(k0 % kRing, k0);
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const bool active = i < nx && j < ny;
  const int c = (threadIdx.y + 1) * SX + threadIdx.x + 1;
  const float inv2 = inv * inv;
  for (int k = k0; k < k1; ++k) {
    load((k + 1) % kRing, k + 1);
    __syncthreads();
    if (active) {
      const float* m = tile[(k + kRing - 1) % kRing];
      const float* o = tile[k % kRing];
      const float* q = tile[(k + 1) % kRing];
      const float p = o[c];
      const float xp = o[c + 1], xm = o[c - 1];
      const float yp = o[c + SX], ym = o[c - SX];
      const float zp = q[c], zm = m[c];
      const float sxx = (xp - 2.0f * p + xm) * inv2;
      const float syy = (yp - 2.0f * p + ym) * inv2;
      const float szz = (zp - 2.0f * p + zm) * inv2;
      const float lap = sxx + syy + szz;
      const float reaction = p * (1.0f - p * p);
      float rhs = lap + reaction;
      if (curvature) {
        // phi_nn = (n.H.n |g|^2 + delta lap) / (|g|^2 + delta): the normal's direction is
        // ill-conditioned where g -> 0, and there the Laplacian takes over
        const float gx = (xp - xm) * (0.5f * inv), gy = (yp - ym) * (0.5f * inv),
                    gz = (zp - zm) * (0.5f * inv);
        const float g2 = gx * gx + gy * gy + gz * gz;
        const float qq = 0.25f * inv2;
        const float sxy = (o[c + SX + 1] - o[c - SX + 1] - o[c + SX - 1] + o[c - SX - 1]) * qq;
        const float sxz = (q[c + 1] - m[c + 1] - q[c - 1] + m[c - 1]) * qq;
        const float syz = (q[c + SX] - m[c + SX] - q[c - SX] + m[c - SX]) * qq;
        const float num = gx * gx * sxx + gy * gy * syy + gz * gz * szz +
                          2.0f * (gx * gy * sxy + gx * gz * sxz + gy * gz * syz);
        rhs = (num + kDelta * lap) / (g2 + kDelta) + reaction;
      }
      out[(long)k * plane + (long)j * nx + i] = p + dtau * rhs;
    }
  }
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
  const dim3 grid((unsigned)((dims[0] + TX - 1) / TX), (unsigned)((dims[1] + TY - 1) / TY),
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
    k_relax<<<grid, dim3(TX, TY)>>>(a, b, dims[0], dims[1], dims[2], (float)(1.0 / hp), (float)dtau,
                                    curvature);
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
