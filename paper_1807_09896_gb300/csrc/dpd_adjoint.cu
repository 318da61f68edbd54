// dpd_adjoint.cu -- reverse-mode derivative of a window of DPD time steps
// (Xu & Meakin, arXiv:1807.09896: pair force Eqs. 3-10, Groot-Warren step,
// bounce-back reflection Eq. 17) with respect to the wall interaction a_fs, the
// dissipation gamma (sigma tied to it by Eq. 8) and the body force g_x, for a
// near-wall velocity-profile loss.
//
// The forward window keeps a checkpoint every K steps.  The backward pass
// recomputes each segment from its checkpoint while recording every step (the
// cell-ordered state, the sort permutation and the cell starts) and then walks
// the recorded steps in reverse.  The pair noise is never stored: it is counter
// based and drawn again.  Events are frozen: which particles were reflected,
// which cell held whom and which profile bin a particle counted in are taken from
// the forward trajectory (the loss is differentiated in the velocities only).
// Per-pair derivatives are binary32; parameter gradients accumulate in binary64.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dpd.h"
#include "dpd_common.cuh"
#include "dpd_engine.h"
#include "dpd_launch.h"
#include "dpd_system.h"

namespace dpd {
namespace {

struct WallBins {
  int axis;
  float lo, hi;    // wall positions along axis
  float inv_width;
  int nbins;
};

// Bin of a particle by its distance to the nearer wall (binary32 decision), or -1.
__device__ __forceinline__ int wall_bin(const WallBins& B, float4 p) {
  const float x = B.axis == 0 ? p.x : (B.axis == 1 ? p.y : p.z);
  const float d = fminf(__fsub_rn(x, B.lo), __fsub_rn(B.hi, x));
  if (!(d >= 0.0f)) return -1;
  const float fb = floorf(__fmul_rn(d, B.inv_width));
  return fb < (float)B.nbins ? (int)fb : -1;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-point scale of the loss bins' velocity sums (|sum| < 2^39 per bin).  Integer
// atomics make the sums, and the loss, independent of the order the warps add in.
constexpr double kBinFix = 16777216.0;  // 2^24

// Forward loss statistics: per bin {count, sum vx} over fluid particles, as integers
// (the sum in units of 2^-24).
__global__ void __launch_bounds__(256) k_wall_profile(const float4* pos, const float4* vel, int n,
                                                      WallBins B, unsigned long long* acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool pending = false;
  int bin = 0;
  double vx = 0.0;
  if (i < n) {
    const float4 p = pos[i];
    if (!is_solid(p.w)) {
      bin = wall_bin(B, p);
      if (bin >= 0) {
        pending = true;
        vx = vel[i].x;
      }
    }
  }
  unsigned mask = __ballot_sync(0xffffffffu, pending);
  while (mask) {
    const int leader = __ffs(mask) - 1;
    const int b0 = __shfl_sync(0xffffffffu, bin, leader);
    const bool mine = pending && bin == b0;
    const unsigned c = __popc(__ballot_sync(0xffffffffu, mine));
    const double s = warp_sum_d(mine ? vx : 0.0);
    if (lane == leader) {
      atomicAdd(acc + 2 * b0, (unsigned long long)c);
      atomicAdd(acc + 2 * b0 + 1, (unsigned long long)__double2ll_rn(s * kBinFix));
    }
    if (mine) pending = false;
    mask = __ballot_sync(0xffffffffu, pending);
  }
}

// Predicted velocity of the window's first force evaluation: vt = v (v_wall for
// solid), no reflection flag.
__global__ void k_window_start(const float4* pos, const float4* vel, float4* vt, int n, float3 vw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 v = vel[i];
  vt[i] = is_solid(pos[i].w) ? make_float4(vw.x, vw.y, vw.z, 0.f) : make_float4(v.x, v.y, v.z, 0.f);
}

// Trilinear phase field and its gradient at a point (same node convention as phi_at).
__device__ __forceinline__ float phi_and_grad(const StepParams& P, float x, float y, float z, float3* g) {
  if (P.phi == nullptr) {
    *g = make_float3(0.f, 0.f, 0.f);
    return 1.0f;
  }
  const float sx = x * P.inv_h, sy = y * P.inv_h, sz = z * P.inv_h;
  const float fx = floorf(sx), fy = floorf(sy), fz = floorf(sz);
  const float tx = sx - fx, ty = sy - fy, tz = sz - fz;
  const int ix0 = wrap_node(__float2int_rd(fx), P.pd[0]), ix1 = wrap_node(__float2int_rd(fx) + 1, P.pd[0]);
  const int iy0 = wrap_node(__float2int_rd(fy), P.pd[1]), iy1 = wrap_node(__float2int_rd(fy) + 1, P.pd[1]);
  const int iz0 = wrap_node(__float2int_rd(fz), P.pd[2]), iz1 = wrap_node(__float2int_rd(fz) + 1, P.pd[2]);
  const long sy_ = P.pd[0];
  const long sz_ = (long)P.pd[0] * P.pd[1];
  const float* G = P.phi;
  const float c000 = G[iz0 * sz_ + iy0 * sy_ + ix0], c100 = G[iz0 * sz_ + iy0 * sy_ + ix1];
  const float c010 = G[iz0 * sz_ + iy1 * sy_ + ix0], c110 = G[iz0 * sz_ + iy1 * sy_ + ix1];
  const float c001 = G[iz1 * sz_ + iy0 * sy_ + ix0], c101 = G[iz1 * sz_ + iy0 * sy_ + ix1];
  const float c011 = G[iz1 * sz_ + iy1 * sy_ + ix0], c111 = G[iz1 * sz_ + iy1 * sy_ + ix1];
  const float ux = 1.f - tx, uy = 1.f - ty, uz = 1.f - tz;
  g->x = ((c100 - c000) * uy * uz + (c110 - c010) * ty * uz + (c101 - c001) * uy * tz +
          (c111 - c011) * ty * tz) * P.inv_h;
  g->y = ((c010 - c000) * ux * uz + (c110 - c100) * tx * uz + (c011 - c001) * ux * tz +
          (c111 - c101) * tx * tz) * P.inv_h;
  g->z = ((c001 - c000) * ux * uy + (c101 - c100) * tx * uy + (c011 - c010) * ux * ty +
          (c111 - c110) * tx * ty) * P.inv_h;
  const float c00 = c000 * ux + c100 * tx, c10 = c010 * ux + c110 * tx;
  const float c01 = c001 * ux + c101 * tx, c11 = c011 * ux + c111 * tx;
  return (c00 * uy + c10 * ty) * uz + (c01 * uy + c11 * ty) * tz;
}

// Adjoint of f(t+dt) = sum_j f_ij(r_ij, vt_ij) with the closing kick folded in.
//
// For target i the total adjoint of its new force is Fb_i = fbar_i + dt/2 vbar_i
// (the kick; reflected particles have no kick).  Because f_ji(-d, -u) = -f_ij(d, u)
// (symmetric noise), the adjoints of the new position and predicted velocity are
//   Rb_i = rbar_i + sum_j J_d(ij)^T (Fb_i - Fb_j),  Vb_i = sum_j J_u(ij)^T (Fb_i - Fb_j)
// (Fb_j = 0 for frozen j).  With f = m e, e = d / r, w = 1 - r, eu = e . u and
// m = w (a - gamma w eu + sigma' xi):
//   J_d^T G = m_r (e.G) e - gamma w^2 (e.G) (u - eu e) / r + m / r (G - (e.G) e)
//   J_u^T G = -gamma w^2 (e.G) e,     m_r = -a + 2 gamma w eu - sigma' xi.
// Parameter adjoints sum over ordered pairs with target i: d f_ij / d a_fs = w e
// (fluid-solid pairs), d f_ij / d gamma = -w^2 eu e + (kBT / sigma) w xi / sqrt(dt) e
// when sigma = sqrt(2 gamma kBT) is tied to gamma (Eq. 8).
// Four lanes per target: lane dz + 1 walks the nine neighbour cells of plane dz
// (dz = -1, 0, 1; the fourth lane idles), and the lanes' sums are combined with two
// shuffles.  The calibration windows are small (tens of thousands of particles), where
// one thread per target left ~5 warps per SM and the kernel waited on its loads.
constexpr int kAdjLanes = 4;
constexpr int kAdjList = 16;  // listed pairs per lane between evaluations

__global__ void __launch_bounds__(128)
k_adj_force(StepParams P, const float4* __restrict__ pos, const float4* __restrict__ vt,
            const uint32_t* __restrict__ start, int n, uint32_t step, const float4* __restrict__ rbar,
            const float4* __restrict__ vbar, const float4* __restrict__ fbar, float4* Rb, float4* Vb,
            float tie_coef, double* tpart) {
  __shared__ int alist[kAdjList][128];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / kAdjLanes, sub = t % kAdjLanes;
  double ta = 0.0, tg = 0.0;
  float Rx = 0.f, Ry = 0.f, Rz = 0.f, Ux = 0.f, Uy = 0.f, Uz = 0.f;
  bool target = false;
  if (i < n) {
    const float4 pi = pos[i];
    target = !is_solid(pi.w);
    if (target && sub < 3) {
      const float4 vti = vt[i];
      const uint32_t idi = id_of(pi.w);
      const float4 fbi = fbar[i], vbi = vbar[i];
      const float kick_i = vti.w == 0.0f ? P.half_dt : 0.0f;
      const float Fx = fbi.x + kick_i * vbi.x, Fy = fbi.y + kick_i * vbi.y, Fz = fbi.z + kick_i * vbi.z;
      if (sub == 1) {  // the target's own rbar, once
        const float4 rbi = rbar[i];
        Rx = rbi.x;
        Ry = rbi.y;
        Rz = rbi.z;
      }
      const int cx = cell_coord(pi.x, P.inv_edge[0], P.nc[0]);
      const int cy = cell_coord(pi.y, P.inv_edge[1], P.nc[1]);
      const int cz = cell_coord(pi.z, P.inv_edge[2], P.nc[2]);
      const int ncx = P.nc[0], ncy = P.nc[1], ncz = P.nc[2];
      // This lane's plane dz of the 27 cells, in the order dy, then dx, then each cell's
      // particles: rows of three cells are one range away from the x seam, single cells
      // on it.  Candidates are tested in rounds of four against the target shifted once
      // per range (a cut of 1 + 8 ulp(L) on r^2 covers that rounding) into a list; the
      // listed pairs are then evaluated in order with the exact minimum-image test, so
      // the pairs and the order of every sum are those of a cell-by-cell walk.
      const float r2cut = fmaf(8.0f * 0x1p-23f, fmaxf(P.L[0], fmaxf(P.L[1], P.L[2])), 1.0f);
      const int dz = sub - 1;
      const int z = wrap_node(cz + dz, ncz);
      const float uz = cz + dz < 0 ? pi.z + P.L[2] : (cz + dz >= ncz ? pi.z - P.L[2] : pi.z);
      const bool inner = cx > 0 && cx < ncx - 1;
      // axes on which some active lane has a range across the periodic seam; elsewhere
      // a listed pair's minimum-image separation is the plain difference
      const unsigned wm = __activemask();
      const bool wrap_x = __any_sync(wm, !inner);
      const bool wrap_y = __any_sync(wm, cy == 0 || cy == ncy - 1);
      const bool wrap_z = __any_sync(wm, cz + dz < 0 || cz + dz >= ncz);
      const int nseg = inner ? 3 : 9;
      int seg = 0, cnt = 0;
      uint32_t j = 0, e = 0;
      float ux = pi.x, uy = pi.y;
      bool more = true;
      for (;;) {
        while (cnt <= kAdjList - 4) {
          if (j == e) {
            if (seg == nseg) {
              more = false;
              break;
            }
            const int dy = (inner ? seg : seg / 3) - 1;
            const int y = wrap_node(cy + dy, ncy);
            uy = cy + dy < 0 ? pi.y + P.L[1] : (cy + dy >= ncy ? pi.y - P.L[1] : pi.y);
            const int row = (z * ncy + y) * ncx;
            if (inner) {
              j = start[row + cx - 1];
              e = start[row + cx + 2];
              ux = pi.x;
            } else {
              const int dx = seg % 3 - 1;
              const int x = wrap_node(cx + dx, ncx);
              ux = cx + dx < 0 ? pi.x + P.L[0] : (cx + dx >= ncx ? pi.x - P.L[0] : pi.x);
              j = start[row + x];
              e = start[row + x + 1];
            }
            ++seg;
          }
          const uint32_t m = min(e - j, 4u);
          if (m == 0u) continue;
          float4 q[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) q[u] = pos[min(j + (uint32_t)u, e - 1u)];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float ddx = ux - q[u].x, ddy = uy - q[u].y, ddz = uz - q[u].z;
            const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
            alist[cnt][threadIdx.x] = (int)(j + u);
            cnt += (u < (int)m) & (r2 < r2cut) & (r2 > 0.0f);
          }
          j += m;
        }
        for (int k = 0; k < cnt; ++k) {
          const uint32_t j = (uint32_t)alist[k][threadIdx.x];
          const float4 pj = pos[j];
          const float ddx = wrap_x ? min_image(pi.x, pj.x, P.L[0], P.halfL[0]) : pi.x - pj.x;
          const float ddy = wrap_y ? min_image(pi.y, pj.y, P.L[1], P.halfL[1]) : pi.y - pj.y;
          const float ddz = wrap_z ? min_image(pi.z, pj.z, P.L[2], P.halfL[2]) : pi.z - pj.z;
          const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
          if (!(r2 < 1.0f && r2 > 0.0f)) continue;
          const float inv_r = rsqrtf(r2);
          const float r = r2 * inv_r;
          const float w = 1.0f - r;
          const float ex = ddx * inv_r, ey = ddy * inv_r, ez = ddz * inv_r;
          const bool solid_j = is_solid(pj.w);
          float ujx, ujy, ujz, a, Gx = Fx, Gy = Fy, Gz = Fz;
          if (solid_j) {
            ujx = P.vw[0]; ujy = P.vw[1]; ujz = P.vw[2];
            a = P.a_fs;
          } else {
            const float4 vtj = vt[j];
            ujx = vtj.x; ujy = vtj.y; ujz = vtj.z;
            a = P.a_ff;
            const float4 fbj = fbar[j], vbj = vbar[j];
            const float kick_j = vtj.w == 0.0f ? P.half_dt : 0.0f;
            Gx -= fbj.x + kick_j * vbj.x;
            Gy -= fbj.y + kick_j * vbj.y;
            Gz -= fbj.z + kick_j * vbj.z;
          }
          const float ux = vti.x - ujx, uy = vti.y - ujy, uz = vti.z - ujz;
          const float eu = ex * ux + ey * uy + ez * uz;
          const float xi = pair_noise(idi, id_of(pj.w), step, P.sys, P.rkey);
          const float m = w * (a - P.gamma * w * eu + P.sigma_rsqdt * xi);
          const float m_r = -a + 2.0f * P.gamma * w * eu - P.sigma_rsqdt * xi;
          const float eG = ex * Gx + ey * Gy + ez * Gz;
          const float gw2 = P.gamma * w * w;
          const float cu = -gw2 * eG * inv_r;
          const float cm = m * inv_r;
          Rx += m_r * eG * ex + cu * (ux - eu * ex) + cm * (Gx - eG * ex);
          Ry += m_r * eG * ey + cu * (uy - eu * ey) + cm * (Gy - eG * ey);
          Rz += m_r * eG * ez + cu * (uz - eu * ez) + cm * (Gz - eG * ez);
          Ux -= gw2 * eG * ex;
          Uy -= gw2 * eG * ey;
          Uz -= gw2 * eG * ez;
          const float eF = ex * Fx + ey * Fy + ez * Fz;
          if (solid_j) ta += (double)(w * eF);
          tg += (double)((-w * w * eu + tie_coef * w * xi) * eF);
        }
        if (!more) break;
        cnt = 0;
      }
    }
  }
  // the target's four lanes are adjacent: add their sums (every lane takes part)
#pragma unroll
  for (int o = 1; o < kAdjLanes; o <<= 1) {
    Rx += __shfl_xor_sync(0xffffffffu, Rx, o);
    Ry += __shfl_xor_sync(0xffffffffu, Ry, o);
    Rz += __shfl_xor_sync(0xffffffffu, Rz, o);
    Ux += __shfl_xor_sync(0xffffffffu, Ux, o);
    Uy += __shfl_xor_sync(0xffffffffu, Uy, o);
    Uz += __shfl_xor_sync(0xffffffffu, Uz, o);
  }
  if (i < n && sub == 0) {
    Rb[i] = target ? make_float4(Rx, Ry, Rz, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    Vb[i] = target ? make_float4(Ux, Uy, Uz, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // each warp adds to its own slot (launches on one stream follow one another, so no
  // two writers meet); k_theta_sum adds the slots in a fixed order
  ta = warp_sum_d(ta);
  tg = warp_sum_d(tg);
  if ((threadIdx.x & 31) == 0) {
    const int w = t >> 5;
    tpart[2 * w] += ta;
    tpart[2 * w + 1] += tg;
  }
}

// Adjoint of the drift, predicted velocity and reflection of one step, from the
// new cell order (index d) back to the previous one (o = perm[d]), plus the loss
// seed at the previous state.
__global__ void __launch_bounds__(256)
k_adj_integrate(StepParams P, const float4* __restrict__ pos_old, const float4* __restrict__ vel_old,
                const float4* __restrict__ frc_old, const float4* __restrict__ pos_new,
                const float4* __restrict__ vt_new, const uint32_t* __restrict__ perm, int n,
                const float4* __restrict__ Rb, const float4* __restrict__ Vb,
                const float4* __restrict__ vbar_new, float4* rbar_old, float4* vbar_old,
                float4* fbar_old, WallBins B, const float* __restrict__ seed_coef, double* tpart) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  double tgx = 0.0;
  if (d < n) {
    const uint32_t o = min(perm[d], (uint32_t)(n - 1));
    const float4 p = pos_old[o];
    float4 rb = make_float4(0.f, 0.f, 0.f, 0.f), vb = rb, fb = rb;
    if (!is_solid(p.w)) {
      const float4 R = Rb[d], U = Vb[d], Vn = vbar_new[d];
      const bool refl = vt_new[d].w != 0.0f;
      if (!refl) {
        rb = make_float4(R.x, R.y, R.z, 0.f);
        vb = make_float4(Vn.x + P.dt * R.x + U.x, Vn.y + P.dt * R.y + U.y, Vn.z + P.dt * R.z + U.z, 0.f);
        fb = make_float4(P.half_dt * Vn.x + P.half_dt2 * R.x + P.lam_dt * U.x,
                         P.half_dt * Vn.y + P.half_dt2 * R.y + P.lam_dt * U.y,
                         P.half_dt * Vn.z + P.half_dt2 * R.z + P.lam_dt * U.z, 0.f);
        tgx = (double)(P.dt * Vn.x + P.half_dt2 * R.x + P.lam_dt * U.x);
      } else {
        const float4 pn = pos_new[d];
        const bool fallback = pn.x == p.x && pn.y == p.y && pn.z == p.z;
        vb = make_float4(-Vn.x - U.x, -Vn.y - U.y, -Vn.z - U.z, 0.f);
        rb = make_float4(R.x, R.y, R.z, 0.f);
        if (!fallback) {
          const float4 v = vel_old[o], f = frc_old[o];
          const float drx = fmaf(P.half_dt2, f.x + P.g[0], P.dt * v.x);
          const float dry = fmaf(P.half_dt2, f.y + P.g[1], P.dt * v.y);
          const float drz = fmaf(P.half_dt2, f.z + P.g[2], P.dt * v.z);
          float3 gn, go;
          const float phn = phi_and_grad(P, p.x + drx, p.y + dry, p.z + drz, &gn);
          const float pho = phi_and_grad(P, p.x, p.y, p.z, &go);
          const float lim = 0.999999f;
          const float pnc = fminf(fmaxf(phn, -lim), lim), poc = fminf(fmaxf(fmaxf(pho, 0.f), -lim), lim);
          const float A = atanhf(-pnc), Bv = atanhf(poc);
          const float s = A / (A + Bv);
          const float sb = -2.0f * (drx * R.x + dry * R.y + drz * R.z);
          const float den = (A + Bv) * (A + Bv);
          const float Ab = sb * Bv / den, Bb = -sb * A / den;
          const float pnb = (fabsf(phn) < lim) ? -Ab / (1.0f - phn * phn) : 0.0f;
          const float pob = (pho > 0.0f && pho < lim) ? Bb / (1.0f - pho * pho) : 0.0f;
          float dbx = (1.0f - 2.0f * s) * R.x + pnb * gn.x;
          float dby = (1.0f - 2.0f * s) * R.y + pnb * gn.y;
          float dbz = (1.0f - 2.0f * s) * R.z + pnb * gn.z;
          rb.x += pnb * gn.x + pob * go.x;
          rb.y += pnb * gn.y + pob * go.y;
          rb.z += pnb * gn.z + pob * go.z;
          vb.x += P.dt * dbx;
          vb.y += P.dt * dby;
          vb.z += P.dt * dbz;
          fb = make_float4(P.half_dt2 * dbx, P.half_dt2 * dby, P.half_dt2 * dbz, 0.f);
          tgx = (double)(P.half_dt2 * dbx);
        }
      }
      if (seed_coef) {
        const int b = wall_bin(B, p);
        if (b >= 0) vb.x += seed_coef[b];
      }
    }
    rbar_old[o] = rb;
    vbar_old[o] = vb;
    fbar_old[o] = fb;
  }
  tgx = warp_sum_d(tgx);
  if ((threadIdx.x & 31) == 0) tpart[d >> 5] += tgx;
}

// theta = (sum of the a_fs and gamma slots of k_adj_force, sum of the g_x slots of
// k_adj_integrate), added in a fixed order: the gradient has the same bits from run to
// run.  One block of kThetaThreads threads.
constexpr int kThetaThreads = 256;
__global__ void __launch_bounds__(kThetaThreads)
k_theta_sum(const double* __restrict__ tpart_f, int nw_f, const double* __restrict__ tpart_i,
            int nw_i, double* out) {
  __shared__ double sh[3][kThetaThreads];
  double a = 0.0, g = 0.0, x = 0.0;
  for (int w = threadIdx.x; w < nw_f; w += kThetaThreads) {
    a += tpart_f[2 * w];
    g += tpart_f[2 * w + 1];
  }
  for (int w = threadIdx.x; w < nw_i; w += kThetaThreads) x += tpart_i[w];
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = g;
  sh[2][threadIdx.x] = x;
  __syncthreads();
  for (int o = kThetaThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = sh[threadIdx.x][0];
}

// Loss seed at the window's last state (same order as the state).
__global__ void k_seed(const float4* pos, int n, WallBins B, const float* coef, float4* vbar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = pos[i];
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!is_solid(p.w)) {
    const int b = wall_bin(B, p);
    if (b >= 0) v.x = coef[b];
  }
  vbar[i] = v;
}

// Three per-particle arrays of one state (in that state's cell order) into id order:
// out[12 id .. 12 id + 11] = a[i], b[i], c[i], ids from the tags of key_pos.
__global__ void k_unsort3(const float4* __restrict__ key_pos, const float4* __restrict__ a,
                          const float4* __restrict__ b, const float4* __restrict__ c, int n,
                          float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t id = id_of(key_pos[i].w);
  if (id >= (uint32_t)n) return;
  out[3 * (size_t)id + 0] = a[i];
  out[3 * (size_t)id + 1] = b[i];
  out[3 * (size_t)id + 2] = c[i];
}

// The record of one step in one launch: the four state arrays, the sort permutation
// and the cell starts, copied to the step's slot of the record.
__global__ void k_record(Arrays src, Arrays dst, const uint32_t* __restrict__ perm,
                         uint32_t* __restrict__ perm_dst, const uint32_t* __restrict__ start,
                         uint32_t* __restrict__ start_dst, int n, int nstart) {
  const int m = n > nstart ? n : nstart;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
    if (q < n) {
      dst.pos[q] = src.pos[q];
      dst.vt[q] = src.vt[q];
      dst.vel[q] = src.vel[q];
      dst.frc[q] = src.frc[q];
      perm_dst[q] = perm[q];
    }
    if (q < nstart) start_dst[q] = start[q];
  }
}

// Carves the adjoint's arrays out of one workspace, each on a 256-byte boundary.  With
// no base it only adds up the bytes (the sizing pass).
struct Carve {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  void alloc(T** p, size_t count) {
    *p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += (sizeof(T) * (count > 0 ? count : 1) + 255) & ~(size_t)255;
  }
};

int afail(dpd_system* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  h->err = buf;
  return code;
}

#define ACU(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return afail(h, DPD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
  } while (0)

inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace
}  // namespace dpd

using dpd::Arrays;
using dpd::DevCounters;

namespace {
// Where dpd_adjoint_window_record puts its record (host memory, entries may be NULL).
struct AdjointRecord {
  float* ckpt;
  float* adj;
  double* seg_grad;
  float* coef;
  uint32_t* seg_step;
};
}  // namespace

static int adjoint_window(dpd_t* h, int nsteps, int ckpt_every, int axis, double wall_lo,
                          double wall_hi, int nbins, double bin_width, const double* target,
                          int tie_sigma, double* loss_out, double grad[3], const AdjointRecord* rec) {
  using namespace dpd;
  if (!h || !target || !grad) return DPD_EINVAL;
  if (!h->loaded) return afail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  if (nsteps < 1 || ckpt_every < 1 || nsteps % ckpt_every != 0)
    return afail(h, DPD_EINVAL, "nsteps must be a positive multiple of ckpt_every");
  if (axis < 0 || axis > 2 || !(wall_hi > wall_lo) || nbins < 1 || nbins > 1024 || !(bin_width > 0))
    return afail(h, DPD_EINVAL, "bad loss layout");
  if (h->reflect_variant != 0) return afail(h, DPD_EINVAL, "the adjoint supports reflect_variant 0");
  if (h->force_law != 0) return afail(h, DPD_EINVAL, "the adjoint supports force_law 0");
  if (h->shear[0] != 0.0 || h->shear[1] != 0.0 || h->shear[2] != 0.0)
    return afail(h, DPD_EINVAL, "the adjoint supports walls moving together (shear 0)");
  if (tie_sigma && !(h->kBT > 0.0 && h->gamma > 0.0))
    return afail(h, DPD_EINVAL, "tying sigma to gamma needs kBT > 0 and gamma > 0");
  Engine& E = h->E;
  if (E.h_ctr[0].status) return engine_status_code(E, E.h_ctr[0].status);
  // the window records complete states (force in frc, velocity kicked) after every
  // step: steps here run their finish pass
  engine_settle(E);
  // Eq. 8, sigma^2 = 2 gamma kBT: the forward window runs with the sigma that the
  // gradient assumes (the system keeps it)
  if (tie_sigma) h->sigma = std::sqrt(2.0 * h->gamma * h->kBT);
  h->params_dirty = true;
  {
    // parameters as set now
    E.h_sys.resize(1);
    E.h_sys[0].P = make_params(h);
    E.h_sys[0].cell_off = 0;
    E.h_sys[0].part_off = 0;
    E.h_sys[0].n = (uint32_t)E.n;
    const int rc = engine_upload_sys(E);
    if (rc) return rc;
    h->params_dirty = false;
  }
  engine_free_graphs(E);
  const StepParams P = E.h_sys[0].P;
  const int n = E.n;
  const int K = ckpt_every, nseg = nsteps / K;
  const size_t nf4 = sizeof(float4) * (size_t)n;
  cudaStream_t st = E.stream;
  WallBins B;
  B.axis = axis;
  B.lo = (float)wall_lo;
  B.hi = (float)wall_hi;
  B.inv_width = (float)(1.0 / bin_width);
  B.nbins = nbins;

  // The record of the steps the reverse pass walks: every state (four arrays), and every
  // step's sort permutation and cell starts.  When the whole window's record fits the
  // budget (option "adjoint_tape_mb") the forward pass keeps it and nothing is recomputed;
  // otherwise the forward pass keeps a checkpoint every K steps and the reverse pass
  // recomputes one segment at a time into a record of K steps.  Both give the same bits.
  const size_t state_bytes = 4 * nf4;
  const size_t step_bytes = sizeof(uint32_t) * ((size_t)n + (size_t)E.ncells + 1);
  const bool whole = (double)((size_t)(nsteps + 1) * state_bytes + (size_t)nsteps * step_bytes) <=
                     h->adjoint_tape_mb * 1048576.0;
  const int T = whole ? nsteps : K;
  std::vector<Arrays> tape(T + 1);
  std::vector<uint32_t*> tperm(T), tstart(T);
  // checkpoints: the four state arrays of each segment start, plus the final state
  std::vector<Arrays> ck(nseg + 1);
  float4 *rb[2], *vb[2], *fb[2], *Rb, *Vb, *zero4;
  unsigned long long* acc;
  // per-warp parameter sums of k_adj_force (two each) and k_adj_integrate (one each), and
  // theta after the reversal of each segment (index seg; index 0 after the window start)
  const int nw_f = nblk((long)n * kAdjLanes, 128) * 4, nw_i = nblk(n, 256) * 8;
  double *tpart_f, *tpart_i, *tsnap;
  float* coef;
  uint32_t *start0, *start_end;  // cell starts of the first and last state of the window
  float4* stage = nullptr;       // id-ordered copy of three per-particle arrays (record API)
  const size_t start_bytes = sizeof(uint32_t) * ((size_t)E.ncells + 1);
  auto layout = [&](Carve& c) {
    for (auto& A : tape) {
      c.alloc(&A.pos, n);
      c.alloc(&A.vt, n);
      c.alloc(&A.vel, n);
      c.alloc(&A.frc, n);
    }
    for (int k = 0; k < T; ++k) {
      c.alloc(&tperm[k], n);
      c.alloc(&tstart[k], (size_t)E.ncells + 1);
    }
    for (int q2 = 0; q2 <= nseg; ++q2) {
      if (whole) {
        ck[q2] = tape[q2 * K];
        continue;
      }
      Arrays& A = ck[q2];
      c.alloc(&A.pos, n);
      c.alloc(&A.vt, n);
      c.alloc(&A.vel, n);
      c.alloc(&A.frc, n);
    }
    for (int q = 0; q < 2; ++q) {
      c.alloc(&rb[q], n);
      c.alloc(&vb[q], n);
      c.alloc(&fb[q], n);
    }
    c.alloc(&Rb, n);
    c.alloc(&Vb, n);
    c.alloc(&zero4, n);
    c.alloc(&start0, (size_t)E.ncells + 1);
    c.alloc(&start_end, (size_t)E.ncells + 1);
    c.alloc(&acc, 2 * (size_t)nbins);
    c.alloc(&tpart_f, 2 * (size_t)nw_f);
    c.alloc(&tpart_i, (size_t)nw_i);
    c.alloc(&tsnap, 3 * (size_t)(nseg + 1));
    c.alloc(&coef, nbins);
    if (rec) c.alloc(&stage, 3 * (size_t)n);
  };
  {
    Carve sizing;
    layout(sizing);
    if (sizing.off > h->adj_ws_bytes) {
      cudaFree(h->d_adj_ws);
      h->d_adj_ws = nullptr;
      h->adj_ws_bytes = 0;
      ACU(cudaMalloc(&h->d_adj_ws, sizing.off));
      h->adj_ws_bytes = sizing.off;
    }
    Carve c;
    c.base = static_cast<char*>(h->d_adj_ws);
    layout(c);
  }
  DevCounters ctr0, ctr_end;

  auto copy_state = [&](const Arrays& dst, const Arrays& src) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(dst.pos, src.pos, nf4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst.vt, src.vt, nf4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst.vel, src.vel, nf4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst.frc, src.frc, nf4, cudaMemcpyDeviceToDevice, st);
    return e;
  };

  // ---- forward window ------------------------------------------------------
  ACU(cudaMemcpyAsync(&ctr0, E.d_ctr, sizeof ctr0, cudaMemcpyDeviceToHost, st));
  ACU(cudaStreamSynchronize(st));
  const uint32_t step0 = ctr0.step;
  // f(0) at the window start, with the current parameters and vt = v(0)
  {
    const Arrays& A = E.arr[E.cur];
    k_window_start<<<nblk(n, 256), 256, 0, st>>>(A.pos, A.vel, A.vt, n,
                                                 make_float3(P.vw[0], P.vw[1], P.vw[2]));
    engine_enqueue_force(E, 0);
  }
  ACU(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 2 * nbins, st));
  ACU(copy_state(ck[0], E.arr[E.cur]));
  ACU(cudaMemcpyAsync(start0, E.cl.start, start_bytes, cudaMemcpyDeviceToDevice, st));
  for (int s = 1; s <= nsteps; ++s) {
    engine_enqueue_step(E, true);
    const Arrays& A = E.arr[E.cur];
    k_wall_profile<<<nblk(n, 256), 256, 0, st>>>(A.pos, A.vel, n, B, acc);
    if (whole) {  // the record of step s (ck[] points into it)
      const int m = n > E.ncells + 1 ? n : E.ncells + 1;
      k_record<<<nblk(m, 256), 256, 0, st>>>(A, tape[s], E.cl.perm, tperm[s - 1], E.cl.start,
                                             tstart[s - 1], n, E.ncells + 1);
    } else if (s % K == 0) {
      ACU(copy_state(ck[s / K], A));
    }
  }
  ACU(cudaGetLastError());
  ACU(cudaMemcpyAsync(start_end, E.cl.start, start_bytes, cudaMemcpyDeviceToDevice, st));
  std::vector<unsigned long long> hacc(2 * nbins);
  ACU(cudaMemcpyAsync(hacc.data(), acc, sizeof(unsigned long long) * 2 * nbins, cudaMemcpyDeviceToHost, st));
  ACU(cudaMemcpyAsync(&ctr_end, E.d_ctr, sizeof ctr_end, cudaMemcpyDeviceToHost, st));
  ACU(cudaStreamSynchronize(st));
  if (ctr_end.status) return engine_status_code(E, ctr_end.status);
  // loss L = sum_b (u_b - target_b)^2 with u_b the mean vx of bin b over the window
  double L = 0.0;
  std::vector<float> hcoef(nbins, 0.0f);
  for (int b = 0; b < nbins; ++b) {
    const double cnt = (double)hacc[2 * b];
    if (cnt <= 0) continue;
    const double u = (double)(long long)hacc[2 * b + 1] / kBinFix / cnt;
    L += (u - target[b]) * (u - target[b]);
    hcoef[b] = (float)(2.0 * (u - target[b]) / cnt);
  }
  ACU(cudaMemcpyAsync(coef, hcoef.data(), sizeof(float) * nbins, cudaMemcpyHostToDevice, st));
  const size_t rec_floats = (size_t)12 * n;
  if (rec) {
    if (rec->coef) memcpy(rec->coef, hcoef.data(), sizeof(float) * nbins);
    if (rec->seg_step)
      for (int q2 = 0; q2 <= nseg; ++q2) rec->seg_step[q2] = step0 + (uint32_t)(q2 * K);
    if (rec->ckpt)
      for (int q2 = 0; q2 <= nseg; ++q2) {
        k_unsort3<<<nblk(n, 256), 256, 0, st>>>(ck[q2].pos, ck[q2].pos, ck[q2].vel, ck[q2].frc, n, stage);
        ACU(cudaMemcpyAsync(rec->ckpt + q2 * rec_floats, stage, sizeof(float) * rec_floats,
                            cudaMemcpyDeviceToHost, st));
      }
  }
  ACU(cudaMemsetAsync(tpart_f, 0, sizeof(double) * 2 * (size_t)nw_f, st));
  ACU(cudaMemsetAsync(tpart_i, 0, sizeof(double) * (size_t)nw_i, st));
  ACU(cudaMemsetAsync(zero4, 0, nf4, st));

  // ---- backward --------------------------------------------------------------
  // adjoints of the last state: vbar from the loss, rbar = fbar = 0
  int q = 0;
  k_seed<<<nblk(n, 256), 256, 0, st>>>(ck[nseg].pos, n, B, coef, vb[q]);
  ACU(cudaMemsetAsync(rb[q], 0, nf4, st));
  ACU(cudaMemsetAsync(fb[q], 0, nf4, st));
  const float tie = tie_sigma ? (float)(h->kBT / h->sigma / std::sqrt(h->dt)) : 0.0f;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    if (rec && rec->adj) {
      // the adjoint of the segment's end state (it includes that state's own loss term)
      k_unsort3<<<nblk(n, 256), 256, 0, st>>>(ck[seg + 1].pos, rb[q], vb[q], fb[q], n, stage);
      ACU(cudaMemcpyAsync(rec->adj + (size_t)(seg + 1) * rec_floats, stage, sizeof(float) * rec_floats,
                          cudaMemcpyDeviceToHost, st));
    }
    const uint32_t seg_step = step0 + (uint32_t)(seg * K);
    const int base = whole ? seg * K : 0;  // the segment's first step in the record
    if (!whole) {
      // recompute the segment, recording every step
      ACU(copy_state(E.arr[E.cur], ck[seg]));
      ACU(cudaMemcpyAsync(&E.d_ctr[0].step, &seg_step, sizeof seg_step, cudaMemcpyHostToDevice, st));
      ACU(copy_state(tape[0], ck[seg]));
      for (int k = 0; k < K; ++k) {
        engine_enqueue_step(E, true);
        const int m = n > E.ncells + 1 ? n : E.ncells + 1;
        k_record<<<nblk(m, 256), 256, 0, st>>>(E.arr[E.cur], tape[k + 1], E.cl.perm, tperm[k],
                                               E.cl.start, tstart[k], n, E.ncells + 1);
      }
    }
    // reverse through the recorded steps
    for (int k = K - 1; k >= 0; --k) {
      const uint32_t step_new = seg_step + (uint32_t)k + 1;
      const Arrays& An = tape[base + k + 1];
      const Arrays& Ao = tape[base + k];
      k_adj_force<<<nblk((long)n * kAdjLanes, 128), 128, 0, st>>>(P, An.pos, An.vt, tstart[base + k], n, step_new, rb[q],
                                                vb[q], fb[q], Rb, Vb, tie, tpart_f);
      const int s_old = seg * K + k;  // global index of the previous state
      k_adj_integrate<<<nblk(n, 256), 256, 0, st>>>(P, Ao.pos, Ao.vel, Ao.frc, An.pos, An.vt,
                                                    tperm[base + k], n, Rb, Vb, vb[q], rb[q ^ 1],
                                                    vb[q ^ 1], fb[q ^ 1], B, s_old >= 1 ? coef : nullptr,
                                                    tpart_i);
      q ^= 1;
    }
    if (rec && rec->seg_grad && seg > 0)
      k_theta_sum<<<1, kThetaThreads, 0, st>>>(tpart_f, nw_f, tpart_i, nw_i, tsnap + 3 * seg);
  }
  if (rec && rec->adj) {
    k_unsort3<<<nblk(n, 256), 256, 0, st>>>(ck[0].pos, rb[q], vb[q], fb[q], n, stage);
    ACU(cudaMemcpyAsync(rec->adj, stage, sizeof(float) * rec_floats, cudaMemcpyDeviceToHost, st));
  }
  // f(0) = f(r0, v0): its parameter dependence, with F-bar = fbar(0) (no kick)
  {
    const Arrays& A0 = ck[0];
    k_adj_force<<<nblk((long)n * kAdjLanes, 128), 128, 0, st>>>(P, A0.pos, A0.vt, start0, n, step0, zero4, zero4,
                                              fb[q], Rb, Vb, tie, tpart_f);
  }
  k_theta_sum<<<1, kThetaThreads, 0, st>>>(tpart_f, nw_f, tpart_i, nw_i, tsnap);
  ACU(cudaGetLastError());
  std::vector<double> theta_snap(3 * (size_t)(nseg + 1), 0.0);
  const size_t nsnap = (rec && rec->seg_grad) ? 3 * (size_t)nseg : 3;
  ACU(cudaMemcpyAsync(theta_snap.data(), tsnap, sizeof(double) * nsnap, cudaMemcpyDeviceToHost, st));
  const double* th = theta_snap.data();
  // recomputed segments repeat steps the forward window ran without error; a status
  // set now would mean the record and the state disagree
  DevCounters ctr_bwd;
  ACU(cudaMemcpyAsync(&ctr_bwd, E.d_ctr, sizeof ctr_bwd, cudaMemcpyDeviceToHost, st));
  ACU(cudaStreamSynchronize(st));
  if (ctr_bwd.status) return engine_status_code(E, ctr_bwd.status);
  // ---- leave the system at the end of the window, as dpd_step would ----------
  ACU(copy_state(E.arr[E.cur], ck[nseg]));
  ACU(cudaMemcpyAsync(E.cl.start, start_end, start_bytes, cudaMemcpyDeviceToDevice, st));
  ACU(cudaMemcpyAsync(E.d_ctr, &ctr_end, sizeof ctr_end, cudaMemcpyHostToDevice, st));
  ACU(cudaStreamSynchronize(st));
  E.h_ctr[0] = ctr_end;
  h->host_step = ctr_end.step;
  // the parameter gradient: a_fs, gamma (sigma tied if requested), g_x
  grad[0] = th[0];
  grad[1] = th[1];
  grad[2] = th[2];
  if (rec && rec->seg_grad) {
    // segment k's share: theta accumulated while reversing it (segment 0 also holds
    // the dependence of f(0) on the parameters); snapshots were taken after the
    // reversal of segments nseg-1 .. 1
    for (int seg = 0; seg < nseg; ++seg) {
      const double* after = &theta_snap[3 * (size_t)seg];
      const double* before = &theta_snap[3 * (size_t)(seg + 1)];
      for (int k2 = 0; k2 < 3; ++k2) rec->seg_grad[3 * seg + k2] = after[k2] - before[k2];
    }
  }
  if (loss_out) *loss_out = L;
  return DPD_OK;
}

extern "C" int dpd_adjoint_window(dpd_t* h, int nsteps, int ckpt_every, int axis, double wall_lo,
                                  double wall_hi, int nbins, double bin_width, const double* target,
                                  int tie_sigma, double* loss_out, double grad[3]) {
  return adjoint_window(h, nsteps, ckpt_every, axis, wall_lo, wall_hi, nbins, bin_width, target,
                        tie_sigma, loss_out, grad, nullptr);
}

extern "C" int dpd_adjoint_window_record(dpd_t* h, int nsteps, int ckpt_every, int axis,
                                         double wall_lo, double wall_hi, int nbins, double bin_width,
                                         const double* target, int tie_sigma, double* loss_out,
                                         double grad[3], float* ckpt, float* adj, double* seg_grad,
                                         float* coef, uint32_t* seg_step) {
  const AdjointRecord rec{ckpt, adj, seg_grad, coef, seg_step};
  return adjoint_window(h, nsteps, ckpt_every, axis, wall_lo, wall_hi, nbins, bin_width, target,
                        tie_sigma, loss_out, grad, &rec);
}
