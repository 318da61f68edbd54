/*
 * dpd_oracle.c -- plain, slow, FP64 CPU oracle for one time step of
 * dissipative particle dynamics (DPD) with phase-field no-slip walls,
 * after Xu & Meakin, "A phase field approach to no slip boundary conditions
 * in dissipative particle dynamics and other particle models for fluid flow
 * in geometrically complex confined systems" (arXiv:1807.09896).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, link or
 * call this file.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA library; the two meet only through the seeded input generators.
 *
 * What it restates, each function citing the passage it follows:
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), and the
 *     Box-Muller transform, to draw the pair noise xi_ij of Eq. 7.
 *   - The pair force of Eqs. 3-10 (conservative, dissipative, random).
 *   - The Groot-Warren modified velocity-Verlet step the paper uses (Sec. II.A,
 *     ref. 35).
 *   - The bounce-back reflection at the phi = 0 surface, located with the
 *     interpolated phase field (Sec. II.C, Eqs. 16-17, Fig. 4).
 *   - Per-bin velocity profile sums (Sec. III.A).
 *
 * Readings where the paper is silent or garbled (each is listed with its
 * reason in the design notes of the repository):
 *   R1  distances from phi use atanh (the inverse of Eq. 14), as the text
 *       around Eq. 17 does; Eq. 16 prints tanh.
 *   R2  Eq. 17's displacement v^t dt is read as the actual drift of the
 *       step, dr = r(t+dt) - r(t) (identical when the force is zero);
 *       reflect_variant = 1 uses v^t dt literally.
 *   R3  a reflected particle leaves the step with v = 2 v_wall - v(t); its
 *       closing half-kick is skipped and its predicted velocity for the new
 *       force is that reversed velocity.
 *   R4  the discrete random force is sigma w_R xi / sqrt(dt).
 *   R5  the reflection test is strict (phi < 0); phi arguments of atanh are
 *       clamped to [-1+1e-6, 1-1e-6]; phi(t) below zero is taken as zero in
 *       the crossing fraction.  If the reflected point still has phi < 0 the
 *       particle goes back to r(t) (fallback), keeping the reversed velocity.
 *   R6  phase field nodes sit at (i, j, k) * h, periodic in every axis, x
 *       fastest in memory; the particle value is trilinear interpolation
 *       (the 3-D form of the paper's "linear interpolation").
 *   R7  pair noise: counter (min id, max id, step, system), key (seed low
 *       word, seed high word); u = ((x >> 9) + 0.5) * 2^-23 from output words
 *       0 and 1; xi = sqrt(-2 ln u0) cos(2 pi u1).
 *   R8  pairs at exactly zero separation contribute nothing (no direction).
 *   R9  solid particles are frozen: they get no force and enter the dissipative
 *       term with velocity v_wall.
 *   R14 a moving wall is a translating solid (Sec. II.C, Couette flow): its
 *       frozen particles move rigidly with it, r += dt v_wall each step (with
 *       v_wall = 0 they never move).
 *   R18 walls may move at different velocities (plane Couette flow): the wall
 *       velocity is the field v_w(r) = v_wall + d S, d the signed distance of
 *       r from the plane r_axis = ref, wrapped into [-L_axis/2, L_axis/2), and
 *       S = d v_w / d r_axis with no component along the axis (the walls
 *       slide in their planes).  A frozen particle moves with v_w at its own
 *       position; a reflected particle leaves with 2 v_w - v, v_w taken at
 *       the crossing point r + (1 - s) dr of Eq. 17.  S = 0 gives R14.
 *   R19 Eq. 24 as printed adds +W' rhat; W' < 0, so the term named repulsive
 *       would attract.  The force is read as minus the derivative of the
 *       energy of Eq. 22, f_i = -sum_j [S^r W'(r^r) - S^a W'(r^a)] rhat_ij,
 *       rhat_ij pointing from j to i.  Fluid-solid pairs use their own
 *       strengths (the paper doubles the fluid-fluid ones); the dissipative
 *       and random parts keep the weights of Eqs. 5-8 with r_c = 1, so both
 *       ranges must be <= 1.
 *   R20 set-up (Sec. II.C): a dense random fluid at the density rho fills the
 *       box, and the phase field classifies it -- fluid where phi >= 0, frozen
 *       solid where phi_min < phi < 0, removed deeper; phi_min is the value of
 *       Eq. 14 at the chosen solid-layer depth.  Positions and velocities come
 *       from Philox4x32-10 streams disjoint from the pair noise.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Parameters, passed from Python as one flat double array.            */
/* ------------------------------------------------------------------ */
enum {
  P_LX, P_LY, P_LZ,          /* periodic box */
  P_AFF, P_AFS, P_ASF, P_ASS,/* a_ij by (type_i, type_j), Eq. 4 */
  P_GAMMA, P_SIGMA, P_KBT,   /* Eqs. 6-8 */
  P_DT, P_LAMBDA,            /* time step and Groot-Warren lambda */
  P_GX, P_GY, P_GZ,          /* body force on fluid particles (Sec. III.A) */
  P_VWX, P_VWY, P_VWZ,       /* wall velocity (Sec. II.C) */
  P_REFLECT_VARIANT,
  P_SHX, P_SHY, P_SHZ,       /* wall shear: d v_wall / d r_axis (reading R18) */
  P_SHAXIS, P_SHREF,         /* its gradient axis and the plane where v_w = v_wall */
  P_FORCE_LAW,               /* 0: Eq. 4 soft repulsion; 1: Eqs. 22-24 */
  P_SR_FF, P_SA_FF,          /* S^r, S^a fluid-fluid (Eq. 22) */
  P_SR_FS, P_SA_FS,          /* S^r, S^a fluid-solid */
  P_R0R, P_R0A,              /* r0^r, r0^a */
  P_SPH_DIM,                 /* D of Eq. 23 */
  P_COUNT
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).                               */
/* One round: two 32x32->64 products of counter words 0 and 2 with the  */
/* round multipliers; the new counter is                                */
/*   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)).  */
/* Between rounds the key is bumped by the Weyl constants.              */
/* ------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (round < 9) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0, 1) from one 32-bit word, reading R7. */
double or_u01(uint32_t x) {
  return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Gaussian pair noise xi_ij of Eq. 7: independent per pair and per step and
 * symmetric in i <-> j (reading R7). */
double or_xi(uint32_t id_a, uint32_t id_b, uint32_t step, uint32_t sys, uint64_t seed) {
  uint32_t lo = id_a < id_b ? id_a : id_b;
  uint32_t hi = id_a < id_b ? id_b : id_a;
  uint32_t ctr[4] = {lo, hi, step, sys};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  or_philox4x32_10(ctr, key, w);
  double u0 = or_u01(w[0]);
  double u1 = or_u01(w[1]);
  return sqrt(-2.0 * log(u0)) * cos(2.0 * M_PI * u1);
}

/* ------------------------------------------------------------------ */
/* Phase field: periodic trilinear interpolation (Sec. II.C, reading R6) */
/* ------------------------------------------------------------------ */
static long wrap_index(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

double or_phi_at(const float* grid, const int dims[3], double h, double x, double y, double z) {
  double p[3] = {x / h, y / h, z / h};
  long i0[3], i1[3];
  double t[3];
  for (int a = 0; a < 3; ++a) {
    double f = floor(p[a]);
    t[a] = p[a] - f;
    i0[a] = wrap_index((long)f, dims[a]);
    i1[a] = wrap_index((long)f + 1, dims[a]);
  }
  double phi = 0.0;
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        long ix = cx ? i1[0] : i0[0];
        long iy = cy ? i1[1] : i0[1];
        long iz = cz ? i1[2] : i0[2];
        double w = (cx ? t[0] : 1.0 - t[0]) * (cy ? t[1] : 1.0 - t[1]) * (cz ? t[2] : 1.0 - t[2]);
        phi += w * (double)grid[(iz * dims[1] + iy) * dims[0] + ix];
      }
  return phi;
}

/* ------------------------------------------------------------------ */
/* Geometry helpers                                                     */
/* ------------------------------------------------------------------ */
/* Minimum-image separation r_i - r_j in a periodic box. */
static void min_image(const double* ri, const double* rj, const double L[3], double d[3]) {
  for (int a = 0; a < 3; ++a) {
    double v = ri[a] - rj[a];
    v -= L[a] * nearbyint(v / L[a]);
    d[a] = v;
  }
}

/* Cell list with cells of edge >= r_c = 1 (only a search aid: the pair set
 * it yields is pinned against the all-pairs search). */
typedef struct {
  int nc[3];
  double edge[3];
  int* head; /* first particle of each cell, -1 if empty */
  int* next; /* next particle in the same cell, -1 at the end */
} cells_t;

static int cell_coord(double x, double edge, int nc) {
  int c = (int)floor(x / edge);
  if (c < 0) c = 0;
  if (c >= nc) c = nc - 1;
  return c;
}

static int cells_build(cells_t* C, int n, const double* pos, const double L[3]) {
  for (int a = 0; a < 3; ++a) {
    C->nc[a] = (int)floor(L[a]);
    if (C->nc[a] < 3) return -1;
    C->edge[a] = L[a] / C->nc[a];
  }
  long ncell = (long)C->nc[0] * C->nc[1] * C->nc[2];
  C->head = (int*)malloc(sizeof(int) * ncell);
  C->next = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  if (!C->head || !C->next) return -2;
  for (long c = 0; c < ncell; ++c) C->head[c] = -1;
  for (int i = n - 1; i >= 0; --i) {
    int cx = cell_coord(pos[3 * i + 0], C->edge[0], C->nc[0]);
    int cy = cell_coord(pos[3 * i + 1], C->edge[1], C->nc[1]);
    int cz = cell_coord(pos[3 * i + 2], C->edge[2], C->nc[2]);
    long c = ((long)cz * C->nc[1] + cy) * C->nc[0] + cx;
    C->next[i] = C->head[c];
    C->head[c] = i;
  }
  return 0;
}

static void cells_free(cells_t* C) {
  free(C->head);
  free(C->next);
}

/* Collect every j != i within the cutoff r < 1 of particle i (Sec. II.A: the
 * sum of Eq. 2 runs over particles closer than r_c).  method 0 searches all
 * particles; method 1 searches the 27 cells around i's cell. */
static int neighbours_of(int i, int n, const double* pos, const double L[3], int method,
                         const cells_t* C, int* out, int cap) {
  int m = 0;
  if (method == 0) {
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3];
      min_image(&pos[3 * i], &pos[3 * j], L, d);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 < 1.0) {
        if (m < cap) out[m] = j;
        ++m;
      }
    }
    return m;
  }
  int cx = cell_coord(pos[3 * i + 0], C->edge[0], C->nc[0]);
  int cy = cell_coord(pos[3 * i + 1], C->edge[1], C->nc[1]);
  int cz = cell_coord(pos[3 * i + 2], C->edge[2], C->nc[2]);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        long nx = wrap_index(cx + dx, C->nc[0]);
        long ny = wrap_index(cy + dy, C->nc[1]);
        long nz = wrap_index(cz + dz, C->nc[2]);
        long c = (nz * C->nc[1] + ny) * C->nc[0] + nx;
        for (int j = C->head[c]; j >= 0; j = C->next[j]) {
          if (j == i) continue;
          double d[3];
          min_image(&pos[3 * i], &pos[3 * j], L, d);
          double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          if (r2 < 1.0) {
            if (m < cap) out[m] = j;
            ++m;
          }
        }
      }
  return m;
}

static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

/* Every unordered pair (i < j) within the cutoff, as (i, j) rows sorted
 * lexicographically.  Returns the pair count; rows beyond cap are dropped. */
long or_pairs(int n, const double* pos, const double* L, int method, long cap, int* pairs) {
  cells_t C;
  memset(&C, 0, sizeof C);
  if (method == 1 && cells_build(&C, n, pos, L) != 0) return -1;
  int* nb = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  long m = 0;
  for (int i = 0; i < n; ++i) {
    int k = neighbours_of(i, n, pos, L, method, &C, nb, n);
    qsort(nb, (size_t)k, sizeof(int), cmp_int);
    for (int q = 0; q < k; ++q) {
      if (nb[q] <= i) continue;
      if (m < cap) {
        pairs[2 * m] = i;
        pairs[2 * m + 1] = nb[q];
      }
      ++m;
    }
  }
  free(nb);
  if (method == 1) cells_free(&C);
  return m;
}

/* Wall velocity at a point whose coordinate along the shear axis is xa (R18). */
static void wall_velocity(const double* P, double xa, double out[3]) {
  const int ax = (int)P[P_SHAXIS];
  const double L = P[P_LX + ax];
  double d = xa - P[P_SHREF];
  d -= L * floor(d / L + 0.5); /* nearest image: d in [-L/2, L/2) */
  out[0] = P[P_VWX] + d * P[P_SHX];
  out[1] = P[P_VWY] + d * P[P_SHY];
  out[2] = P[P_VWZ] + d * P[P_SHZ];
}

/* ------------------------------------------------------------------ */
/* Smoothing function of Eq. 23 (the SPH cubic spline) with support     */
/* scale r0: h = r0 / 2, v = r / h,                                      */
/*   W = alpha_D / h^D * { 1 - 3/2 v^2 + 3/4 v^3   (0 <= v < 1)          */
/*                         1/4 (2 - v)^3           (1 <= v < 2)          */
/*                         0                       (v >= 2) }            */
/* alpha_D = 2/3, 10/(7 pi), 1/pi for D = 1, 2, 3; and its derivative    */
/* dW/dr = alpha_D / h^(D+1) * dw/dv.                                    */
/* ------------------------------------------------------------------ */
static double sph_alpha(int D) {
  return D == 1 ? 2.0 / 3.0 : (D == 2 ? 10.0 / (7.0 * M_PI) : 1.0 / M_PI);
}

double or_sph_W(double r, double r0, int D) {
  const double h = 0.5 * r0, v = r / h;
  double w = 0.0;
  if (v < 1.0) w = 1.0 - 1.5 * v * v + 0.75 * v * v * v;
  else if (v < 2.0) w = 0.25 * (2.0 - v) * (2.0 - v) * (2.0 - v);
  return sph_alpha(D) / pow(h, D) * w;
}

double or_sph_dWdr(double r, double r0, int D) {
  const double h = 0.5 * r0, v = r / h;
  double dw = 0.0;
  if (v < 1.0) dw = -3.0 * v + 2.25 * v * v;
  else if (v < 2.0) dw = -0.75 * (2.0 - v) * (2.0 - v);
  return sph_alpha(D) / pow(h, D + 1) * dw;
}

/* Pair energy of Eq. 22: E = S^r W(r, r0^r) - S^a W(r, r0^a); fs selects the
 * fluid-solid strengths. */
double or_sph_energy(const double* P, double r, int fs) {
  const int D = (int)P[P_SPH_DIM];
  const double Sr = fs ? P[P_SR_FS] : P[P_SR_FF], Sa = fs ? P[P_SA_FS] : P[P_SA_FF];
  return Sr * or_sph_W(r, P[P_R0R], D) - Sa * or_sph_W(r, P[P_R0A], D);
}

/* ------------------------------------------------------------------ */
/* Pair force, Eqs. 3-10:                                              */
/*   f_ij = [ C(r) - gamma w_D (rhat . v_ij) + sigma w_R xi/sqrt(dt) ] rhat */
/*   w_R = 1 - r, w_D = (1 - r)^2 for r < 1, and the conservative part  */
/*   C(r) = a_ij w_C, w_C = 1 - r (Eq. 4; force law 0) or               */
/*   C(r) = -dE/dr of Eq. 22 (Eq. 24 read as -dE/dr, reading R19; law 1). */
/* ------------------------------------------------------------------ */
static void pair_force(const double* P, const double d[3], double r, const double vij[3],
                       int ti, int tj, double xi, double f[3]) {
  double wC = 1.0 - r;
  double wR = wC;
  double wD = wR * wR;
  double e[3] = {d[0] / r, d[1] / r, d[2] / r};
  double ev = e[0] * vij[0] + e[1] * vij[1] + e[2] * vij[2];
  double cons;
  if (P[P_FORCE_LAW] == 0.0) {
    cons = P[P_AFF + 2 * ti + tj] * wC;
  } else {
    const int D = (int)P[P_SPH_DIM], fs = ti != tj;
    const double Sr = fs ? P[P_SR_FS] : P[P_SR_FF], Sa = fs ? P[P_SA_FS] : P[P_SA_FF];
    cons = -(Sr * or_sph_dWdr(r, P[P_R0R], D) - Sa * or_sph_dWdr(r, P[P_R0A], D));
  }
  double mag = cons - P[P_GAMMA] * wD * ev + P[P_SIGMA] * wR * xi / sqrt(P[P_DT]);
  f[0] = mag * e[0];
  f[1] = mag * e[1];
  f[2] = mag * e[2];
}

/* The total pair force on every fluid particle (Eq. 2), evaluated with the
 * predicted velocities vt; solid particles get zero (reading R9).  The
 * noise counter uses `step`.  method 0 = all pairs, 1 = cell list. */
int or_forces_sel(int n, const double* pos, const double* vt, const int* id,
                  const uint8_t* type, const double* P, uint32_t step, uint32_t sys,
                  uint64_t seed, int method, int nsel, const int* sel, double* f, double* fabs_sum);

int or_forces(int n, const double* pos, const double* vt, const int* id, const uint8_t* type,
              const double* P, uint32_t step, uint32_t sys, uint64_t seed, int method,
              double* f) {
  return or_forces_sel(n, pos, vt, id, type, P, step, sys, seed, method, -1, NULL, f, NULL);
}

/* As or_forces, for the particles listed in sel (nsel of them; nsel < 0 means
 * all) -- f and fabs_sum are indexed like sel.  fabs_sum (may be NULL)
 * receives sum_j |f_ij|, the scale against which a force error is measured. */
int or_forces_sel(int n, const double* pos, const double* vt, const int* id,
                  const uint8_t* type, const double* P, uint32_t step, uint32_t sys,
                  uint64_t seed, int method, int nsel, const int* sel, double* f, double* fabs_sum) {
  const double L[3] = {P[P_LX], P[P_LY], P[P_LZ]};
  cells_t C;
  memset(&C, 0, sizeof C);
  if (method == 1 && cells_build(&C, n, pos, L) != 0) return -1;
  int fail = 0;
#pragma omp parallel
  {
    int* nb = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    if (!nb) fail = 1;
    const int nout = nsel < 0 ? n : nsel;
#pragma omp for schedule(static)
    for (int q0 = 0; q0 < nout; ++q0) {
      const int i = nsel < 0 ? q0 : sel[q0];
      double* fo = &f[3 * q0];
      fo[0] = fo[1] = fo[2] = 0.0;
      if (fabs_sum) fabs_sum[q0] = 0.0;
      if (!nb || i < 0 || i >= n || type[i] != 0) continue;
      int k = neighbours_of(i, n, pos, L, method, &C, nb, n);
      for (int q = 0; q < k; ++q) {
        int j = nb[q];
        double d[3];
        min_image(&pos[3 * i], &pos[3 * j], L, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r == 0.0) continue; /* reading R8 */
        double vj[3];
        if (type[j] == 0) {
          vj[0] = vt[3 * j]; vj[1] = vt[3 * j + 1]; vj[2] = vt[3 * j + 2];
        } else {
          wall_velocity(P, pos[3 * j + (int)P[P_SHAXIS]], vj); /* R9, R18 */
        }
        double vij[3] = {vt[3 * i] - vj[0], vt[3 * i + 1] - vj[1], vt[3 * i + 2] - vj[2]};
        double xi = or_xi((uint32_t)id[i], (uint32_t)id[j], step, sys, seed);
        double fij[3];
        pair_force(P, d, r, vij, type[i], type[j], xi, fij);
        fo[0] += fij[0];
        fo[1] += fij[1];
        fo[2] += fij[2];
        if (fabs_sum) fabs_sum[q0] += sqrt(fij[0] * fij[0] + fij[1] * fij[1] + fij[2] * fij[2]);
      }
    }
    free(nb);
  }
  if (method == 1) cells_free(&C);
  return fail ? -2 : 0;
}

/* ------------------------------------------------------------------ */
/* One time step (Sec. II.A integrator of ref. 35; Sec. II.C reflection). */
/*                                                                     */
/* On entry pos, vel, frc hold r(t), v(t) and the pair force f(t); the  */
/* total force is F = f + g for fluid particles.  On exit they hold     */
/* r(t+dt), v(t+dt), f(t+dt), and reflected[i] says whether particle i  */
/* was bounced back.  stats = {reflections, fallbacks}.                 */
/*   r'  = r + dt v + dt^2/2 F                                          */
/*   vt  = v + lambda dt F                                              */
/*   bounce-back of r' at phi = 0 (Eq. 17, readings R1-R5)             */
/*   f(t+dt) = f(r', vt)                                                */
/*   v(t+dt) = v + dt/2 (F(t) + F(t+dt))   (not for reflected particles) */
/* ------------------------------------------------------------------ */
static double clamp_phi(double p) {
  const double lim = 1.0 - 1e-6;
  if (p > lim) return lim;
  if (p < -lim) return -lim;
  return p;
}

static double wrap_coord(double x, double L) {
  double w = x - L * floor(x / L);
  if (w >= L) w -= L;
  if (w < 0.0) w = 0.0;
  return w;
}

/* Wall velocity of every solid particle at its position (zero for fluid). */
void or_wall_velocities(int n, const double* pos, const uint8_t* type, const double* P,
                        double* out) {
  const int ax = (int)P[P_SHAXIS];
  for (int i = 0; i < n; ++i) {
    if (type[i] != 0) {
      wall_velocity(P, pos[3 * i + ax], out + 3 * i);
    } else {
      out[3 * i] = out[3 * i + 1] = out[3 * i + 2] = 0.0;
    }
  }
}

int or_step(int n, double* pos, double* vel, double* frc, const int* id, const uint8_t* type,
            const double* P, const float* grid, const int* dims, double h, uint32_t step_next,
            uint32_t sys, uint64_t seed, int method, uint8_t* reflected, long* stats,
            double* vwall) {
  const double dt = P[P_DT], lam = P[P_LAMBDA];
  const double L[3] = {P[P_LX], P[P_LY], P[P_LZ]};
  const double g[3] = {P[P_GX], P[P_GY], P[P_GZ]};
  const int ax = (int)P[P_SHAXIS];
  double* vt = (double*)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
  double* Fold = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
  if (!vt || !Fold) { free(vt); free(Fold); return -2; }
  long nrefl = 0, nfall = 0;

  for (int i = 0; i < n; ++i) {
    reflected[i] = 0;
    if (type[i] != 0) { /* frozen solid (readings R9, R14, R18): moves with the wall */
      double vw[3];
      wall_velocity(P, pos[3 * i + ax], vw);
      for (int a = 0; a < 3; ++a) {
        vt[3 * i + a] = vw[a];
        Fold[3 * i + a] = 0.0;
        if (vw[a] != 0.0) pos[3 * i + a] = wrap_coord(pos[3 * i + a] + dt * vw[a], L[a]);
        if (vwall) vwall[3 * i + a] = vw[a];
      }
      continue;
    }
    if (vwall) vwall[3 * i] = vwall[3 * i + 1] = vwall[3 * i + 2] = 0.0;
    double F[3], r0[3], v0[3], r1[3], dr[3];
    for (int a = 0; a < 3; ++a) {
      F[a] = frc[3 * i + a] + g[a];
      r0[a] = pos[3 * i + a];
      v0[a] = vel[3 * i + a];
      dr[a] = dt * v0[a] + 0.5 * dt * dt * F[a];
      r1[a] = r0[a] + dr[a];
      vt[3 * i + a] = v0[a] + lam * dt * F[a];
      Fold[3 * i + a] = F[a];
    }
    double phi_new = or_phi_at(grid, dims, h, r1[0], r1[1], r1[2]);
    if (phi_new < 0.0) {
      double phi_old = or_phi_at(grid, dims, h, r0[0], r0[1], r0[2]);
      if (phi_old < 0.0) phi_old = 0.0;
      double A = atanh(-clamp_phi(phi_new)); /* CD of Fig. 4 over sqrt(2) eps */
      double B = atanh(clamp_phi(phi_old));  /* AC of Fig. 4 over sqrt(2) eps */
      double s = A / (A + B);
      double vw[3]; /* wall velocity at the crossing point r + (1 - s) dr (R18) */
      wall_velocity(P, r0[ax] + (1.0 - s) * dr[ax], vw);
      double disp[3];
      for (int a = 0; a < 3; ++a)
        disp[a] = (P[P_REFLECT_VARIANT] == 1.0) ? (v0[a] - vw[a]) * dt : dr[a];
      double rbb[3];
      for (int a = 0; a < 3; ++a) rbb[a] = r1[a] - 2.0 * s * disp[a];
      double phi_bb = or_phi_at(grid, dims, h, rbb[0], rbb[1], rbb[2]);
      if (phi_bb < 0.0) {
        for (int a = 0; a < 3; ++a) rbb[a] = r0[a];
        ++nfall;
      }
      for (int a = 0; a < 3; ++a) {
        r1[a] = rbb[a];
        double vb = 2.0 * vw[a] - v0[a];
        vel[3 * i + a] = vb;
        vt[3 * i + a] = vb;
        if (vwall) vwall[3 * i + a] = vw[a];
      }
      reflected[i] = 1;
      ++nrefl;
    }
    for (int a = 0; a < 3; ++a) pos[3 * i + a] = wrap_coord(r1[a], L[a]);
  }

  int rc = or_forces(n, pos, vt, id, type, P, step_next, sys, seed, method, frc);
  if (rc == 0) {
    for (int i = 0; i < n; ++i) {
      if (type[i] != 0 || reflected[i]) continue;
      for (int a = 0; a < 3; ++a)
        vel[3 * i + a] += 0.5 * dt * (Fold[3 * i + a] + frc[3 * i + a] + g[a]);
    }
  }
  stats[0] = nrefl;
  stats[1] = nfall;
  free(vt);
  free(Fold);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Velocity profile sums over fluid particles (Sec. III.A).             */
/* Bin b of [lo, hi) along `axis`; the bin index is decided in binary32  */
/* arithmetic: b = floor((x - lo) * (nbins / (hi - lo))), so that the     */
/* oracle and the GPU take the same integer decision.  Per bin the five   */
/* sums are {count, sum vx, sum vy, sum vz, sum |v|^2}; they accumulate   */
/* into out (nbins x 5).                                                  */
/* ------------------------------------------------------------------ */
void or_profile(int n, const float* pos4, const double* vel, const uint8_t* type, int axis,
                int nbins, double lo, double hi, double* out) {
  volatile float lo_f = (float)lo;
  volatile float inv_f = (float)((double)nbins / (hi - lo));
  for (int i = 0; i < n; ++i) {
    if (type[i] != 0) continue;
    volatile float x = pos4[4 * i + axis];
    volatile float t = x - lo_f;
    volatile float u = t * inv_f;
    float fb = floorf(u);
    if (!(fb >= 0.0f) || fb >= (float)nbins) continue;
    int b = (int)fb;
    double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
    out[5 * b + 0] += 1.0;
    out[5 * b + 1] += vx;
    out[5 * b + 2] += vy;
    out[5 * b + 3] += vz;
    out[5 * b + 4] += vx * vx + vy * vy + vz * vz;
  }
}

/* Phase field at many points (see or_phi_at). */
void or_phi_many(const float* grid, const int dims[3], double h, long m, const double* pts,
                 double* out) {
  for (long k = 0; k < m; ++k) out[k] = or_phi_at(grid, dims, h, pts[3 * k], pts[3 * k + 1], pts[3 * k + 2]);
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Particle set-up from the phase field (Sec. II.C, reading R20).       */
/* A dense random fluid fills the box: site k of n0 (= round(rho V),    */
/* given by the caller) takes its position from Philox4x32-10 of the    */
/* counter (k, 0xFFFFFFFF, 0xFFFFFFFE, sys) and a Maxwellian velocity   */
/* from (k, 0xFFFFFFFF, 0xFFFFFFFD, sys), key = seed:                   */
/*   r = (u0 Lx, u1 Ly, u2 Lz),                                         */
/*   v = sqrt(kBT) (sqrt(-2 ln u0') cos(2 pi u1'),                      */
/*                  sqrt(-2 ln u0') sin(2 pi u1'),                      */
/*                  sqrt(-2 ln u2') cos(2 pi u3')).                     */
/* The interpolated phase field classifies every site: phi >= 0 fluid,  */
/* phi_min < phi < 0 frozen solid, otherwise removed.  The mean fluid   */
/* velocity is subtracted.  Kept sites are numbered in site order.      */
/* Outputs: site_phi[n0], site_type[n0] (0 fluid, 1 solid, 2 removed),  */
/* and the kept particles pos, vel (n x 3), type (n), site (n).         */
/* Returns n.  have_grid = 0 means phi = +1 everywhere.                 */
/* ------------------------------------------------------------------ */
long or_init_particles(long n0, const double L[3], double kBT, uint64_t seed, uint32_t sys,
                       double phi_min, int have_grid, const float* grid, const int* dims, double h,
                       double* site_phi, uint8_t* site_type, double* pos, double* vel, uint8_t* type,
                       long* site) {
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  long n = 0, nf = 0;
  double mean[3] = {0.0, 0.0, 0.0};
  for (long k = 0; k < n0; ++k) {
    uint32_t ca[4] = {(uint32_t)k, 0xFFFFFFFFu, 0xFFFFFFFEu, sys}, wa[4];
    uint32_t cb[4] = {(uint32_t)k, 0xFFFFFFFFu, 0xFFFFFFFDu, sys}, wb[4];
    or_philox4x32_10(ca, key, wa);
    or_philox4x32_10(cb, key, wb);
    const double r[3] = {or_u01(wa[0]) * L[0], or_u01(wa[1]) * L[1], or_u01(wa[2]) * L[2]};
    const double ra = sqrt(-2.0 * log(or_u01(wb[0]))), rb = sqrt(-2.0 * log(or_u01(wb[2])));
    const double s = sqrt(kBT);
    const double v[3] = {s * ra * cos(2.0 * M_PI * or_u01(wb[1])), s * ra * sin(2.0 * M_PI * or_u01(wb[1])),
                         s * rb * cos(2.0 * M_PI * or_u01(wb[3]))};
    const double phi = have_grid ? or_phi_at(grid, dims, h, r[0], r[1], r[2]) : 1.0;
    const uint8_t t = phi >= 0.0 ? 0 : (phi > phi_min ? 1 : 2);
    site_phi[k] = phi;
    site_type[k] = t;
    if (t == 2) continue;
    for (int a = 0; a < 3; ++a) {
      pos[3 * n + a] = r[a];
      vel[3 * n + a] = t == 0 ? v[a] : 0.0;
    }
    if (t == 0) {
      for (int a = 0; a < 3; ++a) mean[a] += v[a];
      ++nf;
    }
    type[n] = t;
    site[n] = k;
    ++n;
  }
  for (long i = 0; i < n; ++i)
    if (type[i] == 0)
      for (int a = 0; a < 3; ++a) vel[3 * i + a] -= mean[a] / (double)nf;
  return n;
}
