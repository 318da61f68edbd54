/*
 * dpd.h -- C ABI of the GB300 library for one time step of dissipative
 * particle dynamics (DPD) in a confined geometry with phase-field no-slip
 * walls (Xu & Meakin, arXiv:1807.09896).
 *
 * One handle holds one periodic DPD system: its parameters, its phase field
 * phi(x) on a grid, and its particles, all resident on the current CUDA
 * device.  One call of dpd_step advances the system by whole time steps; every
 * step runs, on the GPU:
 *   1. drift r' = r + dt v + dt^2/2 F and predicted velocity
 *      vt = v + lambda dt F of the Groot-Warren modified velocity-Verlet
 *      scheme the paper uses (Sec. II.A, ref. 35), F = f + g on fluid
 *      particles (Eq. 1-2; body force g as in Sec. III.A);
 *   2. bounce-back reflection of every fluid particle whose new position has
 *      phi < 0, at the sharp phi = 0 surface located with the interpolated
 *      phase field (Sec. II.C, Eq. 17, Fig. 4);
 *   3. a cell-list rebuild (counting sort of the particles by cell of edge
 *      >= r_c; each cell holds its particles in the order they had in the
 *      previous step's arrays, which start in id order);
 *   4. the pair force f_i = sum_j f_ij over all j within r_c = 1
 *      (Eq. 2), f_ij = f^C + f^D + f^R of Eqs. 3-10 with the random force
 *      sigma w_R xi_ij / sqrt(dt), xi_ij drawn from Philox4x32-10 keyed by the
 *      pair and the step;
 *   5. the closing half-kick v(t+dt) = v + dt/2 (F(t) + F(t+dt)), skipped
 *      for particles reflected in this step (their velocity is 2 v_w - v, v_w
 *      the wall velocity where the particle crossed phi = 0).
 * Solid (frozen) particles get no force and move with the wall velocity v_w at
 * their position, which is zero unless the walls move (Sec. II.C moving walls):
 * v_w(r) = v_wall + d S, d = r[shear_axis] - shear_ref wrapped into
 * [-L/2, L/2), S = (shear_x, shear_y, shear_z) with no component along the axis
 * (plane Couette walls slide in their planes; S = 0: all walls move together).
 *
 * Conventions.  DPD units: r_c = 1, particle mass 1.  Arrays of 4 floats per
 * particle ("pos4", "vel4", "force4") hold x, y, z and one unused pad float.
 * Particle types: 0 = fluid, 1 = solid.  Particle ids must be a permutation of
 * 0..n-1; state read back with dpd_get_state is in id order.
 *
 * Ownership.  The library copies every input it is given; the caller keeps
 * its buffers.  Outputs go to caller buffers.  `where` says whether a
 * caller pointer is host memory (DPD_HOST) or device memory on the handle's
 * device (DPD_DEVICE).  The library allocates its own device memory in
 * dpd_set_phase_field and dpd_set_particles (never inside dpd_step).
 *
 * Errors.  Every call returns DPD_OK (0) or a negative code below;
 * dpd_last_error gives a message for the last failure on that handle.  A
 * handle is used by one host thread at a time.  All GPU work of a handle runs
 * on one CUDA stream (its own, or the one given to dpd_set_stream).
 */
#ifndef DPD_H_
#define DPD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpd_system dpd_t;

enum {
  DPD_OK = 0,
  DPD_EINVAL = -1,   /* bad argument */
  DPD_ENOMEM = -2,   /* device or host allocation failed */
  DPD_ECUDA = -3,    /* a CUDA call failed */
  DPD_ESTATE = -4,   /* call out of order (e.g. dpd_step before dpd_set_particles) */
  DPD_ELOST = -5,    /* a fluid particle was found at phi < 0 */
  DPD_EBAND = -6,    /* a drift exceeded the band margin of the reflection test */
  DPD_ETIMEOUT = -7, /* reserved for a bounded device wait that gives up: no kernel of
                        this library waits on another block, so none is returned */
  DPD_ENAN = -8,     /* a non-finite position, velocity or force appeared */
  DPD_EOVERFLOW = -9 /* a size limit was exceeded (e.g. a cell holds too many particles) */
};

enum { DPD_HOST = 0, DPD_DEVICE = 1 };

/* Create a system on the current CUDA device.
 * box[3]      periodic box edges (each >= 3 r_c; cells have edge L / floor(L) >= 1).
 * rho         nominal number density, used to report densities in profiles.
 * a_ij[4]     conservative amplitudes a_ff, a_fs, a_sf, a_ss (Eq. 4); only a_ff and
 *             a_fs enter (solid-solid pairs are never evaluated, a_sf = a_fs).
 * gamma       dissipative coefficient (Eq. 6).
 * sigma       random-force coefficient (Eq. 7); Eq. 8 asks sigma^2 = 2 gamma kBT,
 *             which the library does not enforce.
 * kBT         temperature (used for reporting only).
 * dt          time step.
 * body_force  acceleration g added to the force on every fluid particle.
 * Options (dpd_set_option) start at: lambda 0.65, band_margin 0.5,
 * reflect_variant 0, seed 0, system 0, v_wall 0, shear 0, sample_every 0. */
int dpd_create(dpd_t** h, const double box[3], double rho, const double a_ij[4], double gamma,
               double sigma, double kBT, double dt, const double body_force[3]);

/* Set the phase field phi (Sec. II.B): dims[0] x dims[1] x dims[2] float32 node
 * values, x fastest, node (i, j, k) at (i, j, k) * spacing, periodic; dims[a] *
 * spacing must equal box[a].  phi > 0 is fluid, phi < 0 solid, phi = 0 the sharp
 * surface.  The grid is host memory.  Without a phase field phi = +1 everywhere
 * (no reflection).  Must precede dpd_set_particles. */
int dpd_set_phase_field(dpd_t* h, const float* grid, const int dims[3], double spacing);

/* Set up particles from the phase field as Sec. II.C describes: a dense random
 * fluid at the create-time density rho fills the whole box, and the interpolated
 * phase field (set first; without one every site is fluid) classifies each site:
 * phi >= 0 fluid, phi_min < phi < 0 frozen solid, phi <= phi_min removed, with
 * phi_min = tanh(-solid_layer / (sqrt(2) eps)) the value of Eq. 14 at a distance
 * solid_layer inside the solid (eps: option "phase_eps", default 0.5).  Site k of
 * round(rho Lx Ly Lz) takes its position from Philox4x32-10 of the counter
 * (k, 0xFFFFFFFF, 0xFFFFFFFE, system) and a Maxwellian velocity at kBT (Box-Muller)
 * from (k, 0xFFFFFFFF, 0xFFFFFFFD, system), key = seed; the mean fluid velocity is
 * removed; kept sites get ids 0..n-1 in site order.  Deterministic.  Then loads the
 * particles as dpd_set_particles does (errors likewise; DPD_EOVERFLOW if
 * rho V >= 2^30, DPD_EINVAL if solid_layer < 0). */
int dpd_init_particles(dpd_t* h, uint64_t seed, double solid_layer);

/* Load n particles (any order): pos4 positions (wrapped into the box), vel4
 * velocities, id a permutation of 0..n-1, type 0 fluid / 1 solid.  Computes the
 * pair force f(0) at the given state (predicted velocity = v).  Solid
 * velocities are ignored (they move with the wall velocity).  Fails with DPD_ELOST if a fluid
 * particle sits inside the solid, at phi < -1e-4 (a margin for the rounding of binary32
 * positions: a step stores positions rounded, and one just outside the wall can read
 * a phase field a few 1e-6 below zero).  The step counter is kept (see option "step"). */
int dpd_set_particles(dpd_t* h, int n, const float* pos4, const float* vel4, const int* id,
                      const uint8_t* type, int where);

/* Advance nsteps >= 0 time steps.  The device status word is read once at the
 * end; a non-zero status returns DPD_EBAND / DPD_ENAN / DPD_ELOST /
 * DPD_EOVERFLOW and stays set until the next dpd_set_particles. */
int dpd_step(dpd_t* h, int nsteps);

/* Phases of one time step, in launch order, as timed by dpd_time_phases: one
 * kernel each, except the scan (two or three launches). */
enum {
  DPD_PHASE_INTEGRATE = 0, /* counter bump + drift, reflection, cell key and count */
  DPD_PHASE_SCAN = 1,      /* exclusive scan of the cell counts */
  DPD_PHASE_SCATTER = 2,   /* counting-sort scatter of the particle indices */
  DPD_PHASE_CELL_SORT = 3, /* per-cell order (previous index, ascending) */
  DPD_PHASE_GATHER = 4,    /* gather of the particle arrays into cell order */
  DPD_PHASE_FORCE = 5,     /* pair force (Eqs. 3-10); full-shell shapes also finish the kick */
  DPD_PHASE_FINISH = 6,    /* Newton's-third-law shapes: sums -> force, closing kick (else 0) */
  DPD_NPHASES = 7
};

/* Advance nsteps > 0 time steps exactly as dpd_step does, but launched one by one
 * (no graph) with CUDA events between the phases of every step on the handle's
 * stream; ms[DPD_NPHASES] receives each phase's mean duration per step in
 * milliseconds.  Same results and error codes as dpd_step. */
int dpd_time_phases(dpd_t* h, int nsteps, double* ms);

/* Pick the fastest launch shape of the pair-force kernel for this system on this
 * device.  There are two algorithms.  Full-shell shapes evaluate every pair from
 * both sides and sum in binary32 in a fixed order.  Newton's-third-law shapes
 * (option "force_newton3" = 1) evaluate every pair once, give -f_ij to the partner
 * and sum in 64-bit fixed point (2^-32 resolution), then a second kernel applies
 * the closing kick.  Within one algorithm every shape (threads per block, pair-list
 * slots per thread, resident blocks, loop unroll) computes bit-identical results;
 * the two algorithms agree to binary32 rounding.  Both are deterministic.  Each
 * shape is timed over nsteps event-timed steps (after one warm-up step).  The state
 * and counters are then restored, so tuning does not advance the system.
 * ms_per_variant (may be NULL) receives the mean force time of each shape (size:
 * option "force_variants"); chosen (may be NULL) the index now in use (option
 * "force_variant"). */
int dpd_autotune(dpd_t* h, int nsteps, double* ms_per_variant, int* chosen);

/* Copy the state in id order: pos4 / vel4 / force4 (n x 4 floats; the force is
 * the pair force f without the body force; solid particles have f = 0 and the
 * velocity 0; vel4[4 i + 3] is 1 if particle i was reflected in the last step,
 * else 0), id
 * (n ints, equal to 0..n-1) and type (n bytes).  Any output pointer may be
 * NULL.  Synchronises the handle's stream. */
int dpd_get_state(dpd_t* h, float* pos4, float* vel4, float* force4, int* id, uint8_t* type,
                  int where);

/* Velocity profile of the fluid (Sec. III.A): nbins bins of [lo, hi) along axis
 * (0, 1, 2).  Per bin the library accumulates, in FP64, five sums over samples
 * and particles: {count, sum vx, sum vy, sum vz, sum |v|^2}.  mode: 0 = add one
 * sample of the current state and read; 1 = reset the accumulators (and bin
 * layout), add one sample, read; 2 = read only; 3 = reset only.  out is host
 * memory of nbins x 5 doubles (may be NULL for mode 3).  dpd_step also adds a
 * sample every `sample_every` steps (option) with the current bin layout. */
int dpd_velocity_profile(dpd_t* h, int axis, int nbins, double lo, double hi, double* out,
                         int mode);

/* Phase field of an arbitrary geometry (Sec. II.B): relax phi on a periodic grid of
 * dims[0] x dims[1] x dims[2] nodes (x fastest, host memory, updated in place) of
 * spacing h by `iters` explicit Euler steps of size dtau in the pseudo time of
 * Eq. 13, in the scaled coordinates x' = x / eps.  With curvature = 1 the equation is
 * Eq. 15, d phi/dt' = lap' phi + phi (1 - phi^2) - kappa |grad' phi|, whose curvature
 * term keeps curved interfaces in place; with 0 it is Eq. 13 in every direction.
 * Start from a step function (+1 fluid, -1 solid); the steady profile across an
 * interface is tanh(d / (sqrt(2) eps)) (Eq. 14) and the result can be passed to
 * dpd_set_phase_field.  dtau must not exceed (h / eps)^2 / 6, every dimension needs
 * 3 nodes, dims[1] at most 524280 and dims[2] at most 65535 (else DPD_EINVAL).
 * ms_per_iter (may be NULL) receives the mean device time of one step.  Uses the
 * current device and the default stream; messages: dpd_last_error(NULL). */
int dpd_relax_phase_field(float* phi, const int dims[3], double spacing, double eps, int iters,
                          double dtau, int curvature, double* ms_per_iter);

/* Largest nbins accepted by dpd_velocity_profile_noalloc. */
#define DPD_NOALLOC_MAX_BINS 4096

/* Velocity-profile sums of caller-owned particle arrays, with no memory
 * allocation of any kind (no cudaMalloc, cudaFree or allocating library call).
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory -- a framework that owns all device memory through its
 * own pool, a process under a hard memory cap, or a latency-bound loop where an
 * allocation would synchronise the device -- and so cannot create a handle.
 *
 * pos4, vel4  device arrays of n x 4 floats (x, y, z, unused), any order.
 * type        device array of n bytes, 0 = fluid (counted), else skipped.
 * axis, nbins, lo, hi, and the five sums per bin {count, sum vx, sum vy,
 *             sum vz, sum |v|^2}: as dpd_velocity_profile, for this one sample
 *             (nothing accumulates across calls); 1 <= nbins <=
 *             DPD_NOALLOC_MAX_BINS, larger values return DPD_EINVAL.
 * out         nbins x 5 doubles; host memory (where = DPD_HOST, the call then
 *             waits for the result) or device memory (DPD_DEVICE, the copy is
 *             queued on `stream` and the call returns at once).
 * stream      cudaStream_t to run on (NULL: the default stream).
 * The FP64 accumulators live in one fixed device array of DPD_NOALLOC_MAX_BINS x
 * 5 doubles (160 KiB) that every GPU loading the library keeps until the
 * process exits.  Every call shares it: each call clears what it uses first,
 * and calls whose work overlaps on the GPU (e.g. on two streams) race and give
 * wrong sums.  The first call in a CUDA context (per device, and again after a
 * cudaDeviceReset) looks up that array's device address with the device
 * current; make that first call before any stream capture begins.  The array
 * itself comes into being when the library's device code is loaded into the
 * context: under CUDA's default lazy loading that can be inside the first call,
 * so a process that will run under a hard memory cap should make one call
 * (or set CUDA_MODULE_LOADING=EAGER) before the cap applies.
 * Errors: dpd_last_error(NULL) holds the message. */
int dpd_velocity_profile_noalloc(const float* pos4, const float* vel4, const uint8_t* type, int n,
                                 int axis, int nbins, double lo, double hi, double* out, int where,
                                 void* stream);

/* Whole-system diagnostics, FP64: out[0..2] total fluid momentum, out[3] sum
 * |v|^2 over fluid, out[4] fluid count, out[5] reflections so far, out[6]
 * fallbacks so far (reflected point still at phi < 0, particle kept at r(t)),
 * out[7] steps taken (the step counter). */
int dpd_get_stats(dpd_t* h, double out[8]);

/* Set or read a named option: "lambda", "band_margin", "reflect_variant" (0:
 * displacement of the step, 1: v(t) dt as printed in Eq. 17), "seed" (integer
 * <= 2^53), "system" (Philox counter word 3), "v_wall_x|y|z", "shear_x|y|z",
 * "shear_axis" (0-2, default 2), "shear_ref" (the wall velocity field above; a
 * shear component along shear_axis is DPD_EINVAL), "phase_eps" (eps of Eq. 14 for
 * dpd_init_particles, default 0.5), "force_law" (0: the soft
 * repulsion a_ij w of Eq. 4; 1: the attractive/repulsive pair energy of Eq. 22,
 * E = S^r W(r, r0^r) - S^a W(r, r0^a) with the cubic spline W of Eq. 23, whose
 * conservative force is -dE/dr along r_ij (Eq. 24); the dissipative and random
 * forces are unchanged), its parameters "S_r_ff", "S_a_ff", "S_r_fs", "S_a_fs"
 * (fluid-fluid and fluid-solid strengths; defaults 37.5, 18.75, 75, 37.5 as in
 * the paper's wetting example), "r0_r", "r0_a" (ranges in (0, 1]; defaults 0.73,
 * 1), "sph_dim" (D of Eq. 23's normalisation, 1-3; default 3), "sample_every",
 * "a_ff", "a_fs", "gamma", "sigma", "g_x", "g_y", "g_z" (the create-time
 * parameters), "step" (the step counter, part of the noise counter), "use_graph" (1: replay
 * steps from a CUDA graph), "graph_steps" (even number of steps per graph,
 * default 20), "force_variant" (launch shape of the pair-force kernel, see
 * dpd_autotune), "adjoint_tape_mb" (see dpd_adjoint_window).
 * Read-only (dpd_get_option): "ncells", "kernel_launches" (kernels
 * enqueued by stepping calls so far), "kernels_per_step", "force_variants",
 * "force_newton3" (1 if the current shape evaluates each pair once), "scan_tiles"
 * (tiles of 2048 cells in the cell scan). */
int dpd_set_option(dpd_t* h, const char* key, double value);
int dpd_get_option(dpd_t* h, const char* key, double* value);

/* Particle counts currently loaded. */
int dpd_num_particles(dpd_t* h, int* n, int* n_fluid);

/* Reverse-mode gradient of a near-wall velocity-profile loss over a window of
 * nsteps time steps, with respect to (a_fs, gamma, g_x).  The paper has no
 * counterpart (it sets a_fs, gamma and g by hand); this calibrates the wall
 * interaction of Eqs. 4-10 and the body force of Sec. III.A against a target
 * profile.
 * Window: f(0) is recomputed at the current state with the current parameters
 * and predicted velocity v(0); then nsteps steps run exactly as dpd_step (the
 * system ends the call advanced by nsteps, its statistics counted once).
 * Loss: fluid particles are binned by their distance to the nearer wall,
 * d = min(x_axis - wall_lo, wall_hi - x_axis), into nbins bins of width
 * bin_width (binary32 decision); u_b is the mean x velocity of bin b over the
 * states after steps 1..nsteps; L = sum_b (u_b - target[b])^2 (bins never
 * visited are skipped).
 * Gradient: the discrete adjoint of every step (pair force with the noise drawn
 * again from its counter, drift, predicted velocity, closing kick, and Eq. 17
 * reflection including the gradient of the interpolated phase field).  Events
 * are frozen: reflection decisions, cell lists and bin membership are those of
 * the forward trajectory.  tie_sigma = 1 first sets sigma = sqrt(2 gamma kBT)
 * (Eq. 8; the system keeps that sigma) and differentiates through the tie, so
 * d/dgamma includes the random force (DPD_EINVAL unless kBT > 0 and gamma > 0);
 * 0 runs with sigma as set and holds it fixed.  grad[3] receives
 * dL/da_fs, dL/dgamma, dL/dg_x; loss_out (may be NULL) receives L.
 * Memory: the reverse pass walks a record of every step (the state, 64 B per
 * particle, and the step's sort permutation and cell starts).  If the whole
 * window's record fits the budget of option "adjoint_tape_mb" (MiB, default 2048)
 * the forward pass keeps it; otherwise it keeps a checkpoint every ckpt_every steps
 * (nsteps must be a multiple in either case) and the reverse pass recomputes one
 * segment at a time into a record of ckpt_every steps.  Both give the same bits.
 * The device workspace (record, checkpoints, adjoint arrays) is kept by the system
 * for the next window, grown when a window needs more, and freed by dpd_destroy or
 * by setting "adjoint_tape_mb".
 * Determinism: the loss bins are summed with integer atomics (velocity sums in
 * units of 2^-24, |sum| < 2^39 per bin) and the parameter sums in per-warp slots
 * added in a fixed order, so repeated calls on the same state give the same bits.
 * Requires reflect_variant 0, force_law 0 and walls moving together (shear 0);
 * otherwise DPD_EINVAL. */
int dpd_adjoint_window(dpd_t* h, int nsteps, int ckpt_every, int axis, double wall_lo,
                       double wall_hi, int nbins, double bin_width, const double* target,
                       int tie_sigma, double* loss_out, double grad[3]);

/* dpd_adjoint_window, plus a record of its pieces, so that each segment of the
 * window can be checked on its own (the paper has no counterpart).  Host outputs,
 * each may be NULL; nseg = nsteps / ckpt_every, n the particle count:
 * ckpt      (nseg + 1) x n x 12 floats: the state at each checkpoint (steps
 *           0, K, 2K, ...), per particle in id order: position (x, y, z, tag),
 *           velocity (x, y, z, 1 if reflected in the step that produced it),
 *           pair force (x, y, z, 0).
 * adj       (nseg + 1) x n x 12 floats, same layout: the adjoint of that state
 *           (dL/d position, dL/d velocity, dL/d force, each with an unused 4th
 *           float), L linearised at the forward trajectory; it includes the
 *           loss terms of the state itself and of every later state.
 * seg_grad  nseg x 3 doubles: dL/d(a_fs, gamma, g_x) accumulated while reversing
 *           segment k (segment 0 includes the dependence of f(0) on the
 *           parameters); they add up to grad.
 * coef      nbins floats: dL/d(sum of vx in bin b over the window), i.e.
 *           2 (u_b - target_b) / count_b (0 for bins never visited).
 * seg_step  nseg + 1 step counters (noise counter word 2) of the checkpoints.
 * Everything else as dpd_adjoint_window. */
int dpd_adjoint_window_record(dpd_t* h, int nsteps, int ckpt_every, int axis, double wall_lo,
                              double wall_hi, int nbins, double bin_width, const double* target,
                              int tie_sigma, double* loss_out, double grad[3], float* ckpt,
                              float* adj, double* seg_grad, float* coef, uint32_t* seg_step);

/* ---- Batches: many independent systems advanced together ------------------
 * The paper has no counterpart (it runs one system at a time); this is the
 * ensemble form of the same step.  A batch copies the current state of nsys
 * loaded systems into one set of concatenated device arrays; every phase of a
 * step is then one launch over all systems, replayed from a CUDA graph.  Each
 * system keeps its own box, phase field, parameters, seed, system index and step
 * counter: a system advanced in a batch follows bit for bit the trajectory it
 * follows alone.  The member handles are not advanced (their state stays as it
 * was at dpd_batch_create); the batch reads their phase fields and band masks,
 * so they must outlive the batch and keep their phase field.  All members must
 * use the same force_law (DPD_EINVAL).  Error messages of dpd_batch_create:
 * dpd_batch_last_error(NULL). */
typedef struct dpd_batch dpd_batch_t;

int dpd_batch_create(dpd_batch_t** hb, int nsys, dpd_t* const* systems);
/* Advance every system by nsteps steps (graph replay; options "use_graph",
 * "graph_steps" as for a single system).  Errors as dpd_step. */
int dpd_batch_step(dpd_batch_t* hb, int nsteps);
/* As dpd_time_phases / dpd_autotune, over the whole batch. */
int dpd_batch_time_phases(dpd_batch_t* hb, int nsteps, double* ms);
int dpd_batch_autotune(dpd_batch_t* hb, int nsteps, double* ms_per_variant, int* chosen);
/* State of system k (0-based, in the order given to dpd_batch_create), in its
 * own id order; arguments as dpd_get_state. */
int dpd_batch_get_state(dpd_batch_t* hb, int k, float* pos4, float* vel4, float* force4, int* id,
                        uint8_t* type, int where);
/* Diagnostics of system k, as dpd_get_stats. */
int dpd_batch_get_stats(dpd_batch_t* hb, int k, double out[8]);
/* Options "use_graph", "graph_steps", "force_variant"; read-only "force_variants",
 * "kernel_launches", "kernels_per_step", "nsys", "n" (all particles), "ncells". */
int dpd_batch_set_option(dpd_batch_t* hb, const char* key, double value);
int dpd_batch_get_option(dpd_batch_t* hb, const char* key, double* value);
int dpd_batch_num_particles(dpd_batch_t* hb, int k, int* n, int* n_fluid);
int dpd_batch_set_stream(dpd_batch_t* hb, void* stream);
int dpd_batch_destroy(dpd_batch_t* hb);
const char* dpd_batch_last_error(const dpd_batch_t* hb);

/* Run the handle's work on `stream` (a cudaStream_t; NULL selects the handle's
 * own stream). */
int dpd_set_stream(dpd_t* h, void* stream);

/* Free every resource of the handle.  NULL is accepted. */
int dpd_destroy(dpd_t* h);

/* Message of the last failure on h (or of the last failed dpd_create when h is
 * NULL).  Never NULL; the string lives until the next call on h. */
const char* dpd_last_error(const dpd_t* h);

#ifdef __cplusplus
}
#endif

#endif /* DPD_H_ */
