// dpd_system.h -- the handle behind dpd_t (internal; shared by the single-system
// ABI and the batch ABI, which copies systems into one engine).
#pragma once

#include <cstdint>
#include <string>

#include "dpd_common.cuh"
#include "dpd_engine.h"

struct dpd_system {
  // parameters (DPD units)
  double box[3] = {0, 0, 0};
  double rho = 3.0;
  double a[4] = {25, 25, 25, 25};
  double gamma = 4.5, sigma = 3.0, kBT = 1.0, dt = 0.01;
  double lambda = 0.65;
  double g[3] = {0, 0, 0};
  double vw[3] = {0, 0, 0};
  double shear[3] = {0, 0, 0};  // d v_wall / d r_axis (plane Couette walls)
  int shear_axis = 2;
  double shear_ref = 0.0;
  // conservative force law: 0 soft repulsion (Eq. 4), 1 SPH-kernel attraction and
  // repulsion (Eqs. 22-24; defaults: the paper's wetting example)
  int force_law = 0;
  double sph_S[4] = {37.5, 18.75, 75.0, 37.5};  // S^r_ff, S^a_ff, S^r_fs, S^a_fs
  double sph_r0[2] = {0.73, 1.0};               // r0^r, r0^a
  int sph_dim = 3;
  double margin = 0.5;
  double phase_eps = 0.5;  // interface parameter eps of Eq. 14 (used by dpd_init_particles)
  uint64_t seed = 0;
  uint32_t sys = 0;
  int reflect_variant = 0;
  double adjoint_tape_mb = 2048.0;  // budget for keeping a whole adjoint window's record
  // the adjoint's device workspace (record, checkpoints, adjoint arrays): kept between
  // windows, grown when a window needs more, freed by dpd_destroy or adjoint_tape_mb
  void* d_adj_ws = nullptr;
  size_t adj_ws_bytes = 0;
  int sample_every = 0;
  int nc[3] = {0, 0, 0};
  int ncells = 0;
  // phase field and band mask (device)
  float* d_phi = nullptr;
  int pd[3] = {0, 0, 0};
  double h = 0.0;
  uint8_t* d_band = nullptr;
  // particles: one-system engine
  dpd::Engine E;
  int n_fluid = 0;
  bool loaded = false;
  bool params_dirty = true;
  uint64_t host_step = 0;
  // staging for host reads
  float4* d_out4 = nullptr;
  int* d_out_id = nullptr;
  uint8_t* d_out_type = nullptr;
  int out_cap = 0;
  // staging for host inputs of dpd_set_particles (pos and vel, ids, types, id check)
  float4* d_in4 = nullptr;
  int* d_in_id = nullptr;
  uint8_t* d_in_type = nullptr;
  uint32_t* d_seen = nullptr;
  int in_cap = 0;
  // profile accumulators and diagnostics
  double* d_prof = nullptr;
  int prof_cap = 0, prof_axis = 2, prof_nbins = 0;
  double prof_lo = 0, prof_hi = 0;
  double* d_stats = nullptr;
  cudaStream_t own_stream = nullptr;
  std::string err;
};

namespace dpd {
// Kernel parameters of a system, from its host-side settings.
StepParams make_params(const dpd_system* h);
}  // namespace dpd
