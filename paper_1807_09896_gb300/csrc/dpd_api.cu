// dpd_api.cu -- the single-system C ABI of include/dpd.h: handle life cycle,
// device memory, phase field, particle loading and read-back (Xu & Meakin,
// arXiv:1807.09896, Sec. II).  The time steps themselves run in the engine
// (dpd_engine.cu) with one system.
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

using dpd::Arrays;
using dpd::DevCounters;
using dpd::StepParams;

static std::string g_create_error;

namespace dpd {
// Message returned by dpd_last_error(NULL), for entry points without a handle.
void set_global_error(const char* msg) { g_create_error = msg; }

StepParams make_params(const dpd_system* h) {
  StepParams P;
  memset(&P, 0, sizeof P);
  for (int a = 0; a < 3; ++a) {
    P.L[a] = (float)h->box[a];
    P.invL[a] = (float)(1.0 / h->box[a]);
    P.halfL[a] = (float)(0.5 * h->box[a]);
    P.nc[a] = h->nc[a];
    P.inv_edge[a] = (float)(h->nc[a] / h->box[a]);
    P.g[a] = (float)h->g[a];
    P.vw[a] = (float)h->vw[a];
    P.sh[a] = (float)h->shear[a];
    if (h->vw[a] != 0.0 || h->shear[a] != 0.0) P.moving = 1;
    P.pd[a] = h->pd[a];
  }
  P.law = h->force_law;
  {
    const int D = h->sph_dim;
    const double alpha = D == 1 ? 2.0 / 3.0 : (D == 2 ? 10.0 / (7.0 * M_PI) : 1.0 / M_PI);
    const double hr = 0.5 * h->sph_r0[0], ha = 0.5 * h->sph_r0[1];
    const double cr = alpha / std::pow(hr, D + 1), ca = alpha / std::pow(ha, D + 1);
    P.sph_kr_ff = (float)(h->sph_S[0] * cr);
    P.sph_ka_ff = (float)(h->sph_S[1] * ca);
    P.sph_kr_fs = (float)(h->sph_S[2] * cr);
    P.sph_ka_fs = (float)(h->sph_S[3] * ca);
    P.sph_ihr = (float)(1.0 / hr);
    P.sph_iha = (float)(1.0 / ha);
  }
  P.sh_axis = h->shear_axis;
  P.sh_ref = (float)h->shear_ref;
  P.ncells = h->ncells;
  P.dt = (float)h->dt;
  P.half_dt = (float)(0.5 * h->dt);
  P.half_dt2 = (float)(0.5 * h->dt * h->dt);
  P.lam_dt = (float)(h->lambda * h->dt);
  P.a_ff = (float)h->a[0];
  P.a_fs = (float)h->a[1];
  P.gamma = (float)h->gamma;
  P.sigma_rsqdt = (float)(h->sigma / std::sqrt(h->dt));
  P.seed_lo = (uint32_t)(h->seed & 0xffffffffu);
  P.seed_hi = (uint32_t)(h->seed >> 32);
  for (int r = 0; r < 10; ++r) {  // the noise's Philox round keys
    P.rkey[2 * r] = P.seed_lo + (uint32_t)r * 0x9E3779B9u;
    P.rkey[2 * r + 1] = P.seed_hi + (uint32_t)r * 0xBB67AE85u;
  }
  P.sys = h->sys;
  P.reflect_variant = h->reflect_variant;
  P.margin = (float)h->margin;
  P.phi = h->d_phi;
  P.inv_h = h->h > 0 ? (float)(1.0 / h->h) : 0.0f;
  P.band = h->d_band;
  return P;
}
}  // namespace dpd

static int fail(dpd_t* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return code;
}

#define CU(h, call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail((h), DPD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
  } while (0)

template <typename T>
static cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

// Upload the system table when a parameter changed since the last upload.
static int sync_params(dpd_t* h) {
  if (!h->params_dirty) return DPD_OK;
  dpd::Engine& E = h->E;
  E.h_sys.resize(1);
  E.h_sys[0].P = dpd::make_params(h);
  E.h_sys[0].cell_off = 0;
  E.h_sys[0].part_off = 0;
  E.h_sys[0].n = (uint32_t)E.n;
  E.h_sys[0].pad = 0;
  const int rc = dpd::engine_upload_sys(E);
  if (rc) return rc;
  h->params_dirty = false;
  return DPD_OK;
}

static int read_status(dpd_t* h, uint32_t* st) {
  return dpd::engine_read_counters(h->E, st);
}

static int add_profile_sample(dpd_t* h) {
  if (h->prof_nbins <= 0) return DPD_OK;
  dpd::engine_settle(h->E);
  const float lo = (float)h->prof_lo;
  const float inv_w = (float)((double)h->prof_nbins / (h->prof_hi - h->prof_lo));
  const Arrays& A = h->E.arr[h->E.cur];
  dpd::launch_profile(A.pos, A.vel, h->E.n, h->prof_axis, h->prof_nbins, lo, inv_w, h->d_prof,
                      h->E.stream);
  CU(h, cudaGetLastError());
  return DPD_OK;
}

extern "C" {

int dpd_create(dpd_t** out, const double box[3], double rho, const double a_ij[4], double gamma,
               double sigma, double kBT, double dt, const double body_force[3]) {
  if (!out || !box || !a_ij || !body_force) return fail(nullptr, DPD_EINVAL, "null argument");
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (!(box[a] >= 3.0) || !std::isfinite(box[a]))
      return fail(nullptr, DPD_EINVAL, "box edge %d = %g must be finite and >= 3 r_c", a, box[a]);
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, DPD_EINVAL, "dt must be > 0");
  if (!(gamma >= 0.0) || !(sigma >= 0.0) || !(kBT >= 0.0) || !(rho > 0.0))
    return fail(nullptr, DPD_EINVAL, "gamma, sigma, kBT must be >= 0 and rho > 0");
  dpd_t* h = new (std::nothrow) dpd_system();
  if (!h) return fail(nullptr, DPD_ENOMEM, "out of host memory");
  for (int a = 0; a < 3; ++a) {
    h->box[a] = box[a];
    h->g[a] = body_force[a];
    h->nc[a] = (int)std::floor(box[a]);
  }
  for (int k = 0; k < 4; ++k) h->a[k] = a_ij[k];
  h->rho = rho;
  h->gamma = gamma;
  h->sigma = sigma;
  h->kBT = kBT;
  h->dt = dt;
  h->E.err = &h->err;
  const long ncells = (long)h->nc[0] * h->nc[1] * h->nc[2];
  if (ncells > (1L << 30)) {
    delete h;
    return fail(nullptr, DPD_EOVERFLOW, "too many cells (%ld)", ncells);
  }
  h->ncells = (int)ncells;
  cudaError_t e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
  h->E.stream = h->own_stream;
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_stats, 8 * sizeof(double));
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA set-up failed: ") + cudaGetErrorString(e);
    dpd_destroy(h);
    return DPD_ECUDA;
  }
  if (dpd::engine_reserve(h->E, 1, 0, h->ncells) != DPD_OK) {
    g_create_error = h->err;
    dpd_destroy(h);
    return DPD_ECUDA;
  }
  *out = h;
  return DPD_OK;
}

int dpd_set_phase_field(dpd_t* h, const float* grid, const int dims[3], double spacing) {
  if (!h) return DPD_EINVAL;
  if (!grid || !dims || !(spacing > 0.0)) return fail(h, DPD_EINVAL, "null grid or bad spacing");
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 2) return fail(h, DPD_EINVAL, "phase-field dims must be >= 2");
    if (std::fabs(dims[a] * spacing - h->box[a]) > 1e-6 * h->box[a])
      return fail(h, DPD_EINVAL, "dims[%d] * spacing = %g differs from the box edge %g", a,
                  dims[a] * spacing, h->box[a]);
  }
  const size_t nodes = (size_t)dims[0] * dims[1] * dims[2];
  for (size_t k = 0; k < nodes; ++k)
    if (!std::isfinite(grid[k])) return fail(h, DPD_EINVAL, "non-finite phase-field value at node %zu", k);
  dpd::engine_free_graphs(h->E);
  CU(h, cudaStreamSynchronize(h->E.stream));
  cudaFree(h->d_phi);
  cudaFree(h->d_band);
  h->d_phi = nullptr;
  h->d_band = nullptr;
  CU(h, dev_alloc(&h->d_phi, nodes));
  CU(h, dev_alloc(&h->d_band, (size_t)h->ncells));
  CU(h, cudaMemcpyAsync(h->d_phi, grid, nodes * sizeof(float), cudaMemcpyHostToDevice, h->E.stream));
  for (int a = 0; a < 3; ++a) h->pd[a] = dims[a];
  h->h = spacing;
  dpd::launch_band(dpd::make_params(h), h->d_band, h->E.stream);
  CU(h, cudaGetLastError());
  CU(h, cudaStreamSynchronize(h->E.stream));
  h->params_dirty = true;
  h->loaded = false;
  return DPD_OK;
}

int dpd_set_particles(dpd_t* h, int n, const float* pos4, const float* vel4, const int* id,
                      const uint8_t* type, int where) {
  if (!h) return DPD_EINVAL;
  if (n < 0 || (n > 0 && (!pos4 || !vel4 || !id || !type)))
    return fail(h, DPD_EINVAL, "bad particle arrays");
  if (where != DPD_HOST && where != DPD_DEVICE) return fail(h, DPD_EINVAL, "bad `where`");
  if (n >= (1 << 30)) return fail(h, DPD_EOVERFLOW, "too many particles");
  dpd::Engine& E = h->E;
  h->loaded = false;
  // captured graphs stay valid while the buffers, sizes and parameters do (engine_step
  // compares them; engine_reserve drops the graphs when it reallocates)
  int rc = dpd::engine_reserve(E, 1, n, h->ncells);
  if (rc) return rc;
  if (n > h->out_cap) {
    cudaFree(h->d_out4);
    cudaFree(h->d_out_id);
    cudaFree(h->d_out_type);
    h->d_out4 = nullptr;
    h->d_out_id = nullptr;
    h->d_out_type = nullptr;
    h->out_cap = 0;
    CU(h, dev_alloc(&h->d_out4, (size_t)3 * n));
    CU(h, dev_alloc(&h->d_out_id, n));
    CU(h, dev_alloc(&h->d_out_type, n));
    h->out_cap = n;
  }
  h->params_dirty = true;
  rc = sync_params(h);
  if (rc) return rc;
  int nf = 0;
  // Stage the inputs on the device (staging buffers grow only and are kept).
  const bool host = where == DPD_HOST;
  if (n > h->in_cap || !h->d_seen) {
    cudaFree(h->d_in4);
    cudaFree(h->d_in_id);
    cudaFree(h->d_in_type);
    cudaFree(h->d_seen);
    h->d_in4 = nullptr;
    h->d_in_id = nullptr;
    h->d_in_type = nullptr;
    h->d_seen = nullptr;
    h->in_cap = 0;
    const int cap = n > 1 ? n : 1;
    CU(h, dev_alloc(&h->d_in4, (size_t)2 * cap));
    CU(h, dev_alloc(&h->d_in_id, cap));
    CU(h, dev_alloc(&h->d_in_type, cap));
    CU(h, dev_alloc(&h->d_seen, cap));
    h->in_cap = cap;
  }
  float4 *in_pos = nullptr, *in_vel = nullptr;
  int* in_id = nullptr;
  uint8_t* in_type = nullptr;
  uint32_t* seen = h->d_seen;
  std::vector<uint8_t> host_type;
  if (host) {
    in_pos = h->d_in4;
    in_vel = h->d_in4 + n;
    in_id = h->d_in_id;
    in_type = h->d_in_type;
    CU(h, cudaMemcpyAsync(in_pos, pos4, sizeof(float4) * n, cudaMemcpyHostToDevice, E.stream));
    CU(h, cudaMemcpyAsync(in_vel, vel4, sizeof(float4) * n, cudaMemcpyHostToDevice, E.stream));
    CU(h, cudaMemcpyAsync(in_id, id, sizeof(int) * n, cudaMemcpyHostToDevice, E.stream));
    CU(h, cudaMemcpyAsync(in_type, type, n, cudaMemcpyHostToDevice, E.stream));
    for (int i = 0; i < n; ++i) nf += type[i] == 0;
  } else {
    in_pos = (float4*)pos4;
    in_vel = (float4*)vel4;
    in_id = (int*)id;
    in_type = (uint8_t*)type;
    host_type.resize(n);
    CU(h, cudaMemcpyAsync(host_type.data(), type, n, cudaMemcpyDeviceToHost, E.stream));
  }
  CU(h, cudaMemsetAsync(seen, 0, sizeof(uint32_t) * (n > 0 ? n : 1), E.stream));
  // the fixed-point sums start empty (their layout depends on n)
  if (n > 0) CU(h, cudaMemsetAsync(E.facc, 0, sizeof(unsigned long long) * 3 * (size_t)n, E.stream));
  // Status is cleared; the step counter is kept.
  CU(h, cudaMemsetAsync(&E.d_ctr[0].status, 0, sizeof(uint32_t), E.stream));
  E.cur = 0;
  dpd::launch_load(E.h_sys[0].P, in_pos, in_vel, in_id, in_type, E.arr[0], seen, n, E.d_ctr,
                   E.stream);
  dpd::engine_enqueue_sort(E);      // cell order into arr[1]
  dpd::engine_enqueue_force(E, 0);  // f(0) with vt = v(0)
  cudaError_t le = cudaGetLastError();
  cudaError_t se = cudaStreamSynchronize(E.stream);
  if (!host)
    for (int i = 0; i < n; ++i) nf += host_type[i] == 0;
  if (le != cudaSuccess) return fail(h, DPD_ECUDA, "launch failed: %s", cudaGetErrorString(le));
  if (se != cudaSuccess) return fail(h, DPD_ECUDA, "set-up failed: %s", cudaGetErrorString(se));
  uint32_t st = 0;
  rc = read_status(h, &st);
  if (rc) return rc;
  h->n_fluid = nf;
  h->loaded = st == 0;
  h->host_step = E.h_ctr[0].step;
  return dpd::engine_status_code(E, st);
}

int dpd_step(dpd_t* h, int nsteps) {
  if (!h) return DPD_EINVAL;
  if (nsteps < 0) return fail(h, DPD_EINVAL, "nsteps < 0");
  if (!h->loaded) return fail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  dpd::Engine& E = h->E;
  if (E.h_ctr[0].status) return dpd::engine_status_code(E, E.h_ctr[0].status);
  int rc = sync_params(h);
  if (rc) return rc;
  if (h->sample_every > 0 && h->prof_nbins > 0) {
    for (int k = 0; k < nsteps; ++k) {
      dpd::engine_enqueue_step(E);
      h->host_step += 1;
      if (h->host_step % (uint64_t)h->sample_every == 0) {
        rc = add_profile_sample(h);
        if (rc) return rc;
        E.launches += 1;
      }
    }
    CU(h, cudaGetLastError());
  } else {
    rc = dpd::engine_step(E, nsteps);
    if (rc) return rc;
    h->host_step += nsteps;
  }
  uint32_t st = 0;
  rc = read_status(h, &st);
  if (rc) return rc;
  return dpd::engine_status_code(E, st);
}

int dpd_time_phases(dpd_t* h, int nsteps, double* ms) {
  if (!h || !ms) return DPD_EINVAL;
  if (nsteps <= 0) return fail(h, DPD_EINVAL, "nsteps must be > 0");
  if (!h->loaded) return fail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  dpd::Engine& E = h->E;
  if (E.h_ctr[0].status) return dpd::engine_status_code(E, E.h_ctr[0].status);
  int rc = sync_params(h);
  if (rc) return rc;
  rc = dpd::engine_time_phases(E, nsteps, ms);
  h->host_step += nsteps;
  if (rc) return rc;
  uint32_t st = 0;
  rc = read_status(h, &st);
  if (rc) return rc;
  return dpd::engine_status_code(E, st);
}

int dpd_autotune(dpd_t* h, int nsteps, double* ms_per_variant, int* chosen) {
  if (!h) return DPD_EINVAL;
  if (nsteps <= 0) return fail(h, DPD_EINVAL, "nsteps must be > 0");
  if (!h->loaded) return fail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  int rc = sync_params(h);
  if (rc) return rc;
  rc = dpd::engine_autotune(h->E, nsteps, ms_per_variant, chosen);
  if (rc) return rc;
  uint32_t st = 0;
  rc = read_status(h, &st);
  if (rc) return rc;
  return dpd::engine_status_code(h->E, st);
}

int dpd_get_state(dpd_t* h, float* pos4, float* vel4, float* force4, int* id, uint8_t* type,
                  int where) {
  if (!h) return DPD_EINVAL;
  if (where != DPD_HOST && where != DPD_DEVICE) return fail(h, DPD_EINVAL, "bad `where`");
  if (!h->loaded) return fail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  dpd::Engine& E = h->E;
  const int n = E.n;
  dpd::engine_settle(E);
  const Arrays& A = E.arr[E.cur];
  if (where == DPD_DEVICE) {
    dpd::launch_unsort(A, n, (float4*)pos4, (float4*)vel4, (float4*)force4, id, type, E.stream);
    CU(h, cudaGetLastError());
    CU(h, cudaStreamSynchronize(E.stream));
    return DPD_OK;
  }
  float4* op = h->d_out4;
  float4* ov = h->d_out4 + n;
  float4* of = h->d_out4 + 2 * (size_t)n;
  dpd::launch_unsort(A, n, pos4 ? op : nullptr, vel4 ? ov : nullptr, force4 ? of : nullptr,
                     id ? h->d_out_id : nullptr, type ? h->d_out_type : nullptr, E.stream);
  CU(h, cudaGetLastError());
  if (pos4) CU(h, cudaMemcpyAsync(pos4, op, sizeof(float4) * n, cudaMemcpyDeviceToHost, E.stream));
  if (vel4) CU(h, cudaMemcpyAsync(vel4, ov, sizeof(float4) * n, cudaMemcpyDeviceToHost, E.stream));
  if (force4) CU(h, cudaMemcpyAsync(force4, of, sizeof(float4) * n, cudaMemcpyDeviceToHost, E.stream));
  if (id) CU(h, cudaMemcpyAsync(id, h->d_out_id, sizeof(int) * n, cudaMemcpyDeviceToHost, E.stream));
  if (type) CU(h, cudaMemcpyAsync(type, h->d_out_type, n, cudaMemcpyDeviceToHost, E.stream));
  CU(h, cudaStreamSynchronize(E.stream));
  return DPD_OK;
}

int dpd_velocity_profile(dpd_t* h, int axis, int nbins, double lo, double hi, double* out, int mode) {
  if (!h) return DPD_EINVAL;
  if (mode < 0 || mode > 3) return fail(h, DPD_EINVAL, "mode must be 0..3");
  dpd::Engine& E = h->E;
  if (mode == 1 || mode == 3 || h->prof_nbins == 0) {
    if (axis < 0 || axis > 2 || nbins <= 0 || !(hi > lo))
      return fail(h, DPD_EINVAL, "bad profile layout (axis %d, nbins %d, [%g, %g))", axis, nbins, lo, hi);
    if (nbins > h->prof_cap) {
      CU(h, cudaStreamSynchronize(E.stream));
      cudaFree(h->d_prof);
      h->d_prof = nullptr;
      h->prof_cap = 0;
      CU(h, dev_alloc(&h->d_prof, (size_t)5 * nbins));
      h->prof_cap = nbins;
    }
    h->prof_axis = axis;
    h->prof_nbins = nbins;
    h->prof_lo = lo;
    h->prof_hi = hi;
    CU(h, cudaMemsetAsync(h->d_prof, 0, sizeof(double) * 5 * nbins, E.stream));
  } else if (axis != h->prof_axis || nbins != h->prof_nbins || lo != h->prof_lo || hi != h->prof_hi) {
    return fail(h, DPD_EINVAL, "profile layout differs from the accumulated one (reset with mode 1)");
  }
  if (mode == 0 || mode == 1) {
    if (!h->loaded) return fail(h, DPD_ESTATE, "no particles to sample");
    int rc = add_profile_sample(h);
    if (rc) return rc;
  }
  if (mode != 3) {
    if (!out) return fail(h, DPD_EINVAL, "null output");
    CU(h, cudaMemcpyAsync(out, h->d_prof, sizeof(double) * 5 * nbins, cudaMemcpyDeviceToHost, E.stream));
  }
  CU(h, cudaStreamSynchronize(E.stream));
  return DPD_OK;
}

int dpd_get_stats(dpd_t* h, double out[8]) {
  if (!h || !out) return DPD_EINVAL;
  dpd::Engine& E = h->E;
  CU(h, cudaMemsetAsync(h->d_stats, 0, 8 * sizeof(double), E.stream));
  if (h->loaded) dpd::engine_settle(E);
  const Arrays& A = E.arr[E.cur];
  if (h->loaded) dpd::launch_stats(A.pos, A.vel, E.n, h->d_stats, E.stream);
  CU(h, cudaGetLastError());
  double s[8];
  CU(h, cudaMemcpyAsync(s, h->d_stats, 8 * sizeof(double), cudaMemcpyDeviceToHost, E.stream));
  uint32_t st = 0;
  int rc = read_status(h, &st);
  if (rc) return rc;
  for (int k = 0; k < 5; ++k) out[k] = s[k];
  out[5] = (double)E.h_ctr[0].reflections;
  out[6] = (double)E.h_ctr[0].fallbacks;
  out[7] = (double)E.h_ctr[0].step;
  return DPD_OK;
}

int dpd_set_option(dpd_t* h, const char* key, double v) {
  if (!h || !key) return DPD_EINVAL;
  if (!std::isfinite(v)) return fail(h, DPD_EINVAL, "option %s: value must be finite", key);
  const std::string k(key);
  dpd::Engine& E = h->E;
  dpd::engine_free_graphs(E);
  h->params_dirty = true;
  if (k == "lambda") {
    h->lambda = v;
  } else if (k == "a_ff") {
    h->a[0] = v;
  } else if (k == "a_fs") {
    h->a[1] = h->a[2] = v;
  } else if (k == "gamma") {
    if (v < 0) return fail(h, DPD_EINVAL, "gamma must be >= 0");
    h->gamma = v;
  } else if (k == "sigma") {
    if (v < 0) return fail(h, DPD_EINVAL, "sigma must be >= 0");
    h->sigma = v;
  } else if (k == "g_x" || k == "g_y" || k == "g_z") {
    h->g[k.back() - 'x'] = v;
  } else if (k == "band_margin") {
    if (!(v > 0.0) || v > 1.0) return fail(h, DPD_EINVAL, "band_margin must be in (0, 1]");
    h->margin = v;
    if (h->d_phi) {
      dpd::launch_band(dpd::make_params(h), h->d_band, E.stream);
      CU(h, cudaGetLastError());
      CU(h, cudaStreamSynchronize(E.stream));
    }
  } else if (k == "reflect_variant") {
    if (v != 0.0 && v != 1.0) return fail(h, DPD_EINVAL, "reflect_variant must be 0 or 1");
    h->reflect_variant = (int)v;
  } else if (k == "seed") {
    if (v < 0 || v > 9007199254740992.0 || v != std::floor(v))
      return fail(h, DPD_EINVAL, "seed must be an integer in [0, 2^53]");
    h->seed = (uint64_t)v;
  } else if (k == "system") {
    if (v < 0 || v > 4294967295.0 || v != std::floor(v)) return fail(h, DPD_EINVAL, "bad system index");
    h->sys = (uint32_t)v;
  } else if (k == "v_wall_x" || k == "v_wall_y" || k == "v_wall_z") {
    h->vw[k.back() - 'x'] = v;
  } else if (k == "shear_x" || k == "shear_y" || k == "shear_z") {
    const int c = k.back() - 'x';
    if (c == h->shear_axis && v != 0.0)
      return fail(h, DPD_EINVAL, "shear along its own axis would move the walls through the phase field");
    h->shear[c] = v;
  } else if (k == "shear_axis") {
    if (v != 0.0 && v != 1.0 && v != 2.0) return fail(h, DPD_EINVAL, "shear_axis must be 0, 1 or 2");
    if (h->shear[(int)v] != 0.0)
      return fail(h, DPD_EINVAL, "shear along its own axis would move the walls through the phase field");
    h->shear_axis = (int)v;
  } else if (k == "shear_ref") {
    h->shear_ref = v;
  } else if (k == "phase_eps") {
    if (!(v > 0.0)) return fail(h, DPD_EINVAL, "phase_eps must be > 0");
    h->phase_eps = v;
  } else if (k == "force_law") {
    if (v != 0.0 && v != 1.0) return fail(h, DPD_EINVAL, "force_law must be 0 or 1");
    h->force_law = (int)v;
  } else if (k == "S_r_ff" || k == "S_a_ff" || k == "S_r_fs" || k == "S_a_fs") {
    h->sph_S[(k[5] == 's' ? 2 : 0) + (k[2] == 'a' ? 1 : 0)] = v;
  } else if (k == "r0_r" || k == "r0_a") {
    if (!(v > 0.0) || v > 1.0) return fail(h, DPD_EINVAL, "%s must be in (0, 1] (the pair cutoff is 1)", key);
    h->sph_r0[k[3] == 'a' ? 1 : 0] = v;
  } else if (k == "sph_dim") {
    if (v != 1.0 && v != 2.0 && v != 3.0) return fail(h, DPD_EINVAL, "sph_dim must be 1, 2 or 3");
    h->sph_dim = (int)v;
  } else if (k == "sample_every") {
    if (v < 0 || v != std::floor(v)) return fail(h, DPD_EINVAL, "sample_every must be a whole number");
    h->sample_every = (int)v;
  } else if (k == "step") {
    if (v < 0 || v > 4294967295.0 || v != std::floor(v)) return fail(h, DPD_EINVAL, "bad step");
    const uint32_t s = (uint32_t)v;
    CU(h, cudaMemcpyAsync(&E.d_ctr[0].step, &s, sizeof s, cudaMemcpyHostToDevice, E.stream));
    CU(h, cudaStreamSynchronize(E.stream));
    E.h_ctr[0].step = s;
    h->host_step = s;
  } else if (k == "use_graph") {
    E.use_graph = v != 0.0;
  } else if (k == "force_variant") {
    if (v < 0 || v >= dpd::force_variants() || v != std::floor(v))
      return fail(h, DPD_EINVAL, "force_variant must be an integer in [0, %d)", dpd::force_variants());
    E.force_variant = (int)v;
  } else if (k == "graph_steps") {
    if (v < 2 || v > 1000 || v != std::floor(v) || ((int)v & 1))
      return fail(h, DPD_EINVAL, "graph_steps must be an even number in [2, 1000]");
    E.graph_steps = (int)v;
  } else if (k == "adjoint_tape_mb") {
    if (!(v >= 0.0)) return fail(h, DPD_EINVAL, "adjoint_tape_mb must be >= 0");
    h->adjoint_tape_mb = v;
    cudaFree(h->d_adj_ws);  // the next window sizes its workspace anew
    h->d_adj_ws = nullptr;
    h->adj_ws_bytes = 0;
  } else {
    return fail(h, DPD_EINVAL, "unknown option '%s'", key);
  }
  return DPD_OK;
}

int dpd_get_option(dpd_t* h, const char* key, double* v) {
  if (!h || !key || !v) return DPD_EINVAL;
  const std::string k(key);
  const dpd::Engine& E = h->E;
  if (k == "lambda") *v = h->lambda;
  else if (k == "a_ff") *v = h->a[0];
  else if (k == "a_fs") *v = h->a[1];
  else if (k == "gamma") *v = h->gamma;
  else if (k == "sigma") *v = h->sigma;
  else if (k == "kBT") *v = h->kBT;
  else if (k == "dt") *v = h->dt;
  else if (k == "g_x" || k == "g_y" || k == "g_z") *v = h->g[k.back() - 'x'];
  else if (k == "band_margin") *v = h->margin;
  else if (k == "reflect_variant") *v = h->reflect_variant;
  else if (k == "seed") *v = (double)h->seed;
  else if (k == "system") *v = h->sys;
  else if (k == "v_wall_x" || k == "v_wall_y" || k == "v_wall_z") *v = h->vw[k.back() - 'x'];
  else if (k == "shear_x" || k == "shear_y" || k == "shear_z") *v = h->shear[k.back() - 'x'];
  else if (k == "shear_axis") *v = h->shear_axis;
  else if (k == "shear_ref") *v = h->shear_ref;
  else if (k == "force_law") *v = h->force_law;
  else if (k == "phase_eps") *v = h->phase_eps;
  else if (k == "S_r_ff" || k == "S_a_ff" || k == "S_r_fs" || k == "S_a_fs")
    *v = h->sph_S[(k[5] == 's' ? 2 : 0) + (k[2] == 'a' ? 1 : 0)];
  else if (k == "r0_r" || k == "r0_a") *v = h->sph_r0[k[3] == 'a' ? 1 : 0];
  else if (k == "sph_dim") *v = h->sph_dim;
  else if (k == "sample_every") *v = h->sample_every;
  else if (k == "step") *v = (double)h->host_step;
  else if (k == "use_graph") *v = E.use_graph;
  else if (k == "graph_steps") *v = E.graph_steps;
  else if (k == "ncells") *v = h->ncells;
  else if (k == "kernel_launches") *v = (double)E.launches;
  else if (k == "kernels_per_step") *v = dpd::engine_kernels_per_step(E);
  else if (k == "force_variant") *v = E.force_variant;
  else if (k == "force_variants") *v = dpd::force_variants();
  else if (k == "force_newton3") *v = dpd::force_variant_newton3(E.force_variant);
  else if (k == "adjoint_tape_mb") *v = h->adjoint_tape_mb;
  else if (k == "scan_tiles") *v = dpd::scan_blocks(h->ncells);
  else return fail(h, DPD_EINVAL, "unknown option '%s'", key);
  return DPD_OK;
}

int dpd_num_particles(dpd_t* h, int* n, int* n_fluid) {
  if (!h) return DPD_EINVAL;
  if (n) *n = h->E.n;
  if (n_fluid) *n_fluid = h->n_fluid;
  return DPD_OK;
}

int dpd_set_stream(dpd_t* h, void* stream) {
  if (!h) return DPD_EINVAL;
  CU(h, cudaStreamSynchronize(h->E.stream));
  dpd::engine_free_graphs(h->E);
  h->E.stream = stream ? (cudaStream_t)stream : h->own_stream;
  return DPD_OK;
}

int dpd_destroy(dpd_t* h) {
  if (!h) return DPD_OK;
  dpd::engine_free(h->E);
  cudaFree(h->d_adj_ws);
  cudaFree(h->d_out4);
  cudaFree(h->d_out_id);
  cudaFree(h->d_out_type);
  cudaFree(h->d_in4);
  cudaFree(h->d_in_id);
  cudaFree(h->d_in_type);
  cudaFree(h->d_seen);
  cudaFree(h->d_phi);
  cudaFree(h->d_band);
  cudaFree(h->d_prof);
  cudaFree(h->d_stats);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return DPD_OK;
}

const char* dpd_last_error(const dpd_t* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
