// dpd_api.cu -- the C ABI of include/dpd.h: handle life cycle, device memory,
// and the order of kernel launches that makes one DPD time step (Xu & Meakin,
// arXiv:1807.09896, Sec. II).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dpd.h"
#include "dpd_common.cuh"
#include "dpd_launch.h"

using dpd::Arrays;
using dpd::CellList;
using dpd::DevCounters;
using dpd::StepParams;

struct dpd_system {
  // parameters
  double box[3] = {0, 0, 0};
  double rho = 3.0;
  double a[4] = {25, 25, 25, 25};
  double gamma = 4.5, sigma = 3.0, kBT = 1.0, dt = 0.01;
  double lambda = 0.65;
  double g[3] = {0, 0, 0};
  double vw[3] = {0, 0, 0};
  double margin = 0.5;
  uint64_t seed = 0;
  uint32_t sys = 0;
  int reflect_variant = 0;
  int sample_every = 0;
  int use_graph = 1;
  int graph_steps = 20;
  int force_variant = 0;
  int nc[3] = {0, 0, 0};
  int ncells = 0;
  // phase field
  float* d_phi = nullptr;
  int pd[3] = {0, 0, 0};
  double h = 0.0;
  uint8_t* d_band = nullptr;
  // particles
  int n = 0, n_fluid = 0, cap = 0;
  Arrays arr[2] = {};
  int cur = 0;
  CellList cl = {};
  int cl_cells = 0;
  float4* d_out4 = nullptr;  // staging for host reads: 3 x cap float4
  int* d_out_id = nullptr;
  uint8_t* d_out_type = nullptr;
  DevCounters* d_ctr = nullptr;
  DevCounters* h_ctr = nullptr;  // pinned
  double* d_prof = nullptr;
  int prof_cap = 0, prof_axis = 2, prof_nbins = 0;
  double prof_lo = 0, prof_hi = 0;
  double* d_stats = nullptr;
  uint64_t host_step = 0;
  bool loaded = false;
  // stream and graphs
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  uint64_t launches = 0;  // kernels enqueued by dpd_step (graph replays counted per kernel)
  std::string err;
};

// Kernels one time step enqueues: counter bump, drift/reflect/key, three scan
// passes, scatter, per-cell sort, gather, force.
static const int kKernelsPerStep = 9;

static std::string g_create_error;

namespace dpd {
// Message returned by dpd_last_error(NULL), for entry points without a handle.
void set_global_error(const char* msg) { g_create_error = msg; }
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

static void free_graphs(dpd_t* h) {
  for (auto& g : h->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

static void free_particles(dpd_t* h) {
  for (auto& A : h->arr) {
    cudaFree(A.pos);
    cudaFree(A.vt);
    cudaFree(A.vel);
    cudaFree(A.frc);
    A = Arrays{};
  }
  cudaFree(h->cl.key);
  cudaFree(h->cl.rank);
  cudaFree(h->cl.perm);
  cudaFree(h->d_out4);
  cudaFree(h->d_out_id);
  cudaFree(h->d_out_type);
  h->cl.key = h->cl.rank = h->cl.perm = nullptr;
  h->d_out4 = nullptr;
  h->d_out_id = nullptr;
  h->d_out_type = nullptr;
  h->cap = 0;
}

static StepParams make_params(const dpd_t* h) {
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
    P.pd[a] = h->pd[a];
  }
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
  P.sys = h->sys;
  P.reflect_variant = h->reflect_variant;
  P.margin = (float)h->margin;
  P.phi = h->d_phi;
  P.inv_h = h->h > 0 ? (float)(1.0 / h->h) : 0.0f;
  P.band = h->d_band;
  return P;
}

static int ensure_cells(dpd_t* h) {
  if (h->cl_cells == h->ncells && h->cl.count) return DPD_OK;
  cudaFree(h->cl.count);
  cudaFree(h->cl.start);
  cudaFree(h->cl.blocksum);
  CU(h, dev_alloc(&h->cl.count, (size_t)h->ncells));
  CU(h, dev_alloc(&h->cl.start, (size_t)h->ncells + 1));
  CU(h, dev_alloc(&h->cl.blocksum, (size_t)dpd::scan_blocks(h->ncells)));
  CU(h, cudaMemsetAsync(h->cl.count, 0, sizeof(uint32_t) * h->ncells, h->stream));
  h->cl_cells = h->ncells;
  return DPD_OK;
}

static int ensure_particles(dpd_t* h, int n) {
  if (n <= h->cap) return DPD_OK;
  free_particles(h);
  for (auto& A : h->arr) {
    CU(h, dev_alloc(&A.pos, n));
    CU(h, dev_alloc(&A.vt, n));
    CU(h, dev_alloc(&A.vel, n));
    CU(h, dev_alloc(&A.frc, n));
  }
  CU(h, dev_alloc(&h->cl.key, n));
  CU(h, dev_alloc(&h->cl.rank, n));
  CU(h, dev_alloc(&h->cl.perm, n));
  CU(h, dev_alloc(&h->d_out4, (size_t)3 * n));
  CU(h, dev_alloc(&h->d_out_id, n));
  CU(h, dev_alloc(&h->d_out_type, n));
  h->cap = n;
  return DPD_OK;
}

// One time step on the stream: counter bump, drift/reflect/key, scan, sort,
// force + closing kick.  Leaves the new state in arr[cur ^ 1].
static void enqueue_step(dpd_t* h, const StepParams& P, int cur) {
  const Arrays& A = h->arr[cur];
  const Arrays& B = h->arr[cur ^ 1];
  dpd::launch_bump_step(h->d_ctr, h->stream);
  dpd::launch_integrate(P, A, h->cl, h->n, h->d_ctr, h->stream);
  dpd::launch_scan(h->cl, h->ncells, h->n, h->stream);
  dpd::launch_sort(h->cl, A, B, h->n, h->ncells, h->d_ctr, h->stream);
  dpd::launch_force(P, B, h->cl.start, h->n, h->d_ctr, 1, h->force_variant, h->stream);
}

static int status_to_code(dpd_t* h, uint32_t st) {
  if (st == 0) return DPD_OK;
  if (st & dpd::ST_NAN) return fail(h, DPD_ENAN, "non-finite position, velocity or force");
  if (st & dpd::ST_LOST) return fail(h, DPD_ELOST, "a fluid particle is at phi < 0");
  if (st & dpd::ST_BADID) return fail(h, DPD_EINVAL, "ids are not a permutation of 0..n-1");
  if (st & dpd::ST_OVERFLOW) return fail(h, DPD_EOVERFLOW, "a cell holds more particles than the sort capacity");
  if (st & dpd::ST_BAND)
    return fail(h, DPD_EBAND, "a drift exceeded the band margin (%g); reduce dt or raise band_margin", h->margin);
  return fail(h, DPD_ECUDA, "unknown device status %#x", st);
}

static int read_counters(dpd_t* h) {
  CU(h, cudaMemcpyAsync(h->h_ctr, h->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return DPD_OK;
}

static int add_profile_sample(dpd_t* h) {
  if (h->prof_nbins <= 0) return DPD_OK;
  const float lo = (float)h->prof_lo;
  const float inv_w = (float)((double)h->prof_nbins / (h->prof_hi - h->prof_lo));
  const Arrays& A = h->arr[h->cur];
  dpd::launch_profile(A.pos, A.vel, h->n, h->prof_axis, h->prof_nbins, lo, inv_w, h->d_prof, h->stream);
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
  const long ncells = (long)h->nc[0] * h->nc[1] * h->nc[2];
  if (ncells > (1L << 30)) {
    delete h;
    return fail(nullptr, DPD_EOVERFLOW, "too many cells (%ld)", ncells);
  }
  h->ncells = (int)ncells;
  cudaError_t e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_ctr, sizeof(DevCounters));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_ctr, sizeof(DevCounters));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_stats, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->d_ctr, 0, sizeof(DevCounters));
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA set-up failed: ") + cudaGetErrorString(e);
    dpd_destroy(h);
    return DPD_ECUDA;
  }
  memset(h->h_ctr, 0, sizeof(DevCounters));
  h->stream = h->own_stream;
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
  free_graphs(h);
  cudaFree(h->d_phi);
  cudaFree(h->d_band);
  h->d_phi = nullptr;
  h->d_band = nullptr;
  CU(h, dev_alloc(&h->d_phi, nodes));
  CU(h, dev_alloc(&h->d_band, (size_t)h->ncells));
  CU(h, cudaMemcpyAsync(h->d_phi, grid, nodes * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  for (int a = 0; a < 3; ++a) h->pd[a] = dims[a];
  h->h = spacing;
  dpd::launch_band(make_params(h), h->d_band, h->stream);
  CU(h, cudaGetLastError());
  CU(h, cudaStreamSynchronize(h->stream));
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
  free_graphs(h);
  int rc = ensure_cells(h);
  if (rc) return rc;
  rc = ensure_particles(h, n);
  if (rc) return rc;
  int nf = 0;
  // Stage the inputs on the device.
  float4 *in_pos = nullptr, *in_vel = nullptr;
  int* in_id = nullptr;
  uint8_t* in_type = nullptr;
  uint32_t* seen = nullptr;
  std::vector<uint8_t> host_type;
  const bool host = where == DPD_HOST;
  CU(h, dev_alloc(&seen, n));
  if (host) {
    CU(h, dev_alloc(&in_pos, n));
    CU(h, dev_alloc(&in_vel, n));
    CU(h, dev_alloc(&in_id, n));
    CU(h, dev_alloc(&in_type, n));
    CU(h, cudaMemcpyAsync(in_pos, pos4, sizeof(float4) * n, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(in_vel, vel4, sizeof(float4) * n, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(in_id, id, sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(in_type, type, n, cudaMemcpyHostToDevice, h->stream));
    for (int i = 0; i < n; ++i) nf += type[i] == 0;
  } else {
    in_pos = (float4*)pos4;
    in_vel = (float4*)vel4;
    in_id = (int*)id;
    in_type = (uint8_t*)type;
    host_type.resize(n);
    CU(h, cudaMemcpyAsync(host_type.data(), type, n, cudaMemcpyDeviceToHost, h->stream));
  }
  CU(h, cudaMemsetAsync(seen, 0, sizeof(uint32_t) * (n > 0 ? n : 1), h->stream));
  CU(h, cudaMemsetAsync(h->cl.count, 0, sizeof(uint32_t) * h->ncells, h->stream));
  // Status is cleared; the step counter is kept.
  CU(h, cudaMemsetAsync(&h->d_ctr->status, 0, sizeof(uint32_t), h->stream));
  h->n = n;
  const StepParams P = make_params(h);
  Arrays& A = h->arr[0];
  dpd::launch_load(P, in_pos, in_vel, in_id, in_type, A, seen, n, h->d_ctr, h->stream);
  dpd::launch_key(P, A, h->cl, n, h->stream);
  dpd::launch_scan(h->cl, h->ncells, n, h->stream);
  dpd::launch_sort(h->cl, A, h->arr[1], n, h->ncells, h->d_ctr, h->stream);
  dpd::launch_force(P, h->arr[1], h->cl.start, n, h->d_ctr, 0, h->force_variant, h->stream);
  h->cur = 1;
  cudaError_t le = cudaGetLastError();
  cudaError_t se = cudaStreamSynchronize(h->stream);
  cudaFree(seen);
  if (host) {
    cudaFree(in_pos);
    cudaFree(in_vel);
    cudaFree(in_id);
    cudaFree(in_type);
  } else {
    for (int i = 0; i < n; ++i) nf += host_type[i] == 0;
  }
  if (le != cudaSuccess) return fail(h, DPD_ECUDA, "launch failed: %s", cudaGetErrorString(le));
  if (se != cudaSuccess) return fail(h, DPD_ECUDA, "set-up failed: %s", cudaGetErrorString(se));
  rc = read_counters(h);
  if (rc) return rc;
  h->n_fluid = nf;
  h->loaded = h->h_ctr->status == 0;
  h->host_step = h->h_ctr->step;
  return status_to_code(h, h->h_ctr->status);
}

static int build_graph(dpd_t* h, int cur) {
  const StepParams P = make_params(h);
  cudaGraph_t g = nullptr;
  CU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int c = cur;
  for (int k = 0; k < h->graph_steps; ++k) {
    enqueue_step(h, P, c);
    c ^= 1;
  }
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (e != cudaSuccess) return fail(h, DPD_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph[cur], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph[cur] = nullptr;
    return fail(h, DPD_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  return DPD_OK;
}

int dpd_step(dpd_t* h, int nsteps) {
  if (!h) return DPD_EINVAL;
  if (nsteps < 0) return fail(h, DPD_EINVAL, "nsteps < 0");
  if (!h->loaded) return fail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  if (h->h_ctr->status) return status_to_code(h, h->h_ctr->status);
  const StepParams P = make_params(h);
  int left = nsteps;
  while (left > 0) {
    const bool sample_due = h->sample_every > 0 && h->prof_nbins > 0;
    if (h->use_graph && !sample_due && left >= h->graph_steps) {
      if (!h->graph[h->cur]) {
        int rc = build_graph(h, h->cur);
        if (rc) return rc;
      }
      CU(h, cudaGraphLaunch(h->graph[h->cur], h->stream));
      h->launches += (uint64_t)kKernelsPerStep * h->graph_steps;
      // graph_steps is even: the state ends in the same buffer it started in
      h->host_step += h->graph_steps;
      left -= h->graph_steps;
      continue;
    }
    enqueue_step(h, P, h->cur);
    h->launches += kKernelsPerStep;
    h->cur ^= 1;
    h->host_step += 1;
    left -= 1;
    if (sample_due && h->host_step % (uint64_t)h->sample_every == 0) {
      int rc = add_profile_sample(h);
      if (rc) return rc;
      h->launches += 1;
    }
  }
  CU(h, cudaGetLastError());
  int rc = read_counters(h);
  if (rc) return rc;
  return status_to_code(h, h->h_ctr->status);
}

int dpd_time_phases(dpd_t* h, int nsteps, double* ms) {
  if (!h || !ms) return DPD_EINVAL;
  if (nsteps <= 0) return fail(h, DPD_EINVAL, "nsteps must be > 0");
  if (!h->loaded) return fail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  if (h->h_ctr->status) return status_to_code(h, h->h_ctr->status);
  const StepParams P = make_params(h);
  cudaEvent_t ev[DPD_NPHASES + 1];
  for (auto& e : ev) CU(h, cudaEventCreate(&e));
  double acc[DPD_NPHASES] = {0};
  int rc = DPD_OK;
  for (int k = 0; k < nsteps && rc == DPD_OK; ++k) {
    const Arrays& A = h->arr[h->cur];
    const Arrays& B = h->arr[h->cur ^ 1];
    cudaEventRecord(ev[0], h->stream);
    dpd::launch_bump_step(h->d_ctr, h->stream);
    dpd::launch_integrate(P, A, h->cl, h->n, h->d_ctr, h->stream);
    cudaEventRecord(ev[1], h->stream);
    dpd::launch_scan(h->cl, h->ncells, h->n, h->stream);
    cudaEventRecord(ev[2], h->stream);
    dpd::launch_sort(h->cl, A, B, h->n, h->ncells, h->d_ctr, h->stream);
    cudaEventRecord(ev[3], h->stream);
    dpd::launch_force(P, B, h->cl.start, h->n, h->d_ctr, 1, h->force_variant, h->stream);
    cudaEventRecord(ev[4], h->stream);
    h->launches += kKernelsPerStep;
    h->cur ^= 1;
    h->host_step += 1;
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) {
      rc = fail(h, DPD_ECUDA, "timed step failed: %s", cudaGetErrorString(e));
      break;
    }
    for (int q = 0; q < DPD_NPHASES; ++q) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
      acc[q] += t;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  for (int q = 0; q < DPD_NPHASES; ++q) ms[q] = acc[q] / nsteps;
  rc = read_counters(h);
  if (rc) return rc;
  return status_to_code(h, h->h_ctr->status);
}

int dpd_autotune(dpd_t* h, int nsteps, double* ms_per_variant, int* chosen) {
  if (!h) return DPD_EINVAL;
  if (nsteps <= 0) return fail(h, DPD_EINVAL, "nsteps must be > 0");
  if (!h->loaded) return fail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  const int nv = dpd::force_variants();
  int best = h->force_variant;
  double best_ms = 1e300;
  for (int v = 0; v < nv; ++v) {
    h->force_variant = v;
    double ms[DPD_NPHASES];
    int rc = dpd_time_phases(h, 1, ms);  // warm-up of this shape
    if (rc == DPD_OK) rc = dpd_time_phases(h, nsteps, ms);
    if (rc != DPD_OK) return rc;
    if (ms_per_variant) ms_per_variant[v] = ms[DPD_PHASE_FORCE];
    if (ms[DPD_PHASE_FORCE] < best_ms) {
      best_ms = ms[DPD_PHASE_FORCE];
      best = v;
    }
  }
  h->force_variant = best;
  free_graphs(h);
  if (chosen) *chosen = best;
  return DPD_OK;
}

int dpd_get_state(dpd_t* h, float* pos4, float* vel4, float* force4, int* id, uint8_t* type,
                  int where) {
  if (!h) return DPD_EINVAL;
  if (where != DPD_HOST && where != DPD_DEVICE) return fail(h, DPD_EINVAL, "bad `where`");
  if (!h->loaded) return fail(h, DPD_ESTATE, "no valid particle state (call dpd_set_particles)");
  const int n = h->n;
  const Arrays& A = h->arr[h->cur];
  if (where == DPD_DEVICE) {
    dpd::launch_unsort(A, n, (float4*)pos4, (float4*)vel4, (float4*)force4, id, type, h->stream);
    CU(h, cudaGetLastError());
    CU(h, cudaStreamSynchronize(h->stream));
    return DPD_OK;
  }
  float4* op = h->d_out4;
  float4* ov = h->d_out4 + n;
  float4* of = h->d_out4 + 2 * (size_t)n;
  dpd::launch_unsort(A, n, pos4 ? op : nullptr, vel4 ? ov : nullptr, force4 ? of : nullptr,
                     id ? h->d_out_id : nullptr, type ? h->d_out_type : nullptr, h->stream);
  CU(h, cudaGetLastError());
  if (pos4) CU(h, cudaMemcpyAsync(pos4, op, sizeof(float4) * n, cudaMemcpyDeviceToHost, h->stream));
  if (vel4) CU(h, cudaMemcpyAsync(vel4, ov, sizeof(float4) * n, cudaMemcpyDeviceToHost, h->stream));
  if (force4) CU(h, cudaMemcpyAsync(force4, of, sizeof(float4) * n, cudaMemcpyDeviceToHost, h->stream));
  if (id) CU(h, cudaMemcpyAsync(id, h->d_out_id, sizeof(int) * n, cudaMemcpyDeviceToHost, h->stream));
  if (type) CU(h, cudaMemcpyAsync(type, h->d_out_type, n, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return DPD_OK;
}

int dpd_velocity_profile(dpd_t* h, int axis, int nbins, double lo, double hi, double* out, int mode) {
  if (!h) return DPD_EINVAL;
  if (mode < 0 || mode > 3) return fail(h, DPD_EINVAL, "mode must be 0..3");
  if (mode == 1 || mode == 3 || h->prof_nbins == 0) {
    if (axis < 0 || axis > 2 || nbins <= 0 || !(hi > lo))
      return fail(h, DPD_EINVAL, "bad profile layout (axis %d, nbins %d, [%g, %g))", axis, nbins, lo, hi);
    if (nbins > h->prof_cap) {
      cudaFree(h->d_prof);
      h->d_prof = nullptr;
      h->prof_cap = 0;
      CU(h, dev_alloc(&h->d_prof, (size_t)5 * nbins));
      h->prof_cap = nbins;
    }
    free_graphs(h);
    h->prof_axis = axis;
    h->prof_nbins = nbins;
    h->prof_lo = lo;
    h->prof_hi = hi;
    CU(h, cudaMemsetAsync(h->d_prof, 0, sizeof(double) * 5 * nbins, h->stream));
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
    CU(h, cudaMemcpyAsync(out, h->d_prof, sizeof(double) * 5 * nbins, cudaMemcpyDeviceToHost, h->stream));
  }
  CU(h, cudaStreamSynchronize(h->stream));
  return DPD_OK;
}

int dpd_get_stats(dpd_t* h, double out[8]) {
  if (!h || !out) return DPD_EINVAL;
  CU(h, cudaMemsetAsync(h->d_stats, 0, 8 * sizeof(double), h->stream));
  const Arrays& A = h->arr[h->cur];
  if (h->loaded) dpd::launch_stats(A.pos, A.vel, h->n, h->d_stats, h->stream);
  CU(h, cudaGetLastError());
  double s[8];
  CU(h, cudaMemcpyAsync(s, h->d_stats, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  int rc = read_counters(h);
  if (rc) return rc;
  for (int k = 0; k < 5; ++k) out[k] = s[k];
  out[5] = (double)h->h_ctr->reflections;
  out[6] = (double)h->h_ctr->fallbacks;
  out[7] = (double)h->h_ctr->step;
  return DPD_OK;
}

int dpd_set_option(dpd_t* h, const char* key, double v) {
  if (!h || !key) return DPD_EINVAL;
  if (!std::isfinite(v)) return fail(h, DPD_EINVAL, "option %s: value must be finite", key);
  const std::string k(key);
  free_graphs(h);
  if (k == "lambda") {
    h->lambda = v;
  } else if (k == "band_margin") {
    if (!(v > 0.0) || v > 1.0) return fail(h, DPD_EINVAL, "band_margin must be in (0, 1]");
    h->margin = v;
    if (h->d_phi) {
      dpd::launch_band(make_params(h), h->d_band, h->stream);
      CU(h, cudaGetLastError());
      CU(h, cudaStreamSynchronize(h->stream));
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
  } else if (k == "sample_every") {
    if (v < 0 || v != std::floor(v)) return fail(h, DPD_EINVAL, "sample_every must be a whole number");
    h->sample_every = (int)v;
  } else if (k == "step") {
    if (v < 0 || v > 4294967295.0 || v != std::floor(v)) return fail(h, DPD_EINVAL, "bad step");
    const uint32_t s = (uint32_t)v;
    CU(h, cudaMemcpyAsync(&h->d_ctr->step, &s, sizeof s, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    h->host_step = s;
  } else if (k == "use_graph") {
    h->use_graph = v != 0.0;
  } else if (k == "force_variant") {
    if (v < 0 || v >= dpd::force_variants() || v != std::floor(v))
      return fail(h, DPD_EINVAL, "force_variant must be an integer in [0, %d)", dpd::force_variants());
    h->force_variant = (int)v;
  } else if (k == "graph_steps") {
    if (v < 2 || v > 1000 || v != std::floor(v) || ((int)v & 1))
      return fail(h, DPD_EINVAL, "graph_steps must be an even number in [2, 1000]");
    h->graph_steps = (int)v;
  } else {
    return fail(h, DPD_EINVAL, "unknown option '%s'", key);
  }
  return DPD_OK;
}

int dpd_get_option(dpd_t* h, const char* key, double* v) {
  if (!h || !key || !v) return DPD_EINVAL;
  const std::string k(key);
  if (k == "lambda") *v = h->lambda;
  else if (k == "band_margin") *v = h->margin;
  else if (k == "reflect_variant") *v = h->reflect_variant;
  else if (k == "seed") *v = (double)h->seed;
  else if (k == "system") *v = h->sys;
  else if (k == "v_wall_x" || k == "v_wall_y" || k == "v_wall_z") *v = h->vw[k.back() - 'x'];
  else if (k == "sample_every") *v = h->sample_every;
  else if (k == "step") *v = (double)h->host_step;
  else if (k == "use_graph") *v = h->use_graph;
  else if (k == "graph_steps") *v = h->graph_steps;
  else if (k == "ncells") *v = h->ncells;
  else if (k == "kernel_launches") *v = (double)h->launches;
  else if (k == "force_variant") *v = h->force_variant;
  else if (k == "force_variants") *v = dpd::force_variants();
  else if (k == "kernels_per_step") *v = kKernelsPerStep;
  else return fail(h, DPD_EINVAL, "unknown option '%s'", key);
  return DPD_OK;
}

int dpd_num_particles(dpd_t* h, int* n, int* n_fluid) {
  if (!h) return DPD_EINVAL;
  if (n) *n = h->n;
  if (n_fluid) *n_fluid = h->n_fluid;
  return DPD_OK;
}

int dpd_set_stream(dpd_t* h, void* stream) {
  if (!h) return DPD_EINVAL;
  CU(h, cudaStreamSynchronize(h->stream));
  free_graphs(h);
  h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  return DPD_OK;
}

int dpd_destroy(dpd_t* h) {
  if (!h) return DPD_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_graphs(h);
  free_particles(h);
  cudaFree(h->cl.count);
  cudaFree(h->cl.start);
  cudaFree(h->cl.blocksum);
  cudaFree(h->d_phi);
  cudaFree(h->d_band);
  cudaFree(h->d_ctr);
  cudaFree(h->d_prof);
  cudaFree(h->d_stats);
  if (h->h_ctr) cudaFreeHost(h->h_ctr);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return DPD_OK;
}

const char* dpd_last_error(const dpd_t* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
