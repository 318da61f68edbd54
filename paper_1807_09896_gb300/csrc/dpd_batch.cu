// dpd_batch.cu -- many independent DPD systems advanced together: their
// particles and cells are concatenated and every phase of a time step is one
// launch over all of them, replayed from a CUDA graph.  Each system keeps its own
// box, phase field, parameters, noise key and step counter, so a system
// advanced in a batch follows exactly the trajectory it follows alone.
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
using dpd::SysDesc;

struct dpd_batch {
  std::vector<dpd_t*> members;
  std::vector<int> n_fluid;
  dpd::Engine E;
  float4* d_out4 = nullptr;
  int* d_out_id = nullptr;
  uint8_t* d_out_type = nullptr;
  double* d_stats = nullptr;
  int out_cap = 0;
  cudaStream_t own_stream = nullptr;
  std::string err;
};

static std::string g_batch_error;

static int bfail(dpd_batch_t* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b)
    b->err = buf;
  else
    g_batch_error = buf;
  return code;
}

#define BCU(b, call)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bfail((b), DPD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

static Arrays offset(const Arrays& A, size_t off) {
  return Arrays{A.pos + off, A.vt + off, A.vel + off, A.frc + off};
}

static int batch_status(dpd_batch_t* b) {
  uint32_t st = 0;
  int rc = dpd::engine_read_counters(b->E, &st);
  if (rc) return rc;
  return dpd::engine_status_code(b->E, st);
}

extern "C" {

int dpd_batch_create(dpd_batch_t** out, int nsys, dpd_t* const* systems) {
  if (!out || !systems || nsys < 1) return bfail(nullptr, DPD_EINVAL, "need nsys >= 1 systems");
  *out = nullptr;
  long n_total = 0, cells_total = 0;
  for (int k = 0; k < nsys; ++k) {
    dpd_t* h = systems[k];
    if (!h) return bfail(nullptr, DPD_EINVAL, "system %d is NULL", k);
    if (!h->loaded) return bfail(nullptr, DPD_ESTATE, "system %d has no valid particle state", k);
    if (h->E.h_ctr[0].status) return bfail(nullptr, DPD_ESTATE, "system %d has a pending error", k);
    if (h->force_law != systems[0]->force_law)
      return bfail(nullptr, DPD_EINVAL, "system %d uses another force law than system 0", k);
    for (int q = 0; q < k; ++q)
      if (systems[q] == h) return bfail(nullptr, DPD_EINVAL, "system %d appears twice", k);
    n_total += h->E.n;
    cells_total += h->ncells;
  }
  if (n_total >= (1L << 30) || cells_total >= (1L << 30))
    return bfail(nullptr, DPD_EOVERFLOW, "batch too large (%ld particles, %ld cells)", n_total, cells_total);
  dpd_batch_t* b = new (std::nothrow) dpd_batch();
  if (!b) return bfail(nullptr, DPD_ENOMEM, "out of host memory");
  b->E.err = &b->err;
  cudaError_t e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_stats, 8 * sizeof(double));
  if (e != cudaSuccess) {
    g_batch_error = std::string("CUDA set-up failed: ") + cudaGetErrorString(e);
    dpd_batch_destroy(b);
    return DPD_ECUDA;
  }
  b->E.stream = b->own_stream;
  dpd::Engine& E = b->E;
  int rc = dpd::engine_reserve(E, nsys, (int)n_total, (int)cells_total);
  if (rc) {
    g_batch_error = b->err;
    dpd_batch_destroy(b);
    return rc;
  }
  E.h_sys.resize(nsys);
  uint32_t poff = 0, coff = 0;
  int nmax = 0;
  for (int k = 0; k < nsys; ++k) {
    dpd_t* h = systems[k];
    SysDesc& S = E.h_sys[k];
    S.P = dpd::make_params(h);
    S.cell_off = coff;
    S.part_off = poff;
    S.n = (uint32_t)h->E.n;
    S.pad = 0;
    // bring the system's state into the batch (complete, from its own stream)
    dpd::engine_settle(h->E);
    cudaStreamSynchronize(h->E.stream);
    const Arrays src = h->E.arr[h->E.cur];
    const Arrays dst = offset(E.arr[0], poff);
    const size_t bytes = sizeof(float4) * (size_t)h->E.n;
    if (bytes) {
      BCU(b, cudaMemcpyAsync(dst.pos, src.pos, bytes, cudaMemcpyDeviceToDevice, E.stream));
      BCU(b, cudaMemcpyAsync(dst.vt, src.vt, bytes, cudaMemcpyDeviceToDevice, E.stream));
      BCU(b, cudaMemcpyAsync(dst.vel, src.vel, bytes, cudaMemcpyDeviceToDevice, E.stream));
      BCU(b, cudaMemcpyAsync(dst.frc, src.frc, bytes, cudaMemcpyDeviceToDevice, E.stream));
    }
    BCU(b, cudaMemcpyAsync(E.d_ctr + k, h->E.d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToDevice,
                           E.stream));
    b->members.push_back(h);
    b->n_fluid.push_back(h->n_fluid);
    poff += S.n;
    coff += (uint32_t)h->ncells;
    if (h->E.n > nmax) nmax = h->E.n;
  }
  E.cur = 0;
  rc = dpd::engine_upload_sys(E);
  if (rc == DPD_OK) {
    e = cudaMalloc((void**)&b->d_out4, sizeof(float4) * 3 * (size_t)(nmax > 0 ? nmax : 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_out_id, sizeof(int) * (nmax > 0 ? nmax : 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_out_type, (nmax > 0 ? nmax : 1));
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    if (e != cudaSuccess) rc = bfail(b, DPD_ECUDA, "batch set-up failed: %s", cudaGetErrorString(e));
  }
  if (rc) {
    g_batch_error = b->err;
    dpd_batch_destroy(b);
    return rc;
  }
  b->out_cap = nmax;
  uint32_t st = 0;
  rc = dpd::engine_read_counters(E, &st);
  if (rc) {
    g_batch_error = b->err;
    dpd_batch_destroy(b);
    return rc;
  }
  *out = b;
  return DPD_OK;
}

int dpd_batch_step(dpd_batch_t* b, int nsteps) {
  if (!b) return DPD_EINVAL;
  if (nsteps < 0) return bfail(b, DPD_EINVAL, "nsteps < 0");
  for (int k = 0; k < b->E.nsys; ++k)
    if (b->E.h_ctr[k].status) return dpd::engine_status_code(b->E, b->E.h_ctr[k].status);
  int rc = dpd::engine_step(b->E, nsteps);
  if (rc) return rc;
  return batch_status(b);
}

int dpd_batch_time_phases(dpd_batch_t* b, int nsteps, double* ms) {
  if (!b || !ms) return DPD_EINVAL;
  if (nsteps <= 0) return bfail(b, DPD_EINVAL, "nsteps must be > 0");
  int rc = dpd::engine_time_phases(b->E, nsteps, ms);
  if (rc) return rc;
  return batch_status(b);
}

int dpd_batch_autotune(dpd_batch_t* b, int nsteps, double* ms_per_variant, int* chosen) {
  if (!b) return DPD_EINVAL;
  if (nsteps <= 0) return bfail(b, DPD_EINVAL, "nsteps must be > 0");
  int rc = dpd::engine_autotune(b->E, nsteps, ms_per_variant, chosen);
  if (rc) return rc;
  return batch_status(b);
}

int dpd_batch_get_state(dpd_batch_t* b, int k, float* pos4, float* vel4, float* force4, int* id,
                        uint8_t* type, int where) {
  if (!b) return DPD_EINVAL;
  dpd::Engine& E = b->E;
  if (k < 0 || k >= E.nsys) return bfail(b, DPD_EINVAL, "system index %d out of range", k);
  if (where != DPD_HOST && where != DPD_DEVICE) return bfail(b, DPD_EINVAL, "bad `where`");
  const int n = (int)E.h_sys[k].n;
  dpd::engine_settle(E);
  const Arrays A = offset(E.arr[E.cur], E.h_sys[k].part_off);
  if (where == DPD_DEVICE) {
    dpd::launch_unsort(A, n, (float4*)pos4, (float4*)vel4, (float4*)force4, id, type, E.stream);
    BCU(b, cudaGetLastError());
    BCU(b, cudaStreamSynchronize(E.stream));
    return DPD_OK;
  }
  float4* op = b->d_out4;
  float4* ov = b->d_out4 + n;
  float4* of = b->d_out4 + 2 * (size_t)n;
  dpd::launch_unsort(A, n, pos4 ? op : nullptr, vel4 ? ov : nullptr, force4 ? of : nullptr,
                     id ? b->d_out_id : nullptr, type ? b->d_out_type : nullptr, E.stream);
  BCU(b, cudaGetLastError());
  if (pos4) BCU(b, cudaMemcpyAsync(pos4, op, sizeof(float4) * n, cudaMemcpyDeviceToHost, E.stream));
  if (vel4) BCU(b, cudaMemcpyAsync(vel4, ov, sizeof(float4) * n, cudaMemcpyDeviceToHost, E.stream));
  if (force4) BCU(b, cudaMemcpyAsync(force4, of, sizeof(float4) * n, cudaMemcpyDeviceToHost, E.stream));
  if (id) BCU(b, cudaMemcpyAsync(id, b->d_out_id, sizeof(int) * n, cudaMemcpyDeviceToHost, E.stream));
  if (type) BCU(b, cudaMemcpyAsync(type, b->d_out_type, n, cudaMemcpyDeviceToHost, E.stream));
  BCU(b, cudaStreamSynchronize(E.stream));
  return DPD_OK;
}

int dpd_batch_get_stats(dpd_batch_t* b, int k, double out[8]) {
  if (!b || !out) return DPD_EINVAL;
  dpd::Engine& E = b->E;
  if (k < 0 || k >= E.nsys) return bfail(b, DPD_EINVAL, "system index %d out of range", k);
  BCU(b, cudaMemsetAsync(b->d_stats, 0, 8 * sizeof(double), E.stream));
  dpd::engine_settle(E);
  const Arrays A = offset(E.arr[E.cur], E.h_sys[k].part_off);
  dpd::launch_stats(A.pos, A.vel, (int)E.h_sys[k].n, b->d_stats, E.stream);
  BCU(b, cudaGetLastError());
  double s[8];
  BCU(b, cudaMemcpyAsync(s, b->d_stats, 8 * sizeof(double), cudaMemcpyDeviceToHost, E.stream));
  uint32_t st = 0;
  int rc = dpd::engine_read_counters(E, &st);
  if (rc) return rc;
  for (int q = 0; q < 5; ++q) out[q] = s[q];
  out[5] = (double)E.h_ctr[k].reflections;
  out[6] = (double)E.h_ctr[k].fallbacks;
  out[7] = (double)E.h_ctr[k].step;
  return DPD_OK;
}

int dpd_batch_set_option(dpd_batch_t* b, const char* key, double v) {
  if (!b || !key) return DPD_EINVAL;
  if (!std::isfinite(v)) return bfail(b, DPD_EINVAL, "option %s: value must be finite", key);
  const std::string k(key);
  dpd::Engine& E = b->E;
  dpd::engine_free_graphs(E);
  if (k == "use_graph") {
    E.use_graph = v != 0.0;
  } else if (k == "force_variant") {
    if (v < 0 || v >= dpd::force_variants() || v != std::floor(v))
      return bfail(b, DPD_EINVAL, "force_variant must be an integer in [0, %d)", dpd::force_variants());
    E.force_variant = (int)v;
  } else if (k == "graph_steps") {
    if (v < 2 || v > 1000 || v != std::floor(v) || ((int)v & 1))
      return bfail(b, DPD_EINVAL, "graph_steps must be an even number in [2, 1000]");
    E.graph_steps = (int)v;
  } else {
    return bfail(b, DPD_EINVAL, "unknown batch option '%s'", key);
  }
  return DPD_OK;
}

int dpd_batch_get_option(dpd_batch_t* b, const char* key, double* v) {
  if (!b || !key || !v) return DPD_EINVAL;
  const std::string k(key);
  const dpd::Engine& E = b->E;
  if (k == "use_graph") *v = E.use_graph;
  else if (k == "graph_steps") *v = E.graph_steps;
  else if (k == "force_variant") *v = E.force_variant;
  else if (k == "force_variants") *v = dpd::force_variants();
  else if (k == "force_newton3") *v = dpd::force_variant_newton3(E.force_variant);
  else if (k == "kernel_launches") *v = (double)E.launches;
  else if (k == "kernels_per_step") *v = dpd::engine_kernels_per_step(E);
  else if (k == "nsys") *v = E.nsys;
  else if (k == "n") *v = E.n;
  else if (k == "ncells") *v = E.ncells;
  else return bfail(b, DPD_EINVAL, "unknown batch option '%s'", key);
  return DPD_OK;
}

int dpd_batch_num_particles(dpd_batch_t* b, int k, int* n, int* n_fluid) {
  if (!b) return DPD_EINVAL;
  if (k < 0 || k >= b->E.nsys) return bfail(b, DPD_EINVAL, "system index %d out of range", k);
  if (n) *n = (int)b->E.h_sys[k].n;
  if (n_fluid) *n_fluid = b->n_fluid[k];
  return DPD_OK;
}

int dpd_batch_set_stream(dpd_batch_t* b, void* stream) {
  if (!b) return DPD_EINVAL;
  BCU(b, cudaStreamSynchronize(b->E.stream));
  dpd::engine_free_graphs(b->E);
  b->E.stream = stream ? (cudaStream_t)stream : b->own_stream;
  return DPD_OK;
}

int dpd_batch_destroy(dpd_batch_t* b) {
  if (!b) return DPD_OK;
  dpd::engine_free(b->E);
  cudaFree(b->d_out4);
  cudaFree(b->d_out_id);
  cudaFree(b->d_out_type);
  cudaFree(b->d_stats);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
  return DPD_OK;
}

const char* dpd_batch_last_error(const dpd_batch_t* b) {
  return b ? b->err.c_str() : g_batch_error.c_str();
}

}  // extern "C"
