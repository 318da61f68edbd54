// dpd_engine.cu -- launch sequence of one DPD time step over one or more
// independent systems (Xu & Meakin, arXiv:1807.09896, Sec. II): counter bump,
// drift + reflection + cell key, scan, counting sort, pair force + closing kick.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "../../include/dpd.h"
#include "dpd_engine.h"
#include "dpd_launch.h"

namespace dpd {

int engine_fail(Engine& E, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (E.err) *E.err = buf;
  return code;
}

#define ECU(E, call)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return engine_fail((E), DPD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

template <typename T>
static cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

void engine_free_graphs(Engine& E) {
  for (auto& row : E.graph)
    for (auto& g : row) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

static void free_particle_buffers(Engine& E) {
  for (auto& A : E.arr) {
    cudaFree(A.pos);
    cudaFree(A.vt);
    cudaFree(A.vel);
    cudaFree(A.frc);
    A = Arrays{};
  }
  cudaFree(E.cl.key);
  cudaFree(E.cl.perm);
  cudaFree(E.facc);
  E.cl.key = E.cl.perm = nullptr;
  E.facc = nullptr;
  E.cap = 0;
}

static void free_cell_buffers(Engine& E) {
  cudaFree(E.cl.count);
  cudaFree(E.cl.start);
  cudaFree(E.cl.tile_total);
  E.cl.count = E.cl.start = nullptr;
  E.cl.tile_total = nullptr;
  E.cell_cap = 0;
}

void engine_free(Engine& E) {
  if (E.stream) cudaStreamSynchronize(E.stream);
  engine_free_graphs(E);
  free_particle_buffers(E);
  free_cell_buffers(E);
  cudaFree(E.d_sys);
  cudaFree(E.d_ctr);
  if (E.h_ctr) cudaFreeHost(E.h_ctr);
  E.d_sys = nullptr;
  E.d_ctr = nullptr;
  E.h_ctr = nullptr;
  E.sys_cap = 0;
}

int engine_reserve(Engine& E, int nsys, int n, int ncells) {
  if (nsys > E.sys_cap) {
    engine_free_graphs(E);
    cudaFree(E.d_sys);
    cudaFree(E.d_ctr);
    if (E.h_ctr) cudaFreeHost(E.h_ctr);
    E.d_sys = nullptr;
    E.d_ctr = nullptr;
    E.h_ctr = nullptr;
    E.sys_cap = 0;
    ECU(E, dev_alloc(&E.d_sys, nsys));
    ECU(E, dev_alloc(&E.d_ctr, nsys));
    ECU(E, cudaMallocHost((void**)&E.h_ctr, sizeof(DevCounters) * nsys));
    ECU(E, cudaMemsetAsync(E.d_ctr, 0, sizeof(DevCounters) * nsys, E.stream));
    memset(E.h_ctr, 0, sizeof(DevCounters) * nsys);
    E.sys_cap = nsys;
  }
  if (ncells > E.cell_cap) {
    engine_free_graphs(E);
    free_cell_buffers(E);
    ECU(E, dev_alloc(&E.cl.count, ncells));
    ECU(E, dev_alloc(&E.cl.start, (size_t)ncells + 1));
    ECU(E, dev_alloc(&E.cl.tile_total, tile_total_words(scan_blocks(ncells))));
    E.cell_cap = ncells;
  }
  if (n > E.cap) {
    engine_free_graphs(E);
    free_particle_buffers(E);
    for (auto& A : E.arr) {
      ECU(E, dev_alloc(&A.pos, (size_t)n + kPosPad));
      ECU(E, dev_alloc(&A.vt, n));
      ECU(E, dev_alloc(&A.vel, n));
      ECU(E, dev_alloc(&A.frc, n));
    }
    ECU(E, dev_alloc(&E.cl.key, n));
    ECU(E, dev_alloc(&E.cl.perm, n));
    ECU(E, dev_alloc(&E.facc, 3 * (size_t)n));
    ECU(E, cudaMemsetAsync(E.facc, 0, sizeof(unsigned long long) * 3 * (size_t)n, E.stream));
    E.cap = n;
  }
  E.nsys = nsys;
  E.n = n;
  E.ncells = ncells;
  // counts and tile totals must start at zero; every scan leaves them at zero
  ECU(E, cudaMemsetAsync(E.cl.count, 0, sizeof(uint32_t) * (ncells > 0 ? ncells : 1), E.stream));
  ECU(E, cudaMemsetAsync(E.cl.tile_total, 0, sizeof(uint32_t) * tile_total_words(scan_blocks(ncells)),
                         E.stream));
  return DPD_OK;
}

int engine_upload_sys(Engine& E) {
  ECU(E, cudaMemcpyAsync(E.d_sys, E.h_sys.data(), sizeof(SysDesc) * E.nsys, cudaMemcpyHostToDevice,
                         E.stream));
  ECU(E, cudaStreamSynchronize(E.stream));
  return DPD_OK;
}

void engine_enqueue_sort(Engine& E) {
  launch_key(E.d_sys, E.nsys, E.arr[E.cur], E.cl, E.n, E.stream);
  launch_scan(E.cl, E.ncells, E.n, E.stream);
  launch_sort(E.cl, E.arr[E.cur], E.arr[E.cur ^ 1], E.n, E.ncells, E.d_ctr, E.stream);
  E.cur ^= 1;
}

int engine_kernels_per_step(const Engine& E) {
  const int rest = E.n > 0 ? kKernelsPerStepSort + 1 : 0;
  return integrate_kernels(E.n, E.nsys) + scan_kernels(E.ncells) + rest;
}

void engine_enqueue_force(Engine& E, int kick) {
  launch_force(E.h_sys[0].P, E.d_sys, E.nsys, E.arr[E.cur], E.cl.start, E.facc, E.n, E.d_ctr, kick,
               E.force_variant, E.stream);
  E.sums_pending = false;
}

void engine_settle(Engine& E) {
  if (!E.sums_pending) return;
  launch_force_finish(E.h_sys[0].P, E.d_sys, E.nsys, E.arr[E.cur], E.facc, E.n, E.d_ctr, 1, E.stream);
  E.launches += 1;
  E.sums_pending = false;
}

// One step from arr[c] into arr[c ^ 1] (does not touch E.cur).  The drift completes
// whatever the previous step left pending (it reads the device flag).
static void enqueue_step_from(Engine& E, int c, bool finish) {
  const Arrays& A = E.arr[c];
  const Arrays& B = E.arr[c ^ 1];
  launch_integrate(E.h_sys[0].P, E.d_sys, E.nsys, A, E.cl, E.facc, E.sums_pending, E.n, E.d_ctr,
                   E.stream);
  launch_scan(E.cl, E.ncells, E.n, E.stream);
  launch_sort(E.cl, A, B, E.n, E.ncells, E.d_ctr, E.stream);
  launch_force_pairs(E.h_sys[0].P, E.d_sys, E.nsys, B, E.cl.start, E.facc, E.n, E.d_ctr, 1,
                     E.force_variant, E.stream);
  E.sums_pending = force_variant_newton3(E.force_variant);
  if (finish && E.sums_pending) {
    launch_force_finish(E.h_sys[0].P, E.d_sys, E.nsys, B, E.facc, E.n, E.d_ctr, 1, E.stream);
    E.launches += 1;
    E.sums_pending = false;
  }
}

void engine_enqueue_step(Engine& E, bool finish) {
  enqueue_step_from(E, E.cur, finish);
  E.cur ^= 1;
  E.launches += engine_kernels_per_step(E);
}

// Capture graph_steps steps from arr[c], entered with the sums in mode m.
static int build_graph(Engine& E, int c, int m) {
  cudaGraph_t g = nullptr;
  const bool entry = E.sums_pending;
  ECU(E, cudaStreamBeginCapture(E.stream, cudaStreamCaptureModeThreadLocal));
  int cc = c;
  for (int k = 0; k < E.graph_steps; ++k) {
    enqueue_step_from(E, cc, false);
    cc ^= 1;
  }
  E.graph_exit_pending[c][m] = E.sums_pending;
  E.sums_pending = entry;  // nothing ran yet: the replay below moves the state on
  cudaError_t e = cudaStreamEndCapture(E.stream, &g);
  if (e != cudaSuccess)
    return engine_fail(E, DPD_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&E.graph[c][m], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    E.graph[c][m] = nullptr;
    return engine_fail(E, DPD_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  return DPD_OK;
}

static bool any_graph(const Engine& E) {
  for (const auto& row : E.graph)
    for (const auto g : row)
      if (g) return true;
  return false;
}

// True if the captured graphs were built for the engine as it is now.
static bool graph_key_matches(const Engine& E) {
  return E.graph_n == E.n && E.graph_ncells == E.ncells && E.graph_nsys == E.nsys &&
         E.graph_variant == E.force_variant && E.graph_len == E.graph_steps && !E.h_sys.empty() &&
         memcmp(&E.graph_P, &E.h_sys[0].P, sizeof(StepParams)) == 0;
}

int engine_step(Engine& E, int nsteps) {
  if (any_graph(E) && !graph_key_matches(E)) engine_free_graphs(E);
  int left = nsteps;
  while (left > 0) {
    if (E.use_graph && left >= E.graph_steps) {
      const int m = E.sums_pending ? 1 : 0;
      if (!E.graph[E.cur][m]) {
        const int rc = build_graph(E, E.cur, m);
        if (rc) return rc;
        memcpy(&E.graph_P, &E.h_sys[0].P, sizeof(StepParams));
        E.graph_n = E.n;
        E.graph_ncells = E.ncells;
        E.graph_nsys = E.nsys;
        E.graph_variant = E.force_variant;
        E.graph_len = E.graph_steps;
      }
      ECU(E, cudaGraphLaunch(E.graph[E.cur][m], E.stream));
      E.sums_pending = E.graph_exit_pending[E.cur][m];
      // graph_steps is even: the state ends in the buffers it started in
      E.launches += (uint64_t)engine_kernels_per_step(E) * E.graph_steps;
      left -= E.graph_steps;
      continue;
    }
    engine_enqueue_step(E);
    left -= 1;
  }
  ECU(E, cudaGetLastError());
  return DPD_OK;
}

int engine_time_phases(Engine& E, int nsteps, double* ms) {
  cudaEvent_t ev[DPD_NPHASES + 1];
  for (auto& e : ev) ECU(E, cudaEventCreate(&e));
  double acc[DPD_NPHASES] = {0};
  int rc = DPD_OK;
  for (int k = 0; k < nsteps && rc == DPD_OK; ++k) {
    const Arrays& A = E.arr[E.cur];
    const Arrays& B = E.arr[E.cur ^ 1];
    cudaEventRecord(ev[0], E.stream);
    launch_integrate(E.h_sys[0].P, E.d_sys, E.nsys, A, E.cl, E.facc, E.sums_pending, E.n, E.d_ctr,
                     E.stream);
    cudaEventRecord(ev[1], E.stream);
    launch_scan(E.cl, E.ncells, E.n, E.stream);
    cudaEventRecord(ev[2], E.stream);
    launch_scatter(E.cl, E.n, E.ncells, E.d_ctr, E.stream);
    cudaEventRecord(ev[3], E.stream);
    launch_cell_sort(E.cl, E.n, E.ncells, E.d_ctr, E.stream);
    cudaEventRecord(ev[4], E.stream);
    launch_gather(E.cl, A, B, E.n, E.stream);
    cudaEventRecord(ev[5], E.stream);
    launch_force_pairs(E.h_sys[0].P, E.d_sys, E.nsys, B, E.cl.start, E.facc, E.n, E.d_ctr, 1,
                       E.force_variant, E.stream);
    E.sums_pending = force_variant_newton3(E.force_variant);
    cudaEventRecord(ev[6], E.stream);
    // a step launches no finish pass (the next drift does its work): the phase stays
    // in the table, empty, so that the phases of older builds can be compared
    cudaEventRecord(ev[DPD_NPHASES], E.stream);
    E.launches += engine_kernels_per_step(E);
    E.cur ^= 1;
    const cudaError_t e = cudaEventSynchronize(ev[DPD_NPHASES]);
    if (e != cudaSuccess) {
      rc = engine_fail(E, DPD_ECUDA, "timed step failed: %s", cudaGetErrorString(e));
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
  return DPD_OK;
}

int engine_autotune(Engine& E, int nsteps, double* ms_per_variant, int* chosen) {
  const int nv = force_variants();
  // The timing steps must leave no trace: the shapes of the two force algorithms
  // round differently, so the state and counters are kept and put back afterwards
  // (from a complete state: no sums pending).
  engine_settle(E);
  Arrays keep{};
  DevCounters* keep_ctr = nullptr;
  const size_t n = (size_t)E.n;
  ECU(E, dev_alloc(&keep.pos, n));
  ECU(E, dev_alloc(&keep.vt, n));
  ECU(E, dev_alloc(&keep.vel, n));
  ECU(E, dev_alloc(&keep.frc, n));
  ECU(E, dev_alloc(&keep_ctr, (size_t)E.nsys));
  auto copy_state = [&](const Arrays& from, const Arrays& to, const DevCounters* cf, DevCounters* ct) {
    const size_t b = sizeof(float4) * n;
    cudaMemcpyAsync(to.pos, from.pos, b, cudaMemcpyDeviceToDevice, E.stream);
    cudaMemcpyAsync(to.vt, from.vt, b, cudaMemcpyDeviceToDevice, E.stream);
    cudaMemcpyAsync(to.vel, from.vel, b, cudaMemcpyDeviceToDevice, E.stream);
    cudaMemcpyAsync(to.frc, from.frc, b, cudaMemcpyDeviceToDevice, E.stream);
    return cudaMemcpyAsync(ct, cf, sizeof(DevCounters) * E.nsys, cudaMemcpyDeviceToDevice, E.stream);
  };
  int rc = DPD_OK;
  cudaError_t e = copy_state(E.arr[E.cur], keep, E.d_ctr, keep_ctr);
  if (e != cudaSuccess) rc = engine_fail(E, DPD_ECUDA, "autotune: %s", cudaGetErrorString(e));
  const int start_variant = E.force_variant;
  int best = start_variant;
  double best_ms = 1e300;
  for (int v = 0; v < nv && rc == DPD_OK; ++v) {
    E.force_variant = v;
    double ms[DPD_NPHASES];
    rc = engine_time_phases(E, 1, ms);  // warm-up of this shape
    if (rc == DPD_OK) rc = engine_time_phases(E, nsteps, ms);
    engine_settle(E);
    if (rc != DPD_OK) break;
    // whole steps: the Newton's-third-law shapes move the conversion of their sums
    // into the next drift
    double step_ms = 0.0;
    for (int q = 0; q < DPD_NPHASES; ++q) step_ms += ms[q];
    if (ms_per_variant) ms_per_variant[v] = step_ms;
    if (step_ms < best_ms) {
      best_ms = step_ms;
      best = v;
    }
  }
  if (rc == DPD_OK) {
    e = copy_state(keep, E.arr[E.cur], keep_ctr, E.d_ctr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    if (e != cudaSuccess) rc = engine_fail(E, DPD_ECUDA, "autotune: %s", cudaGetErrorString(e));
  } else {
    cudaStreamSynchronize(E.stream);
  }
  cudaFree(keep.pos);
  cudaFree(keep.vt);
  cudaFree(keep.vel);
  cudaFree(keep.frc);
  cudaFree(keep_ctr);
  E.force_variant = rc == DPD_OK ? best : start_variant;
  engine_free_graphs(E);
  if (rc != DPD_OK) return rc;
  if (chosen) *chosen = best;
  return DPD_OK;
}

int engine_read_counters(Engine& E, uint32_t* status) {
  ECU(E, cudaMemcpyAsync(E.h_ctr, E.d_ctr, sizeof(DevCounters) * E.nsys, cudaMemcpyDeviceToHost,
                         E.stream));
  ECU(E, cudaStreamSynchronize(E.stream));
  uint32_t st = 0;
  for (int k = 0; k < E.nsys; ++k) st |= E.h_ctr[k].status;
  *status = st;
  return DPD_OK;
}

int engine_status_code(Engine& E, uint32_t st) {
  if (st == 0) return DPD_OK;
  if (st & ST_NAN) return engine_fail(E, DPD_ENAN, "non-finite position, velocity or force");
  if (st & ST_LOST) return engine_fail(E, DPD_ELOST, "a fluid particle is at phi < 0");
  if (st & ST_BADID) return engine_fail(E, DPD_EINVAL, "ids are not a permutation of 0..n-1");
  if (st & ST_OVERFLOW)
    return engine_fail(E, DPD_EOVERFLOW, "a cell holds more particles than the sort capacity");
  if (st & ST_BAND)
    return engine_fail(E, DPD_EBAND,
                       "a drift exceeded the band margin; reduce dt or raise band_margin");
  return engine_fail(E, DPD_ECUDA, "unknown device status %#x", st);
}

}  // namespace dpd
