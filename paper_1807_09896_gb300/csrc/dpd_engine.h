// dpd_engine.h -- the device state and launch sequence of DPD time steps for one
// or more independent systems held in concatenated arrays (internal).
//
// A single system (dpd_t) is an engine with one system; a batch (dpd_batch_t)
// is an engine with many.  Every phase of a step is one launch over all systems.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "dpd_common.cuh"

namespace dpd {

// Kernels of the reorder in one step: scatter, per-cell sort, gather.  A step also
// enqueues the drift (which advances the noise counter too), the scan passes and the
// force.
constexpr int kKernelsPerStepSort = 3;

struct Engine {
  int nsys = 0, n = 0, ncells = 0;
  int cap = 0, cell_cap = 0, sys_cap = 0;
  Arrays arr[2] = {};
  int cur = 0;  // arrays holding the current state
  CellList cl = {};
  SysDesc* d_sys = nullptr;
  std::vector<SysDesc> h_sys;
  DevCounters* d_ctr = nullptr;  // one per system
  DevCounters* h_ctr = nullptr;  // pinned mirror
  cudaStream_t stream = nullptr;
  // fixed-point pair-force sums of the Newton's-third-law force shapes: 3 per
  // particle, zero between steps (the finish kernel clears what it reads)
  unsigned long long* facc = nullptr;
  // step graphs by the buffers the state starts in and by whether its sums are pending
  // when the graph starts (its first drift differs); exit_pending: the mode it leaves
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool graph_exit_pending[2][2] = {{false, false}, {false, false}};
  // what the graphs were captured with (system 0's parameters travel by value in
  // the kernel arguments; sizes set the grids): a replay with anything else rebuilds
  StepParams graph_P = {};
  int graph_n = -1, graph_ncells = -1, graph_nsys = -1, graph_variant = -1, graph_len = -1;
  int use_graph = 1, graph_steps = 20, force_variant = 0;
  // the last step enqueued ran a Newton's-third-law force kernel and left its force in
  // the fixed-point sums for the next drift (which then runs in its pending form)
  bool sums_pending = false;
  uint64_t launches = 0;
  std::string* err = nullptr;  // where failure messages go
};

int engine_fail(Engine& E, int code, const char* fmt, ...);
// Kernels enqueued per step with the current force shape.
int engine_kernels_per_step(const Engine& E);
// Grow buffers to hold nsys systems, n particles and ncells cells (never shrinks).
int engine_reserve(Engine& E, int nsys, int n, int ncells);
// Copy the host system table to the device (waits for the copy).
int engine_upload_sys(Engine& E);
void engine_free_graphs(Engine& E);
void engine_free(Engine& E);
// Cell build of the state in arr[cur] into arr[cur ^ 1] (set-up, nothing moves).
void engine_enqueue_sort(Engine& E);
// Pair force on arr[cur]; kick = 1 adds dt/2 F(t+dt), completing the closing kick whose
// first half the drift kernel stored in vel.
void engine_enqueue_force(Engine& E, int kick);
// One full time step from arr[cur]; flips cur.  With a Newton's-third-law force shape
// the step leaves its force in the fixed-point sums for the next drift, unless
// finish is set (then the finish pass completes the state, as the adjoint needs).
void engine_enqueue_step(Engine& E, bool finish = false);
// Complete a state left pending by a step (finish pass); a no-op otherwise.  Every
// reader of the state between steps calls this first.
void engine_settle(Engine& E);
// nsteps steps, replayed from CUDA graphs where possible.  Does not wait.
int engine_step(Engine& E, int nsteps);
// nsteps steps launched one by one with events between phases; mean ms per phase.
int engine_time_phases(Engine& E, int nsteps, double* ms);
// Time every force launch shape; keep the fastest.
int engine_autotune(Engine& E, int nsteps, double* ms_per_variant, int* chosen);
// Copy the counters to the host (waits); *status = OR of every system's status.
int engine_read_counters(Engine& E, uint32_t* status);
// Error code and message for a non-zero status word.
int engine_status_code(Engine& E, uint32_t status);

}  // namespace dpd
