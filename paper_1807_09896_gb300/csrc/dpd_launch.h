// dpd_launch.h -- host-side launch wrappers of the DPD kernels (internal).
#pragma once

#include "dpd_common.cuh"

namespace dpd {

// Drift, reflection and cell key of every particle, after advancing each system's
// noise counter (inside the drift launch when nsys <= n, else by a launch of its own).
// P0: parameters of system 0, used directly when nsys == 1.
// pending: the state was left by a Newton's-third-law force kernel, its force still in
// the fixed-point sums facc, which the drift converts (and clears) first.
void launch_integrate(const StepParams& P0, const SysDesc* S, int nsys, const Arrays& A,
                      const CellList& C, unsigned long long* facc, bool pending, int n,
                      DevCounters* ctr, cudaStream_t s);
void launch_key(const SysDesc* S, int nsys, const Arrays& A, const CellList& C, int n,
                cudaStream_t s);
// Kernels one launch_integrate enqueues.
int integrate_kernels(int n, int nsys);
// Tiles of the cell scan (one block each).
int scan_blocks(int ncells);
// Kernels one launch_scan enqueues (one: the scan is a single pass).
int scan_kernels(int ncells);
// Exclusive scan of the cell counts into start (and counts cleared), from the counts
// and the tile totals the drift (or launch_key) left; no block waits on another.
void launch_scan(const CellList& C, int ncells, int n, cudaStream_t s);
// Reorder into cell order: scatter, per-cell sort, gather (launch_sort = all three).
void launch_sort(const CellList& C, const Arrays& src, const Arrays& dst, int n, int ncells,
                 DevCounters* ctr, cudaStream_t s);
void launch_scatter(const CellList& C, int n, int ncells, DevCounters* ctr, cudaStream_t s);
void launch_cell_sort(const CellList& C, int n, int ncells, DevCounters* ctr, cudaStream_t s);
void launch_gather(const CellList& C, const Arrays& src, const Arrays& dst, int n, cudaStream_t s);
// Pair force of the given launch shape; launch_force = the pair kernel, then (for
// the Newton's-third-law shapes) the finish pass, which leaves a complete state.  A
// time step launches the pair kernel alone and leaves the finish to the next drift.
void launch_force(const StepParams& P0, const SysDesc* S, int nsys, const Arrays& A,
                  const uint32_t* start, unsigned long long* facc, int n, DevCounters* ctr, int kick,
                  int variant, cudaStream_t s);
void launch_force_pairs(const StepParams& P0, const SysDesc* S, int nsys, const Arrays& A,
                        const uint32_t* start, unsigned long long* facc, int n, DevCounters* ctr,
                        int kick, int variant, cudaStream_t s);
// Finish pass: pending fixed-point sums -> frc, closing kick (kick = 1), sums cleared.
void launch_force_finish(const StepParams& P0, const SysDesc* S, int nsys, const Arrays& A,
                         unsigned long long* facc, int n, DevCounters* ctr, int kick,
                         cudaStream_t s);
int force_variants();
// Kernels one launch_force of this shape enqueues (1, or 2 with the finish pass).
// True for the Newton's-third-law shapes (fixed-point sums, pending after a step).
bool force_variant_newton3(int variant);
const char* force_variant_name(int v);
void launch_profile(const float4* pos, const float4* vel, int n, int axis, int nbins, float lo,
                    float inv_w, double* acc, cudaStream_t s);
void launch_stats(const float4* pos, const float4* vel, int n, double* acc, cudaStream_t s);
void launch_band(const StepParams& P, uint8_t* band, cudaStream_t s);
void launch_load(const StepParams& P, const float4* in_pos, const float4* in_vel, const int* in_id,
                 const uint8_t* in_type, const Arrays& A, uint32_t* seen, int n, DevCounters* ctr,
                 cudaStream_t s);
void launch_unsort(const Arrays& A, int n, float4* out_pos, float4* out_vel, float4* out_frc,
                   int* out_id, uint8_t* out_type, cudaStream_t s);
void set_global_error(const char* msg);

}  // namespace dpd
