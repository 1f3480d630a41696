// Host-side launchers of the xi-march kernels, one translation unit per precision form
// (march_fp64.cu, march_mixed.cu) so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "wake_common.cuh"

namespace wake {

struct PipeArgs;

constexpr size_t kMaxSmemPerCta = 227 * 1024;

// Precision forms, numbered as the library's WAKE_FP64, WAKE_MIXED and WAKE_MIXED64.
enum Form : int { kFormFP64 = 0, kFormMixed = 1, kFormMixed64 = 2 };

// A compiled march tile: NT threads per CTA, PPT rings per thread (march_tiles.cuh).
struct TileFns {
  int nt, ppt;
  bool wide;  // rings in a global buffer, in chunks of nt x ppt (march_wide.cuh)
  // one CTA per entry of order[0..count-1] (descriptor d[order[i]]), shared memory for n1 nodes
  cudaError_t (*launch)(const SimDesc *d, const int *order, int count, int n1, cudaStream_t s);
  cudaError_t (*prepare)(int n1);  // shared-memory limit for n1 nodes (before any capture)
  size_t (*smem)(int n1);
  int (*occupancy)(int n1);  // CTAs per SM for n1 nodes, 0 if it does not fit
};
// The tile (nt, ppt) of a precision form and geometry (slab: nt = 512, ppt <= 8), if it is
// compiled.
bool march_tile(int form, bool slab, int nt, int ppt, TileFns *out);
bool march_tile_fp64(int nt, int ppt, TileFns *out, bool slab);
bool march_tile_mixed512(int nt, int ppt, TileFns *out, bool slab);
bool march_tile_mixed_small(int nt, int ppt, TileFns *out);
bool march_tile_mixed64(int nt, int ppt, TileFns *out, bool slab);
// The wide mixed march (march_wide.cuh) and its ring buffer for np rings.
TileFns march_tile_wide();
size_t wide_ring_bytes(int np);
// Pipelined steps in the wide form: shared memory fits, co-resident CTAs, launch.
// Pipelined steps in the wide form, CTAs of nt = 256 (two per SM) or 512 threads.
int step_wide_max_ctas(int n1, int nt);
size_t step_wide_window_bytes(int n1);
size_t step_wide_ring_bytes(int np, int nt);
cudaError_t launch_step_wide(const PipeArgs &a, int nt, int ctas, cudaStream_t stream);
// The FP64 wide form (march_wide64.cu): its plain tile, the global bytes one simulation or
// one pipelined CTA needs (ring slots and node arrays), and its pipelined steps.
TileFns march_tile_wide_fp64();
size_t wide_fp64_ring_bytes(int np, int n1);
size_t step_wide_fp64_window_bytes(int n1);
int step_wide_fp64_max_ctas(int n1);
cudaError_t launch_step_wide_fp64(const PipeArgs &a, int ctas, cudaStream_t stream);
// Pipelined steps of many simulations (pipeline.cuh batch_step_kernel), wide form.
struct BatchArgs;
int batch_step_max_ctas(int max_n1, int bnt);
size_t batch_ring_bytes(int max_np, int bnt);
cudaError_t launch_batch_steps(const BatchArgs &b, int max_n1, int bnt, int ctas, cudaStream_t stream);

// Global-memory ring slot storage one simulation needs (0 when the rings live in shared
// memory).
size_t ring_buf_bytes(int form);
// Pipelined beam steps of one simulation (pipeline.cuh): one cooperative launch of up to
// max_ctas CTAs.  step_smem_ok tells whether the pipelined kernel fits shared memory;
// step_max_ctas how many CTAs can be co-resident.
// Global field-window bytes per CTA the form's pipelined step needs (0: in shared memory).
bool step_smem_ok(int form, int n1, int np);
int step_max_ctas(int form, int n1, int np);
size_t step_global_window_bytes(int form, int n1);
cudaError_t launch_step(int form, const PipeArgs &a, int np, int ctas, cudaStream_t stream);
cudaError_t launch_step_mixed64(const PipeArgs &a, int np, int ctas, cudaStream_t stream);
int step_ctas_mixed64(int n1, int np);

// The plain march with the ring trajectory dump (march_traj_kernel), one CTA of 512 threads:
// its shared memory for n1 nodes and np rings (more than kMaxSmemPerCta: no variant fits),
// and its launch on the descriptor d (device).
size_t march_traj_smem_fp64(int n1, int np);
size_t march_traj_smem_mixed(int n1, int np);
cudaError_t launch_march_traj_fp64(const SimDesc *d, int n1, int np, double *traj, int every, bool slab, cudaStream_t s);
cudaError_t launch_march_traj_mixed(const SimDesc *d, int n1, int np, double *traj, int every, bool slab, cudaStream_t s);
// The plain march with trapping (march_trap_kernel) on descriptor d (device); same shared memory.
cudaError_t launch_march_trap_fp64(const SimDesc *d, int n1, int np, cudaStream_t s);
cudaError_t launch_march_trap_mixed(const SimDesc *d, int n1, int np, cudaStream_t s);

}  // namespace wake
