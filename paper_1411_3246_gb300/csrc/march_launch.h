// Host-side launchers of the xi-march kernels, one translation unit per precision form
// (march_fp64.cu, march_mixed.cu) so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "wake_common.cuh"

namespace wake {

struct PipeArgs;

struct MarchLaunch {
  const SimDesc *d_desc;  // n descriptors (device)
  const int *d_order;     // CTA -> simulation (device), largest work first
  int n, max_n1, max_np;
  cudaStream_t stream;
};

// Each returns cudaSuccess or the launch error; ppt_out receives the rings per thread used
// (0 if max_np needs more than the largest compiled variant).
cudaError_t launch_march_fp64(const MarchLaunch &L, int *ppt_out);
cudaError_t launch_march_mixed(const MarchLaunch &L, int *ppt_out);
// Global-memory ring slot storage one simulation needs (0 when the rings live in shared
// memory).
size_t ring_buf_bytes(int precision_fp64);
// Pipelined beam steps of one simulation (pipeline.cuh): one cooperative launch of up to
// max_ctas CTAs.  step_smem_ok tells whether the pipelined kernel fits shared memory;
// step_max_ctas how many CTAs can be co-resident.
bool step_smem_ok(int precision_fp64, int n1, int np);
int step_max_ctas(int precision_fp64, int n1, int np);
cudaError_t launch_step(int precision_fp64, const PipeArgs &a, int np, int ctas, cudaStream_t stream);
// Dynamic shared memory one march CTA needs for n1 nodes and np rings.
size_t march_smem_bytes(int precision_fp64, int n1, int np);

}  // namespace wake
