// Compiled march tiles: a tile is (NT threads per CTA, PPT rings per thread).  Each
// translation unit that instantiates march_kernel registers its tiles through TileFns, so
// the host can launch, size and rank them without knowing which unit compiled them.
#pragma once

#include <mutex>

#include "march.cuh"
#include "march_launch.h"

namespace wake {

// Raise the kernel's dynamic shared-memory limit to what n1 nodes need.  The limit only ever
// grows (it is per kernel, shared by all handles), so a call that finds it high enough makes
// no CUDA call: the planner prepares every class before a step is captured.
template <class Pol, int NT, int PPT>
static cudaError_t tile_prepare(int n1) {
  static std::mutex mu;
  static size_t set = 0;
  const size_t smem = MarchSmem<Pol>::bytes(n1, NT * PPT);
  std::lock_guard<std::mutex> lk(mu);
  if (smem <= set) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(march_kernel<Pol, NT, PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) set = smem;
  return e;
}

template <class Pol, int NT, int PPT>
static cudaError_t tile_launch(const SimDesc *d, const int *order, int count, int n1, cudaStream_t s) {
  const size_t smem = MarchSmem<Pol>::bytes(n1, NT * PPT);
  cudaError_t e = tile_prepare<Pol, NT, PPT>(n1);
  if (e != cudaSuccess) return e;
  march_kernel<Pol, NT, PPT><<<count, NT, smem, s>>>(d, order);
  return cudaGetLastError();
}

template <class Pol, int NT, int PPT>
static size_t tile_smem(int n1) {
  return MarchSmem<Pol>::bytes(n1, NT * PPT);
}

// CTAs of this tile that fit on one SM for n1 nodes (0: it does not fit).
template <class Pol, int NT, int PPT>
static int tile_occupancy(int n1) {
  auto kern = march_kernel<Pol, NT, PPT>;
  const size_t smem = MarchSmem<Pol>::bytes(n1, NT * PPT);
  if (smem > kMaxSmemPerCta) return 0;
  if (tile_prepare<Pol, NT, PPT>(n1) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) return 0;
  return per_sm;
}

template <class Pol, int NT, int PPT>
static TileFns tile_fns() {
  return TileFns{NT, PPT, false, &tile_launch<Pol, NT, PPT>, &tile_prepare<Pol, NT, PPT>, &tile_smem<Pol, NT, PPT>,
                 &tile_occupancy<Pol, NT, PPT>};
}

}  // namespace wake
