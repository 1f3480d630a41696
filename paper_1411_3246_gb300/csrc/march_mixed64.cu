// The FP64-solve split of the xi-march (PolMixed64): FP32 ring arithmetic; FP64 cross-ring
// deposit sums, node arrays, scans and tridiagonal solves; the pipelined step keeps its field
// window in global memory.
#include "march_tiles.cuh"
#include "pipeline.cuh"

namespace wake {

bool march_tile_mixed64(int nt, int ppt, TileFns *out, bool slab) {
  if (nt != 512) return false;
  if (slab) {
    switch (ppt) {
      case 1: *out = tile_fns<SlabOf<PolMixed64>, 512, 1>(); return true;
      case 2: *out = tile_fns<SlabOf<PolMixed64>, 512, 2>(); return true;
      case 4: *out = tile_fns<SlabOf<PolMixed64>, 512, 4>(); return true;
      case 8: *out = tile_fns<SlabOf<PolMixed64>, 512, 8>(); return true;
      default: return false;
    }
  }
  switch (ppt) {
    case 1: *out = tile_fns<PolMixed64, 512, 1>(); return true;
    case 2: *out = tile_fns<PolMixed64, 512, 2>(); return true;
    case 4: *out = tile_fns<PolMixed64, 512, 4>(); return true;
    case 8: *out = tile_fns<PolMixed64, 512, 8>(); return true;
    case 16: *out = tile_fns<PolMixed64, 512, 16>(); return true;
    default: return false;
  }
}

template <class P, int PPT>
static cudaError_t go_step(const PipeArgs &a, int ctas, cudaStream_t stream) {
  auto kern = step_kernel<P, PolMixed64::NT, PPT>;
  const size_t smem = step_smem_bytes<PolMixed64, PolMixed64::NT, PPT>(a.d.nr + 1);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  PipeArgs arg = a;
  void *args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(ctas), dim3(PolMixed64::NT), args, smem, stream);
}
template <int PPT>
static int ctas_step(int n1) {
  auto kern = step_kernel<PolMixed64, PolMixed64::NT, PPT>;
  const size_t smem = step_smem_bytes<PolMixed64, PolMixed64::NT, PPT>(n1);
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PolMixed64::NT, smem) != cudaSuccess) return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}
static int ppt_for(int np) {
  const int ppt = (np + PolMixed64::NT - 1) / PolMixed64::NT;
  return ppt <= 1 ? 1 : ppt <= 2 ? 2 : ppt <= 4 ? 4 : ppt <= 8 ? 8 : ppt <= 16 ? 16 : 0;
}
static size_t step_bytes_for(int n1, int np) {
  switch (ppt_for(np)) {
    case 1: return step_smem_bytes<PolMixed64, PolMixed64::NT, 1>(n1);
    case 2: return step_smem_bytes<PolMixed64, PolMixed64::NT, 2>(n1);
    case 4: return step_smem_bytes<PolMixed64, PolMixed64::NT, 4>(n1);
    case 8: return step_smem_bytes<PolMixed64, PolMixed64::NT, 8>(n1);
    case 16: return step_smem_bytes<PolMixed64, PolMixed64::NT, 16>(n1);
    default: return (size_t)1 << 40;
  }
}
cudaError_t launch_step_mixed64(const PipeArgs &a, int np, int ctas, cudaStream_t stream) {
  if (a.d.slab) {
    switch (ppt_for(np)) {
      case 1: return go_step<SlabOf<PolMixed64>, 1>(a, ctas, stream);
      case 2: return go_step<SlabOf<PolMixed64>, 2>(a, ctas, stream);
      case 4: return go_step<SlabOf<PolMixed64>, 4>(a, ctas, stream);
      case 8: return go_step<SlabOf<PolMixed64>, 8>(a, ctas, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (ppt_for(np)) {
    case 1: return go_step<PolMixed64, 1>(a, ctas, stream);
    case 2: return go_step<PolMixed64, 2>(a, ctas, stream);
    case 4: return go_step<PolMixed64, 4>(a, ctas, stream);
    case 8: return go_step<PolMixed64, 8>(a, ctas, stream);
    case 16: return go_step<PolMixed64, 16>(a, ctas, stream);
    default: return cudaErrorInvalidValue;
  }
}
int step_ctas_mixed64(int n1, int np) {
  if (step_bytes_for(n1, np) > 227 * 1024) return 0;
  switch (ppt_for(np)) {
    case 1: return ctas_step<1>(n1);
    case 2: return ctas_step<2>(n1);
    case 4: return ctas_step<4>(n1);
    case 8: return ctas_step<8>(n1);
    case 16: return ctas_step<16>(n1);
    default: return 0;
  }
}

}  // namespace wake
