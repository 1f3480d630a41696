// Mixed form of the xi-march: FP32 ring and node arithmetic, float-float scans.
#include "march.cuh"
#include "march_launch.h"

namespace wake {

template <int PPT>
static cudaError_t go(const MarchLaunch &L) {
  auto kern = march_kernel<PolMixed, PolMixed::NT, PPT>;
  const size_t smem = MarchSmem<PolMixed>::bytes(L.max_n1, PolMixed::NT * PPT);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<L.n, PolMixed::NT, smem, L.stream>>>(L.d_desc, L.d_order);
  return cudaGetLastError();
}

cudaError_t launch_march_mixed(const MarchLaunch &L, int *ppt_out) {
  const int ppt = (L.max_np + PolMixed::NT - 1) / PolMixed::NT;
  *ppt_out = ppt <= 1 ? 1 : ppt <= 2 ? 2 : ppt <= 4 ? 4 : ppt <= 8 ? 8 : ppt <= 16 ? 16 : 0;
  switch (*ppt_out) {
    case 1: return go<1>(L);
    case 2: return go<2>(L);
    case 4: return go<4>(L);
    case 8: return go<8>(L);
    case 16: return go<16>(L);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wake
