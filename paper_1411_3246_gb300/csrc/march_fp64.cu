// FP64 form of the xi-march (every step in double precision).
#include "march.cuh"
#include "march_launch.h"

namespace wake {

template <int PPT>
static cudaError_t go(const MarchLaunch &L) {
  auto kern = march_kernel<PolFP64, PolFP64::NT, PPT>;
  const size_t smem = MarchSmem<PolFP64>::bytes(L.max_n1, PolFP64::NT * PPT);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<L.n, PolFP64::NT, smem, L.stream>>>(L.d_desc, L.d_order);
  return cudaGetLastError();
}

cudaError_t launch_march_fp64(const MarchLaunch &L, int *ppt_out) {
  const int ppt = (L.max_np + PolFP64::NT - 1) / PolFP64::NT;
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

static int ppt_of(int np, int nt) {
  const int ppt = (np + nt - 1) / nt;
  return ppt <= 1 ? 1 : ppt <= 2 ? 2 : ppt <= 4 ? 4 : ppt <= 8 ? 8 : ppt <= 16 ? 16 : 0;
}

size_t march_smem_bytes(int precision_fp64, int n1, int np) {
  if (precision_fp64) return MarchSmem<PolFP64>::bytes(n1, PolFP64::NT * ppt_of(np, PolFP64::NT));
  return MarchSmem<PolMixed>::bytes(n1, PolMixed::NT * ppt_of(np, PolMixed::NT));
}

size_t ring_buf_bytes(int precision_fp64) {
  // the FP64 form keeps its ring slots in global memory: room for the largest variant
  return precision_fp64 ? RingSoA<double>::bytes(PolFP64::NT * 16) : 0;
}

}  // namespace wake
