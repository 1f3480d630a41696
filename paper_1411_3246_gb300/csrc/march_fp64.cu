// FP64 form of the xi-march (every step in double precision).
#include "march.cuh"
#include "pipeline.cuh"
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


template <int PPT>
static cudaError_t go_step(const PipeArgs &a, int ctas, cudaStream_t stream) {
  auto kern = step_kernel<PolFP64, PolFP64::NT, PPT>;
  const size_t smem = step_smem_bytes<PolFP64, PolFP64::NT, PPT>(a.d.nr + 1);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  PipeArgs arg = a;
  void *args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(ctas), dim3(PolFP64::NT), args, smem, stream);
}
template <int PPT>
static int ctas_step(int n1) {
  auto kern = step_kernel<PolFP64, PolFP64::NT, PPT>;
  const size_t smem = step_smem_bytes<PolFP64, PolFP64::NT, PPT>(n1);
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PolFP64::NT, smem) != cudaSuccess) return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}
static int ppt_for(int np) {
  const int ppt = (np + PolFP64::NT - 1) / PolFP64::NT;
  return ppt <= 1 ? 1 : ppt <= 2 ? 2 : ppt <= 4 ? 4 : ppt <= 8 ? 8 : ppt <= 16 ? 16 : 0;
}
static size_t step_bytes_for(int n1, int np) {
  switch (ppt_for(np)) {
    case 1: return step_smem_bytes<PolFP64, PolFP64::NT, 1>(n1);
    case 2: return step_smem_bytes<PolFP64, PolFP64::NT, 2>(n1);
    case 4: return step_smem_bytes<PolFP64, PolFP64::NT, 4>(n1);
    case 8: return step_smem_bytes<PolFP64, PolFP64::NT, 8>(n1);
    case 16: return step_smem_bytes<PolFP64, PolFP64::NT, 16>(n1);
    default: return (size_t)1 << 40;
  }
}
cudaError_t launch_step_fp64(const PipeArgs &a, int np, int ctas, cudaStream_t stream) {
  switch (ppt_for(np)) {
    case 1: return go_step<1>(a, ctas, stream);
    case 2: return go_step<2>(a, ctas, stream);
    case 4: return go_step<4>(a, ctas, stream);
    case 8: return go_step<8>(a, ctas, stream);
    case 16: return go_step<16>(a, ctas, stream);
    default: return cudaErrorInvalidValue;
  }
}
int step_ctas_fp64(int n1, int np) {
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

cudaError_t launch_step_mixed(const PipeArgs &a, int np, int ctas, cudaStream_t stream);
int step_ctas_mixed(int n1, int np);

bool step_smem_ok(int precision_fp64, int n1, int np) { return step_max_ctas(precision_fp64, n1, np) > 0; }
int step_max_ctas(int precision_fp64, int n1, int np) {
  return precision_fp64 ? step_ctas_fp64(n1, np) : step_ctas_mixed(n1, np);
}
cudaError_t launch_step(int precision_fp64, const PipeArgs &a, int np, int ctas, cudaStream_t stream) {
  return precision_fp64 ? launch_step_fp64(a, np, ctas, stream) : launch_step_mixed(a, np, ctas, stream);
}
}  // namespace wake
