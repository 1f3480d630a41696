// FP64 form of the xi-march (every step in double precision).
#include "march_tiles.cuh"
#include "pipeline.cuh"

namespace wake {

bool march_tile_fp64(int nt, int ppt, TileFns *out, bool slab) {
  if (nt != PolFP64::NT) return false;
  if (slab) {
    switch (ppt) {
      case 1: *out = tile_fns<SlabOf<PolFP64>, 512, 1>(); return true;
      case 2: *out = tile_fns<SlabOf<PolFP64>, 512, 2>(); return true;
      case 4: *out = tile_fns<SlabOf<PolFP64>, 512, 4>(); return true;
      case 8: *out = tile_fns<SlabOf<PolFP64>, 512, 8>(); return true;
      default: return false;
    }
  }
  switch (ppt) {
    case 1: *out = tile_fns<PolFP64, 512, 1>(); return true;
    case 2: *out = tile_fns<PolFP64, 512, 2>(); return true;
    case 4: *out = tile_fns<PolFP64, 512, 4>(); return true;
    case 8: *out = tile_fns<PolFP64, 512, 8>(); return true;
    case 16: *out = tile_fns<PolFP64, 512, 16>(); return true;
    default: return false;
  }
}

bool march_tile(int form, bool slab, int nt, int ppt, TileFns *out) {
  if (form == kFormFP64) return march_tile_fp64(nt, ppt, out, slab);
  if (form == kFormMixed64) return march_tile_mixed64(nt, ppt, out, slab);
  if (nt == 512) return march_tile_mixed512(nt, ppt, out, slab);
  return !slab && march_tile_mixed_small(nt, ppt, out);  // the small tiles are cylindrical only
}

size_t ring_buf_bytes(int form) {
  // the FP64 form keeps its ring slots in global memory: room for the largest variant
  return form == kFormFP64 ? RingSoA<double>::bytes(PolFP64::NT * 16, true) : 0;
}


template <class P, int PPT>
static cudaError_t go_step(const PipeArgs &a, int ctas, cudaStream_t stream) {
  auto kern = step_kernel<P, PolFP64::NT, PPT>;
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
  if (a.d.slab) {  // the slab geometry's kernels (up to 8 rings per thread)
    switch (ppt_for(np)) {
      case 1: return go_step<SlabOf<PolFP64>, 1>(a, ctas, stream);
      case 2: return go_step<SlabOf<PolFP64>, 2>(a, ctas, stream);
      case 4: return go_step<SlabOf<PolFP64>, 4>(a, ctas, stream);
      case 8: return go_step<SlabOf<PolFP64>, 8>(a, ctas, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (ppt_for(np)) {
    case 1: return go_step<PolFP64, 1>(a, ctas, stream);
    case 2: return go_step<PolFP64, 2>(a, ctas, stream);
    case 4: return go_step<PolFP64, 4>(a, ctas, stream);
    case 8: return go_step<PolFP64, 8>(a, ctas, stream);
    case 16: return go_step<PolFP64, 16>(a, ctas, stream);
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

bool step_smem_ok(int form, int n1, int np) { return step_max_ctas(form, n1, np) > 0; }
int step_max_ctas(int form, int n1, int np) {
  return form == kFormFP64 ? step_ctas_fp64(n1, np) : form == kFormMixed64 ? step_ctas_mixed64(n1, np) : step_ctas_mixed(n1, np);
}
size_t step_global_window_bytes(int form, int n1) { return form == kFormMixed64 ? step_window_bytes(n1) : 0; }
cudaError_t launch_step(int form, const PipeArgs &a, int np, int ctas, cudaStream_t stream) {
  return form == kFormFP64 ? launch_step_fp64(a, np, ctas, stream)
                           : form == kFormMixed64 ? launch_step_mixed64(a, np, ctas, stream) : launch_step_mixed(a, np, ctas, stream);
}
}  // namespace wake
