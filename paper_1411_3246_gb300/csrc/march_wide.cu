// The wide form of the xi-march (march_wide.cuh): plain launches (one CTA per simulation) and
// pipelined beam steps with the field window in global memory.
#include "march_launch.h"
#include "march_wide.cuh"
#include "pipeline.cuh"

#include <mutex>

namespace wake {

namespace {

constexpr int kWideNT = PolWide::NT, kWidePPT = 8;

cudaError_t wide_prepare(int n1) {
  static std::mutex mu;
  static size_t set = 0;
  const size_t smem = MarchSmem<PolWide>::bytes(n1, kWideNT * kWidePPT);
  std::lock_guard<std::mutex> lk(mu);
  if (smem <= set) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(march_wide_kernel<PolWide, kWideNT, kWidePPT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) set = smem;
  return e;
}
cudaError_t wide_launch(const SimDesc *d, const int *order, int count, int n1, cudaStream_t s) {
  cudaError_t e = wide_prepare(n1);
  if (e != cudaSuccess) return e;
  march_wide_kernel<PolWide, kWideNT, kWidePPT>
      <<<count, kWideNT, MarchSmem<PolWide>::bytes(n1, kWideNT * kWidePPT), s>>>(d, order);
  return cudaGetLastError();
}
size_t wide_smem(int n1) { return MarchSmem<PolWide>::bytes(n1, kWideNT * kWidePPT); }
int wide_occupancy(int n1) {
  const size_t smem = wide_smem(n1);
  if (smem > kMaxSmemPerCta || wide_prepare(n1) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_wide_kernel<PolWide, kWideNT, kWidePPT>, kWideNT,
                                                    smem) != cudaSuccess)
    return 0;
  return per_sm;
}

size_t step_wide_smem(int n1) {
  return ((MarchSmem<PolWide>::bytes(n1, kWideNT * kWidePPT) + 63) & ~(size_t)63) + 64;
}

}  // namespace

TileFns march_tile_wide() {
  return TileFns{kWideNT, kWidePPT, true, &wide_launch, &wide_prepare, &wide_smem, &wide_occupancy};
}

size_t wide_ring_bytes(int np) { return WideRings<float>::bytes(wide_slots<kWideNT, kWidePPT>(np)); }

size_t step_wide_window_bytes(int n1) { return sizeof(float) * 12 * (size_t)n1; }

template <int NT>
static size_t step_wide_smem_nt(int n1) {
  return ((MarchSmem<PolWide>::bytes(n1, NT * kWidePPT) + 63) & ~(size_t)63) + 64;
}
template <int NT>
static int step_wide_ctas(int n1) {
  auto kern = step_wide_kernel<PolWide, NT, kWidePPT>;
  const size_t smem = step_wide_smem_nt<NT>(n1);
  if (smem > kMaxSmemPerCta || n1 > PolWide::kScanE * NT) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}
template <int NT>
static cudaError_t step_wide_launch(const PipeArgs &a, int ctas, cudaStream_t stream) {
  auto kern = step_wide_kernel<PolWide, NT, kWidePPT>;
  const size_t smem = step_wide_smem_nt<NT>(a.d.nr + 1);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  PipeArgs arg = a;
  void *args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(ctas), dim3(NT), args, smem, stream);
}

int step_wide_max_ctas(int n1, int nt) { return nt == 256 ? step_wide_ctas<256>(n1) : step_wide_ctas<512>(n1); }

size_t step_wide_ring_bytes(int np, int nt) {
  return nt == 256 ? WideRings<float>::bytes(wide_slots<256, kWidePPT>(np)) : wide_ring_bytes(np);
}

cudaError_t launch_step_wide(const PipeArgs &a, int nt, int ctas, cudaStream_t stream) {
  return nt == 256 ? step_wide_launch<256>(a, ctas, stream) : step_wide_launch<512>(a, ctas, stream);
}

// The batched pipelined kernel in CTAs of bnt = 512 or 256 threads (the latter two per SM).
template <int NT>
static int batch_ctas(int max_n1) {
  auto kern = batch_step_kernel<PolWide, NT, kWidePPT>;
  const size_t smem = ((MarchSmem<PolWide>::bytes(max_n1, NT * kWidePPT) + 63) & ~(size_t)63) + 64;
  if (smem > kMaxSmemPerCta || max_n1 > PolWide::kScanE * NT) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}
template <int NT>
static cudaError_t batch_launch(const BatchArgs &b, int max_n1, int ctas, cudaStream_t stream) {
  auto kern = batch_step_kernel<PolWide, NT, kWidePPT>;
  const size_t smem = ((MarchSmem<PolWide>::bytes(max_n1, NT * kWidePPT) + 63) & ~(size_t)63) + 64;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BatchArgs arg = b;
  void *args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(ctas), dim3(NT), args, smem, stream);
}

int batch_step_max_ctas(int max_n1, int bnt) { return bnt == 256 ? batch_ctas<256>(max_n1) : batch_ctas<512>(max_n1); }

size_t batch_ring_bytes(int max_np, int bnt) {
  return bnt == 256 ? WideRings<float>::bytes(wide_slots<256, kWidePPT>(max_np)) : wide_ring_bytes(max_np);
}

cudaError_t launch_batch_steps(const BatchArgs &b, int max_n1, int bnt, int ctas, cudaStream_t stream) {
  return bnt == 256 ? batch_launch<256>(b, max_n1, ctas, stream) : batch_launch<512>(b, max_n1, ctas, stream);
}

}  // namespace wake
