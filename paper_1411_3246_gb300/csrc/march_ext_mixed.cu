// The plain march with an extra hook, one CTA of 512 threads, rings in PPT = 1..16 per thread:
// the ring trajectory dump (march.cuh march_traj_kernel) and plasma-particle trapping
// (march_trap_kernel); mixed form, compiled with the mixed march's fast FP32 division.
#include "march.cuh"
#include "march_launch.h"

namespace wake {

namespace {
template <class P, int PPT>
cudaError_t go_traj(const SimDesc *d, int n1, double *traj, int every, cudaStream_t s) {
  auto kern = march_traj_kernel<P, 512, PPT>;
  const size_t smem = MarchSmem<PolMixed>::bytes(n1, 512 * PPT, true);
  if (smem > kMaxSmemPerCta) return cudaErrorInvalidValue;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<1, 512, smem, s>>>(d, traj, every);
  return cudaGetLastError();
}
int traj_ppt(int np) {
  const int ppt = (np + 511) / 512;
  return ppt <= 1 ? 1 : ppt <= 2 ? 2 : ppt <= 4 ? 4 : ppt <= 8 ? 8 : ppt <= 16 ? 16 : 0;
}
}  // namespace

size_t march_traj_smem_mixed(int n1, int np) {
  const int ppt = traj_ppt(np);
  if (ppt == 0 || n1 > 3 * 512) return (size_t)1 << 40;
  return MarchSmem<PolMixed>::bytes(n1, 512 * ppt, true);
}

template <int PPT>
static cudaError_t go_trap(const SimDesc *d, int n1, cudaStream_t s) {
  auto kern = march_trap_kernel<PolMixed, 512, PPT>;
  const size_t smem = MarchSmem<PolMixed>::bytes(n1, 512 * PPT, true);
  if (smem > kMaxSmemPerCta) return cudaErrorInvalidValue;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<1, 512, smem, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_march_trap_mixed(const SimDesc *d, int n1, int np, cudaStream_t s) {
  switch (traj_ppt(np)) {
    case 1: return go_trap<1>(d, n1, s);
    case 2: return go_trap<2>(d, n1, s);
    case 4: return go_trap<4>(d, n1, s);
    case 8: return go_trap<8>(d, n1, s);
    case 16: return go_trap<16>(d, n1, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_march_traj_mixed(const SimDesc *d, int n1, int np, double *traj, int every, bool slab,
                                     cudaStream_t s) {
  if (slab) {  // the slab geometry's kernels (up to 8 rings per thread)
    switch (traj_ppt(np)) {
      case 1: return go_traj<SlabOf<PolMixed>, 1>(d, n1, traj, every, s);
      case 2: return go_traj<SlabOf<PolMixed>, 2>(d, n1, traj, every, s);
      case 4: return go_traj<SlabOf<PolMixed>, 4>(d, n1, traj, every, s);
      case 8: return go_traj<SlabOf<PolMixed>, 8>(d, n1, traj, every, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (traj_ppt(np)) {
    case 1: return go_traj<PolMixed, 1>(d, n1, traj, every, s);
    case 2: return go_traj<PolMixed, 2>(d, n1, traj, every, s);
    case 4: return go_traj<PolMixed, 4>(d, n1, traj, every, s);
    case 8: return go_traj<PolMixed, 8>(d, n1, traj, every, s);
    case 16: return go_traj<PolMixed, 16>(d, n1, traj, every, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wake
