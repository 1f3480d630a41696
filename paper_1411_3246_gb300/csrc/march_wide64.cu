// The FP64 form of the wide march (march_wide.cuh with PolWideFP64): for boxes beyond the FP64
// tiles (more than 1,024 radial cells or 8,192 rings, up to 2,048 and 65,536).  Its node
// arrays (about 330 KB at 2,049 nodes in FP64) do not fit shared memory, so each CTA carves
// them from a global buffer that follows its ring slots; the arithmetic is the shared wide-march
// code.  Plain launches (one CTA per simulation) and pipelined beam steps.
#include "march_launch.h"
#include "march_wide.cuh"
#include "pipeline.cuh"

namespace wake {

namespace {

using PW = PolWideFP64;
constexpr int kNT = PW::NT, kPPT = 8;

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
// ring slots, then the node arrays, of one simulation (or one CTA of the pipelined steps)
__host__ __device__ inline size_t ring_part(int np) { return align256(WideRings<double>::bytes(wide_slots<kNT, kPPT>(np))); }
__host__ __device__ inline size_t node_part(int n1) { return align256(MarchSmem<PW>::bytes(n1, kNT * kPPT)); }

__global__ void __launch_bounds__(kNT, 1) march_wide_g_kernel(const SimDesc *descs, const int *order) {
  const SimDesc &d = descs[order ? order[blockIdx.x] : blockIdx.x];
  PlainHooks<PW, kNT> hk{(const double *)d.nb, (double *)d.psi, (double *)d.ez, (double *)d.er, (double *)d.bth,
                         d.nr + 1, d.status};
  march_body_wide<PW, kNT, kPPT>(d, (unsigned char *)d.ring_buf + ring_part(d.np), hk);
}

__global__ void __launch_bounds__(kNT, 1) step_wide_g_kernel(PipeArgs a) {
  __shared__ int ctl[2];
  const int n1 = a.d.nr + 1;
  double *win = (double *)((unsigned char *)a.win_bufs + (size_t)blockIdx.x * a.win_stride);
  unsigned char *rb = (unsigned char *)a.ring_bufs + (size_t)blockIdx.x * a.ring_stride;
  for (int t = blockIdx.x; t < a.nsteps; t += gridDim.x) {
    if (threadIdx.x == 0) {
      ctl[0] = 0;
      ctl[1] = 0;
    }
    __syncthreads();
    PipeHooks<PW, kNT> hk{a, t, win, ctl, n1, a.d.nr, a.d.nxi, a.d.dr, a.d.dxi, a.d.rmax, a.d.ximax};
    SimDesc d = a.d;
    d.ring_buf = rb;
    march_body_wide<PW, kNT, kPPT>(d, rb + ring_part(d.np), hk);
    __syncthreads();
    if (ctl[0]) break;
  }
}

cudaError_t g_launch(const SimDesc *d, const int *order, int count, int, cudaStream_t s) {
  march_wide_g_kernel<<<count, kNT, 0, s>>>(d, order);
  return cudaGetLastError();
}
cudaError_t g_prepare(int) { return cudaSuccess; }
size_t g_smem(int) { return 0; }
int g_occupancy(int n1) {
  if (n1 > PW::kScanE * kNT) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_wide_g_kernel, kNT, 0) != cudaSuccess) return 0;
  return per_sm;
}

}  // namespace

TileFns march_tile_wide_fp64() { return TileFns{kNT, kPPT, true, &g_launch, &g_prepare, &g_smem, &g_occupancy}; }

size_t wide_fp64_ring_bytes(int np, int n1) { return ring_part(np) + node_part(n1); }

size_t step_wide_fp64_window_bytes(int n1) { return align256(sizeof(double) * 12 * (size_t)n1); }

int step_wide_fp64_max_ctas(int n1) {
  if (n1 > PW::kScanE * kNT) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_wide_g_kernel, kNT, 0) != cudaSuccess) return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

cudaError_t launch_step_wide_fp64(const PipeArgs &a, int ctas, cudaStream_t stream) {
  PipeArgs arg = a;
  void *args[] = {&arg};
  return cudaLaunchCooperativeKernel((const void *)step_wide_g_kernel, dim3(ctas), dim3(kNT), args, 0, stream);
}

}  // namespace wake
