// FP32 / FP64 fused-multiply-add throughput of this GPU: the ALU peak against which the
// xi-march (an ALU-bound kernel, not HBM- or tensor-bound) is placed on a roofline.  Every
// thread runs 16 independent FMA chains, so the FMA pipes see no dependency stalls; the
// CTAs fill every SM several times over.  Timed with CUDA events on the given stream.
#include <cuda_runtime.h>

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T *sink, int iters, T seed) {
  constexpr int kChains = 16;
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = seed + (T)(threadIdx.x + i) * (T)1e-7;
  const T m = (T)0.9999999, c = (T)1e-7;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], m, c);
  }
  T s = (T)0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == (T)-1.25) sink[blockIdx.x] = s;  // never true: keeps the chains live
}

}  // namespace

extern "C" {

// Runs the FMA kernel in FP32 (fp64 == 0) or FP64: ctas CTAs of 256 threads, iters
// iterations of 16 FMAs per thread, after one untimed launch.  *ms gets the timed launch's
// device time, *flop its floating-point operations (an FMA counts 2).  Returns a
// cudaError_t (0 on success).  Synchronous.
int fp_peak_run(int fp64, int ctas, int iters, void *stream, float *ms, double *flop) {
  cudaStream_t s = (cudaStream_t)stream;
  void *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(double) * (size_t)ctas);
  if (e != cudaSuccess) return (int)e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      if (rep == 1) e = cudaEventRecord(e0, s);
      if (fp64)
        fma_chains_kernel<double><<<ctas, 256, 0, s>>>((double *)sink, iters, 1.0);
      else
        fma_chains_kernel<float><<<ctas, 256, 0, s>>>((float *)sink, iters, 1.0f);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  }
  *flop = 2.0 * 16.0 * 256.0 * (double)ctas * (double)iters;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return (int)e;
}

}  // extern "C"
