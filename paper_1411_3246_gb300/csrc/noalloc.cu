// wake_beam_deposit_noalloc: the beam deposit of wake_beam_deposit for callers that must not
// allocate device memory.  Such callers are, for instance, code running while a caching
// allocator (PyTorch's, or the caller's own pool) holds the device memory, where a cudaMalloc
// could fail or make the pool give back its cached blocks, and code that cannot take the
// device-wide synchronisation of cudaFree among concurrent streams.  Instead of the handle's
// allocated grid, the deposit accumulates in a static device array that is part of the
// module image; the host looks up its address once per device.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/wake.h"
#include "wake_common.cuh"

namespace wake {
void set_last_error(const std::string &msg);
}

using namespace wake;

// Accumulation grid: WAKE_NOALLOC_MAX_NODES doubles (4 MiB).  Zeroed by every call before use.
static __device__ __align__(256) double g_nb_scratch[WAKE_NOALLOC_MAX_NODES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {};  // per device, set by the first call on it

int fail_na(int code, const std::string &msg) {
  set_last_error(msg);
  return code;
}

__global__ void na_zero_kernel(double *acc, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    acc[t] = 0.0;
}

// Bilinear hats of every live particle (drive weight wd for j < n_drive, else ww), as the
// handle's deposit does in its FP64 form.
__global__ void na_deposit_kernel(const double *__restrict__ xyz, const uint8_t *__restrict__ lost, int64_t n,
                                  int64_t n_drive, int nr, int nxi, double rmax, double ximax, double dr,
                                  double dxi, double wd, double ww, double *acc, bool slab) {
  const int n1 = nr + 1;
  const double inv_dr = 1.0 / dr, inv_dxi = 1.0 / dxi;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    if (lost && lost[j]) continue;
    const double x = xyz[j], y = slab ? 0.0 : xyz[n + j], xi = xyz[2 * n + j];  // slab: a sheet beam at y = 0
    const double r = sqrt(x * x + y * y);
    if (!(xi >= 0.0 && xi < ximax && r < rmax)) continue;  // outside the box: lost
    int c, k;
    double f, g;
    locate(r, inv_dr, nr, c, f);
    locate(xi, inv_dxi, nxi, k, g);
    const double w = j < n_drive ? wd : ww;
    double *row = acc + (size_t)k * n1 + c;
    atomicAdd(row, w * (1.0 - f) * (1.0 - g));
    atomicAdd(row + 1, w * f * (1.0 - g));
    atomicAdd(row + n1, w * (1.0 - f) * g);
    atomicAdd(row + n1 + 1, w * f * g);
  }
}

// Divide by the hats' volumes: V_i in r, dxi in xi (dxi/2 at both ends).
__global__ void na_normalize_kernel(const double *__restrict__ acc, double *__restrict__ nb, int nr, int nxi,
                                    double dr, double dxi, bool slab) {
  const int n1 = nr + 1;
  const int64_t tot = (int64_t)(nxi + 1) * n1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / n1), i = (int)(t % n1);
    const double vx = (k == 0 || k == nxi) ? 0.5 * dxi : dxi;
    nb[t] = acc[t] / (node_volume(i, nr, dr, slab) * vx);
  }
}

int blocks_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

}  // namespace

extern "C" int wake_beam_deposit_noalloc(const wake_params *p, const double *xyz, const uint8_t *lost,
                                         void *stream, double *nb) {
  if (!p || !nb) return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: null p or nb");
  if (p->nr < 2 || p->nr > 1024 || p->nxi < 2 || p->nxi > (1 << 20))
    return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: need 2 <= nr <= 1024 and 2 <= nxi <= 2^20");
  const int64_t nodes = (int64_t)(p->nr + 1) * (p->nxi + 1);
  if (nodes > WAKE_NOALLOC_MAX_NODES)
    return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: grid of " + std::to_string(nodes) +
                                    " nodes exceeds WAKE_NOALLOC_MAX_NODES (" +
                                    std::to_string(WAKE_NOALLOC_MAX_NODES) + ")");
  if (p->n_beam < 0 || p->n_drive < 0 || p->n_drive > p->n_beam)
    return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: need 0 <= n_drive <= n_beam");
  if (p->n_beam > 0 && !xyz) return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: null xyz");
  if (!(p->rmax > 0.0) || !(p->ximax > 0.0))
    return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: rmax and ximax must be positive");
  if (!(p->sigma_r > 0.0) || !(p->sigma_zd > 0.0) || (p->n_w != 0.0 && !(p->sigma_zw > 0.0)))
    return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: bunch sizes must be positive");
  if (p->geometry != WAKE_CYLINDRICAL && p->geometry != WAKE_SLAB)
    return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: geometry must be WAKE_CYLINDRICAL or WAKE_SLAB");

  // set-up, once per device: the address of the static accumulation grid
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(WAKE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(WAKE_EINVAL, "wake_beam_deposit_noalloc: device index >= 64");
  double *acc = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void *a = nullptr;
      e = cudaGetSymbolAddress(&a, g_nb_scratch);
      if (e != cudaSuccess || !a)
        return fail_na(WAKE_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = (double *)a;
    }
    acc = g_scratch_addr[dev];
  }

  const cudaStream_t s = (cudaStream_t)stream;
  const double dr = p->rmax / p->nr, dxi = p->ximax / p->nxi;
  // macroparticle weights: each bunch's charge (per 2 pi) of Eq. 12 over its macroparticles
  const double s2pi = std::sqrt(2.0 * 3.14159265358979323846);
  const int64_t nw = p->n_beam - p->n_drive;
  const bool slab = p->geometry == WAKE_SLAB;  // half-slab transverse integral sigma_r sqrt(2 pi)/2
  const double tr = slab ? 0.5 * s2pi * p->sigma_r : p->sigma_r * p->sigma_r;
  const double wd = p->n_drive > 0 ? p->n_d * s2pi * tr * p->sigma_zd / (double)p->n_drive : 0.0;
  const double ww = nw > 0 ? p->n_w * s2pi * tr * p->sigma_zw / (double)nw : 0.0;
  na_zero_kernel<<<blocks_for(nodes), 256, 0, s>>>(acc, nodes);
  if (p->n_beam > 0)
    na_deposit_kernel<<<blocks_for(p->n_beam), 256, 0, s>>>(xyz, lost, p->n_beam, p->n_drive, p->nr, p->nxi,
                                                            p->rmax, p->ximax, dr, dxi, wd, ww, acc, slab);
  na_normalize_kernel<<<blocks_for(nodes), 256, 0, s>>>(acc, nb, p->nr, p->nxi, dr, dxi, slab);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    // a stale address (e.g. after cudaDeviceReset) is looked up again by the next call
    std::lock_guard<std::mutex> lk(g_setup_mu);
    g_scratch_addr[dev] = nullptr;
    return fail_na(WAKE_ECUDA, std::string("wake_beam_deposit_noalloc launch: ") + cudaGetErrorString(e));
  }
  return WAKE_OK;
}
