// The adjoint form: gradients of the witness bunch's mean energy gain and rms energy spread
// (Sec. IV diagnostics) with respect to the witness peak density n_w (its charge), the
// witness delay xi_w - xi_d, the drive length sigma_zd, the plasma temperature u_th (Sec.
// II.A warm plasma) and per-bin multipliers of the witness current profile, through nsteps
// beam steps of deposit -> xi-march -> Boris push.  FP64 throughout.
//
// Forward (wake_adjoint_forward): beam states, beam densities and the field grids of every
// step are kept, and the ring state of every B-th slice of every march (B ~ sqrt(Nxi)).
// Reverse (wake_adjoint_backward): per step, newest first, the Boris push is reversed
// particle by particle (its field adjoints are scattered onto the grid), then the march is
// reversed block by block - each block of B slices is recomputed from its checkpoint with
// its intermediates kept, then reversed slice by slice - giving the adjoint of the step's beam
// density, which the reversed deposit turns into adjoints of the beam positions and weights.
// The arithmetic of each piece is in adjoint_core.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wake.h"
#include "adjoint_core.h"
#include "wake_common.cuh"

namespace wake {
void set_last_error(const std::string &msg);
}

using namespace wake;
using namespace wake::adj;

namespace {

constexpr int kNT = 512;  // threads of the one-CTA march kernels

int afail(int code, const std::string &m) {
  set_last_error(m);
  return code;
}
#define ACUDA(expr)                                                                                       \
  do {                                                                                                    \
    cudaError_t e_ = (expr);                                                                              \
    if (e_ != cudaSuccess) return afail(WAKE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int blocks_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// ---------------------------------------------------------------------------------------
// march kernels (one CTA)
// ---------------------------------------------------------------------------------------

__global__ void __launch_bounds__(kNT, 1) adj_march_fwd_kernel(MarchArgs a) {
  extern __shared__ __align__(16) double sm[];
  const Par P{(int)threadIdx.x, (int)blockDim.x};
  Work W;
  W.carve(sm, a.g.nr + 1);
  __shared__ int bad;
  if (P.tid == 0) bad = 0;
  __syncthreads();
  march_forward_body(P, a, W, &bad);
  if (P.tid == 0 && bad) atomicOr(a.status, bad == 1 ? ST_NUMERIC : ST_ESCAPE);
}

__global__ void __launch_bounds__(kNT, 1) adj_march_rev_kernel(MarchArgs a) {
  extern __shared__ __align__(16) double sm[];
  const Par P{(int)threadIdx.x, (int)blockDim.x};
  Work W;
  W.carve(sm, a.g.nr + 1);
  __shared__ int bad;
  if (P.tid == 0) bad = 0;
  __syncthreads();
  march_reverse_body(P, a, W, &bad);
  if (P.tid == 0 && bad) atomicOr(a.status, bad == 1 ? ST_NUMERIC : ST_ESCAPE);
}

#define GRID_LOOP(j, n) for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < (n); j += (int64_t)gridDim.x * blockDim.x)

__global__ void adj_beam_init_kernel(BeamConst c, BunchSpec q, Beam s, double *wgt, int *bin, const double *nm,
                                     const double *theta, const double *profile) {
  GRID_LOOP(j, c.n) beam_init_one(c, q, s, wgt, bin, nm, theta, profile, j);
}
__global__ void adj_deposit_kernel(BeamConst c, Beam s, const double *wgt, double *nb) {
  GRID_LOOP(j, c.n) deposit_one(c, s, wgt, nb, j);
}
__global__ void adj_normalize_kernel(BoundsRZ b, double *nb) {
  const int n1 = b.nr + 1;
  GRID_LOOP(t, (int64_t)(b.nxi + 1) * n1) nb[t] *= node_scale(b, (int)(t / n1), (int)(t % n1));
}
__global__ void adj_push_kernel(BeamConst c, Beam s0, Beam s1, const double *er, const double *ez, const double *bt) {
  GRID_LOOP(j, c.n) push_one(c, s0, s1, er, ez, bt, j);
}
__global__ void adj_loss_kernel(BeamConst c, Beam s, const double *wgt, double *sums) {
  double v[3] = {0.0, 0.0, 0.0};
  GRID_LOOP(j, c.n) loss_one(c, s, wgt, j, v);
  for (int q = 0; q < 3; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t != 0.0) atomicAdd(&sums[q], t);
  }
}
__global__ void adj_loss_rev_kernel(BeamConst c, Beam s, const double *wgt, const double *sums, double d0, double d1,
                                    Beam lam, double *lw) {
  GRID_LOOP(j, c.n) loss_reverse_one(c, s, wgt, sums, d0, d1, lam, lw, j);
}
__global__ void adj_push_rev_kernel(BeamConst c, Beam s0, const double *er, const double *ez, const double *bt,
                                    Beam lam, double *ler, double *lez, double *lbt) {
  GRID_LOOP(j, c.n) push_reverse_one(c, s0, er, ez, bt, lam, ler, lez, lbt, j);
}
__global__ void adj_deposit_rev_kernel(BeamConst c, Beam s, const double *wgt, const double *lnb, Beam lam, double *lw) {
  GRID_LOOP(j, c.n) deposit_reverse_one(c, s, wgt, lnb, lam, lw, j);
}
__global__ void adj_plasma_init_kernel(int np, int ppc, double dr, double u_th, const double *nm, double *r0,
                                       double *ur0, double *l, double *G0, double *w) {
  GRID_LOOP(j, np) plasma_init_one(ppc, dr, u_th, nm, r0, ur0, l, G0, w, (int)j);
}
__global__ void adj_rho0_kernel(Dims g, const double *r0, const double *w, double *rho0) {
  GRID_LOOP(i, g.nr + 1) rho0[i] = rho0_node(g, r0, w, (int)i);
}
__global__ void adj_theta_kernel(BeamConst c, const double *nm_b, const int *bin, Beam lam0, const double *lwb,
                                 const double *theta, const double *profile, double wu_w, double wu_d, Dims g,
                                 const double *nm_p, const double *r0, const double *lrho0, const double *lG0,
                                 const double *lw_p, const double *ll, const double *lur0, double u_th, int ppc,
                                 double *grad) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  GRID_LOOP(j, c.n) {
    double gb;
    theta_beam_one(c, nm_b, bin, lam0, lwb, theta, profile, wu_w, wu_d, j, v, &gb);
    if (gb != 0.0) atomicAdd(&grad[4 + bin[j]], gb);
  }
  GRID_LOOP(j, g.np) v[3] += theta_ring_one(g, nm_p, r0, lrho0, lG0, lw_p, ll, lur0, u_th, ppc, (int)j);
  for (int q = 0; q < 4; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t != 0.0) atomicAdd(&grad[q], t);
  }
}

}  // namespace

struct wake_adj {
  wake_params p{};
  int nsteps = 0, nbins = 0, B = 0, nblk = 0;
  cudaStream_t stream = nullptr;
  Dims g{};
  BeamConst bc{};
  size_t ng = 0;
  bool have_forward = false;
  std::vector<double> theta;
  // device
  double *theta_d = nullptr, *profile_d = nullptr;
  double *r0 = nullptr, *ur0 = nullptr, *l = nullptr, *G0 = nullptr, *w = nullptr, *rho0 = nullptr;
  double *beam = nullptr;  // (nsteps + 1) x 6 x n
  uint8_t *lost = nullptr;
  double *wgt = nullptr;
  int *bin = nullptr;
  double *nb = nullptr, *ez = nullptr, *er = nullptr, *bth = nullptr;  // nsteps grids each
  double *ckpt = nullptr, *tape = nullptr, *lring = nullptr, *nbh = nullptr, *lnbh = nullptr;
  double *lam = nullptr, *lwb = nullptr;  // 6 x n, n
  double *lez = nullptr, *ler = nullptr, *lbt = nullptr, *lnb = nullptr;  // one grid each
  double *lG0 = nullptr, *lw = nullptr, *ll = nullptr, *lur0 = nullptr, *lrho0 = nullptr;
  double *sums = nullptr, *grad = nullptr;
  const double *nm_p = nullptr, *nm_b = nullptr;  // caller's normals of the last forward
  int *status = nullptr;
};

namespace {

template <class T>
int adalloc(T **p, size_t bytes) {
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) return afail(WAKE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  return WAKE_OK;
}

size_t work_smem(int n1) { return sizeof(double) * (size_t)Work::kCount * n1; }

MarchArgs march_args(wake_adj *a, int t) {
  MarchArgs m{};
  m.g = a->g;
  m.B = a->B;
  m.nblk = a->nblk;
  m.r0 = a->r0;
  m.ur0 = a->ur0;
  m.l = a->l;
  m.G0 = a->G0;
  m.w = a->w;
  m.rho0 = a->rho0;
  m.nb = a->nb + (size_t)t * a->ng;
  m.ez = a->ez + (size_t)t * a->ng;
  m.er = a->er + (size_t)t * a->ng;
  m.bth = a->bth + (size_t)t * a->ng;
  m.ckpt = a->ckpt + (size_t)t * a->nblk * 2 * a->g.np;
  m.tape = a->tape;
  m.lring = a->lring;
  m.lez = a->lez;
  m.ler = a->ler;
  m.lbth = a->lbt;
  m.lnb = a->lnb;
  m.lG0 = a->lG0;
  m.lw = a->lw;
  m.ll = a->ll;
  m.lur0 = a->lur0;
  m.lrho0 = a->lrho0;
  m.nbh = a->nbh;
  m.lnbh = a->lnbh;
  m.status = a->status;
  return m;
}

Beam slot(wake_adj *a, int t) {
  const int64_t n = a->bc.n;
  double *p = a->beam + (size_t)t * 6 * n;
  return Beam{p, p + n, p + 2 * n, p + 3 * n, p + 4 * n, p + 5 * n, a->lost + (size_t)t * n};
}
Beam lam_of(wake_adj *a) {
  const int64_t n = a->bc.n;
  double *p = a->lam;
  return Beam{p, p + n, p + 2 * n, p + 3 * n, p + 4 * n, p + 5 * n, nullptr};
}

}  // namespace

extern "C" {

int wake_adjoint_init(const wake_params *p, int nsteps, int nbins, void *stream, wake_adj **out) {
  if (!p || !out) return afail(WAKE_EINVAL, "wake_adjoint_init: null argument");
  *out = nullptr;
  if (p->nr < 2 || p->nr > 256) return afail(WAKE_EINVAL, "wake_adjoint_init: need 2 <= nr <= 256");
  if (p->nxi < 2 || p->nxi > (1 << 16)) return afail(WAKE_EINVAL, "wake_adjoint_init: need 2 <= nxi <= 65536");
  if (p->ppc < 2 || p->ppc % 2 || (int64_t)p->nr * p->ppc > 8192)
    return afail(WAKE_EINVAL, "wake_adjoint_init: need an even ppc and nr*ppc <= 8192 (warm plasma)");
  if (nsteps < 1 || nbins < 0 || nbins > 1024) return afail(WAKE_EINVAL, "wake_adjoint_init: need nsteps >= 1, 0 <= nbins <= 1024");
  if (p->n_beam < 1 || p->n_drive < 1 || p->n_drive >= p->n_beam)
    return afail(WAKE_EINVAL, "wake_adjoint_init: need a drive and a witness bunch (0 < n_drive < n_beam)");
  if (!(p->rmax > 0) || !(p->ximax > 0) || !(p->sigma_r > 0) || !(p->sigma_zw > 0) || !(p->gamma_b > 1) || !(p->ds > 0))
    return afail(WAKE_EINVAL, "wake_adjoint_init: box, bunch sizes, gamma_b and ds must be positive");
  wake_adj *a = new wake_adj();
  a->p = *p;
  a->nsteps = nsteps;
  a->nbins = nbins;
  a->stream = (cudaStream_t)stream;
  const int n1 = p->nr + 1, np = p->nr * p->ppc;
  a->g = Dims{p->nr, p->nxi, np, p->rmax / p->nr, p->ximax / p->nxi, p->rmax};
  a->B = std::max(1, (int)std::lround(std::sqrt((double)(p->nxi + 1))));
  a->nblk = (p->nxi + 1 + a->B - 1) / a->B;
  a->bc.n = p->n_beam;
  a->bc.n_drive = p->n_drive;
  a->bc.nbins = nbins;
  a->bc.b = BoundsRZ{p->nr, p->nxi, p->rmax / p->nr, p->ximax / p->nxi, p->rmax, p->ximax};
  a->bc.dt = p->ds;
  a->bc.gamma_b = p->gamma_b;
  a->ng = (size_t)(p->nxi + 1) * n1;
  const size_t n = (size_t)p->n_beam, npb = sizeof(double) * np, gb = sizeof(double) * a->ng;
  int rc = WAKE_OK;
  if ((rc = adalloc(&a->theta_d, sizeof(double) * 4)) || (rc = adalloc(&a->profile_d, sizeof(double) * std::max(1, nbins))) ||
      (rc = adalloc(&a->r0, npb)) || (rc = adalloc(&a->ur0, npb)) || (rc = adalloc(&a->l, npb)) ||
      (rc = adalloc(&a->G0, npb)) || (rc = adalloc(&a->w, npb)) || (rc = adalloc(&a->rho0, sizeof(double) * n1)) ||
      (rc = adalloc(&a->beam, sizeof(double) * 6 * n * (nsteps + 1))) || (rc = adalloc(&a->lost, n * (nsteps + 1))) ||
      (rc = adalloc(&a->wgt, sizeof(double) * n)) || (rc = adalloc(&a->bin, sizeof(int) * n)) ||
      (rc = adalloc(&a->nb, gb * nsteps)) || (rc = adalloc(&a->ez, gb * nsteps)) || (rc = adalloc(&a->er, gb * nsteps)) ||
      (rc = adalloc(&a->bth, gb * nsteps)) || (rc = adalloc(&a->ckpt, npb * 2 * a->nblk * nsteps)) ||
      (rc = adalloc(&a->tape, sizeof(double) * slice_tape_doubles(n1, np) * a->B)) ||
      (rc = adalloc(&a->lring, npb * kLring)) || (rc = adalloc(&a->nbh, sizeof(double) * n1)) ||
      (rc = adalloc(&a->lnbh, sizeof(double) * n1)) || (rc = adalloc(&a->lam, sizeof(double) * 6 * n)) ||
      (rc = adalloc(&a->lwb, sizeof(double) * n)) || (rc = adalloc(&a->lez, gb)) || (rc = adalloc(&a->ler, gb)) ||
      (rc = adalloc(&a->lbt, gb)) || (rc = adalloc(&a->lnb, gb)) || (rc = adalloc(&a->lG0, npb)) ||
      (rc = adalloc(&a->lw, npb)) || (rc = adalloc(&a->ll, npb)) || (rc = adalloc(&a->lur0, npb)) ||
      (rc = adalloc(&a->lrho0, sizeof(double) * n1)) || (rc = adalloc(&a->sums, sizeof(double) * 3)) ||
      (rc = adalloc(&a->grad, sizeof(double) * (4 + std::max(1, nbins)))) || (rc = adalloc(&a->status, sizeof(int)))) {
    wake_adjoint_destroy(a);
    return rc;
  }
  if (cudaFuncSetAttribute(adj_march_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)work_smem(n1)) !=
          cudaSuccess ||
      cudaFuncSetAttribute(adj_march_rev_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)work_smem(n1)) !=
          cudaSuccess) {
    wake_adjoint_destroy(a);
    return afail(WAKE_ECUDA, "wake_adjoint_init: shared-memory attribute");
  }
  *out = a;
  return WAKE_OK;
}

int wake_adjoint_forward(wake_adj *a, const double *theta, const double *profile, const double *plasma_normals,
                         const double *beam_normals, double *obs) {
  if (!a || !theta || !plasma_normals || !beam_normals || !obs || (a->nbins > 0 && !profile))
    return afail(WAKE_EINVAL, "wake_adjoint_forward: null argument");
  if (!(theta[0] >= 0.0) || !(theta[2] > 0.0) || !(theta[3] >= 0.0))
    return afail(WAKE_EINVAL, "wake_adjoint_forward: need n_w >= 0, sigma_zd > 0, u_th >= 0");
  const wake_params &p = a->p;
  const cudaStream_t s = a->stream;
  const int n1 = p.nr + 1, np = a->g.np;
  a->theta.assign(theta, theta + 4);
  a->nm_p = plasma_normals;
  a->nm_b = beam_normals;
  ACUDA(cudaMemcpyAsync(a->theta_d, theta, sizeof(double) * 4, cudaMemcpyHostToDevice, s));
  if (a->nbins > 0) ACUDA(cudaMemcpyAsync(a->profile_d, profile, sizeof(double) * a->nbins, cudaMemcpyHostToDevice, s));
  ACUDA(cudaMemsetAsync(a->status, 0, sizeof(int), s));
  // plasma initial slice (warm: mirrored pairs) at temperature u_th = theta[3]
  adj_plasma_init_kernel<<<blocks_of(np), 256, 0, s>>>(np, p.ppc, a->g.dr, theta[3], plasma_normals, a->r0, a->ur0,
                                                       a->l, a->G0, a->w);
  adj_rho0_kernel<<<blocks_of(n1), 256, 0, s>>>(a->g, a->r0, a->w, a->rho0);
  const BunchSpec q{p.sigma_r, p.eps_n, p.xi_d, p.sigma_zw, p.n_d};
  adj_beam_init_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, q, slot(a, 0), a->wgt, a->bin, beam_normals,
                                                          a->theta_d, a->profile_d);
  ACUDA(cudaGetLastError());
  for (int t = 0; t < a->nsteps; ++t) {
    double *nb = a->nb + (size_t)t * a->ng;
    ACUDA(cudaMemsetAsync(nb, 0, sizeof(double) * a->ng, s));
    adj_deposit_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, t), a->wgt, nb);
    adj_normalize_kernel<<<blocks_of((int64_t)a->ng), 256, 0, s>>>(a->bc.b, nb);
    adj_march_fwd_kernel<<<1, kNT, work_smem(n1), s>>>(march_args(a, t));
    adj_push_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, t), slot(a, t + 1), a->er + (size_t)t * a->ng,
                                                       a->ez + (size_t)t * a->ng, a->bth + (size_t)t * a->ng);
    ACUDA(cudaGetLastError());
  }
  ACUDA(cudaMemsetAsync(a->sums, 0, sizeof(double) * 3, s));
  adj_loss_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, a->nsteps), a->wgt, a->sums);
  ACUDA(cudaGetLastError());
  double sums[3];
  int st = 0;
  ACUDA(cudaMemcpyAsync(sums, a->sums, sizeof(sums), cudaMemcpyDeviceToHost, s));
  ACUDA(cudaMemcpyAsync(&st, a->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  ACUDA(cudaStreamSynchronize(s));
  if (st & ST_NUMERIC) return afail(WAKE_ENUMERIC, "adjoint forward: Gamma <= 0 or a non-finite value");
  if (st & ST_ESCAPE) return afail(WAKE_EESCAPE, "adjoint forward: a plasma ring left [0, rmax]");
  if (!(sums[0] > 0.0)) return afail(WAKE_ESTATE, "adjoint forward: no surviving witness particle");
  const double M = sums[1] / sums[0];
  obs[0] = M;
  obs[1] = std::sqrt(std::max(sums[2] / sums[0] - M * M, 0.0));
  a->have_forward = true;
  return WAKE_OK;
}

int wake_adjoint_backward(wake_adj *a, const double *dobs, double *grad) {
  if (!a || !dobs || !grad) return afail(WAKE_EINVAL, "wake_adjoint_backward: null argument");
  if (!a->have_forward) return afail(WAKE_ESTATE, "wake_adjoint_backward before wake_adjoint_forward");
  const wake_params &p = a->p;
  const cudaStream_t s = a->stream;
  const int n1 = p.nr + 1, np = a->g.np;
  const size_t npb = sizeof(double) * np, gb = sizeof(double) * a->ng;
  ACUDA(cudaMemsetAsync(a->lG0, 0, npb, s));
  ACUDA(cudaMemsetAsync(a->lw, 0, npb, s));
  ACUDA(cudaMemsetAsync(a->ll, 0, npb, s));
  ACUDA(cudaMemsetAsync(a->lur0, 0, npb, s));
  ACUDA(cudaMemsetAsync(a->lrho0, 0, sizeof(double) * n1, s));
  ACUDA(cudaMemsetAsync(a->grad, 0, sizeof(double) * (4 + std::max(1, a->nbins)), s));
  Beam lam = lam_of(a);
  adj_loss_rev_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, a->nsteps), a->wgt, a->sums, dobs[0], dobs[1],
                                                         lam, a->lwb);
  ACUDA(cudaGetLastError());
  for (int t = a->nsteps - 1; t >= 0; --t) {
    const size_t off = (size_t)t * a->ng;
    ACUDA(cudaMemsetAsync(a->ler, 0, gb, s));
    ACUDA(cudaMemsetAsync(a->lez, 0, gb, s));
    ACUDA(cudaMemsetAsync(a->lbt, 0, gb, s));
    ACUDA(cudaMemsetAsync(a->lnb, 0, gb, s));
    adj_push_rev_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, t), a->er + off, a->ez + off, a->bth + off,
                                                           lam, a->ler, a->lez, a->lbt);
    adj_march_rev_kernel<<<1, kNT, work_smem(n1), s>>>(march_args(a, t));
    adj_deposit_rev_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, t), a->wgt, a->lnb, lam, a->lwb);
    ACUDA(cudaGetLastError());
  }
  const double s2pi = std::sqrt(2.0 * 3.14159265358979323846);
  const double wu_w = s2pi * p.sigma_r * p.sigma_r * p.sigma_zw / (double)(p.n_beam - p.n_drive);
  const double wu_d = p.n_d * s2pi * p.sigma_r * p.sigma_r / (double)p.n_drive;
  adj_theta_kernel<<<blocks_of(std::max<int64_t>(p.n_beam, np)), 256, 0, s>>>(
      a->bc, a->nm_b, a->bin, lam, a->lwb, a->theta_d, a->profile_d, wu_w, wu_d, a->g, a->nm_p, a->r0, a->lrho0,
      a->lG0, a->lw, a->ll, a->lur0, a->theta[3], p.ppc, a->grad);
  ACUDA(cudaGetLastError());
  int st = 0;
  ACUDA(cudaMemcpyAsync(grad, a->grad, sizeof(double) * (4 + a->nbins), cudaMemcpyDeviceToHost, s));
  ACUDA(cudaMemcpyAsync(&st, a->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  ACUDA(cudaStreamSynchronize(s));
  if (st) return afail(WAKE_ENUMERIC, "adjoint backward: a fault in the recomputed march");
  return WAKE_OK;
}

void wake_adjoint_destroy(wake_adj *a) {
  if (!a) return;
  if (a->stream) cudaStreamSynchronize(a->stream);
  else cudaDeviceSynchronize();
  void *ptrs[] = {a->theta_d, a->profile_d, a->r0, a->ur0, a->l, a->G0, a->w, a->rho0, a->beam, a->lost, a->wgt,
                  a->bin, a->nb, a->ez, a->er, a->bth, a->ckpt, a->tape, a->lring, a->nbh, a->lnbh, a->lam, a->lwb,
                  a->lez, a->ler, a->lbt, a->lnb, a->lG0, a->lw, a->ll, a->lur0, a->lrho0, a->sums, a->grad, a->status};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  delete a;
}

}  // extern "C"
