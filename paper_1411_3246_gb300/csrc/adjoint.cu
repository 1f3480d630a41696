// The adjoint form: gradients of the witness bunch's mean energy gain and rms energy spread
// (Sec. IV diagnostics) with respect to the witness peak density n_w (its charge), the
// witness delay xi_w - xi_d, the drive length sigma_zd, the plasma temperature u_th (Sec.
// II.A warm plasma) and per-bin multipliers of the witness current profile, through nsteps
// beam steps of deposit -> xi-march -> Boris push.  FP64 throughout.
//
// Forward (wake_adjoint_forward): beam states, beam densities and the field grids of every
// step are kept, and either every slice's intermediates (the full tape, when it fits) or the
// ring state of every B-th slice of every march (B ~ sqrt(Nxi)).
// Reverse (wake_adjoint_backward): per step, newest first, the Boris push is reversed
// particle by particle (its field adjoints are scattered onto the grid), then the march is
// reversed slice by slice (block by block from the checkpoints, each block recomputed with its
// intermediates kept, when there is no full tape), giving the adjoint of the step's beam
// density, which the reversed deposit turns into adjoints of the beam positions and weights.
// Both directions run pipelined across the beam steps (adj_fwd_pipe_kernel,
// adj_rev_pipe_kernel) or, as a fallback, one step at a time with one CTA marching.  The
// arithmetic of each piece is in adjoint_core.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
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

// ---------------------------------------------------------------------------------------
// pipelined steps: one CTA per beam step, many steps at once
// ---------------------------------------------------------------------------------------
// Forward.  The march of step t at slice k needs the beam density of rows <= k + 1, i.e. the
// particles of the xi cells <= k + 1 pushed by step t - 1.  The beam is ordered once by the
// xi cell of its initial state (order[], cell c holding positions cstart[c] .. cstart[c+1]-1,
// the lost particles in cell nxi); a particle slips less than a cell over the whole run (the
// host checks the slip rate), so at step t it sits in its cell b or in b + 1.  Step t's CTA
// pushes cell b once its slices b .. b + 2 are solved, deposits the pushed particles into step
// t+1's density grid, and publishes progress[t] = b + 1; step t+1's CTA waits (bounded) for
// progress[t] >= k + 2 before its slice k, and reads those rows through L2 into a private copy.
// Reverse, mirrored in xi and t.  Step t's reverse march needs, before its slice k, the field
// adjoints of slice k: the reversed pushes of the particles of cells >= k - 2, which need the
// adjoints of their state after step t, complete once step t+1 has reversed their deposit.
// Step t+1 reverses the deposit of cell b once its slices >= b - 1 are reversed (the density
// rows b .. b + 2 are then final) and publishes done_rev[t+1] = b.  Per particle the chain of
// adjoint updates therefore runs step by step, as in the sequential form; every value another
// CTA writes during the launch is read through L2.
constexpr int kAdjDrift = 8;  // a particle found outside its sorted cell b and b + 1

struct AdjPipe {
  MarchArgs m;                   // the march's constant part (grid, checkpoints, ring constants)
  int nsteps;
  size_t ng;
  double *nb, *ez, *er, *bth;    // per step, t * ng
  double *ckpt;                  // per step, t * ckpt_stride
  size_t ckpt_stride;
  double *tape, *lring, *nbh, *lnbh, *nbp, *lgrid, *lacc;  // per CTA
  size_t tape_stride, lring_stride, lacc_stride;
  BeamConst bc;
  double *beam;                  // slots t * 6 * n
  uint8_t *lost;                 // slots t * n
  const double *wgt;
  const int *order, *cstart;
  int *progress, *done_rev;
  double *lam, *lwb;
  long long spin_limit;
  double *ftape;                 // full_tape: every slice of every step, t * ftape_stride
  size_t ftape_stride;
};

__device__ __forceinline__ int adj_ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void adj_st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ Beam pipe_slot(const AdjPipe &a, int t) {
  const int64_t n = a.bc.n;
  double *p = a.beam + (size_t)t * 6 * n;
  return Beam{p, p + n, p + 2 * n, p + 3 * n, p + 4 * n, p + 5 * n, a.lost + (size_t)t * n};
}

__device__ __forceinline__ MarchArgs pipe_args(const AdjPipe &a, int t, int cta, bool reverse) {
  MarchArgs m = a.m;
  const int n1 = m.g.nr + 1, np = m.g.np;
  m.nb = reverse ? a.nb + (size_t)t * a.ng : a.nbp + (size_t)cta * a.ng;
  m.ez = a.ez + (size_t)t * a.ng;
  m.er = a.er + (size_t)t * a.ng;
  m.bth = a.bth + (size_t)t * a.ng;
  m.ckpt = a.ckpt + (size_t)t * a.ckpt_stride;
  // every slice of the step when the forward keeps them all, else two blocks per CTA (the
  // reverse recomputes ahead into the second)
  m.tape = a.ftape ? a.ftape + (size_t)t * a.ftape_stride : a.tape + (size_t)cta * 2 * a.tape_stride;
  m.lring = a.lring + (size_t)cta * a.lring_stride;
  m.nbh = a.nbh + (size_t)cta * n1;
  m.lnbh = a.lnbh + (size_t)cta * n1;
  double *lg = a.lgrid + (size_t)cta * 4 * a.ng;
  m.lez = lg;
  m.ler = lg + a.ng;
  m.lbth = lg + 2 * a.ng;
  m.lnb = lg + 3 * a.ng;
  double *la = a.lacc + (size_t)cta * a.lacc_stride;
  m.lG0 = la;
  m.lw = la + np;
  m.ll = la + 2 * (size_t)np;
  m.lur0 = la + 3 * (size_t)np;
  m.lrho0 = la + 4 * (size_t)np;
  return m;
}

// Thread 0 polls *flag until ok(value) (bounded; it also gives up once any CTA has timed out),
// then every thread meets at one barrier: the answer is block-uniform.  ctl[0]: given up.
template <class Ok>
__device__ __forceinline__ bool pipe_wait(const AdjPipe &a, const int *flag, int *ctl, Ok ok) {
  if (threadIdx.x == 0 && !ctl[0]) {
    long long it = 0;
    int v = adj_ld_acquire(flag);
    while (!ok(v)) {
      if (++it > a.spin_limit || (*(volatile int *)a.m.status & ST_TIMEOUT)) {
        atomicOr(a.m.status, ST_TIMEOUT);
        ctl[0] = 1;
        break;
      }
      __nanosleep(128);
      v = adj_ld_acquire(flag);
    }
  }
  __syncthreads();
  return ctl[0] == 0;
}

__global__ void __launch_bounds__(kNT, 1) adj_fwd_pipe_kernel(AdjPipe a) {
  extern __shared__ __align__(16) double sm[];
  const Par P{(int)threadIdx.x, (int)blockDim.x};
  Work W;
  W.carve(sm, a.m.g.nr + 1);
  __shared__ int bad, ctl[1];
  const int nxi = a.m.g.nxi, n1 = a.m.g.nr + 1;
  const double dxi = a.bc.b.dxi;
  for (int t = blockIdx.x; t < a.nsteps; t += gridDim.x) {
    if (P.tid == 0) {
      bad = 0;
      ctl[0] = 0;
    }
    __syncthreads();
    const MarchArgs m = pipe_args(a, t, blockIdx.x, false);
    const Beam s0 = pipe_slot(a, t), s1 = pipe_slot(a, t + 1);
    const double *nbt = a.nb + (size_t)t * a.ng;
    double *nbn = t + 1 < a.nsteps ? a.nb + (size_t)(t + 1) * a.ng : nullptr;
    double *nbp = a.nbp + (size_t)blockIdx.x * a.ng;
    int copied = 0;  // rows of nb[t] in the private copy
    auto before = [&](int k) -> bool {
      const int last = min(nxi, k + 1);
      if (t > 0 && !pipe_wait(a, a.progress + (t - 1), ctl, [&](int v) { return v >= min(nxi, k + 2); })) return false;
      for (int q = copied * n1 + P.tid; q < (last + 1) * n1; q += P.nt) nbp[q] = __ldcg(nbt + q);
      copied = last + 1;
      __syncthreads();
      return true;
    };
    auto push_cell = [&](int b) {
      for (int i = a.cstart[b] + P.tid; i < a.cstart[b + 1]; i += P.nt) {
        const int64_t j = a.order[i];
        if (b < nxi && !rd(s0.lost + j)) {
          int kk;
          double gg;
          cell_of(rd(s0.xi + j), dxi, nxi, kk, gg);
          if (kk != b && kk != b + 1) {  // its fields are not solved yet: flag, keep the state
            atomicOr(a.m.status, kAdjDrift);
            s1.x[j] = rd(s0.x + j); s1.y[j] = rd(s0.y + j); s1.ux[j] = rd(s0.ux + j);
            s1.uy[j] = rd(s0.uy + j); s1.uz[j] = rd(s0.uz + j); s1.xi[j] = rd(s0.xi + j);
            s1.lost[j] = 1;
            continue;
          }
        }
        push_one(a.bc, s0, s1, m.er, m.ez, m.bth, j);
        if (nbn) deposit_scaled_one(a.bc, s1, a.wgt, nbn, j);
      }
      __threadfence();
      __syncthreads();
      if (P.tid == 0) adj_st_release(a.progress + t, b + 1);
    };
    auto after = [&](int k) {
      if (k >= 2) push_cell(k - 2);
    };
    const bool ok = march_forward_body(P, m, W, &bad, before, after, a.ftape != nullptr);
    if (ok) {
      push_cell(nxi - 1);
      push_cell(nxi);  // the particles lost from the start: their state carried to the next slot
    }
    if (P.tid == 0 && bad) atomicOr(a.m.status, bad == 1 ? ST_NUMERIC : ST_ESCAPE);
    __syncthreads();
    if (!ok) break;
  }
}

__global__ void __launch_bounds__(kNT, 1) adj_rev_pipe_kernel(AdjPipe a) {
  extern __shared__ __align__(16) double sm[];
  const Par P{(int)threadIdx.x, (int)blockDim.x};
  Work W;
  W.carve(sm, a.m.g.nr + 1);
  __shared__ int bad, ctl[2];
  const int nxi = a.m.g.nxi;
  const double dxi = a.bc.b.dxi;
  const int64_t n = a.bc.n;
  const Beam lam{a.lam, a.lam + n, a.lam + 2 * n, a.lam + 3 * n, a.lam + 4 * n, a.lam + 5 * n, nullptr};
  for (int it = blockIdx.x; it < a.nsteps; it += gridDim.x) {
    const int t = a.nsteps - 1 - it;
    if (P.tid == 0) {
      bad = 0;
      ctl[0] = 0;
    }
    const MarchArgs m = pipe_args(a, t, blockIdx.x, true);
    double *lg = a.lgrid + (size_t)blockIdx.x * 4 * a.ng;
    for (size_t q = P.tid; q < 4 * a.ng; q += P.nt) lg[q] = 0.0;
    __syncthreads();
    double *ler = lg + a.ng, *lez = lg, *lbt = lg + 2 * a.ng, *lnb = lg + 3 * a.ng;
    const Beam s0 = pipe_slot(a, t);
    int next_push = nxi - 1;  // the highest cell whose push is not yet reversed
    // wait for step t+1 to have reversed the deposit of cell b; while it has not, first do the
    // march's pending work (the recomputation of the block below), then wait (bounded)
    auto ready_for = [&](int b, auto &idle) -> bool {
      if (t + 1 >= a.nsteps) return true;
      if (P.tid == 0) ctl[1] = adj_ld_acquire(a.done_rev + (t + 1)) <= b;
      __syncthreads();
      if (!ctl[1]) idle();
      return pipe_wait(a, a.done_rev + (t + 1), ctl, [&](int v) { return v <= b; });
    };
    auto push_rev_cell = [&](int b, auto &idle) -> bool {
      if (!ready_for(b, idle)) return false;
      for (int i = a.cstart[b] + P.tid; i < a.cstart[b + 1]; i += P.nt) {
        const int64_t j = a.order[i];
        if (s0.lost[j]) continue;
        int kk;
        double gg;
        cell_of(s0.xi[j], dxi, nxi, kk, gg);
        if (kk != b && kk != b + 1) {
          atomicOr(a.m.status, kAdjDrift);
          continue;
        }
        push_reverse_one(a.bc, s0, m.er, m.ez, m.bth, lam, ler, lez, lbt, j);
      }
      __syncthreads();
      return true;
    };
    auto dep_rev_cell = [&](int b) {
      for (int i = a.cstart[b] + P.tid; i < a.cstart[b + 1]; i += P.nt)
        deposit_reverse_one(a.bc, s0, a.wgt, lnb, lam, a.lwb, a.order[i]);
      __threadfence();
      __syncthreads();
      if (P.tid == 0) adj_st_release(a.done_rev + t, b);
    };
    auto pre = [&](int k, auto &idle) -> bool {
      const int lo = k - 2 > 0 ? k - 2 : 0;
      while (next_push >= lo) {
        if (!push_rev_cell(next_push, idle)) return false;
        --next_push;
      }
      return true;
    };
    auto post = [&](int k) {
      if (k + 1 <= nxi - 1) dep_rev_cell(k + 1);
    };
    // two tape buffers: a wait on step t+1 is first used to recompute the block below
    const bool ok = a.ftape ? march_reverse_body(P, m, W, &bad, pre, post, nullptr, true)
                            : march_reverse_body(P, m, W, &bad, pre, post, m.tape + a.tape_stride);
    if (ok) dep_rev_cell(0);
    if (P.tid == 0 && bad) atomicOr(a.m.status, bad == 1 ? ST_NUMERIC : ST_ESCAPE);
    __syncthreads();
    if (!ok) break;
  }
}

// The ring-constant adjoints of every CTA summed: out[q] = sum over CTAs of lacc[cta][q].
__global__ void adj_lacc_sum_kernel(const double *lacc, size_t stride, int ctas, size_t len, double *out) {
  GRID_LOOP(q, (int64_t)len) {
    double s = 0.0;
    for (int c = 0; c < ctas; ++c) s += lacc[(size_t)c * stride + q];
    out[q] += s;
  }
}

// Largest xi slip rate (1 + u_perp^2) / (gamma (gamma + u_z)) of the live particles of a
// state, as the bits of a non-negative double (ordered like unsigned integers).
__global__ void adj_slip_kernel(BeamConst c, Beam s, unsigned long long *out) {
  double mx = 0.0;
  GRID_LOOP(j, c.n) {
    if (s.lost[j]) continue;
    const double up2 = s.ux[j] * s.ux[j] + s.uy[j] * s.uy[j], g = sqrt(1.0 + up2 + s.uz[j] * s.uz[j]);
    mx = fmax(mx, (1.0 + up2) / (g * (g + s.uz[j])));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}
// Counting sort of the particles by the xi cell of a state (lost: cell nxi).
__device__ __forceinline__ int adj_cell(const BeamConst &c, const Beam &s, int64_t j) {
  if (s.lost[j]) return c.b.nxi;
  int k;
  double g;
  cell_of(s.xi[j], c.b.dxi, c.b.nxi, k, g);
  return k;
}
__global__ void adj_cell_count_kernel(BeamConst c, Beam s, int *count) {
  GRID_LOOP(j, c.n) atomicAdd(&count[adj_cell(c, s, j)], 1);
}
// exclusive scan of nb counts into start[0..nb] and cursor (one block of 1024 threads)
__global__ void adj_cell_scan_kernel(const int *count, int *start, int *cursor, int nb) {
  __shared__ int part[1024];
  const int t = threadIdx.x, E = (nb + 1023) / 1024, beg = min(nb, t * E), end = min(nb, beg + E);
  int s = 0;
  for (int q = beg; q < end; ++q) s += count[q];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;
  for (int q = beg; q < end; ++q) {
    start[q] = run;
    cursor[q] = run;
    run += count[q];
  }
  if (t == 1023) start[nb] = part[1023];
}
__global__ void adj_cell_scatter_kernel(BeamConst c, Beam s, int *cursor, int *order) {
  GRID_LOOP(j, c.n) order[atomicAdd(&cursor[adj_cell(c, s, j)], 1)] = (int)j;
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
  // pipelined steps (pipe_ctas > 0): per-CTA scratch, the beam's cell order, the chains
  int pipe_ctas = 0;
  bool pipelined = false;  // the last forward ran pipelined (the backward follows it)
  long long spin_limit = 1LL << 24;
  double *ftape = nullptr;  // the full tape (every slice of every step), when it fits
  size_t ftape_stride = 0;
  double *p_tape = nullptr, *p_lring = nullptr, *p_nbh = nullptr, *p_lnbh = nullptr, *p_nbp = nullptr,
         *p_lgrid = nullptr, *p_lacc = nullptr;
  size_t p_tape_stride = 0, p_lring_stride = 0, p_lacc_stride = 0;
  int *order = nullptr, *cstart = nullptr, *ccount = nullptr, *ccursor = nullptr, *progress = nullptr,
      *done_rev = nullptr;
  unsigned long long *slip = nullptr;
};

namespace {

template <class T>
int adalloc(T **p, size_t bytes) {
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) return afail(WAKE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  return WAKE_OK;
}

size_t work_smem(int n1) { return sizeof(double) * (size_t)Work::kCount * n1; }

AdjPipe pipe_of(wake_adj *a) {
  AdjPipe q{};
  q.m.g = a->g;
  q.m.B = a->B;
  q.m.nblk = a->nblk;
  q.m.r0 = a->r0;
  q.m.ur0 = a->ur0;
  q.m.l = a->l;
  q.m.G0 = a->G0;
  q.m.w = a->w;
  q.m.rho0 = a->rho0;
  q.m.status = a->status;
  q.nsteps = a->nsteps;
  q.ng = a->ng;
  q.nb = a->nb;
  q.ez = a->ez;
  q.er = a->er;
  q.bth = a->bth;
  q.ckpt = a->ckpt;
  q.ckpt_stride = (size_t)a->nblk * 2 * a->g.np;
  q.tape = a->p_tape;
  q.lring = a->p_lring;
  q.nbh = a->p_nbh;
  q.lnbh = a->p_lnbh;
  q.nbp = a->p_nbp;
  q.lgrid = a->p_lgrid;
  q.lacc = a->p_lacc;
  q.tape_stride = a->p_tape_stride;
  q.lring_stride = a->p_lring_stride;
  q.lacc_stride = a->p_lacc_stride;
  q.bc = a->bc;
  q.beam = a->beam;
  q.lost = a->lost;
  q.wgt = a->wgt;
  q.order = a->order;
  q.cstart = a->cstart;
  q.progress = a->progress;
  q.done_rev = a->done_rev;
  q.lam = a->lam;
  q.lwb = a->lwb;
  q.spin_limit = a->spin_limit;
  q.ftape = a->ftape;
  q.ftape_stride = a->ftape_stride;
  return q;
}

// CTAs of the pipelined kernels that can be resident at once (one per SM), at most nsteps.
int pipe_ctas_for(int nsteps, int n1) {
  int dev = 0, sms = 0, f = 0, r = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f, adj_fwd_pipe_kernel, kNT, work_smem(n1)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, adj_rev_pipe_kernel, kNT, work_smem(n1)) != cudaSuccess)
    return 0;
  return std::min(nsteps, std::min(f, r) * sms);
}

cudaError_t launch_pipe(const void *kern, int ctas, size_t smem, const AdjPipe &q, cudaStream_t s) {
  AdjPipe arg = q;
  void *args[] = {&arg};
  return cudaLaunchCooperativeKernel(kern, dim3(ctas), dim3(kNT), args, smem, s);
}

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
  if (p->geometry != WAKE_CYLINDRICAL) return afail(WAKE_EINVAL, "wake_adjoint_init: the adjoint is cylindrical only");
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
          cudaSuccess ||
      cudaFuncSetAttribute(adj_fwd_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)work_smem(n1)) !=
          cudaSuccess ||
      cudaFuncSetAttribute(adj_rev_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)work_smem(n1)) !=
          cudaSuccess) {
    wake_adjoint_destroy(a);
    return afail(WAKE_ECUDA, "wake_adjoint_init: shared-memory attribute");
  }
  if (const char *e = std::getenv("WAKE_SPIN_LIMIT")) a->spin_limit = std::max(0LL, std::atoll(e));
  // pipelined steps: unless WAKE_ADJOINT_PIPELINE=0, when two or more steps can run at once
  const char *pe = std::getenv("WAKE_ADJOINT_PIPELINE");
  const int ctas = (pe && std::atoi(pe) == 0) ? 0 : pipe_ctas_for(nsteps, n1);
  if (ctas >= 2) {
    // every slice's intermediates of every step, when that takes at most a quarter of the free
    // device memory: the reverse then recomputes nothing (its waits on the next step's reverse
    // would otherwise stall on that step's recomputations); else two blocks per CTA
    size_t free_b = 0, total_b = 0;
    const size_t fstride = slice_tape_doubles(n1, np) * (size_t)(p->nxi + 1);
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && sizeof(double) * fstride * nsteps <= free_b / 4 &&
        !(std::getenv("WAKE_ADJOINT_FULL_TAPE") && std::atoi(std::getenv("WAKE_ADJOINT_FULL_TAPE")) == 0)) {
      if ((rc = adalloc(&a->ftape, sizeof(double) * fstride * nsteps))) {
        wake_adjoint_destroy(a);
        return rc;
      }
      a->ftape_stride = fstride;
    }
    a->p_tape_stride = slice_tape_doubles(n1, np) * a->B;
    a->p_lring_stride = (size_t)np * kLring;
    a->p_lacc_stride = (size_t)4 * np + n1;
    if ((!a->ftape && (rc = adalloc(&a->p_tape, sizeof(double) * a->p_tape_stride * 2 * ctas))) ||
        (rc = adalloc(&a->p_lring, sizeof(double) * a->p_lring_stride * ctas)) ||
        (rc = adalloc(&a->p_nbh, sizeof(double) * n1 * ctas)) || (rc = adalloc(&a->p_lnbh, sizeof(double) * n1 * ctas)) ||
        (rc = adalloc(&a->p_nbp, gb * ctas)) || (rc = adalloc(&a->p_lgrid, 4 * gb * ctas)) ||
        (rc = adalloc(&a->p_lacc, sizeof(double) * a->p_lacc_stride * ctas)) ||
        (rc = adalloc(&a->order, sizeof(int) * n)) || (rc = adalloc(&a->cstart, sizeof(int) * (p->nxi + 2))) ||
        (rc = adalloc(&a->ccount, sizeof(int) * (p->nxi + 2))) || (rc = adalloc(&a->ccursor, sizeof(int) * (p->nxi + 2))) ||
        (rc = adalloc(&a->progress, sizeof(int) * nsteps)) || (rc = adalloc(&a->done_rev, sizeof(int) * nsteps)) ||
        (rc = adalloc(&a->slip, sizeof(unsigned long long)))) {
      wake_adjoint_destroy(a);
      return rc;
    }
    a->pipe_ctas = ctas;
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
  a->pipelined = false;
  if (a->pipe_ctas >= 2) {
    // pipelined when no particle can slip a cell over the run: four times the fastest
    // particle's present slip rate over all steps stays below half a cell
    ACUDA(cudaMemsetAsync(a->slip, 0, sizeof(unsigned long long), s));
    adj_slip_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, 0), a->slip);
    ACUDA(cudaGetLastError());
    unsigned long long bits = 0;
    ACUDA(cudaMemcpyAsync(&bits, a->slip, sizeof(bits), cudaMemcpyDeviceToHost, s));
    ACUDA(cudaStreamSynchronize(s));
    double rate;
    std::memcpy(&rate, &bits, sizeof(rate));
    a->pipelined = 4.0 * rate * p.ds * a->nsteps < 0.5 * a->g.dxi;
  }
  if (a->pipelined) {
    const int nbins = p.nxi + 1;
    ACUDA(cudaMemsetAsync(a->ccount, 0, sizeof(int) * (nbins + 1), s));
    adj_cell_count_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, 0), a->ccount);
    adj_cell_scan_kernel<<<1, 1024, 0, s>>>(a->ccount, a->cstart, a->ccursor, nbins);
    adj_cell_scatter_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, 0), a->ccursor, a->order);
    ACUDA(cudaMemsetAsync(a->nb, 0, sizeof(double) * a->ng * a->nsteps, s));
    adj_deposit_kernel<<<blocks_of(p.n_beam), 256, 0, s>>>(a->bc, slot(a, 0), a->wgt, a->nb);
    adj_normalize_kernel<<<blocks_of((int64_t)a->ng), 256, 0, s>>>(a->bc.b, a->nb);
    ACUDA(cudaMemsetAsync(a->progress, 0, sizeof(int) * a->nsteps, s));
    ACUDA(cudaGetLastError());
    ACUDA(launch_pipe((const void *)adj_fwd_pipe_kernel, std::min(a->pipe_ctas, a->nsteps), work_smem(n1), pipe_of(a), s));
  } else {
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
  if (st & ST_TIMEOUT) return afail(WAKE_ETIMEOUT, "adjoint forward: a bounded device wait gave up");
  if (st & kAdjDrift) return afail(WAKE_ESTATE, "adjoint forward: a beam particle slipped more than one xi cell");
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
  if (a->pipelined) {
    const int ctas = std::min(a->pipe_ctas, a->nsteps);
    ACUDA(cudaMemsetAsync(a->p_lacc, 0, sizeof(double) * a->p_lacc_stride * ctas, s));
    ACUDA(cudaMemsetAsync(a->done_rev, 0x7f, sizeof(int) * a->nsteps, s));  // 0x7f7f7f7f: no cell yet
    ACUDA(launch_pipe((const void *)adj_rev_pipe_kernel, ctas, work_smem(n1), pipe_of(a), s));
    const double *la = a->p_lacc;
    adj_lacc_sum_kernel<<<blocks_of(np), 256, 0, s>>>(la, a->p_lacc_stride, ctas, (size_t)np, a->lG0);
    adj_lacc_sum_kernel<<<blocks_of(np), 256, 0, s>>>(la + np, a->p_lacc_stride, ctas, (size_t)np, a->lw);
    adj_lacc_sum_kernel<<<blocks_of(np), 256, 0, s>>>(la + 2 * (size_t)np, a->p_lacc_stride, ctas, (size_t)np, a->ll);
    adj_lacc_sum_kernel<<<blocks_of(np), 256, 0, s>>>(la + 3 * (size_t)np, a->p_lacc_stride, ctas, (size_t)np, a->lur0);
    adj_lacc_sum_kernel<<<blocks_of(n1), 256, 0, s>>>(la + 4 * (size_t)np, a->p_lacc_stride, ctas, (size_t)n1, a->lrho0);
    ACUDA(cudaGetLastError());
  }
  for (int t = a->pipelined ? -1 : a->nsteps - 1; t >= 0; --t) {
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
  if (st & ST_TIMEOUT) return afail(WAKE_ETIMEOUT, "adjoint backward: a bounded device wait gave up");
  if (st & kAdjDrift) return afail(WAKE_ESTATE, "adjoint backward: a beam particle slipped more than one xi cell");
  if (st) return afail(WAKE_ENUMERIC, "adjoint backward: a fault in the recomputed march");
  return WAKE_OK;
}

void wake_adjoint_destroy(wake_adj *a) {
  if (!a) return;
  if (a->stream) cudaStreamSynchronize(a->stream);
  else cudaDeviceSynchronize();
  void *ptrs[] = {a->theta_d, a->profile_d, a->r0, a->ur0, a->l, a->G0, a->w, a->rho0, a->beam, a->lost, a->wgt,
                  a->bin, a->nb, a->ez, a->er, a->bth, a->ckpt, a->tape, a->lring, a->nbh, a->lnbh, a->lam, a->lwb,
                  a->lez, a->ler, a->lbt, a->lnb, a->lG0, a->lw, a->ll, a->lur0, a->lrho0, a->sums, a->grad, a->status,
                  a->ftape, a->p_tape, a->p_lring, a->p_nbh, a->p_lnbh, a->p_nbp, a->p_lgrid, a->p_lacc, a->order, a->cstart,
                  a->ccount, a->ccursor, a->progress, a->done_rev, a->slip};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  delete a;
}

}  // extern "C"
