// Pipelined beam steps.  A beam step is deposit -> xi-march -> push (Sec. II.A, last
// paragraph); consecutive steps are sequential, but the march of step t+1 at slice k only
// needs the beam density of rows <= k+1, i.e. the beam particles of the xi cells <= k+1 pushed
// by step t.  Beam particles slip back in xi by dt (1 - v_z) ~ 1e-9 per step (gamma = 4e4), so
// a particle stays in its cell or moves to the next one.  One persistent cooperative launch
// therefore runs many steps at once, one CTA per SM, each CTA marching its own step a few
// slices behind the previous step's CTA:
//   - step t's CTA keeps the fields of its last slices in shared memory; once slice k is
//     solved it pushes the beam particles in cell b = k - 1 (their fields lie in slices b and
//     b+1) and deposits them straight into the beam-density grid of step t+1;
//   - it then publishes progress[t] = b + 1 (release); step t+1's CTA waits (acquire, bounded)
//     for progress[t] >= k + 2 before it reads rows <= k + 1 of its grid.
// Step t+1 thus trails step t by two slices, which sets the pace of a launch whose steps
// outnumber the SMs.  A particle sorted into cell b that has slipped into a later cell is
// listed and pushed with that cell.  Every step has its own density grid (zeroed before the
// launch), so no grid is reused within a launch.  A wait that exceeds its bound sets
// ST_TIMEOUT and the CTA leaves cleanly; a particle found behind its sorted cell sets ST_DRIFT.
#pragma once

#include "beam.cuh"
#include "march.cuh"
#include "march_wide.cuh"

namespace wake {

constexpr int ST_DRIFT = 8;
constexpr int ST_LISTFULL = 16;  // more slipped particles than a step's lists hold

struct PipeArgs {
  SimDesc d;              // the simulation (plasma, output grids, status)
  void *grids;            // nsteps + 1 beam-density grids (G), grid t at t * ng
  size_t ng;              // nodes per grid
  int *progress;          // nsteps counters: sorted cells pushed by step t
  int nsteps;
  int write_last;         // write the last step's fields to the output grids
  // beam (sorted by xi cell; cell b holds particles bin_start[b] .. bin_start[b+1]-1)
  void *x, *y, *ux, *uy;
  double *xi, *uz;        // FP64, or (BT float) float-float pairs
  uint8_t *flags;
  const int *bin_start;
  void *w;               // per-particle weights (BT)
  double ds;
  float2 ffi, ffx;        // 1/dxi and ximax as float-float pairs
  // the push's constants in FP32 for the mixed form: 1/dr, ds, rmax, and the deposit's
  // 1/(dr^2 dxi) (slab: 1/(dr dxi))
  float f_inv_dr, f_ds, f_rmax, f_wq;
  long long spin_limit;   // polls before a wait gives up
  void *ring_bufs;        // per-CTA ring slot storage (FP64 and wide forms)
  size_t ring_stride;
  void *win_bufs;         // per-CTA field windows in global memory (wide form)
  size_t win_stride;
  // particles found past their sorted cell within the launch: step t lists them (index,
  // target cell) and pushes them with their target.  Two lists per step.  Those found in the
  // next cell (entries made while cell b is pushed, all for cell b + 1, which reads only
  // them) go to a ring of near_cap entries at near_list[t * near_cap ...], defer_cnt[2t]
  // counting every entry made; only two cells' entries are alive at once, so the ring holds
  // a few cells' worth.  The rest (two or more cells on) go to defer_list[t * defer_cap ...],
  // counted in defer_cnt[2t + 1] and read in full by every cell.  target[j] is the latest
  // target any step gave particle j (-1: none).
  int *defer_cnt;
  int2 *defer_list;
  int defer_cap;
  int2 *near_list;
  int near_cap;
  int *target;
};

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <class Pol, int NT>
struct PipeHooks {
  using R = typename Pol::R;
  using G = typename Pol::G;
  using BT = R;
  using W = BeamWide<BT>;
  using Box = typename W::Box;
  static constexpr bool kTraj = false;
  static constexpr bool kTrap = false;
  const PipeArgs &a;
  int t;          // step within the launch
  R *win;         // 4 slices x (E_r, E_z, B_theta) x n1
  int *ctl;       // [0] abort flag, [1] progress seen of step t-1
  int n1, nr, nxi;
  double dr, dxi, rmax, ximax;

  __device__ __forceinline__ const G *grid(int s) const { return (const G *)a.grids + (size_t)s * a.ng; }

  // rows <= k+1 of this step's grid are final once progress[t-1] >= min(nxi, k + 2).  Thread 0
  // polls (bounded; it also gives up as soon as another CTA has timed out), every thread then
  // meets at one barrier, so the decision is uniform.
  __device__ __forceinline__ bool wait_rows(int k) {
    if (t == 0) return true;
    const int need = min(nxi, k + 2);
    if (threadIdx.x == 0 && ctl[1] < need) {
      long long it = 0;
      int v = ld_acquire(&a.progress[t - 1]);
      while (v < need) {
        if (++it > a.spin_limit || (*(volatile int *)a.d.status & ST_TIMEOUT)) {
          flag(a.d.status, ST_TIMEOUT);
          ctl[0] = 1;
          break;
        }
        __nanosleep(128);
        v = ld_acquire(&a.progress[t - 1]);
      }
      ctl[1] = v;
    }
    __syncthreads();
    return ctl[0] == 0;
  }
  __device__ __forceinline__ R nb_row(int row, int m) const { return (R)__ldcg(grid(t) + (size_t)row * n1 + m); }

  __device__ __forceinline__ void slice_done(int k, MarchSmem<Pol> &sm) {
    R *w = win + (size_t)(k & 3) * 3 * n1;
    const bool out = a.write_last && t == a.nsteps - 1;
    G *o1 = (G *)a.d.psi + (size_t)k * n1, *o2 = (G *)a.d.ez + (size_t)k * n1, *o3 = (G *)a.d.er + (size_t)k * n1,
      *o4 = (G *)a.d.bth + (size_t)k * n1;
    for (int m = threadIdx.x; m < n1; m += NT) {
      const R ps = sm.psi[m], e = sm.ez[m], b = sm.bth[m];
      if (!(isfinite(ps) && isfinite(e) && isfinite(b))) flag(a.d.status, ST_NUMERIC);
      const R er = m > 0 ? b - sm.dpsi[m] : (R)0;
      w[m] = er;
      w[n1 + m] = e;
      w[2 * n1 + m] = b;
      if (out) {
        o1[m] = (G)ps;
        o2[m] = (G)e;
        o3[m] = (G)er;
        o4[m] = (G)b;
      }
    }
    __syncthreads();
    if (k >= 1) push_cell(k - 1);
  }
  __device__ __forceinline__ void finish(MarchSmem<Pol> &) {}  // slice nxi pushed cell nxi - 1

  // A particle's state as the push reads it, loaded in one go: the flag, xi and target
  // checks then wait for one round trip to L2 instead of a chain of them.  (Loading several
  // particles per thread ahead of their stores spilled registers of the march and was slower.)
  struct Part {
    BT x, y, ux, uy, w;
    typename W::T xi, uz;
    int tgt;
    uint8_t fl;
  };
  __device__ __forceinline__ void load_part(int j, Part &p) const {
    p.fl = __ldcg(a.flags + j);
    p.xi = W::ldcg(a.xi, j);
    p.tgt = __ldcg(a.target + j);
    p.x = __ldcg((const BT *)a.x + j);
    p.y = __ldcg((const BT *)a.y + j);
    p.ux = __ldcg((const BT *)a.ux + j);
    p.uy = __ldcg((const BT *)a.uy + j);
    p.uz = W::ldcg(a.uz, j);
    p.w = __ldcg((const BT *)a.w + j);
  }

  // Push particle j (state p), found in cell kk (fields of slices kk, kk+1 in the window), and
  // deposit it into the grid of step t+1.
  __device__ __forceinline__ void push_one(int j, const Part &p, int kk, BT g, const Box &bx) {
    BT *X = (BT *)a.x, *Y = (BT *)a.y, *UX = (BT *)a.ux, *UY = (BT *)a.uy;
    G *nbn = (G *)a.grids + (size_t)(t + 1) * a.ng;
    constexpr bool slab = Pol::kSlab;
    constexpr bool f32 = std::is_same_v<BT, float>;  // constants from the arguments: no FP64
    const BT inv_dr = f32 ? (BT)a.f_inv_dr : (BT)(1.0 / dr), dt = f32 ? (BT)a.f_ds : (BT)a.ds,
             Rw = f32 ? (BT)a.f_rmax : (BT)rmax;
    const uint8_t fl = p.fl;
    BT x = p.x, y = p.y, ux = p.ux, uy = p.uy;
    typename W::T xi = p.xi, uzd = p.uz;
    const BT r = sqrt(x * x + y * y);
    int c;
    BT f;
    locate(r, inv_dr, nr, c, f);
    const R *w0 = win + (size_t)(kk & 3) * 3 * n1, *w1 = win + (size_t)((kk + 1) & 3) * 3 * n1;
    const BT a00 = ((BT)1 - f) * ((BT)1 - g), a01 = f * ((BT)1 - g), a10 = ((BT)1 - f) * g, a11 = f * g;
    const BT Er = a00 * w0[c] + a01 * w0[c + 1] + a10 * w1[c] + a11 * w1[c + 1];
    const BT Ez = a00 * w0[n1 + c] + a01 * w0[n1 + c + 1] + a10 * w1[n1 + c] + a11 * w1[n1 + c + 1];
    const BT Bt = a00 * w0[2 * n1 + c] + a01 * w0[2 * n1 + c + 1] + a10 * w1[2 * n1 + c] + a11 * w1[2 * n1 + c + 1];
    boris_step<BT>(x, y, ux, uy, xi, uzd, r, Er, Ez, Bt, dt);
    X[j] = x;
    Y[j] = y;
    UX[j] = ux;
    UY[j] = uy;
    W::st(a.xi, j, xi);
    W::st(a.uz, j, uzd);
    const BT rn = sqrt(x * x + y * y);
    if (!(W::inside(xi, bx) && rn < Rw)) {
      a.flags[j] = fl | 1;
      return;
    }
    // deposit into the next step's grid: bilinear hats over the hat volumes V_i = i dr^2
    // (dr^2/6 on the axis, dr^2 (nr/2 - 1/6) at the wall) in r, dxi (dxi/2 at the two end
    // slices) in xi
    int c2, k2;
    BT f2, g2;
    locate(rn, inv_dr, nr, c2, f2);
    W::cell(xi, bx, nxi, k2, g2);
    // 1 / V_i = iv(i) / dr^2 (slab: iv(i) / dx, the hat width halved at x = 0 and at the wall)
    const BT wq = p.w * (f32 ? (BT)a.f_wq : (BT)(slab ? 1.0 / (dr * dxi) : 1.0 / (dr * dr * dxi)));
    auto iv = [&](int i) -> BT {
      if (slab) return (i == 0 || i == nr) ? (BT)2 : (BT)1;
      return i == 0 ? (BT)6 : (i == nr ? (BT)1 / ((BT)nr * (BT)0.5 - (BT)(1.0 / 6.0)) : (BT)1 / (BT)i);
    };
    const BT ix0 = k2 == 0 ? (BT)2 : (BT)1, ix1 = k2 + 1 == nxi ? (BT)2 : (BT)1;
    const BT v0 = iv(c2), v1 = iv(c2 + 1);
    const BT s00 = wq * v0 * ix0, s01 = wq * v1 * ix0, s10 = wq * v0 * ix1, s11 = wq * v1 * ix1;
    G *row = nbn + (size_t)k2 * n1 + c2;
    atomicAdd(row, (G)(s00 * ((BT)1 - f2) * ((BT)1 - g2)));
    atomicAdd(row + 1, (G)(s01 * f2 * ((BT)1 - g2)));
    atomicAdd(row + n1, (G)(s10 * ((BT)1 - f2) * g2));
    atomicAdd(row + n1 + 1, (G)(s11 * f2 * g2));
  }

  // List particle j (state p), met while cell b is pushed, for the push of cell tgt > b.  A
  // next-cell entry may not overwrite the entries of cell b - 1 that cell b is still reading
  // (from ctl[2] on).
  __device__ __forceinline__ void defer(int b, int j, const Part &p, int tgt) {
    bool ok;
    if (tgt == b + 1) {
      const int q = atomicAdd(a.defer_cnt + 2 * t, 1);
      ok = q - ctl[2] < a.near_cap;
      if (ok) a.near_list[(size_t)t * a.near_cap + q % a.near_cap] = make_int2(j, tgt);
    } else {
      const int q = atomicAdd(a.defer_cnt + 2 * t + 1, 1);
      ok = q < a.defer_cap;
      if (ok) a.defer_list[(size_t)t * a.defer_cap + q] = make_int2(j, tgt);
    }
    if (!ok) {
      flag(a.d.status, ST_LISTFULL);
      return;
    }
    if (tgt > p.tgt) a.target[j] = tgt;
  }

  // A listed particle j for cell b: pushed, listed again if it has slipped on.  (An index
  // outside the sorted beam can only come from a ring slot overwritten after an overflow,
  // which has raised ST_LISTFULL: it is skipped.)
  __device__ __forceinline__ void push_listed(int b, int j, const Box &bx) {
    if (j < 0 || j >= a.bin_start[nxi + 1]) return;
    Part p;
    load_part(j, p);
    if (p.fl & 1) return;
    int kk;
    BT g;
    W::cell(p.xi, bx, nxi, kk, g);
    if (kk > b) {
      defer(b, j, p, kk);
      return;
    }
    if (kk != b) {
      flag(a.d.status, ST_DRIFT);
      return;
    }
    push_one(j, p, kk, g, bx);
  }

  // Push the beam particles sorted into cell b (fields of slices b, b+1 are in the window)
  // and those this step listed for cell b, deposit them into the grid of step t+1; then
  // publish progress[t] = b + 1.  A particle whose cell (or an earlier step's target for it)
  // is past b is listed for that cell: its fields are not all solved yet, or an earlier step
  // may still have to push it there, and the progress chain makes that happen first.
  __device__ void push_cell(int b) {
    const Box bx = W::box(dxi, ximax, a.ffi, a.ffx);
    const int beg = a.bin_start[b], end = a.bin_start[b + 1];
    for (int j = beg + threadIdx.x; j < end; j += NT) {
      Part p;
      load_part(j, p);  // every load of the particle at once, before any branch on them
      if (p.fl & 1) continue;
      int kk;
      BT g;
      W::cell(p.xi, bx, nxi, kk, g);
      const int tgt = max(kk, p.tgt);
      if (tgt > b) {
        defer(b, j, p, tgt);
        continue;
      }
      if (kk != b) {  // behind its sorted cell: cannot happen (xi only grows)
        flag(a.d.status, ST_DRIFT);
        continue;
      }
      push_one(j, p, kk, g, bx);
    }
    __syncthreads();  // every entry counted so far is written
    // this step's listed particles for cell b: the next-cell entries made while cell b - 1 was
    // pushed (ctl[2] .. ctl[3]), and the others whose target is b
    const int2 *near = a.near_list + (size_t)t * a.near_cap;
    const int2 *far = a.defer_list + (size_t)t * a.defer_cap;
    for (int q = ctl[2] + threadIdx.x; q < ctl[3]; q += NT) push_listed(b, __ldcg(near + q % a.near_cap).x, bx);
    const int nf = min(__ldcg(a.defer_cnt + 2 * t + 1), a.defer_cap);
    for (int q = threadIdx.x; q < nf; q += NT) {
      const int2 e = __ldcg(far + q);
      if (e.y == b) push_listed(b, e.x, bx);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      st_release(&a.progress[t], b + 1);
      ctl[2] = ctl[3];  // the entries made while cell b was pushed are cell b + 1's
      ctl[3] = __ldcg(a.defer_cnt + 2 * t);
    }
  }
};

template <class Pol, int NT, int PPT>
__global__ void __launch_bounds__(NT, 1) step_kernel(PipeArgs a) {
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = a.d.nr + 1;
  const size_t base = (MarchSmem<Pol>::bytes(n1, NT * PPT) + 63) & ~(size_t)63;
  R *win;
  int *ctl;
  if constexpr (Pol::kWinGlobal) {  // the field window in this CTA's global buffer
    win = (R *)((unsigned char *)a.win_bufs + (size_t)blockIdx.x * a.win_stride);
    ctl = (int *)(smem_raw + base);
  } else {
    win = (R *)(smem_raw + base);
    ctl = (int *)(win + (size_t)12 * n1);
  }
  for (int t = blockIdx.x; t < a.nsteps; t += gridDim.x) {
    if (threadIdx.x == 0) {
      ctl[0] = 0;
      ctl[1] = 0;
      ctl[2] = 0;  // the next-cell list entries of the cell pushed last
      ctl[3] = 0;
    }
    __syncthreads();
    PipeHooks<Pol, NT> hk{a, t, win, ctl, n1, a.d.nr, a.d.nxi, a.d.dr, a.d.dxi, a.d.rmax, a.d.ximax};
    SimDesc d = a.d;
    if (!Pol::kSmemRings) d.ring_buf = (unsigned char *)a.ring_bufs + (size_t)blockIdx.x * a.ring_stride;
    march_body<Pol, NT, PPT>(d, smem_raw, hk);
    __syncthreads();
    if (ctl[0]) break;
  }
}

// The wide form: rings and the four-slice field window in per-CTA global buffers.
template <class Pol, int NT, int PPT>
__global__ void __launch_bounds__(NT, (NT < 512 ? 512 / NT : 1)) step_wide_kernel(PipeArgs a) {
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = a.d.nr + 1;
  const size_t base = (MarchSmem<Pol>::bytes(n1, NT * PPT) + 63) & ~(size_t)63;
  int *ctl = (int *)(smem_raw + base);
  R *win = (R *)((unsigned char *)a.win_bufs + (size_t)blockIdx.x * a.win_stride);
  for (int t = blockIdx.x; t < a.nsteps; t += gridDim.x) {
    if (threadIdx.x == 0) {
      ctl[0] = 0;
      ctl[1] = 0;
      ctl[2] = 0;  // the next-cell list entries of the cell pushed last
      ctl[3] = 0;
    }
    __syncthreads();
    PipeHooks<Pol, NT> hk{a, t, win, ctl, n1, a.d.nr, a.d.nxi, a.d.dr, a.d.dxi, a.d.rmax, a.d.ximax};
    SimDesc d = a.d;
    d.ring_buf = (unsigned char *)a.ring_bufs + (size_t)blockIdx.x * a.ring_stride;
    march_body_wide<Pol, NT, PPT>(d, smem_raw, hk);
    __syncthreads();
    if (ctl[0]) break;
  }
}

// Pipelined steps of many simulations in one persistent launch.  Work items are (simulation,
// step) pairs in the order the host gives (all steps of a simulation consecutive, largest
// simulations first); CTA c takes items c, c + gridDim.x, ...  An item's predecessor (the
// same simulation's previous step) comes earlier in the order, so with every CTA resident
// the earliest unfinished item can always run.  Every simulation is marched in the wide form.
struct BatchSim {
  PipeArgs p;  // the simulation's pipeline (its grids, progress, beam, lists); nsteps = steps
};
struct BatchArgs {
  const BatchSim *sims;
  const int2 *items;  // (simulation, step)
  int nitems;
  void *ring_bufs, *win_bufs;  // per CTA
  size_t ring_stride, win_stride;
};

template <class Pol, int NT, int PPT>
__global__ void __launch_bounds__(NT, (NT < 512 ? 512 / NT : 1)) batch_step_kernel(BatchArgs b) {
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int i = blockIdx.x; i < b.nitems; i += gridDim.x) {
    const int2 it = b.items[i];
    const PipeArgs &a = b.sims[it.x].p;
    const int n1 = a.d.nr + 1;
    const size_t base = (MarchSmem<Pol>::bytes(n1, NT * PPT) + 63) & ~(size_t)63;
    int *ctl = (int *)(smem_raw + base);
    R *win = (R *)((unsigned char *)b.win_bufs + (size_t)blockIdx.x * b.win_stride);
    if (threadIdx.x == 0) {
      ctl[0] = 0;
      ctl[1] = 0;
      ctl[2] = 0;  // the next-cell list entries of the cell pushed last
      ctl[3] = 0;
    }
    __syncthreads();
    PipeHooks<Pol, NT> hk{a, it.y, win, ctl, n1, a.d.nr, a.d.nxi, a.d.dr, a.d.dxi, a.d.rmax, a.d.ximax};
    SimDesc d = a.d;
    d.ring_buf = (unsigned char *)b.ring_bufs + (size_t)blockIdx.x * b.ring_stride;
    march_body_wide<Pol, NT, PPT>(d, smem_raw, hk);
    __syncthreads();
  }
}

template <class Pol, int NT, int PPT>
size_t step_smem_bytes(int n1) {
  return ((MarchSmem<Pol>::bytes(n1, NT * PPT) + 63) & ~(size_t)63) +
         (Pol::kWinGlobal ? 0 : sizeof(typename Pol::R) * 12 * (size_t)n1) + 64;
}
// Global field-window bytes per CTA of the pipelined step (kWinGlobal forms).
inline size_t step_window_bytes(int n1) { return ((sizeof(float) * 12 * (size_t)n1 + 255) / 256) * 256; }

}  // namespace wake
