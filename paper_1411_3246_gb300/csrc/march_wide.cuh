// The xi-march for boxes whose rings do not fit one CTA's shared memory (up to 2048 radial
// cells and 65,536 rings per slice, the mixed arithmetic of PolWide): the node arrays and
// the radial solves stay in shared memory as in march_body, the ring slots live in a global
// buffer and every ring pass runs over them in chunks of NT x PPT slots (the same per-ring
// code, offset by the chunk).  Every two slices the rings are re-sorted by cell through a
// second buffer; the stage-2 Gamma and force, which march_body keeps in registers between its
// passes, get slot arrays of their own.
#pragma once

#include "march.cuh"

namespace wake {

// Ring slots of the wide march: RingSoA (np_pad slots) followed by the stage-2 G2, F2, and a
// second copy of the ring state (c, f, u_r and the constants) that the re-sort scatters into.
template <class R>
struct WideRings {
  RingSoA<R> s, alt;
  R *G2, *F2;
  __host__ __device__ static size_t bytes(int slots) { return 2 * RingSoA<R>::bytes(slots) + 2 * sizeof(R) * (size_t)slots + 128; }
  __device__ __forceinline__ void carve(void *base, int slots) {
    s.carve(base, slots);
    G2 = (R *)(((uintptr_t)(s.F1 + slots) + 31) & ~(uintptr_t)31);
    F2 = G2 + slots;
    alt.carve((void *)(((uintptr_t)(F2 + slots) + 31) & ~(uintptr_t)31), slots);
  }
};

// A ring's rank in its cell, kept for the scatter in a spare slot array of the ring type:
// stored and read back as raw bits (no arithmetic, so nothing is flushed or rounded).
__device__ __forceinline__ void rank_store(float *p, int v) { *p = __int_as_float(v); }
__device__ __forceinline__ int rank_load(const float *p) { return __float_as_int(*p); }
__device__ __forceinline__ void rank_store(double *p, int v) { *p = __longlong_as_double((long long)v); }
__device__ __forceinline__ int rank_load(const double *p) { return (int)__double_as_longlong(*p); }

// Re-sort the rings of a wide march by cell (counting sort through the second buffer, then
// the buffers swap): rank r goes to chunk r / SLOTS, thread (r % SLOTS) / PPT, ring
// (r % SLOTS) % PPT, so each thread's rings are consecutive in radius again.  Ends with a
// barrier.
template <class Pol, int NT, int PPT>
__device__ __forceinline__ void resort_rings_wide(MarchSmem<Pol> &sm, WideRings<typename Pol::R> &wr, int np, int nr,
                                                  int nch) {
  constexpr int SLOTS = NT * PPT;
  const int t = threadIdx.x, n1 = nr + 1;
  for (int m = t; m < n1; m += NT) sm.cnt[m] = 0;
  __syncthreads();
  for (int ch = 0; ch < nch; ++ch) {
    const int base = ch * SLOTS, npc = np - base < SLOTS ? np - base : SLOTS;
#pragma unroll
    for (int p = 0; p < PPT; ++p)
      if (t * PPT + p < npc) {
        const int sl = base + p * NT + t;
        rank_store(&wr.alt.G1[sl], atomicAdd(&sm.cnt[wr.s.c[sl]], 1));  // rank in its cell
      }
  }
  __syncthreads();
  if (t < 32) {  // exclusive scan of the counts
    const int E = (n1 + 31) / 32, beg = min(n1, t * E), end = min(n1, beg + E);
    int s = 0;
    for (int q = beg; q < end; ++q) s += sm.cnt[q];
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(kFull, incl, o);
      if (t >= o) incl += u;
    }
    int run = incl - s;
    for (int q = beg; q < end; ++q) {
      const int v = sm.cnt[q];
      sm.cnt[q] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int ch = 0; ch < nch; ++ch) {
    const int base = ch * SLOTS, npc = np - base < SLOTS ? np - base : SLOTS;
#pragma unroll
    for (int p = 0; p < PPT; ++p)
      if (t * PPT + p < npc) {
        const int sl = base + p * NT + t;
        const int c = wr.s.c[sl];
        const int r = sm.cnt[c] + rank_load(&wr.alt.G1[sl]);
        const int rr = r % SLOTS;
        const int dl = (r - rr) + (rr % PPT) * NT + rr / PPT;
        wr.alt.c[dl] = c;
        wr.alt.f[dl] = wr.s.f[sl];
        wr.alt.ur[dl] = wr.s.ur[sl];
        wr.alt.lz[dl] = wr.s.lz[sl];
        wr.alt.G0[dl] = wr.s.G0[sl];
        wr.alt.w[dl] = wr.s.w[sl];
      }
  }
  __syncthreads();
  const RingSoA<typename Pol::R> tmp = wr.s;
  wr.s = wr.alt;
  wr.alt = tmp;
}

template <class R>
__device__ __forceinline__ RingSoA<R> shifted(const RingSoA<R> &r, int off) {
  RingSoA<R> o;
  o.c = r.c + off;
  o.f = r.f + off;
  o.ur = r.ur + off;
  o.lz = r.lz + off;
  o.G0 = r.G0 + off;
  o.w = r.w + off;
  o.G1 = r.G1 + off;
  o.F1 = r.F1 + off;
  return o;
}

// Slots a simulation of np rings needs in the wide march (whole chunks).
template <int NT, int PPT>
__host__ __device__ inline int wide_slots(int np) {
  return (np + NT * PPT - 1) / (NT * PPT) * (NT * PPT);
}

template <class Pol, int NT, int PPT, class Hooks>
__device__ __forceinline__ void march_body_wide(const SimDesc &d, unsigned char *smem_raw, Hooks &hk) {
  using R = typename Pol::R;
  using Acc = typename Pol::Acc;
  constexpr int SLOTS = NT * PPT, PRE = Pol::kScanE;
  const int tid = threadIdx.x, nr = d.nr, n1 = nr + 1, np = d.np, nxi = d.nxi;
  const int nch = (np + SLOTS - 1) / SLOTS;
  MarchSmem<Pol> sm;
  sm.carve(smem_raw, n1, SLOTS);
  WideRings<R> wr;
  wr.carve(d.ring_buf, nch * SLOTS);
  const RingSoA<R> &rs = wr.s;  // follows the swaps of the re-sort
  const double drd = d.dr;
  const R h = (R)d.dxi, R_wall = (R)d.rmax, dR = (R)drd, inv_dr = (R)(1.0 / drd);
  const NodeGeo<Pol> geo{sm.invR, sm.invV, sm.alpha, sm.ga, sm.gb, sm.gc, nr, dR, inv_dr, (R)(1.0 / (drd * drd)),
                          (R)(drd / 6.0), (R)(1.0 / (0.5 * nr - 1.0 / 6.0))};
  fill_tables<Pol, NT>(sm, nr, drd);  // the wide form is cylindrical only
  for (int m = tid; m < n1; m += NT) {
    sm.rho[m] = (typename Pol::Q)0;
    sm.jz[m] = sm.chi[m] = sm.T[m] = sm.P[m] = sm.U[m] = sm.K[m] = (Acc)0;
  }
  // chunk ch holds rings ch*SLOTS + t*PPT + p at slot ch*SLOTS + p*NT + t
  for (int ch = 0; ch < nch; ++ch) {
    const int base = ch * SLOTS;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int j = base + tid * PPT + p, sl = base + p * NT + tid;
      if (j < np) {
        const double s = d.r0[j] / drd;
        int c = (int)floor(s);
        c = c < 0 ? 0 : (c > nr - 1 ? nr - 1 : c);
        rs.c[sl] = c;
        rs.f[sl] = (R)(s - (double)c);
        rs.ur[sl] = (R)d.ur0[j];
        rs.lz[sl] = (R)d.lz[j];
        rs.G0[sl] = (R)d.G0[j];
        rs.w[sl] = (R)d.w[j];
      }
    }
  }
  __syncthreads();

  int base = 0;  // slot offset of the chunk the position functors below read
  auto state_pos = [&](int sl, int &c, R &f, R &u_r, R &u_t) {
    sl += base;
    c = rs.c[sl];
    f = rs.f[sl];
    u_r = rs.ur[sl];
    const R r = ((R)c + f) * dR;
    u_t = r > (R)0 ? rs.lz[sl] / r : (R)0;
  };
  auto midpoint_abs = [&](int sl, int &c, R &f, R &u_r, R &u_t) -> R {
    const int c0 = rs.c[sl];
    const R f0 = rs.f[sl], ur0 = rs.ur[sl];
    const R r = ((R)c0 + f0) * dR;
    const R ut = r > (R)0 ? rs.lz[sl] / r : (R)0;
    const R iG = (R)1 / rs.G1[sl];
    const R dx = (R)0.5 * h * ur0 * iG, dy = (R)0.5 * h * ut * iG;
    const R uxh = ur0 + (R)0.5 * h * rs.F1[sl];
    R rr;
    move_ring<R>(c0, f0, r, dx, dy, uxh, ut, inv_dr, dR, nr, c, f, rr, u_r, u_t);
    return rr;
  };
  auto chunk_np = [&](int ch) { return np - ch * SLOTS < SLOTS ? np - ch * SLOTS : SLOTS; };

  // charge of the initial slice = the ion background
  for (int ch = 0; ch < nch; ++ch) {
    const int b0 = ch * SLOTS, npc = chunk_np(ch);
    ChargeWin<Pol> acc;
    acc.init(-8);
#pragma unroll
    for (int p = 0; p < PPT; ++p)
      if (tid * PPT + p < npc) {
        const int sl = b0 + p * NT + tid;
        add_charge<Pol>(sm, acc, p, rs.c[sl], rs.f[sl], rs.w[sl]);
      }
    flush_charge<Pol>(sm, acc, nr);
  }
  __syncthreads();
  for (int m = tid; m < n1; m += NT) sm.rho0[m] = sm.rho[m];
  __syncthreads();

  for (int k = 0; k <= nxi; ++k) {
    if (Pol::kSortEvery > 0 && k > 0 && k % Pol::kSortEvery == 0) resort_rings_wide<Pol, NT, PPT>(sm, wr, np, nr, nch);
    const R *nbk = (k & 1) ? sm.nb1 : sm.nb0, *nbk1 = (k & 1) ? sm.nb0 : sm.nb1;
    if (!hk.wait_rows(k)) break;
    if (k == 0)
      for (int m = tid; m < n1; m += NT) sm.nb0[m] = hk.nb_row(0, m);
    R pre[PRE];
#pragma unroll
    for (int q = 0; q < PRE; ++q) pre[q] = (R)0;
    if (k < nxi) {
#pragma unroll
      for (int q = 0; q < PRE; ++q)
        if (tid + q * NT < n1) pre[q] = hk.nb_row(k + 1, tid + q * NT);
    }
    // ======== stage 1 at xi_k ========
    solve_psi<Pol, NT>(sm, geo, sm.wtot);
    __syncthreads();
    if (k < nxi) {
      R *dst = (k & 1) ? sm.nb0 : sm.nb1;
#pragma unroll
      for (int q = 0; q < PRE; ++q)
        if (tid + q * NT < n1) dst[tid + q * NT] = pre[q];
    }
    for (int i = tid; i < n1; i += NT) sm.rho[i] = (typename Pol::Q)0;
    for (int ch = 0; ch < nch; ++ch) {
      base = ch * SLOTS;
      const int npc = chunk_np(ch);
      R Gs[PPT], gqs[PPT];
      const RingSoA<R> rsc = shifted(rs, base);
      pass_currents<Pol, NT, PPT>(sm, rsc, npc, nr, dR, d.status, state_pos, [&](unsigned miss) {
        warp_misses<NT, PPT>(miss, [&](int sl) { current_miss<Pol>(sm, rsc, sl, dR, d.status, state_pos); });
      }, Gs, gqs);
#pragma unroll
      for (int p = 0; p < PPT; ++p)
        if (tid * PPT + p < npc) {
          rs.G1[base + p * NT + tid] = Gs[p];
          rs.F1[base + p * NT + tid] = gqs[p];
        }
    }
    __syncthreads();
    solve_fields<Pol, NT>(sm, geo, nbk, nbk, sm.wtot);
    __syncthreads();
    hk.slice_done(k, sm);
    if (k == nxi) break;
    for (int i = tid; i < n1; i += NT) sm.jz[i] = sm.chi[i] = sm.T[i] = sm.P[i] = sm.U[i] = sm.K[i] = (Acc)0;
    for (int ch = 0; ch < nch; ++ch) {
      const int b0 = ch * SLOTS, npc = chunk_np(ch);
      ChargeWin<Pol> acc;
      acc.init(-8);
      unsigned miss = 0u;
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        if (tid * PPT + p < npc) {
          const int sl = b0 + p * NT + tid;
          rs.F1[sl] = rs.F1[sl] - interp(sm.bth, rs.c[sl], rs.f[sl]);
          int c;
          R f, u_r, u_t;
          const R rr = midpoint_abs(sl, c, f, u_r, u_t);
          if (!(rr >= (R)0 && rr <= R_wall)) flag(d.status, ST_ESCAPE);
          add_charge_mark<Pol>(sm, acc, p, c, f, rs.w[sl], miss);
        }
      }
      warp_misses<NT, PPT>(miss, [&](int sl) {
        int c;
        R f, u_r, u_t;
        midpoint_abs(b0 + sl, c, f, u_r, u_t);
        ChargeWin<Pol>::direct(sm.rho, c, f, rs.w[b0 + sl]);
      });
      flush_charge<Pol>(sm, acc, nr);
    }
    __syncthreads();
    // ======== stage 2 at xi_k + dxi/2 ========
    solve_psi<Pol, NT>(sm, geo, sm.wtot);
    __syncthreads();
    for (int i = tid; i < n1; i += NT) sm.rho[i] = (typename Pol::Q)0;
    for (int ch = 0; ch < nch; ++ch) {
      base = ch * SLOTS;
      const int npc = chunk_np(ch);
      R Gs[PPT], gqs[PPT];
      auto mid_chunk = [&](int sl, int &c, R &f, R &u_r, R &u_t) { midpoint_abs(sl + base, c, f, u_r, u_t); };
      const RingSoA<R> rsc = shifted(rs, base);
      pass_currents<Pol, NT, PPT>(sm, rsc, npc, nr, dR, d.status, mid_chunk, [&](unsigned miss) {
        warp_misses<NT, PPT>(miss, [&](int sl) { current_miss<Pol>(sm, rsc, sl, dR, d.status, mid_chunk); });
      }, Gs, gqs);
#pragma unroll
      for (int p = 0; p < PPT; ++p)
        if (tid * PPT + p < npc) {
          wr.G2[base + p * NT + tid] = Gs[p];
          wr.F2[base + p * NT + tid] = gqs[p];
        }
    }
    __syncthreads();
    solve_fields<Pol, NT>(sm, geo, nbk, nbk1, sm.wtot);
    __syncthreads();
    // full step from the slice-k state with the midpoint derivative; charge of the new slice
    for (int i = tid; i < n1; i += NT) sm.jz[i] = sm.chi[i] = sm.T[i] = sm.P[i] = sm.U[i] = sm.K[i] = (Acc)0;
    for (int ch = 0; ch < nch; ++ch) {
      const int b0 = ch * SLOTS, npc = chunk_np(ch);
      ChargeWin<Pol> acc;
      acc.init(-8);
      unsigned miss = 0u;
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        if (tid * PPT + p < npc) {
          const int sl = b0 + p * NT + tid;
          int mc;
          R mf, mu_r, mu_t;
          midpoint_abs(sl, mc, mf, mu_r, mu_t);
          const R F2b = wr.F2[sl] - interp(sm.bth, mc, mf);
          const int c0 = rs.c[sl];
          const R f0 = rs.f[sl], ur0 = rs.ur[sl], G1v = rs.G1[sl], F1v = rs.F1[sl];
          const R r = ((R)c0 + f0) * dR;
          const R ut = r > (R)0 ? rs.lz[sl] / r : (R)0;
          const R iG1 = (R)1 / G1v;
          const R xh = r + (R)0.5 * h * ur0 * iG1;
          const R yh = (R)0.5 * h * ut * iG1;
          const R uxh = ur0 + (R)0.5 * h * F1v;
          const R rh = sqrt(xh * xh + yh * yh);
          R ex = (R)1, ey = (R)0;
          if (rh > (R)0) {
            const R irh = (R)1 / rh;
            ex = xh * irh;
            ey = yh * irh;
          }
          const R iG2 = (R)1 / wr.G2[sl];
          const R dx = h * uxh * iG2, dy = h * ut * iG2;
          const R uxn = ur0 + h * F2b * ex, uyn = ut + h * F2b * ey;
          int cn;
          R fn, rn, urn, utn;
          move_ring<R>(c0, f0, r, dx, dy, uxn, uyn, inv_dr, dR, nr, cn, fn, rn, urn, utn);
          if (!(rn >= (R)0 && rn <= R_wall) || !isfinite(urn)) flag(d.status, ST_ESCAPE);
          rs.c[sl] = cn;
          rs.f[sl] = fn;
          rs.ur[sl] = urn;
          add_charge_mark<Pol>(sm, acc, p, cn, fn, rs.w[sl], miss);
        }
      }
      warp_misses<NT, PPT>(miss, [&](int sl) {  // the new positions are in the slots
        ChargeWin<Pol>::direct(sm.rho, rs.c[b0 + sl], rs.f[b0 + sl], rs.w[b0 + sl]);
      });
      flush_charge<Pol>(sm, acc, nr);
    }
    __syncthreads();
  }
  hk.finish(sm);
}

template <class Pol, int NT, int PPT>
__global__ void __launch_bounds__(NT, 1) march_wide_kernel(const SimDesc *descs, const int *order) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SimDesc &d = descs[order ? order[blockIdx.x] : blockIdx.x];
  PlainHooks<Pol, NT> hk{(const typename Pol::G *)d.nb, (typename Pol::G *)d.psi, (typename Pol::G *)d.ez,
                         (typename Pol::G *)d.er, (typename Pol::G *)d.bth, d.nr + 1, d.status};
  march_body_wide<Pol, NT, PPT>(d, smem_raw, hk);
}

}  // namespace wake
