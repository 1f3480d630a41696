// The quasi-static xi-march (Sec. II.A, Eqs. 1-7): one CTA marches one simulation through
// all of its slices, persistent over xi.  The plasma rings live in registers, the node
// arrays of the current slice in shared memory; nothing but the beam density row (in) and
// the field rows (out) touches global memory inside the loop.
//
// Per slice, RK2 (midpoint) in xi; each stage solves the fields for the rings' current
// positions:
//   1. deposit the ring charge (linear hats);
//   2. psi from Gauss's law for the hat density (enclosed charge Phi_m at node m,
//      r_m psi'_m = Phi_m), psi(R) = 0, inward trapezoid sum  -- two block scans;
//   3. per ring: Gamma = Gamma_0 + psi (Eq. 1), gamma and u_z (Eqs. 2-3), a = u_r/Gamma,
//      F0 = (gamma/Gamma) psi' + u_theta^2/(Gamma r) (Eq. 4 without -B); deposit
//      J_z, chi = n/gamma, T = D[w a^2], P = D[w (a^2 psi' - F0)/Gamma], U = D[w a/Gamma]
//      on the nodes and the radial current K_c of each cell;
//   4. E_z = d_xi psi (Eq. 7) by an inward scan of the cell currents; Q = P + E_z U; B_theta
//      from Eq. 6 differentiated in r (Helmholtz form, shift chi) by parallel cyclic
//      reduction; E_r = B_theta - psi';
//   5. per ring: the Cartesian radial force (gamma/Gamma) psi' - B_theta (Eqs. 4-5 with the
//      centrifugal term carried by the local frame).
// Stage 1 at xi_k writes the slice's fields; stage 2 at xi_k + dxi/2 uses n_b averaged over
// slices k and k+1.
#pragma once

#include "wake_common.cuh"

namespace wake {

// Precision policies.  R: ring and node arithmetic (gathers, per-node sources, fields);
// Acc: shared-memory deposit sums; S: tridiagonal (PCR) arithmetic; G: grid element type in
// global memory.  The enclosed-charge and inward field sums are always scanned in FP64.
struct PolFP64 {
  using R = double;
  using Acc = double;
  using S = double;
  using G = double;
  static constexpr int NT = 512;
};
struct PolMixed {
  using R = float;
  using Acc = float;
  using S = float;
  using G = float;
  static constexpr int NT = 1024;
};

template <class Pol>
struct MarchSmem {
  using R = typename Pol::R;
  using Acc = typename Pol::Acc;
  using S = typename Pol::S;
  double *work, *wtot;                       // scan buffer
  Acc *rho0, *rho, *jz, *chi, *T, *P, *U, *K;  // deposits
  R *psi, *dpsi, *ez, *bth;                  // node fields
  R *invR, *invV, *alpha, *ga, *gb, *gc;     // per-simulation tables
  S *ta[2], *tb[2], *tc[2], *td[2];          // PCR buffers

  static size_t bytes(int n1) {
    return sizeof(double) * ((size_t)n1 + 64) + sizeof(Acc) * 8 * (size_t)n1 + sizeof(R) * 10 * (size_t)n1 +
           sizeof(S) * 8 * (size_t)n1 + 256;
  }
  __device__ void carve(unsigned char *base, int n1) {
    double *dp = (double *)base;
    work = dp; dp += n1;
    wtot = dp; dp += 64;
    Acc *ap = (Acc *)dp;
    rho0 = ap; ap += n1;
    rho = ap; ap += n1;
    jz = ap; ap += n1;
    chi = ap; ap += n1;
    T = ap; ap += n1;
    P = ap; ap += n1;
    U = ap; ap += n1;
    K = ap; ap += n1;
    R *rp = (R *)ap;
    psi = rp; rp += n1;
    dpsi = rp; rp += n1;
    ez = rp; rp += n1;
    bth = rp; rp += n1;
    invR = rp; rp += n1;
    invV = rp; rp += n1;
    alpha = rp; rp += n1;
    ga = rp; rp += n1;
    gb = rp; rp += n1;
    gc = rp; rp += n1;
    S *sp = (S *)rp;
    for (int b = 0; b < 2; ++b) {
      ta[b] = sp; sp += n1;
      tb[b] = sp; sp += n1;
      tc[b] = sp; sp += n1;
      td[b] = sp; sp += n1;
    }
  }
};

// One field solve for the rings at radius (pc + pf) dr (cell index pc, offset pf in [0,1])
// with momenta (pur, put).  nbA/nbB: the beam-density rows to average (the same row for
// stage 1).  On return Gam[p] = Gamma of ring p and Fc[p] = (gamma/Gamma) psi'(r_p) -
// B_theta(r_p); the node arrays psi, dpsi, ez, bth hold the fields.
template <class Pol, int NT, int PPT>
__device__ __forceinline__ void solve_stage(MarchSmem<Pol> &sm, const SimDesc &d, int j0,
                                            const int (&pc)[PPT], const typename Pol::R (&pf)[PPT],
                                            const typename Pol::R (&pur)[PPT],
                                            const typename Pol::R (&put)[PPT],
                                            const typename Pol::R (&cG0)[PPT],
                                            const typename Pol::R (&cw)[PPT],
                                            const typename Pol::G *nbA, const typename Pol::G *nbB,
                                            typename Pol::R (&Gam)[PPT], typename Pol::R (&Fc)[PPT]) {
  using R = typename Pol::R;
  using Acc = typename Pol::Acc;
  using S = typename Pol::S;
  const int tid = threadIdx.x, nr = d.nr, n1 = nr + 1, np = d.np;
  const R inv_dr = (R)(1.0 / d.dr);
  const R dr = (R)d.dr;
  const R hdr = (R)(0.5 * d.dr);

  // 1. charge deposit
  for (int i = tid; i < n1; i += NT) {
    sm.rho[i] = (Acc)0;
    sm.jz[i] = (Acc)0;
    sm.chi[i] = (Acc)0;
    sm.T[i] = (Acc)0;
    sm.P[i] = (Acc)0;
    sm.U[i] = (Acc)0;
    sm.K[i] = (Acc)0;
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    if (j0 + p < np) {
      const int c = pc[p];
      const R f = pf[p];
      atomicAdd(&sm.rho[c], (Acc)(cw[p] * ((R)1 - f)));
      atomicAdd(&sm.rho[c + 1], (Acc)(cw[p] * f));
    }
  }
  __syncthreads();

  // 2. psi: enclosed charge Phi_m = sum_{i<m} delta_i + alpha_m delta_m, psi' = Phi/r,
  //    inward trapezoid sum from psi(R) = 0
  for (int m = tid; m < n1; m += NT) sm.work[m] = (double)(sm.rho[m] - sm.rho0[m]);
  __syncthreads();
  block_scan<NT>(sm.work, n1, sm.wtot, false);
  for (int m = tid; m < n1; m += NT) {
    R dp = (R)0;
    if (m > 0) {
      const R v = (R)(sm.rho[m] - sm.rho0[m]);
      dp = ((R)sm.work[m] - ((R)1 - sm.alpha[m]) * v) * sm.invR[m];
    }
    sm.dpsi[m] = dp;
  }
  __syncthreads();
  for (int m = tid; m < n1; m += NT) sm.work[m] = m < nr ? (double)(hdr * (sm.dpsi[m] + sm.dpsi[m + 1])) : 0.0;
  __syncthreads();
  block_scan<NT>(sm.work, n1, sm.wtot, true);
  for (int m = tid; m < n1; m += NT) sm.psi[m] = (R)(-sm.work[m]);
  __syncthreads();

  // 3. ring quantities (Eqs. 1-4) and the current-type deposits
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    if (j0 + p < np) {
      const int c = pc[p];
      const R f = pf[p];
      const R rp = ((R)c + f) * dr;
      const R G = cG0[p] + interp(sm.psi, c, f);
      if (!(G > (R)0)) flag(d.status, ST_NUMERIC);
      const R iG = (R)1 / G;
      const R up2 = pur[p] * pur[p] + put[p] * put[p];
      const R gam = ((R)1 + up2 + G * G) * (R)0.5 * iG;
      const R uz = gam - G;
      const R a = pur[p] * iG;
      const R dp = interp(sm.dpsi, c, f);
      const R cent = rp > (R)0 ? put[p] * put[p] * iG / rp : (R)0;
      const R gq = gam * iG * dp;
      const R F0 = gq + cent;
      const R w = cw[p];
      const R vjz = -w * uz * iG, vchi = w * iG, vT = w * a * a, vP = w * (a * a * dp - F0) * iG, vU = w * a * iG;
      const R g0 = (R)1 - f;
      atomicAdd(&sm.jz[c], (Acc)(vjz * g0));
      atomicAdd(&sm.jz[c + 1], (Acc)(vjz * f));
      atomicAdd(&sm.chi[c], (Acc)(vchi * g0));
      atomicAdd(&sm.chi[c + 1], (Acc)(vchi * f));
      atomicAdd(&sm.T[c], (Acc)(vT * g0));
      atomicAdd(&sm.T[c + 1], (Acc)(vT * f));
      atomicAdd(&sm.P[c], (Acc)(vP * g0));
      atomicAdd(&sm.P[c + 1], (Acc)(vP * f));
      atomicAdd(&sm.U[c], (Acc)(vU * g0));
      atomicAdd(&sm.U[c + 1], (Acc)(vU * f));
      atomicAdd(&sm.K[c], (Acc)(w * a));
      Gam[p] = G;
      Fc[p] = gq;
    }
  }
  __syncthreads();

  // 4a. node densities (divide by the ring volumes); d_xi psi' at the nodes from the cell
  //     currents, then E_z = d_xi psi by the inward trapezoid sum from E_z(R) = 0
  for (int m = tid; m < n1; m += NT) {
    const R iv = sm.invV[m];
    const R nbm = (R)0.5 * ((R)nbA[m] + (R)nbB[m]);
    sm.jz[m] = (Acc)((R)sm.jz[m] * iv - nbm);
    sm.chi[m] = (Acc)((R)sm.chi[m] * iv);
    sm.T[m] = (Acc)((R)sm.T[m] * iv);
    sm.P[m] = (Acc)((R)sm.P[m] * iv);
    sm.U[m] = (Acc)((R)sm.U[m] * iv);
    R dz = (R)0;
    if (m > 0) {
      const R al = sm.alpha[m];
      const R Km = m < nr ? (R)sm.K[m] : (R)0;
      dz = -(((R)1 - al) * (R)sm.K[m - 1] + al * Km) * sm.invR[m] * inv_dr;
    }
    sm.ez[m] = dz;
  }
  __syncthreads();
  for (int m = tid; m < n1; m += NT) sm.work[m] = m < nr ? (double)(hdr * (sm.ez[m] + sm.ez[m + 1])) : 0.0;
  __syncthreads();
  block_scan<NT>(sm.work, n1, sm.wtot, true);
  for (int m = tid; m < n1; m += NT) sm.ez[m] = (R)(-sm.work[m]);
  __syncthreads();
  // 4b. the Helmholtz system for B_theta at nodes 1..nr (row q = i - 1)
  const R i2dr = (R)0.5 * inv_dr;
  for (int q = tid; q < nr; q += NT) {
    const int i = q + 1;
    const R Qi = (R)sm.P[i] + sm.ez[i] * (R)sm.U[i];
    const R Ti = (R)sm.T[i];
    R rhs;
    if (i < nr)
      rhs = ((R)sm.jz[i + 1] - (R)sm.jz[i - 1]) * i2dr + Qi + ((R)sm.T[i + 1] - (R)sm.T[i - 1]) * i2dr +
            Ti * sm.invR[i];
    else
      rhs = Qi + (Ti - (R)sm.T[i - 1]) * inv_dr + Ti * sm.invR[i] - ((R)sm.jz[i - 1] + (R)sm.jz[i]) * inv_dr;
    sm.ta[0][q] = (S)sm.ga[q];
    sm.tb[0][q] = (S)(sm.gb[q] - (R)sm.chi[i]);
    sm.tc[0][q] = (S)sm.gc[q];
    sm.td[0][q] = (S)rhs;
  }
  __syncthreads();
  const int cur = pcr_solve<NT, S>(sm.ta[0], sm.tb[0], sm.tc[0], sm.td[0], sm.ta[1], sm.tb[1], sm.tc[1],
                                   sm.td[1], nr);
  for (int m = tid; m < n1; m += NT) sm.bth[m] = m > 0 ? (R)(sm.td[cur][m - 1] / sm.tb[cur][m - 1]) : (R)0;
  __syncthreads();

  // 5. Cartesian radial force on each ring
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    if (j0 + p < np) {
      Fc[p] = Fc[p] - interp(sm.bth, pc[p], pf[p]);
    }
  }
}

// Move a ring at radius r = (c + f) dr by the Cartesian displacement (dx, dy) from (r, 0)
// and give it the Cartesian momentum (ux, uy).  The new radius is formed as the exact
// increment r' - r = (dx (2r + dx) + dy^2) / (r' + r), applied to the cell offset, so no
// precision is lost to the size of r.  Returns the new cell (cn, fn), the radius rn, and the
// radial / azimuthal momenta; a ring beyond the wall r = nr dr is reflected specularly.
template <class R>
__device__ __forceinline__ void move_ring(int c, R f, R r, R dx, R dy, R ux, R uy, R inv_dr, int nr, int &cn,
                                          R &fn, R &rn, R &urn, R &utn) {
  const R xn = r + dx, yn = dy;
  R rr = sqrt(xn * xn + yn * yn);
  const R den = rr + r;
  const R delta = den > (R)0 ? (dx * ((R)2 * r + dx) + dy * dy) / den : (R)0;
  R s = f + delta * inv_dr;  // offset from node c, in cells
  if (rr > (R)0) {
    urn = (xn * ux + yn * uy) / rr;
    utn = (xn * uy - yn * ux) / rr;
  } else {
    urn = sqrt(ux * ux + uy * uy);
    utn = (R)0;
  }
  R tot = (R)c + s;  // r'/dr
  if (tot > (R)nr) {  // specular reflection at the wall
    s = (R)(2 * (nr - c)) - s;  // r'/dr = 2 nr - (c + s), kept relative to c
    urn = -urn;
    tot = (R)c + s;
  }
  const R fl = floor(s);
  int ci = c + (int)fl;
  R fo = s - fl;
  if (ci > nr - 1) {
    fo += (R)(ci - (nr - 1));
    ci = nr - 1;
  }
  if (ci < 0) {
    fo += (R)ci;
    ci = 0;
  }
  cn = ci;
  fn = fo;
  rn = tot / inv_dr;
}

template <class Pol, int NT, int PPT>
__global__ void __launch_bounds__(NT, 1) march_kernel(const SimDesc *descs, const int *order) {
  using R = typename Pol::R;
  using G = typename Pol::G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SimDesc d = descs[order ? order[blockIdx.x] : blockIdx.x];
  const int tid = threadIdx.x, nr = d.nr, n1 = nr + 1, np = d.np, nxi = d.nxi;
  MarchSmem<Pol> sm;
  sm.carve(smem_raw, n1);
  const double dr = d.dr;
  const R h = (R)d.dxi, R_wall = (R)d.rmax;

  // per-simulation node tables: 1/r_m, 1/V_m, alpha_m, and the geometric part of the
  // B_theta rows (central differences; a half cell at the wall)
  for (int m = tid; m < n1; m += NT) {
    sm.invR[m] = (R)(m > 0 ? 1.0 / ((double)m * dr) : 0.0);
    sm.invV[m] = (R)(1.0 / node_volume(m, nr, dr));
    sm.alpha[m] = (R)(m > 0 ? node_alpha(m, nr) : 0.0);
    if (m < nr) {
      const int i = m + 1;
      const double idr2 = 1.0 / (dr * dr), rm = i - 0.5, rp = i + 0.5;
      double a, b, c;
      if (i < nr) {
        a = (i - 1) / rm * idr2;
        c = (i + 1) / rp * idr2;
        b = -(double)i * (1.0 / rp + 1.0 / rm) * idr2;
      } else {
        a = 2.0 * (i - 1) / rm * idr2;
        c = 0.0;
        b = -2.0 * (double)i / rm * idr2;
      }
      sm.ga[m] = (R)(m == 0 ? 0.0 : a);
      sm.gb[m] = (R)b;
      sm.gc[m] = (R)c;
    }
  }
  // rings: contiguous chunk of PPT per thread.  A ring's radius is kept as a cell index c
  // and an offset f in [0,1] (r = (c + f) dr), so its position resolution is uniform over
  // the box in either precision; moves are applied as exact radial displacements.
  const int j0 = tid * PPT;
  const R dR = (R)dr, inv_dr = (R)(1.0 / dr);
  int rc[PPT];
  R rf[PPT], ur[PPT], lz[PPT], cG0[PPT], cw[PPT];
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const int j = j0 + p;
    if (j < np) {
      const double s = d.r0[j] / dr;
      int c = (int)floor(s);
      c = c < 0 ? 0 : (c > nr - 1 ? nr - 1 : c);
      rc[p] = c;
      rf[p] = (R)(s - (double)c);
      ur[p] = (R)d.ur0[j];
      lz[p] = (R)d.lz[j];
      cG0[p] = (R)d.G0[j];
      cw[p] = (R)d.w[j];
    } else {
      rc[p] = 0;
      rf[p] = ur[p] = lz[p] = cw[p] = (R)0;
      cG0[p] = (R)1;
    }
  }
  __syncthreads();
  // ion background: the deposit of the unperturbed electrons (same arithmetic as a stage)
  {
    for (int i = tid; i < n1; i += NT) sm.rho[i] = 0;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      if (j0 + p < np) {
        atomicAdd(&sm.rho[rc[p]], (typename Pol::Acc)(cw[p] * ((R)1 - rf[p])));
        atomicAdd(&sm.rho[rc[p] + 1], (typename Pol::Acc)(cw[p] * rf[p]));
      }
    }
    __syncthreads();
    for (int i = tid; i < n1; i += NT) sm.rho0[i] = sm.rho[i];
    __syncthreads();
  }

  const G *nb = (const G *)d.nb;
  G *opsi = (G *)d.psi, *oez = (G *)d.ez, *oer = (G *)d.er, *obth = (G *)d.bth;
  int pc[PPT];
  R pf[PPT], pur[PPT], put[PPT], G1[PPT], F1[PPT], G2[PPT], F2[PPT];

  for (int k = 0; k <= nxi; ++k) {
    const G *nbk = nb + (size_t)k * n1;
    // stage 1 at xi_k
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const R r = ((R)rc[p] + rf[p]) * dR;
      pc[p] = rc[p];
      pf[p] = rf[p];
      pur[p] = ur[p];
      put[p] = r > (R)0 ? lz[p] / r : (R)0;
    }
    solve_stage<Pol, NT, PPT>(sm, d, j0, pc, pf, pur, put, cG0, cw, nbk, nbk, G1, F1);
    // fields of slice k
    {
      G *o1 = opsi + (size_t)k * n1, *o2 = oez + (size_t)k * n1, *o3 = oer + (size_t)k * n1,
        *o4 = obth + (size_t)k * n1;
      for (int m = tid; m < n1; m += NT) {
        const R ps = sm.psi[m], e = sm.ez[m], b = sm.bth[m];
        if (!(isfinite(ps) && isfinite(e) && isfinite(b))) flag(d.status, ST_NUMERIC);
        o1[m] = (G)ps;
        o2[m] = (G)e;
        o3[m] = m > 0 ? (G)(b - sm.dpsi[m]) : (G)0;
        o4[m] = (G)b;
      }
    }
    if (k == nxi) break;
    __syncthreads();
    // midpoint state in the local Cartesian frame (x, y) = (r, 0), (u_x, u_y) = (u_r, u_theta)
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const R r = ((R)rc[p] + rf[p]) * dR;
      const R ut = put[p];
      const R dx = (R)0.5 * h * ur[p] / G1[p], dy = (R)0.5 * h * ut / G1[p];
      const R uxh = ur[p] + (R)0.5 * h * F1[p], uyh = ut;
      int cn;
      R fn, rr, urr, utt;
      move_ring<R>(rc[p], rf[p], r, dx, dy, uxh, uyh, inv_dr, nr, cn, fn, rr, urr, utt);
      if (j0 + p < np && !(rr >= (R)0 && rr <= R_wall)) flag(d.status, ST_ESCAPE);
      pc[p] = cn;
      pf[p] = fn;
      pur[p] = urr;
      put[p] = utt;
    }
    // stage 2 at xi_k + dxi/2
    solve_stage<Pol, NT, PPT>(sm, d, j0, pc, pf, pur, put, cG0, cw, nbk, nbk + n1, G2, F2);
    // full step from the slice-k state with the midpoint derivative
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const R r = ((R)rc[p] + rf[p]) * dR;
      const R ut = r > (R)0 ? lz[p] / r : (R)0;
      const R xh = r + (R)0.5 * h * ur[p] / G1[p];
      const R yh = (R)0.5 * h * ut / G1[p];
      const R uxh = ur[p] + (R)0.5 * h * F1[p];
      const R uyh = ut;
      const R rh = sqrt(xh * xh + yh * yh);
      R ex = (R)1, ey = (R)0;
      if (rh > (R)0) {
        ex = xh / rh;
        ey = yh / rh;
      }
      const R dx = h * uxh / G2[p], dy = h * uyh / G2[p];
      const R uxn = ur[p] + h * F2[p] * ex, uyn = ut + h * F2[p] * ey;
      int cn;
      R fn, rn, urn, utn;
      move_ring<R>(rc[p], rf[p], r, dx, dy, uxn, uyn, inv_dr, nr, cn, fn, rn, urn, utn);
      if (j0 + p < np && (!(rn >= (R)0 && rn <= R_wall) || !isfinite(urn))) flag(d.status, ST_ESCAPE);
      if (j0 + p < np) {
        rc[p] = cn;
        rf[p] = fn;
        ur[p] = urn;
      }
    }
    __syncthreads();
  }
}

}  // namespace wake
