// Reverse-mode differentiation of the quasi-static step: the xi-march of Sec. II.A (RK2
// stages, hat deposits, the Gauss and E_z scans, the B_theta Helmholtz solve) and the beam
// push of Eqs. 8-11, in FP64.  Each forward routine here has a reverse routine that takes the
// adjoints of its outputs and accumulates the adjoints of its inputs (a vector-Jacobian
// product of the discrete scheme, not of a continuum approximation).
//
// The code is plain C++ with __host__ __device__ qualifiers.  Block-parallel loops go through
// Par (thread index, thread count, barrier): a CUDA block runs them with its threads, the
// host with one "thread", so the same arithmetic can be checked on a CPU.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define ADJ_HD __host__ __device__
#else
#define ADJ_HD
#endif

namespace wake {
namespace adj {

struct Par {
  int tid, nt;
  ADJ_HD void sync() const {
#ifdef __CUDA_ARCH__
    __syncthreads();
#endif
  }
};

// v is finite (not NaN or infinite): v - v is 0 exactly then.
ADJ_HD inline bool finite(double v) { return v - v == 0.0; }

// A load of a value another CTA may have written in the same launch (the pipelined steps):
// from L2 on the device (never a stale L1 line), a plain load on the host.
ADJ_HD inline double rd(const double *p) {
#ifdef __CUDA_ARCH__
  return __ldcg(p);
#else
  return *p;
#endif
}
ADJ_HD inline uint8_t rd(const uint8_t *p) {
#ifdef __CUDA_ARCH__
  return __ldcg(p);
#else
  return *p;
#endif
}

ADJ_HD inline void add_to(double *p, double v) {
#ifdef __CUDA_ARCH__
  atomicAdd(p, v);
#else
  *p += v;
#endif
}

// Inclusive sums out(i, S_i), S_i = sum_{j <= i} in(j) (or sum_{j >= i} when reverse), over
// i = 0..n-1.  One warp on the device (lanes hold consecutive chunks), serial on the host.
// All threads must call it; it ends with a barrier.
template <class In, class Out>
ADJ_HD void par_scan(const Par &P, int n, bool reverse, In in, Out out) {
#ifdef __CUDA_ARCH__
  if (P.tid < 32) {
    const int lane = P.tid, chunk = (n + 31) / 32, b = lane * chunk, e = b + chunk < n ? b + chunk : n;
    double s = 0.0;
    for (int q = b; q < e; ++q) s += in(reverse ? n - 1 - q : q);
    double incl = s;
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    double run = incl - s;
    for (int q = b; q < e; ++q) {
      const int i = reverse ? n - 1 - q : q;
      run += in(i);
      out(i, run);
    }
  }
  P.sync();
#else
  double run = 0.0;
  for (int q = 0; q < n; ++q) {
    const int i = reverse ? n - 1 - q : q;
    run += in(i);
    out(i, run);
  }
#endif
}

struct Dims {
  int nr, nxi, np;
  double dr, dxi, R;
};

ADJ_HD inline double vol(int i, int nr, double dr) {
  return i == 0 ? dr * dr / 6.0 : (i == nr ? dr * ((double)nr * dr / 2.0 - dr / 6.0) : (double)i * dr * dr);
}
ADJ_HD inline double alpha(int m, int nr) { return m == nr ? 1.0 : 0.5 - 1.0 / (6.0 * (double)m); }
ADJ_HD inline void cell_of(double r, double dr, int nr, int &c, double &f) {
  const double s = r / dr;
  int i = (int)floor(s);
  i = i < 0 ? 0 : (i > nr - 1 ? nr - 1 : i);
  c = i;
  f = s - (double)i;
}

// ---------------------------------------------------------------------------------------
// Tridiagonal systems a_q x_{q-1} + b_q x_q + c_q x_{q+1} = d_q (q = 0..n-1, a_0 = c_{n-1} = 0)
// by parallel cyclic reduction.  Ping-pong between (a, b, c, d) and (a2, b2, c2, d2); x may
// alias neither.  Ends with a barrier.
// ---------------------------------------------------------------------------------------
ADJ_HD inline void pcr(const Par &P, int n, double *a, double *b, double *c, double *d, double *a2, double *b2,
                       double *c2, double *d2, double *x) {
  double *A = a, *B = b, *C = c, *D = d, *A2 = a2, *B2 = b2, *C2 = c2, *D2 = d2;
  for (int s = 1; s < n; s <<= 1) {
    for (int q = P.tid; q < n; q += P.nt) {
      const int lo = q - s, hi = q + s;
      double na = 0.0, nb = B[q], nc = 0.0, nd = D[q];
      if (lo >= 0) {
        const double k1 = A[q] / B[lo];
        nb -= k1 * C[lo];
        nd -= k1 * D[lo];
        na = -k1 * A[lo];
      }
      if (hi < n) {
        const double k2 = C[q] / B[hi];
        nb -= k2 * A[hi];
        nd -= k2 * D[hi];
        nc = -k2 * C[hi];
      }
      A2[q] = na;
      B2[q] = nb;
      C2[q] = nc;
      D2[q] = nd;
    }
    P.sync();
    double *t;
    t = A; A = A2; A2 = t;
    t = B; B = B2; B2 = t;
    t = C; C = C2; C2 = t;
    t = D; D = D2; D2 = t;
  }
  for (int q = P.tid; q < n; q += P.nt) x[q] = D[q] / B[q];
  P.sync();
}

// ---------------------------------------------------------------------------------------
// One field stage (the radial solves of one slice, Eqs. 6-7, with the deposits they need).
// ---------------------------------------------------------------------------------------

// Node arrays of one stage (each n1 = nr + 1 long).
struct Nodes {
  double *rho, *dpsi, *psi, *jz, *chi, *T, *P, *U, *K, *dez, *ez, *Q, *bth;
  static constexpr int kCount = 13;
  ADJ_HD void carve(double *base, int n1) {
    double **f[kCount] = {&rho, &dpsi, &psi, &jz, &chi, &T, &P, &U, &K, &dez, &ez, &Q, &bth};
    for (int i = 0; i < kCount; ++i) *f[i] = base + (size_t)i * n1;
  }
};
// Per-ring values of one stage (each np long): its inputs and what the reverse pass reuses.
struct Rings {
  double *r, *ur, *ut, *Gam, *gam, *dp, *bf;
  static constexpr int kCount = 7;
  ADJ_HD void carve(double *base, int np) {
    double **f[kCount] = {&r, &ur, &ut, &Gam, &gam, &dp, &bf};
    for (int i = 0; i < kCount; ++i) *f[i] = base + (size_t)i * np;
  }
};
// Scratch shared by the stages: tridiagonal rows and their ping-pong copies (n1 each), and
// the adjoint node arrays.
struct Work {
  double *ta, *tb, *tc, *td, *a2, *b2, *c2, *d2;
  double *l_rho, *l_dpsi, *l_psi, *l_jz, *l_chi, *l_T, *l_P, *l_U, *l_K, *l_dez, *l_ez, *l_Q, *l_td, *l_bth;
  static constexpr int kCount = 22;
  ADJ_HD void carve(double *base, int n1) {
    double **f[kCount] = {&ta, &tb, &tc, &td, &a2, &b2, &c2, &d2, &l_rho, &l_dpsi, &l_psi,
                          &l_jz, &l_chi, &l_T, &l_P, &l_U, &l_K, &l_dez, &l_ez, &l_Q, &l_td, &l_bth};
    for (int i = 0; i < kCount; ++i) *f[i] = base + (size_t)i * n1;
  }
};

ADJ_HD inline double interp(const double *v, int c, double f) { return (1.0 - f) * v[c] + f * v[c + 1]; }

// Rows of the B_theta system (unknowns at nodes 1..nr, row q = node q + 1): central
// differences, a half cell at the wall, B_0 = 0.  Writes ta, tb, tc (tb includes -chi).
ADJ_HD inline void helmholtz_rows(const Par &P, const Dims &g, const Nodes &S, Work &W) {
  const int nr = g.nr;
  const double idr2 = 1.0 / (g.dr * g.dr);
  for (int i = 1 + P.tid; i <= nr; i += P.nt) {
    const int q = i - 1;
    const double rm = i - 0.5;
    if (i < nr) {
      const double rp = i + 0.5;
      W.ta[q] = q == 0 ? 0.0 : (i - 1) / rm * idr2;
      W.tc[q] = (i + 1) / rp * idr2;
      W.tb[q] = -(double)i * (1.0 / rp + 1.0 / rm) * idr2 - S.chi[i];
    } else {
      W.ta[q] = q == 0 ? 0.0 : 2.0 * (i - 1) / rm * idr2;
      W.tc[q] = 0.0;
      W.tb[q] = -2.0 * (double)i / rm * idr2 - S.chi[i];
    }
  }
}

// Forward stage: rings (R.r, R.ur, R.ut; constants G0, w), ion charge rho0 and beam density
// nb on this slice's nodes -> node fields in S and, per ring, Gamma (R.Gam) and the Cartesian
// radial force Fc (Eq. 4 without its centrifugal term).  Also keeps gamma, psi'(r_j) and
// B(r_j) per ring for the reverse pass.  Sets *bad when a Gamma <= 0.  Ends with a barrier.
ADJ_HD inline void stage_forward(const Par &P, const Dims &g, const Rings &R, const double *G0, const double *w,
                                 const double *rho0, const double *nb, Nodes &S, Work &W, double *Fc, int *bad) {
  const int nr = g.nr, n1 = nr + 1, np = g.np;
  const double dr = g.dr;
  for (int i = P.tid; i < n1; i += P.nt) S.rho[i] = S.jz[i] = S.chi[i] = S.T[i] = S.P[i] = S.U[i] = S.K[i] = 0.0;
  P.sync();
  for (int j = P.tid; j < np; j += P.nt) {
    int c;
    double f;
    cell_of(R.r[j], dr, nr, c, f);
    add_to(&S.rho[c], w[j] * (1.0 - f));
    add_to(&S.rho[c + 1], w[j] * f);
  }
  P.sync();
  // Gauss: psi'_m = (sum_{i<m} delta_i + alpha_m delta_m) / r_m, delta = rho - rho0
  par_scan(P, n1, false, [&](int i) { return S.rho[i] - rho0[i]; },
           [&](int m, double incl) {
             if (m == 0) {
               S.dpsi[0] = 0.0;
               return;
             }
             const double dl = S.rho[m] - rho0[m];
             S.dpsi[m] = (incl - dl + alpha(m, nr) * dl) / (m * dr);
           });
  // psi(R) = 0, inward trapezoid
  par_scan(P, n1, true, [&](int m) { return m < nr ? 0.5 * dr * (S.dpsi[m] + S.dpsi[m + 1]) : 0.0; },
           [&](int m, double incl) { S.psi[m] = -incl; });
  for (int j = P.tid; j < np; j += P.nt) {
    const double r = R.r[j], ur = R.ur[j], ut = R.ut[j];
    int c;
    double f;
    cell_of(r, dr, nr, c, f);
    const double Gam = G0[j] + interp(S.psi, c, f);
    if (!(Gam > 0.0)) *bad = 1;
    const double up2 = ur * ur + ut * ut;
    const double gam = (1.0 + up2 + Gam * Gam) / (2.0 * Gam), uz = gam - Gam;
    const double a = ur / Gam, dp = interp(S.dpsi, c, f);
    const double cent = r > 0.0 ? ut * ut / (Gam * r) : 0.0;
    const double F0 = (gam / Gam) * dp + cent;
    R.Gam[j] = Gam;
    R.gam[j] = gam;
    R.dp[j] = dp;
    const double wj = w[j];
    const double vjz = -wj * uz / Gam, vchi = wj / Gam, vT = wj * a * a, vP = wj * (a * a * dp - F0) / Gam,
                 vU = wj * a / Gam;
    add_to(&S.jz[c], vjz * (1.0 - f));
    add_to(&S.jz[c + 1], vjz * f);
    add_to(&S.chi[c], vchi * (1.0 - f));
    add_to(&S.chi[c + 1], vchi * f);
    add_to(&S.T[c], vT * (1.0 - f));
    add_to(&S.T[c + 1], vT * f);
    add_to(&S.P[c], vP * (1.0 - f));
    add_to(&S.P[c + 1], vP * f);
    add_to(&S.U[c], vU * (1.0 - f));
    add_to(&S.U[c + 1], vU * f);
    add_to(&S.K[c], wj * a);
  }
  P.sync();
  for (int i = P.tid; i < n1; i += P.nt) {
    const double V = vol(i, nr, dr);
    S.jz[i] = S.jz[i] / V - nb[i];
    S.chi[i] /= V;
    S.T[i] /= V;
    S.P[i] /= V;
    S.U[i] /= V;
    double dz = 0.0;
    if (i > 0) {
      const double al = alpha(i, nr), Km = i < nr ? S.K[i] : 0.0;
      dz = -((1.0 - al) * S.K[i - 1] + al * Km) / dr / (i * dr);
    }
    S.dez[i] = dz;
  }
  P.sync();
  par_scan(P, n1, true, [&](int m) { return m < nr ? 0.5 * dr * (S.dez[m] + S.dez[m + 1]) : 0.0; },
           [&](int m, double incl) { S.ez[m] = -incl; });
  for (int i = P.tid; i < n1; i += P.nt) S.Q[i] = S.P[i] + S.ez[i] * S.U[i];
  P.sync();
  helmholtz_rows(P, g, S, W);
  for (int i = 1 + P.tid; i <= nr; i += P.nt) {
    const int q = i - 1;
    if (i < nr)
      W.td[q] = (S.jz[i + 1] - S.jz[i - 1]) / (2.0 * dr) + S.Q[i] + (S.T[i + 1] - S.T[i - 1]) / (2.0 * dr) +
                S.T[i] / (i * dr);
    else
      W.td[q] = S.Q[i] + (S.T[i] - S.T[i - 1]) / dr + S.T[i] / (i * dr) - (S.jz[i - 1] + S.jz[i]) / dr;
  }
  P.sync();
  pcr(P, nr, W.ta, W.tb, W.tc, W.td, W.a2, W.b2, W.c2, W.d2, S.bth + 1);
  if (P.tid == 0) S.bth[0] = 0.0;
  P.sync();
  for (int j = P.tid; j < np; j += P.nt) {
    int c;
    double f;
    cell_of(R.r[j], dr, nr, c, f);
    const double bf = interp(S.bth, c, f);
    R.bf[j] = bf;
    Fc[j] = (R.gam[j] / R.Gam[j]) * R.dp[j] - bf;
  }
  P.sync();
}

// Reverse stage.  Given the adjoints of the stage's outputs - per ring lG (of Gamma) and lF
// (of Fc), per node lez, ler, lbth (of E_z, E_r = B - psi', B; NULL for a stage whose fields
// are not an output) - adds the adjoints of its inputs: per ring lr, lur, lut, lG0, lw; per
// node lnb (beam density, scaled by nb_scale) and lrho0.  S, R hold the stage's forward
// values; W is scratch.  Ends with a barrier.
ADJ_HD inline void stage_reverse(const Par &P, const Dims &g, const Rings &R, const double *G0, const double *w,
                                 const Nodes &S, Work &W, const double *lG, const double *lF, const double *lez,
                                 const double *ler, const double *lbth, double *lr, double *lur, double *lut,
                                 double *lG0, double *lw, double *lnb, double nb_scale, double *lrho0,
                                 double *lgam_s, double *lGam_s, double *ldp_s) {
  const int nr = g.nr, n1 = nr + 1, np = g.np;
  const double dr = g.dr;
  for (int i = P.tid; i < n1; i += P.nt) {
    W.l_rho[i] = W.l_dpsi[i] = W.l_psi[i] = W.l_jz[i] = W.l_chi[i] = W.l_T[i] = W.l_P[i] = W.l_U[i] = 0.0;
    W.l_K[i] = W.l_dez[i] = W.l_Q[i] = W.l_td[i] = 0.0;
    double lb = lbth ? lbth[i] : 0.0, ld = 0.0;
    if (ler && i > 0) {  // E_r = B - psi'
      lb += ler[i];
      ld -= ler[i];
    }
    W.l_bth[i] = lb;
    W.l_dpsi[i] = ld;
    W.l_ez[i] = lez ? lez[i] : 0.0;
  }
  P.sync();
  // Fc = (gamma/Gamma) psi'(r) - B(r), Gamma output
  for (int j = P.tid; j < np; j += P.nt) {
    int c;
    double f;
    cell_of(R.r[j], dr, nr, c, f);
    const double iG = 1.0 / R.Gam[j], gam = R.gam[j], dp = R.dp[j], lFj = lF[j];
    lgam_s[j] = lFj * dp * iG;
    lGam_s[j] = lG[j] - lFj * gam * dp * iG * iG;
    ldp_s[j] = lFj * gam * iG;
    const double lbf = -lFj;
    add_to(&W.l_bth[c], lbf * (1.0 - f));
    add_to(&W.l_bth[c + 1], lbf * f);
    lr[j] += lbf * (S.bth[c + 1] - S.bth[c]) / dr;
  }
  P.sync();
  // B = A(chi)^-1 td: l_td = A^-T l_B (rows 1..nr), l_chi_i += l_td_q B_i.  A^T has
  // sub-diagonal c_{q-1} and super-diagonal a_{q+1}.
  helmholtz_rows(P, g, S, W);
  P.sync();
  for (int q = P.tid; q < nr; q += P.nt) {
    W.a2[q] = q > 0 ? W.tc[q - 1] : 0.0;
    W.c2[q] = q + 1 < nr ? W.ta[q + 1] : 0.0;
    W.d2[q] = W.l_bth[q + 1];
  }
  P.sync();
  pcr(P, nr, W.a2, W.tb, W.c2, W.d2, W.ta, W.b2, W.tc, W.td, W.l_td);
  // td rows -> l_jz, l_Q, l_T; l_chi
  for (int i = 1 + P.tid; i <= nr; i += P.nt) {
    const int q = i - 1;
    const double lt = W.l_td[q];
    add_to(&W.l_chi[i], lt * S.bth[i]);
    add_to(&W.l_Q[i], lt);
    if (i < nr) {
      add_to(&W.l_jz[i + 1], lt / (2.0 * dr));
      add_to(&W.l_jz[i - 1], -lt / (2.0 * dr));
      add_to(&W.l_T[i + 1], lt / (2.0 * dr));
      add_to(&W.l_T[i - 1], -lt / (2.0 * dr));
      add_to(&W.l_T[i], lt / (i * dr));
    } else {
      add_to(&W.l_T[i], lt * (1.0 / dr + 1.0 / (i * dr)));
      add_to(&W.l_T[i - 1], -lt / dr);
      add_to(&W.l_jz[i - 1], -lt / dr);
      add_to(&W.l_jz[i], -lt / dr);
    }
  }
  P.sync();
  // Q = P + E_z U
  for (int i = P.tid; i < n1; i += P.nt) {
    const double lq = W.l_Q[i];
    W.l_P[i] += lq;
    W.l_ez[i] += lq * S.U[i];
    W.l_U[i] += lq * S.ez[i];
  }
  P.sync();
  // E_z_m = -sum_{i=m}^{nr-1} dr/2 (dez_i + dez_{i+1}):  l_dez_j = -dr/2 ([j<nr] L_j + L_{j-1}),
  // L_j = sum_{m<=j} l_ez_m
  par_scan(P, n1, false, [&](int m) { return W.l_ez[m]; }, [&](int m, double incl) { W.l_Q[m] = incl; });
  for (int j = P.tid; j < n1; j += P.nt)
    W.l_dez[j] = -0.5 * dr * ((j < nr ? W.l_Q[j] : 0.0) + (j > 0 ? W.l_Q[j - 1] : 0.0));
  P.sync();
  // dez_m = -((1-alpha_m) K_{m-1} + alpha_m K_m [m<nr]) / (m dr^2); node normalisation
  for (int i = P.tid; i < n1; i += P.nt) {
    double lk = 0.0;
    if (i < nr) {
      lk -= W.l_dez[i + 1] * (1.0 - alpha(i + 1, nr)) / ((i + 1) * dr * dr);
      if (i > 0) lk -= W.l_dez[i] * alpha(i, nr) / (i * dr * dr);
    }
    W.l_K[i] = lk;
    const double V = vol(i, nr, dr);
    lnb[i] -= nb_scale * W.l_jz[i];
    W.l_jz[i] /= V;
    W.l_chi[i] /= V;
    W.l_T[i] /= V;
    W.l_P[i] /= V;
    W.l_U[i] /= V;
  }
  P.sync();
  // per ring: deposits, F0, gamma/u_z, Gamma = G0 + psi(r)
  for (int j = P.tid; j < np; j += P.nt) {
    const double r = R.r[j], ur = R.ur[j], ut = R.ut[j];
    int c;
    double f;
    cell_of(r, dr, nr, c, f);
    const double Gam = R.Gam[j], gam = R.gam[j], dp = R.dp[j], uz = gam - Gam, wj = w[j];
    const double iG = 1.0 / Gam, iG2 = iG * iG, ir = r > 0.0 ? 1.0 / r : 0.0;
    const double up2 = ur * ur + ut * ut, a = ur * iG;
    const double cent = ut * ut * iG * ir;
    const double F0 = gam * iG * dp + cent;
    const double vjz = -wj * uz * iG, vchi = wj * iG, vT = wj * a * a, vP = wj * (a * a * dp - F0) * iG,
                 vU = wj * a * iG;
    const double g0 = 1.0 - f, g1 = f;
    const double ljz = W.l_jz[c] * g0 + W.l_jz[c + 1] * g1, lchi = W.l_chi[c] * g0 + W.l_chi[c + 1] * g1,
                 lT = W.l_T[c] * g0 + W.l_T[c + 1] * g1, lP = W.l_P[c] * g0 + W.l_P[c + 1] * g1,
                 lU = W.l_U[c] * g0 + W.l_U[c + 1] * g1, lK = W.l_K[c];
    double lf = vjz * (W.l_jz[c + 1] - W.l_jz[c]) + vchi * (W.l_chi[c + 1] - W.l_chi[c]) +
                vT * (W.l_T[c + 1] - W.l_T[c]) + vP * (W.l_P[c + 1] - W.l_P[c]) + vU * (W.l_U[c + 1] - W.l_U[c]);
    double lrj = lf / dr;
    lw[j] += (-ljz * uz + lchi + lP * (a * a * dp - F0) + lU * a) * iG + lT * a * a + lK * a;
    double luz = -ljz * wj * iG;
    double lGam = lGam_s[j] + (ljz * wj * uz - lchi * wj - lP * wj * (a * a * dp - F0) - lU * wj * a) * iG2;
    double la = lT * 2.0 * wj * a + (lP * wj * 2.0 * a * dp + lU * wj) * iG + lK * wj;
    double ldp = ldp_s[j] + lP * wj * a * a * iG;
    const double lF0 = -lP * wj * iG;
    double lgam = lgam_s[j] + lF0 * dp * iG;
    lGam -= lF0 * gam * dp * iG2;
    ldp += lF0 * gam * iG;
    const double lcent = lF0;
    double lutj = 0.0;
    if (r > 0.0) {
      lutj += lcent * 2.0 * ut * iG * ir;
      lGam -= lcent * cent * iG;
      lrj -= lcent * cent * ir;
    }
    double lurj = la * iG;
    lGam -= la * a * iG;
    // gamma = (1 + up2 + Gam^2)/(2 Gam), u_z = gamma - Gam
    lgam += luz;
    lGam -= luz;
    const double lup2 = 0.5 * lgam * iG;
    lGam += lgam * (0.5 - 0.5 * (1.0 + up2) * iG2);
    lurj += 2.0 * ur * lup2;
    lutj += 2.0 * ut * lup2;
    // psi'(r) and psi(r) gathers
    add_to(&W.l_dpsi[c], ldp * g0);
    add_to(&W.l_dpsi[c + 1], ldp * g1);
    lrj += ldp * (S.dpsi[c + 1] - S.dpsi[c]) / dr;
    lG0[j] += lGam;
    add_to(&W.l_psi[c], lGam * g0);
    add_to(&W.l_psi[c + 1], lGam * g1);
    lrj += lGam * (S.psi[c + 1] - S.psi[c]) / dr;
    lr[j] += lrj;
    lur[j] += lurj;
    lut[j] += lutj;
  }
  P.sync();
  // psi_m = -sum_{i=m}^{nr-1} dr/2 (psi'_i + psi'_{i+1})
  par_scan(P, n1, false, [&](int m) { return W.l_psi[m]; }, [&](int m, double incl) { W.l_Q[m] = incl; });
  for (int j = P.tid; j < n1; j += P.nt)
    W.l_dpsi[j] += -0.5 * dr * ((j < nr ? W.l_Q[j] : 0.0) + (j > 0 ? W.l_Q[j - 1] : 0.0));
  P.sync();
  // psi'_m = (sum_{i<m} delta_i + alpha_m delta_m) / (m dr):
  // l_delta_i = sum_{m>i} l_psi'_m / (m dr) + [i>0] alpha_i l_psi'_i / (i dr)
  par_scan(P, n1, true, [&](int m) { return m > 0 ? W.l_dpsi[m] / (m * dr) : 0.0; },
           [&](int m, double incl) { W.l_td[m] = incl; });
  for (int i = P.tid; i < n1; i += P.nt) {
    const double own = i > 0 ? W.l_dpsi[i] / (i * dr) : 0.0;
    const double ld = (W.l_td[i] - own) + (i > 0 ? alpha(i, nr) * own : 0.0);
    W.l_rho[i] = ld;
    lrho0[i] -= ld;
  }
  P.sync();
  for (int j = P.tid; j < np; j += P.nt) {
    int c;
    double f;
    cell_of(R.r[j], dr, nr, c, f);
    lw[j] += W.l_rho[c] * (1.0 - f) + W.l_rho[c + 1] * f;
    lr[j] += w[j] * (W.l_rho[c + 1] - W.l_rho[c]) / dr;
  }
  P.sync();
}

// ---------------------------------------------------------------------------------------
// One slice of the march (RK2 midpoint in a local Cartesian frame, Sec. II.A): the slice
// state (r, u_r) and the ring constants l, G0, w -> stage 1 at xi_k (output fields), the
// midpoint, stage 2 at xi_k + dxi/2, the full step to slice k+1.
// ---------------------------------------------------------------------------------------

// Per-ring values of the midpoint and full step (each np long).
struct Mid {
  double *G1, *F1, *xh, *yh, *uxh, *uyh, *G2, *F2, *reflh;
  static constexpr int kCount = 9;
  ADJ_HD void carve(double *base, int np) {
    double **f[kCount] = {&G1, &F1, &xh, &yh, &uxh, &uyh, &G2, &F2, &reflh};
    for (int i = 0; i < kCount; ++i) *f[i] = base + (size_t)i * np;
  }
};

// Midpoint state from stage 1 (R1: r, u_r, u_theta, with M.G1, M.F1) into R2 (r, u_r,
// u_theta), specular reflection at the wall.  Sets *bad if a ring leaves [0, R].
ADJ_HD inline void midpoint(const Par &P, const Dims &g, const Rings &R1, Mid &M, Rings &R2, int *bad) {
  const double h = 0.5 * g.dxi;
  for (int j = P.tid; j < g.np; j += P.nt) {
    const double xh = R1.r[j] + h * R1.ur[j] / M.G1[j], yh = h * R1.ut[j] / M.G1[j];
    const double uxh = R1.ur[j] + h * M.F1[j], uyh = R1.ut[j];
    M.xh[j] = xh;
    M.yh[j] = yh;
    M.uxh[j] = uxh;
    M.uyh[j] = uyh;
    double rr = sqrt(xh * xh + yh * yh), urr, utt;
    if (rr > 0.0) {
      urr = (xh * uxh + yh * uyh) / rr;
      utt = (xh * uyh - yh * uxh) / rr;
    } else {
      urr = sqrt(uxh * uxh + uyh * uyh);
      utt = 0.0;
    }
    double refl = 0.0;
    if (rr > g.R) {
      rr = 2.0 * g.R - rr;
      urr = -urr;
      refl = 1.0;
    }
    if (!(rr >= 0.0 && rr <= g.R)) *bad = 2;
    M.reflh[j] = refl;
    R2.r[j] = rr;
    R2.ur[j] = urr;
    R2.ut[j] = utt;
  }
  P.sync();
}

// Full step from the slice state (R1) with the stage-2 values (M) to (rn, urn).
ADJ_HD inline void full_step(const Par &P, const Dims &g, const Rings &R1, const Mid &M, double *rn, double *urn,
                             int *bad) {
  const double dxi = g.dxi;
  for (int j = P.tid; j < g.np; j += P.nt) {
    const double xh = M.xh[j], yh = M.yh[j];
    const double rr = sqrt(xh * xh + yh * yh);
    double ex = 1.0, ey = 0.0;
    if (rr > 0.0) {
      ex = xh / rr;
      ey = yh / rr;
    }
    const double xn = R1.r[j] + dxi * M.uxh[j] / M.G2[j], yn = dxi * M.uyh[j] / M.G2[j];
    const double uxn = R1.ur[j] + dxi * M.F2[j] * ex, uyn = R1.ut[j] + dxi * M.F2[j] * ey;
    double r2 = sqrt(xn * xn + yn * yn);
    double u2 = r2 > 0.0 ? (xn * uxn + yn * uyn) / r2 : sqrt(uxn * uxn + uyn * uyn);
    if (r2 > g.R) {
      r2 = 2.0 * g.R - r2;
      u2 = -u2;
    }
    if (!(r2 >= 0.0 && r2 <= g.R) || !finite(u2)) *bad = 2;
    rn[j] = r2;
    urn[j] = u2;
  }
  P.sync();
}

// Reverse of the full step: lrn, lurn (adjoints of the new state) -> adds to lr, lur, lut
// (slice state) and writes lG2, lF2 (stage-2 outputs) and lxh, lyh, luxh, luyh (midpoint).
ADJ_HD inline void full_step_reverse(const Par &P, const Dims &g, const Rings &R1, const Mid &M, const double *lrn,
                                     const double *lurn, double *lr, double *lur, double *lut, double *lG2,
                                     double *lF2, double *lxh, double *lyh, double *luxh, double *luyh) {
  const double dxi = g.dxi;
  for (int j = P.tid; j < g.np; j += P.nt) {
    const double xh = M.xh[j], yh = M.yh[j], G2 = M.G2[j], F2 = M.F2[j], uxh = M.uxh[j], uyh = M.uyh[j];
    const double rr = sqrt(xh * xh + yh * yh);
    double ex = 1.0, ey = 0.0;
    if (rr > 0.0) {
      ex = xh / rr;
      ey = yh / rr;
    }
    const double iG2 = 1.0 / G2;
    const double xn = R1.r[j] + dxi * uxh * iG2, yn = dxi * uyh * iG2;
    const double uxn = R1.ur[j] + dxi * F2 * ex, uyn = R1.ut[j] + dxi * F2 * ey;
    const double r2 = sqrt(xn * xn + yn * yn), ir2 = 1.0 / r2;
    const double u2 = (xn * uxn + yn * uyn) * ir2;
    double lr2 = lrn[j], lu2 = lurn[j];
    if (r2 > g.R) {
      lr2 = -lr2;
      lu2 = -lu2;
    }
    double lxn = lr2 * xn * ir2 + lu2 * (uxn - u2 * xn * ir2) * ir2;
    double lyn = lr2 * yn * ir2 + lu2 * (uyn - u2 * yn * ir2) * ir2;
    const double luxn = lu2 * xn * ir2, luyn = lu2 * yn * ir2;
    lur[j] += luxn;
    lut[j] += luyn;
    double lF = luxn * dxi * ex + luyn * dxi * ey;
    const double lex = luxn * dxi * F2, ley = luyn * dxi * F2;
    lr[j] += lxn;
    double lux = lxn * dxi * iG2, luy = lyn * dxi * iG2;
    double lG = -(lxn * uxh + lyn * uyh) * dxi * iG2 * iG2;
    double lx = 0.0, ly = 0.0;
    if (rr > 0.0) {
      const double irr = 1.0 / rr, ir3 = irr * irr * irr;
      lx = lex * (irr - xh * xh * ir3) - ley * yh * xh * ir3;
      ly = -lex * xh * yh * ir3 + ley * (irr - yh * yh * ir3);
    }
    lG2[j] = lG;
    lF2[j] = lF;
    lxh[j] = lx;
    lyh[j] = ly;
    luxh[j] = lux;
    luyh[j] = luy;
  }
  P.sync();
}

// Reverse of the midpoint: lr2, lur2, lut2 (adjoints of the stage-2 inputs) plus the
// partial lxh.. from the full step -> adds to lr, lur, lut (slice state) and writes lG1, lF1.
ADJ_HD inline void midpoint_reverse(const Par &P, const Dims &g, const Rings &R1, const Mid &M, const Rings &R2,
                                    const double *lr2, const double *lur2, const double *lut2, const double *lxh0,
                                    const double *lyh0, const double *luxh0, const double *luyh0, double *lr,
                                    double *lur, double *lut, double *lG1, double *lF1) {
  const double h = 0.5 * g.dxi;
  for (int j = P.tid; j < g.np; j += P.nt) {
    const double xh = M.xh[j], yh = M.yh[j], uxh = M.uxh[j], uyh = M.uyh[j];
    const double rr = sqrt(xh * xh + yh * yh);
    double lrr = lr2[j], lurr = lur2[j];
    const double lutt = lut2[j];
    if (M.reflh[j] != 0.0) {
      lrr = -lrr;
      lurr = -lurr;
    }
    double lxh = lxh0[j], lyh = lyh0[j], luxh = luxh0[j], luyh = luyh0[j];
    if (rr > 0.0) {
      const double irr = 1.0 / rr;
      const double urr = (xh * uxh + yh * uyh) * irr, utt = (xh * uyh - yh * uxh) * irr;
      lxh += (lrr * xh + lurr * (uxh - urr * xh * irr) + lutt * (uyh - utt * xh * irr)) * irr;
      lyh += (lrr * yh + lurr * (uyh - urr * yh * irr) + lutt * (-uxh - utt * yh * irr)) * irr;
      luxh += (lurr * xh - lutt * yh) * irr;
      luyh += (lurr * yh + lutt * xh) * irr;
    }
    const double iG1 = 1.0 / M.G1[j], ur = R1.ur[j], ut = R1.ut[j];
    lr[j] += lxh;
    lur[j] += lxh * h * iG1 + luxh;
    lut[j] += lyh * h * iG1 + luyh;
    lG1[j] = -(lxh * ur + lyh * ut) * h * iG1 * iG1;
    lF1[j] = luxh * h;
  }
  P.sync();
}

// ---------------------------------------------------------------------------------------
// Beam (Eq. 12 bunches, Eqs. 8-11 Boris push, deposit on the (r, xi) nodes)
// ---------------------------------------------------------------------------------------

struct BoundsRZ {
  int nr, nxi;
  double dr, dxi, rmax, ximax;
};

// Bilinear node weights of a point: cell (c, k), offsets (f, g).
ADJ_HD inline void cell_rz(const BoundsRZ &b, double r, double xi, int &c, double &f, int &k, double &gg) {
  cell_of(r, b.dr, b.nr, c, f);
  cell_of(xi, b.dxi, b.nxi, k, gg);
}

// Boris step with the fields (Er, Ez, Bt) at the particle.  In/out: x, y, ux, uy, uz, xi.
ADJ_HD inline void boris(double &x, double &y, double &ux, double &uy, double &uz, double &xi, double Er, double Ez,
                         double Bt, double dt) {
  const double h = -0.5 * dt;
  const double r = sqrt(x * x + y * y);
  const double cs = r > 0.0 ? x / r : 0.0, sn = r > 0.0 ? y / r : 0.0;
  const double Ex = Er * cs, Ey = Er * sn, Bx = -Bt * sn, By = Bt * cs;
  const double mx = ux + h * Ex, my = uy + h * Ey, mz = uz + h * Ez;
  const double gm = sqrt(1.0 + mx * mx + my * my + mz * mz);
  const double tx = h * Bx / gm, ty = h * By / gm;
  const double px = mx - mz * ty, py = my + mz * tx, pz = mz + (mx * ty - my * tx);
  const double s = 2.0 / (1.0 + tx * tx + ty * ty);
  const double sx = s * tx, sy = s * ty;
  const double uxn = mx - pz * sy + h * Ex, uyn = my + pz * sx + h * Ey;
  const double uzn = uz + (2.0 * h * Ez + (px * sy - py * sx));
  const double up2 = uxn * uxn + uyn * uyn;
  const double gam = sqrt(1.0 + up2 + uzn * uzn);
  x += dt * uxn / gam;
  y += dt * uyn / gam;
  xi += dt * (1.0 + up2) / (gam * (gam + uzn));
  ux = uxn;
  uy = uyn;
  uz = uzn;
}

// Reverse of boris(): (x, y, ux, uy, uz, xi) is the state BEFORE the step; l* hold the
// adjoints of the state after it and are replaced by those before it; lEr, lEz, lBt receive
// the adjoints of the gathered fields.
ADJ_HD inline void boris_reverse(double x, double y, double ux, double uy, double uz, double Er, double Ez,
                                 double Bt, double dt, double &lx, double &ly, double &lux, double &luy,
                                 double &luz, double &lxi, double &lEr, double &lEz, double &lBt) {
  const double h = -0.5 * dt;
  const double r = sqrt(x * x + y * y);
  const double cs = r > 0.0 ? x / r : 0.0, sn = r > 0.0 ? y / r : 0.0;
  const double Ex = Er * cs, Ey = Er * sn, Bx = -Bt * sn, By = Bt * cs;
  const double mx = ux + h * Ex, my = uy + h * Ey, mz = uz + h * Ez;
  const double gm2 = 1.0 + mx * mx + my * my + mz * mz, gm = sqrt(gm2);
  const double tx = h * Bx / gm, ty = h * By / gm;
  const double px = mx - mz * ty, py = my + mz * tx, pz = mz + (mx * ty - my * tx);
  const double den = 1.0 + tx * tx + ty * ty, s = 2.0 / den;
  const double sx = s * tx, sy = s * ty;
  const double uxn = mx - pz * sy + h * Ex, uyn = my + pz * sx + h * Ey;
  const double uzn = uz + (2.0 * h * Ez + (px * sy - py * sx));
  const double up2 = uxn * uxn + uyn * uyn;
  const double gam2 = 1.0 + up2 + uzn * uzn, gam = sqrt(gam2);
  // xi' = xi + dt (1 + up2) / (gam (gam + uzn)), x' = x + dt uxn / gam, y' = y + dt uyn / gam
  const double D = gam * (gam + uzn), Nn = 1.0 + up2;
  double luxn = lux, luyn = luy, luzn = luz;  // adjoints of the new momenta
  double lgam = 0.0, lup2 = 0.0;
  // xi
  lup2 += lxi * dt / D;
  const double lD = -lxi * dt * Nn / (D * D);
  lgam += lD * (2.0 * gam + uzn);
  luzn += lD * gam;
  // x, y
  luxn += lx * dt / gam;
  luyn += ly * dt / gam;
  lgam += -lx * dt * uxn / (gam * gam) - ly * dt * uyn / (gam * gam);
  // gam = sqrt(1 + up2 + uzn^2)
  lup2 += lgam / (2.0 * gam);
  luzn += lgam * uzn / gam;
  luxn += lup2 * 2.0 * uxn;
  luyn += lup2 * 2.0 * uyn;
  // uzn = uz + 2 h Ez + px sy - py sx
  double luz0 = luzn, lEz_ = luzn * 2.0 * h;
  double lpx = luzn * sy, lpy = -luzn * sx, lsy = luzn * px, lsx = -luzn * py;
  // uxn = mx - pz sy + h Ex; uyn = my + pz sx + h Ey
  double lmx = luxn, lpz = -luxn * sy + luyn * sx, lEx = luxn * h, lmy = luyn, lEy = luyn * h;
  lsy += -luxn * pz;
  lsx += luyn * pz;
  // sx = s tx, sy = s ty, s = 2 / den
  double ltx = lsx * s, lty = lsy * s;
  const double ls = lsx * tx + lsy * ty;
  const double lden = -ls * 2.0 / (den * den);
  ltx += lden * 2.0 * tx;
  lty += lden * 2.0 * ty;
  // pz = mz + mx ty - my tx; py = my + mz tx; px = mx - mz ty
  double lmz = lpz + lpy * tx - lpx * ty;
  lmx += lpz * ty + lpx;
  lmy += -lpz * tx + lpy;
  lty += lpz * mx - lpx * mz;
  ltx += -lpz * my + lpy * mz;
  // tx = h Bx / gm, ty = h By / gm
  double lBx = ltx * h / gm, lBy = lty * h / gm;
  const double lgm = -ltx * h * Bx / gm2 - lty * h * By / gm2;
  // gm = sqrt(1 + mx^2 + my^2 + mz^2)
  lmx += lgm * mx / gm;
  lmy += lgm * my / gm;
  lmz += lgm * mz / gm;
  // mx = ux + h Ex, my = uy + h Ey, mz = uz + h Ez
  lux = lmx;
  luy = lmy;
  luz = luz0 + lmz;
  lEx += lmx * h;
  lEy += lmy * h;
  lEz_ += lmz * h;
  // Ex = Er cs, Ey = Er sn, Bx = -Bt sn, By = Bt cs
  lEr = lEx * cs + lEy * sn;
  lBt = -lBx * sn + lBy * cs;
  lEz = lEz_;
  const double lcs = lEx * Er + lBy * Bt, lsn = lEy * Er - lBx * Bt;
  if (r > 0.0) {
    const double r3 = r * r * r;
    lx += lcs * (1.0 / r - x * x / r3) - lsn * x * y / r3;
    ly += -lcs * x * y / r3 + lsn * (1.0 / r - y * y / r3);
  }
  // lxi unchanged: the step adds to xi
}


// ---------------------------------------------------------------------------------------
// The march of one beam step with checkpoints, and its reverse
// ---------------------------------------------------------------------------------------

struct MarchArgs {
  Dims g;
  int B, nblk;                 // checkpoint interval and block count
  const double *r0, *ur0, *l, *G0, *w, *rho0;
  const double *nb;            // this step's beam density grid
  double *ez, *er, *bth;       // forward: output grids
  double *ckpt;                // nblk x 2 x np: (r, u_r) at slices 0, B, 2B, ...
  double *tape;                // per-slice intermediates of one block
  double *lring;               // per-ring adjoint scratch (kLring x np)
  const double *lez, *ler, *lbth;  // reverse: field adjoints (grids)
  double *lnb;                 // reverse: beam-density adjoint grid (accumulated)
  double *lG0, *lw, *ll, *lur0;    // reverse: ring-constant adjoints (accumulated over steps)
  double *lrho0;               // reverse: ion-charge adjoint (accumulated)
  double *nbh, *lnbh;          // n1 scratch
  int *status;
};

constexpr int kLring = 24;

// One block-slice's tape: stage nodes, stage rings, midpoint.
struct SliceTape {
  Nodes S1, S2;
  Rings R1, R2;
  Mid M;
};
ADJ_HD inline size_t slice_tape_doubles(int n1, int np) {
  return (size_t)2 * Nodes::kCount * n1 + (size_t)2 * Rings::kCount * np + (size_t)Mid::kCount * np;
}
ADJ_HD inline SliceTape slice_tape(double *base, int s, int n1, int np) {
  SliceTape t;
  double *p = base + (size_t)s * slice_tape_doubles(n1, np);
  t.S1.carve(p, n1);
  p += (size_t)Nodes::kCount * n1;
  t.S2.carve(p, n1);
  p += (size_t)Nodes::kCount * n1;
  t.R1.carve(p, np);
  p += (size_t)Rings::kCount * np;
  t.R2.carve(p, np);
  p += (size_t)Rings::kCount * np;
  t.M.carve(p, np);
  return t;
}

// No-op hooks of the march bodies (the sequential form and the host build).
struct NoHook {
  template <class... A>
  ADJ_HD bool operator()(A &&...) const {
    return true;
  }
};

// Forward slices k0 .. k1-1 starting from the state in T[0].R1 (r, u_r), each slice's
// intermediates in tape slot k - k0 when keep, else all in slot 0.  Writes the stage-1 output
// fields when a.ez is set and checkpoints when ckpt_out.  before(k) runs at the start of
// slice k (false: stop, block-uniform), after(k) once slice k's output fields are written.
// Returns false if before() stopped the march.
template <class Before = NoHook, class After = NoHook>
ADJ_HD inline bool march_slices(const Par &P, const MarchArgs &a, Work &W, int k0, int k1, bool keep, bool outputs,
                                bool ckpt_out, int *bad, Before &&before = Before(), After &&after = After()) {
  const Dims &g = a.g;
  const int n1 = g.nr + 1, np = g.np;
  for (int k = k0; k < k1; ++k) {
    if (!before(k)) return false;
    const int s = keep ? k - k0 : 0;
    SliceTape T = slice_tape(a.tape, s, n1, np);
    if (ckpt_out && k % a.B == 0) {
      double *ck = a.ckpt + (size_t)(k / a.B) * 2 * np;
      for (int j = P.tid; j < np; j += P.nt) {
        ck[j] = T.R1.r[j];
        ck[np + j] = T.R1.ur[j];
      }
    }
    for (int j = P.tid; j < np; j += P.nt) T.R1.ut[j] = T.R1.r[j] > 0.0 ? a.l[j] / T.R1.r[j] : 0.0;
    P.sync();
    stage_forward(P, g, T.R1, a.G0, a.w, a.rho0, a.nb + (size_t)k * n1, T.S1, W, T.M.F1, bad);
    for (int j = P.tid; j < np; j += P.nt) T.M.G1[j] = T.R1.Gam[j];
    if (outputs)
      for (int i = P.tid; i < n1; i += P.nt) {
        a.ez[(size_t)k * n1 + i] = T.S1.ez[i];
        a.bth[(size_t)k * n1 + i] = T.S1.bth[i];
        a.er[(size_t)k * n1 + i] = i > 0 ? T.S1.bth[i] - T.S1.dpsi[i] : 0.0;
      }
    P.sync();
    after(k);
    if (k == g.nxi) break;
    midpoint(P, g, T.R1, T.M, T.R2, bad);
    for (int i = P.tid; i < n1; i += P.nt) a.nbh[i] = 0.5 * (a.nb[(size_t)k * n1 + i] + a.nb[(size_t)(k + 1) * n1 + i]);
    P.sync();
    stage_forward(P, g, T.R2, a.G0, a.w, a.rho0, a.nbh, T.S2, W, T.M.F2, bad);
    for (int j = P.tid; j < np; j += P.nt) T.M.G2[j] = T.R2.Gam[j];
    P.sync();
    // next slice's state: the next tape slot, or slot 0 (in place is not possible: the
    // full step reads R1), so through the per-ring scratch
    double *rn = a.lring + 0 * (size_t)np, *urn = a.lring + 1 * (size_t)np;
    full_step(P, g, T.R1, T.M, rn, urn, bad);
    const int sn = keep ? s + 1 : 0;
    if (k + 1 < k1 || !keep) {
      SliceTape Tn = slice_tape(a.tape, sn, n1, np);
      for (int j = P.tid; j < np; j += P.nt) {
        Tn.R1.r[j] = rn[j];
        Tn.R1.ur[j] = urn[j];
      }
    }
    P.sync();
  }
  return true;
}

// Forward march of one beam step: fields of every slice to a.ez/a.er/a.bth, checkpoints of
// the ring state every a.B slices, or (full_tape) every slice's intermediates on the tape,
// a.tape then holding Nxi + 1 slices.  W is the caller's scratch (Work::kCount x n1).  Hooks as
// march_slices; returns false if before() stopped the march.
template <class Before = NoHook, class After = NoHook>
ADJ_HD inline bool march_forward_body(const Par &P, const MarchArgs &a, Work &W, int *bad, Before &&before = Before(),
                                      After &&after = After(), bool full_tape = false) {
  SliceTape T = slice_tape(a.tape, 0, a.g.nr + 1, a.g.np);
  for (int j = P.tid; j < a.g.np; j += P.nt) {
    T.R1.r[j] = a.r0[j];
    T.R1.ur[j] = a.ur0[j];
  }
  P.sync();
  return march_slices(P, a, W, 0, a.g.nxi + 1, full_tape, true, !full_tape, bad, before, after);
}

// Per-ring adjoint scratch rows in a.lring.
enum {
  LR_RN = 0, LR_URN, LR_LRN, LR_LURN, LR_LR, LR_LUR, LR_LUT, LR_LG1, LR_LF1, LR_LG2, LR_LF2, LR_LXH, LR_LYH,
  LR_LUXH, LR_LUYH, LR_LR2, LR_LUR2, LR_LUT2, LR_SGAM, LR_SGAMMA, LR_SDP, LR_ZERO
};

// Reverse march of one beam step (the adjoints of its output fields in a.lez/a.ler/a.lbth):
// block by block from the last, each recomputed from its checkpoint with its intermediates on
// the tape, then reversed slice by slice.  Adds the beam-density adjoint to a.lnb and the
// ring-constant adjoints to a.lG0, a.lw, a.ll, a.lur0, a.lrho0.  pre(k) runs before slice k
// is reversed (false: stop, block-uniform; the field adjoints of slice k must be complete
// when it returns true), post(k) once it is (rows >= k + 1 of a.lnb are then final).  Returns
// false if pre() stopped it.  With a second tape buffer tape2, pre(k, idle) is also given
// idle(): a block-uniform call that recomputes the block below into the other buffer (once;
// it returns false when there is nothing left to do), for a pre() that would otherwise wait;
// without one, or if idle() was not called, the block below is recomputed after the current
// one is reversed.  full_tape: the forward kept every slice on a.tape (march_forward_body's
// full_tape); nothing is recomputed.
template <class Pre = NoHook, class Post = NoHook>
ADJ_HD inline bool march_reverse_body(const Par &P, const MarchArgs &a, Work &W, int *bad, Pre &&pre = Pre(),
                                      Post &&post = Post(), double *tape2 = nullptr, bool full_tape = false) {
  const Dims &g = a.g;
  const int n1 = g.nr + 1, np = g.np;
  double *L[LR_ZERO + 1];
  for (int q = 0; q <= LR_ZERO; ++q) L[q] = a.lring + (size_t)q * np;
  for (int j = P.tid; j < np; j += P.nt) {
    L[LR_LRN][j] = L[LR_LURN][j] = 0.0;
    L[LR_ZERO][j] = 0.0;
  }
  P.sync();
  double *bufs[2] = {a.tape, tape2 ? tape2 : a.tape};
  // recompute block blk from its checkpoint into tape buffer buf
  auto recompute = [&](int blk, double *buf) {
    const int k0 = blk * a.B, k1 = k0 + a.B < g.nxi + 1 ? k0 + a.B : g.nxi + 1;
    MarchArgs ab = a;
    ab.tape = buf;
    SliceTape T0 = slice_tape(buf, 0, n1, np);
    const double *ck = a.ckpt + (size_t)blk * 2 * np;
    for (int j = P.tid; j < np; j += P.nt) {
      T0.R1.r[j] = ck[j];
      T0.R1.ur[j] = ck[np + j];
    }
    P.sync();
    march_slices(P, ab, W, k0, k1, true, false, false, bad);
  };
  int cur = 0;
  const int nblk = full_tape ? 1 : a.nblk;
  if (!full_tape) recompute(a.nblk - 1, bufs[cur]);
  for (int blk = nblk - 1; blk >= 0; --blk) {
    const int k0 = full_tape ? 0 : blk * a.B;
    const int k1 = full_tape ? g.nxi + 1 : (k0 + a.B < g.nxi + 1 ? k0 + a.B : g.nxi + 1);
    bool below_done = false;
    auto idle = [&]() -> bool {
      if (blk == 0 || below_done || !tape2) return false;
      recompute(blk - 1, bufs[cur ^ 1]);
      below_done = true;
      return true;
    };
    for (int k = k1 - 1; k >= k0; --k) {
      if (!pre(k, idle)) return false;
      SliceTape T = slice_tape(bufs[cur], k - k0, n1, np);
      for (int j = P.tid; j < np; j += P.nt) L[LR_LR][j] = L[LR_LUR][j] = L[LR_LUT][j] = 0.0;
      P.sync();
      const double *lG1 = L[LR_ZERO], *lF1 = L[LR_ZERO];
      if (k < g.nxi) {
        full_step_reverse(P, g, T.R1, T.M, L[LR_LRN], L[LR_LURN], L[LR_LR], L[LR_LUR], L[LR_LUT], L[LR_LG2],
                          L[LR_LF2], L[LR_LXH], L[LR_LYH], L[LR_LUXH], L[LR_LUYH]);
        for (int j = P.tid; j < np; j += P.nt) L[LR_LR2][j] = L[LR_LUR2][j] = L[LR_LUT2][j] = 0.0;
        for (int i = P.tid; i < n1; i += P.nt) a.lnbh[i] = 0.0;
        P.sync();
        stage_reverse(P, g, T.R2, a.G0, a.w, T.S2, W, L[LR_LG2], L[LR_LF2], nullptr, nullptr, nullptr, L[LR_LR2],
                      L[LR_LUR2], L[LR_LUT2], a.lG0, a.lw, a.lnbh, 1.0, a.lrho0, L[LR_SGAM], L[LR_SGAMMA],
                      L[LR_SDP]);
        for (int i = P.tid; i < n1; i += P.nt) {
          a.lnb[(size_t)k * n1 + i] += 0.5 * a.lnbh[i];
          a.lnb[(size_t)(k + 1) * n1 + i] += 0.5 * a.lnbh[i];
        }
        midpoint_reverse(P, g, T.R1, T.M, T.R2, L[LR_LR2], L[LR_LUR2], L[LR_LUT2], L[LR_LXH], L[LR_LYH],
                         L[LR_LUXH], L[LR_LUYH], L[LR_LR], L[LR_LUR], L[LR_LUT], L[LR_LG1], L[LR_LF1]);
        lG1 = L[LR_LG1];
        lF1 = L[LR_LF1];
      }
      stage_reverse(P, g, T.R1, a.G0, a.w, T.S1, W, lG1, lF1, a.lez + (size_t)k * n1, a.ler + (size_t)k * n1,
                    a.lbth + (size_t)k * n1, L[LR_LR], L[LR_LUR], L[LR_LUT], a.lG0, a.lw, a.lnb + (size_t)k * n1,
                    1.0, a.lrho0, L[LR_SGAM], L[LR_SGAMMA], L[LR_SDP]);
      // u_theta = l / r
      for (int j = P.tid; j < np; j += P.nt) {
        const double r = T.R1.r[j], lut = L[LR_LUT][j];
        double lr = L[LR_LR][j];
        if (r > 0.0) {
          a.ll[j] += lut / r;
          lr -= lut * a.l[j] / (r * r);
        }
        L[LR_LRN][j] = lr;
        L[LR_LURN][j] = L[LR_LUR][j];
      }
      P.sync();
      post(k);
    }
    if (blk > 0) {
      if (!below_done) recompute(blk - 1, bufs[cur ^ 1]);
      cur ^= 1;
    }
  }
  // slice 0 starts from (r0, u_r0): r0 is fixed, u_r0 = u_th n_r
  for (int j = P.tid; j < np; j += P.nt) a.lur0[j] += L[LR_LURN][j];
  P.sync();
  return true;
}


// ---------------------------------------------------------------------------------------
// Beam of the adjoint form: FP64 state, per-particle weights (per-particle bodies)
// ---------------------------------------------------------------------------------------

struct Beam {
  double *x, *y, *ux, *uy, *uz, *xi;
  uint8_t *lost;
};
struct BeamConst {
  int64_t n, n_drive;
  int nbins;
  BoundsRZ b;
  double dt, gamma_b;
};
struct BunchSpec {
  double sigma_r, eps_n, xi_d, sigma_zw, n_d;
};

// Eq. 12 bunches with theta = (n_w, delay, sigma_zd, u_th) and the witness profile: particle
// j's position, momentum, weight and witness bin (bins span xi_w +- 3 sigma_zw, by the
// particle's normal draw).
ADJ_HD inline void beam_init_one(const BeamConst &c, const BunchSpec &q, Beam s, double *wgt, int *bin,
                                 const double *nm, const double *theta, const double *profile, int64_t j) {
  const double n_w = theta[0], delay = theta[1], szd = theta[2];
  const double su = q.eps_n / q.sigma_r, s2pi = sqrt(2.0 * 3.14159265358979323846);
  const int64_t nw = c.n - c.n_drive;
  const double wd = c.n_drive > 0 ? q.n_d * s2pi * q.sigma_r * q.sigma_r * szd / (double)c.n_drive : 0.0;
  const double ww = nw > 0 ? n_w * s2pi * q.sigma_r * q.sigma_r * q.sigma_zw / (double)nw : 0.0;
  const bool drive = j < c.n_drive;
  const double z = nm[4 * c.n + j];
  const double x = q.sigma_r * nm[j], y = q.sigma_r * nm[c.n + j];
  const double xi = drive ? q.xi_d + szd * z : q.xi_d + delay + q.sigma_zw * z;
  int b = -1;
  double w = wd;
  if (!drive) {
    b = (int)floor((z + 3.0) * c.nbins / 6.0);
    b = b < 0 ? 0 : (b > c.nbins - 1 ? c.nbins - 1 : b);
    w = ww * (c.nbins > 0 ? profile[b] : 1.0);
  }
  s.x[j] = x;
  s.y[j] = y;
  s.ux[j] = su * nm[2 * c.n + j];
  s.uy[j] = su * nm[3 * c.n + j];
  s.uz[j] = c.gamma_b;
  s.xi[j] = xi;
  s.lost[j] = (xi >= 0.0 && xi < c.b.ximax && sqrt(x * x + y * y) < c.b.rmax) ? 0 : 1;
  wgt[j] = w;
  bin[j] = b;
}

// Raw bilinear deposit of particle j's weight on the (r, xi) nodes.
ADJ_HD inline void deposit_one(const BeamConst &c, const Beam &s, const double *wgt, double *nb, int64_t j) {
  if (s.lost[j]) return;
  const int n1 = c.b.nr + 1;
  int cr, k;
  double f, gx;
  cell_rz(c.b, sqrt(s.x[j] * s.x[j] + s.y[j] * s.y[j]), s.xi[j], cr, f, k, gx);
  double *row = nb + (size_t)k * n1 + cr;
  const double w = wgt[j];
  add_to(row, w * (1.0 - f) * (1.0 - gx));
  add_to(row + 1, w * f * (1.0 - gx));
  add_to(row + n1, w * (1.0 - f) * gx);
  add_to(row + n1 + 1, w * f * gx);
}

// 1 / (hat volume) of node (k, i): V_i in r, dxi in xi (dxi/2 at both ends).
ADJ_HD inline double node_scale(const BoundsRZ &b, int k, int i) {
  const double vx = (k == 0 || k == b.nxi) ? 0.5 * b.dxi : b.dxi;
  return 1.0 / (vol(i, b.nr, b.dr) * vx);
}

ADJ_HD inline void gather3(const BoundsRZ &b, const double *er, const double *ez, const double *bt, int c, double f,
                           int k, double gx, double &Er, double &Ez, double &Bt) {
  const int n1 = b.nr + 1;
  const size_t i0 = (size_t)k * n1 + c;
  const double a00 = (1.0 - f) * (1.0 - gx), a01 = f * (1.0 - gx), a10 = (1.0 - f) * gx, a11 = f * gx;
  Er = a00 * er[i0] + a01 * er[i0 + 1] + a10 * er[i0 + n1] + a11 * er[i0 + n1 + 1];
  Ez = a00 * ez[i0] + a01 * ez[i0 + 1] + a10 * ez[i0 + n1] + a11 * ez[i0 + n1 + 1];
  Bt = a00 * bt[i0] + a01 * bt[i0 + 1] + a10 * bt[i0 + n1] + a11 * bt[i0 + n1 + 1];
}

// Particle j from state s0 to s1: gather, Boris step, lost check.
ADJ_HD inline void push_one(const BeamConst &c, const Beam &s0, Beam s1, const double *er, const double *ez,
                            const double *bt, int64_t j) {
  double x = rd(s0.x + j), y = rd(s0.y + j), ux = rd(s0.ux + j), uy = rd(s0.uy + j), uz = rd(s0.uz + j), xi = rd(s0.xi + j);
  uint8_t lost = rd(s0.lost + j);
  if (!lost) {
    int cr, k;
    double f, gx, Er, Ez, Bt;
    cell_rz(c.b, sqrt(x * x + y * y), xi, cr, f, k, gx);
    gather3(c.b, er, ez, bt, cr, f, k, gx, Er, Ez, Bt);
    boris(x, y, ux, uy, uz, xi, Er, Ez, Bt, c.dt);
    if (!(xi >= 0.0 && xi < c.b.ximax && sqrt(x * x + y * y) < c.b.rmax)) lost = 1;
  }
  s1.x[j] = x;
  s1.y[j] = y;
  s1.ux[j] = ux;
  s1.uy[j] = uy;
  s1.uz[j] = uz;
  s1.xi[j] = xi;
  s1.lost[j] = lost;
}

// Witness sums of particle j: v[0] += w, v[1] += w g, v[2] += w g^2, g = gamma - gamma_b.
ADJ_HD inline void loss_one(const BeamConst &c, const Beam &s, const double *wgt, int64_t j, double *v) {
  if (j < c.n_drive || s.lost[j]) return;
  const double gm = sqrt(1.0 + s.ux[j] * s.ux[j] + s.uy[j] * s.uy[j] + s.uz[j] * s.uz[j]) - c.gamma_b;
  v[0] += wgt[j];
  v[1] += wgt[j] * gm;
  v[2] += wgt[j] * gm * gm;
}

// Seed of the reverse pass for particle j: L = d0 mean + d1 rms, mean = S1/W,
// rms = sqrt(S2/W - mean^2), over the surviving witness particles.
ADJ_HD inline void loss_reverse_one(const BeamConst &c, const Beam &s, const double *wgt, const double *sums, double d0,
                                    double d1, Beam lam, double *lw, int64_t j) {
  const double W = sums[0], M = sums[1] / W, var0 = sums[2] / W - M * M, var = var0 > 0.0 ? var0 : 0.0,
               sd = sqrt(var);
  lam.x[j] = lam.y[j] = lam.ux[j] = lam.uy[j] = lam.uz[j] = lam.xi[j] = 0.0;
  lw[j] = 0.0;
  if (j < c.n_drive || s.lost[j] || !(W > 0.0)) return;
  const double gam = sqrt(1.0 + s.ux[j] * s.ux[j] + s.uy[j] * s.uy[j] + s.uz[j] * s.uz[j]);
  const double gm = gam - c.gamma_b, wj = wgt[j];
  double lg = d0 * wj / W;
  double lwj = d0 * (gm - M) / W;
  if (sd > 0.0) {
    lg += d1 * wj * (gm - M) / (W * sd);
    lwj += d1 * ((gm - M) * (gm - M) - var) / (2.0 * W * sd);
  }
  lam.ux[j] = lg * s.ux[j] / gam;
  lam.uy[j] = lg * s.uy[j] / gam;
  lam.uz[j] = lg * s.uz[j] / gam;
  lw[j] = lwj;
}

// Reverse of particle j's push: lam holds the adjoint of state t+1 and becomes that of state t;
// the field adjoints go onto the grids (bilinear, transposed).
ADJ_HD inline void push_reverse_one(const BeamConst &c, const Beam &s0, const double *er, const double *ez,
                                    const double *bt, Beam lam, double *ler, double *lez, double *lbt, int64_t j) {
  if (s0.lost[j]) return;
  const int n1 = c.b.nr + 1;
  const double x = s0.x[j], y = s0.y[j], xi = s0.xi[j];
  const double r = sqrt(x * x + y * y);
  int cr, k;
  double f, gx, Er, Ez, Bt;
  cell_rz(c.b, r, xi, cr, f, k, gx);
  gather3(c.b, er, ez, bt, cr, f, k, gx, Er, Ez, Bt);
  double lx = rd(lam.x + j), ly = rd(lam.y + j), lux = rd(lam.ux + j), luy = rd(lam.uy + j), luz = rd(lam.uz + j),
         lxi = rd(lam.xi + j);
  double lEr = 0.0, lEz = 0.0, lBt = 0.0;
  boris_reverse(x, y, s0.ux[j], s0.uy[j], s0.uz[j], Er, Ez, Bt, c.dt, lx, ly, lux, luy, luz, lxi, lEr, lEz, lBt);
  const size_t i0 = (size_t)k * n1 + cr;
  const double a00 = (1.0 - f) * (1.0 - gx), a01 = f * (1.0 - gx), a10 = (1.0 - f) * gx, a11 = f * gx;
  add_to(&ler[i0], lEr * a00);
  add_to(&ler[i0 + 1], lEr * a01);
  add_to(&ler[i0 + n1], lEr * a10);
  add_to(&ler[i0 + n1 + 1], lEr * a11);
  add_to(&lez[i0], lEz * a00);
  add_to(&lez[i0 + 1], lEz * a01);
  add_to(&lez[i0 + n1], lEz * a10);
  add_to(&lez[i0 + n1 + 1], lEz * a11);
  add_to(&lbt[i0], lBt * a00);
  add_to(&lbt[i0 + 1], lBt * a01);
  add_to(&lbt[i0 + n1], lBt * a10);
  add_to(&lbt[i0 + n1 + 1], lBt * a11);
  // the gather's weights move with the particle: d/df and d/dg of the bilinear form
  double lf = 0.0, lg = 0.0;
  const double *vs[3] = {er, ez, bt};
  const double ls[3] = {lEr, lEz, lBt};
  for (int q = 0; q < 3; ++q) {
    const double *v = vs[q];
    lf += ls[q] * ((1.0 - gx) * (v[i0 + 1] - v[i0]) + gx * (v[i0 + n1 + 1] - v[i0 + n1]));
    lg += ls[q] * ((1.0 - f) * (v[i0 + n1] - v[i0]) + f * (v[i0 + n1 + 1] - v[i0 + 1]));
  }
  if (r > 0.0) {
    lx += lf / c.b.dr * x / r;
    ly += lf / c.b.dr * y / r;
  }
  lxi += lg / c.b.dxi;
  lam.x[j] = lx;
  lam.y[j] = ly;
  lam.ux[j] = lux;
  lam.uy[j] = luy;
  lam.uz[j] = luz;
  lam.xi[j] = lxi;
}

// Reverse of particle j's deposit at step t: the density adjoint lnb -> its position and weight.
ADJ_HD inline void deposit_reverse_one(const BeamConst &c, const Beam &s, const double *wgt, const double *lnb,
                                       Beam lam, double *lw, int64_t j) {
  if (s.lost[j]) return;
  const int n1 = c.b.nr + 1;
  const double x = s.x[j], y = s.y[j], r = sqrt(x * x + y * y);
  int cr, k;
  double f, gx;
  cell_rz(c.b, r, s.xi[j], cr, f, k, gx);
  const size_t i0 = (size_t)k * n1 + cr;
  const double L00 = lnb[i0] * node_scale(c.b, k, cr), L01 = lnb[i0 + 1] * node_scale(c.b, k, cr + 1),
               L10 = lnb[i0 + n1] * node_scale(c.b, k + 1, cr),
               L11 = lnb[i0 + n1 + 1] * node_scale(c.b, k + 1, cr + 1);
  const double w = wgt[j];
  lw[j] = rd(lw + j) + (L00 * (1.0 - f) * (1.0 - gx) + L01 * f * (1.0 - gx) + L10 * (1.0 - f) * gx + L11 * f * gx);
  const double lf = w * ((1.0 - gx) * (L01 - L00) + gx * (L11 - L10));
  const double lg = w * ((1.0 - f) * (L10 - L00) + f * (L11 - L01));
  if (r > 0.0) {
    lam.x[j] = rd(lam.x + j) + lf / c.b.dr * x / r;
    lam.y[j] = rd(lam.y + j) + lf / c.b.dr * y / r;
  }
  lam.xi[j] = rd(lam.xi + j) + lg / c.b.dxi;
}

// deposit_one with the division by the hats' volumes folded in (node_scale per node): the
// normalised density in one pass, for the pipelined steps that deposit into the next step's
// grid as each cell of the beam is pushed.
ADJ_HD inline void deposit_scaled_one(const BeamConst &c, const Beam &s, const double *wgt, double *nb, int64_t j) {
  if (s.lost[j]) return;
  const int n1 = c.b.nr + 1;
  int cr, k;
  double f, gx;
  cell_rz(c.b, sqrt(s.x[j] * s.x[j] + s.y[j] * s.y[j]), s.xi[j], cr, f, k, gx);
  double *row = nb + (size_t)k * n1 + cr;
  const double w = wgt[j];
  add_to(row, w * (1.0 - f) * (1.0 - gx) * node_scale(c.b, k, cr));
  add_to(row + 1, w * f * (1.0 - gx) * node_scale(c.b, k, cr + 1));
  add_to(row + n1, w * (1.0 - f) * gx * node_scale(c.b, k + 1, cr));
  add_to(row + n1 + 1, w * f * gx * node_scale(c.b, k + 1, cr + 1));
}

// Initial plasma slice, ring j (Sec. II.A, warm Maxwellian): cell c = j / ppc holds ppc/2
// radii, each shared by a mirrored pair of draws; u = u_th n, gamma0 = sqrt(1 + u^2),
// Gamma0 = gamma0 - u_z, l = r u_theta, w = r dr/ppc (Gamma0/gamma0) (the flux factor 1 - v_z0).
ADJ_HD inline void plasma_init_one(int ppc, double dr, double u_th, const double *nm, double *r0, double *ur0,
                                   double *l, double *G0, double *w, int j) {
  const int c = j / ppc, m = j % ppc;
  const double r = ((double)c + ((double)(m / 2) + 0.5) / (double)(ppc / 2)) * dr;
  const double ur = u_th * nm[3 * j], ut = u_th * nm[3 * j + 1], uz = u_th * nm[3 * j + 2];
  const double g0 = sqrt(1.0 + ur * ur + ut * ut + uz * uz);
  r0[j] = r;
  ur0[j] = ur;
  l[j] = r * ut;
  G0[j] = g0 - uz;
  w[j] = r * dr / (double)ppc * ((g0 - uz) / g0);
}

// Ion charge at node i: the deposit of the unperturbed rings.
ADJ_HD inline double rho0_node(const Dims &g, const double *r0, const double *w, int i) {
  double s = 0.0;
  for (int j = 0; j < g.np; ++j) {
    int c;
    double f;
    cell_of(r0[j], g.dr, g.nr, c, f);
    if (c == i) s += w[j] * (1.0 - f);
    if (c + 1 == i) s += w[j] * f;
  }
  return s;
}

// Contributions of beam particle j to the gradient: g4[0] n_w, g4[1] delay, g4[2] sigma_zd
// (the profile bin's share is returned in *gbin).  wu_w: witness weight per unit n_w and
// unit multiplier; wu_d: drive weight per unit sigma_zd.
ADJ_HD inline void theta_beam_one(const BeamConst &c, const double *nm_b, const int *bin, const Beam &lam0,
                                  const double *lwb, const double *theta, const double *profile, double wu_w,
                                  double wu_d, int64_t j, double *g4, double *gbin) {
  *gbin = 0.0;
  if (j < c.n_drive) {
    g4[2] += lam0.xi[j] * nm_b[4 * c.n + j] + lwb[j] * wu_d;
  } else {
    const double m = c.nbins > 0 ? profile[bin[j]] : 1.0;
    g4[0] += lwb[j] * wu_w * m;
    g4[1] += lam0.xi[j];
    *gbin = lwb[j] * wu_w * theta[0];
  }
}

// Contribution of plasma ring j to d/du_th: u = u_th n, gamma0 = sqrt(1 + u^2),
// G0 = gamma0 - u_z, l = r0 u_theta, u_r0 = u_th n_r, w = r0 dr/ppc G0/gamma0 (the ion charge
// rho0 carries w too).
ADJ_HD inline double theta_ring_one(const Dims &g, const double *nm_p, const double *r0, const double *lrho0,
                                    const double *lG0, const double *lw_p, const double *ll, const double *lur0,
                                    double u_th, int ppc, int j) {
  const double nr_ = nm_p[3 * j], nt = nm_p[3 * j + 1], nz = nm_p[3 * j + 2];
  const double n2 = nr_ * nr_ + nt * nt + nz * nz, g0 = sqrt(1.0 + u_th * u_th * n2);
  const double G0 = g0 - u_th * nz;
  const double dg0 = u_th * n2 / g0, dG0 = dg0 - nz;
  const double base = r0[j] * g.dr / (double)ppc;
  const double dw = base * (dG0 * g0 - G0 * dg0) / (g0 * g0);
  int cc;
  double f;
  cell_of(r0[j], g.dr, g.nr, cc, f);
  const double lwj = lw_p[j] + lrho0[cc] * (1.0 - f) + lrho0[cc + 1] * f;
  return lur0[j] * nr_ + ll[j] * r0[j] * nt + lG0[j] * dG0 + lwj * dw;
}

}  // namespace adj
}  // namespace wake
