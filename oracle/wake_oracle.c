/*
 * wake_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the quasi-static (QS)
 * r-xi plasma-wakefield method of Jain, Palastro, Antonsen, Mori & An, "Plasma wakefield
 * acceleration studies using the quasi-static code WAKE" (arXiv:1411.3246).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load this library.  It shares no code, header or constant with the CUDA
 * path; the only thing both sides see is the arrays of standard normals that the seeded
 * input module draws.
 *
 * Units: lengths k_p^-1, time omega_p^-1, momenta u = p/(m c), potentials m c^2/e, fields
 * E_0 = m c omega_p / e, densities n_p, currents e n_p c.  Plasma and beam electrons have
 * charge -1 and mass 1; the ions are immobile with density 1.  All radial "volumes" and
 * weights are per 2*pi (a ring of radius r and width dr has volume r dr).
 *
 * What the paper fixes (Sec. II.A):
 *   Eq. 1   gamma - u_z + q psi = gamma_0 - u_z0, i.e. for q = -1
 *           Gamma := gamma - u_z = Gamma_0 + psi, Gamma_0 = gamma_0 - u_z0.
 *   Eq. 2-3 gamma = (1 + u_perp^2 + Gamma^2) / (2 Gamma),  u_z = (1 + u_perp^2 - Gamma^2)/(2 Gamma).
 *   p_theta = l_z / r (l_z conserved).
 *   Eq. 4   du_r/dxi = (gamma/Gamma) dpsi/dr + u_theta^2/(Gamma r) - B_theta.
 *   Eq. 5   dr/dxi = u_r / Gamma.
 *   Eq. 6   (1/r) d_r (r B_theta) = d_xi^2 psi + J_z.
 *   Eq. 7   d_xi d_r psi = J_r.
 *   Eq. 8-11 beam: Lorentz force of E = (E_r, E_z), B = B_theta in t; d xi/dt = 1 - v_z.
 *   Eq. 12  two-bunch bi-Gaussian driver density.
 * What the paper leaves open is read as follows (the same reading as the CUDA path):
 *   - node-centred grid r_i = i dr (i = 0..nr), xi_k = k dxi (k = 0..nxi);
 *   - linear-hat radial deposit divided by the hats' ring volumes V_0 = dr^2/6,
 *     V_i = r_i dr, V_nr = dr (r_nr/2 - dr/6); the ion background is the deposit of the
 *     unperturbed electrons;
 *   - psi from Gauss minus Ampere-z, lap_perp psi = n_e (1 - v_z) - 1, in flux form with
 *     psi(R) = 0 (conducting wall); E_z = d_xi psi from Eq. 7 with the radial current of
 *     each cell; B_theta from Eq. 6 differentiated in r, with d_xi J_r expanded by Eqs. 4-5
 *     (a Helmholtz equation whose shift is chi = n/gamma);
 *   - RK2 (midpoint) in xi, the transverse motion integrated in a local Cartesian frame
 *     (which carries the u_theta^2/(Gamma r) term of Eq. 4 exactly), l_z re-imposed after
 *     each step, specular reflection at r = R;
 *   - Boris push for the beam (Eqs. 8-11), d xi/dt written without cancellation.
 * Slab geometry (geometry = 1; Sec. I: WAKE handles slab as well as cylindrical geometry) is
 * read as the same model with d/dy = 0 in place of d/dtheta = 0: r becomes x >= 0 with the
 * plane x = 0 a mirror plane (psi even, E_x and B_y odd), volumes per unit area (hats of
 * width dx, halved at x = 0 and at the wall), lap_perp = d_x^2 and (1/r) d_r(r .) = d_x, the
 * conserved transverse momentum u_y (in place of l_z) entering gamma only, so Eq. 4 loses its
 * centrifugal term; a sheet that crosses x = 0 is replaced by its mirror image (x, u_x) ->
 * (-x, -u_x).  The beam is a sheet beam at y = 0 (u_y = 0), its density folded onto x >= 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENUMERIC (-4)
#define ORC_EESCAPE (-6)

typedef struct {
  int32_t nr, nxi, ppc, pad0;
  double rmax, ximax, u_th;
  double n_d, n_w, sigma_r, sigma_zd, sigma_zw, xi_d, xi_w;
  double gamma_b, eps_n, ds;
  int64_t n_beam, n_drive;
  int32_t geometry, pad1; /* 0: cylindrical (r, xi); 1: slab (x, xi) */
} orc_params;

#define ORC_SLAB(p) ((p)->geometry == 1)

/* ------------------------------------------------------------------------------------ */
/* Grid helpers                                                                           */
/* ------------------------------------------------------------------------------------ */

/* Ring volume (per 2 pi) of the linear hat centred on node i: int hat_i(r) r dr.  Slab: the
 * hat's width on x >= 0, dx (dx/2 at x = 0 and at the wall). */
static double node_volume(int i, int nr, double dr, int slab) {
  if (slab) return (i == 0 || i == nr) ? 0.5 * dr : dr;
  if (i == 0) return dr * dr / 6.0;
  if (i == nr) return dr * ((double)nr * dr / 2.0 - dr / 6.0);
  return (double)i * dr * dr;
}

/* Fraction of hat m's ring volume that lies inside r_m: alpha_m = 1/2 - 1/(6m) for
 * 1 <= m < nr, 1 at the wall node (its hat has no outer half).  Slab: 1/2, 1 at the wall. */
static double node_alpha(int m, int nr, int slab) {
  if (m == nr) return 1.0;
  if (slab) return 0.5;
  return 0.5 - 1.0 / (6.0 * (double)m);
}

/* The metric of Gauss's law at node m (1/r_m; slab 1) and the curvature of (1/r) d_r(r .)
 * (1/r_m; slab 0). */
static double node_metric(int m, double dr, int slab) { return slab ? 1.0 : 1.0 / (m * dr); }
static double node_curv(int m, double dr, int slab) { return slab ? 0.0 : 1.0 / (m * dr); }

/* Cell index c (0..nr-1) and fractional offset f in [0,1] of radius r. */
static void locate(double r, double dr, int nr, int *c, double *f) {
  double s = r / dr;
  int i = (int)floor(s);
  if (i < 0) i = 0;
  if (i > nr - 1) i = nr - 1;
  *c = i;
  *f = s - (double)i;
}

static double interp(const double *v, double r, double dr, int nr) {
  int c;
  double f;
  locate(r, dr, nr, &c, &f);
  return (1.0 - f) * v[c] + f * v[c + 1];
}

/* ------------------------------------------------------------------------------------ */
/* Eqs. 2-3: gamma and u_z from the QS invariant                                          */
/* ------------------------------------------------------------------------------------ */

void orc_gamma_uz(double uperp2, double Gam, double *gamma, double *uz) {
  *gamma = (1.0 + uperp2 + Gam * Gam) / (2.0 * Gam);
  *uz = (1.0 + uperp2 - Gam * Gam) / (2.0 * Gam);
}

/* ------------------------------------------------------------------------------------ */
/* Plasma initial slice (Sec. II.A, warm plasma with Maxwellian momenta)                  */
/* ------------------------------------------------------------------------------------ */

/* Particle j = c*ppc + m of cell c.  Cold plasma: ppc rings at r0 = (c + (m+1/2)/ppc) dr.
 * Warm plasma: ppc/2 ring positions per cell, each used by a mirrored pair of draws.
 * Ring weight (per 2 pi) w = r0 dr / ppc times the QS flux factor 1 - v_z0 = Gamma0/gamma0
 * (a QS macroparticle carries the flux of electrons through a xi = const plane).
 * u = u_th * normals; gamma0 = sqrt(1 + u^2); Gamma0 = gamma0 - u_z0; l = r0 u_theta0.
 * Slab: sheets with w = dx / ppc times the flux factor and l = u_y0 (conserved). */
int orc_plasma_init(const orc_params *p, const double *normals, double *r0, double *ur0,
                    double *l, double *G0, double *w) {
  const int nr = p->nr, ppc = p->ppc;
  const double dr = p->rmax / nr;
  const int warm = (p->u_th != 0.0), slab = ORC_SLAB(p);
  if (nr < 2 || ppc < 1 || (warm && (ppc % 2 != 0 || normals == NULL))) return ORC_EINVAL;
  for (int c = 0; c < nr; ++c) {
    for (int m = 0; m < ppc; ++m) {
      const int j = c * ppc + m;
      double r;
      if (warm)
        r = ((double)c + ((double)(m / 2) + 0.5) / (double)(ppc / 2)) * dr;
      else
        r = ((double)c + ((double)m + 0.5) / (double)ppc) * dr;
      double ur = 0.0, ut = 0.0, uz = 0.0;
      if (warm) {
        ur = p->u_th * normals[3 * j + 0];
        ut = p->u_th * normals[3 * j + 1];
        uz = p->u_th * normals[3 * j + 2];
      }
      const double g0 = sqrt(1.0 + ur * ur + ut * ut + uz * uz);
      r0[j] = r;
      ur0[j] = ur;
      l[j] = slab ? ut : r * ut;
      G0[j] = g0 - uz;
      w[j] = (slab ? dr : r * dr) / (double)ppc * ((g0 - uz) / g0);
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Eq. 12: two-bunch driver density on the nodes (frozen analytic driver)                 */
/* ------------------------------------------------------------------------------------ */

double orc_nb_eq12(const orc_params *p, double r, double xi) {
  double radial = exp(-r * r / (2.0 * p->sigma_r * p->sigma_r));
  double ad = (xi - p->xi_d) / p->sigma_zd;
  double lon = p->n_d * exp(-0.5 * ad * ad);
  if (p->n_w != 0.0) {
    double aw = (xi - p->xi_w) / p->sigma_zw;
    lon += p->n_w * exp(-0.5 * aw * aw);
  }
  return radial * lon;
}

void orc_nb_analytic(const orc_params *p, double *nb) {
  const int nr = p->nr, nxi = p->nxi;
  const double dr = p->rmax / nr, dxi = p->ximax / nxi;
  for (int k = 0; k <= nxi; ++k)
    for (int i = 0; i <= nr; ++i) nb[(size_t)k * (nr + 1) + i] = orc_nb_eq12(p, i * dr, k * dxi);
}

/* ------------------------------------------------------------------------------------ */
/* Tridiagonal solve (Thomas algorithm): a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i       */
/* ------------------------------------------------------------------------------------ */

int orc_tridiag(int n, const double *a, const double *b, const double *c, const double *d,
                double *x) {
  double *cp = (double *)malloc(sizeof(double) * n);
  double *dp = (double *)malloc(sizeof(double) * n);
  if (!cp || !dp) {
    free(cp);
    free(dp);
    return ORC_ENOMEM;
  }
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int i = 1; i < n; ++i) {
    double m = b[i] - a[i] * cp[i - 1];
    cp[i] = c[i] / m;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* One slice: deposit (Sec. II.A sources) and radial field solves (Eqs. 6-7)             */
/* ------------------------------------------------------------------------------------ */

/* Node arrays written by orc_solve_slice, each (nr+1) long, at out + SL_x * (nr+1). */
enum {
  SL_PSI = 0, /* psi                                                   */
  SL_DPSI,    /* d psi / dr at the nodes                               */
  SL_EZ,      /* E_z = d_xi psi                                        */
  SL_BTH,     /* B_theta                                               */
  SL_ER,      /* E_r = B_theta - d psi/dr                              */
  SL_RHO,     /* raw charge deposit sum_j w_j hat_i(r_j) (electrons)   */
  SL_JZ,      /* total J_z = J_z,plasma + J_z,beam                     */
  SL_CHI,     /* chi = n/gamma = D[w/Gamma]                            */
  SL_T,       /* T = D[w a^2], a = u_r/Gamma                           */
  SL_Q,       /* Q (Helmholtz source from d_xi J_r)                    */
  SL_KCELL,   /* per-cell radial current sum_{j in cell} w_j a_j       */
  SL_COUNT
};

/*
 * Field solve for one slice, given the plasma rings (r_j, u_rj, u_thetaj, Gamma0_j, w_j),
 * the raw ion charge rho0 (deposit of the unperturbed electrons) and the beam density nb on
 * the nodes of this slice.
 *
 *  psi:  Gauss minus Ampere-z gives lap_perp psi = n_e (1 - v_z) - 1 (the beam's own
 *        rho_b - J_zb = -n_b (1 - v_b) is dropped).  Flux form on the node cells:
 *        r_{i+1/2} (psi_{i+1} - psi_i)/dr = Phi_i = sum_{i'<=i} (rho_i' - rho0_i'),
 *        psi(R) = 0.  This is an exact discrete Gauss law.
 *  E_z:  Eq. 7 with E_z = d_xi psi:  d_r E_z = J_r, E_z(R) = 0.  The radial current of
 *        cell c, J_r,c+1/2 = -(sum_{j in c} w_j u_rj/Gamma_j)/(r_{c+1/2} dr), makes E_z the
 *        exact xi-derivative of the discrete psi for continuously moving rings.
 *  B_th: Eq. 6 differentiated in r, with Eq. 7 for d_xi E_z:
 *          d_r[(1/r) d_r(r B)] = d_r J_z + d_xi J_r,
 *        and d_xi J_r expanded with Eqs. 4-5 along the ring trajectories:
 *          d_xi J_r = chi B + Q + (1/r) d_r(r T),
 *          chi = D[w/Gamma], T = D[w a^2],
 *          Q = D[w (a^2 psi' - F0)/Gamma] + E_z D[w a/Gamma],
 *          F0 = (gamma/Gamma) psi' + u_theta^2/(Gamma r)   (Eq. 4 without -B),
 *          using d Gamma/dxi = E_z + a psi' (Eq. 1).
 *        So (d_r (1/r) d_r r - chi) B = d_r J_z + Q + (1/r) d_r (r T), with B(0) = 0 and
 *        (1/r) d_r(r B) = J_z at r = R (there E_z = 0 for all xi).  Central differences on
 *        the nodes, a half cell at the wall; diagonally dominant, solved by Thomas.
 *  E_r = B_theta - d psi/dr (the paper's E_r - B_theta = -d_r psi, Fig. 7).
 *  Slab (x, xi): psi'_m = Phi_m, d_xi psi'_m = -((1 - alpha_m) K_{m-1} + alpha_m K_m)/dx,
 *        and (d_x^2 - chi) B_y = d_x J_z + Q + d_x T with F0 = (gamma/Gamma) psi' (no
 *        centrifugal term), B_y(0) = 0 (odd) and d_x B_y = J_z at the wall.
 *
 * Optional per-particle outputs: Gamma_j and the Cartesian radial force
 * Fc_j = (gamma/Gamma) psi'(r_j) - B(r_j) (Eq. 4 without its centrifugal term).
 * Returns ORC_ENUMERIC if any Gamma <= 0 or a value is not finite.
 */
int orc_solve_slice(const orc_params *p, int np, const double *r, const double *ur,
                    const double *ut, const double *G0, const double *w, const double *rho0,
                    const double *nb, double *out, double *Gam_out, double *Fc_out) {
  const int nr = p->nr, n1 = nr + 1, slab = ORC_SLAB(p);
  const double dr = p->rmax / nr;
  double *psi = out + SL_PSI * n1, *dpsi = out + SL_DPSI * n1, *ez = out + SL_EZ * n1;
  double *bth = out + SL_BTH * n1, *er = out + SL_ER * n1, *rho = out + SL_RHO * n1;
  double *jz = out + SL_JZ * n1, *chi = out + SL_CHI * n1, *T = out + SL_T * n1;
  double *Q = out + SL_Q * n1, *K = out + SL_KCELL * n1;
  double *P = (double *)calloc(n1, sizeof(double));
  double *U = (double *)calloc(n1, sizeof(double));
  double *Gp = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
  double *ga = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
  double *ta = (double *)malloc(sizeof(double) * n1);
  double *tb = (double *)malloc(sizeof(double) * n1);
  double *tc = (double *)malloc(sizeof(double) * n1);
  double *td = (double *)malloc(sizeof(double) * n1);
  double *dph = (double *)malloc(sizeof(double) * n1);
  int status = ORC_OK;
  if (!P || !U || !Gp || !ga || !ta || !tb || !tc || !td || !dph) {
    status = ORC_ENOMEM;
    goto done;
  }
  for (int i = 0; i < SL_COUNT * n1; ++i) out[i] = 0.0;

  /* electron charge deposit (linear hats) */
  for (int j = 0; j < np; ++j) {
    int c;
    double f;
    locate(r[j], dr, nr, &c, &f);
    rho[c] += w[j] * (1.0 - f);
    rho[c + 1] += w[j] * f;
  }
  /* psi: Gauss's law for the piecewise-linear density sum_i S_i hat_i(r) that the hat
   * deposit represents.  The enclosed charge at node m is
   *   Phi_m = sum_{i<m} (rho_i - rho0_i) + alpha_m (rho_m - rho0_m),
   *   alpha_m = (int_{r_{m-1}}^{r_m} hat_m r dr) / V_m  (= 1/2 - 1/(6m); 1 at the wall),
   * so psi'_m = Phi_m / r_m exactly for that density; psi(R) = 0 and psi is the inward
   * trapezoid sum of psi'. */
  {
    double C = 0.0;
    dpsi[0] = 0.0;
    for (int m = 1; m <= nr; ++m) {
      C += rho[m - 1] - rho0[m - 1];
      const double Phi = C + node_alpha(m, nr, slab) * (rho[m] - rho0[m]);
      dpsi[m] = Phi * node_metric(m, dr, slab);
    }
    psi[nr] = 0.0;
    for (int m = nr - 1; m >= 0; --m) psi[m] = psi[m + 1] - 0.5 * dr * (dpsi[m] + dpsi[m + 1]);
  }
  /* per-ring QS quantities (Eqs. 1-3) and the current-type deposits; a ring of zero weight (a
   * ring promoted to a beam particle by the trapping of orc_march_trap) takes no part */
  for (int j = 0; j < np; ++j) {
    if (w[j] == 0.0) {
      Gp[j] = 1.0;
      ga[j] = 1.0;
      continue;
    }
    const double Gam = G0[j] + interp(psi, r[j], dr, nr);
    if (!(Gam > 0.0)) {
      status = ORC_ENUMERIC;
      goto done;
    }
    const double up2 = ur[j] * ur[j] + ut[j] * ut[j];
    double gam, uz;
    orc_gamma_uz(up2, Gam, &gam, &uz);
    const double a = ur[j] / Gam;
    const double dp = interp(dpsi, r[j], dr, nr);
    const double cent = (!slab && r[j] > 0.0) ? ut[j] * ut[j] / (Gam * r[j]) : 0.0;
    const double F0 = (gam / Gam) * dp + cent;
    Gp[j] = Gam;
    ga[j] = gam;
    int c;
    double f;
    locate(r[j], dr, nr, &c, &f);
    const double wj = w[j];
    const double v_jz = -wj * uz / Gam;
    const double v_chi = wj / Gam;
    const double v_T = wj * a * a;
    const double v_P = wj * (a * a * dp - F0) / Gam;
    const double v_U = wj * a / Gam;
    jz[c] += v_jz * (1.0 - f);
    jz[c + 1] += v_jz * f;
    chi[c] += v_chi * (1.0 - f);
    chi[c + 1] += v_chi * f;
    T[c] += v_T * (1.0 - f);
    T[c + 1] += v_T * f;
    P[c] += v_P * (1.0 - f);
    P[c + 1] += v_P * f;
    U[c] += v_U * (1.0 - f);
    U[c + 1] += v_U * f;
    K[c] += wj * a;
  }
  for (int i = 0; i <= nr; ++i) {
    const double V = node_volume(i, nr, dr, slab);
    jz[i] = jz[i] / V - nb[i]; /* beam J_z = -n_b (v_b = c) */
    chi[i] /= V;
    T[i] /= V;
    P[i] /= V;
    U[i] /= V;
  }
  /* E_z = d_xi psi (Eq. 7): the hat deposit of a ring moving at dr/dxi = a changes by
   * d_xi rho_i = (K_{i-1} - K_i)/dr, K_c = sum_{j in cell c} w_j a_j, so
   *   d_xi Phi_m = -((1 - alpha_m) K_{m-1} + alpha_m K_m) / dr,
   * and E_z is the inward trapezoid sum of d_xi psi'_m = d_xi Phi_m / r_m from E_z(R) = 0:
   * the exact xi-derivative of the discrete psi for continuously moving rings. */
  {
    double *dez = dph; /* d_xi psi' at the nodes */
    dez[0] = 0.0;
    for (int m = 1; m <= nr; ++m) {
      const double al = node_alpha(m, nr, slab);
      const double Km = (m < nr) ? K[m] : 0.0;
      dez[m] = -((1.0 - al) * K[m - 1] + al * Km) / dr * node_metric(m, dr, slab);
    }
    ez[nr] = 0.0;
    for (int m = nr - 1; m >= 0; --m) ez[m] = ez[m + 1] - 0.5 * dr * (dez[m] + dez[m + 1]);
  }
  for (int i = 0; i <= nr; ++i) Q[i] = P[i] + ez[i] * U[i];

  /* B_theta: unknowns at nodes 1..nr (row q = i-1) */
  {
    const double idr2 = 1.0 / (dr * dr);
    for (int i = 1; i < nr; ++i) {
      const int q = i - 1;
      const double rm = (i - 0.5), rp = (i + 0.5);
      if (slab) { /* d_x^2 */
        ta[q] = idr2;
        tc[q] = idr2;
        tb[q] = -2.0 * idr2 - chi[i];
      } else {    /* d_r (1/r) d_r r */
        ta[q] = (i - 1) / rm * idr2;
        tc[q] = (i + 1) / rp * idr2;
        tb[q] = -(double)i * (1.0 / rp + 1.0 / rm) * idr2 - chi[i];
      }
      td[q] = (jz[i + 1] - jz[i - 1]) / (2.0 * dr) + Q[i] + (T[i + 1] - T[i - 1]) / (2.0 * dr) +
              T[i] * node_curv(i, dr, slab);
    }
    {
      const int i = nr, q = nr - 1;
      const double rm = (i - 0.5);
      ta[q] = slab ? 2.0 * idr2 : 2.0 * (i - 1) / rm * idr2;
      tc[q] = 0.0;
      tb[q] = (slab ? -2.0 * idr2 : -2.0 * (double)i / rm * idr2) - chi[i];
      td[q] = Q[i] + (T[i] - T[i - 1]) / dr + T[i] * node_curv(i, dr, slab) - (jz[i - 1] + jz[i]) / dr;
    }
    ta[0] = 0.0; /* B_0 = 0 */
    int s = orc_tridiag(nr, ta, tb, tc, td, bth + 1);
    if (s != ORC_OK) {
      status = s;
      goto done;
    }
    bth[0] = 0.0;
  }
  for (int i = 0; i <= nr; ++i) er[i] = bth[i] - dpsi[i];
  er[0] = 0.0;
  for (int i = 0; i < SL_COUNT * n1; ++i)
    if (!isfinite(out[i])) {
      status = ORC_ENUMERIC;
      goto done;
    }
  for (int j = 0; j < np; ++j) {
    const double dp = interp(dpsi, r[j], dr, nr);
    const double b = interp(bth, r[j], dr, nr);
    if (Gam_out) Gam_out[j] = Gp[j];
    if (Fc_out) Fc_out[j] = w[j] == 0.0 ? 0.0 : (ga[j] / Gp[j]) * dp - b;
  }
done:
  free(P);
  free(U);
  free(Gp);
  free(ga);
  free(ta);
  free(tb);
  free(tc);
  free(td);
  free(dph);
  return status;
}

/* Raw charge deposit of rings at radii r with weights w (the ion background rho0 is this
 * deposit evaluated on the unperturbed electrons). */
void orc_deposit_charge(const orc_params *p, int np, const double *r, const double *w,
                        double *rho) {
  const int nr = p->nr;
  const double dr = p->rmax / nr;
  for (int i = 0; i <= nr; ++i) rho[i] = 0.0;
  for (int j = 0; j < np; ++j) {
    int c;
    double f;
    locate(r[j], dr, nr, &c, &f);
    rho[c] += w[j] * (1.0 - f);
    rho[c + 1] += w[j] * f;
  }
}

/* ------------------------------------------------------------------------------------ */
/* The xi-march (Sec. II.A; the plasma is solved with the beam frozen, Sec. I)            */
/* ------------------------------------------------------------------------------------ */

/*
 * March the plasma through the box for a frozen beam density nb ((nxi+1) x (nr+1), slice
 * major).  Fields at node slices k = 0..nxi are written to psi, ez, er, bth (same layout,
 * any may be NULL).  Optional traj receives (r_j, u_rj, Gamma_j) at every slice:
 * traj[(k*3 + 0)*np + j] etc.
 *
 * One slice step is RK2 (midpoint) in xi.  Stage 1 solves the fields at xi_k with the rings
 * at their slice-k state and stores them; stage 2 solves at xi_k + dxi/2 with the rings at
 * the midpoint state and nb averaged over slices k and k+1.  Each ring is advanced in a local
 * Cartesian frame (x, y) = (r, 0), (u_x, u_y) = (u_r, u_theta):
 *     dx_perp/dxi = u_perp / Gamma,   du_perp/dxi = Fc rhat,
 * which is Eqs. 4-5 with the centrifugal term carried by the frame; afterwards
 * r = |x_perp|, u_r = x_perp . u_perp / r and u_theta = l / r.
 */
/*
 * orc_march with plasma-particle trapping (Sec. I: plasma particles that meet a threshold
 * condition are promoted to beam particles, which then follow the full equations of motion).
 * Reading (the paper cites the conditions to earlier work and gives none): a ring whose
 * stage-1 Gamma = gamma - u_z = Gamma_0 + psi (Eq. 1) at slice k is below gamma_t moves almost
 * with the wake (1 - v_z = Gamma/gamma) and leaves the quasi-static plasma there: it still
 * counts in slice k's fields, then its weight drops to zero and it no longer moves.  Each
 * promotion is recorded in trap[7 * t ..] = (ring j, slice k, r, u_r, u_theta, Gamma, w_j),
 * at most max_trap of them (*ntrap counts all).  gamma_t <= 0: no trapping (orc_march).
 */
int orc_march_trap(const orc_params *p, const double *r0, const double *ur0, const double *l,
                   const double *G0, const double *w_in, const double *nb, double gamma_t, double *psi,
                   double *ez, double *er, double *bth, double *traj, double *trap, int max_trap,
                   int *ntrap);
int orc_march(const orc_params *p, const double *r0, const double *ur0, const double *l,
              const double *G0, const double *w, const double *nb, double *psi, double *ez,
              double *er, double *bth, double *traj) {
  int nt = 0;
  return orc_march_trap(p, r0, ur0, l, G0, w, nb, 0.0, psi, ez, er, bth, traj, NULL, 0, &nt);
}
int orc_march_trap(const orc_params *p, const double *r0, const double *ur0, const double *l,
                   const double *G0, const double *w_in, const double *nb, double gamma_t, double *psi,
                   double *ez, double *er, double *bth, double *traj, double *trap, int max_trap,
                   int *ntrap) {
  const int nr = p->nr, nxi = p->nxi, n1 = nr + 1, slab = ORC_SLAB(p);
  const int np = p->nr * p->ppc;
  const double dr = p->rmax / nr, dxi = p->ximax / nxi, R = p->rmax;
  int status = ORC_OK;
  *ntrap = 0;
  if (slab && gamma_t > 0.0) return ORC_EINVAL; /* trapping is read for the cylinder only */
  double *r = (double *)malloc(sizeof(double) * np);
  double *ur = (double *)malloc(sizeof(double) * np);
  double *ut = (double *)malloc(sizeof(double) * np);
  double *rh = (double *)malloc(sizeof(double) * np);
  double *urh = (double *)malloc(sizeof(double) * np);
  double *uth = (double *)malloc(sizeof(double) * np);
  double *xh = (double *)malloc(sizeof(double) * np);
  double *yh = (double *)malloc(sizeof(double) * np);
  double *uxh = (double *)malloc(sizeof(double) * np);
  double *uyh = (double *)malloc(sizeof(double) * np);
  double *G1 = (double *)malloc(sizeof(double) * np);
  double *F1 = (double *)malloc(sizeof(double) * np);
  double *G2 = (double *)malloc(sizeof(double) * np);
  double *F2 = (double *)malloc(sizeof(double) * np);
  double *rho0 = (double *)malloc(sizeof(double) * n1);
  double *nbh = (double *)malloc(sizeof(double) * n1);
  double *sl = (double *)malloc(sizeof(double) * SL_COUNT * n1);
  double *w = (double *)malloc(sizeof(double) * np); /* weights; zero once a ring is promoted */
  if (!r || !ur || !ut || !rh || !urh || !uth || !xh || !yh || !uxh || !uyh || !G1 || !F1 ||
      !G2 || !F2 || !rho0 || !nbh || !sl || !w) {
    status = ORC_ENOMEM;
    goto done;
  }
  for (int j = 0; j < np; ++j) {
    r[j] = r0[j];
    ur[j] = ur0[j];
    w[j] = w_in[j];
  }
  orc_deposit_charge(p, np, r0, w, rho0);

  for (int k = 0; k <= nxi; ++k) {
    /* u_theta = l_z / r (slab: the conserved u_y) */
    for (int j = 0; j < np; ++j) ut[j] = slab ? l[j] : ((r[j] > 0.0) ? l[j] / r[j] : 0.0);
    /* stage 1 at xi_k */
    status = orc_solve_slice(p, np, r, ur, ut, G0, w, rho0, nb + (size_t)k * n1, sl, G1, F1);
    if (status != ORC_OK) goto done;
    if (psi) memcpy(psi + (size_t)k * n1, sl + SL_PSI * n1, sizeof(double) * n1);
    if (ez) memcpy(ez + (size_t)k * n1, sl + SL_EZ * n1, sizeof(double) * n1);
    if (er) memcpy(er + (size_t)k * n1, sl + SL_ER * n1, sizeof(double) * n1);
    if (bth) memcpy(bth + (size_t)k * n1, sl + SL_BTH * n1, sizeof(double) * n1);
    if (traj)
      for (int j = 0; j < np; ++j) {
        traj[((size_t)k * 3 + 0) * np + j] = r[j];
        traj[((size_t)k * 3 + 1) * np + j] = ur[j];
        traj[((size_t)k * 3 + 2) * np + j] = G1[j];
      }
    /* promotion of the rings that fell below the threshold at this slice */
    for (int j = 0; j < np; ++j)
      if (w[j] != 0.0 && G1[j] < gamma_t) {
        if (*ntrap < max_trap) {
          double *e = trap + 7 * (size_t)(*ntrap);
          e[0] = (double)j;
          e[1] = (double)k;
          e[2] = r[j];
          e[3] = ur[j];
          e[4] = ut[j];
          e[5] = G1[j];
          e[6] = w[j];
        }
        ++*ntrap;
        w[j] = 0.0;
      }
    if (k == nxi) break;

    /* midpoint state (a promoted ring stays where it is) */
    for (int j = 0; j < np; ++j) {
      if (w[j] == 0.0) {
        rh[j] = r[j];
        urh[j] = ur[j];
        uth[j] = ut[j];
        xh[j] = r[j];
        yh[j] = 0.0;
        uxh[j] = ur[j];
        uyh[j] = ut[j];
        continue;
      }
      /* the frame's y axis: the azimuth (cylinder); in the slab u_y moves nothing that matters
       * (d/dy = 0), so the frame is the x line and r = |x| mirrors a sheet that crosses x = 0 */
      const double uyf = slab ? 0.0 : ut[j];
      xh[j] = r[j] + 0.5 * dxi * ur[j] / G1[j];
      yh[j] = 0.5 * dxi * uyf / G1[j];
      uxh[j] = ur[j] + 0.5 * dxi * F1[j];
      uyh[j] = uyf;
      double rr = sqrt(xh[j] * xh[j] + yh[j] * yh[j]);
      double urr, utt;
      if (rr > 0.0) {
        urr = (xh[j] * uxh[j] + yh[j] * uyh[j]) / rr;
        utt = (xh[j] * uyh[j] - yh[j] * uxh[j]) / rr;
      } else {
        urr = sqrt(uxh[j] * uxh[j] + uyh[j] * uyh[j]);
        utt = 0.0;
      }
      if (rr > R) { /* specular reflection at the wall */
        rr = 2.0 * R - rr;
        urr = -urr;
      }
      if (!(rr >= 0.0 && rr <= R)) {
        status = ORC_EESCAPE;
        goto done;
      }
      rh[j] = rr;
      urh[j] = urr;
      uth[j] = slab ? l[j] : utt;
    }
    for (int i = 0; i < n1; ++i) nbh[i] = 0.5 * (nb[(size_t)k * n1 + i] + nb[(size_t)(k + 1) * n1 + i]);
    /* stage 2 at xi_k + dxi/2 */
    status = orc_solve_slice(p, np, rh, urh, uth, G0, w, rho0, nbh, sl, G2, F2);
    if (status != ORC_OK) goto done;
    /* full step */
    for (int j = 0; j < np; ++j) {
      if (w[j] == 0.0) continue;
      double ex = 1.0, ey = 0.0;
      const double rr = sqrt(xh[j] * xh[j] + yh[j] * yh[j]);
      if (rr > 0.0) {
        ex = xh[j] / rr;
        ey = yh[j] / rr;
      }
      const double xn = r[j] + dxi * uxh[j] / G2[j];
      const double yn = dxi * uyh[j] / G2[j];
      const double uxn = ur[j] + dxi * F2[j] * ex;
      const double uyn = (slab ? 0.0 : ut[j]) + dxi * F2[j] * ey;
      double rn = sqrt(xn * xn + yn * yn);
      double urn = (rn > 0.0) ? (xn * uxn + yn * uyn) / rn : sqrt(uxn * uxn + uyn * uyn);
      if (rn > R) {
        rn = 2.0 * R - rn;
        urn = -urn;
      }
      if (!(rn >= 0.0 && rn <= R) || !isfinite(urn)) {
        status = ORC_EESCAPE;
        goto done;
      }
      r[j] = rn;
      ur[j] = urn;
    }
  }
done:
  free(r);
  free(ur);
  free(ut);
  free(rh);
  free(urh);
  free(uth);
  free(xh);
  free(yh);
  free(uxh);
  free(uyh);
  free(G1);
  free(F1);
  free(G2);
  free(F2);
  free(rho0);
  free(nbh);
  free(sl);
  free(w);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Beam driver (Eq. 12 initial condition, Eqs. 8-11 push)                                 */
/* ------------------------------------------------------------------------------------ */

/* Macroparticle weights (per 2 pi) of the drive and witness bunches: the charge of the
 * Eq. 12 bunch, n sqrt(2 pi) sigma_r^2 sigma_z, over its macroparticle count. */
void orc_beam_weights(const orc_params *p, double *wd, double *ww) {
  const double s2pi = sqrt(2.0 * 3.14159265358979323846);
  const int64_t nw = p->n_beam - p->n_drive;
  /* transverse integral of exp(-r^2/2 sigma^2): r dr gives sigma^2; the slab's x >= 0 half,
   * on which the folded sheet beam lies, gives sigma sqrt(2 pi) / 2 */
  const double tr = ORC_SLAB(p) ? 0.5 * s2pi * p->sigma_r : p->sigma_r * p->sigma_r;
  *wd = (p->n_drive > 0) ? p->n_d * s2pi * tr * p->sigma_zd / (double)p->n_drive : 0.0;
  *ww = (nw > 0) ? p->n_w * s2pi * tr * p->sigma_zw / (double)nw : 0.0;
}

/* Beam state from normals (5 x n): x = sigma_r n0, y = sigma_r n1, u_x = (eps_n/sigma_r) n2,
 * u_y = (eps_n/sigma_r) n3, xi = xi_c + sigma_z n4 (drive: first n_drive), u_z = gamma_b.
 * Slab: a sheet beam, y = u_y = 0 (rows 1 and 3 unused).
 * A particle outside 0 <= xi < L or r >= R is marked lost. */
void orc_beam_init(const orc_params *p, const double *normals, double *x, double *y,
                   double *xi, double *ux, double *uy, double *uz, uint8_t *lost) {
  const int64_t n = p->n_beam;
  const double su = p->eps_n / p->sigma_r;
  for (int64_t j = 0; j < n; ++j) {
    const int drive = j < p->n_drive;
    const int slab = ORC_SLAB(p);
    x[j] = p->sigma_r * normals[0 * n + j];
    y[j] = slab ? 0.0 : p->sigma_r * normals[1 * n + j];
    ux[j] = su * normals[2 * n + j];
    uy[j] = slab ? 0.0 : su * normals[3 * n + j];
    xi[j] = drive ? p->xi_d + p->sigma_zd * normals[4 * n + j] : p->xi_w + p->sigma_zw * normals[4 * n + j];
    uz[j] = p->gamma_b;
    const double r = sqrt(x[j] * x[j] + y[j] * y[j]);
    lost[j] = !(xi[j] >= 0.0 && xi[j] < p->ximax && r < p->rmax);
  }
}

/* Beam density on the (nxi+1) x (nr+1) nodes: bilinear hats in (r, xi) divided by the hats'
 * volumes (V_i in r; dxi, or dxi/2 at the two end slices, in xi).  Lost particles skipped.
 * wmul (NULL: all 1) multiplies particle j's charge: a witness current profile other than
 * the Gaussian of Eq. 12 (Sec. IV studies the witness current). */
void orc_beam_deposit_w(const orc_params *p, const double *x, const double *y, const double *xi,
                        const uint8_t *lost, const double *wmul, double *nb);
void orc_beam_deposit(const orc_params *p, const double *x, const double *y, const double *xi,
                      const uint8_t *lost, double *nb) {
  orc_beam_deposit_w(p, x, y, xi, lost, NULL, nb);
}
void orc_beam_deposit_w(const orc_params *p, const double *x, const double *y, const double *xi,
                        const uint8_t *lost, const double *wmul, double *nb) {
  const int nr = p->nr, nxi = p->nxi, n1 = nr + 1;
  const double dr = p->rmax / nr, dxi = p->ximax / nxi;
  double wd, ww;
  orc_beam_weights(p, &wd, &ww);
  memset(nb, 0, sizeof(double) * (size_t)(nxi + 1) * n1);
  for (int64_t j = 0; j < p->n_beam; ++j) {
    if (lost[j]) continue;
    const double wj = (j < p->n_drive ? wd : ww) * (wmul ? wmul[j] : 1.0);
    const double r = sqrt(x[j] * x[j] + y[j] * y[j]);
    int c, k;
    double f, g;
    locate(r, dr, nr, &c, &f);
    locate(xi[j], dxi, nxi, &k, &g);
    nb[(size_t)k * n1 + c] += wj * (1 - f) * (1 - g);
    nb[(size_t)k * n1 + c + 1] += wj * f * (1 - g);
    nb[(size_t)(k + 1) * n1 + c] += wj * (1 - f) * g;
    nb[(size_t)(k + 1) * n1 + c + 1] += wj * f * g;
  }
  for (int k = 0; k <= nxi; ++k) {
    const double vx = (k == 0 || k == nxi) ? 0.5 * dxi : dxi;
    for (int i = 0; i <= nr; ++i) nb[(size_t)k * n1 + i] /= node_volume(i, nr, dr, ORC_SLAB(p)) * vx;
  }
}

/* One beam step of length dt = ds: Boris push (Boris 1970) of Eqs. 8-11 with charge -1 in
 * the lab-frame fields E = (E_r x/r, E_r y/r, E_z), B = (-B_theta y/r, B_theta x/r, 0),
 * gathered bilinearly in (r, xi).  Momentum lives at half steps.  Then
 * x_perp += dt u_perp/gamma and xi += dt (1 + u_perp^2)/(gamma (gamma + u_z)) (= dt (1 - v_z)).
 * A particle that leaves 0 <= xi < L or r < R is marked lost and no longer moves. */
void orc_beam_push(const orc_params *p, double *x, double *y, double *xi, double *ux,
                   double *uy, double *uz, uint8_t *lost, const double *er, const double *ez,
                   const double *bth) {
  const int nr = p->nr, nxi = p->nxi, n1 = nr + 1;
  const double dr = p->rmax / nr, dxi = p->ximax / nxi, dt = p->ds;
  for (int64_t j = 0; j < p->n_beam; ++j) {
    if (lost[j]) continue;
    const double r = sqrt(x[j] * x[j] + y[j] * y[j]);
    int c, k;
    double f, g;
    locate(r, dr, nr, &c, &f);
    locate(xi[j], dxi, nxi, &k, &g);
    const size_t i00 = (size_t)k * n1 + c, i01 = i00 + 1, i10 = i00 + n1, i11 = i10 + 1;
    const double w00 = (1 - f) * (1 - g), w01 = f * (1 - g), w10 = (1 - f) * g, w11 = f * g;
    const double Er = w00 * er[i00] + w01 * er[i01] + w10 * er[i10] + w11 * er[i11];
    const double Ez = w00 * ez[i00] + w01 * ez[i01] + w10 * ez[i10] + w11 * ez[i11];
    const double Bt = w00 * bth[i00] + w01 * bth[i01] + w10 * bth[i10] + w11 * bth[i11];
    const double cs = r > 0.0 ? x[j] / r : 0.0, sn = r > 0.0 ? y[j] / r : 0.0;
    const double Ex = Er * cs, Ey = Er * sn, Bx = -Bt * sn, By = Bt * cs;
    const double h = -0.5 * dt; /* q dt / 2 with q = -1 */
    double mx = ux[j] + h * Ex, my = uy[j] + h * Ey, mz = uz[j] + h * Ez;
    const double gm = sqrt(1.0 + mx * mx + my * my + mz * mz);
    const double tx = h * Bx / gm, ty = h * By / gm, tz = 0.0;
    const double px = mx + (my * tz - mz * ty), py = my + (mz * tx - mx * tz), pz = mz + (mx * ty - my * tx);
    const double s = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz);
    const double sx = s * tx, sy = s * ty, sz = s * tz;
    mx += py * sz - pz * sy;
    my += pz * sx - px * sz;
    mz += px * sy - py * sx;
    ux[j] = mx + h * Ex;
    uy[j] = my + h * Ey;
    uz[j] = mz + h * Ez;
    const double up2 = ux[j] * ux[j] + uy[j] * uy[j];
    const double gam = sqrt(1.0 + up2 + uz[j] * uz[j]);
    x[j] += dt * ux[j] / gam;
    y[j] += dt * uy[j] / gam;
    xi[j] += dt * (1.0 + up2) / (gam * (gam + uz[j]));
    const double rn = sqrt(x[j] * x[j] + y[j] * y[j]);
    if (!(xi[j] >= 0.0 && xi[j] < p->ximax && rn < p->rmax)) lost[j] = 1;
  }
}

/* Witness diagnostics (Sec. IV, energy gain and spread): out[0] surviving witness count,
 * out[1] mean gamma, out[2] rms gamma spread (absolute), out[3] surviving drive count,
 * out[4] drive mean gamma. */
void orc_diagnostics(const orc_params *p, const double *ux, const double *uy, const double *uz,
                     const uint8_t *lost, double *out) {
  double nw = 0, sw = 0, sw2 = 0, nd = 0, sd = 0;
  const double ref = p->gamma_b;
  for (int64_t j = 0; j < p->n_beam; ++j) {
    if (lost[j]) continue;
    const double g = sqrt(1.0 + ux[j] * ux[j] + uy[j] * uy[j] + uz[j] * uz[j]) - ref;
    if (j >= p->n_drive) {
      nw += 1;
      sw += g;
      sw2 += g * g;
    } else {
      nd += 1;
      sd += g;
    }
  }
  out[0] = nw;
  out[1] = nw > 0 ? ref + sw / nw : 0.0;
  out[2] = nw > 0 ? sqrt(fmax(sw2 / nw - (sw / nw) * (sw / nw), 0.0)) : 0.0;
  out[3] = nd;
  out[4] = nd > 0 ? ref + sd / nd : 0.0;
}

/* Witness observables weighted by charge (Sec. IV: mean energy gain and energy spread of the
 * witness): out[0] = sum w g / sum w, out[1] = sqrt(sum w (g - out[0])^2 / sum w) over the
 * surviving witness particles, g = gamma - gamma_b, w = wmul[j] (NULL: all 1). */
void orc_witness_obs(const orc_params *p, const double *ux, const double *uy, const double *uz,
                     const uint8_t *lost, const double *wmul, double *out) {
  double W = 0.0, S1 = 0.0;
  for (int64_t j = p->n_drive; j < p->n_beam; ++j) {
    if (lost[j]) continue;
    const double w = wmul ? wmul[j] : 1.0;
    W += w;
    S1 += w * (sqrt(1.0 + ux[j] * ux[j] + uy[j] * uy[j] + uz[j] * uz[j]) - p->gamma_b);
  }
  const double M = W > 0.0 ? S1 / W : 0.0;
  double S2 = 0.0;
  for (int64_t j = p->n_drive; j < p->n_beam; ++j) {
    if (lost[j]) continue;
    const double w = wmul ? wmul[j] : 1.0;
    const double d = sqrt(1.0 + ux[j] * ux[j] + uy[j] * uy[j] + uz[j] * uz[j]) - p->gamma_b - M;
    S2 += w * d * d;
  }
  out[0] = M;
  out[1] = W > 0.0 ? sqrt(S2 / W) : 0.0;
}

/* A full run (Sec. II.A, last paragraph): for each beam step, deposit the beam, march the
 * plasma with the beam frozen, then push the beam once.  Fields of the last march are left
 * in er, ez, bth, psi (any may be NULL).  orc_run_w takes per-particle charge multipliers
 * (orc_beam_deposit_w). */
int orc_run_w(const orc_params *p, int nsteps, const double *r0, const double *ur0,
              const double *l, const double *G0, const double *w, double *x, double *y,
              double *xi, double *ux, double *uy, double *uz, uint8_t *lost, const double *wmul,
              double *psi, double *ez, double *er, double *bth);
int orc_run(const orc_params *p, int nsteps, const double *r0, const double *ur0,
            const double *l, const double *G0, const double *w, double *x, double *y,
            double *xi, double *ux, double *uy, double *uz, uint8_t *lost, double *psi,
            double *ez, double *er, double *bth) {
  return orc_run_w(p, nsteps, r0, ur0, l, G0, w, x, y, xi, ux, uy, uz, lost, NULL, psi, ez, er, bth);
}
int orc_run_w(const orc_params *p, int nsteps, const double *r0, const double *ur0,
              const double *l, const double *G0, const double *w, double *x, double *y,
              double *xi, double *ux, double *uy, double *uz, uint8_t *lost, const double *wmul,
              double *psi, double *ez, double *er, double *bth) {
  const size_t ng = (size_t)(p->nxi + 1) * (p->nr + 1);
  double *nb = (double *)malloc(sizeof(double) * ng);
  double *fer = (double *)malloc(sizeof(double) * ng);
  double *fez = (double *)malloc(sizeof(double) * ng);
  double *fbt = (double *)malloc(sizeof(double) * ng);
  int status = ORC_OK;
  if (!nb || !fer || !fez || !fbt) {
    status = ORC_ENOMEM;
    goto done;
  }
  for (int s = 0; s < nsteps; ++s) {
    orc_beam_deposit_w(p, x, y, xi, lost, wmul, nb);
    status = orc_march(p, r0, ur0, l, G0, w, nb, psi, fez, fer, fbt, NULL);
    if (status != ORC_OK) goto done;
    orc_beam_push(p, x, y, xi, ux, uy, uz, lost, fer, fez, fbt);
  }
  if (ez) memcpy(ez, fez, sizeof(double) * ng);
  if (er) memcpy(er, fer, sizeof(double) * ng);
  if (bth) memcpy(bth, fbt, sizeof(double) * ng);
done:
  free(nb);
  free(fer);
  free(fez);
  free(fbt);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Trapping: promoted plasma particles as beam particles (Sec. I)                         */
/* ------------------------------------------------------------------------------------ */

/* Beam density with explicit per-particle weights (charge per 2 pi), for n particles: the
 * bilinear hats of orc_beam_deposit_w divided by the hats' volumes. */
void orc_beam_deposit_wt(const orc_params *p, int64_t n, const double *x, const double *y,
                         const double *xi, const uint8_t *lost, const double *wt, double *nb) {
  const int nr = p->nr, nxi = p->nxi, n1 = nr + 1;
  const double dr = p->rmax / nr, dxi = p->ximax / nxi;
  memset(nb, 0, sizeof(double) * (size_t)(nxi + 1) * n1);
  for (int64_t j = 0; j < n; ++j) {
    if (lost[j]) continue;
    const double r = sqrt(x[j] * x[j] + y[j] * y[j]);
    int c, k;
    double f, g;
    locate(r, dr, nr, &c, &f);
    locate(xi[j], dxi, nxi, &k, &g);
    nb[(size_t)k * n1 + c] += wt[j] * (1 - f) * (1 - g);
    nb[(size_t)k * n1 + c + 1] += wt[j] * f * (1 - g);
    nb[(size_t)(k + 1) * n1 + c] += wt[j] * (1 - f) * g;
    nb[(size_t)(k + 1) * n1 + c + 1] += wt[j] * f * g;
  }
  for (int k = 0; k <= nxi; ++k) {
    const double vx = (k == 0 || k == nxi) ? 0.5 * dxi : dxi;
    for (int i = 0; i <= nr; ++i) nb[(size_t)k * n1 + i] /= node_volume(i, nr, dr, ORC_SLAB(p)) * vx;
  }
}

/*
 * nsteps beam steps with trapping.  The beam has room for cap particles, *n_cur of them in
 * use (the first p->n_beam are the bunches; tag 0 drive, 1 witness), with weights wt.  Each
 * step: deposit the beam, march with orc_march_trap, append one beam particle per promoted ring
 * - at (x, y) = (r, 0), xi = xi_k, momentum (u_r, u_theta, u_z) with u_z from Eqs. 2-3 for its
 * Gamma, weight w_j ds (the ring's flux through a xi plane over one beam step), tag 2; lost if
 * it is outside the box, dropped (counted in *n_dropped) once the beam is full - then push all
 * particles in use (Eqs. 8-11).  The fields of the last march are left in psi, ez, er, bth.
 */
int orc_run_trap(const orc_params *p, int nsteps, const double *r0, const double *ur0,
                 const double *l, const double *G0, const double *w, double gamma_t, int64_t cap,
                 int64_t *n_cur, double *x, double *y, double *xi, double *ux, double *uy,
                 double *uz, uint8_t *lost, double *wt, uint8_t *tag, int64_t *n_dropped,
                 double *psi, double *ez, double *er, double *bth) {
  const size_t ng = (size_t)(p->nxi + 1) * (p->nr + 1);
  const int np = p->nr * p->ppc;
  const double dxi = p->ximax / p->nxi;
  double *nb = (double *)malloc(sizeof(double) * ng);
  double *fer = (double *)malloc(sizeof(double) * ng);
  double *fez = (double *)malloc(sizeof(double) * ng);
  double *fbt = (double *)malloc(sizeof(double) * ng);
  double *trap = (double *)malloc(sizeof(double) * 7 * (size_t)np);
  int status = ORC_OK;
  *n_dropped = 0;
  if (!nb || !fer || !fez || !fbt || !trap) {
    status = ORC_ENOMEM;
    goto done;
  }
  for (int s = 0; s < nsteps; ++s) {
    orc_beam_deposit_wt(p, *n_cur, x, y, xi, lost, wt, nb);
    int nt = 0;
    status = orc_march_trap(p, r0, ur0, l, G0, w, nb, gamma_t, psi, fez, fer, fbt, NULL, trap, np, &nt);
    if (status != ORC_OK) goto done;
    for (int t = 0; t < nt; ++t) {
      const double *e = trap + 7 * (size_t)t;
      if (*n_cur >= cap) {
        ++*n_dropped;
        continue;
      }
      const int64_t q = (*n_cur)++;
      const double G = e[5], up2 = e[3] * e[3] + e[4] * e[4];
      x[q] = e[2];
      y[q] = 0.0;
      xi[q] = e[1] * dxi;
      ux[q] = e[3];
      uy[q] = e[4];
      uz[q] = (1.0 + up2 - G * G) / (2.0 * G); /* Eq. 3 */
      lost[q] = !(xi[q] >= 0.0 && xi[q] < p->ximax && e[2] < p->rmax);
      wt[q] = e[6] * p->ds;
      tag[q] = 2;
    }
    orc_params pn = *p;
    pn.n_beam = *n_cur;
    orc_beam_push(&pn, x, y, xi, ux, uy, uz, lost, fer, fez, fbt);
  }
  if (ez) memcpy(ez, fez, sizeof(double) * ng);
  if (er) memcpy(er, fer, sizeof(double) * ng);
  if (bth) memcpy(bth, fbt, sizeof(double) * ng);
done:
  free(nb);
  free(fer);
  free(fez);
  free(fbt);
  free(trap);
  return status;
}
