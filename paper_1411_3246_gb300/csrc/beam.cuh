// Beam-driver and set-up kernels: the Eq. 12 bunches, their (r, xi) deposit, the Boris push
// of Eqs. 8-11, witness diagnostics, and the initial plasma slice of Sec. II.A.
//
// Beam state is SoA: x, y, u_x, u_y in the policy's type BT (float in the mixed form).  xi
// and u_z need more than FP32: u_z ~ gamma_b = 4e4 changes by O(1) per step and xi slips by
// ~1e-9 per step.  The FP64 form keeps them in FP64; the mixed form keeps each as a
// float-float pair (BeamWide below) in the same 8-byte slot, so that its push runs without
// FP64 instructions.  The kicks themselves are computed in BT either way.  A
// flag byte per particle holds bit 0 = lost, bit 1 = witness and bit 2 = a plasma particle
// promoted by trapping; orig holds the particle's index in the caller's order (the beam is
// kept sorted by xi cell for the pipelined step).  With trapping the arrays have room for
// n_cap >= n particles: the bunches' n, then the promoted particles (the unused slots lost).
#pragma once

#include "wake_common.cuh"

namespace wake {

struct BeamDesc {
  int64_t n, n_drive;
  int64_t n_cap;           // slots in the arrays (n plus room for promoted particles)
  int nr, nxi;
  double rmax, ximax, dr, dxi, ds, gamma_b;
  double wd, ww;           // macroparticle weights of the drive and witness bunches
  void *x, *y, *ux, *uy;   // BT
  double *xi, *uz;         // 8-byte slots: FP64, or (BT float) float-float pairs
  uint8_t *lost;           // flags: bit 0 lost, bit 1 witness, bit 2 promoted (trapping)
  int *orig;               // index in the caller's order
  void *w;                 // per-particle weight (BT): charge per 2 pi
  void *nb;                // beam-density grid (G)
  const void *er, *ez, *bth;  // fields of the last march (G)
  double *diag;            // 5 accumulators
  int slab;                // slab geometry: a sheet beam at y = u_y = 0, folded onto x >= 0
  float2 ffi, ffx;         // 1/dxi and ximax as float-float pairs (the mixed form's xi tests)
};

// A double as a float-float pair (hi, lo): hi = v rounded to FP32, lo = the rest rounded.
__host__ __device__ inline float2 ff_pair(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// The beam's xi and u_z in the form's wide type T.  FP64 form: double.  Mixed form: a
// float-float pair (hi, lo) with |lo| <= ulp(hi)/2, about 48 significant bits.  A sum adds
// an FP32 increment by Knuth's two-sum of the high parts and renormalises.  The cell of xi is
// the floor of the float-float product xi (1/dxi), decided by exact comparisons: it does not
// decrease as xi grows (a particle cannot be found behind a cell it has reached), and the
// sort by cell and the push both call cell(), so they agree on every particle.
template <class BT>
struct BeamWide;

template <>
struct BeamWide<double> {
  using T = double;
  struct Box {
    double inv_dxi, ximax;
  };
  __device__ static Box box(double dxi, double ximax, float2, float2) { return {1.0 / dxi, ximax}; }
  __device__ static T ld(const double *p, int64_t j) { return p[j]; }
  __device__ static T ldcg(const double *p, int64_t j) { return __ldcg(p + j); }
  __device__ static void st(double *p, int64_t j, T v) { p[j] = v; }
  __device__ static T from(double v) { return v; }
  __device__ static double to(T v) { return v; }
  __device__ static double lead(T v) { return v; }
  __device__ static void add(T &v, double d) { v += d; }
  __device__ static bool inside(T xi, const Box &bx) { return xi >= 0.0 && xi < bx.ximax; }
  __device__ static void cell(T xi, const Box &bx, int nxi, int &k, double &g) { locate(xi, bx.inv_dxi, nxi, k, g); }
};

template <>
struct BeamWide<float> {
  using T = float2;
  struct Box {
    float2 inv_dxi, ximax;
  };
  __device__ static Box box(double, double, float2 ffi, float2 ffx) { return {ffi, ffx}; }
  __device__ static T ld(const double *p, int64_t j) { return reinterpret_cast<const float2 *>(p)[j]; }
  __device__ static T ldcg(const double *p, int64_t j) { return __ldcg(reinterpret_cast<const float2 *>(p) + j); }
  __device__ static void st(double *p, int64_t j, T v) { reinterpret_cast<float2 *>(p)[j] = v; }
  __device__ static T from(double v) { return ff_pair(v); }
  __device__ static double to(T v) { return (double)v.x + (double)v.y; }
  __device__ static float lead(T v) { return v.x; }
  __device__ static void add(T &v, float d) {
    const float s = v.x + d, bv = s - v.x;
    const float e = ((v.x - (s - bv)) + (d - bv)) + v.y;  // the rounding error of s, plus lo
    const float h = s + e;
    v = make_float2(h, e - (h - s));
  }
  // 0 <= xi < ximax, the pairs compared high part first
  __device__ static bool inside(T xi, const Box &bx) {
    const bool ge0 = xi.x > 0.0f || (xi.x == 0.0f && xi.y >= 0.0f);
    const bool lt = xi.x < bx.ximax.x || (xi.x == bx.ximax.x && xi.y < bx.ximax.y);
    return ge0 && lt;
  }
  // The cell is floor(p + e) for the float-float product p + e of xi and 1/dxi: decided by
  // exact comparisons of p - floor(p) (exact) with -e, not by a rounded sum, so that a
  // particle is not put back a cell by rounding as xi grows.
  __device__ static void cell(T xi, const Box &bx, int nxi, int &k, float &g) {
    const float p = xi.x * bx.inv_dxi.x;
    const float e = fmaf(xi.x, bx.inv_dxi.y, fmaf(xi.y, bx.inv_dxi.x, fmaf(xi.x, bx.inv_dxi.x, -p)));
    float kf = floorf(p);
    const float r = p - kf;  // exact, in [0, 1)
    if (r < -e)
      kf -= 1.0f;
    else if (r - 1.0f >= -e)  // exact where it can hold (r >= 1/2)
      kf += 1.0f;
    const float f = (p - kf) + e;
    int i = (int)kf;
    i = i < 0 ? 0 : (i > nxi - 1 ? nxi - 1 : i);
    k = i;
    g = f + (kf - (float)i);
  }
};

struct BunchInit {
  double sigma_r, eps_n, xi_d, sigma_zd, xi_w, sigma_zw, gamma_b;
};

// The slots past the bunches (room for promoted particles): empty, that is lost.
template <class BT>
__device__ __forceinline__ void clear_tail(const BeamDesc &b) {
  for (int64_t j = b.n + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b.n_cap;
       j += (int64_t)gridDim.x * blockDim.x) {
    ((BT *)b.x)[j] = ((BT *)b.y)[j] = ((BT *)b.ux)[j] = ((BT *)b.uy)[j] = (BT)0;
    BeamWide<BT>::st(b.xi, j, BeamWide<BT>::from(0.0));
    BeamWide<BT>::st(b.uz, j, BeamWide<BT>::from(0.0));
    b.lost[j] = 1;
    b.orig[j] = (int)j;
    ((BT *)b.w)[j] = (BT)0;
  }
}

// Eq. 12 bunches from standard normals (rows x, y, u_x, u_y, xi of a 5 x n array).  Slab: a
// sheet beam, y = u_y = 0 (rows 1 and 3 unused).
template <class BT>
__global__ void beam_init_kernel(BeamDesc b, BunchInit q, const double *__restrict__ nm) {
  const double su = q.eps_n / q.sigma_r;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b.n; j += (int64_t)gridDim.x * blockDim.x) {
    const bool drive = j < b.n_drive;
    const double x = q.sigma_r * nm[j], y = b.slab ? 0.0 : q.sigma_r * nm[b.n + j];
    const double xi = drive ? q.xi_d + q.sigma_zd * nm[4 * b.n + j] : q.xi_w + q.sigma_zw * nm[4 * b.n + j];
    ((BT *)b.x)[j] = (BT)x;
    ((BT *)b.y)[j] = (BT)y;
    ((BT *)b.ux)[j] = (BT)(su * nm[2 * b.n + j]);
    ((BT *)b.uy)[j] = (BT)(b.slab ? 0.0 : su * nm[3 * b.n + j]);
    BeamWide<BT>::st(b.xi, j, BeamWide<BT>::from(xi));
    BeamWide<BT>::st(b.uz, j, BeamWide<BT>::from(q.gamma_b));
    const double r = sqrt(x * x + y * y);
    b.lost[j] = (uint8_t)((xi >= 0.0 && xi < b.ximax && r < b.rmax) ? 0 : 1) | (uint8_t)(drive ? 0 : 2);
    b.orig[j] = (int)j;
    ((BT *)b.w)[j] = (BT)(drive ? b.wd : b.ww);
  }
  clear_tail<BT>(b);
}

// A beam given by the caller: xyz rows x, y, xi, u_x, u_y, u_z (6 x n, FP64), weights w (NULL:
// the Eq. 12 bunch weights), witness tags (NULL: the particles from n_drive on).  Particles
// outside 0 <= xi < ximax, r < rmax are lost.  Slab: y and u_y are taken as 0.
template <class BT>
__global__ void beam_set_kernel(BeamDesc b, const double *__restrict__ xyz, const double *__restrict__ w,
                                const uint8_t *__restrict__ tag) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b.n; j += (int64_t)gridDim.x * blockDim.x) {
    const bool witness = tag ? tag[j] != 0 : j >= b.n_drive;
    const double x = xyz[j], y = b.slab ? 0.0 : xyz[b.n + j], xi = xyz[2 * b.n + j];
    ((BT *)b.x)[j] = (BT)x;
    ((BT *)b.y)[j] = (BT)y;
    ((BT *)b.ux)[j] = (BT)xyz[3 * b.n + j];
    ((BT *)b.uy)[j] = (BT)(b.slab ? 0.0 : xyz[4 * b.n + j]);
    BeamWide<BT>::st(b.xi, j, BeamWide<BT>::from(xi));
    BeamWide<BT>::st(b.uz, j, BeamWide<BT>::from(xyz[5 * b.n + j]));
    const double r = sqrt(x * x + y * y);
    b.lost[j] = (uint8_t)((xi >= 0.0 && xi < b.ximax && r < b.rmax) ? 0 : 1) | (uint8_t)(witness ? 2 : 0);
    b.orig[j] = (int)j;
    ((BT *)b.w)[j] = (BT)(w ? w[j] : (witness ? b.ww : b.wd));
  }
  clear_tail<BT>(b);
}

// Raw bilinear deposit of the beam weights on the (r, xi) nodes (grid zeroed beforehand):
// particles j0, j0 + stride, ...
template <class BT, class G>
__device__ __forceinline__ void deposit_range(const BeamDesc &b, int64_t j0, int64_t stride) {
  G *nb = (G *)b.nb;
  const int n1 = b.nr + 1;
  using W = BeamWide<BT>;
  const BT inv_dr = (BT)(1.0 / b.dr);
  const typename W::Box bx = W::box(b.dxi, b.ximax, b.ffi, b.ffx);
  for (int64_t j = j0; j < b.n_cap; j += stride) {
    const uint8_t fl = b.lost[j];
    if (fl & 1) continue;
    const BT x = ((const BT *)b.x)[j], y = ((const BT *)b.y)[j];
    const BT r = sqrt(x * x + y * y);
    int c, k;
    BT f, gg;
    locate(r, inv_dr, b.nr, c, f);
    W::cell(W::ld(b.xi, j), bx, b.nxi, k, gg);
    const BT w = ((const BT *)b.w)[j];
    G *row = nb + (size_t)k * n1 + c;
    atomicAdd(row, (G)(w * ((BT)1 - f) * ((BT)1 - gg)));
    atomicAdd(row + 1, (G)(w * f * ((BT)1 - gg)));
    atomicAdd(row + n1, (G)(w * ((BT)1 - f) * gg));
    atomicAdd(row + n1 + 1, (G)(w * f * gg));
  }
}
template <class BT, class G>
__global__ void beam_deposit_kernel(BeamDesc b) {
  deposit_range<BT, G>(b, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Divide the raw deposit by the hats' volumes: V_i in r, dxi in xi (dxi/2 at both ends).
template <class G>
__device__ __forceinline__ void normalize_range(G *nb, int nr, int nxi, double dr, double dxi, int slab, int64_t t0,
                                                int64_t stride) {
  const int n1 = nr + 1;
  const int64_t tot = (int64_t)(nxi + 1) * n1;
  for (int64_t t = t0; t < tot; t += stride) {
    const int k = (int)(t / n1), i = (int)(t % n1);
    const double vx = (k == 0 || k == nxi) ? 0.5 * dxi : dxi;
    nb[t] = (G)((double)nb[t] / (node_volume(i, nr, dr, slab != 0) * vx));
  }
}
template <class G>
__global__ void nb_normalize_kernel(G *nb, int nr, int nxi, double dr, double dxi, int slab) {
  normalize_range<G>(nb, nr, nxi, dr, dxi, slab, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                     (int64_t)gridDim.x * blockDim.x);
}

// Eq. 12 on the nodes (frozen analytic driver).
template <class G>
__global__ void nb_analytic_kernel(G *nb, int nr, int nxi, double dr, double dxi, double n_d, double n_w,
                                   double sr, double szd, double szw, double xd, double xw) {
  const int n1 = nr + 1;
  const int64_t tot = (int64_t)(nxi + 1) * n1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / n1), i = (int)(t % n1);
    nb[t] = (G)nb_eq12(i * dr, k * dxi, n_d, n_w, sr, szd, szw, xd, xw);
  }
}

// One Boris step (Eqs. 8-11 are the Lorentz force of E = (E_r rhat, E_z), B = B_theta
// thetahat on a charge -1) with the fields (Er, Ez, Bt) gathered at the particle: momentum at
// half steps; x_perp += dt u_perp/gamma; xi += dt (1 + u_perp^2)/(gamma (gamma + u_z)).  The
// u_z kick 2 h E_z + (p x s)_z and the xi increment are formed in BT and added to the wide
// u_z and xi.
template <class BT>
__device__ __forceinline__ void boris_step(BT &x, BT &y, BT &ux, BT &uy, typename BeamWide<BT>::T &xi,
                                           typename BeamWide<BT>::T &uzd, BT r, BT Er, BT Ez, BT Bt, BT dt) {
  using W = BeamWide<BT>;
  const BT h = (BT)-0.5 * dt;  // q dt / 2 with q = -1
  const BT cs = r > (BT)0 ? x / r : (BT)0, sn = r > (BT)0 ? y / r : (BT)0;
  const BT Ex = Er * cs, Ey = Er * sn, Bx = -Bt * sn, By = Bt * cs;
  const BT uz = (BT)W::lead(uzd);
  const BT mx = ux + h * Ex, my = uy + h * Ey, mz = uz + h * Ez;
  const BT gm = sqrt((BT)1 + mx * mx + my * my + mz * mz);
  const BT tx = h * Bx / gm, ty = h * By / gm;
  const BT px = mx - mz * ty, py = my + mz * tx, pz = mz + (mx * ty - my * tx);
  const BT s = (BT)2 / ((BT)1 + tx * tx + ty * ty);
  const BT sx = s * tx, sy = s * ty;
  ux = mx - pz * sy + h * Ex;
  uy = my + pz * sx + h * Ey;
  W::add(uzd, (BT)2 * h * Ez + (px * sy - py * sx));
  const BT uzn = (BT)W::lead(uzd);
  const BT up2 = ux * ux + uy * uy;
  const BT gam = sqrt((BT)1 + up2 + uzn * uzn);
  x += dt * ux / gam;
  y += dt * uy / gam;
  W::add(xi, dt * ((BT)1 + up2) / (gam * (gam + uzn)));
}

// One beam step through the grid fields of the last march, bilinear gather in (r, xi):
// particles j0, j0 + stride, ...
template <class BT, class G>
__device__ __forceinline__ void push_range(const BeamDesc &b, int64_t j0, int64_t stride) {
  const G *er = (const G *)b.er, *ez = (const G *)b.ez, *bt = (const G *)b.bth;
  BT *X = (BT *)b.x, *Y = (BT *)b.y, *UX = (BT *)b.ux, *UY = (BT *)b.uy;
  const int n1 = b.nr + 1;
  using W = BeamWide<BT>;
  const BT inv_dr = (BT)(1.0 / b.dr), dt = (BT)b.ds, Rw = (BT)b.rmax;
  const typename W::Box bx = W::box(b.dxi, b.ximax, b.ffi, b.ffx);
  for (int64_t j = j0; j < b.n_cap; j += stride) {
    if (b.lost[j] & 1) continue;
    BT x = X[j], y = Y[j], ux = UX[j], uy = UY[j];
    typename W::T xi = W::ld(b.xi, j), uzd = W::ld(b.uz, j);
    const BT r = sqrt(x * x + y * y);
    int c, k;
    BT f, g;
    locate(r, inv_dr, b.nr, c, f);
    W::cell(xi, bx, b.nxi, k, g);
    const size_t i00 = (size_t)k * n1 + c;
    const BT w00 = ((BT)1 - f) * ((BT)1 - g), w01 = f * ((BT)1 - g), w10 = ((BT)1 - f) * g, w11 = f * g;
    const BT Er = w00 * (BT)er[i00] + w01 * (BT)er[i00 + 1] + w10 * (BT)er[i00 + n1] + w11 * (BT)er[i00 + n1 + 1];
    const BT Ez = w00 * (BT)ez[i00] + w01 * (BT)ez[i00 + 1] + w10 * (BT)ez[i00 + n1] + w11 * (BT)ez[i00 + n1 + 1];
    const BT Bt = w00 * (BT)bt[i00] + w01 * (BT)bt[i00 + 1] + w10 * (BT)bt[i00 + n1] + w11 * (BT)bt[i00 + n1 + 1];
    boris_step<BT>(x, y, ux, uy, xi, uzd, r, Er, Ez, Bt, dt);
    X[j] = x;
    Y[j] = y;
    UX[j] = ux;
    UY[j] = uy;
    W::st(b.xi, j, xi);
    W::st(b.uz, j, uzd);
    const BT rn = sqrt(x * x + y * y);
    if (!(W::inside(xi, bx) && rn < Rw)) b.lost[j] |= 1;
  }
}
template <class BT, class G>
__global__ void beam_push_kernel(BeamDesc b) {
  push_range<BT, G>(b, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Batched forms over the simulations of a handle: blockIdx.y is the simulation; simulations
// without a beam (n == 0, the frozen analytic driver) are left alone.
template <class G>
__global__ void nb_zero_batch_kernel(const BeamDesc *bs) {
  const BeamDesc &b = bs[blockIdx.y];
  if (b.n == 0) return;
  const int64_t tot = (int64_t)(b.nxi + 1) * (b.nr + 1);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    ((G *)b.nb)[t] = (G)0;
}
template <class BT, class G>
__global__ void beam_deposit_batch_kernel(const BeamDesc *bs) {
  const BeamDesc b = bs[blockIdx.y];
  deposit_range<BT, G>(b, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}
template <class G>
__global__ void nb_normalize_batch_kernel(const BeamDesc *bs) {
  const BeamDesc &b = bs[blockIdx.y];
  if (b.n == 0) return;
  normalize_range<G>((G *)b.nb, b.nr, b.nxi, b.dr, b.dxi, b.slab, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                     (int64_t)gridDim.x * blockDim.x);
}
template <class BT, class G>
__global__ void beam_push_batch_kernel(const BeamDesc *bs) {
  const BeamDesc b = bs[blockIdx.y];
  push_range<BT, G>(b, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Witness / drive sums in FP64: counts, sum(gamma - gamma_b), sum(gamma - gamma_b)^2.
template <class BT>
__global__ void beam_diag_kernel(BeamDesc b) {
  const BT *UX = (const BT *)b.ux, *UY = (const BT *)b.uy;
  double nw = 0, sw = 0, sw2 = 0, nd = 0, sd = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b.n_cap; j += (int64_t)gridDim.x * blockDim.x) {
    if (b.lost[j] & 5) continue;  // lost, or a promoted plasma particle (neither bunch)
    const double ux = UX[j], uy = UY[j], uz = BeamWide<BT>::to(BeamWide<BT>::ld(b.uz, j));
    const double g = sqrt(1.0 + ux * ux + uy * uy + uz * uz) - b.gamma_b;
    if (b.lost[j] & 2) {
      nw += 1;
      sw += g;
      sw2 += g * g;
    } else {
      nd += 1;
      sd += g;
    }
  }
  double v[5] = {nw, sw, sw2, nd, sd};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
    if ((threadIdx.x & 31) == 0 && t != 0.0) atomicAdd(&b.diag[q], t);
  }
}

// Initial plasma slice (Sec. II.A): cell c, ring m.  Cold: ppc radii (c + (m+1/2)/ppc) dr;
// warm: ppc/2 radii, each shared by a mirrored pair of draws.  u = u_th * normals,
// gamma0 = sqrt(1 + u^2), Gamma0 = gamma0 - u_z0, l_z = r u_theta0,
// w = r dr/ppc * Gamma0/gamma0 (the quasi-static flux factor 1 - v_z0).  Slab: sheets,
// w = dx/ppc * Gamma0/gamma0, and lz holds the conserved u_y0.
static __global__ void plasma_init_kernel(int nr, int ppc, double dr, double u_th, const double *__restrict__ nm,
                                   double *r0, double *ur0, double *lz, double *G0, double *w, int slab) {
  const int np = nr * ppc;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += gridDim.x * blockDim.x) {
    const int c = j / ppc, m = j % ppc;
    const bool warm = nm != nullptr;
    const double r = warm ? ((double)c + ((double)(m / 2) + 0.5) / (double)(ppc / 2)) * dr
                          : ((double)c + ((double)m + 0.5) / (double)ppc) * dr;
    double ur = 0.0, ut = 0.0, uz = 0.0;
    if (warm) {
      ur = u_th * nm[3 * j];
      ut = u_th * nm[3 * j + 1];
      uz = u_th * nm[3 * j + 2];
    }
    const double g0 = sqrt(1.0 + ur * ur + ut * ut + uz * uz);
    r0[j] = r;
    ur0[j] = ur;
    lz[j] = slab ? ut : r * ut;
    G0[j] = g0 - uz;
    w[j] = (slab ? dr : r * dr) / (double)ppc * ((g0 - uz) / g0);
  }
}

// Counting sort of the beam by xi cell (lost particles go to the extra bin nxi).
// The cell is found exactly as the push finds it (BeamWide<BT>::cell).
template <class BT>
__device__ __forceinline__ int beam_bin(const BeamDesc &b, const typename BeamWide<BT>::Box &bx, int64_t j) {
  if (b.lost[j] & 1) return b.nxi;
  int k;
  BT g;
  BeamWide<BT>::cell(BeamWide<BT>::ld(b.xi, j), bx, b.nxi, k, g);
  return k;
}
// Slip rates dxi/dt = (1 + u_perp^2) / (gamma (gamma + u_z)) of the live beam: the largest, as
// the bits of a non-negative double (ordered like unsigned integers) in *out, and a histogram
// of floor(log2(span / rate)) (clamped to 0..63; span / rate = steps until the particle has
// slipped a given span) in hist.  Both zeroed before.
template <class BT>
__global__ void beam_slip_kernel(BeamDesc b, double span, unsigned long long *out, int *hist) {
  __shared__ int sh[64];  // the block's histogram, added to hist once per bin
  for (int q = threadIdx.x; q < 64; q += blockDim.x) sh[q] = 0;
  __syncthreads();
  double m = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b.n_cap; j += (int64_t)gridDim.x * blockDim.x) {
    if (b.lost[j] & 1) continue;
    const double ux = ((const BT *)b.ux)[j], uy = ((const BT *)b.uy)[j];
    const double uz = BeamWide<BT>::to(BeamWide<BT>::ld(b.uz, j));
    const double up2 = ux * ux + uy * uy, g = sqrt(1.0 + up2 + uz * uz);
    const double rate = (1.0 + up2) / (g * (g + uz));
    m = fmax(m, rate);
    const double steps = rate > 0.0 ? span / rate : 1e300;
    const int q = steps < 1.0 ? 0 : (steps >= 9.2e18 ? 63 : min(63, 63 - __clzll((long long)steps)));
    atomicAdd(&sh[q], 1);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
  __syncthreads();
  for (int q = threadIdx.x; q < 64; q += blockDim.x)
    if (sh[q]) atomicAdd(&hist[q], sh[q]);
}
template <class BT>
__global__ void bin_count_kernel(BeamDesc b, int *count) {
  const typename BeamWide<BT>::Box bx = BeamWide<BT>::box(b.dxi, b.ximax, b.ffi, b.ffx);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b.n_cap; j += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&count[beam_bin<BT>(b, bx, j)], 1);
}
// The largest of the counts of bins 0 .. n-1, into *out (zeroed before).
static __global__ void bin_max_kernel(const int *count, int n, int *out) {
  int m = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) m = max(m, count[q]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}
// exclusive scan of nbins counts into start[0..nbins] (one block of 1024 threads)
static __global__ void bin_scan_kernel(const int *count, int *start, int *cursor, int nbins) {
  __shared__ int part[1024];
  const int t = threadIdx.x, E = (nbins + 1023) / 1024, beg = t * E, end = min(nbins, beg + E);
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
  if (t == 1023) start[nbins] = part[1023];
}
template <class BT>
__global__ void bin_scatter_kernel(BeamDesc b, BeamDesc dst, int *cursor) {
  const typename BeamWide<BT>::Box bx = BeamWide<BT>::box(b.dxi, b.ximax, b.ffi, b.ffx);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b.n_cap; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = atomicAdd(&cursor[beam_bin<BT>(b, bx, j)], 1);
    ((BT *)dst.x)[q] = ((const BT *)b.x)[j];
    ((BT *)dst.y)[q] = ((const BT *)b.y)[j];
    ((BT *)dst.ux)[q] = ((const BT *)b.ux)[j];
    ((BT *)dst.uy)[q] = ((const BT *)b.uy)[j];
    BeamWide<BT>::st(dst.xi, q, BeamWide<BT>::ld(b.xi, j));
    BeamWide<BT>::st(dst.uz, q, BeamWide<BT>::ld(b.uz, j));
    dst.lost[q] = b.lost[j];
    dst.orig[q] = b.orig[j];
    ((BT *)dst.w)[q] = ((const BT *)b.w)[j];
  }
}
// Scatter the beam back to the caller's order: out rows x, y, xi, u_x, u_y, u_z (6 x n).
template <class BT>
__global__ void beam_unpermute_kernel(BeamDesc b, double *xyz, uint8_t *lost) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < b.n_cap; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b.orig[j];
    if (o >= b.n) continue;  // a promoted particle (wake_trapped returns those)
    if (xyz) {
      xyz[0 * b.n + o] = (double)((const BT *)b.x)[j];
      xyz[1 * b.n + o] = (double)((const BT *)b.y)[j];
      xyz[2 * b.n + o] = BeamWide<BT>::to(BeamWide<BT>::ld(b.xi, j));
      xyz[3 * b.n + o] = (double)((const BT *)b.ux)[j];
      xyz[4 * b.n + o] = (double)((const BT *)b.uy)[j];
      xyz[5 * b.n + o] = BeamWide<BT>::to(BeamWide<BT>::ld(b.uz, j));
    }
    if (lost) lost[o] = b.lost[j] & 1;
  }
}

// Promoted plasma particles into the beam (trapping, Sec. I): entry q of the march's list
// (ring j, slice k, r, u_r, u_theta, Gamma, w) becomes the particle in slot n + *used + rank_q,
// rank_q the entry's place in (k, j) order, so that the slots do not depend on the order the
// march's atomics produced: at (x, y) = (r, 0), xi = k dxi, momentum (u_r, u_theta, u_z) with
// u_z = (1 + u_perp^2 - Gamma^2) / (2 Gamma) (Eqs. 2-3), weight w ds (the ring's flux over one
// beam step), flags promoted (and lost outside the box).  Entries that do not fit the arrays
// are counted in *dropped.  One block; *used advances by the entries placed.
template <class BT>
__global__ void trap_append_kernel(BeamDesc b, const double *__restrict__ list, const int *__restrict__ count, int cap,
                                   int64_t *used, int64_t *dropped) {
  const int nl = min(*count, cap);
  const int64_t base = *used, room = b.n_cap - b.n - base;
  for (int q = threadIdx.x; q < nl; q += blockDim.x) {
    const double *e = list + 7 * (size_t)q;
    const double key = e[1] * 1e9 + e[0];  // slice-major, then ring
    int rank = 0;
    for (int m = 0; m < nl; ++m) {
      const double km = list[7 * (size_t)m + 1] * 1e9 + list[7 * (size_t)m];
      rank += km < key;
    }
    if (rank >= room) continue;
    const int64_t j = b.n + base + rank;
    const double r = e[2], ur = e[3], ut = e[4], G = e[5], up2 = ur * ur + ut * ut;
    const double xi = e[1] * b.dxi;
    ((BT *)b.x)[j] = (BT)r;
    ((BT *)b.y)[j] = (BT)0;
    ((BT *)b.ux)[j] = (BT)ur;
    ((BT *)b.uy)[j] = (BT)ut;
    BeamWide<BT>::st(b.uz, j, BeamWide<BT>::from((1.0 + up2 - G * G) / (2.0 * G)));
    BeamWide<BT>::st(b.xi, j, BeamWide<BT>::from(xi));
    b.lost[j] = (uint8_t)4 | (uint8_t)((xi >= 0.0 && xi < b.ximax && r < b.rmax) ? 0 : 1);
    b.orig[j] = (int)j;
    ((BT *)b.w)[j] = (BT)(e[6] * b.ds);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int64_t placed = nl < room ? nl : (room > 0 ? room : 0);
    *used = base + placed;
    *dropped += (int64_t)(*count) - placed;
  }
}

// The promoted particles (slots n .. n + used - 1) to caller arrays: xyz rows x, y, xi, u_x,
// u_y, u_z of stride cap_out (FP64), weights w, lost flags.
template <class BT>
__global__ void trapped_out_kernel(BeamDesc b, int64_t used, int64_t cap_out, double *xyz, double *w, uint8_t *lost) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < used; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = b.n + q;
    if (xyz) {
      xyz[0 * cap_out + q] = (double)((const BT *)b.x)[j];
      xyz[1 * cap_out + q] = (double)((const BT *)b.y)[j];
      xyz[2 * cap_out + q] = BeamWide<BT>::to(BeamWide<BT>::ld(b.xi, j));
      xyz[3 * cap_out + q] = (double)((const BT *)b.ux)[j];
      xyz[4 * cap_out + q] = (double)((const BT *)b.uy)[j];
      xyz[5 * cap_out + q] = BeamWide<BT>::to(BeamWide<BT>::ld(b.uz, j));
    }
    if (w) w[q] = (double)((const BT *)b.w)[j];
    if (lost) lost[q] = b.lost[j] & 1;
  }
}

template <class Src>
__global__ void widen_kernel(const Src *__restrict__ in, double *__restrict__ out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (double)in[t];
}

}  // namespace wake
