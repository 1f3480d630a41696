// Device-side helpers shared by the march and beam kernels of libwake.
//
// Grid conventions (Sec. II.A; readings stated in the library header): node-centred radial
// nodes r_i = i dr, i = 0..nr; xi nodes xi_k = k dxi, k = 0..nxi; linear hats in r with
// ring volumes V_0 = dr^2/6, V_i = r_i dr, V_nr = dr (r_nr/2 - dr/6) (per 2 pi).  Slab
// geometry (x, xi), x >= 0 with a mirror plane at x = 0: hat widths V_i = dx, halved at x = 0
// and at the wall (per unit area).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wake {

// Sticky per-simulation status bits (device word), mapped to WAKE_E* codes on the host.
enum : int { ST_NUMERIC = 1, ST_ESCAPE = 2, ST_TIMEOUT = 4 };

constexpr unsigned kFull = 0xffffffffu;

// Everything one CTA needs about one simulation.  Grids are (nxi+1) x (nr+1), slice-major;
// their element type is double (FP64) or float (mixed) as the kernel's policy says.
struct SimDesc {
  int nr, nxi, np, has_beam;
  double rmax, ximax, dr, dxi;
  const double *r0, *ur0, *lz, *G0, *w;  // ring constants (set by wake_load_plasma)
  void *ring_buf;                        // ring slot arrays in global memory (FP64 form)
  const void *nb;                        // beam density n_b on the nodes
  void *psi, *ez, *er, *bth;             // march output
  int *status;
  // trapping (march_trap_kernel): threshold, promotion list of trap_cap entries of 7 doubles
  double gamma_t;
  double *trap;
  int *trap_count;
  int trap_cap;
  int slab;  // slab geometry: r is x, lz holds the conserved u_y
};

// Cell index c in [0, nr-1] and offset f = r/dr - c (f in [0,1] for 0 <= r <= rmax).
// Clamped, so a non-finite r never indexes out of bounds.
template <class R>
__device__ __forceinline__ void locate(R r, R inv_dr, int nr, int &c, R &f) {
  R s = r * inv_dr;
  R fl = floor(s);
  int i = (int)fl;
  i = i < 0 ? 0 : (i > nr - 1 ? nr - 1 : i);
  c = i;
  f = s - (R)i;
}

template <class T, class R>
__device__ __forceinline__ R interp(const T *v, int c, R f) {
  return ((R)1 - f) * (R)v[c] + f * (R)v[c + 1];
}

__host__ __device__ __forceinline__ double node_volume(int i, int nr, double dr, bool slab = false) {
  if (slab) return (i == 0 || i == nr) ? 0.5 * dr : dr;
  return i == 0 ? dr * dr / 6.0 : (i == nr ? dr * ((double)nr * dr / 2.0 - dr / 6.0) : (double)i * dr * dr);
}

// Fraction of hat m's ring volume that lies inside r_m (1/2 - 1/(6m); 1 at the wall; slab 1/2).
__host__ __device__ __forceinline__ double node_alpha(int m, int nr, bool slab = false) {
  return m == nr ? 1.0 : (slab ? 0.5 : 0.5 - 1.0 / (6.0 * (double)m));
}

// Eq. 12: the two-bunch driver density.
__host__ __device__ __forceinline__ double nb_eq12(double r, double xi, double n_d, double n_w,
                                                   double sr, double szd, double szw, double xd,
                                                   double xw) {
  const double ad = (xi - xd) / szd;
  double lon = n_d * exp(-0.5 * ad * ad);
  if (n_w != 0.0) {
    const double aw = (xi - xw) / szw;
    lon += n_w * exp(-0.5 * aw * aw);
  }
  return exp(-r * r / (2.0 * sr * sr)) * lon;
}

__device__ __forceinline__ void flag(int *status, int bit) { atomicOr(status, bit); }

// Block-wide in-place inclusive scan of a[0..n-1] (suffix scan if reverse), n arbitrary:
// each thread sums a contiguous chunk, warps scan the chunk sums with shuffles, warp 0
// scans the warp totals.  Ends with a barrier; wtot needs NT/32 doubles.
template <int NT>
__device__ __forceinline__ void block_scan(double *a, int n, double *wtot, bool reverse) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int E = (n + NT - 1) / NT;
  const int beg = tid * E, end = min(n, beg + E);
  double s = 0.0;
  for (int q = beg; q < end; ++q) s += a[reverse ? n - 1 - q : q];
  double incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    double t = lane < NT / 32 ? wtot[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += u;
    }
    if (lane < NT / 32) wtot[lane] = t;
  }
  __syncthreads();
  double run = incl - s + (warp > 0 ? wtot[warp - 1] : 0.0);
  for (int q = beg; q < end; ++q) {
    const int i = reverse ? n - 1 - q : q;
    run += a[i];
    a[i] = run;
  }
  __syncthreads();
}

// Parallel cyclic reduction (Hockney) for a tridiagonal system of n rows:
//   a_q x_{q-1} + b_q x_q + c_q x_{q+1} = d_q,  a_0 = c_{n-1} = 0.
// Each step eliminates the couplings at distance s and doubles s; after ceil(log2 n) steps
// every row is decoupled and x_q = d_q / b_q.  Arrays are double-buffered (A -> B -> A ...);
// returns which buffer holds the result (0 = first).  Ends with a barrier.
template <int NT, class S>
__device__ __forceinline__ int pcr_solve(S *a0, S *b0, S *c0, S *d0, S *a1, S *b1, S *c1, S *d1,
                                         int n) {
  int cur = 0;
  for (int s = 1; s < n; s <<= 1) {
    S *a = cur ? a1 : a0, *b = cur ? b1 : b0, *c = cur ? c1 : c0, *d = cur ? d1 : d0;
    S *an = cur ? a0 : a1, *bn = cur ? b0 : b1, *cn = cur ? c0 : c1, *dn = cur ? d0 : d1;
    for (int q = threadIdx.x; q < n; q += NT) {
      S aq = a[q], bq = b[q], cq = c[q], dq = d[q];
      S na = (S)0, nc = (S)0;
      if (q - s >= 0) {
        const S k1 = aq / b[q - s];
        bq -= c[q - s] * k1;
        dq -= d[q - s] * k1;
        na = -a[q - s] * k1;
      }
      if (q + s < n) {
        const S k2 = cq / b[q + s];
        bq -= a[q + s] * k2;
        dq -= d[q + s] * k2;
        nc = -c[q + s] * k2;
      }
      an[q] = na;
      bn[q] = bq;
      cn[q] = nc;
      dn[q] = dq;
    }
    __syncthreads();
    cur ^= 1;
  }
  return cur;
}

}  // namespace wake
