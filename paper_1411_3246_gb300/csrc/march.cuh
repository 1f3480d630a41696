// The quasi-static xi-march (Sec. II.A, Eqs. 1-7): one CTA marches one simulation through
// all of its slices, persistent over xi.
//
// Per slice, RK2 (midpoint) in xi; each stage solves the fields for the rings' positions in
// four phases separated by block barriers, every phase run by all threads of the CTA:
//   P0  psi from Gauss's law for the hat charge density (enclosed charge Phi_m at node m,
//       r_m psi'_m = Phi_m), psi(R) = 0, inward trapezoid sum: two block-wide scans over
//       the nodes (solve_psi);
//   P1  per ring: Gamma = Gamma_0 + psi (Eq. 1), gamma and u_z (Eqs. 2-3), a = u_r/Gamma,
//       F0 = (gamma/Gamma) psi' + u_theta^2/(Gamma r) (Eq. 4 without -B); deposit J_z,
//       chi = n/gamma, T = D[w a^2], P = D[w (a^2 psi' - F0)/Gamma], U = D[w a/Gamma] on the
//       nodes and the radial current K_c of each cell (pass_currents);
//   P2  E_z = d_xi psi (Eq. 7) by a block-wide inward scan of the cell currents; Q = P + E_z U;
//       B_theta from Eq. 6 differentiated in r (Helmholtz form, shift chi), a tridiagonal
//       system solved by block-wide parallel cyclic reduction on row sums (solve_fields);
//   P3  per ring: the Cartesian radial force (gamma/Gamma) psi' - B_theta (Eqs. 4-5 with the
//       centrifugal term carried by the local frame), the move to the next stage's position,
//       and that position's charge deposit (linear hats).
// Stage 1 at xi_k writes the slice's fields; stage 2 at xi_k + dxi/2 uses n_b averaged over
// slices k and k+1.
//
// Layout.  Ring state lives in slot arrays (structure of arrays, slot p*NT + t for the p-th
// ring of thread t): shared memory in the mixed form, global memory in the FP64 form.  A
// thread's rings are consecutive in radius (the mixed form re-sorts them by cell every two
// slices), so its deposits are summed over a window of three cells in registers, combined
// across the lanes of a warp that share a window by segmented shuffle sums, and flushed with
// one shared-memory atomic per segment, node and array.  The node scans run block-wide (each
// thread up to kScanE consecutive nodes, warp shuffles, one warp for the warp totals) in a
// wide type: FP64, or float-float pairs on the FP32 pipe.
#pragma once

#include "wake_common.cuh"
#include <type_traits>

namespace wake {

// ---------------------------------------------------------------------------------------
// wide accumulation type: FP64, or a float-float pair (Dekker / Knuth two-sum), which keeps
// ~48 significant bits on the FP32 pipe
// ---------------------------------------------------------------------------------------
struct FF {
  float h, l;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  const float h = s + e;
  return FF{h, e - (h - s)};
}
__device__ __forceinline__ double wide_add(double a, double b) { return a + b; }
__device__ __forceinline__ FF wide_add(FF a, FF b) { return ff_add(a, b); }
__device__ __forceinline__ double wide_shfl_up(double a, int o) { return __shfl_up_sync(kFull, a, o); }
__device__ __forceinline__ FF wide_shfl_up(FF a, int o) {
  return FF{__shfl_up_sync(kFull, a.h, o), __shfl_up_sync(kFull, a.l, o)};
}
__device__ __forceinline__ double wide_shfl_down(double a, int o) { return __shfl_down_sync(kFull, a, o); }
__device__ __forceinline__ double wide_shfl_idx(double a, int l) { return __shfl_sync(kFull, a, l); }
__device__ __forceinline__ FF wide_shfl_idx(FF a, int l) { return FF{__shfl_sync(kFull, a.h, l), __shfl_sync(kFull, a.l, l)}; }
__device__ __forceinline__ FF wide_shfl_down(FF a, int o) {
  return FF{__shfl_down_sync(kFull, a.h, o), __shfl_down_sync(kFull, a.l, o)};
}
template <class W>
__device__ __forceinline__ W wide_zero();
template <>
__device__ __forceinline__ double wide_zero<double>() { return 0.0; }
template <>
__device__ __forceinline__ FF wide_zero<FF>() { return FF{0.f, 0.f}; }
__device__ __forceinline__ float wide_value(FF x) { return x.h + x.l; }
__device__ __forceinline__ double wide_value(double x) { return x; }
template <class W, class R>
__device__ __forceinline__ W wide_of(R x);
template <>
__device__ __forceinline__ double wide_of<double, double>(double x) { return x; }
template <>
__device__ __forceinline__ FF wide_of<FF, float>(float x) { return FF{x, 0.f}; }

// exclusive prefix over the lanes of one warp of per-lane totals (lane 0 gets 0)
template <class W>
__device__ __forceinline__ W warp_excl_prefix(W v, int lane) {
  W incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const W t = wide_shfl_up(incl, o);
    if (lane >= o) incl = wide_add(incl, t);
  }
  const W ex = wide_shfl_up(incl, 1);
  return lane == 0 ? wide_zero<W>() : ex;
}
// exclusive suffix over the lanes of one warp (lane 31 gets 0)
template <class W>
__device__ __forceinline__ W warp_excl_suffix(W v, int lane) {
  W incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const W t = wide_shfl_down(incl, o);
    if (lane + o < 32) incl = wide_add(incl, t);
  }
  const W ex = wide_shfl_down(incl, 1);
  return lane == 31 ? wide_zero<W>() : ex;
}

// ---------------------------------------------------------------------------------------
// precision policies.  R: ring arithmetic; N: node arrays and the radial solves; Acc:
// current-type deposit sums across rings (a thread's own rings are summed in R first); Q:
// charge deposit sums (psi comes from the small difference rho - rho0 of two large sums, so
// the mixed forms sum exact float-float products as 64-bit integers, which makes rho - rho0
// exact); G: grid element type in global memory; W: scan type.  Mixed: rings in shared
// memory, re-sorted by cell every kSortEvery slices, node coefficients computed on the fly.
// FP64: rings in global memory in their initial order, node coefficients from tables (FP64
// division is slow on this chip).  kWinGlobal: the pipelined step keeps its field window in
// global memory (its shared memory is full).
// ---------------------------------------------------------------------------------------
struct PolFP64 {
  using R = double;
  using N = double;
  using Acc = double;
  using Q = double;  // charge deposit sums
  using G = double;
  using W = double;
  static constexpr int NT = 512;
  static constexpr int kSortEvery = 0;
  static constexpr bool kSmemRings = false;
  static constexpr bool kTables = true;
  static constexpr bool kWinGlobal = false;
  static constexpr bool kSlab = false;  // geometry: see SlabOf
  static constexpr bool kDeferMisses = false;  // out-of-window rings deposited after the ring loops
  static constexpr bool kWarpPCR = false;      // the tridiagonal solve finished per warp
  static constexpr int kScanE = 3;  // nodes per thread in the block scans: n1 <= kScanE * NT
};
struct PolMixed {
  using R = float;
  using N = float;
  using Acc = float;
  using Q = long long;  // charge deposit sums: 64-bit fixed point, 2^-44 resolution
  using G = float;
  using W = FF;
  static constexpr int NT = 512;
  static constexpr int kSortEvery = 2;
  static constexpr bool kSmemRings = true;
  static constexpr bool kTables = false;
  static constexpr bool kWinGlobal = false;
  static constexpr bool kSlab = false;  // geometry: see SlabOf
  static constexpr bool kDeferMisses = true;  // out-of-window rings deposited after the ring loops
  static constexpr bool kWarpPCR = true;      // the tridiagonal solve finished per warp
  static constexpr int kScanE = 3;
};
// The precision split in which only the particle arithmetic is FP32: each ring's push and its
// deposit terms (and a thread's sum over its own few rings) in FP32; the per-slice reductions
// across rings (current sums in FP64, charge in exact fixed point), the node arrays, the scans
// and the tridiagonal solve in FP64.
struct PolMixed64 {
  using R = float;
  using N = double;
  using Acc = double;
  using Q = long long;
  using G = float;
  using W = double;
  static constexpr int NT = 512;
  static constexpr int kSortEvery = 2;
  static constexpr bool kSmemRings = true;
  static constexpr bool kTables = false;
  static constexpr bool kWinGlobal = true;
  static constexpr bool kSlab = false;  // geometry: see SlabOf
  static constexpr bool kDeferMisses = true;  // out-of-window rings deposited after the ring loops
  static constexpr bool kWarpPCR = true;      // the tridiagonal solve finished per warp
  static constexpr int kScanE = 3;
};
// The mixed arithmetic for boxes too large for one CTA's shared memory to hold the rings
// (up to 2048 radial cells and 65,536 rings): rings in global memory, processed in chunks,
// re-sorted by cell every two slices; block scans of up to 5 nodes per thread.
struct PolWide {
  using R = float;
  using N = float;
  using Acc = float;
  using Q = long long;
  using G = float;
  using W = FF;
  static constexpr int NT = 512;
  static constexpr int kSortEvery = 2;  // rings re-sorted by cell through a second global buffer
  static constexpr bool kSmemRings = false;
  static constexpr bool kTables = false;
  static constexpr bool kWinGlobal = false;
  static constexpr bool kSlab = false;  // geometry: see SlabOf
  static constexpr bool kDeferMisses = false;  // out-of-window rings deposited after the ring loops
  static constexpr bool kWarpPCR = false;      // the tridiagonal solve finished per warp
  static constexpr int kScanE = 5;
};

// The FP64 arithmetic for boxes too large for one CTA's shared memory (the wide form): rings in
// global memory as PolWide, and the node arrays too (in FP64 they exceed shared memory at
// 2,049 nodes), in a per-CTA global buffer the wide kernels of march_wide64.cu carve.
struct PolWideFP64 {
  using R = double;
  using N = double;
  using Acc = double;
  using Q = double;
  using G = double;
  using W = double;
  static constexpr int NT = 512;
  static constexpr int kSortEvery = 2;
  static constexpr bool kSmemRings = false;
  static constexpr bool kTables = false;
  static constexpr bool kWinGlobal = false;
  static constexpr bool kSlab = false;  // geometry: see SlabOf
  static constexpr bool kDeferMisses = false;  // out-of-window rings deposited after the ring loops
  static constexpr bool kWarpPCR = false;      // the tridiagonal solve finished per warp
  static constexpr int kScanE = 5;
};
// The slab geometry (x, xi) of a policy (Sec. I: WAKE handles slab and cylindrical geometry):
// d/dy = 0 in place of d/dtheta = 0, x >= 0 with a mirror plane at x = 0, volumes per unit
// area, lap_perp = d_x^2, Eq. 6 as d_x B_y = d_xi^2 psi + J_z, and the conserved u_y (kept in
// the l_z slot) entering gamma only.  A separate instantiation, so the cylindrical kernels
// carry no geometry test.
template <class P>
struct SlabOf : P {
  static constexpr bool kSlab = true;
};

// Ring slot arrays: cell index, offset in the cell, u_r, the constants l_z, Gamma_0, w, and
// the stage-1 Gamma and radial force kept for the full step; with ids, each slot also carries
// its ring's initial index (it follows the ring through the re-sorts; the trajectory dump
// uses it).
template <class R>
struct RingSoA {
  int *c;
  R *f, *ur, *lz, *G0, *w, *G1, *F1;
  int *id = nullptr;
  __host__ __device__ static size_t bytes(int slots, bool ids = false) {
    return sizeof(int) * (size_t)slots + 32 + 7 * sizeof(R) * (size_t)slots + (ids ? sizeof(int) * (size_t)slots + 32 : 0);
  }
  __device__ __forceinline__ void carve(void *base, int slots, bool ids = false) {
    c = (int *)base;
    R *p = (R *)(((uintptr_t)(c + slots) + 31) & ~(uintptr_t)31);
    f = p; p += slots;
    ur = p; p += slots;
    lz = p; p += slots;
    G0 = p; p += slots;
    w = p; p += slots;
    G1 = p; p += slots;
    F1 = p; p += slots;
    id = ids ? (int *)(((uintptr_t)p + 31) & ~(uintptr_t)31) : nullptr;
  }
};

template <class Pol>
struct MarchSmem {
  using R = typename Pol::R;
  using N = typename Pol::N;
  using Acc = typename Pol::Acc;
  typename Pol::Q *rho0, *rho;                  // charge deposits
  Acc *jz, *chi, *T, *P, *U, *K;                // current-type deposits
  N *psi, *dpsi, *ez, *bth;                     // node fields
  R *nb0, *nb1;                                 // beam-density rows (double buffer)
  N *ta, *tb, *tc, *td;                         // tridiagonal rows (a, row sum, c, rhs)
  N *invR, *invV, *alpha, *ga, *gb, *gc;        // tables (FP64 form; the mixed forms keep
                                                // invR = 1/(m dr) and ga = 1/(j + 1/2) only)
  int *cnt;                                     // re-sort counts
  int *qn;                                      // entries in the out-of-window ring queue
  typename Pol::W *wtot;                        // block-scan warp totals
  RingSoA<R> rings;                             // ring slots (mixed form)

  __host__ __device__ static size_t bytes(int n1, int slots, bool ids = false) {
    size_t b = sizeof(typename Pol::W) * 64 + sizeof(typename Pol::Q) * 2 * (size_t)n1 + sizeof(Acc) * 6 * (size_t)n1 +
               sizeof(N) * 4 * (size_t)n1 + sizeof(R) * 2 * (size_t)n1 + sizeof(N) * 4 * ((size_t)n1 + 32) + 256;
    b += sizeof(N) * (Pol::kTables ? 6 : 2) * (size_t)n1;
    if (Pol::kSortEvery > 0) b += sizeof(int) * ((size_t)n1 + 32);
    if (Pol::kSmemRings) b += RingSoA<R>::bytes(slots, ids) + 32;
    return b + 64;
  }
  __device__ void carve(unsigned char *base, int n1, int slots, bool ids = false) {
    wtot = (typename Pol::W *)base;
    typename Pol::Q *qp = (typename Pol::Q *)(wtot + 64);
    rho0 = qp; qp += n1;
    rho = qp; qp += n1;
    Acc *ap = (Acc *)qp;
    jz = ap; ap += n1;
    chi = ap; ap += n1;
    T = ap; ap += n1;
    P = ap; ap += n1;
    U = ap; ap += n1;
    K = ap; ap += n1;
    N *rp = (N *)ap;
    psi = rp; rp += n1;
    dpsi = rp; rp += n1;
    ez = rp; rp += n1;
    bth = rp; rp += n1;
    ta = rp; rp += n1 + 32;
    tb = rp; rp += n1 + 32;
    tc = rp; rp += n1 + 32;
    td = rp; rp += n1 + 32;
    invR = invV = alpha = ga = gb = gc = nullptr;
    invR = rp; rp += n1;
    ga = rp; rp += n1;
    if (Pol::kTables) {
      invV = rp; rp += n1;
      alpha = rp; rp += n1;
      gb = rp; rp += n1;
      gc = rp; rp += n1;
    }
    R *bp = (R *)rp;
    nb0 = bp; bp += n1;
    nb1 = bp; bp += n1;
    int *ip = (int *)(((uintptr_t)bp + 7) & ~(uintptr_t)7);
    cnt = nullptr;
    if (Pol::kSortEvery > 0) {
      cnt = ip;
      ip += n1 + 32;
    }
    qn = ip;
    ip += 16;
    if (Pol::kSmemRings) rings.carve((void *)(((uintptr_t)ip + 31) & ~(uintptr_t)31), slots, ids);
  }
  // The out-of-window ring queue: slot ids in the tridiagonal rows, which are free from the end
  // of one solve to the start of the next (a ring pass and the deposits that follow it)
  __device__ __forceinline__ int *queue() const { return (int *)ta; }
  __device__ __forceinline__ int queue_cap(int n1) const { return (int)(4 * ((size_t)n1 + 32) * sizeof(N) / sizeof(int)); }
};

// ---------------------------------------------------------------------------------------
// node geometry: 1/r_m, 1/V_m, alpha_m and the B_theta rows (central differences, a half
// cell at the wall), from tables or computed on the fly
// ---------------------------------------------------------------------------------------
// division of the solves: the mixed form is compiled with the fast approximate '/'
__device__ __forceinline__ float div_rn(float a, float b) { return a / b; }
__device__ __forceinline__ double div_rn(double a, double b) { return a / b; }

template <class Pol>
struct NodeGeo {
  using R = typename Pol::N;  // node arithmetic
  const R *t_invR, *t_invV, *t_alpha, *t_ga, *t_gb, *t_gc;
  int nr;
  R dr, inv_dr, inv_dr2, dr_6, v_wall_inv;
  static constexpr bool slab = Pol::kSlab;  // lap_perp = d_x^2, hat widths per unit area
  // the metric of Gauss's law at node m, 1/r_m (slab 1), and the curvature term of
  // (1/r) d_r(r .), 1/r_m (slab 0)
  __device__ __forceinline__ R metric(int m) const { return slab ? (R)1 : t_invR[m]; }
  __device__ __forceinline__ R curv(int m) const { return slab ? (R)0 : t_invR[m]; }
  __device__ __forceinline__ R invV(int m) const {
    if (Pol::kTables) return t_invV[m];
    // V_m = m dr^2 in the interior; dr^2/6 on the axis; dr^2 (nr/2 - 1/6) at the wall.  Slab:
    // dx, dx/2 on the mirror plane and at the wall
    if (slab) return (m == 0 || m == nr) ? (R)2 * inv_dr : inv_dr;
    return m == 0 ? (R)6 * inv_dr2 : (m == nr ? inv_dr2 * v_wall_inv : t_invR[m] * inv_dr);
  }
  __device__ __forceinline__ R alpha(int m) const {
    if (Pol::kTables) return t_alpha[m];
    if (slab) return m == 0 ? (R)0 : (m == nr ? (R)1 : (R)0.5);
    return m == 0 ? (R)0 : (m == nr ? (R)1 : (R)0.5 - t_invR[m] * dr_6);
  }
  // row q (node i = q + 1): a_q x_{q-1} + b_q x_q + c_q x_{q+1}, without the -chi shift, and
  // its row sum a + b + c.  The row sum is the small margin of diagonal dominance (about
  // -1/(r_{i-1/2} r_{i+1/2}) against a diagonal of -2/dr^2), so it is formed directly, never
  // as the difference of the large coefficients.  1/(j + 1/2) comes from the table ga in the
  // mixed form.
  __device__ __forceinline__ void row(int q, R &a, R &c, R &sum) const {
    if (Pol::kTables) {
      a = t_ga[q];
      c = t_gc[q];
      sum = t_ga[q] + t_gb[q] + t_gc[q];  // FP64: the cancellation costs ~1e-13 of the margin
      return;
    }
    const int i = q + 1;
    if (slab) {  // d_x^2: a row sum of zero in the interior, the margin is chi alone
      a = q == 0 ? (R)0 : (i < nr ? inv_dr2 : (R)2 * inv_dr2);
      c = i < nr ? inv_dr2 : (R)0;
      sum = q == 0 ? (i < nr ? -inv_dr2 : (R)-2 * inv_dr2) : (R)0;
      return;
    }
    const R ihm = t_ga[i - 1], ihp = t_ga[i];  // 1/(i - 1/2), 1/(i + 1/2)
    if (i < nr) {
      a = q == 0 ? (R)0 : (R)(i - 1) * ihm * inv_dr2;
      c = (R)(i + 1) * ihp * inv_dr2;
      sum = q == 0 ? (R)(-4.0 / 3.0) * inv_dr2 : -(ihm * ihp) * inv_dr2;
    } else {
      a = q == 0 ? (R)0 : (R)(2 * (i - 1)) * ihm * inv_dr2;
      c = (R)0;
      sum = q == 0 ? (R)-2 * (R)i * ihm * inv_dr2 : (R)-2 * ihm * inv_dr2;
    }
  }
};

template <class Pol, int NT>
__device__ __forceinline__ void fill_tables(MarchSmem<Pol> &sm, int nr, double dr) {
  using R = typename Pol::N;
  constexpr bool slab = Pol::kSlab;
  for (int m = threadIdx.x; m <= nr; m += NT) {
    sm.invR[m] = (R)(m > 0 ? 1.0 / ((double)m * dr) : 0.0);
    if constexpr (Pol::kTables) {
      sm.invV[m] = (R)(1.0 / node_volume(m, nr, dr, slab));
      sm.alpha[m] = (R)(m > 0 ? node_alpha(m, nr, slab) : 0.0);
      if (m < nr) {
        const int i = m + 1;
        const double idr2 = 1.0 / (dr * dr), rm = i - 0.5, rp = i + 0.5;
        double a, b, c;
        if (slab) {  // d_x^2, a half cell at the wall
          a = i < nr ? idr2 : 2.0 * idr2;
          c = i < nr ? idr2 : 0.0;
          b = -2.0 * idr2;
        } else if (i < nr) {
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
    } else {
      sm.ga[m] = (R)(1.0 / ((double)m + 0.5));
    }
  }
}

// Charge sums.  FP64 form: plain doubles.  Mixed form: 64-bit fixed point (2^44 units).  A
// ring's share w f is the exact float-float product (two-product by FMA) rounded once to the
// fixed-point grid, and its share w (1 - f) is the ring's fixed-point weight minus that, so
// the two add up to the same integer on every slice; window, warp and shared-memory sums
// are integer and exact, so rho - rho0 loses nothing to cancellation.
constexpr double kQScale = 17592186044416.0;  // 2^44
__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = a * b;
  return FF{p, __fmaf_rn(a, b, -p)};
}
// x rounded to the nearest integer (ties to even), as a 64-bit integer, from 32-bit
// instructions only (the 64-bit conversions run on the slow FP64 pipe): below 2^31 in
// magnitude the 32-bit conversion rounds it; above, x has 24 significant bits and is an
// integer, given exactly by its significand shifted by its exponent.  |x| < 2^63.
__device__ __forceinline__ long long f2q(float x) {
  const int b = __float_as_int(x);
  int e = ((b >> 23) & 0xff) - 150;  // x = m 2^e
  e = e < 0 ? 0 : (e > 40 ? 40 : e);
  const long long m = (long long)((b & 0x7fffff) | 0x800000) << e;
  const bool small = fabsf(x) < 2147483648.f;
  const long long r = (long long)__float2int_rn(small ? x : 0.f);
  return small ? r : (b < 0 ? -m : m);
}
__device__ __forceinline__ long long ff_to_q(FF x) { return f2q(x.h * (float)kQScale) + f2q(x.l * (float)kQScale); }
template <class Q, class W>
__device__ __forceinline__ W q_to_wide(Q d);
template <>
__device__ __forceinline__ double q_to_wide<double, double>(double d) { return d; }
template <>
__device__ __forceinline__ double q_to_wide<long long, double>(long long d) {
  return (double)d * (1.0 / kQScale);  // exact: |d| < 2^53 and the scale is a power of two
}
template <>
__device__ __forceinline__ FF q_to_wide<long long, FF>(long long d) {
  // the integer (|d| < 2^48) as the float-float sum of three exact floats (32-bit conversions
  // only), i.e. its correctly rounded float and the exact remainder, then the exact
  // power-of-two rescale
  const int dh = (int)(d >> 32);
  const unsigned dl = (unsigned)d;
  const FF x = ff_add(ff_add(FF{(float)dh * 4294967296.f, 0.f}, FF{(float)(int)(dl >> 16) * 65536.f, 0.f}),
                      FF{(float)(int)(dl & 0xffffu), 0.f});
  const float s = (float)(1.0 / kQScale);
  return FF{x.h * s, x.l * s};
}

// Block-wide parallel cyclic reduction on the row-sum form (see pcr_rowsum_solve below), every
// doubling over the block with a barrier.  Double-buffered; returns the buffer holding the
// result (x_q = d_q / s_q there).  Ends with a barrier.
template <int NT, class S>
__device__ __forceinline__ int pcr_rowsum(S *a0, S *s0, S *c0, S *d0, S *a1, S *s1, S *c1, S *d1, int n) {
  int cur = 0;
  for (int k = 1; k < n; k <<= 1) {
    const S *a = cur ? a1 : a0, *sm_ = cur ? s1 : s0, *c = cur ? c1 : c0, *d = cur ? d1 : d0;
    S *an = cur ? a0 : a1, *sn = cur ? s0 : s1, *cn = cur ? c0 : c1, *dn = cur ? d0 : d1;
    for (int q = threadIdx.x; q < n; q += NT) {
      const S aq = a[q], cq = c[q];
      S sq = sm_[q], dq = d[q], na = (S)0, nc = (S)0;
      if (q - k >= 0) {
        const S bm = sm_[q - k] - a[q - k] - c[q - k];
        const S k1 = aq / bm;
        sq -= k1 * sm_[q - k];
        dq -= k1 * d[q - k];
        na = -a[q - k] * k1;
      }
      if (q + k < n) {
        const S bp = sm_[q + k] - a[q + k] - c[q + k];
        const S k2 = cq / bp;
        sq -= k2 * sm_[q + k];
        dq -= k2 * d[q + k];
        nc = -c[q + k] * k2;
      }
      an[q] = na;
      sn[q] = sq;
      cn[q] = nc;
      dn[q] = dq;
    }
    __syncthreads();
    cur ^= 1;
  }
  return cur;
}

// Parallel cyclic reduction (Hockney) on rows a_q x_{q-1} + b_q x_q + c_q x_{q+1} = d_q
// stored as (a, s = a + b + c, c, d).  For this M-matrix (a, c >= 0, s < 0) the eliminated
// row sum s' = s - k1 s_{q-k} - k2 s_{q+k} (k1 = a_q/b_{q-k}, k2 = c_q/b_{q+k}, both <= 0)
// adds terms of one sign, so the margin of diagonal dominance is never lost to cancellation;
// b = s - a - c likewise.  After ceil(log2 n) doublings a = c = 0 and x_q = d_q / s_q.
//
// The first doublings (strides 1 .. ns/2) run over the block, double-buffered, one barrier
// each.  They leave ns independent systems, rows r, r + ns, r + 2 ns, ... (ns the smallest
// power of two >= NT/32 with n <= 32 ns); each is finished by one warp, lane l holding row
// r + ns l, with the remaining doublings (lane strides 1 .. 16) done by shuffles.  The
// arithmetic is that of the block form, stride for stride.  out(q, x_q) receives the solution.
template <int NT, class S, class Out>
__device__ __forceinline__ void pcr_rowsum_solve(S *a0, S *s0, S *c0, S *d0, S *a1, S *s1, S *c1, S *d1, int n,
                                                 Out &&out) {
  constexpr int W = NT / 32;
  int ns = W;
  while (32 * ns < n) ns <<= 1;
  int cur = 0;
  for (int k = 1; k < ns && k < n; k <<= 1) {
    const S *a = cur ? a1 : a0, *sm_ = cur ? s1 : s0, *c = cur ? c1 : c0, *d = cur ? d1 : d0;
    S *an = cur ? a0 : a1, *sn = cur ? s0 : s1, *cn = cur ? c0 : c1, *dn = cur ? d0 : d1;
    for (int q = threadIdx.x; q < n; q += NT) {
      const S aq = a[q], cq = c[q];
      S sq = sm_[q], dq = d[q], na = (S)0, nc = (S)0;
      if (q - k >= 0) {
        const S bm = sm_[q - k] - a[q - k] - c[q - k];
        const S k1 = aq / bm;
        sq -= k1 * sm_[q - k];
        dq -= k1 * d[q - k];
        na = -a[q - k] * k1;
      }
      if (q + k < n) {
        const S bp = sm_[q + k] - a[q + k] - c[q + k];
        const S k2 = cq / bp;
        sq -= k2 * sm_[q + k];
        dq -= k2 * d[q + k];
        nc = -c[q + k] * k2;
      }
      an[q] = na;
      sn[q] = sq;
      cn[q] = nc;
      dn[q] = dq;
    }
    __syncthreads();
    cur ^= 1;
  }
  const S *a = cur ? a1 : a0, *sm_ = cur ? s1 : s0, *c = cur ? c1 : c0, *d = cur ? d1 : d0;
  const int lane = threadIdx.x & 31;
  for (int r = threadIdx.x >> 5; r < ns; r += W) {
    const int q = r + ns * lane;
    const bool on = q < n;  // rows past n: the identity (their neighbours' couplings to them are zero)
    S aq = on ? a[q] : (S)0, sq = on ? sm_[q] : (S)1, cq = on ? c[q] : (S)0, dq = on ? d[q] : (S)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const S am = __shfl_up_sync(kFull, aq, o), smm = __shfl_up_sync(kFull, sq, o);
      const S cm = __shfl_up_sync(kFull, cq, o), dm = __shfl_up_sync(kFull, dq, o);
      const S ap = __shfl_down_sync(kFull, aq, o), spp = __shfl_down_sync(kFull, sq, o);
      const S cp = __shfl_down_sync(kFull, cq, o), dp = __shfl_down_sync(kFull, dq, o);
      S s2 = sq, d2 = dq, na = (S)0, nc = (S)0;
      if (lane >= o) {
        const S bm = smm - am - cm;
        const S k1 = aq / bm;
        s2 -= k1 * smm;
        d2 -= k1 * dm;
        na = -am * k1;
      }
      if (lane + o < 32) {
        const S bp = spp - ap - cp;
        const S k2 = cq / bp;
        s2 -= k2 * spp;
        d2 -= k2 * dp;
        nc = -cp * k2;
      }
      aq = na;
      sq = s2;
      cq = nc;
      dq = d2;
    }
    if (on) out(q, dq / sq);
  }
}

// ---------------------------------------------------------------------------------------
// node solves (all threads of the CTA)
// ---------------------------------------------------------------------------------------

// Block-wide inclusive scan (suffix scan if Reverse) of n values, fused with its producer and
// consumer: in(m) gives element m, out(m, s) receives the scan at m.  Each thread holds up to
// EMAX consecutive elements in registers; warps scan the thread totals with shuffles, and
// after one barrier every warp scans the NT/32 warp totals itself for its offset.  Contains
// one barrier and ends with another.
template <int NT, int EMAX, bool Reverse, class W, class In, class Out>
__device__ __forceinline__ void block_scan_fused(int n, W *wtot, In &&in, Out &&out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  static_assert(NW <= 32, "one warp scans the warp totals");
  const int E = (n + NT - 1) / NT;  // <= EMAX
  const int beg = tid * E;
  W v[EMAX];
  W tot = wide_zero<W>();
#pragma unroll
  for (int j = 0; j < EMAX; ++j) {
    const int q = beg + j;
    v[j] = wide_zero<W>();
    if (j < E && q < n) {
      v[j] = in(Reverse ? n - 1 - q : q);
      tot = wide_add(tot, v[j]);
    }
  }
  W incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const W t = wide_shfl_up(incl, o);
    if (lane >= o) incl = wide_add(incl, t);
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  // this warp's offset: the sum of the totals of the warps before it
  W t = lane < warp ? wtot[lane] : wide_zero<W>();
#pragma unroll
  for (int o = 1; o < NW; o <<= 1) t = wide_add(t, wide_shfl_down(t, o));
  W run = wide_shfl_idx(t, 0);
  const W below = wide_shfl_up(incl, 1);
  if (lane > 0) run = wide_add(run, below);
#pragma unroll
  for (int j = 0; j < EMAX; ++j) {
    const int q = beg + j;
    if (j < E && q < n) {
      run = wide_add(run, v[j]);
      out(Reverse ? n - 1 - q : q, run);
    }
  }
  __syncthreads();
}

// psi from the charge deposit in sm.rho: Phi_m = sum_{i<m} delta_i + alpha_m delta_m,
// psi'_m = Phi_m / r_m, psi(R) = 0, psi = inward trapezoid sum of psi'.  Ends with a barrier.
template <class Pol, int NT>
__device__ __forceinline__ void solve_psi(MarchSmem<Pol> &sm, const NodeGeo<Pol> &geo, typename Pol::W *wtot) {
  using R = typename Pol::N;
  using W = typename Pol::W;
  const int nr = geo.nr, n1 = nr + 1;
  block_scan_fused<NT, Pol::kScanE, false, W>(
      n1, wtot, [&](int m) { return q_to_wide<typename Pol::Q, W>(sm.rho[m] - sm.rho0[m]); },
      [&](int m, W incl) {
        R dp = (R)0;
        if (m > 0) {
          const R v = (R)wide_value(q_to_wide<typename Pol::Q, W>(sm.rho[m] - sm.rho0[m]));
          dp = (R)wide_value(wide_add(incl, wide_of<W, R>(-((R)1 - geo.alpha(m)) * v))) * geo.metric(m);
        }
        sm.dpsi[m] = dp;
      });
  const R hdr = (R)0.5 * geo.dr;
  block_scan_fused<NT, Pol::kScanE, true, W>(
      n1, wtot, [&](int m) { return wide_of<W, R>(m < nr ? hdr * (sm.dpsi[m] + sm.dpsi[m + 1]) : (R)0); },
      [&](int m, W incl) { sm.psi[m] = -(R)wide_value(incl); });
}

// E_z, the Helmholtz system for B_theta and its PCR solve, from the current-type deposits
// and the beam-density rows nbA, nbB (averaged).  Ends with a barrier.
template <class Pol, int NT>
__device__ __forceinline__ void solve_fields(MarchSmem<Pol> &sm, const NodeGeo<Pol> &geo, const typename Pol::R *nbA,
                                             const typename Pol::R *nbB, typename Pol::W *wtot) {
  using R = typename Pol::N;
  using W = typename Pol::W;
  using Acc = typename Pol::Acc;
  const int tid = threadIdx.x, nr = geo.nr, n1 = nr + 1;
  const R inv_dr = geo.inv_dr, hdr = (R)0.5 * geo.dr;
  // d_xi psi'_m = -((1 - alpha_m) K_{m-1} + alpha_m K_m) / (dr r_m), from the K deposits
  auto dxi_dpsi = [&](int m) -> R {
    if (m == 0) return (R)0;
    const R al = geo.alpha(m);
    const R Km = m < nr ? (R)sm.K[m] : (R)0;
    return -(((R)1 - al) * (R)sm.K[m - 1] + al * Km) * geo.metric(m) * inv_dr;
  };
  // E_z: inward trapezoid sum from E_z(R) = 0
  block_scan_fused<NT, Pol::kScanE, true, W>(
      n1, wtot, [&](int m) { return wide_of<W, R>(m < nr ? hdr * (dxi_dpsi(m) + dxi_dpsi(m + 1)) : (R)0); },
      [&](int m, W incl) { sm.ez[m] = -(R)wide_value(incl); });
  // node densities (deposit / hat volume; J_z less the beam density averaged over the two
  // rows) read where the rows need them
  auto dens = [&](const Acc *v, int m) -> R { return (R)v[m] * geo.invV(m); };
  auto jz_node = [&](int m) -> R { return (R)sm.jz[m] * geo.invV(m) - (R)0.5 * ((R)nbA[m] + (R)nbB[m]); };
  // rows q = 0..nr-1 (node i = q + 1): central differences, a half cell at the wall
  const R i2dr = (R)0.5 * inv_dr;
  for (int q = tid; q < nr; q += NT) {
    const int i = q + 1;
    const R Qi = dens(sm.P, i) + sm.ez[i] * dens(sm.U, i);
    const R Ti = dens(sm.T, i);
    R a, c, sgeo;
    geo.row(q, a, c, sgeo);
    R rhs;
    if (i < nr)
      rhs = (jz_node(i + 1) - jz_node(i - 1)) * i2dr + Qi + (dens(sm.T, i + 1) - dens(sm.T, i - 1)) * i2dr +
            Ti * geo.curv(i);
    else
      rhs = Qi + (Ti - dens(sm.T, i - 1)) * inv_dr + Ti * geo.curv(i) - (jz_node(i - 1) + jz_node(i)) * inv_dr;
    sm.ta[q] = a;
    sm.tb[q] = sgeo - dens(sm.chi, i);  // row sum a + b + c (both terms negative)
    sm.tc[q] = c;
    sm.td[q] = rhs;
  }
  __syncthreads();
  // parallel cyclic reduction (on row sums); the second buffer reuses the deposit arrays J_z, chi, T, P,
  // which are dead once the rows are set up (they are zeroed before the next pass B)
  static_assert(sizeof(Acc) == sizeof(R), "PCR buffer reuses deposit arrays");
  if constexpr (Pol::kWarpPCR) {
    pcr_rowsum_solve<NT, R>(sm.ta, sm.tb, sm.tc, sm.td, (R *)sm.jz, (R *)sm.chi, (R *)sm.T, (R *)sm.P, nr,
                            [&](int q, R x) { sm.bth[q + 1] = x; });  // row q is node q + 1
    if (tid == 0) sm.bth[0] = (R)0;
  } else {
    const int cur = pcr_rowsum<NT, R>(sm.ta, sm.tb, sm.tc, sm.td, (R *)sm.jz, (R *)sm.chi, (R *)sm.T, (R *)sm.P, nr);
    const R *bb = cur ? (const R *)sm.chi : sm.tb, *dd = cur ? (const R *)sm.P : sm.td;  // row sum = diagonal now
    for (int m = tid; m < n1; m += NT) sm.bth[m] = m > 0 ? dd[m - 1] / bb[m - 1] : (R)0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// ring moves and windowed deposits
// ---------------------------------------------------------------------------------------

// Move a ring at radius r = (c + f) dr by the Cartesian displacement (dx, dy) from (r, 0)
// and give it the Cartesian momentum (ux, uy).  The new radius is formed as the exact
// increment r' - r = (dx (2r + dx) + dy^2) / (r' + r), applied to the cell offset, so no
// precision is lost to the size of r.  Returns the new cell (cn, fn), the radius rn, and the
// radial / azimuthal momenta; a ring beyond the wall r = nr dr is reflected specularly.
template <class R>
__device__ __forceinline__ void move_ring(int c, R f, R r, R dx, R dy, R ux, R uy, R inv_dr, R dr, int nr,
                                          int &cn, R &fn, R &rn, R &urn, R &utn) {
  const R xn = r + dx, yn = dy;
  const R rr = sqrt(xn * xn + yn * yn);
  const R den = rr + r;
  const R delta = den > (R)0 ? (dx * ((R)2 * r + dx) + dy * dy) / den : (R)0;
  R s = f + delta * inv_dr;  // offset from node c, in cells
  if (rr > (R)0) {
    const R irr = (R)1 / rr;
    urn = (xn * ux + yn * uy) * irr;
    utn = (xn * uy - yn * ux) * irr;
  } else {
    urn = sqrt(ux * ux + uy * uy);
    utn = (R)0;
  }
  if ((R)c + s > (R)nr) {  // specular reflection at the wall: r'/dr -> 2 nr - r'/dr
    s = (R)(2 * (nr - c)) - s;
    urn = -urn;
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
  rn = ((R)ci + fo) * dr;
}

// Window of three cells c0..c0+2 (four nodes) summed in registers; a ring outside the
// window deposits directly.
template <class R, int NV>
struct WindowAcc {
  int c0 = -1;
  R n[4][NV];
  __device__ __forceinline__ void init(int c) {
    c0 = c;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < NV; ++q) n[a][q] = (R)0;
  }
  // the hat weights (1 - f, f) placed on the window's nodes o, o + 1 once, then one
  // multiply-add per node and value
  __device__ __forceinline__ bool add(int c, R f, const R (&v)[NV]) {
    const int o = c - c0;
    if (o < 0 || o > 2) return false;
    const R g = (R)1 - f;
    const R w0 = o == 0 ? g : (R)0, w1 = o == 0 ? f : (o == 1 ? g : (R)0);
    const R w2 = o == 1 ? f : (o == 2 ? g : (R)0), w3 = o == 2 ? f : (R)0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      n[0][q] += v[q] * w0;
      n[1][q] += v[q] * w1;
      n[2][q] += v[q] * w2;
      n[3][q] += v[q] * w3;
    }
    return true;
  }
};

// Warp segments: maximal runs of consecutive lanes with the same key (a window's first
// cell).  sum() is the inclusive segmented sum from the segment's head; the segment's tail
// lane then holds the total, so one lane per segment issues the shared-memory atomics
// (same-address atomics of one instruction serialise).
struct WarpSeg {
  int lane, seg_start, tail_lane, max_len;
  bool is_tail;
  __device__ __forceinline__ explicit WarpSeg(int key) {
    lane = threadIdx.x & 31;
    const int kprev = __shfl_up_sync(kFull, key, 1);
    const int knext = __shfl_down_sync(kFull, key, 1);
    const bool head = lane == 0 || kprev != key;
    is_tail = lane == 31 || knext != key;
    const unsigned heads = __ballot_sync(kFull, head);
    const unsigned tails = __ballot_sync(kFull, is_tail);
    seg_start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    tail_lane = __ffs(tails & (0xffffffffu << lane)) - 1;
    max_len = __reduce_max_sync(kFull, (unsigned)(lane - seg_start + 1));
  }
  // Inclusive segmented sums of N values from the segment's head, in place.  The strides
  // double while they are below the warp's longest segment: a longer stride would add
  // nothing (no lane is that far into its segment), so the sums equal those of all five
  // steps.  The bound is warp-uniform.
  template <class T, int N>
  __device__ __forceinline__ void sum_n(T (&v)[N]) const {
    for (int o = 1; o < max_len; o <<= 1) {
      const bool take = lane - o >= seg_start;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const T u = __shfl_up_sync(kFull, v[i], o);
        if (take) v[i] += u;
      }
    }
  }
};

// A ring's charge contributions to the node pair (c, c+1) in the form's charge-window type.
template <class Pol>
struct ChargeWin;
template <>
struct ChargeWin<PolFP64> {
  int c0 = -1;
  double n[4];
  __device__ __forceinline__ void init(int c) {
    c0 = c;
    n[0] = n[1] = n[2] = n[3] = 0.0;
  }
  __device__ __forceinline__ bool add(int c, double f, double w) {
    const int o = c - c0;
    if (o < 0 || o > 2) return false;
    const double lo = w * (1.0 - f), hi = w * f;
    n[0] += o == 0 ? lo : 0.0;
    n[1] += o == 0 ? hi : (o == 1 ? lo : 0.0);
    n[2] += o == 1 ? hi : (o == 2 ? lo : 0.0);
    n[3] += o == 2 ? hi : 0.0;
    return true;
  }
  __device__ __forceinline__ static void direct(double *rho, int c, double f, double w) {
    atomicAdd(&rho[c], w * (1.0 - f));
    atomicAdd(&rho[c + 1], w * f);
  }
  __device__ __forceinline__ double node(int a) const { return n[a]; }
};
template <>
struct ChargeWin<PolMixed> {
  int c0 = -1;
  long long n[4];
  __device__ __forceinline__ void init(int c) {
    c0 = c;
    n[0] = n[1] = n[2] = n[3] = 0;
  }
  // w f as an exact float-float product, w and w f in fixed point, w (1 - f) = w - w f there
  __device__ __forceinline__ static void split(float f, float w, long long &qlo, long long &qhi) {
    const FF hi = two_prod(w, f);
    qhi = ff_to_q(hi);
    qlo = f2q(w * (float)kQScale) - qhi;
  }
  __device__ __forceinline__ bool add(int c, float f, float w) {
    const int o = c - c0;
    if (o < 0 || o > 2) return false;
    long long lo, hi;
    split(f, w, lo, hi);
    n[0] += o == 0 ? lo : 0ll;
    n[1] += o == 0 ? hi : (o == 1 ? lo : 0ll);
    n[2] += o == 1 ? hi : (o == 2 ? lo : 0ll);
    n[3] += o == 2 ? hi : 0ll;
    return true;
  }
  __device__ __forceinline__ static void direct(long long *rho, int c, float f, float w) {
    long long lo, hi;
    split(f, w, lo, hi);
    atomicAdd((unsigned long long *)&rho[c], (unsigned long long)lo);
    atomicAdd((unsigned long long *)&rho[c + 1], (unsigned long long)hi);
  }
  __device__ __forceinline__ long long node(int a) const { return n[a]; }
};

template <>
struct ChargeWin<PolWide> : ChargeWin<PolMixed> {};
template <>
struct ChargeWin<PolMixed64> : ChargeWin<PolMixed> {};
template <>
struct ChargeWin<PolWideFP64> : ChargeWin<PolFP64> {};
template <class P>
struct ChargeWin<SlabOf<P>> : ChargeWin<P> {};


__device__ __forceinline__ void q_atomic_add(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void q_atomic_add(long long *p, long long v) {
  atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

// Flush a charge window into rho over the warp.  All lanes of the warp call it.
template <class Pol>
__device__ __forceinline__ void flush_charge(MarchSmem<Pol> &sm, const ChargeWin<Pol> &acc, int nr) {
  using Q = typename Pol::Q;
  const WarpSeg seg(acc.c0);
  Q t[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) t[a] = acc.node(a);
  seg.sum_n(t);
#pragma unroll
  for (int a = 0; a < 4; ++a)  // a node no ring of the segment touched is not added to
    if (seg.is_tail && acc.c0 >= 0 && acc.c0 + a <= nr && t[a] != (Q)0) q_atomic_add(&sm.rho[acc.c0 + a], t[a]);
}

// Charge deposit of one ring through a window (direct atomics outside it).
template <class Pol>
__device__ __forceinline__ void add_charge(MarchSmem<Pol> &sm, ChargeWin<Pol> &acc, int p, int c,
                                           typename Pol::R f, typename Pol::R w) {
  if (p == 0) acc.init(c);
  if (!acc.add(c, f, w)) ChargeWin<Pol>::direct(sm.rho, c, f, w);
}
// Charge deposit of ring p through the window; a ring outside it is marked in miss (bit p) and
// left to warp_misses.
template <class Pol>
__device__ __forceinline__ void add_charge_mark(MarchSmem<Pol> &sm, ChargeWin<Pol> &acc, int p, int c,
                                                typename Pol::R f, typename Pol::R w, unsigned &miss) {
  if (p == 0) acc.init(c);
  if (!acc.add(c, f, w)) {
    if constexpr (Pol::kDeferMisses)
      miss |= 1u << p;
    else
      ChargeWin<Pol>::direct(sm.rho, c, f, w);  // the policy deposits in the loop
  }
}

// ---------------------------------------------------------------------------------------
// ring passes
// ---------------------------------------------------------------------------------------

// The i-th (from 0) out-of-window ring of the warp, counted ring index p first and lane second,
// when mp[p] holds the lanes that marked ring p: returns its slot.
template <int NT, int PPT>
__device__ __forceinline__ int warp_miss_slot(const unsigned (&mp)[PPT], int i) {
  int before = 0, pp = 0, rank = 0;
  unsigned m = 0u;
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const int n = __popc(mp[p]);
    if (i >= before && i < before + n) {
      pp = p;
      rank = i - before;
      m = mp[p];
    }
    before += n;
  }
  for (int r = 0; r < rank; ++r) m &= m - 1u;  // drop the rank lowest lanes
  return pp * NT + (int)(threadIdx.x & ~31u) + (__ffs(m) - 1);
}

// Marks of the thread's out-of-window rings (bit p: ring p), shared over the warp: lane l
// handles the warp's l-th, (l+32)-th, ... marked ring through fn(slot).  All lanes call.
template <int NT, int PPT, class Fn>
__device__ __forceinline__ void warp_misses(unsigned miss, Fn &&fn) {
  unsigned mp[PPT];
  int tot = 0;
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    mp[p] = __ballot_sync(kFull, (miss >> p) & 1u);
    tot += __popc(mp[p]);
  }
  if (tot == 0) return;
  __syncwarp();  // the slots the owners wrote in the pass are visible to the warp
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < tot; i0 += 32)
    if (i0 + lane < tot) fn(warp_miss_slot<NT, PPT>(mp, i0 + lane));
}

// The same marks handed to the whole CTA: the warp reserves entries of the queue (one shared
// atomic) and stores the marked rings' slots; drain_queue, after the pass's barrier, spreads
// them over all warps.  Rings past the queue's capacity are handled by the warp through
// fn(slot).  All lanes call.
template <int NT, int PPT, class Pol, class Fn>
__device__ __forceinline__ void queue_misses(MarchSmem<Pol> &sm, int n1, unsigned miss, Fn &&fn) {
  unsigned mp[PPT];
  int tot = 0;
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    mp[p] = __ballot_sync(kFull, (miss >> p) & 1u);
    tot += __popc(mp[p]);
  }
  if (tot == 0) return;
  const int lane = threadIdx.x & 31, cap = sm.queue_cap(n1);
  int base = 0;
  if (lane == 0) base = atomicAdd(sm.qn, tot);
  base = __shfl_sync(kFull, base, 0);
  int *q = sm.queue();
  __syncwarp();
  for (int i0 = 0; i0 < tot; i0 += 32) {
    const int i = i0 + lane;
    if (i < tot) {
      const int sl = warp_miss_slot<NT, PPT>(mp, i);
      if (base + i < cap)
        q[base + i] = sl;
      else
        fn(sl);
    }
  }
}

// Take the queue's entries over all threads (entry i to warp i mod (NT/32), so that a burst
// of entries from one warp is spread over the CTA), then empty it.  Call after the barrier that
// ends the pass; contains a barrier when the queue is not empty.
template <int NT, class Pol, class Fn>
__device__ __forceinline__ void drain_queue(MarchSmem<Pol> &sm, int n1, Fn &&fn) {
  const int n = min(*sm.qn, sm.queue_cap(n1));
  if (n == 0) return;  // block-uniform
  constexpr int W = NT / 32;
  const int *q = sm.queue();
  for (int i = (threadIdx.x & 31) * W + (threadIdx.x >> 5); i < n; i += NT) fn(q[i]);
  __syncthreads();
  if (threadIdx.x == 0) *sm.qn = 0;
}

// One ring's current-type deposit values (the source terms of Eqs. 4-7: J_z, chi, T, P, U and
// the K share), its Gamma and (gamma/Gamma) psi', at cell c, offset f, momenta (u_r, u_theta).
template <class Pol>
__device__ __forceinline__ void current_values(const MarchSmem<Pol> &sm, const RingSoA<typename Pol::R> &rs, int sl,
                                               int c, typename Pol::R f, typename Pol::R u_r, typename Pol::R u_t,
                                               typename Pol::R dr, int *status, typename Pol::R (&v)[5],
                                               typename Pol::R &ka, typename Pol::R &G, typename Pol::R &g) {
  using R = typename Pol::R;
  constexpr bool slab = Pol::kSlab;
  const R rp = ((R)c + f) * dr;
  G = rs.G0[sl] + interp(sm.psi, c, f);
  if (!(G > (R)0)) flag(status, ST_NUMERIC);
  const R iG = (R)1 / G;
  const R up2 = u_r * u_r + u_t * u_t;
  const R gam = ((R)1 + up2 + G * G) * (R)0.5 * iG;
  const R uz = gam - G;
  const R a = u_r * iG;
  const R dp = interp(sm.dpsi, c, f);
  const R cent = (!slab && rp > (R)0) ? u_t * u_t * iG / rp : (R)0;  // Eq. 4's centrifugal term (cylinder)
  g = gam * iG * dp;
  const R w = rs.w[sl];
  v[0] = -w * uz * iG;
  v[1] = w * iG;
  v[2] = w * a * a;
  v[3] = w * (a * a * dp - g - cent) * iG;
  v[4] = w * a * iG;
  ka = w * a;
}

// The current deposit of one ring straight into the node arrays (shared atomics).
template <class Pol>
__device__ __forceinline__ void current_direct(MarchSmem<Pol> &sm, int c, typename Pol::R f,
                                               const typename Pol::R (&v)[5], typename Pol::R ka) {
  using Acc = typename Pol::Acc;
  const typename Pol::R g0 = (typename Pol::R)1 - f;
  Acc *arr[5] = {sm.jz, sm.chi, sm.T, sm.P, sm.U};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    atomicAdd(&arr[q][c], (Acc)(v[q] * g0));
    atomicAdd(&arr[q][c + 1], (Acc)(v[q] * f));
  }
  atomicAdd(&sm.K[c], (Acc)ka);
}

// A ring outside the window, at slot sl, through the position functor pos_slot: its values
// formed again by the same arithmetic and deposited straight into the node arrays.
template <class Pol, class PosSlot>
__device__ __forceinline__ void current_miss(MarchSmem<Pol> &sm, const RingSoA<typename Pol::R> &rs, int sl,
                                             typename Pol::R dr, int *status, PosSlot &&pos_slot) {
  using R = typename Pol::R;
  int c;
  R f, u_r, u_t, v[5], ka, G, g;
  pos_slot(sl, c, f, u_r, u_t);
  current_values<Pol>(sm, rs, sl, c, f, u_r, u_t, dr, status, v, ka, G, g);
  current_direct<Pol>(sm, c, f, v, ka);
}

// Pass B: ring quantities at the position given by pos(sl, c, f, u_r, u_theta) and the
// current-type deposits.  Gam[p] = Gamma, gq[p] = (gamma/Gamma) psi'(r).  All threads call.
// A ring outside the thread's window is only marked in the loop (an atomic there would order
// every later ring's loads behind it); on_miss(mask) receives the thread's marks after the loop
// (all lanes call it) and sees to those rings' deposits (current_miss).
template <class Pol, int NT, int PPT, bool kTrap = false, class Pos, class OnMiss>
__device__ __forceinline__ void pass_currents(MarchSmem<Pol> &sm, const RingSoA<typename Pol::R> &rs, int np,
                                              int nr, typename Pol::R dr, int *status, Pos &&pos, OnMiss &&on_miss,
                                              typename Pol::R (&Gam)[PPT], typename Pol::R (&gq)[PPT]) {
  using R = typename Pol::R;
  using Acc = typename Pol::Acc;
  const int t = threadIdx.x;
  WindowAcc<R, 5> acc;
  acc.init(-8);
  R kw[3] = {(R)0, (R)0, (R)0};
  unsigned miss = 0u;
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    Gam[p] = (R)1;
    gq[p] = (R)0;
    if (t * PPT + p < np) {
      const int sl = p * NT + t;
      int c;
      R f, u_r, u_t;
      if constexpr (std::is_invocable_v<Pos, int, int, int &, R &, R &, R &>)
        pos(p, sl, c, f, u_r, u_t);
      else
        pos(sl, c, f, u_r, u_t);
      if (p == 0) acc.init(c);
      if constexpr (kTrap)
        if (rs.w[sl] == (R)0) continue;  // promoted to a beam particle: no longer in the plasma
      R v[5], ka, G, g;
      current_values<Pol>(sm, rs, sl, c, f, u_r, u_t, dr, status, v, ka, G, g);
      if (acc.add(c, f, v)) {
        const int o = c - acc.c0;
        kw[0] += o == 0 ? ka : (R)0;
        kw[1] += o == 1 ? ka : (R)0;
        kw[2] += o == 2 ? ka : (R)0;
      } else if constexpr (Pol::kDeferMisses) {
        miss |= 1u << p;
      } else {
        current_direct<Pol>(sm, c, f, v, ka);
      }
      Gam[p] = G;
      gq[p] = g;
    }
  }
  if constexpr (Pol::kDeferMisses) on_miss(miss);
  const WarpSeg seg(acc.c0);
  const int c = acc.c0;
  const bool emit = seg.is_tail && c >= 0;
  Acc tot[23];  // the thread's window sums, then summed across rings in the deposit type
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int a = 0; a < 4; ++a) tot[q * 4 + a] = (Acc)acc.n[a][q];
#pragma unroll
  for (int a = 0; a < 3; ++a) tot[20 + a] = (Acc)kw[a];
  seg.sum_n(tot);
  // The window's last nodes are often untouched (a thread's rings span one or two cells where
  // the plasma is dense), and the shared-memory adds are the pass's costliest part: zero sums
  // are not added.
  Acc *arr[5] = {sm.jz, sm.chi, sm.T, sm.P, sm.U};
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (emit && c + a <= nr && tot[q * 4 + a] != (Acc)0) atomicAdd(&arr[q][c + a], (Acc)tot[q * 4 + a]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (emit && c + a < nr && tot[20 + a] != (Acc)0) atomicAdd(&sm.K[c + a], (Acc)tot[20 + a]);
}

// Re-sort the rings of the CTA by cell (counting sort) so that each thread's rings are
// consecutive in radius again.  Rings in the three cells c0..c0+2 of the thread's first ring
// are counted in registers, combined over warp segments and take their bases with one atomic
// per cell and segment; others take a rank with their own atomic.  The slot arrays are
// permuted in place through registers.  Order within a cell follows the atomics.
template <class Pol, int NT, int PPT, bool kIds = false>
__device__ __forceinline__ void resort_rings(MarchSmem<Pol> &sm, const RingSoA<typename Pol::R> &rs, int np, int nr) {
  using R = typename Pol::R;
  const int t = threadIdx.x, n1 = nr + 1;
  for (int m = t; m < n1; m += NT) sm.cnt[m] = 0;
  int rc[PPT], rid[kIds ? PPT : 1];
  R rf[PPT], rur[PPT], rlz[PPT], rG0[PPT], rw[PPT];
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    rc[p] = 0;
    rf[p] = rur[p] = rlz[p] = rG0[p] = rw[p] = (R)0;
    if constexpr (kIds) rid[p] = 0;
    if (t * PPT + p < np) {
      const int sl = p * NT + t;
      rc[p] = rs.c[sl];
      rf[p] = rs.f[sl];
      rur[p] = rs.ur[sl];
      rlz[p] = rs.lz[sl];
      rG0[p] = rs.G0[sl];
      rw[p] = rs.w[sl];
      if constexpr (kIds) rid[p] = rs.id[sl];
    }
  }
  __syncthreads();
  int rank[PPT];
  {
    const int c0 = t * PPT < np ? rc[0] : -8;
    int cw[3] = {0, 0, 0};
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      rank[p] = 0;
      if (t * PPT + p < np) {
        const int o = rc[p] - c0;
        if (o >= 0 && o <= 2) {
          rank[p] = o == 0 ? cw[0] : (o == 1 ? cw[1] : cw[2]);
          cw[0] += o == 0;
          cw[1] += o == 1;
          cw[2] += o == 2;
        } else {
          rank[p] = atomicAdd(&sm.cnt[rc[p]], 1) | (1 << 30);
        }
      }
    }
    const WarpSeg seg(c0);
    int base[3], inc[3] = {cw[0], cw[1], cw[2]};
    seg.sum_n(inc);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int incl = inc[a];
      int b = 0;
      if (seg.is_tail && c0 >= 0 && c0 + a < nr && incl > 0) b = atomicAdd(&sm.cnt[c0 + a], incl);
      b = __shfl_sync(kFull, b, seg.tail_lane);
      base[a] = b + incl - cw[a];
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p)
      if (t * PPT + p < np) {
        if (rank[p] & (1 << 30)) {
          rank[p] &= ~(1 << 30);
        } else {
          const int o = rc[p] - c0;
          rank[p] += o == 0 ? base[0] : (o == 1 ? base[1] : base[2]);
        }
      }
  }
  __syncthreads();
  // exclusive scan of the counts (warp 0)
  if (t < 32) {
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
  // scatter: rank r goes to thread r / PPT, ring r % PPT, slot (r % PPT) * NT + r / PPT
#pragma unroll
  for (int p = 0; p < PPT; ++p)
    if (t * PPT + p < np) {
      const int r = sm.cnt[rc[p]] + rank[p];
      const int sl = (r % PPT) * NT + r / PPT;
      rs.c[sl] = rc[p];
      rs.f[sl] = rf[p];
      rs.ur[sl] = rur[p];
      rs.lz[sl] = rlz[p];
      rs.G0[sl] = rG0[p];
      rs.w[sl] = rw[p];
      if constexpr (kIds) rs.id[sl] = rid[p];
    }
  __syncthreads();
}

// The march of one simulation by one CTA.  Hooks supply the beam-density rows and receive
// each slice's fields (see PlainHooks; the pipelined beam step adds its own):
//   bool wait_rows(int k)           rows k, k+1 may be read (false: give up, block-uniform)
//   R    nb_row(int row, int m)     beam density at node m of a row
//   void slice_done(int k, sm)      stage-1 fields of slice k are in sm (psi, dpsi, ez, bth)
//   void finish(sm)                 after the last slice
//   kTraj, ring_state<NT, PPT>(k, rs, np)
//                                   (kTraj true only) the slice-k state of the thread's own
//                                   rings, with their stage-1 Gamma in rs.G1; the slots carry
//                                   ring ids
//   kTrap, trap_rings<NT, PPT>(k, rs, np)
//                                   (kTrap true only) after slice k's stage-1 pass: the hook may
//                                   promote the thread's own rings (their weight set to zero);
//                                   a ring of zero weight no longer takes part or moves
template <class Pol, int NT, int PPT, class Hooks>
__device__ __forceinline__ void march_body(const SimDesc &d, unsigned char *smem_raw, Hooks &hk) {
  using R = typename Pol::R;
  using G = typename Pol::G;
  using Acc = typename Pol::Acc;
  const int tid = threadIdx.x, nr = d.nr, n1 = nr + 1, np = d.np, nxi = d.nxi;
  constexpr int SLOTS = NT * PPT;
  constexpr bool kTrap = Hooks::kTrap;
  constexpr bool kIds = Hooks::kTraj || kTrap;
  MarchSmem<Pol> sm;
  sm.carve(smem_raw, n1, SLOTS, kIds);
  RingSoA<R> rs;
  if (Pol::kSmemRings)
    rs = sm.rings;
  else
    rs.carve(d.ring_buf, SLOTS, kIds);
  const double drd = d.dr;
  const R h = (R)d.dxi, R_wall = (R)d.rmax, dR = (R)drd, inv_dr = (R)(1.0 / drd);
  using N = typename Pol::N;
  constexpr bool slab = Pol::kSlab;
  if ((d.slab != 0) != slab) {  // a descriptor of the other geometry: refuse, touch nothing
    if (tid == 0) flag(d.status, ST_NUMERIC);
    return;
  }
  const NodeGeo<Pol> geo{sm.invR, sm.invV, sm.alpha, sm.ga, sm.gb, sm.gc, nr, (N)drd, (N)(1.0 / drd), (N)(1.0 / (drd * drd)),
                          (N)(drd / 6.0), (N)(1.0 / (0.5 * nr - 1.0 / 6.0))};
  fill_tables<Pol, NT>(sm, nr, drd);
  for (int m = tid; m < n1; m += NT) {
    sm.rho[m] = (typename Pol::Q)0;
    sm.jz[m] = sm.chi[m] = sm.T[m] = sm.P[m] = sm.U[m] = sm.K[m] = (Acc)0;
  }
  if (tid == 0) *sm.qn = 0;
  // rings: thread t holds rings t*PPT .. t*PPT+PPT-1 (consecutive in radius), slot p*NT + t.
  // A ring's radius is a cell index c and an offset f in [0,1] (r = (c + f) dr), so its
  // position resolution is uniform over the box; moves are exact radial displacements.
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const int j = tid * PPT + p, sl = p * NT + tid;
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
      if constexpr (kIds) rs.id[sl] = j;
    }
  }
  __syncthreads();

  // positions of the stages: the slice state (stage 1), and the midpoint reached from it with
  // the stage-1 derivative in the local Cartesian frame (x, y) = (r, 0), (u_x, u_y) =
  // (u_r, u_theta) (stage 2), computed once per slice in the midpoint deposit and kept in
  // registers for stage 2 and the full step
  // u_theta = l_z / r; in the slab, lz holds the conserved u_y, which enters gamma only and
  // moves nothing (d/dy = 0): the Cartesian frame below is then the x line, and r = |x| puts a
  // sheet that crosses x = 0 in place of its mirror image
  auto state_pos = [&](int sl, int &c, R &f, R &u_r, R &u_t) {
    c = rs.c[sl];
    f = rs.f[sl];
    u_r = rs.ur[sl];
    const R r = ((R)c + f) * dR;
    u_t = slab ? rs.lz[sl] : (r > (R)0 ? rs.lz[sl] / r : (R)0);
  };
  auto midpoint = [&](int sl, int &c, R &f, R &u_r, R &u_t) -> R {
    const int c0 = rs.c[sl];
    const R f0 = rs.f[sl], ur0 = rs.ur[sl];
    const R r = ((R)c0 + f0) * dR;
    const R ut = slab ? (R)0 : (r > (R)0 ? rs.lz[sl] / r : (R)0);  // the frame's y momentum
    const R iG = (R)1 / rs.G1[sl];
    const R dx = (R)0.5 * h * ur0 * iG, dy = (R)0.5 * h * ut * iG;
    const R uxh = ur0 + (R)0.5 * h * rs.F1[sl];
    R rr;
    move_ring<R>(c0, f0, r, dx, dy, uxh, ut, inv_dr, dR, nr, c, f, rr, u_r, u_t);
    if (slab) u_t = rs.lz[sl];
    return rr;
  };
  auto mid_slot = [&](int sl, int &c, R &f, R &u_r, R &u_t) { midpoint(sl, c, f, u_r, u_t); };
  // out-of-window rings: those of the current passes queued and drained by the CTA after the
  // pass, those of the charge passes (two atomics each) deposited by their own warp
  auto cur_miss1 = [&](int sl) { current_miss<Pol>(sm, rs, sl, dR, d.status, state_pos); };
  auto cur_miss2 = [&](int sl) { current_miss<Pol>(sm, rs, sl, dR, d.status, mid_slot); };
  auto chg_miss_mid = [&](int sl) {
    const R w = rs.w[sl];
    if (kTrap && w == (R)0) return;  // a promoted ring deposits nothing
    int c;
    R f, u_r, u_t;
    midpoint(sl, c, f, u_r, u_t);
    ChargeWin<Pol>::direct(sm.rho, c, f, w);
  };
  auto chg_miss_full = [&](int sl) {  // the new positions are in the slots
    const R w = rs.w[sl];
    if (w != (R)0) ChargeWin<Pol>::direct(sm.rho, rs.c[sl], rs.f[sl], w);
  };

  // charge of the initial slice; it is also the ion background (the deposit of the
  // unperturbed electrons), so psi starts exactly at zero
  {
    ChargeWin<Pol> acc;
    acc.init(-8);
#pragma unroll
    for (int p = 0; p < PPT; ++p)
      if (tid * PPT + p < np) {
        const int sl = p * NT + tid;
        add_charge<Pol>(sm, acc, p, rs.c[sl], rs.f[sl], rs.w[sl]);
      }
    flush_charge<Pol>(sm, acc, nr);
  }
  __syncthreads();
  for (int m = tid; m < n1; m += NT) sm.rho0[m] = sm.rho[m];
  __syncthreads();

  R G2[PPT], F2[PPT];
  for (int k = 0; k <= nxi; ++k) {
    if (Pol::kSortEvery > 0 && k > 0 && k % Pol::kSortEvery == 0) resort_rings<Pol, NT, PPT, kIds>(sm, rs, np, nr);
    const R *nbk = (k & 1) ? sm.nb1 : sm.nb0, *nbk1 = (k & 1) ? sm.nb0 : sm.nb1;
    if (!hk.wait_rows(k)) break;
    if (k == 0)  // row 0 is first read in P2, after two barriers
      for (int m = tid; m < n1; m += NT) sm.nb0[m] = hk.nb_row(0, m);
    // prefetch beam-density row k+1 (stored in phase P1); n1 <= 3 NT
    R pre[3] = {(R)0, (R)0, (R)0};
    if (k < nxi) {
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (tid + q * NT < n1) pre[q] = hk.nb_row(k + 1, tid + q * NT);
    }
    // ======== stage 1 at xi_k ========
    solve_psi<Pol, NT>(sm, geo, sm.wtot);  // P0
    __syncthreads();
    if (k < nxi) {  // P1
      R *dst = (k & 1) ? sm.nb0 : sm.nb1;
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (tid + q * NT < n1) dst[tid + q * NT] = pre[q];
    }
    for (int i = tid; i < n1; i += NT) sm.rho[i] = (typename Pol::Q)0;
    {
      R Gs[PPT], gqs[PPT];
      pass_currents<Pol, NT, PPT, kTrap>(
          sm, rs, np, nr, dR, d.status, state_pos,
          [&](unsigned miss) { queue_misses<NT, PPT>(sm, n1, miss, cur_miss1); }, Gs, gqs);
#pragma unroll
      for (int p = 0; p < PPT; ++p)
        if (tid * PPT + p < np) {
          rs.G1[p * NT + tid] = Gs[p];
          rs.F1[p * NT + tid] = gqs[p];
        }
      if constexpr (Hooks::kTraj) hk.template ring_state<NT, PPT>(k, rs, np);
    }
    __syncthreads();
    drain_queue<NT>(sm, n1, cur_miss1);
    if constexpr (kTrap) hk.template trap_rings<NT, PPT>(k, rs, np);  // after every stage-1 deposit
    solve_fields<Pol, NT>(sm, geo, nbk, nbk, sm.wtot);  // P2
    __syncthreads();
    // P3: fields of slice k, then the move to the midpoint and its charge deposit
    hk.slice_done(k, sm);
    if (k == nxi) break;
    for (int i = tid; i < n1; i += NT) sm.jz[i] = sm.chi[i] = sm.T[i] = sm.P[i] = sm.U[i] = sm.K[i] = (Acc)0;
    // the midpoint of each ring, kept in registers for stage 2 and the full step
    int MC[PPT];
    R MF[PPT], MUR[PPT], MUT[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      MC[p] = 0;
      MF[p] = MUR[p] = MUT[p] = (R)0;
    }
    {
      ChargeWin<Pol> acc;
      acc.init(-8);
      unsigned miss = 0u;
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        if (tid * PPT + p < np) {
          const int sl = p * NT + tid;
          rs.F1[sl] = rs.F1[sl] - interp(sm.bth, rs.c[sl], rs.f[sl]);
          int c;
          R f, u_r, u_t;
          R rr;
          if (kTrap && rs.w[sl] == (R)0) {  // a promoted ring stays where it is
            state_pos(sl, c, f, u_r, u_t);
            rr = ((R)c + f) * dR;
          } else {
            rr = midpoint(sl, c, f, u_r, u_t);
          }
          if (!(rr >= (R)0 && rr <= R_wall)) flag(d.status, ST_ESCAPE);
          MC[p] = c;
          MF[p] = f;
          MUR[p] = u_r;
          MUT[p] = u_t;
          add_charge_mark<Pol>(sm, acc, p, c, f, rs.w[sl], miss);
        }
      }
      warp_misses<NT, PPT>(miss, chg_miss_mid);
      flush_charge<Pol>(sm, acc, nr);
    }
    __syncthreads();
    // ======== stage 2 at xi_k + dxi/2 ========
    solve_psi<Pol, NT>(sm, geo, sm.wtot);  // P0
    __syncthreads();
    for (int i = tid; i < n1; i += NT) sm.rho[i] = (typename Pol::Q)0;  // P1
    pass_currents<Pol, NT, PPT, kTrap>(sm, rs, np, nr, dR, d.status,
                                [&](int p, int, int &c, R &f, R &u_r, R &u_t) {
                                  c = MC[p];
                                  f = MF[p];
                                  u_r = MUR[p];
                                  u_t = MUT[p];
                                },
                                [&](unsigned miss) { queue_misses<NT, PPT>(sm, n1, miss, cur_miss2); }, G2, F2);
    __syncthreads();
    drain_queue<NT>(sm, n1, cur_miss2);
    solve_fields<Pol, NT>(sm, geo, nbk, nbk1, sm.wtot);  // P2
    __syncthreads();
    // P3: full step from the slice-k state with the midpoint derivative, and the charge
    // deposit of the new slice
    for (int i = tid; i < n1; i += NT) sm.jz[i] = sm.chi[i] = sm.T[i] = sm.P[i] = sm.U[i] = sm.K[i] = (Acc)0;
    {
      ChargeWin<Pol> acc;
      acc.init(-8);
      unsigned miss = 0u;
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        if (tid * PPT + p < np) {
          const int sl = p * NT + tid;
          if (kTrap && rs.w[sl] == (R)0) {  // a promoted ring: no move, no charge
            add_charge_mark<Pol>(sm, acc, p, rs.c[sl], rs.f[sl], (R)0, miss);
            continue;
          }
          const R F2b = F2[p] - interp(sm.bth, MC[p], MF[p]);  // at the midpoint
          const int c0 = rs.c[sl];
          const R f0 = rs.f[sl], ur0 = rs.ur[sl], G1v = rs.G1[sl], F1v = rs.F1[sl];
          const R r = ((R)c0 + f0) * dR;
          const R ut = slab ? (R)0 : (r > (R)0 ? rs.lz[sl] / r : (R)0);  // the frame's y momentum
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
          const R iG2 = (R)1 / G2[p];
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
      warp_misses<NT, PPT>(miss, chg_miss_full);
      flush_charge<Pol>(sm, acc, nr);
    }
    __syncthreads();
  }
  hk.finish(sm);
}

// Plain march: beam density from the simulation's grid, fields to its output grids.
template <class Pol, int NT>
struct PlainHooks {
  using R = typename Pol::R;
  using G = typename Pol::G;
  static constexpr bool kTraj = false;
  static constexpr bool kTrap = false;
  const G *nb;
  G *opsi, *oez, *oer, *obth;
  int n1;
  int *status;
  __device__ __forceinline__ bool wait_rows(int) { return true; }
  __device__ __forceinline__ R nb_row(int row, int m) const { return (R)nb[(size_t)row * n1 + m]; }
  __device__ __forceinline__ void slice_done(int k, MarchSmem<Pol> &sm) {
    if (!opsi) return;  // a timing probe of the tile autotuner keeps no output
    G *o1 = opsi + (size_t)k * n1, *o2 = oez + (size_t)k * n1, *o3 = oer + (size_t)k * n1, *o4 = obth + (size_t)k * n1;
    for (int m = threadIdx.x; m < n1; m += NT) {
      const R ps = sm.psi[m], e = sm.ez[m], b = sm.bth[m];
      if (!(isfinite(ps) && isfinite(e) && isfinite(b))) flag(status, ST_NUMERIC);
      o1[m] = (G)ps;
      o2[m] = (G)e;
      o3[m] = m > 0 ? (G)(b - sm.dpsi[m]) : (G)0;
      o4[m] = (G)b;
    }
  }
  __device__ __forceinline__ void finish(MarchSmem<Pol> &) {}
};

// One CTA per simulation.  Tiles of fewer threads ask for more CTAs per SM, within the
// same 128 registers per thread.
template <class Pol, int NT, int PPT>
__global__ void __launch_bounds__(NT, (NT < 512 ? 512 / NT : 1)) march_kernel(const SimDesc *descs, const int *order) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SimDesc &d = descs[order ? order[blockIdx.x] : blockIdx.x];
  PlainHooks<Pol, NT> hk{(const typename Pol::G *)d.nb, (typename Pol::G *)d.psi, (typename Pol::G *)d.ez,
                         (typename Pol::G *)d.er, (typename Pol::G *)d.bth, d.nr + 1, d.status};
  march_body<Pol, NT, PPT>(d, smem_raw, hk);
}

// The plain march that also records the rings' trajectories (Sec. IV, Figs. 4-5): at every
// slice k that is a multiple of `every`, ring j's radius, u_r and Gamma go to
// traj[((k / every) * 3 + q) * np + j], q = 0, 1, 2 (j its index in the initial slice).
template <class Pol, int NT>
struct TrajHooks : PlainHooks<Pol, NT> {
  static constexpr bool kTraj = true;
  double *traj;
  int every;
  double dr;
  template <int NT_, int PPT>
  __device__ __forceinline__ void ring_state(int k, const RingSoA<typename Pol::R> &rs, int np) const {
    if (k % every) return;
    double *row = traj + (size_t)(k / every) * 3 * np;
#pragma unroll
    for (int p = 0; p < PPT; ++p)
      if (threadIdx.x * PPT + p < np) {
        const int sl = p * NT_ + threadIdx.x, j = rs.id[sl];
        row[j] = ((double)rs.c[sl] + (double)rs.f[sl]) * dr;
        row[np + j] = (double)rs.ur[sl];
        row[2 * (size_t)np + j] = (double)rs.G1[sl];
      }
  }
};

// The plain march with plasma-particle trapping (Sec. I: plasma particles past a threshold
// become beam particles).  After slice k's stage-1 pass every ring of nonzero weight whose
// Gamma = Gamma_0 + psi (Eq. 1) is below gamma_t is promoted: its weight drops to zero (it
// still counted in slice k's fields) and an entry (ring j, slice k, r, u_r, u_theta, Gamma, w)
// goes to list[7 q], q taken from *count (entries past cap are counted, not written).
template <class Pol, int NT>
struct TrapHooks : PlainHooks<Pol, NT> {
  using R = typename Pol::R;
  static constexpr bool kTrap = true;
  double gamma_t;
  double *list;
  int *count;
  int cap;
  double dr;
  template <int NT_, int PPT>
  __device__ __forceinline__ void trap_rings(int k, const RingSoA<R> &rs, int np) const {
#pragma unroll
    for (int p = 0; p < PPT; ++p)
      if (threadIdx.x * PPT + p < np) {
        const int sl = p * NT_ + threadIdx.x;
        const R w = rs.w[sl];
        if (w != (R)0 && (double)rs.G1[sl] < gamma_t) {
          const int q = atomicAdd(count, 1);
          if (q < cap) {
            const double r = ((double)rs.c[sl] + (double)rs.f[sl]) * dr;
            double *e = list + 7 * (size_t)q;
            e[0] = (double)rs.id[sl];
            e[1] = (double)k;
            e[2] = r;
            e[3] = (double)rs.ur[sl];
            e[4] = r > 0.0 ? (double)rs.lz[sl] / r : 0.0;
            e[5] = (double)rs.G1[sl];
            e[6] = (double)w;
          }
          rs.w[sl] = (R)0;
        }
      }
  }
};

template <class Pol, int NT, int PPT>
__global__ void __launch_bounds__(NT, 1) march_trap_kernel(const SimDesc *desc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SimDesc &d = *desc;
  TrapHooks<Pol, NT> hk;
  hk.nb = (const typename Pol::G *)d.nb;
  hk.opsi = (typename Pol::G *)d.psi;
  hk.oez = (typename Pol::G *)d.ez;
  hk.oer = (typename Pol::G *)d.er;
  hk.obth = (typename Pol::G *)d.bth;
  hk.n1 = d.nr + 1;
  hk.status = d.status;
  hk.gamma_t = d.gamma_t;
  hk.list = d.trap;
  hk.count = d.trap_count;
  hk.cap = d.trap_cap;
  hk.dr = d.dr;
  march_body<Pol, NT, PPT>(d, smem_raw, hk);
}

template <class Pol, int NT, int PPT>
__global__ void __launch_bounds__(NT, 1) march_traj_kernel(const SimDesc *desc, double *traj, int every) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SimDesc &d = *desc;
  TrajHooks<Pol, NT> hk;
  hk.nb = (const typename Pol::G *)d.nb;
  hk.opsi = (typename Pol::G *)d.psi;
  hk.oez = (typename Pol::G *)d.ez;
  hk.oer = (typename Pol::G *)d.er;
  hk.obth = (typename Pol::G *)d.bth;
  hk.n1 = d.nr + 1;
  hk.status = d.status;
  hk.traj = traj;
  hk.every = every;
  hk.dr = d.dr;
  march_body<Pol, NT, PPT>(d, smem_raw, hk);
}

}  // namespace wake
