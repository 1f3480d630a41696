// Host build of the library's adjoint (paper_1411_3246_gb300/csrc/adjoint_core.h): the same
// forward and reverse bodies the CUDA kernels run, executed by one host thread in the order
// wake_adjoint_forward and wake_adjoint_backward launch them, so that the CPU test suite can
// check the library's gradient against finite differences of the oracle without a GPU.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../include/wake.h"
#include "../paper_1411_3246_gb300/csrc/adjoint_core.h"

using namespace wake::adj;

extern "C" int adj_host_gradient(const wake_params *p, int nsteps, int nbins, const double *theta,
                                 const double *profile, const double *nm_p, const double *nm_b, const double *dobs,
                                 double *obs, double *grad) {
  const Par P{0, 1};
  const int nr = p->nr, n1 = nr + 1, np = p->nr * p->ppc;
  const int64_t n = p->n_beam;
  const Dims g{nr, p->nxi, np, p->rmax / nr, p->ximax / p->nxi, p->rmax};
  const int B = std::max(1, (int)std::lround(std::sqrt((double)(p->nxi + 1))));
  const int nblk = (p->nxi + 1 + B - 1) / B;
  const size_t ng = (size_t)(p->nxi + 1) * n1;
  BeamConst c{};
  c.n = n;
  c.n_drive = p->n_drive;
  c.nbins = nbins;
  c.b = BoundsRZ{nr, p->nxi, g.dr, g.dxi, p->rmax, p->ximax};
  c.dt = p->ds;
  c.gamma_b = p->gamma_b;
  std::vector<double> r0(np), ur0(np), l(np), G0(np), w(np), rho0(n1);
  for (int j = 0; j < np; ++j) plasma_init_one(p->ppc, g.dr, theta[3], nm_p, r0.data(), ur0.data(), l.data(), G0.data(), w.data(), j);
  for (int i = 0; i < n1; ++i) rho0[i] = rho0_node(g, r0.data(), w.data(), i);
  std::vector<double> beam((size_t)6 * n * (nsteps + 1)), wgt(n);
  std::vector<uint8_t> lost((size_t)n * (nsteps + 1));
  std::vector<int> bin(n);
  auto slot = [&](int t) {
    double *q = beam.data() + (size_t)t * 6 * n;
    return Beam{q, q + n, q + 2 * n, q + 3 * n, q + 4 * n, q + 5 * n, lost.data() + (size_t)t * n};
  };
  std::vector<double> nb(ng * nsteps), ez(ng * nsteps), er(ng * nsteps), bt(ng * nsteps);
  std::vector<double> ckpt((size_t)np * 2 * nblk * nsteps), tape(slice_tape_doubles(n1, np) * B);
  std::vector<double> lring((size_t)np * 24), nbh(n1), lnbh(n1), work((size_t)Work::kCount * n1);
  std::vector<double> lam((size_t)6 * n), lwb(n), lez(ng), ler(ng), lbt(ng), lnb(ng);
  std::vector<double> lG0(np), lw(np), ll(np), lur0(np), lrho0(n1);
  const BunchSpec q{p->sigma_r, p->eps_n, p->xi_d, p->sigma_zw, p->n_d};
  for (int64_t j = 0; j < n; ++j) beam_init_one(c, q, slot(0), wgt.data(), bin.data(), nm_b, theta, profile, j);
  Work W;
  W.carve(work.data(), n1);
  auto args = [&](int t) {
    MarchArgs m{};
    m.g = g;
    m.B = B;
    m.nblk = nblk;
    m.r0 = r0.data();
    m.ur0 = ur0.data();
    m.l = l.data();
    m.G0 = G0.data();
    m.w = w.data();
    m.rho0 = rho0.data();
    m.nb = nb.data() + (size_t)t * ng;
    m.ez = ez.data() + (size_t)t * ng;
    m.er = er.data() + (size_t)t * ng;
    m.bth = bt.data() + (size_t)t * ng;
    m.ckpt = ckpt.data() + (size_t)t * nblk * 2 * np;
    m.tape = tape.data();
    m.lring = lring.data();
    m.lez = lez.data();
    m.ler = ler.data();
    m.lbth = lbt.data();
    m.lnb = lnb.data();
    m.lG0 = lG0.data();
    m.lw = lw.data();
    m.ll = ll.data();
    m.lur0 = lur0.data();
    m.lrho0 = lrho0.data();
    m.nbh = nbh.data();
    m.lnbh = lnbh.data();
    return m;
  };
  int bad = 0;
  for (int t = 0; t < nsteps; ++t) {
    double *nbt = nb.data() + (size_t)t * ng;
    std::memset(nbt, 0, sizeof(double) * ng);
    for (int64_t j = 0; j < n; ++j) deposit_one(c, slot(t), wgt.data(), nbt, j);
    for (size_t i = 0; i < ng; ++i) nbt[i] *= node_scale(c.b, (int)(i / n1), (int)(i % n1));
    march_forward_body(P, args(t), W, &bad);
    for (int64_t j = 0; j < n; ++j)
      push_one(c, slot(t), slot(t + 1), er.data() + (size_t)t * ng, ez.data() + (size_t)t * ng, bt.data() + (size_t)t * ng, j);
  }
  if (bad) return -4;
  double sums[3] = {0, 0, 0};
  for (int64_t j = 0; j < n; ++j) loss_one(c, slot(nsteps), wgt.data(), j, sums);
  const double M = sums[1] / sums[0];
  obs[0] = M;
  obs[1] = std::sqrt(std::max(sums[2] / sums[0] - M * M, 0.0));
  if (!dobs) return 0;
  Beam L{lam.data(), lam.data() + n, lam.data() + 2 * n, lam.data() + 3 * n, lam.data() + 4 * n, lam.data() + 5 * n, nullptr};
  for (int64_t j = 0; j < n; ++j) loss_reverse_one(c, slot(nsteps), wgt.data(), sums, dobs[0], dobs[1], L, lwb.data(), j);
  for (int t = nsteps - 1; t >= 0; --t) {
    std::fill(ler.begin(), ler.end(), 0.0);
    std::fill(lez.begin(), lez.end(), 0.0);
    std::fill(lbt.begin(), lbt.end(), 0.0);
    std::fill(lnb.begin(), lnb.end(), 0.0);
    for (int64_t j = 0; j < n; ++j)
      push_reverse_one(c, slot(t), er.data() + (size_t)t * ng, ez.data() + (size_t)t * ng, bt.data() + (size_t)t * ng,
                       L, ler.data(), lez.data(), lbt.data(), j);
    march_reverse_body(P, args(t), W, &bad);
    for (int64_t j = 0; j < n; ++j) deposit_reverse_one(c, slot(t), wgt.data(), lnb.data(), L, lwb.data(), j);
  }
  const double s2pi = std::sqrt(2.0 * 3.14159265358979323846);
  const double wu_w = s2pi * p->sigma_r * p->sigma_r * p->sigma_zw / (double)(p->n_beam - p->n_drive);
  const double wu_d = p->n_d * s2pi * p->sigma_r * p->sigma_r / (double)p->n_drive;
  for (int i = 0; i < 4 + nbins; ++i) grad[i] = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double gb;
    theta_beam_one(c, nm_b, bin.data(), L, lwb.data(), theta, profile, wu_w, wu_d, j, grad, &gb);
    if (gb != 0.0) grad[4 + bin[j]] += gb;
  }
  for (int j = 0; j < np; ++j)
    grad[3] += theta_ring_one(g, nm_p, r0.data(), lrho0.data(), lG0.data(), lw.data(), ll.data(), lur0.data(), theta[3], p->ppc, j);
  return bad ? -4 : 0;
}
