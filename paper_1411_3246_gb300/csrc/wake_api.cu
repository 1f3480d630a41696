// libwake: the C ABI declared in include/wake.h.  Host-side bookkeeping only: scratch
// allocation per simulation, argument checks, kernel launches on the handle's stream, and
// the sticky device status words.  All arithmetic of the method runs in the kernels of
// march.cuh and beam.cuh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wake.h"
#include "beam.cuh"
#include "march_launch.h"
#include "pipeline.cuh"

using namespace wake;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return fail(WAKE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct Sim {
  wake_params p{};
  int np = 0;
  size_t ng = 0;  // grid nodes (nxi+1)(nr+1)
  double *r0 = nullptr, *ur0 = nullptr, *lz = nullptr, *G0 = nullptr, *w = nullptr;
  void *ring_buf = nullptr;  // ring slot arrays in global memory (FP64 form)
  void *nb = nullptr, *psi = nullptr, *ez = nullptr, *er = nullptr, *bth = nullptr;
  void *bx = nullptr, *by = nullptr, *bux = nullptr, *buy = nullptr;
  double *bxi = nullptr, *buz = nullptr;
  uint8_t *blost = nullptr;  // flags: bit 0 lost, bit 1 witness
  int *orig = nullptr;       // index of each particle in the caller's order
  void *bwt = nullptr, *bwt2 = nullptr;  // per-particle weights (and the sort's second copy)
  // second copy of the beam for the re-sort by xi cell, and the cell table
  void *bx2 = nullptr, *by2 = nullptr, *bux2 = nullptr, *buy2 = nullptr;
  double *bxi2 = nullptr, *buz2 = nullptr;
  uint8_t *blost2 = nullptr;
  int *orig2 = nullptr, *bin_count = nullptr, *bin_start = nullptr, *bin_cursor = nullptr;
  unsigned long long *slip = nullptr;  // largest xi slip rate of the beam (double bits)
  // pipelined steps: per-step beam-density grids, progress counters, per-CTA ring storage
  void *pgrids = nullptr;
  int pgrid_cap = 0;
  int *progress = nullptr;
  void *pring = nullptr;
  size_t pring_bytes = 0;
  int *defer_cnt = nullptr, *target = nullptr;  // pipelined steps: slipped-particle lists
  size_t target_n = 0;                           // entries of target
  int2 *defer_list = nullptr;
  size_t defer_bytes = 0;
  int2 *near_list = nullptr;  // pipelined steps: the next-cell rings
  size_t near_bytes = 0;
  int *status = nullptr;
  // trapping (wake_set_trapping): beam slots for promoted particles, the march's promotions
  int64_t n_cap = 0;            // beam slots: n_beam, plus room for promoted particles
  double trap_gamma = 0.0;      // promotion threshold on Gamma (0: no trapping)
  double *trap_list = nullptr;  // one march's promotions: np entries of 7 doubles
  int *trap_count = nullptr;
  int64_t *trap_used = nullptr;  // [0] promoted particles in the beam, [1] promotions dropped
  bool trap_pending = false;     // a march's promotions not yet appended to the beam
  bool plasma = false, beam = false, marched = false;
  bool fields_bound = false;  // psi, ez, er, bth are the caller's (wake_bind_fields): never freed
  bool wide = false;  // marched by the wide form (rings in a global buffer)
};

size_t gsize(int precision) { return precision == WAKE_FP64 ? sizeof(double) : sizeof(float); }

// Global ring storage a simulation's march needs: FP64 form and wide form only.
size_t sim_ring_bytes(int precision, const Sim &s) {
  if (s.wide) return precision == WAKE_FP64 ? wide_fp64_ring_bytes(s.np, s.p.nr + 1) : wide_ring_bytes(s.np);
  return ring_buf_bytes(precision);
}

// x-extent of a batched launch (blockIdx.y is the simulation): up to 64 blocks of 256 per
// simulation, each striding over that simulation's particles or nodes.
int batch_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 64)); }

int grid_blocks(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

namespace wake {
// Error message of an entry point defined in another translation unit.
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace wake

struct wake_sim {
  int n = 0, precision = 0;
  cudaStream_t stream = nullptr;
  std::vector<Sim> sims;
  std::vector<SimDesc> h_desc;  // host copy of d_desc
  SimDesc *d_desc = nullptr;
  int *d_order = nullptr;
  double *d_diag = nullptr;
  int max_n1 = 0, max_np = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;  // around each pipelined launch
  int ev_used = 0;
  // march tiles: simulations grouped by the tile the autotuner chose (planned at the first march)
  struct TileClass {
    TileFns fns;
    int n1max = 0, off = 0, count = 0;
    cudaStream_t side = nullptr;  // class 0 runs on the handle's stream
    cudaEvent_t done = nullptr;
  };
  bool planned = false;
  std::vector<TileClass> classes;
  std::vector<int> tile_of;  // per simulation: its class
  cudaEvent_t fork = nullptr;
  SimDesc *d_probe = nullptr;  // autotuner probe descriptor, status word, all-zero CTA map
  int *d_probe_status = nullptr, *d_probe_order = nullptr;
  int tile_nt_forced = 0;  // WAKE_TILE_NT
  BeamDesc *d_bdesc = nullptr;  // per simulation (several simulations: the batched beam kernels)
  int64_t max_beam = 0;
  size_t max_ng = 0;
  cudaGraphExec_t step_graph = nullptr;  // one batched step, captured at the first wake_step
  bool batch_pipeline = true;             // WAKE_BATCH_PIPELINE=0: batched steps by the graph
  int batch_nt = 256;                     // threads per CTA of the pipelined batch (256 or 512)
  long long spin_limit = 1LL << 24;       // polls of >= 128 ns before a pipelined wait gives up
                                          // (WAKE_SPIN_LIMIT)
  int step_form = 0;                      // one simulation's pipelined steps: 0 tile (or wide 512 when
                                          // no tile fits), 256 / 512 wide form (WAKE_STEP_FORM)
  void *bp_rings = nullptr, *bp_sims = nullptr, *bp_items = nullptr;  // pipelined batch scratch
  size_t bp_rings_bytes = 0, bp_sims_bytes = 0, bp_items_bytes = 0;
};

namespace {

void free_sim(Sim &s) {
  if (s.fields_bound) s.psi = s.ez = s.er = s.bth = nullptr;  // the caller's memory
  void *ptrs[] = {s.r0, s.ur0, s.lz, s.G0, s.w, s.ring_buf, s.nb, s.psi, s.ez, s.er, s.bth, s.bx, s.by, s.bux, s.buy,
                  s.bxi, s.buz, s.blost, s.status, s.orig, s.bx2, s.by2, s.bux2, s.buy2, s.bxi2, s.buz2, s.blost2,
                  s.orig2, s.bin_count, s.bin_start, s.bin_cursor, s.slip, s.pgrids, s.progress, s.pring,
                  s.defer_cnt, s.target, s.defer_list, s.near_list, s.bwt, s.bwt2, s.trap_list, s.trap_count,
                  s.trap_used};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  s = Sim();
}

int check_params(const wake_params &p, int prec0) {
  if (p.precision != WAKE_FP64 && p.precision != WAKE_MIXED && p.precision != WAKE_MIXED64)
    return fail(WAKE_EINVAL, "precision must be WAKE_FP64, WAKE_MIXED or WAKE_MIXED64");
  if (p.precision != prec0) return fail(WAKE_EINVAL, "all simulations of one handle must share the precision");
  const bool small = p.precision == WAKE_MIXED64;  // the FP64-solve split has no wide form
  if (p.nr < 2 || p.nr > (small ? 1024 : 2048))
    return fail(WAKE_EINVAL, "nr must be in [2, 1024] (FP64-solve) or [2, 2048] (FP64, mixed)");
  if (p.nxi < 2 || p.nxi > (1 << 20)) return fail(WAKE_EINVAL, "nxi must be in [2, 2^20]");
  if (p.ppc < 1 || (int64_t)p.nr * p.ppc > (small ? 8192 : 65536))
    return fail(WAKE_EINVAL, "need ppc >= 1 and nr*ppc <= 8192 (FP64-solve) or 65536 (FP64, mixed)");
  if (p.u_th < 0.0 || (p.u_th > 0.0 && p.ppc % 2)) return fail(WAKE_EINVAL, "a warm plasma needs u_th > 0 and an even ppc");
  if (!(p.rmax > 0.0) || !(p.ximax > 0.0)) return fail(WAKE_EINVAL, "rmax and ximax must be positive");
  if (p.n_beam < 0 || p.n_drive < 0 || p.n_drive > p.n_beam) return fail(WAKE_EINVAL, "need 0 <= n_drive <= n_beam");
  if (!(p.sigma_r > 0.0) || !(p.sigma_zd > 0.0) || (p.n_w != 0.0 && !(p.sigma_zw > 0.0)))
    return fail(WAKE_EINVAL, "bunch sizes must be positive");
  if (p.n_beam > 0 && (!(p.gamma_b > 1.0) || !(p.ds > 0.0))) return fail(WAKE_EINVAL, "a beam needs gamma_b > 1 and ds > 0");
  if (p.geometry != WAKE_CYLINDRICAL && p.geometry != WAKE_SLAB)
    return fail(WAKE_EINVAL, "geometry must be WAKE_CYLINDRICAL or WAKE_SLAB");
  return WAKE_OK;
}

template <class T>
int dalloc(T **p, size_t bytes) {
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) return fail(WAKE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  return WAKE_OK;
}

// The pipelined steps' per-particle targets, one per beam slot (promoted particles included).
int alloc_target(Sim &s) {
  const size_t n = (size_t)(s.n_cap > s.p.n_beam ? s.n_cap : s.p.n_beam);
  if (s.target && s.target_n >= n) return WAKE_OK;
  if (s.target) cudaFree(s.target);
  s.target = nullptr;
  s.target_n = 0;
  const int rc = dalloc(&s.target, sizeof(int) * n);
  if (rc == WAKE_OK) s.target_n = n;
  return rc;
}

// Entries of a step's next-cell ring: the entries of two consecutive cells are alive at
// once, each cell's at most the particles sorted into it (and a few listed again), so four
// times the densest cell suffices.
int near_ring(const Sim &s, int occ) {
  return (int)std::min<int64_t>((int64_t)4 * occ + 1024, (int64_t)s.n_cap + 1024);
}
int alloc_near(Sim &s, int cap, int ch) {
  const size_t need = sizeof(int2) * (size_t)cap * ch;
  if (s.near_bytes >= need) return WAKE_OK;
  if (s.near_list) cudaFree(s.near_list);
  s.near_list = nullptr;
  s.near_bytes = 0;
  const int rc = dalloc(&s.near_list, need);
  if (rc == WAKE_OK) s.near_bytes = need;
  return rc;
}

// The beam arrays of simulation s for s.n_cap particles (any earlier ones freed).
int alloc_beam(wake_sim *h, Sim &s) {
  void **old[] = {&s.bx, &s.by, &s.bux, &s.buy, (void **)&s.bxi, (void **)&s.buz, (void **)&s.blost, (void **)&s.orig,
                  &s.bx2, &s.by2, &s.bux2, &s.buy2, (void **)&s.bxi2, (void **)&s.buz2, (void **)&s.blost2,
                  (void **)&s.orig2, (void **)&s.bin_count, (void **)&s.bin_start, (void **)&s.bin_cursor,
                  (void **)&s.slip, &s.bwt, &s.bwt2};
  for (void **q : old)
    if (*q) {
      cudaFree(*q);
      *q = nullptr;
    }
  const size_t bt = gsize(h->precision) * (size_t)s.n_cap, nbm = (size_t)s.n_cap;
  int rc;
  if ((rc = dalloc(&s.bx, bt)) || (rc = dalloc(&s.by, bt)) || (rc = dalloc(&s.bux, bt)) || (rc = dalloc(&s.buy, bt)) ||
      (rc = dalloc(&s.bxi, sizeof(double) * nbm)) || (rc = dalloc(&s.buz, sizeof(double) * nbm)) ||
      (rc = dalloc(&s.blost, nbm)) || (rc = dalloc(&s.orig, sizeof(int) * nbm)) || (rc = dalloc(&s.bx2, bt)) ||
      (rc = dalloc(&s.by2, bt)) || (rc = dalloc(&s.bux2, bt)) || (rc = dalloc(&s.buy2, bt)) ||
      (rc = dalloc(&s.bxi2, sizeof(double) * nbm)) || (rc = dalloc(&s.buz2, sizeof(double) * nbm)) ||
      (rc = dalloc(&s.blost2, nbm)) || (rc = dalloc(&s.orig2, sizeof(int) * nbm)) ||
      (rc = dalloc(&s.bin_count, sizeof(int) * (s.p.nxi + 2))) ||
      (rc = dalloc(&s.bin_start, sizeof(int) * (s.p.nxi + 2))) ||
      (rc = dalloc(&s.bin_cursor, sizeof(int) * (s.p.nxi + 2))) ||
      (rc = dalloc(&s.slip, sizeof(unsigned long long) + 64 * sizeof(int))) || (rc = dalloc(&s.bwt, bt)) ||
      (rc = dalloc(&s.bwt2, bt)))
    return rc;
  return WAKE_OK;
}

// The pipelined push's FP32 constants (the mixed form reads them instead of forming them in
// FP64 per particle).
void push_consts(PipeArgs &a, const wake_params &p) {
  const double dr = p.rmax / p.nr, dxi = p.ximax / p.nxi;
  a.f_inv_dr = (float)(1.0 / dr);
  a.f_ds = (float)p.ds;
  a.f_rmax = (float)p.rmax;
  a.f_wq = (float)(p.geometry == WAKE_SLAB ? 1.0 / (dr * dxi) : 1.0 / (dr * dr * dxi));
}

BeamDesc beam_desc(const Sim &s, double *diag) {
  BeamDesc b{};
  const wake_params &p = s.p;
  b.n = p.n_beam;
  b.n_drive = p.n_drive;
  b.n_cap = s.n_cap > p.n_beam ? s.n_cap : p.n_beam;
  b.nr = p.nr;
  b.nxi = p.nxi;
  b.rmax = p.rmax;
  b.ximax = p.ximax;
  b.dr = p.rmax / p.nr;
  b.dxi = p.ximax / p.nxi;
  b.ds = p.ds;
  b.gamma_b = p.gamma_b;
  // macroparticle weight = bunch charge (per 2 pi) of Eq. 12, n sqrt(2 pi) sigma_r^2 sigma_z,
  // over the bunch's macroparticle count (slab: per unit area of the half slab, the transverse
  // integral sigma_r sqrt(2 pi)/2 in place of sigma_r^2)
  const double s2pi = std::sqrt(2.0 * 3.14159265358979323846);
  const int64_t nw = p.n_beam - p.n_drive;
  const double tr = p.geometry == WAKE_SLAB ? 0.5 * s2pi * p.sigma_r : p.sigma_r * p.sigma_r;
  b.wd = p.n_drive > 0 ? p.n_d * s2pi * tr * p.sigma_zd / (double)p.n_drive : 0.0;
  b.ww = nw > 0 ? p.n_w * s2pi * tr * p.sigma_zw / (double)nw : 0.0;
  b.slab = p.geometry == WAKE_SLAB;
  b.ffi = ff_pair(1.0 / b.dxi);
  b.ffx = ff_pair(b.ximax);
  b.x = s.bx;
  b.y = s.by;
  b.ux = s.bux;
  b.uy = s.buy;
  b.xi = s.bxi;
  b.uz = s.buz;
  b.lost = s.blost;
  b.orig = s.orig;
  b.w = s.bwt;
  b.nb = s.nb;
  b.er = s.er;
  b.ez = s.ez;
  b.bth = s.bth;
  b.diag = diag;
  return b;
}

constexpr int kProbeSlices = 48;
constexpr int kMaxProbeCtas = 152 * 16;

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Compiled tiles that can march simulation s: NT x PPT >= Np rings, Nr+1 <= 3 NT nodes (a
// thread holds at most three nodes in the block scans), shared memory within one CTA's limit.
std::vector<TileFns> tile_candidates(const wake_sim *h, const Sim &s) {
  std::vector<TileFns> out;
  const int n1 = s.p.nr + 1;
  for (int nt : {128, 256, 512}) {
    if (h->precision != WAKE_MIXED && nt != 512) continue;
    if (h->tile_nt_forced && nt != h->tile_nt_forced) continue;  // -1: the wide form only
    if (n1 > 3 * nt) continue;
    const int ppt = pow2_at_least((s.np + nt - 1) / nt);
    TileFns f;
    if (!march_tile(h->precision, s.p.geometry == WAKE_SLAB, nt, ppt, &f)) continue;
    if (f.smem(n1) > kMaxSmemPerCta) continue;
    out.push_back(f);
  }
  if (s.p.geometry == WAKE_SLAB) return out;  // the wide forms are cylindrical only
  if (out.empty() && h->precision == WAKE_MIXED && (!h->tile_nt_forced || h->tile_nt_forced == -1)) {
    const TileFns f = march_tile_wide();
    if (n1 <= 5 * f.nt && f.smem(n1) <= kMaxSmemPerCta) out.push_back(f);
  }
  if (out.empty() && h->precision == WAKE_FP64 && (!h->tile_nt_forced || h->tile_nt_forced == -1)) {
    const TileFns f = march_tile_wide_fp64();  // node arrays in global memory
    if (n1 <= 5 * f.nt) out.push_back(f);
  }
  return out;
}

// Throughput score of tile f on simulation s: a probe march of kProbeSlices slices run by as
// many CTAs as fill the GPU (all on s, outputs discarded), CTAs x slices per ms.
int probe_tile(wake_sim *h, const Sim &s, const SimDesc &d, const TileFns &f, double *score) {
  const int n1 = s.p.nr + 1;
  int occ = f.occupancy(n1), dev = 0, sms = 0;
  if (occ < 1) {
    *score = 0.0;
    return WAKE_OK;
  }
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int ctas = std::min(kMaxProbeCtas, occ * sms);
  SimDesc pd = d;
  pd.nxi = std::min(d.nxi, kProbeSlices);
  pd.psi = pd.ez = pd.er = pd.bth = nullptr;
  pd.status = h->d_probe_status;
  CUDA_TRY(cudaMemcpyAsync(h->d_probe, &pd, sizeof(SimDesc), cudaMemcpyHostToDevice, h->stream));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(WAKE_ECUDA, "cudaEventCreate");
  }
  cudaError_t e = f.launch(h->d_probe, h->d_probe_order, ctas, n1, h->stream);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
  if (e == cudaSuccess) e = f.launch(h->d_probe, h->d_probe_order, ctas, n1, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(WAKE_ECUDA, std::string("tile probe: ") + cudaGetErrorString(e));
  *score = ms > 0.0f ? (double)ctas * pd.nxi / ms : 0.0;
  return WAKE_OK;
}

// Choose a tile per simulation (the best probe score per distinct (Nr, Np); the only
// candidate when there is one) and group the simulations by tile, each group largest work
// first.  Synchronous (the probes are timed).
int plan_tiles(wake_sim *h) {
  std::vector<SimDesc> desc(h->n);
  CUDA_TRY(cudaMemcpyAsync(desc.data(), h->d_desc, sizeof(SimDesc) * h->n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  std::vector<std::pair<long long, TileFns>> chosen_by_shape;  // key nr * 2^20 + np
  std::vector<TileFns> pick(h->n);
  for (int i = 0; i < h->n; ++i) {
    const Sim &s = h->sims[i];
    const long long key = (long long)s.p.nr * (1 << 20) + s.np;
    bool found = false;
    for (auto &kv : chosen_by_shape)
      if (kv.first == key) {
        pick[i] = kv.second;
        found = true;
      }
    if (found) continue;
    std::vector<TileFns> cand = tile_candidates(h, s);
    if (cand.empty()) return fail(WAKE_EINVAL, "no compiled march tile fits a simulation's Nr and rings");
    TileFns best = cand.back();  // the 512-thread tile when there is no choice to make
    if (cand.size() > 1 && h->n > 1) {
      // representative: the simulation of this shape with the most slices
      int rep = i;
      for (int j = i + 1; j < h->n; ++j)
        if ((long long)h->sims[j].p.nr * (1 << 20) + h->sims[j].np == key && h->sims[j].p.nxi > h->sims[rep].p.nxi) rep = j;
      double best_score = -1.0;
      for (const TileFns &f : cand) {
        double sc = 0.0;
        int rc = probe_tile(h, h->sims[rep], desc[rep], f, &sc);
        if (rc) return rc;
        if (sc > best_score) {
          best_score = sc;
          best = f;
        }
      }
    }
    chosen_by_shape.push_back({key, best});
    pick[i] = best;
  }
  // group by tile, largest work first within a group
  h->classes.clear();
  h->tile_of.assign(h->n, 0);
  for (int i = 0; i < h->n; ++i) {
    int c = -1;
    for (size_t q = 0; q < h->classes.size(); ++q)
      if (h->classes[q].fns.nt == pick[i].nt && h->classes[q].fns.ppt == pick[i].ppt &&
          h->classes[q].fns.wide == pick[i].wide)
        c = (int)q;
    if (c < 0) {
      wake_sim::TileClass tc;
      tc.fns = pick[i];
      h->classes.push_back(tc);
      c = (int)h->classes.size() - 1;
    }
    h->tile_of[i] = c;
    h->classes[c].n1max = std::max(h->classes[c].n1max, h->sims[i].p.nr + 1);
  }
  std::vector<int> order;
  for (size_t c = 0; c < h->classes.size(); ++c) {
    std::vector<int> mine;
    for (int i = 0; i < h->n; ++i)
      if (h->tile_of[i] == (int)c) mine.push_back(i);
    std::stable_sort(mine.begin(), mine.end(), [&](int a, int b) {
      return (double)h->sims[a].np * h->sims[a].p.nxi > (double)h->sims[b].np * h->sims[b].p.nxi;
    });
    const cudaError_t ep = h->classes[c].fns.prepare(h->classes[c].n1max);
    if (ep != cudaSuccess) return fail(WAKE_ECUDA, std::string("march tile set-up: ") + cudaGetErrorString(ep));
    h->classes[c].off = (int)order.size();
    h->classes[c].count = (int)mine.size();
    order.insert(order.end(), mine.begin(), mine.end());
    if (c > 0) {
      CUDA_TRY(cudaStreamCreateWithFlags(&h->classes[c].side, cudaStreamNonBlocking));
      CUDA_TRY(cudaEventCreateWithFlags(&h->classes[c].done, cudaEventDisableTiming));
    }
  }
  if (h->classes.size() > 1 && !h->fork) CUDA_TRY(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
  CUDA_TRY(cudaMemcpyAsync(h->d_order, order.data(), sizeof(int) * h->n, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->planned = true;
  return WAKE_OK;
}

// One march of every simulation: one launch per tile class, the classes on forked streams
// joined back to the handle's stream.
int launch_march(wake_sim *h) {
  int rc;
  if (!h->planned && (rc = plan_tiles(h))) return rc;
  const size_t nc = h->classes.size();
  if (nc > 1) CUDA_TRY(cudaEventRecord(h->fork, h->stream));
  for (size_t c = 0; c < nc; ++c) {
    auto &k = h->classes[c];
    cudaStream_t st = c == 0 ? h->stream : k.side;
    if (c > 0) CUDA_TRY(cudaStreamWaitEvent(st, h->fork, 0));
    const cudaError_t e = k.fns.launch(h->d_desc, h->d_order + k.off, k.count, k.n1max, st);
    if (e != cudaSuccess) return fail(WAKE_ECUDA, std::string("march launch: ") + cudaGetErrorString(e));
    if (c > 0) CUDA_TRY(cudaEventRecord(k.done, st));
  }
  for (size_t c = 1; c < nc; ++c) CUDA_TRY(cudaStreamWaitEvent(h->stream, h->classes[c].done, 0));
  return WAKE_OK;
}

int check_handle(wake_sim *h, int sim) {
  if (!h) return fail(WAKE_EINVAL, "null handle");
  if (sim < 0 || sim >= h->n) return fail(WAKE_EINVAL, "simulation index out of range");
  return WAKE_OK;
}

}  // namespace

extern "C" {

const char *wake_last_error(void) { return g_err.c_str(); }

int wake_init(const wake_params *p, int n_sims, void *stream, wake_sim **out) {
  if (!p || !out || n_sims < 1) return fail(WAKE_EINVAL, "wake_init: null pointer or n_sims < 1");
  *out = nullptr;
  for (int i = 0; i < n_sims; ++i) {
    int rc = check_params(p[i], p[0].precision);
    if (rc) return rc;
  }
  wake_sim *h = new wake_sim();
  h->n = n_sims;
  h->precision = p[0].precision;
  h->stream = (cudaStream_t)stream;
  h->sims.resize(n_sims);
  if (const char *t = std::getenv("WAKE_TILE_NT")) h->tile_nt_forced = std::atoi(t);
  if (const char *t = std::getenv("WAKE_BATCH_PIPELINE")) h->batch_pipeline = std::atoi(t) != 0;
  if (const char *t = std::getenv("WAKE_BATCH_NT")) h->batch_nt = std::atoi(t) == 512 ? 512 : 256;
  if (const char *t = std::getenv("WAKE_STEP_FORM")) h->step_form = std::atoi(t);
  if (const char *t = std::getenv("WAKE_SPIN_LIMIT")) h->spin_limit = std::max(0LL, std::atoll(t));
  const size_t gs = gsize(h->precision);
  int rc = WAKE_OK;
  for (int i = 0; i < n_sims && rc == WAKE_OK; ++i) {
    Sim &s = h->sims[i];
    s.p = p[i];
    s.np = p[i].nr * p[i].ppc;
    s.ng = (size_t)(p[i].nxi + 1) * (p[i].nr + 1);
    {
      const std::vector<TileFns> cand = tile_candidates(h, s);
      s.wide = !cand.empty() && cand.back().wide;
      if (cand.empty() && p[i].geometry == WAKE_SLAB) {
        rc = fail(WAKE_EINVAL, "wake_init: a slab simulation needs the shared-memory march (nr*ppc <= 4096 within one CTA)");
        break;
      }
    }
    h->max_n1 = std::max(h->max_n1, p[i].nr + 1);
    h->max_np = std::max(h->max_np, s.np);
    const size_t pb = sizeof(double) * s.np;
    if ((rc = dalloc(&s.r0, pb)) || (rc = dalloc(&s.ur0, pb)) || (rc = dalloc(&s.lz, pb)) || (rc = dalloc(&s.G0, pb)) ||
        (rc = dalloc(&s.w, pb)) ||
        (sim_ring_bytes(h->precision, s) > 0 && (rc = dalloc(&s.ring_buf, sim_ring_bytes(h->precision, s)))) ||
        (rc = dalloc(&s.nb, gs * s.ng)) || (rc = dalloc(&s.psi, gs * s.ng)) ||
        (rc = dalloc(&s.ez, gs * s.ng)) || (rc = dalloc(&s.er, gs * s.ng)) || (rc = dalloc(&s.bth, gs * s.ng)) ||
        (rc = dalloc(&s.status, sizeof(int))))
      break;
    if (cudaMemsetAsync(s.status, 0, sizeof(int), h->stream) != cudaSuccess) {
      rc = fail(WAKE_ECUDA, "cudaMemsetAsync(status)");
      break;
    }
    if (p[i].n_beam > 0) {
      s.n_cap = p[i].n_beam;
      if ((rc = alloc_beam(h, s))) break;
    } else {
      // frozen analytic driver (Eq. 12) on the nodes
      const double dr = p[i].rmax / p[i].nr, dxi = p[i].ximax / p[i].nxi;
      const int nb = grid_blocks((int64_t)s.ng, 256);
      if (h->precision == WAKE_FP64)
        nb_analytic_kernel<double><<<nb, 256, 0, h->stream>>>((double *)s.nb, p[i].nr, p[i].nxi, dr, dxi, p[i].n_d,
                                                              p[i].n_w, p[i].sigma_r, p[i].sigma_zd, p[i].sigma_zw,
                                                              p[i].xi_d, p[i].xi_w);
      else
        nb_analytic_kernel<float><<<nb, 256, 0, h->stream>>>((float *)s.nb, p[i].nr, p[i].nxi, dr, dxi, p[i].n_d,
                                                             p[i].n_w, p[i].sigma_r, p[i].sigma_zd, p[i].sigma_zw,
                                                             p[i].xi_d, p[i].xi_w);
      if (cudaGetLastError() != cudaSuccess) {
        rc = fail(WAKE_ECUDA, "nb_analytic_kernel launch");
        break;
      }
    }
  }
  if (rc == WAKE_OK)
    for (int i = 0; i < n_sims && rc == WAKE_OK; ++i)
      if (tile_candidates(h, h->sims[i]).empty())
        rc = fail(WAKE_EINVAL, "nr and nr*ppc too large for one march CTA's shared memory");
  if (rc == WAKE_OK && h->n > 1) {
    std::vector<BeamDesc> bd(n_sims);
    for (int i = 0; i < n_sims; ++i) {
      bd[i] = beam_desc(h->sims[i], nullptr);
      h->max_beam = std::max<int64_t>(h->max_beam, h->sims[i].p.n_beam);
      h->max_ng = std::max(h->max_ng, h->sims[i].ng);
    }
    if ((rc = dalloc(&h->d_bdesc, sizeof(BeamDesc) * n_sims)) == WAKE_OK &&
        cudaMemcpyAsync(h->d_bdesc, bd.data(), sizeof(BeamDesc) * n_sims, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      rc = fail(WAKE_ECUDA, "wake_init: beam descriptor upload");
    if (rc == WAKE_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = fail(WAKE_ECUDA, "wake_init: sync");
  }
  if (rc == WAKE_OK && h->n > 1) {
    if ((rc = dalloc(&h->d_probe, sizeof(SimDesc))) == WAKE_OK && (rc = dalloc(&h->d_probe_status, sizeof(int))) == WAKE_OK &&
        (rc = dalloc(&h->d_probe_order, sizeof(int) * kMaxProbeCtas)) == WAKE_OK) {
      if (cudaMemsetAsync(h->d_probe_order, 0, sizeof(int) * kMaxProbeCtas, h->stream) != cudaSuccess ||
          cudaMemsetAsync(h->d_probe_status, 0, sizeof(int), h->stream) != cudaSuccess)
        rc = fail(WAKE_ECUDA, "wake_init: probe scratch");
    }
  }
  if (rc == WAKE_OK) {
    // descriptors; CTAs take the simulations largest-work first (LPT order)
    std::vector<SimDesc> desc(n_sims);
    std::vector<int> order(n_sims);
    for (int i = 0; i < n_sims; ++i) {
      const Sim &s = h->sims[i];
      SimDesc &d = desc[i];
      d.nr = s.p.nr;
      d.nxi = s.p.nxi;
      d.np = s.np;
      d.has_beam = s.p.n_beam > 0;
      d.slab = s.p.geometry == WAKE_SLAB;
      d.rmax = s.p.rmax;
      d.ximax = s.p.ximax;
      d.dr = s.p.rmax / s.p.nr;
      d.dxi = s.p.ximax / s.p.nxi;
      d.r0 = s.r0;
      d.ur0 = s.ur0;
      d.lz = s.lz;
      d.G0 = s.G0;
      d.w = s.w;
      d.ring_buf = s.ring_buf;
      d.nb = s.nb;
      d.psi = s.psi;
      d.ez = s.ez;
      d.er = s.er;
      d.bth = s.bth;
      d.status = s.status;
      order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return (double)desc[a].np * desc[a].nxi > (double)desc[b].np * desc[b].nxi;
    });
    h->h_desc = desc;
    if ((rc = dalloc(&h->d_desc, sizeof(SimDesc) * n_sims)) == WAKE_OK &&
        (rc = dalloc(&h->d_order, sizeof(int) * n_sims)) == WAKE_OK &&
        (rc = dalloc(&h->d_diag, sizeof(double) * 5 * n_sims)) == WAKE_OK) {
      if (cudaMemcpyAsync(h->d_desc, desc.data(), sizeof(SimDesc) * n_sims, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
          cudaMemcpyAsync(h->d_order, order.data(), sizeof(int) * n_sims, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess)
        rc = fail(WAKE_ECUDA, "wake_init: descriptor upload");
    }
  }
  if (rc != WAKE_OK) {
    wake_destroy(h);
    return rc;
  }
  *out = h;
  return WAKE_OK;
}

int wake_load_plasma(wake_sim *h, int sim, const double *normals) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  Sim &s = h->sims[sim];
  if (s.p.u_th > 0.0 && !normals) return fail(WAKE_EINVAL, "a warm plasma needs the momentum normals");
  const double dr = s.p.rmax / s.p.nr;
  plasma_init_kernel<<<grid_blocks(s.np, 256), 256, 0, h->stream>>>(s.p.nr, s.p.ppc, dr, s.p.u_th,
                                                                     s.p.u_th > 0.0 ? normals : nullptr, s.r0, s.ur0,
                                                                     s.lz, s.G0, s.w, s.p.geometry == WAKE_SLAB);
  CUDA_TRY(cudaGetLastError());
  s.plasma = true;
  return WAKE_OK;
}

int wake_load_beam(wake_sim *h, int sim, const double *normals) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  Sim &s = h->sims[sim];
  if (s.p.n_beam == 0) return fail(WAKE_EINVAL, "simulation has no beam (n_beam == 0)");
  if (!normals) return fail(WAKE_EINVAL, "null beam normals");
  BeamDesc b = beam_desc(s, nullptr);
  BunchInit q{s.p.sigma_r, s.p.eps_n, s.p.xi_d, s.p.sigma_zd, s.p.xi_w, s.p.sigma_zw, s.p.gamma_b};
  const int nb = grid_blocks(s.p.n_beam, 256);
  if (h->precision == WAKE_FP64)
    beam_init_kernel<double><<<nb, 256, 0, h->stream>>>(b, q, normals);
  else
    beam_init_kernel<float><<<nb, 256, 0, h->stream>>>(b, q, normals);
  CUDA_TRY(cudaGetLastError());
  s.beam = true;
  return WAKE_OK;
}

int wake_set_beam(wake_sim *h, int sim, const double *xyz, const double *w, const uint8_t *tag) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  Sim &s = h->sims[sim];
  if (s.p.n_beam == 0) return fail(WAKE_EINVAL, "simulation has no beam (n_beam == 0)");
  if (!xyz) return fail(WAKE_EINVAL, "null beam state");
  BeamDesc b = beam_desc(s, nullptr);
  const int nb = grid_blocks(s.p.n_beam, 256);
  if (h->precision == WAKE_FP64)
    beam_set_kernel<double><<<nb, 256, 0, h->stream>>>(b, xyz, w, tag);
  else
    beam_set_kernel<float><<<nb, 256, 0, h->stream>>>(b, xyz, w, tag);
  CUDA_TRY(cudaGetLastError());
  s.beam = true;
  return WAKE_OK;
}

int wake_beam_deposit(wake_sim *h) {
  if (!h) return fail(WAKE_EINVAL, "null handle");
  if (h->n > 1) {  // one launch per phase over all simulations
    for (auto &s : h->sims)
      if (s.p.n_beam > 0 && !s.beam) return fail(WAKE_ESTATE, "wake_beam_deposit before wake_load_beam");
    if (h->max_beam == 0) return WAKE_OK;
    const dim3 gg(batch_blocks((int64_t)h->max_ng), h->n), gb(batch_blocks(h->max_beam), h->n);
    if (h->precision == WAKE_FP64) {
      nb_zero_batch_kernel<double><<<gg, 256, 0, h->stream>>>(h->d_bdesc);
      beam_deposit_batch_kernel<double, double><<<gb, 256, 0, h->stream>>>(h->d_bdesc);
      nb_normalize_batch_kernel<double><<<gg, 256, 0, h->stream>>>(h->d_bdesc);
    } else {
      nb_zero_batch_kernel<float><<<gg, 256, 0, h->stream>>>(h->d_bdesc);
      beam_deposit_batch_kernel<float, float><<<gb, 256, 0, h->stream>>>(h->d_bdesc);
      nb_normalize_batch_kernel<float><<<gg, 256, 0, h->stream>>>(h->d_bdesc);
    }
    CUDA_TRY(cudaGetLastError());
    return WAKE_OK;
  }
  for (int i = 0; i < h->n; ++i) {
    Sim &s = h->sims[i];
    if (s.p.n_beam == 0) continue;
    if (!s.beam) return fail(WAKE_ESTATE, "wake_beam_deposit before wake_load_beam");
    BeamDesc b = beam_desc(s, nullptr);
    CUDA_TRY(cudaMemsetAsync(s.nb, 0, gsize(h->precision) * s.ng, h->stream));
    const int nb = grid_blocks(s.p.n_beam, 256), ng = grid_blocks((int64_t)s.ng, 256);
    if (h->precision == WAKE_FP64) {
      beam_deposit_kernel<double, double><<<nb, 256, 0, h->stream>>>(b);
      nb_normalize_kernel<double><<<ng, 256, 0, h->stream>>>((double *)s.nb, s.p.nr, s.p.nxi, b.dr, b.dxi, b.slab);
    } else {
      beam_deposit_kernel<float, float><<<nb, 256, 0, h->stream>>>(b);
      nb_normalize_kernel<float><<<ng, 256, 0, h->stream>>>((float *)s.nb, s.p.nr, s.p.nxi, b.dr, b.dxi, b.slab);
    }
    CUDA_TRY(cudaGetLastError());
  }
  return WAKE_OK;
}

int wake_set_trapping(wake_sim *h, int sim, double gamma_t, int64_t capacity) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  Sim &s = h->sims[sim];
  if (h->n != 1) return fail(WAKE_EINVAL, "wake_set_trapping: trapping needs a handle of one simulation");
  if (s.p.n_beam == 0) return fail(WAKE_EINVAL, "wake_set_trapping: trapping needs a particle beam (n_beam > 0)");
  if (s.p.geometry == WAKE_SLAB) return fail(WAKE_EINVAL, "wake_set_trapping: trapping is cylindrical only");
  if (!(gamma_t >= 0.0) || capacity < 0 || s.p.n_beam + capacity > ((int64_t)1 << 31) - 1)
    return fail(WAKE_EINVAL, "wake_set_trapping: need gamma_t >= 0 and 0 <= capacity < 2^31 - n_beam");
  if (s.beam) return fail(WAKE_ESTATE, "wake_set_trapping: call it before wake_load_beam / wake_set_beam");
  const int n1 = s.p.nr + 1;
  const size_t smem = h->precision == WAKE_FP64 ? march_traj_smem_fp64(n1, s.np) : march_traj_smem_mixed(n1, s.np);
  if (h->precision == WAKE_MIXED64 || s.wide || smem > kMaxSmemPerCta)
    return fail(WAKE_EINVAL, "wake_set_trapping: FP64 and mixed handles whose simulation fits one 512-thread march CTA");
  s.n_cap = s.p.n_beam + capacity;
  if ((rc = alloc_beam(h, s))) return rc;
  if (!s.trap_list && ((rc = dalloc(&s.trap_list, sizeof(double) * 7 * (size_t)s.np)) ||
                       (rc = dalloc(&s.trap_count, sizeof(int))) || (rc = dalloc(&s.trap_used, 2 * sizeof(int64_t)))))
    return rc;
  CUDA_TRY(cudaMemsetAsync(s.trap_count, 0, sizeof(int), h->stream));
  CUDA_TRY(cudaMemsetAsync(s.trap_used, 0, 2 * sizeof(int64_t), h->stream));
  s.trap_gamma = gamma_t;
  s.trap_pending = false;
  SimDesc &d = h->h_desc[sim];
  d.gamma_t = gamma_t;
  d.trap = s.trap_list;
  d.trap_count = s.trap_count;
  d.trap_cap = s.np;
  CUDA_TRY(cudaMemcpyAsync(h->d_desc + sim, &d, sizeof(SimDesc), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));  // d is host memory that may change
  return WAKE_OK;
}

int wake_trapped(wake_sim *h, int sim, double *xyz, double *w, uint8_t *lost, int64_t *count, int64_t *dropped) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  Sim &s = h->sims[sim];
  if (!s.trap_used) return fail(WAKE_ESTATE, "wake_trapped: trapping is not set (wake_set_trapping)");
  int64_t u[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(u, s.trap_used, sizeof(u), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (count) *count = u[0];
  if (dropped) *dropped = u[1];
  if (u[0] > 0 && (xyz || w || lost)) {
    const BeamDesc b = beam_desc(s, nullptr);
    const int64_t cap = s.n_cap - s.p.n_beam;
    const int nb = grid_blocks(u[0], 256);
    if (h->precision == WAKE_FP64)
      trapped_out_kernel<double><<<nb, 256, 0, h->stream>>>(b, u[0], cap, xyz, w, lost);
    else
      trapped_out_kernel<float><<<nb, 256, 0, h->stream>>>(b, u[0], cap, xyz, w, lost);
    CUDA_TRY(cudaGetLastError());
  }
  return WAKE_OK;
}

int wake_plasma_march(wake_sim *h) {
  if (!h) return fail(WAKE_EINVAL, "null handle");
  for (auto &s : h->sims)
    if (!s.plasma) return fail(WAKE_ESTATE, "wake_plasma_march before wake_load_plasma");
  if (h->n == 1 && h->sims[0].trap_gamma > 0.0) {  // the march that promotes rings
    Sim &s = h->sims[0];
    CUDA_TRY(cudaMemsetAsync(s.trap_count, 0, sizeof(int), h->stream));
    const int n1 = s.p.nr + 1;
    const cudaError_t e = h->precision == WAKE_FP64 ? launch_march_trap_fp64(h->d_desc, n1, s.np, h->stream)
                                                    : launch_march_trap_mixed(h->d_desc, n1, s.np, h->stream);
    if (e != cudaSuccess) return fail(WAKE_ECUDA, std::string("trapping march launch: ") + cudaGetErrorString(e));
    s.trap_pending = true;
    s.marched = true;
    return WAKE_OK;
  }
  int rc = launch_march(h);
  if (rc) return rc;
  for (auto &s : h->sims) s.marched = true;
  return WAKE_OK;
}

int wake_plasma_march_traj(wake_sim *h, int sim, int every, double *traj) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  if (every < 1 || !traj) return fail(WAKE_EINVAL, "wake_plasma_march_traj: every >= 1 and a trajectory buffer are needed");
  Sim &s = h->sims[sim];
  if (!s.plasma) return fail(WAKE_ESTATE, "wake_plasma_march_traj before wake_load_plasma");
  const int n1 = s.p.nr + 1;
  if (h->precision == WAKE_MIXED64) return fail(WAKE_EINVAL, "wake_plasma_march_traj: FP64 and mixed forms only");
  const bool fp64 = h->precision == WAKE_FP64;
  const size_t smem = fp64 ? march_traj_smem_fp64(n1, s.np) : march_traj_smem_mixed(n1, s.np);
  if (s.wide || smem > kMaxSmemPerCta)
    return fail(WAKE_EINVAL, "wake_plasma_march_traj: the simulation does not fit one 512-thread march CTA "
                             "(nr + 1 <= 1536 nodes and its rings in shared memory)");
  const bool slab = s.p.geometry == WAKE_SLAB;
  const cudaError_t e = fp64 ? launch_march_traj_fp64(h->d_desc + sim, n1, s.np, traj, every, slab, h->stream)
                             : launch_march_traj_mixed(h->d_desc + sim, n1, s.np, traj, every, slab, h->stream);
  if (e != cudaSuccess) return fail(WAKE_ECUDA, std::string("trajectory march launch: ") + cudaGetErrorString(e));
  s.marched = true;
  return WAKE_OK;
}

int wake_bind_fields(wake_sim *h, int sim, void *psi, void *ez, void *er, void *bth) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  if (!psi || !ez || !er || !bth) return fail(WAKE_EINVAL, "wake_bind_fields: null field pointer");
  Sim &s = h->sims[sim];
  if (s.marched || h->step_graph) return fail(WAKE_ESTATE, "wake_bind_fields after a march or step");
  if (!s.fields_bound) {  // the library's own grids are no longer needed
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    void *own[] = {s.psi, s.ez, s.er, s.bth};
    for (void *q : own)
      if (q) cudaFree(q);
  }
  s.psi = psi;
  s.ez = ez;
  s.er = er;
  s.bth = bth;
  s.fields_bound = true;
  // every descriptor that carries the field pointers: the march's, and the batched beam's
  SimDesc &d = h->h_desc[sim];
  d.psi = psi;
  d.ez = ez;
  d.er = er;
  d.bth = bth;
  CUDA_TRY(cudaMemcpyAsync(h->d_desc + sim, &d, sizeof(SimDesc), cudaMemcpyHostToDevice, h->stream));
  if (h->d_bdesc) {
    const BeamDesc b = beam_desc(s, nullptr);
    CUDA_TRY(cudaMemcpyAsync(h->d_bdesc + sim, &b, sizeof(BeamDesc), cudaMemcpyHostToDevice, h->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));  // the host copies above may be reused
  return WAKE_OK;
}

int wake_beam_push_steps(wake_sim *h, int nsteps) {
  if (!h || nsteps < 0) return fail(WAKE_EINVAL, "wake_beam_push_steps: null handle or nsteps < 0");
  for (int t = 0; t < nsteps; ++t) {
    const int rc = wake_beam_push(h);
    if (rc) return rc;
  }
  return WAKE_OK;
}

int wake_beam_push(wake_sim *h) {
  if (!h) return fail(WAKE_EINVAL, "null handle");
  if (h->n > 1) {
    for (auto &s : h->sims)
      if (s.p.n_beam > 0 && (!s.beam || !s.marched))
        return fail(WAKE_ESTATE, "wake_beam_push needs a loaded beam and a march");
    if (h->max_beam == 0) return WAKE_OK;
    const dim3 gb(batch_blocks(h->max_beam), h->n);
    if (h->precision == WAKE_FP64)
      beam_push_batch_kernel<double, double><<<gb, 256, 0, h->stream>>>(h->d_bdesc);
    else
      beam_push_batch_kernel<float, float><<<gb, 256, 0, h->stream>>>(h->d_bdesc);
    CUDA_TRY(cudaGetLastError());
    return WAKE_OK;
  }
  for (int i = 0; i < h->n; ++i) {
    Sim &s = h->sims[i];
    if (s.p.n_beam == 0) continue;
    if (!s.beam || !s.marched) return fail(WAKE_ESTATE, "wake_beam_push needs a loaded beam and a march");
    BeamDesc b = beam_desc(s, nullptr);
    if (s.trap_pending) {  // the last march's promoted rings join the beam before the push
      if (h->precision == WAKE_FP64)
        trap_append_kernel<double><<<1, 1024, 0, h->stream>>>(b, s.trap_list, s.trap_count, s.np, s.trap_used,
                                                             s.trap_used + 1);
      else
        trap_append_kernel<float><<<1, 1024, 0, h->stream>>>(b, s.trap_list, s.trap_count, s.np, s.trap_used,
                                                            s.trap_used + 1);
      CUDA_TRY(cudaGetLastError());
      s.trap_pending = false;
    }
    const int nb = grid_blocks(b.n_cap, 256);
    if (h->precision == WAKE_FP64)
      beam_push_kernel<double, double><<<nb, 256, 0, h->stream>>>(b);
    else
      beam_push_kernel<float, float><<<nb, 256, 0, h->stream>>>(b);
    CUDA_TRY(cudaGetLastError());
  }
  return WAKE_OK;
}

namespace {

// Sort the beam of simulation s by xi cell (lost particles last) into the second copy and
// swap the copies; bin_start then gives the range of each cell.
int sort_beam(wake_sim *h, Sim &s, int *occ) {
  BeamDesc b = beam_desc(s, nullptr);
  BeamDesc d = b;
  d.x = s.bx2;
  d.y = s.by2;
  d.ux = s.bux2;
  d.uy = s.buy2;
  d.xi = s.bxi2;
  d.uz = s.buz2;
  d.lost = s.blost2;
  d.orig = s.orig2;
  d.w = s.bwt2;
  const int nbins = s.p.nxi + 1;
  CUDA_TRY(cudaMemsetAsync(s.bin_count, 0, sizeof(int) * (nbins + 1), h->stream));
  const int blocks = grid_blocks(s.p.n_beam, 256);
  if (h->precision == WAKE_FP64) {
    bin_count_kernel<double><<<blocks, 256, 0, h->stream>>>(b, s.bin_count);
    bin_scan_kernel<<<1, 1024, 0, h->stream>>>(s.bin_count, s.bin_start, s.bin_cursor, nbins);
    bin_scatter_kernel<double><<<blocks, 256, 0, h->stream>>>(b, d, s.bin_cursor);
  } else {
    bin_count_kernel<float><<<blocks, 256, 0, h->stream>>>(b, s.bin_count);
    bin_scan_kernel<<<1, 1024, 0, h->stream>>>(s.bin_count, s.bin_start, s.bin_cursor, nbins);
    bin_scatter_kernel<float><<<blocks, 256, 0, h->stream>>>(b, d, s.bin_cursor);
  }
  CUDA_TRY(cudaGetLastError());
  if (occ) {  // the densest cell (bins 0 .. nxi - 1) into the unused last count
    bin_max_kernel<<<std::max(1, std::min(152, (nbins + 255) / 256)), 256, 0, h->stream>>>(s.bin_count, nbins - 1,
                                                                                      s.bin_count + nbins);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(occ, s.bin_count + nbins, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  std::swap(s.bx, s.bx2);
  std::swap(s.by, s.by2);
  std::swap(s.bux, s.bux2);
  std::swap(s.buy, s.buy2);
  std::swap(s.bxi, s.bxi2);
  std::swap(s.buz, s.buz2);
  std::swap(s.blost, s.blost2);
  std::swap(s.orig, s.orig2);
  std::swap(s.bwt, s.bwt2);
  return WAKE_OK;
}

// The beam's slip rates at the start of a launch.  A particle may slip any distance over a
// launch (pipeline.cuh lists it for the cell it reached), but less than one cell per step.
//   *ok: the fastest particle, with 4x headroom for its rate to grow (u_perp^2 grows with the
//        betatron motion), slips at most half a cell per step (else the steps are taken one
//        launch sequence at a time);
//   hist[q]: particles that, at twice their present rate, slip two cells after [2^q, 2^(q+1))
//        steps - a launch of L steps lists at most those of the buckets with 2^q < L.
// Synchronises the stream.
int slip_stats(wake_sim *h, Sim &s, bool *ok, long long *hist) {
  BeamDesc b = beam_desc(s, nullptr);
  const double dxi = s.p.ximax / s.p.nxi;
  CUDA_TRY(cudaMemsetAsync(s.slip, 0, sizeof(unsigned long long) + 64 * sizeof(int), h->stream));
  int *dh = (int *)(s.slip + 1);
  const int blocks = grid_blocks(s.p.n_beam, 256);
  const double span = 2.0 * dxi / (2.0 * s.p.ds);  // steps_j = span / rate_j
  if (h->precision == WAKE_FP64)
    beam_slip_kernel<double><<<blocks, 256, 0, h->stream>>>(b, span, s.slip, dh);
  else
    beam_slip_kernel<float><<<blocks, 256, 0, h->stream>>>(b, span, s.slip, dh);
  CUDA_TRY(cudaGetLastError());
  unsigned long long buf[1 + 32] = {};
  CUDA_TRY(cudaMemcpyAsync(buf, s.slip, sizeof(unsigned long long) + 64 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  double rate;
  std::memcpy(&rate, &buf[0], sizeof(rate));
  *ok = !(4.0 * s.p.ds * rate > 0.5 * dxi);
  const int *hc = (const int *)(buf + 1);
  for (int q = 0; q < 64; ++q) hist[q] = hc[q];
  return WAKE_OK;
}

int step_sequential(wake_sim *h, int nsteps) {
  for (int t = 0; t < nsteps; ++t) {
    int rc;
    if ((rc = wake_beam_deposit(h)) || (rc = wake_plasma_march(h)) || (rc = wake_beam_push(h))) return rc;
  }
  return WAKE_OK;
}

int upload_beam_descs(wake_sim *h) {
  std::vector<BeamDesc> bd(h->n);
  for (int i = 0; i < h->n; ++i) bd[i] = beam_desc(h->sims[i], nullptr);
  CUDA_TRY(cudaMemcpyAsync(h->d_bdesc, bd.data(), sizeof(BeamDesc) * h->n, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));  // bd is a host temporary
  return WAKE_OK;
}

// Several simulations with beams, mixed form: pipelined steps of all of them in one
// persistent launch (pipeline.cuh batch_step_kernel), every simulation in the wide form.
// Returns WAKE_OK after running, or a positive value when the path does not apply (the
// caller then takes the graph path).
int step_batch_pipelined(wake_sim *h, int nsteps) {
  if (h->precision != WAKE_MIXED || !h->batch_pipeline) return 1;
  int max_n1 = 0, max_np = 0;
  for (auto &s : h->sims) {
    if (s.p.n_beam == 0 || !s.beam || !s.plasma) return 1;
    if (s.p.geometry == WAKE_SLAB) return 1;  // the batch pipeline marches the wide (cylindrical) form
    max_n1 = std::max(max_n1, s.p.nr + 1);
    max_np = std::max(max_np, s.np);
  }
  const int ctas_max = batch_step_max_ctas(max_n1, h->batch_nt);
  if (ctas_max < 1) return 1;
  int rc;
  // every beam must slip less than half a cell per step (4x headroom), as for one simulation
  for (auto &s : h->sims) {
    BeamDesc b = beam_desc(s, nullptr);
    CUDA_TRY(cudaMemsetAsync(s.slip, 0, sizeof(unsigned long long) + 64 * sizeof(int), h->stream));
    const double span = 2.0 * (s.p.ximax / s.p.nxi) / (2.0 * s.p.ds);
    beam_slip_kernel<float><<<grid_blocks(s.p.n_beam, 256), 256, 0, h->stream>>>(b, span, s.slip, (int *)(s.slip + 1));
  }
  CUDA_TRY(cudaGetLastError());
  // the largest slip rate and the histogram of steps per cell of each simulation
  std::vector<unsigned long long> slip((size_t)h->n * 33);
  for (int i = 0; i < h->n; ++i)
    CUDA_TRY(cudaMemcpyAsync(&slip[(size_t)i * 33], h->sims[i].slip, sizeof(unsigned long long) + 64 * sizeof(int),
                             cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->n; ++i) {
    double rate;
    std::memcpy(&rate, &slip[(size_t)i * 33], sizeof(rate));
    const Sim &s = h->sims[i];
    if (4.0 * s.p.ds * rate > 0.5 * (s.p.ximax / s.p.nxi)) return 1;
  }
  // steps per launch: the per-step density grids of all simulations within half the free memory
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  size_t per_step = 0;
  for (auto &s : h->sims) per_step += sizeof(float) * s.ng;
  const int chmax = (int)std::max<size_t>(1, std::min<size_t>(nsteps, free_b / 2 / per_step - 1));
  // per-CTA ring and window buffers
  const int ctas = ctas_max;
  const size_t rb = batch_ring_bytes(max_np, h->batch_nt), wb = step_wide_window_bytes(max_n1);
  if (h->bp_rings_bytes < (rb + wb) * ctas) {
    if (h->bp_rings) cudaFree(h->bp_rings);
    h->bp_rings = nullptr;
    h->bp_rings_bytes = 0;
    if ((rc = dalloc(&h->bp_rings, (rb + wb) * ctas))) return rc;
    h->bp_rings_bytes = (rb + wb) * ctas;
  }
  // simulations largest work first
  std::vector<int> order(h->n);
  for (int i = 0; i < h->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)h->sims[a].np * (h->sims[a].p.nxi + 1) > (double)h->sims[b].np * (h->sims[b].p.nxi + 1);
  });
  int done = 0;
  while (done < nsteps) {
    const int ch = std::min(nsteps - done, chmax);
    std::vector<BatchSim> bs(h->n);
    for (int i = 0; i < h->n; ++i) {
      Sim &s = h->sims[i];
      const size_t gbytes = sizeof(float) * s.ng;
      const int dcap = (int)std::min<int64_t>(s.p.n_beam, 4096);
      if (s.pgrid_cap < ch + 1) {
        void *old[] = {s.pgrids, s.progress, s.defer_cnt};
        for (void *q : old)
          if (q) cudaFree(q);
        s.pgrids = nullptr;
        s.progress = nullptr;
        s.defer_cnt = nullptr;
        s.pgrid_cap = 0;
        if ((rc = dalloc(&s.pgrids, gbytes * (ch + 1))) || (rc = dalloc(&s.progress, sizeof(int) * ch)) ||
            (rc = dalloc(&s.defer_cnt, 2 * sizeof(int) * ch)))
          return rc;
        s.pgrid_cap = ch + 1;
      }
      if (s.defer_bytes < sizeof(int2) * (size_t)dcap * ch) {
        if (s.defer_list) cudaFree(s.defer_list);
        s.defer_list = nullptr;
        s.defer_bytes = 0;
        if ((rc = dalloc(&s.defer_list, sizeof(int2) * (size_t)dcap * ch))) return rc;
        s.defer_bytes = sizeof(int2) * (size_t)dcap * ch;
      }
      if ((rc = alloc_target(s))) return rc;
      int occ = 0;
      if ((rc = sort_beam(h, s, &occ))) return rc;
      const int ncap = near_ring(s, occ);
      if ((rc = alloc_near(s, ncap, ch))) return rc;
      BeamDesc b = beam_desc(s, nullptr);
      b.nb = s.pgrids;
      CUDA_TRY(cudaMemsetAsync(s.pgrids, 0, gbytes * (ch + 1), h->stream));
      beam_deposit_kernel<float, float><<<grid_blocks(s.p.n_beam, 256), 256, 0, h->stream>>>(b);
      nb_normalize_kernel<float><<<grid_blocks((int64_t)s.ng, 256), 256, 0, h->stream>>>((float *)s.pgrids, s.p.nr, s.p.nxi,
                                                                                       b.dr, b.dxi, b.slab);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaMemsetAsync(s.progress, 0, sizeof(int) * ch, h->stream));
      CUDA_TRY(cudaMemsetAsync(s.defer_cnt, 0, 2 * sizeof(int) * ch, h->stream));
      CUDA_TRY(cudaMemsetAsync(s.target, 0xff, sizeof(int) * s.target_n, h->stream));
      PipeArgs &a = bs[i].p;
      a = PipeArgs{};
      SimDesc &d = a.d;
      d.nr = s.p.nr;
      d.nxi = s.p.nxi;
      d.np = s.np;
      d.has_beam = 1;
      d.slab = s.p.geometry == WAKE_SLAB;
      d.rmax = s.p.rmax;
      d.ximax = s.p.ximax;
      d.dr = s.p.rmax / s.p.nr;
      d.dxi = s.p.ximax / s.p.nxi;
      d.r0 = s.r0;
      d.ur0 = s.ur0;
      d.lz = s.lz;
      d.G0 = s.G0;
      d.w = s.w;
      d.psi = s.psi;
      d.ez = s.ez;
      d.er = s.er;
      d.bth = s.bth;
      d.status = s.status;
      a.grids = s.pgrids;
      a.ng = s.ng;
      a.progress = s.progress;
      a.nsteps = ch;
      a.write_last = 1;
      a.x = b.x;
      a.y = b.y;
      a.ux = b.ux;
      a.uy = b.uy;
      a.xi = b.xi;
      a.uz = b.uz;
      a.flags = b.lost;
      a.bin_start = s.bin_start;
      a.w = b.w;
      a.ds = s.p.ds;
      a.ffi = b.ffi;
      a.ffx = b.ffx;
      push_consts(a, s.p);
      a.spin_limit = h->spin_limit;
      a.defer_cnt = s.defer_cnt;
      a.defer_list = s.defer_list;
      a.defer_cap = dcap;
      a.near_list = s.near_list;
      a.near_cap = ncap;
      a.target = s.target;
    }
    if ((rc = upload_beam_descs(h))) return rc;  // the sort swapped the beam copies
    std::vector<int2> items;
    items.reserve((size_t)h->n * ch);
    for (int i : order)
      for (int t = 0; t < ch; ++t) items.push_back(make_int2(i, t));
    const size_t sb = sizeof(BatchSim) * h->n, ib = sizeof(int2) * items.size();
    if (h->bp_sims_bytes < sb) {
      if (h->bp_sims) cudaFree(h->bp_sims);
      h->bp_sims = nullptr;
      h->bp_sims_bytes = 0;
      if ((rc = dalloc(&h->bp_sims, sb))) return rc;
      h->bp_sims_bytes = sb;
    }
    if (h->bp_items_bytes < ib) {
      if (h->bp_items) cudaFree(h->bp_items);
      h->bp_items = nullptr;
      h->bp_items_bytes = 0;
      if ((rc = dalloc(&h->bp_items, ib))) return rc;
      h->bp_items_bytes = ib;
    }
    CUDA_TRY(cudaMemcpyAsync(h->bp_sims, bs.data(), sb, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->bp_items, items.data(), ib, cudaMemcpyHostToDevice, h->stream));
    BatchArgs ba{};
    ba.sims = (const BatchSim *)h->bp_sims;
    ba.items = (const int2 *)h->bp_items;
    ba.nitems = (int)items.size();
    ba.ring_bufs = h->bp_rings;
    ba.ring_stride = rb;
    ba.win_bufs = (char *)h->bp_rings + rb * ctas;
    ba.win_stride = wb;
    const int nctas = std::min(ctas, ba.nitems);
    if (h->ev_used == (int)h->ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> q{};
      CUDA_TRY(cudaEventCreate(&q.first));
      if (cudaEventCreate(&q.second) != cudaSuccess) {
        cudaEventDestroy(q.first);
        return fail(WAKE_ECUDA, "cudaEventCreate");
      }
      h->ev.push_back(q);
    }
    CUDA_TRY(cudaEventRecord(h->ev[h->ev_used].first, h->stream));
    const cudaError_t e = launch_batch_steps(ba, max_n1, h->batch_nt, nctas, h->stream);
    if (e != cudaSuccess) return fail(WAKE_ECUDA, std::string("pipelined batch launch: ") + cudaGetErrorString(e));
    CUDA_TRY(cudaEventRecord(h->ev[h->ev_used].second, h->stream));
    ++h->ev_used;
    // the host arrays are read by the copies above: finish them before bs and items go
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (auto &s : h->sims) {
      CUDA_TRY(cudaMemcpyAsync(s.nb, (char *)s.pgrids + sizeof(float) * s.ng * (ch - 1), sizeof(float) * s.ng,
                               cudaMemcpyDeviceToDevice, h->stream));
      s.marched = true;
    }
    done += ch;
  }
  return WAKE_OK;
}

// Several simulations: one step is the batched deposit, one march launch per tile class
// (forked streams), the batched push.  The step is captured once as a CUDA graph and
// replayed; on the legacy default stream, or while the caller is capturing, the launches
// are issued directly.
int step_batched(wake_sim *h, int nsteps) {
  int rc;
  for (auto &s : h->sims)
    if (!s.plasma) return fail(WAKE_ESTATE, "wake_step before wake_load_plasma");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (h->stream) CUDA_TRY(cudaStreamIsCapturing(h->stream, &cs));
  if (!h->planned) {
    if (cs != cudaStreamCaptureStatusNone)
      return fail(WAKE_ESTATE, "the first march of a handle times its tiles: make it before any stream capture");
    if ((rc = plan_tiles(h))) return rc;
  }
  if (!h->stream || cs != cudaStreamCaptureStatusNone) return step_sequential(h, nsteps);
  if (!h->step_graph) {
    CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    rc = step_sequential(h, 1);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(WAKE_ECUDA, std::string("step capture: ") + cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&h->step_graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->step_graph = nullptr;
      return fail(WAKE_ECUDA, std::string("step graph: ") + cudaGetErrorString(ei));
    }
  }
  for (int t = 0; t < nsteps; ++t) CUDA_TRY(cudaGraphLaunch(h->step_graph, h->stream));
  return WAKE_OK;
}

// nsteps beam steps of a single simulation as pipelined cooperative launches (pipeline.cuh).
// Per launch: sort the beam by xi cell, deposit the first step's density into grid 0, zero
// the grids of the later steps and the progress counters, launch.
int step_pipelined(wake_sim *h, int nsteps, int ctas_max, int wide_nt) {
  Sim &s = h->sims[0];
  const int fp64 = h->precision == WAKE_FP64;
  const size_t gs = gsize(h->precision), gbytes = gs * s.ng;
  // every step of a launch owns a density grid: up to a quarter of the free memory
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const int chmax = (int)std::min<size_t>(1024, std::max<size_t>(1, free_b / 4 / gbytes - 1));
  const int wnt = wide_nt;  // 0: the tiled step kernel
  const bool wide64 = wnt && fp64;  // the FP64 wide form: node arrays in the ring buffer
  const size_t rb = wide64 ? wide_fp64_ring_bytes(s.np, s.p.nr + 1)
                           : (wnt ? step_wide_ring_bytes(s.np, wnt) : ring_buf_bytes(h->precision));
  const size_t wb = wide64 ? step_wide_fp64_window_bytes(s.p.nr + 1)
                           : (wnt ? step_wide_window_bytes(s.p.nr + 1) : step_global_window_bytes(h->precision, s.p.nr + 1));
  int rc, done = 0, last_ch = 0;
  // the lists of slipped particles: up to 16 GB (or an eighth of the free memory) for a launch
  const size_t list_budget = std::min<size_t>((size_t)16 << 30, free_b / 8);
  while (done < nsteps) {
    bool ok = false;
    long long hist[64];
    if ((rc = slip_stats(h, s, &ok, hist))) return rc;
    if (!ok) return step_sequential(h, nsteps - done);  // a beam slipping this fast: one step at a time
    // the longest launch whose lists - as long as the budget allows, the prediction being
    // only a guide for a fresh beam whose u_perp is still growing - hold twice the predicted
    // count
    long long L = std::min<long long>(nsteps - done, chmax), dcap_l = 0;
    for (;;) {
      // the second list holds the particles two or more cells past their sorted cell: at most
      // those that slip a cell in fewer than L steps
      long long pred = 0;
      for (int q = 0; q < 64 && (1LL << q) < L; ++q) pred += hist[q];
      dcap_l = std::min<long long>(s.p.n_beam, (long long)(list_budget / (sizeof(int2) * (size_t)L)));
      if (2 * pred <= dcap_l || L == 1) break;
      L = L > ctas_max ? (L - 1) / ctas_max * ctas_max : L / 2;
    }
    dcap_l = std::max<long long>(dcap_l, 1);
    // a launch that does not finish the call ends on a whole wave (the next launch waits for
    // it to drain); one that does keeps every remaining step (its last wave overlaps the
    // tail of the one before)
    if (L < nsteps - done && L >= ctas_max) L = L / ctas_max * ctas_max;
    const int ch = (int)std::max<long long>(1, L);
    const int dcap = (int)dcap_l;
    if (s.pgrid_cap < ch + 1) {
      void *old[] = {s.pgrids, s.progress, s.defer_cnt};
      for (void *q : old)
        if (q) cudaFree(q);
      s.pgrids = nullptr;
      s.progress = nullptr;
      s.defer_cnt = nullptr;
      s.pgrid_cap = 0;
      const int cap = std::min(nsteps, chmax);
      if ((rc = dalloc(&s.pgrids, gbytes * (cap + 1))) || (rc = dalloc(&s.progress, sizeof(int) * cap)) ||
          (rc = dalloc(&s.defer_cnt, 2 * sizeof(int) * cap)))
        return rc;
      s.pgrid_cap = cap + 1;
    }
    if (s.defer_bytes < sizeof(int2) * (size_t)dcap * ch) {
      if (s.defer_list) cudaFree(s.defer_list);
      s.defer_list = nullptr;
      s.defer_bytes = 0;
      if ((rc = dalloc(&s.defer_list, sizeof(int2) * (size_t)dcap * ch))) return rc;
      s.defer_bytes = sizeof(int2) * (size_t)dcap * ch;
    }
    if ((rc = alloc_target(s))) return rc;
    const int ctas = std::min(ch, ctas_max);
    if (rb + wb > 0 && s.pring_bytes < (rb + wb) * ctas) {
      if (s.pring) cudaFree(s.pring);
      s.pring = nullptr;
      s.pring_bytes = 0;
      if ((rc = dalloc(&s.pring, (rb + wb) * ctas))) return rc;
      s.pring_bytes = (rb + wb) * ctas;
    }
    int occ = 0;
    if ((rc = sort_beam(h, s, &occ))) return rc;
    const int ncap = near_ring(s, occ);
    if ((rc = alloc_near(s, ncap, ch))) return rc;
    const BeamDesc bd = beam_desc(s, nullptr);
    {  // beam density of the launch's first step
      BeamDesc b = bd;
      b.nb = s.pgrids;
      CUDA_TRY(cudaMemsetAsync(s.pgrids, 0, gbytes, h->stream));
      const int nbk = grid_blocks(s.p.n_beam, 256), ngk = grid_blocks((int64_t)s.ng, 256);
      if (fp64) {
        beam_deposit_kernel<double, double><<<nbk, 256, 0, h->stream>>>(b);
        nb_normalize_kernel<double><<<ngk, 256, 0, h->stream>>>((double *)s.pgrids, s.p.nr, s.p.nxi, b.dr, b.dxi, b.slab);
      } else {
        beam_deposit_kernel<float, float><<<nbk, 256, 0, h->stream>>>(b);
        nb_normalize_kernel<float><<<ngk, 256, 0, h->stream>>>((float *)s.pgrids, s.p.nr, s.p.nxi, b.dr, b.dxi, b.slab);
      }
      CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(cudaMemsetAsync((char *)s.pgrids + gbytes, 0, gbytes * ch, h->stream));
    CUDA_TRY(cudaMemsetAsync(s.progress, 0, sizeof(int) * ch, h->stream));
    CUDA_TRY(cudaMemsetAsync(s.defer_cnt, 0, 2 * sizeof(int) * ch, h->stream));
    CUDA_TRY(cudaMemsetAsync(s.target, 0xff, sizeof(int) * s.target_n, h->stream));  // -1: no target
    PipeArgs a{};
    SimDesc &d = a.d;
    d.nr = s.p.nr;
    d.nxi = s.p.nxi;
    d.np = s.np;
    d.has_beam = 1;
    d.slab = s.p.geometry == WAKE_SLAB;
    d.rmax = s.p.rmax;
    d.ximax = s.p.ximax;
    d.dr = s.p.rmax / s.p.nr;
    d.dxi = s.p.ximax / s.p.nxi;
    d.r0 = s.r0;
    d.ur0 = s.ur0;
    d.lz = s.lz;
    d.G0 = s.G0;
    d.w = s.w;
    d.ring_buf = s.ring_buf;
    d.nb = nullptr;
    d.psi = s.psi;
    d.ez = s.ez;
    d.er = s.er;
    d.bth = s.bth;
    d.status = s.status;
    a.grids = s.pgrids;
    a.ng = s.ng;
    a.progress = s.progress;
    a.nsteps = ch;
    a.write_last = 1;
    a.x = bd.x;
    a.y = bd.y;
    a.ux = bd.ux;
    a.uy = bd.uy;
    a.xi = bd.xi;
    a.uz = bd.uz;
    a.flags = bd.lost;
    a.bin_start = s.bin_start;
    a.w = bd.w;
    a.ds = s.p.ds;
    a.ffi = bd.ffi;
    a.ffx = bd.ffx;
    push_consts(a, s.p);
    a.spin_limit = h->spin_limit;  // polls of >= 128 ns: by default a wait gives up after seconds
    a.ring_bufs = s.pring;
    a.ring_stride = rb;
    a.win_bufs = wb > 0 ? (char *)s.pring + rb * ctas : nullptr;
    a.win_stride = wb;
    a.defer_cnt = s.defer_cnt;
    a.defer_list = s.defer_list;
    a.defer_cap = dcap;
    a.near_list = s.near_list;
    a.near_cap = ncap;
    a.target = s.target;
    if (h->ev_used == (int)h->ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> q{};
      CUDA_TRY(cudaEventCreate(&q.first));
      if (cudaEventCreate(&q.second) != cudaSuccess) {
        cudaEventDestroy(q.first);
        return fail(WAKE_ECUDA, "cudaEventCreate");
      }
      h->ev.push_back(q);
    }
    CUDA_TRY(cudaEventRecord(h->ev[h->ev_used].first, h->stream));
    const cudaError_t e = wide64 ? launch_step_wide_fp64(a, ctas, h->stream)
                                 : (wnt ? launch_step_wide(a, wnt, ctas, h->stream) : launch_step(h->precision, a, s.np, ctas, h->stream));
    if (e != cudaSuccess) return fail(WAKE_ECUDA, std::string("pipelined step launch: ") + cudaGetErrorString(e));
    CUDA_TRY(cudaEventRecord(h->ev[h->ev_used].second, h->stream));
    ++h->ev_used;
    done += ch;
    last_ch = ch;
    // the density the launch's last march used
    CUDA_TRY(cudaMemcpyAsync(s.nb, (char *)s.pgrids + gbytes * (last_ch - 1), gbytes, cudaMemcpyDeviceToDevice,
                             h->stream));
    s.marched = true;
  }
  return WAKE_OK;
}

}  // namespace

int wake_step(wake_sim *h, int nsteps) {
  if (!h || nsteps < 0) return fail(WAKE_EINVAL, "wake_step: null handle or nsteps < 0");
  h->ev_used = 0;
  if (nsteps == 0) return WAKE_OK;
  if (h->n == 1 && h->sims[0].trap_gamma > 0.0) return step_sequential(h, nsteps);  // trapping: step by step
  if (h->n == 1 && h->sims[0].p.n_beam > 0) {
    Sim &s = h->sims[0];
    if (!s.beam || !s.plasma) return fail(WAKE_ESTATE, "wake_step needs wake_load_plasma and wake_load_beam");
    int wnt = s.wide ? 512 : 0;
    if (h->precision == WAKE_MIXED && (h->step_form == 256 || h->step_form == 512)) wnt = h->step_form;
    const int ctas = (wnt && h->precision == WAKE_FP64) ? step_wide_fp64_max_ctas(s.p.nr + 1)
                     : wnt ? step_wide_max_ctas(s.p.nr + 1, wnt) : step_max_ctas(h->precision, s.p.nr + 1, s.np);
    if (ctas > 0) return step_pipelined(h, nsteps, ctas, wnt);
  }
  if (h->n > 1) {
    const int rc = step_batch_pipelined(h, nsteps);
    if (rc <= 0) return rc;
    return step_batched(h, nsteps);
  }
  return step_sequential(h, nsteps);
}

int wake_tile(wake_sim *h, int sim, int *nt, int *ppt) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  if (!nt || !ppt) return fail(WAKE_EINVAL, "wake_tile: null output");
  *nt = *ppt = 0;
  if (h->planned) {
    const TileFns &f = h->classes[h->tile_of[sim]].fns;
    *nt = f.nt;
    *ppt = f.ppt;
  }
  return WAKE_OK;
}

int wake_step_kernel_ms(wake_sim *h, float *ms) {
  if (!h || !ms) return fail(WAKE_EINVAL, "wake_step_kernel_ms: null argument");
  float tot = 0.0f;
  for (int i = 0; i < h->ev_used; ++i) {
    float t = 0.0f;
    CUDA_TRY(cudaEventSynchronize(h->ev[i].second));
    CUDA_TRY(cudaEventElapsedTime(&t, h->ev[i].first, h->ev[i].second));
    tot += t;
  }
  *ms = tot;
  return WAKE_OK;
}

int wake_get_fields(wake_sim *h, int sim, double *psi, double *ez, double *er, double *bth) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  Sim &s = h->sims[sim];
  if (!s.marched) return fail(WAKE_ESTATE, "wake_get_fields before a march");
  void *src[4] = {s.psi, s.ez, s.er, s.bth};
  double *dst[4] = {psi, ez, er, bth};
  for (int q = 0; q < 4; ++q) {
    if (!dst[q]) continue;
    if (h->precision == WAKE_FP64) {
      CUDA_TRY(cudaMemcpyAsync(dst[q], src[q], sizeof(double) * s.ng, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      widen_kernel<float><<<grid_blocks((int64_t)s.ng, 256), 256, 0, h->stream>>>((const float *)src[q], dst[q], (int64_t)s.ng);
      CUDA_TRY(cudaGetLastError());
    }
  }
  return WAKE_OK;
}

int wake_get_nb(wake_sim *h, int sim, double *nb) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  Sim &s = h->sims[sim];
  if (!nb) return fail(WAKE_EINVAL, "null output");
  if (h->precision == WAKE_FP64) {
    CUDA_TRY(cudaMemcpyAsync(nb, s.nb, sizeof(double) * s.ng, cudaMemcpyDeviceToDevice, h->stream));
  } else {
    widen_kernel<float><<<grid_blocks((int64_t)s.ng, 256), 256, 0, h->stream>>>((const float *)s.nb, nb, (int64_t)s.ng);
    CUDA_TRY(cudaGetLastError());
  }
  return WAKE_OK;
}

int wake_get_beam(wake_sim *h, int sim, double *xyz, uint8_t *lost) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  Sim &s = h->sims[sim];
  if (!s.beam) return fail(WAKE_ESTATE, "wake_get_beam before wake_load_beam");
  const int64_t n = s.p.n_beam;
  BeamDesc b = beam_desc(s, nullptr);
  const int nb = grid_blocks(n, 256);
  if (h->precision == WAKE_FP64)
    beam_unpermute_kernel<double><<<nb, 256, 0, h->stream>>>(b, xyz, lost);
  else
    beam_unpermute_kernel<float><<<nb, 256, 0, h->stream>>>(b, xyz, lost);
  CUDA_TRY(cudaGetLastError());
  return WAKE_OK;
}

int wake_diagnostics(wake_sim *h, double *out_host) {
  if (!h || !out_host) return fail(WAKE_EINVAL, "wake_diagnostics: null argument");
  CUDA_TRY(cudaMemsetAsync(h->d_diag, 0, sizeof(double) * 5 * h->n, h->stream));
  for (int i = 0; i < h->n; ++i) {
    Sim &s = h->sims[i];
    if (s.p.n_beam == 0 || !s.beam) continue;
    BeamDesc b = beam_desc(s, h->d_diag + 5 * i);
    const int nb = grid_blocks(s.p.n_beam, 256);
    if (h->precision == WAKE_FP64)
      beam_diag_kernel<double><<<nb, 256, 0, h->stream>>>(b);
    else
      beam_diag_kernel<float><<<nb, 256, 0, h->stream>>>(b);
    CUDA_TRY(cudaGetLastError());
  }
  std::vector<double> acc(5 * h->n);
  CUDA_TRY(cudaMemcpyAsync(acc.data(), h->d_diag, sizeof(double) * 5 * h->n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->n; ++i) {
    const double *a = &acc[5 * i];
    const double gb = h->sims[i].p.gamma_b;
    double *o = out_host + 5 * i;
    o[0] = a[0];
    o[1] = a[0] > 0 ? gb + a[1] / a[0] : 0.0;
    o[2] = a[0] > 0 ? std::sqrt(std::max(a[2] / a[0] - (a[1] / a[0]) * (a[1] / a[0]), 0.0)) : 0.0;
    o[3] = a[3];
    o[4] = a[3] > 0 ? gb + a[4] / a[3] : 0.0;
  }
  return WAKE_OK;
}

int wake_status(wake_sim *h, int sim) {
  int rc = check_handle(h, sim);
  if (rc) return rc;
  int st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, h->sims[sim].status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (st & ST_NUMERIC) return fail(WAKE_ENUMERIC, "Gamma <= 0 or a non-finite field in the march");
  if (st & ST_ESCAPE) return fail(WAKE_EESCAPE, "a plasma ring left [0, rmax]");
  if (st & ST_TIMEOUT) return fail(WAKE_ETIMEOUT, "a bounded device wait gave up");
  if (st & ST_DRIFT) return fail(WAKE_ESTATE, "a beam particle was found behind the xi cell it was sorted into");
  if (st & ST_LISTFULL) return fail(WAKE_ESTATE, "more beam particles slipped past their xi cells than a pipelined step's lists hold");
  return WAKE_OK;
}

void wake_destroy(wake_sim *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (auto &s : h->sims) free_sim(s);
  if (h->d_desc) cudaFree(h->d_desc);
  if (h->d_order) cudaFree(h->d_order);
  if (h->d_diag) cudaFree(h->d_diag);
  if (h->d_probe) cudaFree(h->d_probe);
  if (h->d_probe_status) cudaFree(h->d_probe_status);
  if (h->d_probe_order) cudaFree(h->d_probe_order);
  for (auto &k : h->classes) {
    if (k.side) cudaStreamDestroy(k.side);
    if (k.done) cudaEventDestroy(k.done);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->step_graph) cudaGraphExecDestroy(h->step_graph);
  if (h->bp_rings) cudaFree(h->bp_rings);
  if (h->bp_sims) cudaFree(h->bp_sims);
  if (h->bp_items) cudaFree(h->bp_items);
  if (h->d_bdesc) cudaFree(h->d_bdesc);
  for (auto &q : h->ev) {
    cudaEventDestroy(q.first);
    cudaEventDestroy(q.second);
  }
  delete h;
}

}  // extern "C"
