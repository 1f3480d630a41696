/*
 * wake.h -- C ABI of libwake, a GB300 (sm_103a) implementation of the quasi-static r-xi
 * plasma-wakefield method of Jain, Palastro, Antonsen, Mori & An, "Plasma wakefield
 * acceleration studies using the quasi-static code WAKE" (arXiv:1411.3246).
 *
 * Conventions (all entry points):
 *   - Units are normalised: lengths k_p^-1, time omega_p^-1, momenta m c, potentials
 *     m c^2/e, fields E_0 = m c omega_p/e, densities n_p.  Electrons have charge -1.
 *   - Array arguments are DEVICE pointers owned by the caller unless stated otherwise;
 *     the library never frees them.  The library owns only the scratch it allocates in
 *     wake_init and frees in wake_destroy.
 *   - Calls are asynchronous on the CUDA stream given to wake_init, except those documented
 *     as synchronous (wake_diagnostics, wake_status).
 *   - Every call returns WAKE_OK (0) or a negative WAKE_E* code; wake_last_error() gives a
 *     thread-local message for the last failure.  A numeric fault inside a kernel is sticky
 *     in a per-simulation device status word and is reported by wake_status.
 *   - Grids are node-centred: r_i = i dr (i = 0..nr, dr = rmax/nr) and xi_k = k dxi
 *     (k = 0..nxi, dxi = ximax/nxi); a grid array is (nxi+1) x (nr+1), slice-major
 *     (index k*(nr+1) + i).
 */
#ifndef WAKE_H
#define WAKE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WAKE_OK 0
#define WAKE_EINVAL (-1)   /* bad argument or parameter                              */
#define WAKE_ENOMEM (-2)   /* device allocation failed                               */
#define WAKE_ECUDA (-3)    /* CUDA runtime error (launch or copy)                    */
#define WAKE_ENUMERIC (-4) /* Gamma <= 0 or a non-finite value in the march          */
#define WAKE_ETIMEOUT (-5) /* a bounded device wait gave up                          */
#define WAKE_EESCAPE (-6)  /* a plasma ring left [0, rmax]                           */
#define WAKE_ESTATE (-7)   /* call out of order (e.g. push before any march)         */

#define WAKE_FP64 0    /* FP64 throughout                                            */
#define WAKE_MIXED 1   /* FP32 particle arithmetic and fields; charge sums in exact    */
                       /* fixed point, scans in float-float, FP32 tridiagonal solve;   */
                       /* the beam's xi and u_z held as float-float pairs              */
#define WAKE_MIXED64 2 /* FP32 particle arithmetic and fields; the sums across rings,  */
                       /* the scans and the tridiagonal solve in FP64 (charge sums in  */
                       /* exact fixed point); beam as in WAKE_MIXED                    */

/*
 * Parameters of one simulation (Sec. II, Eq. 12, Table I notation):
 *   nr, nxi      radial and longitudinal cells of the box [0, rmax] x [0, ximax]
 *   ppc          plasma rings per radial cell (even when u_th > 0)
 *   precision    WAKE_FP64, WAKE_MIXED or WAKE_MIXED64 (all simulations of one handle must
 *                agree)
 *   u_th         thermal momentum of the Maxwellian plasma, per component (0: cold)
 *   n_d, n_w, sigma_r, sigma_zd, sigma_zw, xi_d, xi_w
 *                the two-bunch driver density of Eq. 12
 *   gamma_b, eps_n   beam Lorentz factor and normalised emittance (u_perp spread
 *                    eps_n/sigma_r)
 *   ds           beam time step (Eqs. 8-11)
 *   n_beam       beam macroparticles (0: the driver is Eq. 12 itself, frozen)
 *   n_drive      the first n_drive beam particles form the drive bunch, the rest the
 *                witness
 */
typedef struct wake_params {
  int32_t nr, nxi, ppc, precision;
  double rmax, ximax, u_th;
  double n_d, n_w, sigma_r, sigma_zd, sigma_zw, xi_d, xi_w;
  double gamma_b, eps_n, ds;
  int64_t n_beam, n_drive;
  int32_t geometry; /* WAKE_CYLINDRICAL (0) or WAKE_SLAB (1) */
  int32_t reserved; /* 0 */
} wake_params;

/*
 * Geometry (Sec. I: WAKE handles cylindrical and slab geometry).  WAKE_CYLINDRICAL is the
 * (r, xi) model of Sec. II.A.  WAKE_SLAB reads it with d/dy = 0 in place of d/dtheta = 0: the
 * transverse coordinate is x >= 0 with a mirror plane at x = 0 (psi and E_z even, E_x and B_y
 * odd) and a conducting wall at x = rmax; volumes are per unit area (hat widths dx, halved at
 * x = 0 and at the wall); lap_perp = d_x^2 and Eq. 6 reads d_x B_y = d_xi^2 psi + J_z; the
 * plasma particles are sheets whose conserved u_y enters gamma only (Eq. 4 has no centrifugal
 * term); the beam is a sheet beam at y = u_y = 0, its density folded onto x >= 0 with the
 * bunch weight n sqrt(2 pi) sigma_z * sigma_r sqrt(2 pi)/2 (the half-slab integral).  The
 * fields keep their names: er is E_x, bth is B_y.  Slab simulations use the 512-thread
 * shared-memory march forms with up to 8 rings per thread (nr*ppc <= 4096, and within one
 * CTA's shared memory), and have no trapping and no adjoint.
 */
#define WAKE_CYLINDRICAL 0
#define WAKE_SLAB 1

typedef struct wake_sim wake_sim; /* opaque handle: n_sims independent simulations */

/*
 * Create n_sims independent simulations, p[0..n_sims-1] (sizes may differ), bound to the
 * CUDA stream `stream` (a cudaStream_t; NULL = legacy default stream).  Allocates all
 * scratch: plasma rings, beam state, the beam-density and field grids.  A simulation with
 * n_beam == 0 gets the frozen analytic driver of Eq. 12 on its nodes.
 * Errors: WAKE_EINVAL (geometry not 0 or 1, or a slab simulation too large for the shared-memory
 * march; sizes out of range: 2 <= nxi, 1 <= ppc; FP64 and mixed 2 <= nr <= 2048
 * and nr*ppc <= 65536 (beyond 1,024 cells or 8,192 rings the FP64 form marches in its wide
 * form, node arrays in global memory, far slower); WAKE_MIXED64 2 <= nr <= 1024, nr*ppc <= 8192
 * and within one CTA's shared memory (about 4,500 rings at nr = 512); precision mismatch),
 * WAKE_ENOMEM, WAKE_ECUDA.
 */
int wake_init(const wake_params *p, int n_sims, void *stream, wake_sim **out);

/*
 * Initial plasma slice of simulation `sim` (Sec. II.A): rings at their cell positions,
 * weights with the quasi-static flux factor 1 - v_z0, Gamma_0 = gamma_0 - u_z0 (Eq. 1),
 * l_z = r u_theta0.  `normals` is a device array of nr*ppc*3 standard normals
 * (u_r, u_theta, u_z per ring, row-major, mirrored in pairs), scaled by u_th; it may be
 * NULL only for a cold plasma (u_th == 0).  Must be called before the first march.
 */
int wake_load_plasma(wake_sim *s, int sim, const double *normals);

/*
 * Initial beam of simulation `sim` (Eq. 12 bunches): `normals` is a device array of
 * 5 x n_beam standard normals (rows x, y, u_x, u_y, xi); x = sigma_r n, u_perp =
 * (eps_n/sigma_r) n, xi = xi_d + sigma_zd n (drive) or xi_w + sigma_zw n (witness),
 * u_z = gamma_b.  Particles outside 0 <= xi < ximax or r >= rmax start lost.
 */
int wake_load_beam(wake_sim *s, int sim, const double *normals);

/*
 * A beam of simulation `sim` given by the caller (a beam from another code, another bunch
 * shape, or a state saved with wake_get_beam): xyz is a device array of 6 x n_beam doubles in
 * wake_get_beam's layout (rows x, y, xi, u_x, u_y, u_z); w a device array of n_beam charge
 * weights per 2 pi (NULL: the Eq. 12 bunch weights, as wake_load_beam gives them); tag a
 * device array of n_beam bytes, nonzero for witness particles (NULL: the particles from
 * n_drive on).  Particles outside 0 <= xi < ximax, r < rmax start lost.  Replaces the beam
 * state; wake_get_beam returns particles in this order.  Slab geometry: y and u_y are taken
 * as 0 (a sheet beam).
 */
int wake_set_beam(wake_sim *s, int sim, const double *xyz, const double *w, const uint8_t *tag);

/* Beam -> (r, xi) grid density of every simulation with a beam (bilinear hats divided by
 * the hats' ring volumes).  Needs wake_load_beam. */
int wake_beam_deposit(wake_sim *s);

/*
 * The quasi-static xi-march of every simulation with its beam frozen (Sec. II.A, Eqs. 1-7):
 * per slice, RK2 push of the plasma rings, deposit, and the radial solves for psi, E_z,
 * B_theta and E_r, written to the handle's field grids.  Needs wake_load_plasma (and a
 * beam deposit for simulations with a beam).
 */
int wake_plasma_march(wake_sim *s);

/*
 * The march of simulation `sim` alone, as wake_plasma_march does it (fields to the handle's
 * grids), that also records the plasma rings' trajectories (Sec. IV, Figs. 4-5: electron
 * trajectories in the cold and the warm plasma).  At every slice k = 0, every, 2 every, ...
 * <= nxi, ring j's radius r, radial momentum u_r and Gamma = gamma - u_z (Eq. 1, at the slice's
 * first RK2 stage) go to traj[((k / every) * 3 + q) * np + j], q = 0 (r), 1 (u_r), 2 (Gamma),
 * np = nr * ppc, j the ring's index in the initial slice (cell-major, as wake_load_plasma
 * lays the rings out).
 *   every  >= 1
 *   traj   device, (nxi / every + 1) * 3 * np doubles, caller-owned, overwritten
 * One CTA of 512 threads runs the march, so the simulation must fit one: nr + 1 <= 1536 and
 * its rings in shared memory (the tile form; not the wide form of wake_tile).  WAKE_FP64 and
 * WAKE_MIXED handles only.  Asynchronous.
 * Errors: WAKE_EINVAL (bad sim, every < 1, null traj, too large), WAKE_ESTATE (no plasma),
 * WAKE_ECUDA.
 */
int wake_plasma_march_traj(wake_sim *s, int sim, int every, double *traj);

/* One beam time step of length ds (Eqs. 8-11, Boris) through the fields of the last march,
 * for every simulation with a beam.  Needs a march. */
int wake_beam_push(wake_sim *s);

/* nsteps beam time steps through the same fields (the wake of the last march held frozen:
 * the beam pushed as test particles, with no deposit or march in between); nsteps >= 0.
 * Errors as wake_beam_push. */
int wake_beam_push_steps(wake_sim *s, int nsteps);

/*
 * Caller-owned field grids for simulation `sim` (Eqs. 6-7 output): from now on every march
 * and step writes psi, E_z, E_r and B_theta (slab: E_x, B_y) of the simulation straight into
 * these device arrays, and the beam push reads them there; the library frees its own grids and
 * never frees these.  Each is (nxi + 1) x (nr + 1), slice-major, double (WAKE_FP64) or float
 * (mixed forms), and must stay valid until wake_destroy.  wake_get_fields still copies from
 * them.  Call before the first march or step of the handle.  Synchronises the stream.
 * Errors: WAKE_EINVAL (bad sim, a null pointer), WAKE_ESTATE (after a march or step), WAKE_ECUDA.
 */
int wake_bind_fields(wake_sim *s, int sim, void *psi, void *ez, void *er, void *bth);

/*
 * nsteps x (wake_beam_deposit, wake_plasma_march, wake_beam_push).  With several
 * simulations of the mixed form that all have beams, every simulation's steps run pipelined
 * (as below) in one persistent cooperative launch, largest simulations first, each march in
 * the wide form (the environment variable WAKE_BATCH_PIPELINE=0, read by wake_init, turns
 * this off).  Otherwise, with several simulations, one step is a batched deposit, one march
 * launch per tile class (concurrent streams) and a batched push; the first call captures that
 * step as a CUDA graph on the handle's stream and every call replays it nsteps times (on the
 * legacy default stream, or while the caller's stream is capturing, the launches are issued
 * directly).  With one simulation
 * that has a beam, the steps run pipelined: the beam is sorted by xi cell and one
 * cooperative launch marches up to one step per SM, each step two slices behind the one
 * before, pushing each cell of the beam as soon as its fields are solved (same arithmetic as
 * the separate calls; only the order of the deposit sums differs).  A step whose wait for the
 * step before it gives up (after WAKE_SPIN_LIMIT polls of >= 128 ns, the environment variable
 * read by wake_init; default 2^24) leaves cleanly and raises WAKE_ETIMEOUT through wake_status.
 * A particle that slips past the cell it was sorted into during a launch is pushed with the
 * cell it has reached.  The beam must slip less than a cell per step: a beam whose fastest
 * particle, measured at the start of each launch, slips more than 1/8 of a cell per step
 * takes the separate calls (the check synchronises the stream once per launch).  A particle
 * found behind the cell it was sorted into, or more slipped particles than the launch's
 * lists hold, raise WAKE_ESTATE through wake_status.
 */
int wake_step(wake_sim *s, int nsteps);

/*
 * The march tile simulation `sim` runs in: nt threads per CTA, ppt rings per thread.  With
 * several simulations the first march chooses each simulation's tile by timing the compiled
 * candidates on a short probe march (synchronous: make that first march before any stream
 * capture); the environment variable WAKE_TILE_NT (128, 256 or 512), read by wake_init,
 * restricts the choice to one width.  A mixed simulation too large for any tile (more than
 * 768 radial cells with more than 4096 rings, up to nr = 2048 and 65,536 rings) runs in the
 * wide form, which keeps its rings in a global buffer and processes them in chunks of
 * 512 x 8 (nt = 512, ppt = 8 here); WAKE_TILE_NT=-1 forces the wide form.  Before the first
 * march both are 0.  Instrumentation and tuning: the paper has no counterpart.
 */
int wake_tile(wake_sim *s, int sim, int *nt, int *ppt);

/*
 * Device time in milliseconds of the pipelined step kernels launched by the last wake_step
 * call (0 if it took the separate calls), measured with CUDA events on the handle's stream;
 * synchronous.  Instrumentation only: the paper has no counterpart.
 */
int wake_step_kernel_ms(wake_sim *s, float *ms);

/*
 * Plasma-particle trapping for simulation `sim` (Sec. I: plasma particles that meet a
 * threshold condition are promoted to beam particles, which then follow the full equations
 * of motion, Eqs. 8-11).  The paper gives no condition; the library's reading: after the first
 * RK2 stage of a slice, a ring whose Gamma = gamma - u_z = Gamma_0 + psi (Eq. 1) is below
 * gamma_t moves almost with the wake (1 - v_z = Gamma / gamma) and leaves the quasi-static
 * plasma (it still counts in that slice's fields; its weight is zero from then on).  Before
 * the next push, each promoted ring becomes one beam particle: at (x, y) = (r, 0), xi = the
 * slice's, momentum (u_r, u_theta, u_z) with u_z from Eqs. 2-3 for its Gamma, charge weight
 * w ds (the ring's flux over one beam step), neither drive nor witness (wake_diagnostics
 * leaves it out); in the field equations it is a beam particle like the bunches.  The beam's
 * arrays get room for `capacity` promoted particles; promotions beyond it are counted and
 * dropped.  The same plasma is marched every step, so a ring may be promoted at every step.
 *   gamma_t   threshold (> 0; 0 keeps the arrays but promotes nothing)
 *   capacity  promoted particles the beam can hold (>= 0)
 * Needs a handle of one simulation with a particle beam, FP64 or WAKE_MIXED, cylindrical, that
 * fits one 512-thread march CTA; call it before wake_load_beam / wake_set_beam (the beam's arrays are
 * reallocated).  With trapping on, wake_step takes the separate calls (deposit, march, push).
 * Errors: WAKE_EINVAL, WAKE_ESTATE (beam already loaded), WAKE_ENOMEM, WAKE_ECUDA.
 */
int wake_set_trapping(wake_sim *s, int sim, double gamma_t, int64_t capacity);

/*
 * The particles promoted so far in simulation `sim`, in the order they were promoted (by beam
 * step, then slice, then ring): *count of them (host), and *dropped promotions that found no
 * room (host).  Any of xyz (6 x capacity doubles, rows x, y, xi, u_x, u_y, u_z), w (capacity
 * charge weights) and lost (capacity bytes) may be NULL; the first *count entries of each are
 * written (device arrays).  Synchronous.
 */
int wake_trapped(wake_sim *s, int sim, double *xyz, double *w, uint8_t *lost, int64_t *count, int64_t *dropped);

/* Copy the last march's fields of `sim` to caller-owned device arrays of (nxi+1)*(nr+1)
 * doubles each (any pointer may be NULL). */
int wake_get_fields(wake_sim *s, int sim, double *psi, double *ez, double *er, double *bth);

/* Copy the beam-density grid of `sim` ((nxi+1)*(nr+1) doubles, device). */
int wake_get_nb(wake_sim *s, int sim, double *nb);

/* Copy the beam state of `sim`: xyz is 6 x n_beam doubles (rows x, y, xi, u_x, u_y, u_z),
 * lost is n_beam bytes (1 = lost); either may be NULL.  Device pointers. */
int wake_get_beam(wake_sim *s, int sim, double *xyz, uint8_t *lost);

/* Witness and drive statistics of every simulation (Sec. IV), synchronous.  out_host holds
 * 5 doubles per simulation: surviving witness count, witness mean gamma, witness rms gamma
 * spread, surviving drive count, drive mean gamma. */
int wake_diagnostics(wake_sim *s, double *out_host);

/* Synchronous: WAKE_OK, or the sticky error of simulation `sim` (WAKE_ENUMERIC,
 * WAKE_EESCAPE, WAKE_ETIMEOUT) raised by a kernel. */
int wake_status(wake_sim *s, int sim);

/*
 * Largest grid, in nodes (nxi+1)*(nr+1), that wake_beam_deposit_noalloc accepts: its
 * accumulation grid is a static device array of this many doubles (4 MiB).
 */
#define WAKE_NOALLOC_MAX_NODES 524288

/*
 * wake_beam_deposit without a handle and without allocating any memory: the beam density on
 * the (r, xi) nodes of the grid that p describes, from a beam the caller holds.  The paper
 * has no counterpart.  It serves callers that must not allocate device memory: code running
 * while a caching allocator (PyTorch's, or the caller's own pool) holds the device's memory,
 * where a cudaMalloc could fail or make the pool give back its cached blocks, and code that
 * cannot take the device-wide synchronisation of cudaFree among concurrent streams.
 *   p       host pointer; reads nr, nxi, rmax, ximax, n_d, n_w, sigma_r, sigma_zd, sigma_zw,
 *           n_beam and n_drive (the bunch macroparticle weights, as wake_beam_deposit takes
 *           them); precision is ignored (FP64 throughout)
 *   xyz     device, 6 x n_beam doubles in wake_get_beam's layout (rows x, y, xi, u_x, u_y,
 *           u_z; only x, y and xi are read, y not in the slab geometry); the first n_drive
 *           particles are the drive bunch
 *   lost    device, n_beam bytes, nonzero = lost (NULL: none lost); a particle outside
 *           0 <= xi < ximax, r < rmax also counts as lost
 *   stream  a cudaStream_t of the current device (NULL = legacy default stream); the call is
 *           asynchronous
 *   nb      device output, (nxi+1)*(nr+1) doubles, overwritten
 * The arithmetic is that of wake_beam_deposit's FP64 form; results agree up to the order of
 * the atomic sums.  Scratch: a static device array of WAKE_NOALLOC_MAX_NODES doubles, which
 * each call zeroes on `stream` before it accumulates there; larger grids are rejected.  The
 * first call on a device looks up that array's address (cudaGetSymbolAddress), which may load
 * the library's device code: make it before any stream capture.  The address is cached per
 * device index; the cache is dropped when a launch fails, and does not survive
 * cudaDeviceReset (after a reset, a call whose launch fails returns WAKE_ECUDA and the next
 * call looks the address up again).  Calls that overlap in time
 * (on other streams or from other host threads) share the array and race: order them on one
 * stream.
 * Errors: WAKE_EINVAL (null p or nb, xyz NULL with n_beam > 0, sizes or grid out of range),
 * WAKE_ECUDA.
 */
int wake_beam_deposit_noalloc(const wake_params *p, const double *xyz, const uint8_t *lost, void *stream,
                              double *nb);

/*
 * The adjoint form: gradients of the witness bunch's observables (Sec. IV: mean energy gain
 * <gamma - gamma_b> and rms energy spread over the surviving witness particles, weighted by
 * their charge) after nsteps beam steps, with respect to
 *   theta[0] = n_w          witness peak density of Eq. 12 (its charge is proportional)
 *   theta[1] = xi_w - xi_d  witness delay
 *   theta[2] = sigma_zd     drive bunch length (its peak density n_d held fixed)
 *   theta[3] = u_th         plasma temperature (Sec. II.A Maxwellian)
 * and nbins multipliers of the witness current profile: witness macroparticle j carries
 * weight n_w-bunch weight x profile[b], b its bin of xi_w +- 3 sigma_zw (from its initial
 * draw).  FP64 throughout.  The paper differentiates nothing: this form serves the parameter
 * studies of its Sec. IV.
 * The beam steps run pipelined (unless WAKE_ADJOINT_PIPELINE=0, or a beam slips fast enough to
 * cross a xi cell within the run, or fewer than two steps fit): one CTA marches each step, a
 * few slices behind the step before, pushing each xi cell of the beam as soon as its fields
 * are solved; the reverse runs the same way in -xi, each step a few slices behind the step
 * after it.  The reverse needs every slice's intermediates: the forward keeps them all when
 * they take at most a quarter of the free device memory at wake_adjoint_init (about
 * nsteps x (Nxi + 1) x (2 x 13 (Nr + 1) + 23 Np) x 8 bytes; WAKE_ADJOINT_FULL_TAPE=0 declines),
 * else it keeps the ring state every ~sqrt(Nxi + 1) slices and the reverse recomputes each
 * block from it.  The waits are bounded (WAKE_SPIN_LIMIT polls of >= 128 ns; a wait that gives
 * up returns WAKE_ETIMEOUT).
 *
 * wake_adjoint_init: p gives the grid, box, bunches (n_d, sigma_r, sigma_zw, xi_d, gamma_b,
 * eps_n, ds, n_beam, n_drive; the theta entries of p are ignored).  Cylindrical geometry
 * only.  Needs nr <= 256, an even
 * ppc, 0 < n_drive < n_beam, 0 <= nbins <= 1024.  Allocates everything (beam states, densities
 * and fields of every step: about (nsteps + 1) x 49 x n_beam + nsteps x 32 x (Nxi+1)(Nr+1)
 * bytes, plus the tape above and per-CTA scratch).
 * wake_adjoint_forward: theta (host, 4), profile (host, nbins; NULL if nbins == 0),
 * plasma_normals (device, nr*ppc*3 mirrored pairs as wake_load_plasma takes them) and
 * beam_normals (device, 5 x n_beam as wake_load_beam takes them; both must stay valid until
 * the next forward) -> obs (host, 2): mean gain, rms spread.  Synchronous.
 * wake_adjoint_backward: dobs (host, 2) = dL/dobs -> grad (host, 4 + nbins) = dL/dtheta,
 * dL/dprofile, for the last forward.  Synchronous.
 * Errors: WAKE_EINVAL, WAKE_ENOMEM, WAKE_ECUDA, WAKE_ENUMERIC, WAKE_EESCAPE, WAKE_ETIMEOUT,
 * WAKE_ESTATE (no surviving witness, backward before forward, or a beam particle that slipped
 * more than one xi cell during a pipelined run).
 */
typedef struct wake_adj wake_adj;
int wake_adjoint_init(const wake_params *p, int nsteps, int nbins, void *stream, wake_adj **out);
int wake_adjoint_forward(wake_adj *a, const double *theta, const double *profile, const double *plasma_normals,
                         const double *beam_normals, double *obs);
int wake_adjoint_backward(wake_adj *a, const double *dobs, double *grad);
void wake_adjoint_destroy(wake_adj *a);

/* Thread-local message describing the last failed call (never NULL). */
const char *wake_last_error(void);

/* Free all scratch of the handle (synchronises its stream). */
void wake_destroy(wake_sim *s);

#ifdef __cplusplus
}
#endif
#endif /* WAKE_H */
