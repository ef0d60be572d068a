/*
 * otf_md.h - C ABI of the GB300 on-the-fly property library.
 *
 * The library runs a Lennard-Jones molecular-dynamics system on one GPU and
 * computes, while it runs, the quantities of arXiv 2503.07526 ("DL_POLY 5:
 * Calculation of system properties on the fly for very large systems via
 * massive parallelism"): the system stress tensor and heat flux every step
 * (Sec. 2.3), multiple-tau correlators of the off-diagonal stress, the heat
 * flux and every atom's velocity (Sec. 2.2, Appendix D Algorithms 1-2), and
 * Green-Kubo integrals of them (Sec. 2.3 Eqs. (visc), (therm)).
 *
 * Conventions shared by every call:
 *  - Every function returns an int status: MD_OK (0) or a negative MD_E*
 *    code; md_last_error() then holds a message for the calling thread.  No
 *    C++ exception crosses this boundary.
 *  - Positions, velocities and forces are component-major arrays [3][n]
 *    (all x, then all y, then all z) in the caller's atom order.  Stress
 *    tensors and per-particle virials use the order xx, yy, zz, xy, xz, yz.
 *  - The library copies every input and keeps no caller pointer.  Handles
 *    are owned by the library and released with md_free / corr_free.
 *  - All GPU work is enqueued on the CUDA stream given at creation
 *    (a cudaStream_t passed as void*, NULL for the legacy default stream).
 *    Calls that hand results to the host synchronise that stream.
 *  - Units are the caller's; the tests use LJ reduced units
 *    (eps = sigma = m = kB = 1).
 */
#ifndef OTF_MD_H
#define OTF_MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exported from libotfmd.so (the library is built with hidden visibility). */
#if defined(__GNUC__)
#define OTF_API __attribute__((visibility("default")))
#else
#define OTF_API
#endif

/* Status codes. */
#define MD_OK 0
#define MD_EINVAL (-1)   /* invalid argument or parameter */
#define MD_ENOMEM (-2)   /* device or host allocation failed */
#define MD_ECUDA (-3)    /* a CUDA runtime call failed */
#define MD_ESTATE (-4)   /* the system left its valid state: non-finite
                            coordinates, a neighbour list or cell over its
                            capacity, fewer than 3 cells per side */
#define MD_ETIMEOUT (-5) /* a bounded device wait gave up */
#define MD_ECAP (-6)     /* output buffer too small; *n holds the size needed */

/* Arithmetic of the MD path. */
#define MD_PREC_FP64 0   /* every step in FP64 */
#define MD_PREC_MIXED 1  /* FP32 forces, per-particle fluxes and correlator
                            products; FP64 positions, velocities, global
                            reductions and correlator lag sums */

/* Where caller arrays live. */
#define MD_MEM_HOST 0
#define MD_MEM_DEVICE 1

/* Correlators owned by an MD system (md_corr). */
#define MD_CORR_STRESS 0   /* 3 series: sigma_xy, sigma_xz, sigma_yz */
#define MD_CORR_HEATFLUX 1 /* 3 series: q_x, q_y, q_z */
#define MD_CORR_VACF 2     /* 3n series: v_x of every atom, then v_y, then v_z;
                              read out per component, averaged over atoms */
#define MD_CORR_MASSFLUX 3 /* cross correlator, 6 series per replica:
                              <q_a(0) j_a(t)> for a = x, y, z, then
                              <j_a(0) j_a(t)>, with j the partial momentum
                              density of one species (Sec. 2.3, multi-component
                              kappa).  For a binary system (total momentum
                              zero) the mass-flux corrected conductivity is
                              V/T^2 [I_qq - I_qj^2 / I_jj], I the time
                              integrals of the component means of the heat-flux,
                              cross and partial momentum correlations. */

/* Interaction (md_params.potential). */
#define MD_POT_LJ 0          /* Lennard-Jones (eps, sigma), optionally energy-shifted */
#define MD_POT_BUCK_EWALD 1  /* Buckingham A exp(-r/rho) - C/r^6 between every pair
                                plus Coulomb by Ewald: real-space erfc term
                                within rc, smooth particle-mesh Ewald in
                                reciprocal space (single systems only) */

/* Pair evaluation. */
#define MD_PAIR_VERLET 0 /* Verlet neighbour lists built from link cells,
                            rebuilt when an atom has moved skin/2 */
#define MD_PAIR_CELLS 1  /* direct link-cell evaluation every step */
#define MD_PAIR_TILES 2  /* mixed-precision Lennard-Jones only: Verlet lists
                            (same skin rule) over tiles of at most 3 x 2 x 2
                            cells; each tile's CTA stages the tile and its
                            one-cell shell in shared memory, in the tile's own
                            frame, and the lists hold 16-bit offsets into that
                            window.  md_init returns MD_EINVAL when the
                            expected window exceeds the shared-memory capacity
                            (4,095 atoms); a window that outgrows it during a
                            run stops md_step with MD_ESTATE. */

/* Multiple-tau parameters of one correlator (Sec. 2.2: b blocks of p points
 * with block averages of m samples; u = update interval in MD steps).
 * p must be a multiple of m, 2 <= p <= 64, 1 <= b <= 32, m >= 1.  u = 0
 * disables the correlator. */
typedef struct {
  int32_t b, p, m, u;
} corr_spec;

typedef struct {
  int64_t n;          /* atoms, 2 .. 2^26 - 1 (over all replicas of a batch too) */
  double box;         /* edge of the periodic cubic box */
  double eps, sigma;  /* Lennard-Jones parameters */
  double rc;          /* cutoff radius; box >= 3 (rc + skin) */
  int32_t shift;      /* 1: energy-shifted potential (U(rc) subtracted) */
  int32_t ntypes;     /* 1..8 atom types (mass only) */
  double mass[8];     /* mass of each type */
  double dt;          /* time step */
  int32_t precision;  /* MD_PREC_FP64 or MD_PREC_MIXED */
  int32_t pair_mode;  /* MD_PAIR_VERLET or MD_PAIR_CELLS */
  double skin;        /* Verlet skin (MD_PAIR_VERLET); 0 rebuilds every step */
  int32_t max_neighbors; /* neighbour-list capacity per atom; 0 = automatic */
  int32_t use_graph;  /* 1: md_step replays CUDA graphs (8 steps at a time, each step's
                         correlator pushes on a second stream beside the next step; one graph
                         of 1..7 steps for the rest of a call), each captured the first time a
                         call needs it; 0: direct launches */
  int32_t autotune;   /* 1: md_init times launch shapes on the system itself and
                         keeps the fastest (md_get_config).  MD_PAIR_VERLET:
                         the pair kernel at 64/128/256 threads per CTA and the
                         list build (j-parallel at 2/4/8, i-parallel and staged
                         at 4/8 warps per CTA).  MD_PAIR_TILES: the cell tiles
                         (at most 3x2x2, 2x2x2 or 3x3x2 cells, those whose
                         windows fit) at 1.0/1.1/1.3 times the mean tile in
                         threads per CTA, scored as one pair launch plus an
                         eighth of a list build.  Tilings round coordinates in
                         different frames, so results can differ from the
                         untuned handle at FP32 rounding level. */
  corr_spec stress, heatflux, vacf; /* the three correlators of Sec. 2.3/2.7 */
  int32_t list_build; /* neighbour-list build when not autotuned: 0 = the
                         library's default, 1 = j-parallel, 2 = i-parallel,
                         3 = staged (all give the same lists in the same
                         order) */
  int32_t potential;  /* MD_POT_LJ or MD_POT_BUCK_EWALD */
  double charge[8];   /* MD_POT_BUCK_EWALD: charge of each type */
  double buck_A, buck_rho, buck_C; /* MD_POT_BUCK_EWALD: Buckingham parameters
                         (one set for every pair of types; no energy shift) */
  double coulomb;     /* MD_POT_BUCK_EWALD: ke = 1/(4 pi eps0) in the caller's
                         units (14.399645 eV Angstrom / e^2 for eV, Angstrom, e) */
  double ewald_alpha; /* MD_POT_BUCK_EWALD: Ewald splitting parameter */
  int32_t mesh;       /* MD_POT_BUCK_EWALD: SPME mesh points per side (even,
                         >= order) */
  int32_t order;      /* MD_POT_BUCK_EWALD: B-spline order: 4, 6 or 8 */
  int32_t flux_species; /* atom type whose partial momentum density j is
                         observed and correlated with q (MD_CORR_MASSFLUX) */
  corr_spec massflux; /* MD_CORR_MASSFLUX settings (u = 0: off) */
  int32_t window_slots; /* MD_PAIR_TILES: shared-memory window capacity per tile in
                           atoms + 1 (0 = automatic: the largest window expected at
                           1.2 times the mean density, or one atom per sigma^3, plus
                           64); at most 4,096.  A window that needs more stops
                           md_init or md_step with MD_ESTATE. */
} md_params;

typedef struct {
  const double *r;     /* [3][n] positions (wrapped into the box by md_init) */
  const double *v;     /* [3][n] velocities */
  const int32_t *type; /* [n] type of each atom, or NULL for all type 0 */
  int32_t mem;         /* MD_MEM_HOST or MD_MEM_DEVICE for the three arrays */
} md_system;

/* One replica of a batch (md_init_replicas): its own atoms, box, positions
 * [3][n], velocities [3][n] and types (NULL: all type 0). */
typedef struct {
  int64_t n;
  double box;
  const double *r;
  const double *v;
  const int32_t *type;
} md_replica;

/* Launch shapes and sizes chosen for a system (md_get_config). */
typedef struct {
  int32_t replicas;
  int32_t pair_threads;   /* threads per CTA of the pair kernel */
  int32_t build_warps;    /* warps per CTA of the neighbour-list build */
  int32_t max_neighbors;  /* neighbour-list capacity per atom */
  int64_t atoms, cells;   /* totals over all replicas */
  int32_t build_kind;     /* 0: j-parallel list build, 1: i-parallel, 2: staged,
                             3: tile windows (MD_PAIR_TILES) */
  int64_t vacf_input_bytes; /* device bytes of the per-atom velocity correlator's
                               input slots (0 when that correlator is off) */
  int64_t tiles;            /* MD_PAIR_TILES: tiles (CTAs of the pair kernel); else 0 */
  int32_t window_capacity;  /* MD_PAIR_TILES: shared-memory window slots per tile */
  int32_t tile_threads;     /* MD_PAIR_TILES: threads per tile CTA */
  int32_t tile_extent[3];   /* MD_PAIR_TILES: largest tile extent in cells along x, y, z
                               (3 2 2 unless the autotuner picked another tiling) */
} md_config;

/* Observables of the last completed step (Sec. 2.3). */
typedef struct {
  int64_t step;        /* steps completed since md_init */
  double U, K, T;      /* potential and kinetic energy, T = 2K/(3n-3) */
  double sigma[6];     /* pressure tensor: (sum m v v + sum_i W_i) / V */
  double q[3];         /* heat flux: sum_i (E_i v_i + W_i v_i) / V */
  double T_mean;       /* mean of T over the steps since md_init */
  int64_t rebuilds;    /* cell sorts / neighbour-list builds since md_init */
  double j[3];         /* partial momentum density of the flux species:
                          sum over its atoms of m v / V */
} md_obs;

typedef struct md_handle_s md_handle;
typedef struct corr_handle_s corr_handle;

/* Creates a system: copies r, v, type, builds the cell-sorted layout,
 * evaluates forces, per-particle energies and virials at t = 0 and the
 * observables (no correlator sample is taken at t = 0).  Link cells of edge
 * >= rc + skin (Sec. 1 "linked cells").  Errors: MD_EINVAL for bad
 * parameters (including fewer than 3 cells per side), MD_ENOMEM, MD_ECUDA,
 * MD_ESTATE for non-finite input. */
OTF_API int md_init(const md_params *p, const md_system *s, void *cuda_stream, md_handle **out);

/* A batch of independent replicas (sizes, densities and temperatures may
 * differ; the LJ parameters, time step, precision and correlator settings of
 * p are shared; p->n and p->box are ignored).  Their atoms, cells and
 * reduction CTAs are laid end to end, so every kernel of a step covers all
 * replicas and one captured graph launch advances the whole batch.  Every
 * replica needs at least 256 atoms and 3 cells per side; the per-atom
 * velocity correlator must be off (vacf.u = 0).  The stress and heat-flux
 * correlators then hold 3 series per replica (replica r: series 3r..3r+2,
 * read with corr_read(group = 3r + k)).  mem says where all the replicas'
 * arrays live.  Otherwise as md_init; the other md_* calls apply to all
 * replicas (md_observables reports replica 0). */
OTF_API int md_init_replicas(const md_params *p, const md_replica *reps, int32_t count, int32_t mem,
                             void *cuda_stream, md_handle **out);

/* Advances nsteps velocity-Verlet NVE steps (Sec. 1).  Each step: half
 * kick and drift; neighbour-list rebuild when needed; pair forces with
 * per-particle energy and virial; half kick; reduction to U, K, sigma, q;
 * correlator samples of the stress and heat flux every stress.u /
 * heatflux.u steps and of every atom's velocity every vacf.u steps
 * (Algorithm 1; with vacf.p <= 16 the velocity samples wait in device slots
 * and are applied eight at a time; samples short of a full block stay there
 * across calls and are applied by the next readout of the velocity
 * correlator (corr_read, corr_raw, corr_read_rows), so a readout always
 * holds every step taken).
 * Everything stays on the device.  Synchronises the stream at the end and
 * returns MD_ESTATE if a device check failed (the state is then
 * undefined). */
OTF_API int md_step(md_handle *h, int64_t nsteps);

/* Observables of the last step (synchronises); replica 0 of a batch. */
OTF_API int md_observables(md_handle *h, md_obs *out);

/* Observables of replica r of a batch (synchronises). */
OTF_API int md_replica_observables(md_handle *h, int32_t r, md_obs *out);
/* The observables of every replica at once: out [count], count = the number
 * of replicas (MD_EINVAL otherwise).  One device read; synchronises. */
OTF_API int md_replica_observables_all(md_handle *h, md_obs *out, int32_t count);

/* Per-particle state in the caller's atom order: positions (wrapped into
 * [0, box)), velocities, forces, potential energies [n] and virials [6][n]
 * (W_i = 1/2 sum_j r_ij (x) f_ij).  Any pointer may be NULL.  mem says where
 * the outputs live.  Synchronises. */
OTF_API int md_get_particles(md_handle *h, double *r, double *v, double *F, double *epot,
                     double *W, int32_t mem);

/* Multiplies every velocity by lambda (velocity-rescaling equilibration;
 * not part of the correlated run) and refreshes the observables. */
OTF_API int md_scale_velocities(md_handle *h, double lambda);

/* Per-replica velocity rescaling: replica r's velocities times lambda[r]
 * (host array of one factor per replica). */
OTF_API int md_replica_scale_velocities(md_handle *h, const double *lambda);

/* Replica count, total atoms and cells, list capacity and the launch shapes
 * in use (after autotuning when md_params.autotune was set). */
OTF_API int md_get_config(md_handle *h, md_config *out);

/* Clears the correlators and the running temperature mean of a system, so
 * that a production run can start after equilibration. */
OTF_API int md_reset_correlators(md_handle *h);

/* Borrowed view of a correlator of the system (MD_CORR_*); valid until
 * md_free; do not pass it to corr_free or corr_push. */
OTF_API int md_corr(md_handle *h, int32_t which, corr_handle **out);

/* Kernel classes timed by md_set_timing / md_kernel_times. */
#define MD_K_INTEGRATE 0 /* half kick + drift + skin check */
#define MD_K_REBUILD 1   /* cell counting sort + neighbour-list build */
#define MD_K_PAIR 2      /* pair forces, per-particle energy and virial */
#define MD_K_REDUCE 3    /* half kick + stress / heat-flux reduction + their
                            correlator samples */
#define MD_K_VACF 4      /* per-atom velocity correlator sample */
#define MD_K_SPME 5      /* reciprocal-space Ewald (MD_POT_BUCK_EWALD) */
#define MD_NKCLASS 6

/* on = 1: the following md_step calls bracket every kernel class with CUDA
 * events and add its device time to counters; on = 0 stops that.  Enabling
 * clears the counters.  With graphs on (md_params.use_graph), enabling
 * captures graphs that carry the event records (8 steps, and 1..7 steps for
 * a call's remainder), so the times are those of the normal launch path
 * (the correlator pushes then overlap the next step's kernels, and their
 * times include that sharing of the GPU); without graphs every step launches
 * directly between events. */
OTF_API int md_set_timing(md_handle *h, int32_t on);

/* Accumulated device milliseconds [MD_NKCLASS] and launches [MD_NKCLASS]
 * per kernel class since timing was enabled (host arrays). */
OTF_API int md_kernel_times(md_handle *h, double *ms, int64_t *launches);

OTF_API void md_free(md_handle *h);

/* A free-standing correlator over nseries series pushed in lockstep
 * (Sec. 2.2 "any pair of observables can be correlated").  Series are split
 * into contiguous groups of group_size; a group's readout is the mean of its
 * series' correlations.  cross = 0: autocorrelation of x; cross = 1: x
 * with y.  precision: MD_PREC_FP64 (FP64 ring and products) or
 * MD_PREC_MIXED (FP32 ring and products, FP64 lag sums).  dt_unit: time
 * between two pushes (readout times are lag * m^(k-1) * dt_unit). */
typedef struct {
  int32_t b, p, m;
  int32_t cross;
  int64_t nseries;
  int64_t group_size;
  int32_t precision;
  double dt_unit;
} corr_params;

OTF_API int corr_create(const corr_params *cp, void *cuda_stream, corr_handle **out);

/* One sample per series (Algorithm 1 applied to every series): x [nseries]
 * and, for cross correlators, y [nseries]; FP64, in host or device memory
 * (mem).  Host input is copied before the call returns. */
OTF_API int corr_push(corr_handle *c, const double *x, const double *y, int64_t nseries, int32_t mem);

/* Readout of group g (Algorithm 2), or of the mean over all groups when
 * g = -1: writes up to cap (time, value) points to host arrays and the
 * number of points to *n; MD_ECAP (with *n set) when cap is too small.
 * Synchronises. */
OTF_API int corr_read(corr_handle *c, int64_t g, double *times, double *values, int64_t cap, int64_t *n);

/* Raw lag sums [ngroups][b][p] (sums over each group's series), product
 * counts per series [b][p] and the number of blocks used (host arrays). */
OTF_API int corr_raw(corr_handle *c, double *values, int64_t *count, int32_t *blocks_used);

/* Number of samples pushed so far. */
OTF_API int corr_pushes(corr_handle *c, int64_t *n);

OTF_API int corr_reset(corr_handle *c);
OTF_API void corr_free(corr_handle *c);

/* Green-Kubo integral (Sec. 2.3 Eqs. (visc), (therm)): prefactor times the
 * integral of the piecewise-linear interpolant of (t[i], c[i]) from t[0] to
 * min(t_cut, t[n-1]) (trapezoid rule).  running (nullable, [n]) receives
 * prefactor times the integral from t[0] to t[i].  Host arrays; t must be
 * strictly increasing.  Viscosity: prefactor V / (kB T); conductivity with
 * c = <q(t).q(0)>: V / (3 kB T^2). */
OTF_API int gk_integrate(const double *t, const double *c, int64_t n, double t_cut, double prefactor,
                 double *integral, double *running);

/* Allocation-free observables: the paper has no counterpart to this call.
 * It exists for host programs that cannot call cudaMalloc while they run,
 * such as engines that hand all device memory to their own fixed pool at
 * start-up, or pipelines that must not take the device-wide synchronisation
 * cudaMalloc / cudaFree may cause.  It computes, from caller device arrays
 * (FP64): obs[12] = U, K, T = 2K/(3n-3), sigma[6] (xx yy zz xy xz yz) and
 * q[3], with sigma = (sum_i m_i v_i v_i + sum_i W_i) / volume and
 * q = sum_i (E_i v_i + W_i v_i) / volume, E_i = m_i v_i^2 / 2 + epot_i;
 * v [3][n], epot [n], W [6][n], mass_of [n], obs [12] device output.  The
 * work is enqueued on cuda_stream and the call returns without waiting.
 * Its scratch is a fixed array inside the library (partial sums for 1024
 * CTAs, about 90 KB per GPU, held until the process exits); n may be up to
 * 2^27 - 1 and larger n is rejected with MD_EINVAL.  The first call on each
 * device looks up that array's address and clears its completion counter on
 * cuda_stream, ahead of its own launch, so make that first call before any
 * stream capture.  All calls on one device share the array: calls that
 * overlap on the GPU race. */
OTF_API int md_observables_noalloc(int64_t n, double volume, const double *v, const double *epot,
                                   const double *W, const double *mass_of, double *obs,
                                   void *cuda_stream);

/* Measurement utility (the paper has no counterpart): the FP32 FMA rate of
 * the current GPU, which sets the roofline of the pair kernel.  Launches a
 * grid that fills every SM (occupancy-limited CTAs of 256 threads), each
 * thread running 8 independent chains of dependent FMAs for iters x 16
 * steps: scalar fma.rn.f32 (paired = 0) or fma.rn.f32x2 on register pairs
 * (paired = 1, two FMAs per instruction).  One warm-up launch, then reps
 * launches timed with CUDA events on cuda_stream.  Outputs (host):
 * flops per launch (2 per FMA), device milliseconds per launch, and the SM
 * count.  Allocates and frees a small output buffer and synchronises the
 * stream.  Errors: MD_EINVAL for iters or reps < 1 or a null output,
 * MD_ECUDA for a failed CUDA call. */
OTF_API int md_fp32_peak(int32_t paired, int64_t iters, int32_t reps, void *cuda_stream,
                         double *flops_per_launch, double *ms_per_launch, int32_t *sm_count);

/* Message of the last failed call on this thread ("" if none). */
OTF_API const char *md_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OTF_MD_H */
