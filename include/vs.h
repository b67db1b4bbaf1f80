/*
 * vs.h -- C ABI of the GB300 vortex-field smoothing library (libvs.so).
 *
 * Method: Virgili, Kamleh & Leinweber, "Smoothing algorithms for projected
 * center-vortex gauge fields", arXiv:2203.09764.  The library smooths a
 * Z(3)-projected centre-vortex gauge field on one GPU:
 *   load (Sec. I, Eqs. centre_project / centre_element)
 *   -> centrifuge preconditioning (Sec. IV, Eqs. lambda_j / lambda_k)
 *   -> annealed stout smoothing with standard or over-improved staples
 *      (Sec. II.A Eqs. stout / generator, Sec. III Eq. over-improvement,
 *       Sec. V.B annealed Euler Wilson flow) and the vortex-preservation
 *      accept/reject test (Sec. VI)
 *   -> vortex check and Wilson action (Sec. I, Sec. V).
 *
 * Conventions shared by every call:
 *   dims[4] = {Lx, Ly, Lz, Lt}; every extent must be a positive multiple of 4
 *     (the annealed schedule colours links by (2 x_mu + sum_{nu != mu} x_nu) mod 4).
 *   Host link arrays: double [4][V][3][3][2] (direction major, then the
 *     lexicographic site s = x + Lx*(y + Ly*(z + Lz*t)), then the row-major
 *     3x3 matrix as (re, im) pairs).  Host label arrays: int8_t [4][V] in
 *     {-1, 0, +1}, same ordering.
 *   `where` selects whether a caller pointer is host memory (VS_HOST) or CUDA
 *     device memory (VS_DEVICE) of the field's device.
 *   The caller keeps ownership of every buffer it passes in; the library
 *     copies what it needs before the call returns (host) or before work on
 *     the field's stream that follows the call (device).
 *   A field holds no data until vs_load_field, vs_load_cooled or
 *     vs_field_restore: every other call that reads or updates its links or
 *     labels returns EINVAL before that.
 *   Every call returns a vs_status; on failure vs_last_error() describes it.
 *     No C++ exception crosses this boundary.  Calls on one vs_field are not
 *     thread safe; distinct fields may be used from distinct threads.
 */
#ifndef VS_H
#define VS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vs_status;
enum {
    VS_OK = 0,
    VS_EINVAL = 1,       /* bad argument; nothing was launched */
    VS_ENOMEM = 2,       /* device or host allocation failed */
    VS_EBUSY = 3,        /* serving queue is full */
    VS_EAGAIN = 4,       /* result not ready (poll with timeout 0) */
    VS_ETIMEDOUT = 5,    /* poll timed out */
    VS_EDEVICE = 6,      /* CUDA error or device error word set */
    VS_EUNSUPPORTED = 7, /* combination not built */
    VS_ENOTFOUND = 8,    /* unknown ticket */
    VS_ECANCELED = 9     /* job was cancelled (vs_result.status) */
};

enum { VS_FP64 = 0, VS_FP32 = 1 };            /* arithmetic and storage precision */
enum { VS_LINK18 = 0, VS_LINK12 = 1 };        /* 18 reals, or rows 1-2 with row 3 rebuilt */
enum { VS_ANNEALED = 0, VS_SIMULTANEOUS = 1 };
enum { VS_HOST = 0, VS_DEVICE = 1 };

typedef struct vs_ctx vs_ctx;
typedef struct vs_field vs_field;

/* Device allocator hooks: return a device pointer of at least `bytes` bytes
 * (aligned to 256 bytes) or NULL; free_fn releases it. */
typedef void *(*vs_alloc_fn)(size_t bytes, void *user);
typedef void (*vs_free_fn)(void *ptr, void *user);

typedef struct {
    int32_t device;             /* CUDA device ordinal */
    vs_alloc_fn alloc;          /* NULL: cudaMalloc */
    vs_free_fn free_fn;         /* NULL: cudaFree */
    void *alloc_user;
    uint64_t hbm_budget_bytes;  /* serving admission cap on device bytes; 0 = no cap */
    int32_t max_slots;          /* serving: jobs on the device at once; 0 -> 8 */
    int32_t max_queue;          /* serving: waiting jobs before VS_EBUSY; 0 -> 1024 */
} vs_options;

/* Thread-local description of the last failure on this thread. */
const char *vs_last_error(void);

/* Library version and the device code architecture it was built for. */
const char *vs_version(void);

vs_status vs_create(const vs_options *opt, vs_ctx **out);
void vs_destroy(vs_ctx *ctx);

/* Allocate a field (links + resident reference labels) on the context's
 * device.  stream: a cudaStream_t to run on, or NULL for a library-owned
 * stream.  EINVAL: an extent not a positive multiple of 4, more than 2^30
 * plane positions (sites, plus the layout's unused positions when Lx/4 is 5,
 * 6 or 7; see vs_field_describe), or an unknown precision/storage;
 * EUNSUPPORTED: FP64 with 12-real storage. */
vs_status vs_field_create(vs_ctx *ctx, const int32_t dims[4], int32_t precision,
                          int32_t storage, void *stream, vs_field **out);
/* Device memory of a field: the links (4 V x 18 or 12 reals), two label planes
 * (8 V bytes) and a few KB of counters, allocated here.  One staging buffer is
 * allocated on first need, grown to the largest need and kept until
 * vs_field_destroy: host transfers of links or a gauge field (288 V or 144 V
 * bytes), of labels (4 V) and of per-site observables (24 V), and the second
 * field buffer of the simultaneous schedules and the RK3 stages (one field's
 * links).  Device-side transfers (`where` = VS_DEVICE) need no staging. */
void vs_field_destroy(vs_field *f);

/* Load, Sec. I Eqs. (centre_project)/(centre_element): exactly one of
 * links / labels is non-NULL.  With links, the reference labels n_mu(x) are the
 * Z(3) sectors of arg Tr U of the given links; with labels, every link becomes
 * exp(2 pi i n/3) I.  The labels stay resident as the vortex-preservation
 * reference until the next load.  EINVAL: both or neither input, a label
 * outside {-1,0,1} (device input is not scanned). */
vs_status vs_load_field(vs_field *f, const double *links, const int8_t *labels, int32_t where);

/* Hot start from a seed: every link an independent Haar SU(3) matrix, then
 * n_cool sweeps of annealed MaxReTr cooling (Sec. III, alpha = 1, plaquette
 * staples, three passes over the SU(2) subgroups), then projection of every
 * link to its Z(3) element, which also becomes the reference labels.  This is
 * the synthetic stand-in for a gauge-fixed Monte-Carlo ensemble member. */
vs_status vs_load_cooled(vs_field *f, uint64_t seed, int32_t n_cool);

/* Centrifuge preconditioning, Sec. IV: every link at once from the original
 * labels; staple phase sigma = m 2pi/18 with integer m, a random pair (j,k)
 * per link from SplitMix64 value (mu*V + s) of `seed` mod 3 selecting
 * (1,2),(2,3),(3,1); lambda^j = lambda + delta, lambda^k = lambda - delta,
 * delta = omega (sigma - lambda).  EINVAL unless 0 <= omega < 1/4 (the bound
 * that keeps every label, Sec. IV.A), or if the field is in a random gauge
 * (vs_gauge_transform comes after the centrifuge). */
vs_status vs_centrifuge(vs_field *f, double omega, uint64_t seed);

typedef struct {
    int32_t kind;                 /* VS_ANNEALED or VS_SIMULTANEOUS */
    const double *rho_per_sweep;  /* host [n_sweeps] step sizes, or NULL for constant rho */
    int32_t reunit_every;         /* FP32: re-unitarise (Gram-Schmidt in FP32) every k sweeps; 0 = never */
    int32_t action_every;         /* record <S> in stats every k sweeps; 0 = never */
    int32_t fp64_redecide;        /* FP32 with vortex preservation: a candidate whose FP32 trace lies within
                                     the FP32 band of a sector edge (n_undecidable below) is left unwritten
                                     by its class launch and decided again in FP64 from the same stored
                                     links before the next class (1), or decided in FP32 (0, the default
                                     when sched is NULL).  The FP64 pass sits between dependent class
                                     launches on GB300's FP64 pipe (~60 us per candidate): with ~80 such
                                     candidates per sweep at 32^3x64 a sweep takes 2.8x as long.  A
                                     candidate accepted in FP64 whose FP32-rounded link would carry
                                     another label keeps the old link. */
} vs_anneal;

typedef struct {
    int64_t n_accept;             /* candidates written */
    int64_t n_reject;             /* candidates refused by the vortex-preservation test */
    int64_t n_fp64_exp;           /* FP32 mode: exponentials redone in FP64 (|rho Q| large) */
    double action;                /* <S>/beta after the sweep, when recorded */
    int32_t has_action;
    int32_t n_singular;           /* vs_smooth_ape: blocked matrices with no projection (link kept) */
    /* Vortex-preservation diagnostics (Sec. VI; the n_diff counts of the
     * paper's tables) of vs_smooth, vs_smooth_aus and vs_smooth_ape; -1 / NaN
     * from vs_flow_rk3: */
    int64_t n_label_diff;         /* candidates whose Z(3) label (Sec. I) differs from the reference label;
                                     with vortex preservation these are the rejections, without it the
                                     label differences after the sweep */
    int64_t n_undecidable;        /* candidates whose trace lies within the rounding band of a sector
                                     edge (in trace units: FP32 arithmetic 2e-6, FP32 candidates decided
                                     again in FP64 1e-6, FP64 1e-12), where another rounding could
                                     decide the test differently; outside it the decision equals that
                                     of exact arithmetic on the stored links (FP32 arithmetic: on the
                                     stored links up to that band) */
    double min_margin;            /* smallest angular distance of a candidate's arg Tr from a sector edge
                                     (radians) */
    int64_t n_fp64_redecided;     /* FP32 candidates decided in FP64 (vs_anneal.fp64_redecide); their
                                     undecidable band is then that of the FP32 storage of the links
                                     (1e-6), not of FP32 arithmetic */
} vs_sweep_stats;

/* n_sweeps of stout smoothing, Eqs. (stout)/(generator), with
 * Sigma = c0 (plaquette staples) + c1 (rectangles), c0 = (5 - 2 eps)/3,
 * c1 = (eps - 1)/(12 u0^2) (Eq. over-improvement; eps = 1 is standard).
 * Annealed: for mu = 0..3, for colour c = 0..3, all links of that class at
 * once, in place (Sec. III.A masked updates; Sec. V.B: Euler Wilson flow with
 * step rho).  Simultaneous: every link from the previous sweep's field.
 * vortex_preserve != 0: a candidate is written only if its Z(3) label equals
 * the original reference label (Sec. VI).  sched may be NULL (annealed,
 * constant rho, re-unitarise every 10 sweeps in FP32, no action).  stats:
 * NULL, or [n_sweeps] filled before return (the call then waits for the
 * device).  Without stats the call only enqueues.  EINVAL: n_sweeps < 0,
 * non-finite rho/eps, u0 <= 0.  EDEVICE: CUDA error or device error word. */
vs_status vs_smooth(vs_field *f, int32_t n_sweeps, double rho, double epsilon, double u0,
                    const vs_anneal *sched, int32_t vortex_preserve, vs_sweep_stats *stats);

/* n_sweeps of annealed U-link smearing with MaxReTr reunitarisation (AUS,
 * Sec. III Eqs. V and maxReTr; Sec. III.A; the smoother of the paper's CP
 * and VP recipes): for mu = 0..3, colour 0..3, every link of the class at
 * once, V = (1 - alpha) U + (alpha / 6) Sigma(eps, u0) with the staples of
 * Eq. over-improvement, then n_hits passes over the SU(2) subgroups (1,2),
 * (2,3), (1,3) maximise Re Tr(U V^dag) starting from U (a subgroup with
 * k = sqrt(det T) = 0 is skipped).  vortex_preserve: Sec. VI test against the
 * original labels.  FP32: re-unitarise every reunit_every sweeps (0 = never).
 * alpha = 1 with eps = 1 is cooling.  stats as for vs_smooth (no action).
 * EINVAL: alpha outside [0, 1], n_hits < 1, non-finite eps, u0 <= 0. */
vs_status vs_smooth_aus(vs_field *f, int32_t n_sweeps, double alpha, double epsilon, double u0,
                        int32_t n_hits, int32_t reunit_every, int32_t vortex_preserve,
                        vs_sweep_stats *stats);

/* n_sweeps of APE blocking with unit circle projection (Sec. II.C, Eqs. V, W
 * and P_ucp): V = (1 - alpha) U + (alpha / 6) Sigma(eps, u0) with the staples
 * of Eq. over-improvement, U <- W / cbrt(det W), W = V (V^dag V)^{-1/2}, the
 * principal cube root (arg det W in (-pi, pi]).  schedule VS_SIMULTANEOUS
 * is APE smearing (every link from the previous sweep's field);
 * VS_ANNEALED is annealed U-link smearing with UCP (AUS+UCP, Sec. VII.A), in
 * the colour order of vs_smooth.  A blocked matrix with
 * det(V^dag V) <= 1e-24 (Tr(V^dag V)/3)^3 has no projection: the link is kept
 * and counted in stats[].n_singular.  vortex_preserve: Sec. VI test against
 * the original labels.  FP32: re-unitarise every reunit_every sweeps (0 =
 * never).  stats as for vs_smooth (no action).  EINVAL: alpha outside
 * [0, 1], bad schedule, non-finite eps, u0 <= 0. */
vs_status vs_smooth_ape(vs_field *f, int32_t n_sweeps, double alpha, double epsilon, double u0,
                        int32_t schedule, int32_t reunit_every, int32_t vortex_preserve,
                        vs_sweep_stats *stats);

/* n_steps of the Wilson flow dU/dtau = Q[U] U (Sec. V.B; Q of Eq. generator
 * with the staples Sigma(eps, u0), eps = 1: the Wilson flow) by the
 * third-order Runge-Kutta scheme of Luscher (JHEP 08 (2010) 071), step size
 * `step`: with Z_i = step Q[W_i] on every link,
 *   W_1 = exp(Z_0/4) W_0, W_2 = exp(8 Z_1/9 - 17 Z_0/36) W_1,
 *   U(tau + step) = exp(3 Z_2/4 - 8 Z_1/9 + 17 Z_0/36) W_2,
 * each stage from the whole field of the previous one.  Allocates a
 * 4 x 9 x V exponent buffer (field precision) on first use, kept with the
 * field.  No vortex preservation (the flow of a centre-vortex field is
 * trivial, Sec. V.B).  FP32: re-unitarise every reunit_every steps.  stats:
 * NULL or [n_steps] (n_fp64_exp per step).  EINVAL: step < 0 or non-finite,
 * non-finite eps, u0 <= 0. */
vs_status vs_flow_rk3(vs_field *f, int32_t n_steps, double step, double epsilon, double u0,
                      int32_t reunit_every, vs_sweep_stats *stats);

/* One colour class (mu, colour) of the annealed schedule, as vs_smooth runs it. */
vs_status vs_subsweep(vs_field *f, int32_t mu, int32_t colour, double rho, double epsilon,
                      double u0, int32_t vortex_preserve);

typedef struct {
    int64_t n_links;
    int64_t n_label_diff;         /* links whose current Z(3) label != reference */
    int64_t n_charge_diff;        /* plaquettes whose centre charge != reference (Sec. I) */
    int64_t n_near_boundary;      /* links with arg Tr U within 1e-5 rad of a sector edge */
    double min_margin;            /* smallest angular distance of arg Tr U from a sector edge */
} vs_vortex_report;

typedef struct {
    double mean_S;                /* <S>/beta, the Wilson action density (Sec. V) */
    double mean_SR;               /* <S_R>/beta, the reconstructed action from clover F */
    double Q;                     /* total topological charge sum_x q(x) */
} vs_observables_out;

/* Smoothness observables, Sec. V: clover field strength F_munu(x) (mean of the
 * four plaquette leaves at x, F = (C - C^dag)/(2i), traceless, lattice units
 * -- the coupling of Eq. 1LFST absorbed), the one-loop topological charge
 * density q(x) = eps_{mu nu rho sigma} Tr(F_munu F_rhosigma)/(32 pi^2)
 * (Eq. 1LTopQ), and the reconstructed action S_R(x)/beta = 1/72
 * sum_{mu != nu} Tr(F_munu^2)/2, normalised so that S_R/S -> 1 on smooth
 * fields (the paper's smoothness condition <S> ~ <S_R>; its printed
 * normalisation is garbled).  Optional per-site densities S(x)/beta,
 * S_R(x)/beta, q(x): double [V] in lexicographic order, host or device per
 * `where`.  Products in the field precision, sums in FP64.  Synchronous. */
vs_status vs_observables(vs_field *f, vs_observables_out *out, double *S_site, double *SR_site,
                         double *q_site, int32_t where);

/* Correlation of two per-site densities, Sec. VII Eq. (correlation_s) and the
 * C^q equation after it:
 *   C_XY = <a(x) b(x)> / (sqrt<a(x)^2> sqrt<b(x)^2>),
 * <.> the mean over the field's V sites (the paper's form: not
 * mean-subtracted).  a, b: double [V] (any site order, the same for both; e.g.
 * the lexicographic densities of vs_observables of two smoothed fields of
 * this field's dims), host or device per `where`; the field supplies the
 * lattice size, the stream and (for host input) its staging buffer.  Sums in
 * FP64 in a fixed order.  Synchronous.  EINVAL: NULL arguments, bad `where`,
 * a density that is zero on every site. */
vs_status vs_correlation(vs_field *f, const double *a, const double *b, int32_t where, double *C);

/* Vortex-structure check of the current field against the reference. Synchronous. */
vs_status vs_vortex_check(vs_field *f, vs_vortex_report *out);

/* Vortex check that allocates no device memory.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory at the point where they need the check -- code running while a CUDA
 * graph is being captured on another stream of the thread (the global
 * capture mode forbids allocating and synchronising calls), a serving loop
 * under a hard memory cap that must not call into cudaMalloc (which can block
 * on the whole device or fail under pressure), or a host that hands the
 * library preallocated buffers and forbids any other allocation.  It runs the
 * same kernels as vs_vortex_check on buffers the caller owns: links and
 * ref_labels are device pointers in the layout of a field with these dims,
 * precision and storage, and gauge is the field's random gauge transformation
 * G (Sec. V.D; the test then runs in the original gauge, on G^dag(x) U
 * G(x+mu), as vs_vortex_check does) or NULL for a field in its original gauge
 * -- vs_field_describe gives all three.  The result goes to the caller's host
 * struct.  Its scratch (one byte per link plus eight counters) is a fixed
 * array of VS_NOALLOC_MAX_LINKS bytes compiled into the library, which every
 * GPU that loads the library keeps until the process exits.  EINVAL for
 * lattices with more than VS_NOALLOC_MAX_LINKS links (2,097,152 sites, e.g.
 * 32^3 x 64).  Runs on the calling thread's current device, which must own
 * the buffers.
 *
 * Once per device the library looks up the scratch there, loads the check's
 * kernels and pins a 64-byte mapped host block (its only allocation, and on
 * the host): vs_create does this for its device, vs_noalloc_prepare for any
 * device, and otherwise the first call on a device does it (with the
 * thread's capture mode relaxed for those calls, so a first call made while
 * another stream captures neither fails nor invalidates the capture).  The
 * call waits for its own work without a synchronising CUDA call: its last
 * kernel writes the report and a sequence number to the mapped block, which
 * the host watches.  Calls on one device are serialised on the host and
 * share the scratch; one call's kernels finish before the next call on that
 * device launches any, except after a call that gave up waiting (EDEVICE
 * after 30 s without a result): its kernels may still be running, so later
 * calls on that device return EBUSY until its result has been published.
 * `stream`: where the kernels run; while another stream captures, give a
 * non-blocking stream (work on the legacy default stream, NULL, synchronises
 * with the blocking streams, which a capture forbids). */
#define VS_NOALLOC_MAX_LINKS (8 * 1024 * 1024)
vs_status vs_vortex_check_noalloc(const void *links, const int8_t *ref_labels, const void *gauge,
                                  const int32_t dims[4], int32_t precision, int32_t storage, void *stream,
                                  vs_vortex_report *out);

/* The once-per-device set-up of vs_vortex_check_noalloc, for a device on which
 * no vs_create ran: afterwards its calls there allocate nothing at all. */
vs_status vs_noalloc_prepare(int32_t device);

/* Mean Wilson action density <S>/beta, Sec. V: (1/V) sum_x 1/72 sum_{mu != nu}
 * Re Tr(1 - P_munu(x)); products in the field precision, sums in FP64 with a
 * fixed reduction order.  Synchronous. */
vs_status vs_action(vs_field *f, double *mean_S);

/* Copy out the current links (FP64, host layout above) or labels. */
vs_status vs_read_field(vs_field *f, double *links_out, int32_t where);
vs_status vs_read_labels(vs_field *f, int8_t *labels_out, int32_t where);     /* reference */

/* Number of links with a NaN or Inf entry (a guard for diverging or singular
 * updates; 0 for every workload).  Synchronous. */
vs_status vs_field_count_nonfinite(vs_field *f, int64_t *n_links);

/* Checkpoint and resume (not in the paper).  vs_field_checkpoint writes the
 * links (FP64 [4][V][3][3] complex, as vs_read_field), the reference labels
 * (int8 [4][V], as vs_read_labels) and the number of sweeps since the last
 * load (it sets the phase of the periodic re-unitarisation) to caller-owned
 * buffers on the host or the device (`where`); synchronous for the host.
 * vs_field_restore loads them into a field of the same dims, precision and
 * storage.  The kernels are deterministic, so N + M sweeps equal N sweeps,
 * checkpoint, restore into any field, then M sweeps, bit for bit (FP32 links
 * are exact in FP64; 12-real storage rebuilds row 2 the same way).
 * EINVAL: NULL buffers, a field not loaded, sweeps_done < 0, host labels
 * outside {-1, 0, 1}; EUNSUPPORTED: a field in a random gauge (checkpoint
 * before vs_gauge_transform). */
vs_status vs_field_checkpoint(vs_field *f, double *links_out, int8_t *labels_out, int64_t *sweeps_done,
                              int32_t where);
vs_status vs_field_restore(vs_field *f, const double *links, const int8_t *labels, int64_t sweeps_done,
                           int32_t where);
vs_status vs_current_labels(vs_field *f, int8_t *labels_out, int32_t where);  /* of current links */

/* Random gauge transformation (Sec. V.D): U_mu(x) -> G(x) U_mu(x) G^dag(x+mu)
 * for every link, with G: double [V][3][3][2] (lexicographic sites, SU(3)
 * matrices; host or device per `where`).  The field keeps G: from then on the
 * vortex-preservation test, the re-unitarisation guard and vs_vortex_check use
 * the label of G^dag(x) U G(x+mu) against the original labels (Sec. VI, the
 * test in the original gauge).  Reloading the field drops G.  EINVAL if the
 * field is already transformed. */
vs_status vs_gauge_transform(vs_field *f, const double *G, int32_t where);

/* Re-unitarise every link now: Gram-Schmidt of rows 1-2 in the field's precision, row 3 =
 * conj(r1 x r2); no label test (the periodic pass inside the smoothers keeps a link whose
 * label would change). */
vs_status vs_reunitarise(vs_field *f);

/* Wait for all work queued on the field's stream; EDEVICE on a device error. */
vs_status vs_synchronize(vs_field *f);

/* Device-time profile of the subsweep launches made by vs_smooth while
 * profiling is on: total milliseconds of the colour-class update chains (CUDA
 * events around each sweep's chain on the field's stream) and the number of
 * class-update launches they contain. */
vs_status vs_set_profiling(vs_field *f, int32_t on);
vs_status vs_get_profile(vs_field *f, double *chain_ms, int64_t *n_launches);

typedef struct {
    int32_t dims[4];
    int32_t precision, storage;
    int64_t n_sites;
    int64_t plane_stride;          /* P: positions per vector plane, n_sites or more (see below) */
    int32_t n_components;          /* NC: 18 or 12 stored reals per link */
    int32_t device;                /* CUDA device ordinal that holds the field */
    void *links;                   /* device: direction mu at element mu*NC*P, in blocks of
                                      16 plane positions (16*NC reals each); inside a block
                                      one vector chunk of the 16 links after another: FP32
                                      18 reals = 4 float4 chunks (complex entries 0-1, 2-3,
                                      4-5, 6-7) + 1 float2 chunk (entry 8); FP32 12 reals =
                                      3 float4 chunks; FP64 = 9 double2 chunks (one entry
                                      each); position i is element i mod 16 of its block's
                                      chunks */
    int8_t *labels;                /* device: [4][plane_stride] reference labels */
    void *stream;
    void *gauge;                   /* device: the random gauge transformation G of vs_gauge_transform
                                      (18 reals per site in the field precision, laid out as
                                      direction 0 of 18-real links), or NULL in the original gauge */
} vs_field_desc;

/* Device layout of a field.  Site positions (the index of the labels and of
 * the link blocks) follow the lexicographic rows (y, z, t), and inside each
 * x-row the sites are grouped by x mod 4: position row * 4Qp + (x mod 4) * Qp
 * + x/4 (see vs_layout_index), where Qp = Lx/4, except Qp = 8 when Lx/4 is 5,
 * 6 or 7: a group of one colour class's sites then fills one 128-byte line
 * of a float4 chunk run instead of straddling two, and the positions
 * Lx/4 .. 7 of each group hold no link (plane_stride = 4 Qp Ly Lz Lt, a
 * multiple of 256).  The links of position i are in block i / 16 of their
 * direction, element i mod 16 of each of its chunks (vs_field_desc.links). */
vs_status vs_field_describe(const vs_field *f, vs_field_desc *out);

/* Position of site (x,y,z,t) in the device layout (above). */
int64_t vs_layout_index(const int32_t dims[4], const int32_t x[4]);

/* Number of kernels the library has launched directly in this process (CUDA
 * graph replays of the serving loop are not counted). */
int64_t vs_kernel_launches(void);

/* Diagnostic: exp(X) for n traceless anti-Hermitian 3x3 matrices by the
 * kernels' Cayley-Hamilton series, in the given precision.  X, E: host
 * double [n][3][3][2]. */
vs_status vs_debug_expm(vs_ctx *ctx, const double *X, int32_t n, int32_t precision, double *E);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of smoothing jobs                          */
/* ---------------------------------------------------------------------- */

typedef struct {
    int32_t dims[4];
    int32_t precision, storage;
    const int8_t *labels;          /* host [4][V] reference labels, or NULL: vs_load_cooled(seed, n_cool) */
    uint64_t seed;
    int32_t n_cool;
    int32_t vortex_preserve;
    double omega;                  /* centrifuge angle; < 0 skips the centrifuge */
    uint64_t centrifuge_seed;
    double rho, epsilon, u0;
    int32_t n_sweeps;
    int32_t reunit_every;
    double *links_out;             /* optional host [4][V][3][3][2], written before completion */
    int32_t fp64_redecide;         /* as vs_anneal.fp64_redecide (0: FP32 decisions) */
} vs_job;

typedef struct {
    double action;                 /* <S>/beta of the smoothed field */
    int64_t n_reject;              /* vortex-preservation rejections over all sweeps */
    int64_t n_label_diff;          /* label differences after the last sweep */
    double t_submit_ms, t_admit_ms, t_done_ms;  /* on the context's monotonic clock */
    vs_status status;
    int32_t pad;
} vs_result;

/* Queue a job (the library copies it, and its labels).  Never waits on the
 * GPU.  EBUSY when max_queue jobs are waiting; EINVAL on bad parameters. */
vs_status vs_submit(vs_ctx *ctx, const vs_job *job, int64_t *ticket);

/* Result of a job: OK (and the ticket is retired), EAGAIN if not done and
 * timeout_ms == 0, ETIMEDOUT after timeout_ms (< 0: wait without limit). */
vs_status vs_poll(vs_ctx *ctx, int64_t ticket, int32_t timeout_ms, vs_result *out);

/* Cancel a queued or running job; its slot and memory are released at the
 * next sweep boundary.  ENOTFOUND for unknown or retired tickets. */
vs_status vs_cancel(vs_ctx *ctx, int64_t ticket);

typedef struct {
    int64_t submitted, completed, cancelled, running, waiting;
    uint64_t bytes_in_use, peak_bytes_in_use;
    /* chunk graphs (a job's sweeps are replayed in chunks of reunit_every
     * sweeps from a captured CUDA graph): instantiated anew, or taken from the
     * idle graphs of the same shape and updated with the job's pointers */
    int64_t graphs_instantiated, graphs_reused;
} vs_serve_stats;

vs_status vs_serve_stats_get(vs_ctx *ctx, vs_serve_stats *out);

/* Milliseconds on the context's monotonic clock (the clock of vs_result). */
double vs_now_ms(vs_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* VS_H */
