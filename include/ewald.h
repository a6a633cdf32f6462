/*
 * ewald.h - C ABI of the GB300 Ewald-summation library (libewald_gb300.so).
 *
 * The library evaluates the periodic Coulomb (Ewald) energy of a batch of
 * quantum Monte Carlo walkers and the energy change of single-particle moves
 * (Thorpe, Smith, Hasnip & Drummond, "Acceleration of the CASINO quantum
 * Monte Carlo software using GPUs and OpenACC": Sec. 2.2, Eqs. (2)-(4) in 3D
 * and Eqs. (5)-(6) in 2D, with every charge in the plane z = 0 or, for
 * layered cells, at up to EWALD_MAX_LAYERS heights; Sec. 2.1 for the
 * single-particle moves of VMC/DMC).
 *
 * Conventions
 *   - alpha ("gamma" below) is the screening parameter of erfc(alpha r); it
 *     is the square root of the paper's gamma.
 *   - Lattices are dim x dim, row-major, row i = lattice vector a_i (bohr).
 *     The cell must be right-handed (det > 0).
 *   - Positions are Cartesian, row-major [W][N][dim] (walker, particle, axis).
 *   - Energies are in hartree (Coulomb constant 1).
 *   - Every call that takes "on_device" reads or writes the caller's array
 *     in device memory when on_device != 0, and in host memory otherwise.
 *     Device arrays are accessed on the context's stream, in stream order.
 *     Host outputs are complete when the call returns (the call synchronises
 *     the stream); host inputs may be reused as soon as the call returns.
 *   - The caller owns every array it passes; the library copies what it
 *     needs and keeps no caller pointer.  The library owns all state it
 *     allocates (walker positions, rho(G), tables) and frees it in the
 *     matching destroy call.
 *   - Every int-returning call returns EWALD_OK (0) or an error code.  The
 *     last error is also kept per context (ewald_last_error).  Errors found
 *     inside kernels (coincident particles, a move index out of range) are
 *     reported by the next call that synchronises the stream, or by
 *     ewald_batch_sync.
 */
#ifndef EWALD_GB300_H
#define EWALD_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ewald_ctx ewald_ctx;     /* one periodic system: cell, charges, tables */
typedef struct ewald_batch ewald_batch; /* W walkers of one system, state on the device */

/* Arithmetic of the kernels (paper Sec. 6: single vs double precision).
 * EWALD_FP64: every kernel in FP64.
 * EWALD_MIXED: erfc, sin/cos and per-tile sums in FP32 with compensated
 * accumulation; per-walker reductions, rho(G) and constants in FP64.
 * EWALD_FP64_TIERED: FP64 results (the FP64 cutoffs and error bound) with
 * the real-space sum split by term size: a pair image whose erfc(alpha r)
 * is above 1e-7 is evaluated in FP64 from the exact fixed-point geometry
 * and FP64 charges, the smaller ones (their FP32 error is below 1e-14 of
 * the pair's 1/r) and the image tests in FP32.  Every other kernel
 * (structure factor, moves, batched and serving forms) runs as EWALD_FP64;
 * ewald_get_info reports this value. */
typedef enum { EWALD_FP64 = 0, EWALD_MIXED = 1, EWALD_FP64_TIERED = 2 } ewald_precision;

enum {
    EWALD_OK = 0,
    EWALD_ERR_ARG = 1,         /* bad dimension, NULL, size < 1, non-finite value, k out of range */
    EWALD_ERR_LATTICE = 2,     /* singular or left-handed lattice */
    EWALD_ERR_COINCIDENT = 3,  /* two particles (or images) closer than 1e-10 of the cell size */
    EWALD_ERR_NO_PROPOSAL = 4, /* accept without a pending propose */
    EWALD_ERR_OOM = 5,         /* device or host allocation failed, or over the memory budget */
    EWALD_ERR_CUDA = 6,        /* a CUDA runtime call failed */
    EWALD_ERR_TIMEOUT = 7,     /* a bounded device-side wait expired */
    EWALD_ERR_STATE = 8,       /* call not valid in the object's current state */
    EWALD_ERR_CANCELLED = 9    /* the serving request was cancelled (ewald_server_cancel) */
};

typedef struct {
    int dim;                     /* 2 or 3 */
    const double *lattice;       /* [dim][dim] host memory, rows = lattice vectors */
    int n_mobile;                /* number of moving particles (electrons), >= 1 */
    const double *mobile_charge; /* [n_mobile] host memory */
    int n_fixed;                 /* number of fixed particles (ions), >= 0 */
    const double *fixed_pos;     /* [n_fixed][dim] host memory, Cartesian (may be NULL if 0) */
    const double *fixed_charge;  /* [n_fixed] host memory (may be NULL if 0) */
    double gamma;                /* alpha of erfc(alpha r); <= 0 picks a balanced alpha */
    double g_cutoff;             /* |G| cutoff; <= 0: exp(-G^2/4alpha^2) (3D) or
                                    erfc(G/2alpha) (2D) reaches 1e-16 */
    double r_cutoff;             /* real-space cutoff; <= 0: erfc(alpha r) reaches 1e-16
                                    (EWALD_FP64) or 1e-10 (EWALD_MIXED: images beyond
                                    add less than FP32 resolves; see ewald_get_info) */
    int precision;               /* ewald_precision */
    int resum_every;             /* accepted moves between rho(G) rebuilds; 0 -> 64 */
    /* Layered 2D systems (paper Eqs. (5)-(6) with z != 0: bilayers, charges
     * above or below the plane).  dim 2 only; NULL = every particle at z = 0.
     * Particles with equal heights (exactly equal doubles) form a layer; at
     * most EWALD_MAX_LAYERS distinct heights among all particles.  A move
     * changes the in-plane position only: heights belong to the context.
     * Height differences must keep |z_i - z_j| * g_cutoff <= 600. */
    const double *mobile_z;      /* [n_mobile] host memory, or NULL */
    const double *fixed_z;       /* [n_fixed] host memory, or NULL */
} ewald_desc;

#define EWALD_MAX_LAYERS 4

/* Read-only facts about a context (for tests, manifests and tuning). */
typedef struct {
    int dim, n_mobile, n_fixed, precision;
    double alpha, r_cutoff, g_cutoff;
    double volume;        /* Omega (3D) or area A (2D) */
    int n_g_half;         /* G vectors kept, one of each +-G pair */
    int n_images;         /* distinct lattice vectors that may meet the real-space cutoff */
    int subcell_bits;     /* real-space displacement cells: 2^bits per axis */
    int pair_tile;        /* particles per side of a real-space pair tile (32, 64, 128; 256 in the mixed form) */
    int max_candidates;   /* longest candidate-image list of a displacement cell */
    int n_runs, run_len;  /* G rows split into runs of <= run_len consecutive n1 */
    double e_madelung;    /* 1/2 sum q^2 sum_{R!=0} erfc(alpha R)/R  (all charges) */
    double e_self;        /* -(alpha/sqrt(pi)) sum q^2                (all charges) */
    double e_background;  /* -pi Q^2/(2 Omega alpha^2) (3D), -sqrt(pi) Q^2/(A alpha) (2D);
                             layered 2D: -(pi/A) sum_{L,L'} Q_L Q_L' g(z_L - z_L'),
                             g(z) = z erf(alpha z) + exp(-alpha^2 z^2)/(alpha sqrt(pi)) */
    double e_fixed_real;  /* real-space pair sum among fixed particles */
    int n_layers;         /* distinct particle heights (1 unless the desc gave heights) */
    int mixed_direct;     /* mixed form: 1 if the energy kernels' pair loop evaluates the two
                             images nearest to each displacement cell's centre as one masked
                             term without testing them first (chosen at set-up where those two
                             lie inside r_cutoff for at least 3/4 of the displacements), else 0 */
} ewald_info;

/* Create a context: validates the description, builds the G list, the image
 * lists and the constants in FP64 on the host (paper Sec. 6.1 keeps these
 * set-up tables in double precision) and uploads them once (Sec. 2.2: the
 * Ewald data move to the GPU at the outset).  cuda_stream is a cudaStream_t;
 * NULL makes the library create a blocking stream of its own.  On error
 * *out is set to NULL. */
int ewald_create(const ewald_desc *desc, void *cuda_stream, ewald_ctx **out);
void ewald_destroy(ewald_ctx *ctx);
int ewald_get_info(const ewald_ctx *ctx, ewald_info *info);

/* Plan a context without creating it: runs the same host set-up as
 * ewald_create (validation, cutoffs, G list, image and candidate lists,
 * constants, all in FP64; paper Sec. 6.1) and its default real-space tiling,
 * and fills *info as ewald_get_info would for the new context.  Touches no
 * GPU and allocates no device memory, so it also works on a machine without
 * one (sizing, manifests, tests of the set-up).  A tiling cached through
 * EWALD_TUNE_CACHE is not applied.  Errors: those of ewald_create's
 * validation (EWALD_ERR_ARG, EWALD_ERR_OOM); EWALD_ERR_ARG for a NULL
 * argument.  info is caller-owned host memory. */
int ewald_plan(const ewald_desc *desc, ewald_info *info);
/* The half-space G list in the library's storage order: nvec[n_g_half][dim]
 * integer coordinates on the reciprocal basis (host memory). */
int ewald_get_gvectors(const ewald_ctx *ctx, int *nvec);
/* Last error recorded on the context (sticky until the next successful call
 * that checks it). */
int ewald_last_error(const ewald_ctx *ctx);
const char *ewald_strerror(int code);
/* How the library was built: EWALD_BUILD_DEBUG_CHECKS set for the debug
 * build (libewald_gb300_debug.so, compiled with -DEWALD_DEBUG), whose
 * kernels check their ring and queue fill levels, candidate-list, G-slot
 * and particle indices, skip an out-of-range access and report it as
 * EWALD_ERR_STATE on the next synchronising call.  Not in the paper: a
 * development aid, for tiny cases compared with the ordinary build. */
#define EWALD_BUILD_DEBUG_CHECKS 1
int ewald_build_flags(void);
/* A one-line description of the context's last failure (argument checked,
 * CUDA call and its error string, ...); valid until the next call on the
 * context.  Never NULL. */
const char *ewald_last_error_message(const ewald_ctx *ctx);

/* Walker batches.  A batch owns the walkers' positions (fixed-point
 * fractional coordinates), their rho(G) and the pending moves.  Before the
 * first energy or move the positions must be set.
 *
 * Host arrays (on_device = 0) may be ordinary or page-locked memory
 * (cudaMallocHost, cudaHostRegister); page-locked arrays are copied by DMA
 * directly, others through the batch's staging buffer.  Either way the call
 * has finished with the caller's array when it returns. */
int ewald_batch_create(ewald_ctx *ctx, int n_walkers, ewald_batch **out);
void ewald_batch_destroy(ewald_batch *b);
/* pos: [W][N][dim] Cartesian.  Positions are stored wrapped into the cell;
 * get_positions returns the wrapped positions.  rho(G) follows new
 * positions: it is rebuilt by the next energy, or before the next call that
 * reads it (propose, resum, get_rho). */
int ewald_batch_set_positions(ewald_batch *b, const double *pos, int on_device);
int ewald_batch_get_positions(ewald_batch *b, double *pos, int on_device);
/* Synchronise the context's stream and report errors raised by kernels. */
int ewald_batch_sync(ewald_batch *b);

/* Full Ewald energy of every walker, e_out[W] (paper Eq. (2) with Eqs. (3)-(4)
 * or (5)-(6)).  Also rebuilds each walker's rho(G) from scratch. */
int ewald_energy(ewald_batch *b, double *e_out, int on_device);
/* Same, with components comp_out[W][5] =
 * {E_real, E_madelung, E_recip, E_self, E_background}; E_real includes the
 * fixed-fixed pairs, and the other four include every charge.  Sum = energy. */
int ewald_energy_components(ewald_batch *b, double *comp_out, int on_device);

/* Propose moving particle k[w] of every walker w to r_new[w][dim]
 * (Cartesian) and return the Ewald energy change de_out[W].  The move is
 * remembered as pending; a second propose replaces it.  Cost O(N + N_G)
 * per walker.  k, r_new and de_out are all host or all device arrays. */
int ewald_propose_move(ewald_batch *b, const int *k, const double *r_new, double *de_out,
                       int on_device);
/* Apply the pending moves of the walkers with accept[w] != 0: position and
 * rho(G) += delta(G) in FP64.  Every resum_every accepted moves of a walker
 * its rho(G) is rebuilt from scratch.  EWALD_ERR_NO_PROPOSAL if nothing is
 * pending. */
int ewald_accept_move(ewald_batch *b, const unsigned char *accept, int on_device);
/* Rebuild rho(G) of every walker from its positions. */
int ewald_resum(ewald_batch *b);
/* rho(G) of every walker, rho_out[W][n_layers][n_g_half][2] (re, im), G in
 * the order of ewald_get_gvectors, layers in increasing height (n_layers = 1
 * unless the context has heights); includes the fixed particles'
 * contribution. */
int ewald_batch_get_rho(ewald_batch *b, double *rho_out, int on_device);

/* Batched form: walkers of several batches - of different systems (N,
 * cell, dimension 2 or 3, charges), all of one precision - evaluated by one
 * persistent kernel launch per call.  The work items (walker x chunk of G
 * runs, walker x pair tile) are ordered longest first at creation and taken
 * by the CTAs from an atomic counter; the CTA that finishes a walker's last
 * item adds up its energy in a fixed order, so a result does not depend on
 * the schedule or the other batches and equals the single-batch
 * ewald_energy of that walker to rounding.  The launch is
 * captured once in a CUDA graph and replayed by every call.  The batches
 * must keep their positions set and outlive the multi object; their
 * contexts' streams are ordered with the multi's own stream by events.
 * (Paper Sec. 5.1 splits the Ewald sum into independent real- and
 * reciprocal-space loops; here those loops of many systems share one
 * launch.) */
typedef struct ewald_multi ewald_multi;
int ewald_multi_create(ewald_batch *const *batches, int n_batches, ewald_multi **out);
/* e_out[sum_b W_b]: energies of every walker, batches in creation order.
 * Also rebuilds every walker's rho(G), like ewald_energy. */
int ewald_multi_energy(ewald_multi *m, double *e_out, int on_device);
void ewald_multi_destroy(ewald_multi *m);

/* Serving form: continuous batching of walker batches from concurrent runs.
 * A request is W walkers of one system (a context of the server's
 * precision, see below) that each make n_steps single-particle moves: particle k
 * uniform, Gaussian displacement of standard deviation sigma per axis,
 * accepted with probability accept_prob (there is no wave function here),
 * all drawn on the device from a counter-based SplitMix64 stream of the
 * request's seed.  precision: EWALD_MIXED takes mixed contexts, EWALD_FP64
 * FP64 and tiered ones (moves by the plain FP64 kernel), EWALD_FP64_TIERED
 * tiered ones (moves by the tiered kernel: real space split by term size,
 * reciprocal part and rho(G) in FP64).  Requests queue on submission and are admitted between
 * steps while the server's walker slots and device-memory budget allow;
 * from admission on their rho(G) stays on the device.  Every step advances
 * every active request by one move in one persistent launch (replayed from
 * a CUDA graph), whatever the mix of systems; finished requests are retired
 * between steps.  A walker's result is the same alone and in any mix.
 * Results: the final energy of every walker (initial Ewald energy plus the
 * accepted energy changes) and its number of accepted moves.  The contexts
 * must outlive the server.  (Paper Sec. 2.1: VMC and DMC are sequences of
 * single-particle moves; Sec. 2.2: the Ewald data stay on the device.)
 * hbm_budget_bytes <= 0 takes 80% of the free device memory. */
typedef struct ewald_server ewald_server;
int ewald_server_create(int precision, int max_walkers, double hbm_budget_bytes, void *cuda_stream,
                        ewald_server **out);
void ewald_server_destroy(ewald_server *srv);
/* pos: host [n_walkers][N][dim], copied.  *request_id receives the id. */
int ewald_server_submit(ewald_server *srv, ewald_ctx *system, const double *pos, int n_walkers,
                        int n_steps, double sigma, double accept_prob, unsigned long long seed,
                        int *request_id);
/* Retire finished requests, admit queued ones, and queue one move of every
 * active request; returns without waiting for the device. */
int ewald_server_step(ewald_server *srv, int *n_active, int *n_queued);
/* EWALD_OK and the results (host arrays [W], either may be NULL) once the
 * request is done, EWALD_ERR_STATE before, EWALD_ERR_CANCELLED after
 * ewald_server_cancel; latency_ms = submission to completion as seen by the
 * host. */
int ewald_server_result(ewald_server *srv, int request_id, double *energies, int *n_accepted,
                        double *latency_ms);
/* Ids of requests that finished since the last call (up to max_ids, the
 * rest on the next call; *n receives the count): a host loop can fetch just
 * those results instead of polling every pending request. */
int ewald_server_completed(ewald_server *srv, int *ids, int max_ids, int *n);
/* Device bytes that admission counts against the server's memory budget
 * for a request of n_walkers walkers of system (its batch state and
 * upload buffer), in *bytes.  A request above the budget is refused by
 * ewald_server_submit with EWALD_ERR_OOM; queued requests wait until the
 * bytes of the active ones plus theirs fit.  Not in the paper. */
int ewald_server_request_bytes(const ewald_ctx *system, int n_walkers, double *bytes);
/* Cancel a request from the host.  A queued request leaves the queue; an
 * active one stops moving: it is retired at the next ewald_server_step
 * (its device memory returned, stream-ordered, after the moves already
 * queued), without results.  Either way it is reported once by
 * ewald_server_completed, and ewald_server_result answers
 * EWALD_ERR_CANCELLED.  The other requests are unaffected (every walker's
 * result is the same alone and in any mix).  EWALD_ERR_STATE if the request
 * has already finished or was cancelled; EWALD_ERR_ARG for an unknown id.
 * Not in the paper: a serving-loop facility. */
int ewald_server_cancel(ewald_server *srv, int request_id);
/* Wait until everything queued on the server's stream has run. */
int ewald_server_drain(ewald_server *srv);
const char *ewald_server_error_message(const ewald_server *srv);

/* Autotuner.  Times the real-space kernel on (up to 512 of) the batch's
 * walkers for every allowed real-space tiling - pair tiles of 32, 64 or 128
 * particles per side (also 256 in the mixed form) x 2^bits displacement
 * cells per axis (candidate lists <= 48 KB) x, in the mixed form, CTAs of
 * 256 or 512 threads - and the structure-factor kernel for 1 to 4 chunks of
 * G runs per walker (the threads of its CTAs), and keeps the fastest of
 * each in the batch's context.  With
 * cache_path (may be NULL) the result is looked up first and stored after
 * tuning in a small JSON file keyed by the system's shape and the GPU name;
 * ewald_create also applies a cached tiling when the environment variable
 * EWALD_TUNE_CACHE names such a file.  Retune before creating multi objects
 * that include the context: a multi keeps the tiling it was created with. */
typedef struct {
    int pair_tile, subcell_bits;
    double ms;       /* real-space kernel time of the chosen tiling, ms */
    int n_tried;     /* tilings timed (0 if taken from the cache) */
    int from_cache;
    int real_threads;  /* threads per real-space CTA of the chosen tiling */
    int sfac_chunks;   /* structure-factor chunks per walker chosen */
    double sfac_ms;    /* structure-factor kernel time with them, ms */
} ewald_tune_result;
int ewald_autotune(ewald_batch *b, const char *cache_path, ewald_tune_result *res);

/* Splitting parameter by measurement (alpha balancing).  alpha moves work
 * between the real-space sum (~alpha^-3) and the reciprocal sum (~alpha^3)
 * without changing the energy (paper Eq. (2): v_E does not depend on gamma,
 * up to the cutoff tolerances); the best balance depends on the precision,
 * the system and the GPU.  For desc (r_cutoff and g_cutoff must be <= 0:
 * they follow alpha) this times the full energy of the sample pos
 * [n_walkers][N][dim] (host memory, Cartesian) on trial contexts at alpha =
 * a0 x {0.6 ... 3} around a0 (desc->gamma if > 0, else the balanced
 * default), refines around the fastest, and returns it in *alpha_out and
 * its time per walker (microseconds) in *us_per_walker (may be NULL).
 * Trials the cell cannot take (cutoffs too large) are skipped.  Uses
 * cuda_stream like ewald_create; synchronises it.  Errors: EWALD_ERR_ARG
 * for bad arguments, the starting context's error, EWALD_ERR_CUDA if no
 * trial could be timed (e.g. coincident particles in the sample). */
int ewald_tune_alpha(const ewald_desc *desc, void *cuda_stream, int n_walkers, const double *pos, double *alpha_out,
                     double *us_per_walker);

/* Full energies without any device allocation at call time.  Meant for
 * callers that cannot call cudaMalloc while they compute (a host framework
 * that owns all device memory through its own pool and would see a foreign
 * allocation fragment it, an embedded code that reserves memory up front).
 * Every precision form of the context computes what ewald_energy computes
 * (the tiered form with its double-float structure factor).
 * pos [n_walkers][N][dim] and e_out [n_walkers] are device arrays of the
 * caller; status_out (device int, may be NULL) receives 0, or bit 1 for
 * coincident particles and bit 4 for a non-finite position.  All
 * intermediates live in one static device array of 32 MiB that every GPU
 * which loads the library holds until the process exits; n_walkers beyond
 * what fits for this system returns EWALD_ERR_OOM with the limit in
 * ewald_last_error_message.  Work is queued on the context's stream and the
 * call returns without waiting.  Calls that overlap on the GPU (other
 * streams, other contexts, other threads) share that array and race: keep
 * them ordered.  The first call on each device looks up the array's device
 * address; make that first call before any stream capture.  There is no
 * counterpart in the paper: this is a deployment convenience. */
int ewald_energy_noalloc(ewald_ctx *ctx, const double *pos, int n_walkers, double *e_out, int *status_out);

/* Kernel timers of a context (in the spirit of the paper's per-subroutine
 * timers, Sec. 3.2).  When enabled, every kernel the context launches is
 * bracketed by CUDA events on its stream.  ewald_get_timing synchronises
 * the stream, writes the accumulated device milliseconds and launch counts
 * of the EWALD_N_KERNELS kernels (ms[EWALD_N_KERNELS], launches[...], host
 * memory; either may be NULL), and resets them.  Kernel order: ingest,
 * structure factor, real space, combine, propose, accept, resum. */
#define EWALD_N_KERNELS 7
int ewald_set_timing(ewald_ctx *ctx, int enable);
int ewald_get_timing(ewald_ctx *ctx, double *ms, long long *launches);

/* Two-body plane-wave Jastrow term (paper Sec. 2.3, Eqs. (7), (9), (10)):
 *   J_p = sum_{i<j} p(r_i - r_j),  p(r) = sum_{m=1}^{n_stars} a_m sum_{G in star_m^+} cos(G.r)
 * over the mobile particles (electrons) of each walker, with a star read as
 * a shell of simulation-cell reciprocal-lattice vectors of equal |G| counted
 * from the shortest, star_m^+ one of each +-G pair.
 * ewald_jastrow_p_set stores the stars' G vectors and coefficients a[n_stars]
 * (host memory, 1 <= n_stars <= 64) on the context; ewald_jastrow_p_count
 * gives the number of G vectors kept.  ewald_jastrow_p writes, per walker,
 * j_out[W] and optionally grad_out[W][N][dim] = dJ_p/dr_i and
 * lap_out[W][N] = Laplacian of J_p with respect to r_i (either may be NULL);
 * all three on the device or on the host together (on_device).  Positions
 * are the batch's; phases are exact (fixed-point) in both precisions;
 * EWALD_FP64 sums in FP64, EWALD_MIXED in compensated FP32 with rho(G) and
 * J_p in FP64.  Errors: EWALD_ERR_STATE without positions or stars. */
int ewald_jastrow_p_set(ewald_ctx *ctx, int n_stars, const double *a);
int ewald_jastrow_p_count(const ewald_ctx *ctx, int *n_g);
int ewald_jastrow_p(ewald_batch *b, double *j_out, double *grad_out, double *lap_out, int on_device);

/* Polynomial two-body Jastrow term (paper Sec. 2.3, Eqs. (7), (8)):
 *   J_u = sum_{i<j} u(r_ij),  u(r) = (r - L_u)^C sum_{l=0}^{n_u} alpha_l r^l for r < L_u, 0 beyond,
 * over the mobile particles of each walker, r_ij the nearest-image distance.
 * Mobile particles 0 .. n_up-1 have spin up, the others spin down; pairs of
 * like spins use alpha_like[0..n_u], unlike spins alpha_unlike[0..n_u]
 * (host memory).  alpha_*[1] is ignored: the Kato cusp condition u'(0) =
 * Gamma fixes alpha_1 = Gamma/(-L_u)^C + C alpha_0/L_u, Gamma = 1/4 (like)
 * and 1/2 (unlike) in 3D, 1/3 and 1 in 2D.  Requirements: 0 <= n_up <=
 * n_mobile, 1 <= C <= 8, 1 <= n_u <= 24, 0 < L_u < half the shortest
 * lattice vector (EWALD_ERR_ARG otherwise).  ewald_jastrow_u_set stores
 * the term on the context (replacing an earlier one; it synchronises the
 * context's stream).  ewald_jastrow_u writes j_out[W] and optionally
 * grad_out[W][N][dim] and lap_out[W][N] (the gradient and Laplacian with
 * respect to each particle; either may be NULL), all on the device or all
 * on the host (on_device).  EWALD_FP64: FP64 throughout; EWALD_MIXED: FP32
 * terms in compensated FP32 sums, J_u added up in FP64.  Errors:
 * EWALD_ERR_STATE without positions or without a u term; coincident
 * particles set the batch's status (EWALD_ERR_COINCIDENT at the next
 * synchronising call). */
int ewald_jastrow_u_set(ewald_ctx *ctx, int n_up, double L_u, int C, int n_u, const double *alpha_like,
                        const double *alpha_unlike);
int ewald_jastrow_u(ewald_batch *b, double *j_out, double *grad_out, double *lap_out, int on_device);

/* Measured arithmetic peaks of the current GPU, for the rooflines of the
 * ALU-bound kernels: FP32 FMA and FP64 FMA in TFLOP/s (2 flop per FMA) and
 * the special-function unit's rsqrt rate in Tops/s.  Runs a few
 * milliseconds of multiply-add chains on a private stream and synchronises
 * it; any output pointer may be NULL.  Not part of the method: a
 * measurement aid (the paper quantifies GPU performance against peaks in
 * Sec. 4). */
int ewald_measure_peaks(double *fp32_tflops, double *fp64_tflops, double *mufu_tops);

/* The mixed form's FP32 real-space term erfc(alpha r)/r (Eq. (3), second
 * term) for n values of r^2 (host arrays, r2[i] > 0 and finite), evaluated
 * on the GPU by the scalar function and by its paired form (two terms per
 * lane with FFMA2/FADD2/FMUL2) into scalar_out[n] and paired_out[n].  The
 * real-space kernels use the paired form; the two are meant to agree bit
 * for bit.  A diagnostic for tests: synchronous, allocates and frees its
 * own device buffers.  EWALD_ERR_ARG for n < 0, null arrays, alpha not
 * positive and finite or an r^2 that is not. */
int ewald_pair_terms(int n, const float *r2, double alpha, float *scalar_out, float *paired_out);
/* The tiered form's head-term arithmetic (double-float 1/r by Newton steps,
 * piecewise-Taylor erfc; FP32 pipe only) on n FP64 values of r^2 (host
 * arrays), erfc(alpha r)/r returned in FP64 in out[n].  Same diagnostic
 * terms and errors as ewald_pair_terms; alpha r must stay below 4, the
 * head range (erfc(alpha r) > 1e-7 means alpha r < 3.77). */
int ewald_pair_terms_df(int n, const double *r2, double alpha, double *out);

#ifdef __cplusplus
}
#endif
#endif
