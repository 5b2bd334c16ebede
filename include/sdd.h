/*
 * libsdd -- GB300 (sm_103a) Monte Carlo evaluation of the Feynman-Kac
 * representation of the TE (E-polarisation) magnetotelluric equation at the
 * interface nodes of a stochastic domain decomposition (Bihlo, Farquharson,
 * Haynes, Loredo-Osti, arXiv:1603.09311).
 *
 * The operation (Sec. 2.2 and Sec. 3.1).  For the TE mode the diffusion
 * coefficient of the discontinuous elliptic problem is constant, so the
 * equation is, in dimensionless form,
 *     Lap u = i kappa(x) u   in the rectangle Omega,   u = g on dOmega,
 * with kappa(x) = omega mu sigma(x) L^2 >= 0 piecewise constant over
 * materials.  By the Kac-Feynman formula (Sec. 2.2)
 *     u(x0) = E[ g(beta_tau) exp(-i (1/2) int_0^tau kappa(beta_s) ds) ],
 * beta a standard 2D Brownian motion started at x0.  The library simulates
 * beta with the Euler-Maruyama scheme of Sec. 3.1, ends each walk with the
 * boundary-hitting rule of the first-exit-time estimate (linear interpolation
 * on overshoot, Brownian-bridge test with one uniform when both ends are
 * inside), counts the Euler steps spent in each material (the occupation
 * times T_m of Sec. 3.1) and averages g(exit) exp(-i (1/2) sum_m kappa_m T_m)
 * over the walks (the Monte Carlo estimator of Sec. 3.1).  One walk serves
 * every evaluation e (a row kappa[e][.] of phase rates, e.g. a frequency),
 * because the TE walk does not depend on kappa.
 *
 * Around that path the library also provides:
 *  - TM models: vertical strips whose diffusion coefficient jumps, walked
 *    with the interface rules of Sec. 3.1 (sdd_model_desc.diffusion);
 *  - interpolation between Monte Carlo nodes along an interface (Sec. 5):
 *    sdd_interpolate, sdd_interface_values_interp;
 *  - apparent resistivity and phase at measurement sites (Sec. 2.1,
 *    Sec. 4.2): sdd_apparent_resistivity;
 *  - the RBF-FD sub-domain solve that completes the decomposition
 *    (Sec. 3.2): sdd_rbffd_weights, sdd_rbffd_solve;
 *  - batched, graph, allocation-free, asynchronous and served launches of
 *    the walk;
 *  - raw sums of path ranges and their fixed-order reduction, for an
 *    evaluation split across processes (sdd_range_sums, sdd_reduce_sums).
 *
 * Conventions common to all entry points:
 *  - z grows downwards; air is z < 0, earth z >= 0.
 *  - All arrays are dense, row-major, little-endian, in the units stated.
 *  - The caller owns every array it passes.  Host arrays are read (or
 *    written) before the call returns; device arrays passed to the *_device
 *    entry points must stay valid until the work queued on the stream ends.
 *  - The library owns the device copy of the model and its scratch buffers
 *    (work-item table, per-item partial sums, counters) until sdd_destroy.
 *  - Every entry point returns an sdd_status.  On any status other than
 *    SDD_OK and SDD_E_TRUNCATED the outputs are undefined.  SDD_E_TRUNCATED
 *    means some walks reached max_steps: they are left out of the averages,
 *    the outputs are valid and stats->truncated counts them.
 *  - A context may be used from one host thread at a time, except that
 *    asynchronous requests (sdd_interface_values_async) may be submitted to
 *    one context from several threads.
 */
#ifndef SDD_H
#define SDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SDD_OK = 0,
    SDD_E_ARG = 1,         /* invalid argument (message via sdd_last_error) */
    SDD_E_OOM = 2,         /* device or host allocation failed */
    SDD_E_CUDA = 3,        /* a CUDA runtime call failed */
    SDD_E_TRUNCATED = 4,   /* results valid; some walks hit max_steps */
    SDD_E_CANCELLED = 5,   /* serving request cancelled */
    SDD_E_TIMEOUT = 6,     /* a bounded wait gave up */
    SDD_E_UNSUPPORTED = 7, /* no kernel for this configuration */
    SDD_E_BUSY = 8         /* serving admission refused: no slot or memory */
} sdd_status;

#define SDD_MAX_MATERIALS 8
#define SDD_MAX_EVAL 32
#define SDD_MAX_SHAPES 16

typedef struct sdd_ctx sdd_ctx;
typedef struct sdd_request sdd_request;

/* Rectangular domain Omega = [x_min, x_max] x [z_min, z_max]. */
typedef struct {
    double x_min, x_max, z_min, z_max;
} sdd_domain;

enum { SDD_SHAPE_RECT = 0, SDD_SHAPE_TRIANGLE = 1 };

/* One material region.  RECT: half-open [v0, v1) x [v2, v3).  TRIANGLE:
 * closed triangle with vertices (v0, v1), (v2, v3), (v4, v5), either
 * orientation.  Later shapes override earlier ones and the background. */
typedef struct {
    int32_t kind;
    int32_t material;
    double v[6];
} sdd_shape;

/* Dirichlet data g on dOmega.
 * SDD_G_COLUMNS: the one-dimensional layered TE solution of Sec. 2.1 --
 *   for a column with earth rate k_c: u = exp(-k z) (z >= 0), u = 1 - k z
 *   (z < 0, air), k = sqrt(i k_c) with Re k >= 0.  The left wall uses the
 *   column of material g_left, the right wall that of g_right (rates from
 *   the evaluation's kappa row), top and bottom interpolate linearly in x
 *   between the two corner values.
 * SDD_G_AFFINE: g = a + b x + c z, complex a, b, c in g_coef
 *   (a_re, a_im, b_re, b_im, c_re, c_im); harmonic, for checks.
 * SDD_G_X2MZ2: g = x^2 - z^2; harmonic, for checks.
 * SDD_G_TM_COSH (TM mode only): g = (z + 1) cosh(a x), a = sqrt(i kappa_{e,s} / D_s)
 *   with Re a >= 0 for the strip s of x: the exact solution of the analytic
 *   test model of Sec. 4.1 when its one interface is at x = 0.
 * SDD_G_TM_FLUX (TM mode only): g = int_{x_min}^x ds / D(s), the solution with
 *   kappa = 0 and the same flux D u' = 1 in every strip. */
enum { SDD_G_COLUMNS = 0, SDD_G_AFFINE = 1, SDD_G_X2MZ2 = 2, SDD_G_TM_COSH = 3, SDD_G_TM_FLUX = 4 };

/* Conductivity model.  Material of a point: if raster != NULL, the cell
 * (clamp(floor((x - x_min) nx / (x_max - x_min))), same for z) of the int8
 * raster [nz][nx]; otherwise bg_air (z < 0) or bg_earth (z >= 0) overridden
 * by the shapes in order.  kappa[e][m] >= 0 is the dimensionless phase rate
 * of material m in evaluation e.
 *
 * TM mode (diffusion != NULL): the diffusion coefficient jumps across
 * vertical interfaces (Sec. 2.2, the Helmholtz equation per sub-domain with
 * flux continuity; the interface rules of Sec. 3.1).  Material m is the strip
 * [interfaces[m-1], interfaces[m]) (the first from x_min, the last to x_max)
 * with diffusion D_m, and D_m Lap u = i kappa_{e,m} u there; kappa may then
 * be negative.  Shapes, raster and background are not used, and g_kind is
 * AFFINE, X2MZ2, TM_COSH or TM_FLUX. */
typedef struct {
    sdd_domain domain;
    int32_t n_materials;   /* K, 1..SDD_MAX_MATERIALS */
    int32_t n_eval;        /* E, 1..SDD_MAX_EVAL */
    const double *kappa;   /* host, [n_eval][n_materials], copied */
    int32_t bg_air, bg_earth;
    const sdd_shape *shapes; /* host, copied; may be NULL if n_shapes == 0 */
    int32_t n_shapes;        /* 0..SDD_MAX_SHAPES */
    const int8_t *raster;    /* host, [nz][nx] material ids, copied; or NULL */
    int32_t nx, nz;          /* raster size: each side 1..2^20 cells, nx * nz <= 2^31 */
    int32_t g_kind;
    int32_t g_left, g_right;
    double g_coef[6];
    const double *diffusion;  /* host, [n_materials] D_m > 0, copied; NULL = TE mode */
    const double *interfaces; /* host, [n_materials - 1] strictly increasing, inside
                                 (x_min, x_max), copied; TM mode only */
} sdd_model_desc;

enum { SDD_FP32 = 0, SDD_FP64 = 1 };

/* Launch options; zero means automatic. */
typedef struct {
    int32_t precision;     /* SDD_FP32: single-precision walk, FP64 sums.
                              SDD_FP64: double-precision walk (parity mode). */
    int64_t max_steps;     /* per-walk step cap, 0..2^26; 0 = ceil(20 / dt).  Rounded
                              up to a multiple of 8 (a single-precision walk
                              advances 8 Euler steps per iteration) */
    int32_t block_threads; /* threads per CTA (multiple of 32, <= 256); 0 = auto */
    int32_t ctas_per_sm;   /* persistent CTAs per SM; 0 = occupancy limit */
    int32_t chunk_paths;   /* > 0: work items of this many paths (the last one of a
                              node shorter); 0 = guided sizes (guided_factor) */
    int32_t use_graph;     /* sdd_interface_values_device: 1 = run the device work as a
                              CUDA graph cached in the context (updated in place on
                              later calls, re-instantiated only when its shape changes) */
    int32_t guided_factor; /* guided work items (chunk_paths == 0): cut in rounds, each
                              node's item taking ceil(R / (guided_factor x warps)) paths,
                              R the paths not yet cut, rounded up to a multiple of 32,
                              at least 32; the queue hands them out in cut order, so
                              they shrink toward its end.  0 = auto (tuned, else 2) */
} sdd_config;

typedef struct {
    uint64_t steps;      /* Euler steps simulated (exiting steps included) */
    uint64_t walks;      /* walks simulated */
    uint64_t truncated;  /* walks that reached max_steps */
    double kernel_ms;    /* device time of the walk kernel (CUDA events) */
    int32_t launches;    /* kernels launched by the call */
    int32_t items;       /* work items (node, path chunk) */
    int32_t grid;        /* CTAs of the persistent walk kernel */
    int32_t block;       /* threads per CTA */
    uint64_t h2d_bytes;  /* host-to-device bytes copied by the call */
    uint64_t d2h_bytes;  /* device-to-host bytes copied by the call */
    double post_ms;      /* device time of the kernels that follow the walks (CUDA
                            events; sdd_interface_values_interp and
                            sdd_apparent_resistivity, 0 elsewhere) */
} sdd_stats;

/* Create a context on the current CUDA device and copy the model to it.
 * Errors: SDD_E_ARG (bad sizes, material ids out of range, kappa < 0 or not
 * finite, empty domain), SDD_E_OOM, SDD_E_CUDA.  *out is NULL on error. */
sdd_status sdd_create(const sdd_model_desc *model, sdd_ctx **out);

/* Free the context and everything it owns.  NULL is allowed. */
void sdd_destroy(sdd_ctx *ctx);

/* Interface-node values, host buffers, synchronous (Sec. 3.1 estimator).
 *   nodes_xz  host, [n_nodes][2] (x, z), each strictly inside the domain
 *   node_ids  host, [n_nodes] RNG node ids, or NULL for 0..n_nodes-1
 *   n_paths   host, [n_nodes] walks per node, 1 .. 2^31-1
 *   dt        Euler time step (standard Brownian clock), > 0
 *   seed      64-bit Philox4x32-10 key; step n of walk (node id i, path r)
 *             uses the two words of counter (n>>1, r, i, 0) (words 0,1 for even
 *             n, 2,3 for odd n): SDD_FP32 takes its two normals from their low
 *             23 bits and its bridge uniform from the other 18 bits; SDD_FP64
 *             takes its normals from the full words and its bridge uniform
 *             from counter (n, r, i, 1).  Results do not depend on the launch
 *   cfg       options, or NULL for defaults
 *   mean      host out, [n_nodes][n_eval][2] (re, im) sample means
 *   se        host out, [n_nodes][n_eval][2] standard errors of re and im
 *             (sqrt of the unbiased sample variance / N)
 *   stats     host out, nullable
 * n_nodes == 0 is allowed and does nothing.  The host-to-device copies of
 * the inputs and the device-to-host copies of the outputs are part of the
 * call. */
sdd_status sdd_interface_values(sdd_ctx *ctx, const double *nodes_xz, const uint32_t *node_ids,
                                int32_t n_nodes, const int64_t *n_paths, double dt,
                                uint64_t seed, const sdd_config *cfg, double *mean, double *se,
                                sdd_stats *stats);

/* Same computation on device buffers, queued on `stream` (a cudaStream_t;
 * NULL = legacy default stream); returns once the work is queued.
 *   d_nodes_xz  device, [n_nodes][2]
 *   d_node_ids  device, [n_nodes], or NULL for 0..n_nodes-1
 *   n_paths     HOST, [n_nodes] (the work-item table is planned on the host)
 *   d_mean, d_se device outputs, layouts as above
 *   d_counters  device, 3 x uint64 (steps, walks, truncated) written by the
 *               call, or NULL
 * The context's scratch buffers are reused by the next call on the same
 * context, so calls on one context must be ordered on one stream. */
sdd_status sdd_interface_values_device(sdd_ctx *ctx, const double *d_nodes_xz,
                                       const uint32_t *d_node_ids, int32_t n_nodes,
                                       const int64_t *n_paths, double dt, uint64_t seed,
                                       const sdd_config *cfg, double *d_mean, double *d_se,
                                       uint64_t *d_counters, void *stream);

/* Interface-node values at a target standard error, host buffers,
 * synchronous.  Each node first runs paths 0 .. n_pilot-1; from their sample
 * variance it gets N = clamp(ceil(max_e (var_re + var_im) / target_se^2),
 * n_pilot, n_max) walks in all, and paths n_pilot .. N-1 are run in a second
 * launch.  The sums of the two phases are added in fixed order, so the result
 * equals sdd_interface_values with n_paths = N up to FP64 summation order.
 *   n_pilot, n_max  2 <= n_pilot <= n_max <= 2^31-1
 *   target_se       complex standard error aimed at, sqrt(var_re + var_im)/sqrt(N)
 *   n_used          host out, [n_nodes] N of each node, nullable
 * Other arguments as sdd_interface_values.  A node reaching n_max may stay
 * above target_se; compare se with target_se to count the nodes that met it. */
sdd_status sdd_interface_values_target(sdd_ctx *ctx, const double *nodes_xz,
                                       const uint32_t *node_ids, int32_t n_nodes,
                                       int64_t n_pilot, int64_t n_max, double target_se,
                                       double dt, uint64_t seed, const sdd_config *cfg,
                                       double *mean, double *se, int64_t *n_used,
                                       sdd_stats *stats);

/* One model's share of a batched launch. */
typedef struct {
    sdd_ctx *ctx;               /* the model (created by sdd_create) */
    const double *nodes_xz;     /* host, [n_nodes][2] */
    const uint32_t *node_ids;   /* host, [n_nodes] RNG node ids, or NULL for 0..n_nodes-1 */
    int32_t n_nodes;
    const int64_t *n_paths;     /* host, [n_nodes] */
    double *mean;               /* host out, [n_nodes][n_eval][2] */
    double *se;                 /* host out, [n_nodes][n_eval][2] */
} sdd_batch_entry;

/* Interface-node values of several models in ONE launch of the persistent
 * walk kernel, host buffers, synchronous (the estimator of Sec. 3.1 for each
 * entry).  The models must be raster models on the same device with the same
 * domain, raster size, n_eval and g_kind; 1..256 entries.  Walk (node id i,
 * path r) of an entry uses the same Philox stream as in sdd_interface_values
 * with the same seed, so each entry's result equals its result computed
 * alone, up to FP64 summation order.  The first entry's context lends its
 * scratch buffers.  Errors: SDD_E_ARG (mismatched models, bad nodes),
 * SDD_E_UNSUPPORTED (non-raster model, SDD_FP64). */
sdd_status sdd_batch_values(const sdd_batch_entry *entries, int32_t n_entries, double dt,
                            uint64_t seed, const sdd_config *cfg, sdd_stats *stats);

/* Pick the launch shape for a workload by timing it: threads per CTA in
 * {128, 192, 256} x guided factor in {1, 2, 4, 8} (which sets the sizes of
 * the work items), two runs each of sdd_interface_values on the given nodes.
 * The fastest shape is kept in the context and used by later calls whose
 * block_threads, chunk_paths and guided_factor are automatic; with the
 * environment variable SDD_TUNE_CACHE naming a file, it is also appended
 * there and read by new contexts with the same device, lookup program,
 * materials bound, evaluations, precision and decade of dt.
 *   base   options whose block_threads, chunk_paths and guided_factor are 0,
 *          or NULL
 *   best   out (nullable): base with the chosen block_threads and
 *          guided_factor (chunk_paths 0: guided items)
 *   best_steps_per_s  out (nullable): walk-steps/s of the chosen shape
 * Library-level design choice: the paper has no launch shapes. */
sdd_status sdd_autotune(sdd_ctx *ctx, const double *nodes_xz, int32_t n_nodes,
                        const int64_t *n_paths, double dt, uint64_t seed, const sdd_config *base,
                        sdd_config *best, double *best_steps_per_s);

/* Per-path records of walks (node id, paths p0 .. p0+count-1) started at
 * (x0, z0), host buffers, synchronous -- the individual steps of Sec. 3.1
 * for comparison path by path:
 *   steps     [count] Euler steps taken (the exiting step included)
 *   counts    [count][n_materials] steps whose end point lies in material m
 *   exit_xzt  [count][3] exit point x, z and hit fraction theta of the last step
 *   wall      [count] 0 left, 1 right, 2 top, 3 bottom, -1 truncated
 *   m_last    [count] material of the last point inside (receives theta dt)
 * Every output pointer may be NULL except steps. */
sdd_status sdd_walk_records(sdd_ctx *ctx, double x0, double z0, uint32_t node_id, uint32_t p0,
                            int32_t count, double dt, uint64_t seed, const sdd_config *cfg,
                            int64_t *steps, int64_t *counts, double *exit_xzt, int32_t *wall,
                            int32_t *m_last);

/* Per-path occupation records, for TE and TM models (a TM model's interface
 * hits split a step's time between two strips, Sec. 3.1; sdd_walk_records
 * rejects TM models with SDD_E_UNSUPPORTED):
 *   steps     [count] Euler steps taken (the exiting step included)
 *   occ       [count][n_materials] time spent in material m in units of dt,
 *             without the theta of the last step (TE: the step counts)
 *   exit_xzt, wall, m_last  as in sdd_walk_records
 *   hits      [count] interface randomisations (TM; 0 in TE)
 * Every output pointer may be NULL except steps. */
sdd_status sdd_walk_occupation(sdd_ctx *ctx, double x0, double z0, uint32_t node_id, uint32_t p0,
                               int32_t count, double dt, uint64_t seed, const sdd_config *cfg,
                               int64_t *steps, double *occ, double *exit_xzt, int32_t *wall,
                               int32_t *m_last, int64_t *hits);

/* Limits of sdd_interface_values_noalloc: nodes per call, work items per call
 * (the path chunks are widened until the items fit), and the size in bytes of
 * the scratch array the library keeps for it on every device that loads it. */
#define SDD_NOALLOC_MAX_NODES 4096
#define SDD_NOALLOC_MAX_ITEMS 8192
#define SDD_NOALLOC_SCRATCH_BYTES 8602112

/* The computation of sdd_interface_values_device, for callers that must not
 * allocate device memory -- hosts that hand out all device memory from their
 * own arena, processes whose memory another framework's caching allocator
 * already holds, loops that cannot afford the synchronisation of cudaMalloc
 * and cudaFree.  It calls no cudaMalloc, cudaFree or other allocating routine:
 * its per-call scratch (work items, partial sums, counters) is a fixed device
 * array of SDD_NOALLOC_SCRATCH_BYTES compiled into the library, which every
 * GPU that loads the library holds until the process exits; the context's own
 * scratch buffers are not used.  The paper has no counterpart: this is a
 * deployment variant of the same estimator.
 *   Arguments and outputs as sdd_interface_values_device (ctx from
 *   sdd_create; d_nodes_xz, d_node_ids, d_mean, d_se, d_counters device; n_paths
 *   host; stream a cudaStream_t or NULL), except that cfg->use_graph must be 0:
 *   this call launches its kernels directly.  n_paths is also read by an
 *   asynchronous copy queued on the stream: if it is page-locked memory, keep
 *   it unchanged until the stream has passed the call.
 *   Errors: SDD_E_ARG for more than SDD_NOALLOC_MAX_NODES nodes, a request whose
 *   work items cannot fit SDD_NOALLOC_MAX_ITEMS, or a context created on another
 *   device than the current one; SDD_E_UNSUPPORTED for cfg->use_graph != 0; the
 *   checks of sdd_interface_values_device.
 * The first call on a device looks up the array's device address (set-up); make
 * that first call before any stream capture.  The address is kept for the life
 * of the process: after cudaDeviceReset on a device, this entry point must not
 * be called on that device again.  All calls share the one array,
 * which keeps the last call's contents (each call clears what must start at
 * zero): calls that overlap on the GPU -- on two streams or from two host
 * threads -- race and must be ordered by the caller. */
sdd_status sdd_interface_values_noalloc(sdd_ctx *ctx, const double *d_nodes_xz,
                                        const uint32_t *d_node_ids, int32_t n_nodes,
                                        const int64_t *n_paths, double dt, uint64_t seed,
                                        const sdd_config *cfg, double *d_mean, double *d_se,
                                        uint64_t *d_counters, void *stream);

/* ------------------------------------------------------------------------
 * Asynchronous requests: the evaluation of sdd_interface_values (the Monte
 * Carlo estimator of Sec. 3.1 at every node), queued without waiting.
 *
 * sdd_interface_values_async copies its inputs (nodes_xz, node_ids nullable,
 * n_paths; host arrays, free to reuse on return), queues the walks, the
 * reduction and the download of the results on `stream` (a cudaStream_t; NULL
 * gives the request a stream of its own) and returns a request in *out.  The
 * request owns its device and page-locked host scratch, so a context may have
 * several requests in flight, submitted from several host threads.  Results
 * equal those of sdd_interface_values on the same inputs (the same plan and
 * walks), up to the FP64 summation order within a work item.
 *   sdd_poll      SDD_E_BUSY while running; then the request's status:
 *                 SDD_OK, SDD_E_TRUNCATED, SDD_E_CANCELLED or an error.
 *   sdd_wait      waits up to timeout_ms (< 0: no limit); SDD_E_TIMEOUT if
 *                 the request is still running then, else as sdd_poll.
 *   sdd_cancel    stops handing out walks: the walks already started end,
 *                 the rest are skipped, and the request ends with
 *                 SDD_E_CANCELLED (outputs undefined).  A request cancelled
 *                 while it still waits behind earlier work on its stream
 *                 keeps the cancel: it ends once the walks its warps take
 *                 before the flag arrives (one per lane at most) have ended.
 *                 Returns at once.
 *   sdd_request_result  copies mean [n_nodes][n_eval][2] and se (as
 *                 sdd_interface_values) and stats (nullable) once the request
 *                 has ended with SDD_OK or SDD_E_TRUNCATED; otherwise returns
 *                 its status (SDD_E_BUSY while running).
 *   sdd_request_free  waits for the request's GPU work, then frees it.
 * Errors at submission: those of sdd_interface_values; SDD_E_UNSUPPORTED for
 * cfg->use_graph != 0; SDD_E_ARG for a context of another device. */
sdd_status sdd_interface_values_async(sdd_ctx *ctx, const double *nodes_xz, const uint32_t *node_ids,
                                      int32_t n_nodes, const int64_t *n_paths, double dt, uint64_t seed,
                                      const sdd_config *cfg, void *stream, sdd_request **out);
sdd_status sdd_poll(sdd_request *req);
sdd_status sdd_wait(sdd_request *req, int64_t timeout_ms);
sdd_status sdd_cancel(sdd_request *req);
sdd_status sdd_request_result(sdd_request *req, double *mean, double *se, sdd_stats *stats);
void sdd_request_free(sdd_request *req);

/* ------------------------------------------------------------------------
 * Path ranges and their reduction: one evaluation split across processes.
 *
 * The walks of a node are independent, and so are the nodes (Sec. 5), so an
 * evaluation can be cut into ranges -- a node and a contiguous range of its
 * paths -- that different processes (one per GPU) evaluate.  A range's raw
 * sums are those of the Monte Carlo estimator of Sec. 3.1 over its walks,
 * which keep the Philox streams (node id, path) they have in a whole-node
 * call.  The node's mean and standard errors follow from the sums of its
 * ranges added in range order, so they do not depend on which process
 * evaluated which range.
 *
 * sdd_range_sums: range i is paths [path_begin[i], path_begin[i] +
 * path_count[i]) of the node at nodes_xz[i] (host, [n_ranges][2]) under RNG
 * node id node_ids[i] (host, nullable: i).  path_count[i] in 1..2^31-1,
 * path_begin[i] >= 0 and path_begin[i] + path_count[i] <= 2^32.  Outputs (host):
 *   sums    [n_ranges][n_eval][4]  sum re, sum im, sum re^2, sum im^2 of the
 *           samples g(exit) exp(-i (1/2) sum_m kappa_{e,m} T_m) of the walks
 *           that reached the boundary;
 *   n_valid [n_ranges]             those walks (truncated ones left out).
 * Errors: as sdd_interface_values; SDD_E_ARG for a range outside 0..2^32;
 * SDD_E_UNSUPPORTED for cfg->use_graph != 0.  Synchronous. */
sdd_status sdd_range_sums(sdd_ctx *ctx, const double *nodes_xz, const uint32_t *node_ids,
                          int32_t n_ranges, const int64_t *path_begin, const int64_t *path_count,
                          double dt, uint64_t seed, const sdd_config *cfg, double *sums,
                          int64_t *n_valid, sdd_stats *stats);

/* The same with device buffers, queued on stream (cudaStream_t or NULL):
 * d_nodes_xz [n_ranges][2], d_node_ids [n_ranges] (nullable), d_sums
 * [n_ranges][n_eval][4], d_n_valid [n_ranges], d_counters [3] (nullable:
 * steps, walks, truncated walks); path_begin and path_count are host arrays.
 * Like sdd_interface_values_device it uses the context's scratch buffers, as
 * do sdd_reduce_sums and sdd_reduce_sums_device: calls on one context must be
 * ordered on one stream. */
sdd_status sdd_range_sums_device(sdd_ctx *ctx, const double *d_nodes_xz, const uint32_t *d_node_ids,
                                 int32_t n_ranges, const int64_t *path_begin,
                                 const int64_t *path_count, double dt, uint64_t seed,
                                 const sdd_config *cfg, double *d_sums, int64_t *d_n_valid,
                                 uint64_t *d_counters, void *stream);

/* Mean and standard errors per node and evaluation from range sums:
 * range_node [n_ranges] (host) is the node 0..n_nodes-1 of each range,
 * nondecreasing; the sums of a node's ranges are added in range order, then
 * mean = sum / N and se = sqrt(unbiased variance / N) per component, N the
 * node's n_valid total (NaN where N = 0, and se NaN where N = 1).  sums and
 * n_valid are laid out as sdd_range_sums writes them; mean and se are
 * [n_nodes][n_eval][2].  ctx gives n_eval and the device; host buffers,
 * synchronous. */
sdd_status sdd_reduce_sums(sdd_ctx *ctx, int32_t n_nodes, int32_t n_ranges, const int32_t *range_node,
                           const double *sums, const int64_t *n_valid, double *mean, double *se);

/* The same on device buffers, queued on stream; range_node stays on the host. */
sdd_status sdd_reduce_sums_device(sdd_ctx *ctx, int32_t n_nodes, int32_t n_ranges,
                                  const int32_t *range_node, const double *d_sums,
                                  const int64_t *d_n_valid, double *d_mean, double *d_se,
                                  void *stream);

/* ------------------------------------------------------------------------
 * Interpolation along an interface (Sec. 5: the stochastic solution is
 * computed at some points of an interface only and the other interface
 * values are interpolated).  The paper names the idea and gives no scheme;
 * the one implemented here is:
 *  - the nodes of one interface are an ordered polyline p_0 .. p_{n-1} and
 *    the interpolation variable is its arc length s_i = sum_{k<i} |p_{k+1} - p_k|;
 *  - each real component (re and im of each evaluation) is interpolated on
 *    its own, piecewise linearly in s (SDD_INTERP_LINEAR) or by the natural
 *    cubic spline in s, second derivative zero at both end knots
 *    (SDD_INTERP_SPLINE);
 *  - both interpolants are linear in the knot values, v(s) = sum_j c_j(s) v_j,
 *    and the knots' estimates are independent, so the standard error given
 *    at s is sqrt(sum_j c_j(s)^2 se_j^2): the Monte Carlo part of the error,
 *    not the interpolation error.
 * Both entry points run on the current CUDA device in FP64, allocate their
 * own device scratch and return when the results are in the host arrays. */
#define SDD_INTERP_LINEAR 0
#define SDD_INTERP_SPLINE 1
#define SDD_INTERP_MAX_SPLINE_KNOTS 4096 /* the spline keeps an n x n FP64 table */
#define SDD_INTERP_MAX_NODES (1 << 20)

/* Interpolate knot data to target arc lengths.
 *   knots_s     host, [n_knots] strictly increasing, finite; n_knots >= 2
 *               (<= SDD_INTERP_MAX_SPLINE_KNOTS for the spline)
 *   values      host, [n_knots][n_vals] real components at the knots
 *   se          host, [n_knots][n_vals] their standard errors, or NULL
 *   targets_s   host, [n_targets] within [knots_s[0], knots_s[n_knots-1]]
 *   kind        SDD_INTERP_LINEAR or SDD_INTERP_SPLINE
 *   out_values  host out, [n_targets][n_vals]
 *   out_se      host out, [n_targets][n_vals], or NULL (written only when se
 *               is given)
 * A target belongs to the segment [s_i, s_{i+1}] with the largest i <= n-2
 * such that s_i <= target; a target on a knot gets that knot's value.
 * Errors: SDD_E_ARG (sizes, kind, knots not increasing, a target outside the
 * knot range, NULL arrays), SDD_E_CUDA.  n_targets == 0 does nothing. */
sdd_status sdd_interpolate(const double *knots_s, int32_t n_knots, const double *values,
                           const double *se, int32_t n_vals, const double *targets_s,
                           int32_t n_targets, int32_t kind, double *out_values, double *out_se);

/* Interface values at every node of an interface polyline from walks at every
 * stride-th node: the Monte Carlo nodes ("knots") are nodes 0, stride,
 * 2 stride, ... and always node n_nodes-1.  Each knot runs n_paths walks with
 * its index along the polyline as RNG node id, so its estimate equals the one
 * sdd_interface_values gives that node in a call on the whole polyline with
 * node ids 0 .. n_nodes-1; the other nodes get the interpolated values and
 * propagated standard errors described above.
 *   nodes_xz   host, [n_nodes][2] in interface order, 2 <= n_nodes <=
 *              SDD_INTERP_MAX_NODES, consecutive nodes distinct, each strictly
 *              inside the domain
 *   stride     >= 1 (1: every node runs walks)
 *   n_paths    walks per Monte Carlo node, 1 .. 2^31-1
 *   kind       SDD_INTERP_LINEAR or SDD_INTERP_SPLINE (at most
 *              SDD_INTERP_MAX_SPLINE_KNOTS knots)
 *   mean, se   host out, [n_nodes][n_eval][2], layouts as sdd_interface_values
 *   stats      host out, nullable: the walks of the knots
 *   dt, seed, cfg as sdd_interface_values.
 * Returns the status of the walks (SDD_OK or SDD_E_TRUNCATED) or an error. */
sdd_status sdd_interface_values_interp(sdd_ctx *ctx, const double *nodes_xz, int32_t n_nodes,
                                       int32_t stride, int64_t n_paths, int32_t kind, double dt,
                                       uint64_t seed, const sdd_config *cfg, double *mean,
                                       double *se, sdd_stats *stats);

/* ------------------------------------------------------------------------
 * Apparent resistivity and phase at measurement sites (Sec. 2.1: the
 * secondary fields H^x = -(1/(i omega mu)) dE^y/dz (TE) and
 * E^x = (1/sigma) dH^y/dz (TM), rho_a = |E/H|^2 / (omega mu) and
 * phi = arg(E/H) with E/H = E^y/H^x (TE) or E^x/H^y (TM); Sec. 4.2: the
 * solution at three points near the surface of each site, the z-derivative
 * by the centred difference).
 *
 * Site i = (x, z0) runs n_paths walks at (x, z0 - h), (x, z0), (x, z0 + h)
 * under node ids 3i, 3i+1, 3i+2.  With u the primary field there (E^y of a
 * TE model, H^y of a TM model), u_z = (u(z0 + h) - u(z0 - h)) / (2h), and
 * kappa_ref[e] = omega_e mu sigma_ref L^2 the rate a reference conductivity
 * sigma_ref would have in evaluation e, the library returns, in units of
 * rho_ref = 1/sigma_ref:
 *   TE  rho = kappa_ref |u / u_z|^2,        phi = arg(-i u / u_z)
 *   TM  rho = D^2 |u_z / u|^2 / kappa_ref,  phi = arg(u_z / u)
 * where D = sigma_ref / sigma is the diffusion of the strip holding x (a TM
 * model's D_m Lap u = i kappa u is the TM equation times sigma_ref / sigma_m
 * when kappa = omega mu sigma_ref L^2 in every strip).  A uniform half-space
 * gives rho = sigma_ref / sigma and phi = 45 degrees (TE) or -135 degrees
 * (TM); phases are in radians in (-pi, pi].
 * Standard errors are first order in the six real inputs (re and im of the
 * three points, taken as independent).
 *   sites_xz   host, [n_sites][2]; every point strictly inside the domain
 *   h          > 0, the centred-difference half step
 *   n_paths    walks per point, 1 .. 2^31-1
 *   kappa_ref  host, [n_eval], finite and > 0
 *   rho, phase host out, [n_sites][n_eval]
 *   rho_se, phase_se  host out, [n_sites][n_eval], nullable
 *   u0, uz     host out, [n_sites][n_eval][2] (re, im): the primary field at
 *              the site and its centred z-derivative (dimensionless), nullable
 *   stats      host out, nullable: the walks of all 3 n_sites points
 *   dt, seed, cfg as sdd_interface_values.
 * Returns the status of the walks (SDD_OK or SDD_E_TRUNCATED) or an error.
 * Runs on the current device; host arrays in and out. */
#define SDD_MT_MAX_SITES (1 << 20)
sdd_status sdd_apparent_resistivity(sdd_ctx *ctx, const double *sites_xz, int32_t n_sites, double h,
                                    int64_t n_paths, const double *kappa_ref, double dt,
                                    uint64_t seed, const sdd_config *cfg, double *rho, double *phase,
                                    double *rho_se, double *phase_se, double *u0, double *uz,
                                    sdd_stats *stats);

/* The arithmetic of sdd_apparent_resistivity on given three-point values:
 *   values, se  host, [n_sites][3][n_eval][2]: estimates (re, im) and their
 *               standard errors at (x, z0 - h), (x, z0), (x, z0 + h)
 *   d_site      host, [n_sites] diffusion of each site's strip (TM), or NULL (TE)
 *   h, kappa_ref, rho, phase, rho_se, phase_se, u0, uz as sdd_apparent_resistivity.
 * Errors: SDD_E_ARG, SDD_E_CUDA. */
sdd_status sdd_apparent_from_values(const double *values, const double *se, int32_t n_sites,
                                    int32_t n_eval, double h, const double *kappa_ref,
                                    const double *d_site, double *rho, double *phase,
                                    double *rho_se, double *phase_se, double *u0, double *uz);

/* ------------------------------------------------------------------------
 * RBF-FD sub-domain solve (Sec. 3.2).  Once the interface values are known,
 * a sub-domain of constant rate kappa (TE: Lap u = i kappa u; a TM strip of
 * diffusion D: the same with kappa / D) is solved on its own nodes by
 * radial-basis-function finite differences:
 *  - the stencil of a node is the node and its n_stencil - 1 nearest nodes
 *    (by squared distance dx*dx + dz*dz, ties to the lower index);
 *  - the weights of the Laplacian at node x_0 solve A w = b, A_ij =
 *    phi(|x_i - x_j|) over the stencil, b_j = Lap phi(|x - x_j|) at x_0, with
 *    the multiquadric phi(r) = sqrt(1 + (eps r)^2), so
 *    Lap phi = (2 eps^2 + eps^4 r^2) / phi^3 (the paper builds d^2/dx^2 and
 *    d^2/dz^2 separately; their sum has these weights);
 *  - every non-Dirichlet node i gets sum_j w_ij u_j - i kappa_i u_i = 0, the
 *    Dirichlet nodes' terms on the right-hand side, and the system is solved
 *    by BiCGStab with a Jacobi preconditioner to |b - K x| <= tol |b|.
 * The paper uses n_stencil = 9 and eps = 1/2000 per metre with 100-125 m
 * spacing (eps h about 0.05).  FP64 on the current device; host arrays. */
#define SDD_RBFFD_MAX_NODES (1 << 18) /* the neighbour search scans all nodes */
#define SDD_RBFFD_MAX_STENCIL 16

typedef struct {
    int32_t unknowns;     /* non-Dirichlet nodes */
    int32_t iterations;   /* BiCGStab iterations */
    double rel_residual;  /* |b - K x| / |b| of the returned solution */
    double knn_ms;        /* device time of the neighbour search */
    double weights_ms;    /* device time of the weights */
    double solve_ms;      /* device time of assembly and BiCGStab (with its polls) */
} sdd_rbffd_stats;

/* Stencils and Laplacian weights of every node.
 *   nodes_xz   host, [n][2] finite, distinct; n_stencil <= n <= SDD_RBFFD_MAX_NODES
 *   n_stencil  2 .. SDD_RBFFD_MAX_STENCIL (9 in the paper)
 *   eps        shape parameter, > 0
 *   stencil    host out, [n][n_stencil] node indices, the node itself first
 *   weights    host out, [n][n_stencil]
 * Errors: SDD_E_ARG (sizes, eps, non-finite nodes, a singular stencil
 * matrix from coincident nodes), SDD_E_CUDA. */
sdd_status sdd_rbffd_weights(const double *nodes_xz, int32_t n, int32_t n_stencil, double eps,
                             int32_t *stencil, double *weights);

/* Sub-domain solution.
 *   dirichlet  host, [n] 1 = value given (interface or outer boundary), 0 = unknown
 *   values     host, [n][2] (re, im), read at Dirichlet nodes
 *   kappa      host, [n] rate of the equation at each node
 *   tol        relative residual to reach, > 0; max_iter >= 1
 *   u          host out, [n][2]: the values at Dirichlet nodes, the solution
 *              elsewhere (the last iterate when not converged)
 *   stats      host out, nullable
 * Errors: SDD_E_ARG, SDD_E_CUDA; SDD_E_TIMEOUT when BiCGStab did not reach
 * tol within max_iter or broke down (u and stats are still written). */
sdd_status sdd_rbffd_solve(const double *nodes_xz, int32_t n, const uint8_t *dirichlet,
                           const double *values, const double *kappa, int32_t n_stencil, double eps,
                           double tol, int32_t max_iter, double *u, sdd_rbffd_stats *stats);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.
 *
 * A server evaluates requests -- one raster model and its interface nodes
 * each -- on one device.  Requests are admitted while a slot (and, with
 * max_bytes, device memory) is free.  Each phase of a request (its pilot or
 * fixed-count walks, then the top-up walks sized from the pilot) is cut
 * into pieces of whole nodes of at most max_batch_walks walks; a worker
 * thread packs queued pieces, first in first out, into launches of the
 * persistent walk kernel over many models, with up to n_streams launches in
 * flight, so new requests start while earlier ones are still on the GPU and
 * the tail of one launch overlaps the next.
 * Every walk uses the server's seed and the request's node ids as Philox
 * stream, so a request's result does not depend on what it was batched with
 * (up to FP64 summation order).  All requests must match the server's
 * domain, raster size, n_eval and g_kind.
 * ---------------------------------------------------------------------- */
typedef struct sdd_server sdd_server;

typedef struct {
    sdd_domain domain;        /* every request's domain */
    int32_t nx, nz;           /* every request's raster size (limits as in sdd_model_desc) */
    int32_t n_eval;           /* every request's number of evaluations */
    int32_t g_kind;           /* every request's boundary-data kind */
    int32_t max_requests;     /* admission slots: admitted and not yet collected, 1..4096 */
    int64_t max_bytes;        /* device bytes admitted requests may hold; 0 = slots only */
    int32_t n_streams;        /* batched launches in flight at once, 1..8 */
    int32_t max_batch_models; /* requests per launch, 1..256 */
    int64_t max_batch_walks;  /* walks per launch; a request's phase is cut into pieces
                                 of whole nodes to fit; 0 = 2^24 */
    double dt;                /* Euler time step of every walk */
    uint64_t seed;            /* Philox key of every walk */
    sdd_config launch;        /* launch options; precision must be SDD_FP32 */
} sdd_server_config;

typedef struct {
    const sdd_model_desc *model; /* raster model, copied at submission */
    const double *nodes_xz;      /* host, [n_nodes][2], copied */
    const uint32_t *node_ids;    /* host, [n_nodes] or NULL for 0..n_nodes-1, copied */
    int32_t n_nodes;             /* 1..65536 */
    const int64_t *n_paths;      /* host, [n_nodes] fixed walk counts, or NULL for ... */
    double target_se;            /* ... adaptive counts at this complex standard error */
    int64_t n_pilot, n_max;      /* adaptive: pilot walks and cap per node */
} sdd_request_desc;

typedef struct {
    double queue_us;    /* submission to its first launch */
    double latency_us;  /* submission to completion */
    uint64_t walks;     /* walks run for the request */
    uint64_t truncated; /* of which reached max_steps */
    int32_t launches;   /* batched launches the request took part in */
    int32_t status;     /* SDD_OK, SDD_E_TRUNCATED, SDD_E_CANCELLED or an error */
} sdd_request_stats;

typedef struct {
    uint64_t submitted, refused, completed, cancelled;
    uint64_t launches;          /* batched launches */
    uint64_t steps, walks;      /* Euler steps and walks of all launches */
    double gpu_busy_ms;         /* sum of the launches' walk-kernel times */
    int32_t in_flight;          /* admitted, not yet collected */
    int64_t bytes_in_use;       /* device bytes held by admitted requests */
} sdd_server_stats;

/* Create a server on the current device: worker thread, n_streams streams,
 * an arena of max_requests material maps (two-level tile form, at most
 * about nx x nz + nx x nz / 64 bytes each) and per-stream scratch.
 * Errors: SDD_E_ARG, SDD_E_OOM, SDD_E_CUDA. */
sdd_status sdd_server_create(const sdd_server_config *cfg, sdd_server **out);

/* Stop the worker (running launches finish first) and free everything;
 * requests not collected are discarded.  NULL is allowed. */
void sdd_server_destroy(sdd_server *srv);

/* Admit a request; *id identifies it.  SDD_E_BUSY when no slot or not enough
 * of max_bytes is free (nothing is kept; retry later), SDD_E_ARG when the
 * request does not match the server or is malformed. */
sdd_status sdd_server_submit(sdd_server *srv, const sdd_request_desc *req, uint64_t *id);

/* *done = 1 once the request has finished (or was cancelled). */
sdd_status sdd_server_poll(sdd_server *srv, uint64_t id, int32_t *done);

/* Block until the request finishes or timeout_ms passes (< 0: no limit);
 * SDD_E_TIMEOUT if it did not finish in time. */
sdd_status sdd_server_wait(sdd_server *srv, uint64_t id, int64_t timeout_ms);

/* Copy a finished request's results and free its slot: mean and se
 * [n_nodes][n_eval][2], n_used [n_nodes] (nullable), stats (nullable).
 * Returns the request's status (SDD_OK, SDD_E_TRUNCATED, SDD_E_CANCELLED, ...);
 * SDD_E_BUSY if it has not finished; SDD_E_ARG for an unknown id. */
sdd_status sdd_server_result(sdd_server *srv, uint64_t id, double *mean, double *se,
                             int64_t *n_used, sdd_request_stats *stats);

/* Cancel a request: if it is not on the GPU it ends at once, otherwise when
 * its launch ends; its results are then discarded.  Collect it with
 * sdd_server_result to free its slot. */
sdd_status sdd_server_cancel(sdd_server *srv, uint64_t id);

/* Counters of the server since its creation. */
sdd_status sdd_server_get_stats(sdd_server *srv, sdd_server_stats *out);

/* Number of evaluations and materials of the context's model. */
int32_t sdd_n_eval(const sdd_ctx *ctx);
int32_t sdd_n_materials(const sdd_ctx *ctx);

/* Material-lookup programs of the single-precision walk: how the occupation
 * update of Sec. 3.1 (the step's time to the material of the new point)
 * finds the material.  The one-shape programs count steps by region (earth
 * side of the surface, inside the shape) and form the material counts at the
 * walk's exit; they are chosen only for a shape wholly on one side of z = 0. */
#define SDD_PROGRAM_LAYERS 0    /* layered background (air z < 0, earth z >= 0) only */
#define SDD_PROGRAM_RECT 1      /* one rectangle on one side of the surface */
#define SDD_PROGRAM_TRIANGLE 2  /* one triangle on one side of the surface */
#define SDD_PROGRAM_SHAPES4 3   /* up to 4 shapes, or one shape across the surface */
#define SDD_PROGRAM_SHAPES16 4  /* up to 16 shapes */
#define SDD_PROGRAM_RASTER 5    /* int8 raster through its tile map */
#define SDD_PROGRAM_CONTACT 6   /* one rectangle that is the earth right of x0 (vertical contact) */
#define SDD_PROGRAM_TM 8        /* TM walk over vertical strips */

/* The lookup program sdd_create would give a model, decided on the host by
 * the same code; no CUDA call and no allocation, so it works without a GPU.
 *   model: as for sdd_create (read only, not kept).
 *   *program: one of SDD_PROGRAM_*.
 *   *shape_side (nullable): for SDD_PROGRAM_RECT, _TRIANGLE and _CONTACT 0 when
 *   the shape lies in the earth and 1 when it lies in the air; -1 otherwise.
 * Errors: SDD_E_ARG for a NULL model or program, and every model check of
 * sdd_create. */
sdd_status sdd_model_program(const sdd_model_desc *model, int32_t *program, int32_t *shape_side);

/* The work items one evaluation is cut into, as a launch with `warps`
 * resident warps cuts them (node values are independent, Sec. 5, so every
 * node's paths are split into (node, path range) items that the warps take
 * from one queue); host only, no CUDA call.
 *   n_paths [n_nodes] host; warps >= 1; guided_factor >= 1 (guided items of
 *   about 1 / (guided_factor x warps) of the paths not yet cut, multiples of
 *   32 shrinking toward the end of the queue) used when chunk_paths == 0,
 *   else fixed items of chunk_paths paths, node by node.
 *   node, path0, count [max_items] host, written in queue order; *n_items
 *   the number of items.
 * Errors: SDD_E_ARG for n_nodes < 0, a negative path count, warps < 1,
 * guided_factor < 1, chunk_paths < 0, a NULL pointer, or a plan of more than
 * max_items items (*n_items then holds the number needed). */
sdd_status sdd_plan_items(int32_t n_nodes, const int64_t *n_paths, int32_t warps, int32_t guided_factor,
                          int32_t chunk_paths, int32_t max_items, int32_t *node, uint32_t *path0,
                          int32_t *count, int32_t *n_items);

/* Static description of a status; never NULL. */
const char *sdd_status_str(sdd_status s);

/* Message of the last error raised on this host thread ("" if none). */
const char *sdd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SDD_H */
