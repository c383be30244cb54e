/*
 * abd.h -- C ABI of the GB300 (sm_103a) implementation of distributed Affine
 * Body Dynamics with consensus ADMM ("Distributed Affine Body Dynamics with
 * Adaptive Consensus", SIGGRAPH 2026).
 *
 * One time step (abd_step) is: the implicit-Euler incremental potential of
 * affine bodies (Sec. 3, Eq. 1) split over spatial slab partitions (Sec. 4,
 * Fig. 2), each partition minimising its replica-weighted local objective
 * (Eq. 3) plus the consensus penalty (Eq. 5) by projected Newton with
 * CCD-filtered backtracking; then the consensus average (Eq. 6), the dual
 * update (Eq. 7), the stopping metrics (Eq. 8-10), the CCD-certified merge
 * (Sec. 4.2) and the mass-aware, residual-driven penalty (Sec. 4.3).  Every
 * partition of every scene runs on the one GPU the library was created on; no
 * call communicates across GPUs.
 *
 * Conventions
 *   - q of one body: 12 doubles (p0,p1,p2, A00,A01,A02, A10,A11,A12, A20,A21,A22);
 *     world position x = A * xbar + p, A row-major.  At creation the rest
 *     vertices of every dynamic body are recentred at its centre of mass and p
 *     is shifted so that world positions are unchanged; abd_state_get/set use
 *     that centred convention.
 *   - Body kinds: ABD_DYNAMIC (12 DoFs), ABD_STATIC (fixed collider),
 *     ABD_KINEMATIC (prescribed motion: still 12 DoFs of the solve, but its
 *     predicted state is its prescribed pose -- p moved by its linear velocity,
 *     A rotated by R(omega h) about its centre of mass, no gravity -- and its
 *     inertia carries a weight of 1e6, so contacts cannot move it measurably off
 *     the prescription; abd_body_props reports the weighted mass and moment).
 *   - Ground planes are axis-aligned: distance = sign * x[axis] - offset.
 *   - All pointers in the descriptors are HOST pointers owned by the caller;
 *     the library copies what it needs before returning.
 *   - Return values: 0 = ABD_OK; > 0 warnings; < 0 errors (no exceptions cross
 *     the ABI).  abd_last_error() gives the text of the last error of a scene.
 *   - A scene handle is not thread-safe: use one host thread per scene.
 */
#ifndef ABD_H
#define ABD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ABD_DYNAMIC = 0, ABD_STATIC = 1, ABD_KINEMATIC = 2 };
enum { ABD_FP64 = 0, ABD_MIXED = 1 };
enum { ABD_RHO_FIXED = 0, ABD_RHO_ADAPTIVE = 1 };

enum {
    ABD_OK = 0,
    ABD_ADMM_MAXITER = 1,       /* K ADMM rounds without convergence; merge check passed, z accepted */
    ABD_NEWTON_MAXITER = 2,     /* some local solve hit max_newton */
    ABD_FELL_BACK_MONOLITHIC = 3, /* K rounds and the merge check failed: step re-solved on one partition */
    ABD_DT_SPLIT = 4,           /* a blocked merge was retaken as two steps of h/2 (dt_split_max > 0) */
    ABD_E_INVALID = -1,
    ABD_E_OOM = -2,
    ABD_E_CUDA = -3,
    ABD_E_PAIR_OVERFLOW = -4,
    ABD_E_DEVICE_TIMEOUT = -5,
    ABD_E_PENETRATION = -6,     /* the step ended with a pair at distance <= 0 */
    ABD_E_UNSUPPORTED = -7
};

typedef struct abd_scene abd_scene;

/* Scene description (meshes, bodies, ground planes).  Arrays are host memory. */
typedef struct {
    int32_t n_meshes;
    const int32_t *mesh_n_verts;   /* [n_meshes] */
    const int32_t *mesh_n_tris;    /* [n_meshes] */
    const double *mesh_xbar;       /* [sum verts][3] rest positions, mesh frame */
    const int32_t *mesh_tris;      /* [sum tris][3] mesh-local vertex indices, closed and outward for dynamic bodies */
    int32_t n_bodies;
    const int32_t *body_mesh;      /* [B] */
    const double *body_density;    /* [B] kg/m^3 (dynamic bodies) */
    const double *body_kappa;      /* [B] orthogonality stiffness kappa of kappa V ||A A^T - I||_F^2 */
    const int32_t *body_kind;      /* [B] ABD_DYNAMIC, ABD_STATIC or ABD_KINEMATIC */
    const double *body_q0;         /* [B][12] initial q in the mesh frame */
    const double *body_v0;         /* [B][12] initial qdot, or NULL for zero */
    const double *body_omega;      /* [B][3] angular velocity of ABD_KINEMATIC bodies about their centre of
                                      mass (world frame, rad/s), or NULL; their linear velocity is
                                      body_v0[0..3] */
    int32_t n_planes;              /* <= 8 */
    const int32_t *plane_axis;     /* [n_planes] 0, 1 or 2 */
    const double *plane_sign;      /* [n_planes] +1 or -1 */
    const double *plane_offset;    /* [n_planes] */
    double gravity[3];
} abd_scene_desc;

/* Slab partition (Sec. 4, Fig. 2): n_slabs slabs along `axis` separated by the
 * planes gamma_1..gamma_{n_slabs-1} (NULL: equal widths over the dynamic
 * bodies' extent at the start of each step).  Overlap width
 * w = max(alpha * v_max * h, w_min), w_min <= 0 meaning the smallest dynamic
 * body AABB diagonal.  A body is replicated on every slab whose range widened
 * by w/2 meets its AABB; membership is recomputed at the start of every step. */
typedef struct {
    int32_t axis;
    int32_t n_slabs;               /* 1..64 */
    const double *planes;          /* [n_slabs - 1] or NULL */
    double alpha;                  /* 2 in the paper */
    double w_min;
    /* Control-based load balancing (Sec. 5.2):
     * after every step each plane between slabs i and i+1 moves by
     * -(pd_kp T + pd_kd (T - T_prev)) along the axis, T = (tau_i - tau_{i+1}) /
     * (tau_i + tau_{i+1}) from the smoothed work tau of the two slabs, so the
     * slower slab shrinks (abd_pd_update).  Work of a slab in a step = its Newton
     * iterations x its slots (its partitions share every launch on this GPU,
     * so they have no separate clocks).  Smoothing tau <- pd_smooth tau_prev +
     * (1 - pd_smooth) tau_step.  pd_kp = pd_kd = 0: planes fixed (default). */
    double pd_kp, pd_kd, pd_smooth;
} abd_partition_desc;

/* Step parameters.  Defaults: abd_step_params_default(). */
typedef struct {
    double h;                      /* time step (s) */
    double dhat;                   /* barrier activation distance (m) */
    double kappa_barrier;          /* barrier stiffness; <= 0: 10 * mean dynamic mass * |g| / dhat */
    int32_t precision;             /* ABD_FP64 or ABD_MIXED (FP32 assembly and PCG, FP64 CCD/energies/residuals) */
    int32_t rho_mode;              /* ABD_RHO_FIXED or ABD_RHO_ADAPTIVE */
    double beta, tau, mu, sigma_min, sigma_max; /* Sec. 4.3: 1, 2, 5, 1e-3, 1e3 */
    double theta;                  /* Eq. 8 threshold */
    double newton_tol;             /* |dq|_inf / (h l) < newton_tol ends a local solve */
    int32_t max_admm, max_newton, max_halvings;
    double pcg_rtol;               /* PCG stop: FP64, |r|_2 <= pcg_rtol |r_0|_2; mixed, the block-Jacobi
                                      preconditioned residual z = P r (in the units of q, body by body)
                                      |z|_inf <= pcg_rtol |z_0|_inf */
    int32_t pcg_max;
    double accd_s, accd_c;         /* additive CCD gap fraction and step factor */
    int32_t dt_split_max;          /* adaptive time stepping (Sec. 4.2, Fig. 4): when the merge check
                                      blocks after K rounds, retake the step from the same state as two
                                      steps of h/2, recursively up to this depth, before the one-partition
                                      fallback; 0 (default) disables it; at most 16 */
    int32_t mixed_fp64_first;      /* ABD_MIXED only: 1 (default) takes the first Newton iteration of every
                                      local solve with FP64 assembly and PCG, the later ones in FP32 -- the
                                      first step is the long one, and an FP32 Hessian's rounding can steer
                                      its line search into another local minimum of the non-convex
                                      contact energy; 0: every iteration in FP32 */
} abd_step_params;

typedef struct {
    int32_t status;
    int32_t admm_iters;            /* local-solve rounds */
    int32_t newton_iters;          /* Newton iterations summed over partitions and rounds */
    int32_t n_partitions, n_shared, n_slots;
    int64_t pcg_iters;             /* PCG iterations summed over Newton iterations */
    int64_t n_candidates_peak, n_active_peak;
    double r_inf, s_inf, delta_inf, min_distance, l, kappa_barrier, w;
    /* host wall clock split after Table 1's columns: t_solve_ms = the local
     * Newton solves, including their broad phase, narrow phase and CCD, which
     * run inside each Newton iteration (and its CUDA graph); t_coll_ms is
     * therefore 0 (abd_kernel_stats splits device time by kernel instead);
     * t_sync_ms = consensus, residuals and the merge check; t_total_ms =
     * the whole step */
    double t_solve_ms, t_coll_ms, t_sync_ms, t_total_ms;
    int64_t kernel_launches;       /* kernels of this library launched by the step */
    int32_t pcg_cluster;           /* largest thread-block cluster size of the step's PCG launches */
    int32_t pcg_unstaged;          /* 1: some PCG CTA read off-diagonal entries that did not fit in its
                                      shared memory from the owners' shared memory directly */
    int32_t list_redo;             /* Newton iterations redone because a pair list outgrew its buffer
                                      (the buffer is grown and the iteration repeated from its start) */
    int32_t reserved0;
} abd_step_stats;

/* --- scene ---------------------------------------------------------------- */

/* Copy the description to the device and compute per-body constants (mass,
 * second moment, volume, edges).  The affine degrees of freedom q = (p, A),
 * x = A xbar + p, and the mass matrix of each body follow Sec. 3 (the
 * affine-body setting of Eq. 1, whose inertia term uses M): mass and second
 * moment are integrated over the closed mesh, and the rest vertices are
 * recentred at the centre of mass so that M = diag(m I3, S, S, S) in q order.
 * `cuda_stream` is a cudaStream_t (NULL: the
 * legacy default stream) on which every later call on this scene enqueues
 * work; the current CUDA device becomes the scene's device.
 * Errors: ABD_E_INVALID (bad indices, open or inverted dynamic or kinematic
 * mesh, more than 8 planes, unknown kind), ABD_E_OOM, ABD_E_CUDA. */
int abd_scene_create(const abd_scene_desc *desc, void *cuda_stream, abd_scene **out);
void abd_scene_destroy(abd_scene *s);

/* counts[0..3] = bodies, vertices, triangles, edges (edges are the unique
 * undirected triangle edges, sorted by (min, max) mesh vertex index). */
int abd_scene_counts(const abd_scene *s, int64_t counts[4]);

/* Mass m, centre of mass (mesh frame), second moment S (row-major 3x3) and
 * volume of body b (ABD mass matrix M = diag(m I3, S, S, S) in q order). */
int abd_body_props(const abd_scene *s, int32_t b, double *m, double com[3], double S[9], double *V);

/* Set the slab partition used by later steps (default: one slab). */
int abd_partition(abd_scene *s, const abd_partition_desc *desc);

/* Body membership of the partition computed at the current state with the
 * given step size (bit i of mask[b] set = body b replicated on slab i); w_out
 * receives the overlap width. Host buffers. */
int abd_partition_masks(abd_scene *s, double h, uint64_t *mask, double *w_out);

/* Advance one time step of p->h (Eq. 1 by consensus ADMM over the current
 * partition, Eq. 5-10).  Blocks until the step is complete.  Returns a
 * status: 0, a positive warning (the step was taken) or a negative error
 * (the step did not complete; abd_last_error describes it).  With
 * p->dt_split_max > 0, a step whose merge check fails after K rounds is
 * retaken from its start state as two steps of h/2 (each with
 * dt_split_max - 1) and returns ABD_DT_SPLIT;
 * stats then sum the ADMM rounds and Newton iterations of every attempt and
 * report the second half step's residuals and minimum distance.  A scene
 * whose bodies are all static has no unknowns: the step returns 0 at once
 * (one ADMM round, no Newton iteration) and changes no state.
 * ABD_E_PENETRATION: the state after the step has a contact pair or a
 * vertex-plane pair at distance <= 0 (stats->min_distance); the state is
 * kept as computed, so the caller can inspect or restore it. */
int abd_step(abd_scene *s, const abd_step_params *p, abd_step_stats *stats);

/* Level-1 broad phase (overlapping slot pairs) of later steps: mode 0 (the
 * default) uses a spatial hash when some partition holds at least 1024 slots
 * and otherwise tests every pair within each partition; 1 always tests
 * every pair within each partition; 2 always uses the hash (a uniform grid of
 * cells 1.01 x the largest slot box, counting-sorted into buckets, at most
 * 27 cells visited per slot).  Both give the same pair set (the broad phase
 * of Sec. 6's candidate pairs, whose method the paper leaves open).
 * ABD_E_INVALID for another mode. */
int abd_scene_broadphase(abd_scene *s, int32_t mode);

/* Initial capacity, in pair records, of the scene's device pair lists
 * (candidates, active pairs, line-search pairs; the cluster-pair list gets
 * four times as many).  Lists grow by themselves when a count exceeds its
 * buffer (the Newton iteration is then redone, abd_step_stats.list_redo), so
 * this only trades memory against redone iterations; values below 16 are
 * raised to 16.  The library's own service, not a step of the method.
 * ABD_E_INVALID for pairs < 0. */
int abd_scene_reserve(abd_scene *s, int64_t pairs);

/* Host copies of the state (q, qdot), [B][12] each; either may be NULL.  This
 * is the state at the end of a frame of Alg. 1: shared bodies at their
 * consensus z, internal bodies at their only replica, and the velocity
 * qdot = (q^{t+1} - q^t) / h of the merge.  Arrays are caller-owned host
 * memory of n_bodies rows (ABD_E_INVALID when n_bodies differs from the
 * scene's body count); abd_state_set copies the caller's arrays to the device
 * and takes effect at the next step. */
int abd_state_get(const abd_scene *s, double *q, double *v, int64_t n_bodies);
int abd_state_set(abd_scene *s, const double *q, const double *v, int64_t n_bodies);

/* Device pointers of the resident state ([B][12] doubles each), valid until
 * the scene is destroyed; writes through them take effect at the next step. */
int abd_state_device(abd_scene *s, double **q, double **v);

/* Broad phase on caller-given vertex positions (host [V][3] doubles, global
 * vertex order; x1 NULL for the static set, else the set swept from x0 to
 * x1), one slab, inflation dhat/2 per side: writes up to `cap` triples
 * (type 0 = point-triangle (vertex, triangle), 1 = edge-edge (i < j)) in
 * unspecified order to `out` (host) and the total count to n_out. */
int abd_candidates(abd_scene *s, const double *x0, const double *x1, double dhat, int32_t *out, int64_t cap,
                   int64_t *n_out);

/* The same query as abd_candidates without allocating device memory, for
 * callers that must not call cudaMalloc/cudaFree themselves or through this
 * library (a plugin inside a framework whose allocator owns the GPU's memory
 * budget; latency-critical loops that cannot absorb the device-wide
 * synchronisation an allocation may cause).  The paper has no counterpart:
 * this is a service of this library, not a step of the method.
 *   x0, x1: DEVICE pointers, [V][3] doubles in global vertex order (x1 NULL:
 *           static set); out: DEVICE pointer to `cap` int32 triples (type, i, j)
 *           as in abd_candidates; n_out: host pointer, total count (entries
 *           beyond cap are counted, not written).  Inputs and outputs stay the
 *           caller's.
 *   Intermediates live in one 32 MiB array of static device memory, held by
 *   every GPU on which the library is loaded until the process exits.  The
 *   first call on a device looks up that array's address; make that first call
 *   before any stream capture on the device.  All calls share the array: calls
 *   whose work overlaps on the GPU (other host threads, other streams) race.
 *   Limits: at most 131072 bodies (ABD_E_INVALID beyond) and
 *   (32 MiB - 64 B x bodies - about 1.5 KiB of headers) / 8 overlapping body
 *   pairs (ABD_E_PAIR_OVERFLOW beyond): about 4.19 million for small scenes,
 *   3.1 million at the body limit; each error comes with a message in
 *   abd_last_error().  When more than `cap` candidates exist, the first `cap`
 *   found are written, *n_out receives the full count and the call returns
 *   ABD_OK.  Blocks until done. */
int abd_candidates_noalloc(abd_scene *s, const double *x0, const double *x1, double dhat, int32_t *out, int64_t cap,
                           int64_t *n_out);

/* Slab planes the next step will use (the explicit or load-balanced planes,
 * else the equal-width planes of the last step): up to `cap` values into
 * `planes`, the count (n_slabs - 1) in *n. */
int abd_partition_planes(const abd_scene *s, double *planes, int32_t cap, int32_t *n);

/* The load-balancing law alone (pure host function, no device work): for the
 * n_slabs - 1 planes, T[i] = (tau[i] - tau[i+1]) / (tau[i] + tau[i+1]) (0 when
 * both are 0) and delta[i] = -(kp T[i] + kd (T[i] - T_prev[i])), the plane
 * shift along the axis.  T_prev may be NULL (zeros). */
int abd_pd_update(int32_t n_slabs, const double *tau, const double *T_prev, double kp, double kd, double *delta,
                  double *T);

/* ---------------------------------------------------------------------------
 * Batched world: n independent scenes (uneven subdomains) in one scene
 * object.  Each scene becomes one partition; every phase of every scene's
 * Newton iteration (broad phase, assembly, PCG, CCD, line search) runs in the
 * same kernel launches, each partition converging on its own (its local solve
 * is Eq. 5 without shared bodies), and the steady-state iteration is replayed
 * as one CUDA graph.  Each scene keeps its own scale l (Eq. 8) and default
 * barrier stiffness, its static bodies collide only with its own bodies, and
 * scenes never collide with one another, so each scene's step is the one it
 * takes alone (up to the order of floating-point sums).  The paper solves one
 * scene; this packing is this library's batching of many.
 *   descs: n scene descriptions (host, copied); all must have the same ground
 *          planes and gravity (ABD_E_INVALID otherwise); n <= 256.
 *   Bodies are concatenated in scene order: abd_state_get/set and
 *   abd_body_props index the concatenation; abd_batch_layout gives each
 *   scene's first body.  abd_partition is rejected (the scenes are the
 *   partitions).  abd_candidates on a batched world treats the caller's
 *   positions as one scene. */
int abd_scene_create_batch(const abd_scene_desc *descs, int32_t n, void *cuda_stream, abd_scene **out);

/* Body offsets of the scenes of a batched world: body_off[0..n] (up to cap
 * values, host), *n = number of scenes (1 and [0, B] for an ordinary scene). */
int abd_batch_layout(const abd_scene *s, int64_t *body_off, int32_t cap, int32_t *n);

/* Newton iterations of each partition (each scene of a batched world) summed
 * over the ADMM rounds of the last step: up to cap values into iters (host),
 * the partition count in *n. */
int abd_partition_newton(const abd_scene *s, int32_t *iters, int32_t cap, int32_t *n);

/* Membership of partition `part` as the last abd_step built it (Sec. 4: a
 * dynamic body belongs to every slab its w-inflated box meets).  `bodies`
 * receives up to `cap` body indices of the partition and `shared` up to
 * `cap_shared` indices of those that also belong to another partition (the
 * replicated bodies B_ij); *n and *n_shared receive the full counts.  Either
 * array may be NULL to query counts.  ABD_E_INVALID for a partition index out
 * of range or before the first step. */
int abd_partition_get(const abd_scene *s, int32_t part, int32_t *bodies, int32_t cap, int32_t *n, int32_t *shared,
                      int32_t cap_shared, int32_t *n_shared);

/* ---------------------------------------------------------------------------
 * Serving: many independent scenes on one GPU.  The paper solves one scene;
 * this runtime has no counterpart there.  A server owns `n_streams` worker
 * threads, each with its own CUDA stream.  A submitted request (a scene, its
 * partition, step parameters and a number of steps) waits in FIFO order until
 * its estimated device memory fits the HBM budget; a free worker then creates
 * the scene on its stream, advances it `n_steps` steps with q, v, z, u and the
 * contact lists resident on the device, copies the final state to host memory
 * owned by the server and frees the scene.  Requests on different workers
 * overlap on the device, and a request admitted while others run starts as
 * soon as a worker and memory are free (continuous batching).  Each request's
 * arithmetic is that of abd_step on its own scene, so its result does not
 * depend on what else runs.
 * ------------------------------------------------------------------------- */
typedef struct abd_server abd_server;

typedef struct {
    int32_t device;           /* CUDA device of every scene */
    int32_t n_streams;        /* worker threads = concurrent scenes (>= 1) */
    int64_t hbm_budget_bytes; /* admission budget; 0: 80% of the free device memory at create */
} abd_server_desc;

enum { ABD_REQ_QUEUED = 0, ABD_REQ_RUNNING = 1, ABD_REQ_DONE = 2 };

typedef struct {
    int32_t state;         /* ABD_REQ_* */
    int32_t status;        /* worst step status (0 OK, > 0 warning, < 0 error; an error ends the request) */
    int32_t steps_done;
    int32_t n_bodies;
    int64_t est_bytes;     /* admission estimate of the request's device memory */
    double queue_ms;       /* submit -> admitted */
    double run_ms;         /* admitted -> done (scene creation, steps, state read-back) */
    double step_ms_p50;    /* per-step wall-clock latency (abd_step call) */
    double step_ms_p99;
    abd_step_stats last;   /* statistics of the last step */
} abd_request_info;

/* Create a server (threads started, streams created on `device`).  The
 * descriptor is copied.  ABD_E_INVALID for n_streams < 1. */
int abd_server_create(const abd_server_desc *desc, abd_server **out);

/* Queue a request.  Every array behind `scene` (and `part`, `params`) is
 * copied before return, so the caller may free them.  `part` NULL: one
 * partition (monolithic).  `params` NULL: abd_step_params_default().
 * *ticket identifies the request in the calls below. */
int abd_server_submit(abd_server *srv, const abd_scene_desc *scene, const abd_partition_desc *part,
                      const abd_step_params *params, int32_t n_steps, int64_t *ticket);

/* Queue a request on a resident scene named by `key` (non-zero).  The first
 * request of a key gives the scene (and optionally its partition; arrays
 * copied before return); it builds the scene, which then stays on the
 * device after the request -- its state q, v and its workspace (consensus z,
 * dual u, pair lists, captured Newton-iteration graph) -- on a CUDA stream of
 * its own.  Later requests of the key pass scene = NULL and continue from the
 * state the previous one left; requests of one key run one at a time in
 * submission order, while other keys' requests overlap with them.  A resident
 * scene holds its admission estimate of the HBM budget; when a request does
 * not fit, idle resident scenes are evicted, least recently used first
 * (their state is kept in host memory and the scene is rebuilt at its next
 * request).  ABD_E_INVALID for key 0, a first request without a scene, or a
 * scene given again for a live key.  Results, latencies and errors are read
 * per ticket as for abd_server_submit.  Not in the paper: this is the
 * library's serving runtime. */
int abd_server_submit_keyed(abd_server *srv, int64_t key, const abd_scene_desc *scene,
                            const abd_partition_desc *part, const abd_step_params *params, int32_t n_steps,
                            int64_t *ticket);

/* Free the resident scene of `key` once its queued requests are done (its
 * key may then name a new scene).  ABD_E_INVALID for an unknown key. */
int abd_server_release(abd_server *srv, int64_t key);

/* Current state of a request (non-blocking), or, for abd_server_wait, its
 * state once it is done.  ABD_E_INVALID for an unknown ticket. */
int abd_server_poll(abd_server *srv, int64_t ticket, abd_request_info *info);
int abd_server_wait(abd_server *srv, int64_t ticket, abd_request_info *info);

/* Final q and v ([n_bodies][12] each, host) of a done request; per-step
 * latencies (ms, up to `cap`) with their count in *n.  ABD_E_INVALID when the
 * request is not done or the sizes do not match; the request's error code if
 * it failed. */
int abd_server_result(abd_server *srv, int64_t ticket, double *q, double *v, int64_t n_bodies);
int abd_server_latencies(abd_server *srv, int64_t ticket, double *ms, int32_t cap, int32_t *n);

/* Last error text of a request (empty when none). */
const char *abd_server_error(abd_server *srv, int64_t ticket);

/* Wait for queued and running requests, stop the workers, free everything. */
void abd_server_destroy(abd_server *srv);

/* Per-kernel timing of the last steps (enabled by abd_profile(s, 1)): for the
 * kernel named `name`, launches, total device milliseconds (CUDA events on
 * the scene's stream) and algorithmic bytes moved. */
int abd_profile(abd_scene *s, int32_t enable);
int abd_kernel_stats(const abd_scene *s, const char *name, int64_t *launches, double *total_ms, double *bytes);

abd_step_params abd_step_params_default(void);
const char *abd_status_string(int code);
const char *abd_last_error(const abd_scene *s);

#ifdef __cplusplus
}
#endif
#endif
