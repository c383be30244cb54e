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
 *   - Body kinds: ABD_DYNAMIC (12 DoFs), ABD_STATIC (fixed collider).
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
    ABD_E_INVALID = -1,
    ABD_E_OOM = -2,
    ABD_E_CUDA = -3,
    ABD_E_PAIR_OVERFLOW = -4,
    ABD_E_DEVICE_TIMEOUT = -5,
    ABD_E_PENETRATION = -6,
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
    const int32_t *body_kind;      /* [B] ABD_DYNAMIC or ABD_STATIC */
    const double *body_q0;         /* [B][12] initial q in the mesh frame */
    const double *body_v0;         /* [B][12] initial qdot, or NULL for zero */
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
    double pcg_rtol;               /* relative residual of the block-Jacobi PCG */
    int32_t pcg_max;
    double accd_s, accd_c;         /* additive CCD gap fraction and step factor */
} abd_step_params;

typedef struct {
    int32_t status;
    int32_t admm_iters;            /* local-solve rounds */
    int32_t newton_iters;          /* Newton iterations summed over partitions and rounds */
    int32_t n_partitions, n_shared, n_slots;
    int64_t pcg_iters;             /* PCG iterations summed over Newton iterations */
    int64_t n_candidates_peak, n_active_peak;
    double r_inf, s_inf, delta_inf, min_distance, l, kappa_barrier, w;
    double t_solve_ms, t_coll_ms, t_sync_ms, t_total_ms; /* host wall clock split (Table 1 columns) */
    int64_t kernel_launches;       /* kernels of this library launched by the step */
} abd_step_stats;

/* --- scene ---------------------------------------------------------------- */

/* Copy the description to the device and compute per-body constants (mass,
 * second moment, volume, edges).  `cuda_stream` is a cudaStream_t (NULL: the
 * legacy default stream) on which every later call on this scene enqueues
 * work; the current CUDA device becomes the scene's device.
 * Errors: ABD_E_INVALID (bad indices, open or inverted dynamic mesh, more
 * than 8 planes, kinematic body), ABD_E_OOM, ABD_E_CUDA. */
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

/* Advance one time step.  Blocks until the step is complete. */
int abd_step(abd_scene *s, const abd_step_params *p, abd_step_stats *stats);

/* Host copies of the state (q, qdot), [B][12] each; either may be NULL. */
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
 *   Limits: at most 131072 bodies (ABD_E_INVALID beyond) and about 4 million
 *   overlapping body pairs (ABD_E_PAIR_OVERFLOW beyond), each with a message
 *   in abd_last_error().  Blocks until done. */
int abd_candidates_noalloc(abd_scene *s, const double *x0, const double *x1, double dhat, int32_t *out, int64_t cap,
                           int64_t *n_out);

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
