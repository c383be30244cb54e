/*
 * abd_oracle.h -- FP64, single-threaded CPU oracle of distributed ABD-IPC.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no code, header,
 * table or helper with the CUDA library; the two meet only through the seeded
 * scene generators, which hold none of the method's arithmetic.
 *
 * What it computes (paper "Distributed Affine Body Dynamics with Adaptive
 * Consensus"):
 *   - the implicit-Euler incremental potential of affine bodies (Eq. 1),
 *   - the replica-weighted local objective F_i (Eq. 3),
 *   - the local projected-Newton solve with the consensus penalty (Eq. 5),
 *   - the consensus and dual updates (Eq. 6, Eq. 7),
 *   - the stopping metrics (Eq. 8-10), the CCD-certified merge (Sec. 4.2),
 *   - mass-aware rho initialisation and residual-driven adaptation (Sec. 4.3).
 * Details that the paper defers to the ABD and IPC papers (orthogonality
 * potential, log barrier, distance types, edge-edge mollifier, additive CCD)
 * follow the readings listed in the design notes; each function says which.
 *
 * All arrays are row-major, double precision, caller-owned.  q of one body is
 * (p0,p1,p2, A00,A01,A02, A10,A11,A12, A20,A21,A22), x = A*xbar + p.
 */
#ifndef ABD_ORACLE_H
#define ABD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_DYNAMIC = 0, ORC_STATIC = 1, ORC_KINEMATIC = 2 };
enum { ORC_OK = 0, ORC_ADMM_MAXITER = 1, ORC_NEWTON_MAXITER = 2, ORC_FELL_BACK = 3, ORC_DT_SPLIT = 4,
       ORC_E_INVALID = -1, ORC_E_OOM = -2, ORC_E_NOT_SPD = -3, ORC_E_PENETRATION = -6 };

typedef struct {
    int32_t n_meshes;
    const int32_t *mesh_n_verts, *mesh_n_tris;
    const double *mesh_xbar;   /* concatenated [sum V][3] */
    const int32_t *mesh_tris;  /* concatenated [sum T][3], mesh-local */
    int32_t n_bodies;
    const int32_t *body_mesh;
    const double *body_density, *body_kappa;
    const int32_t *body_kind;
    const double *body_q0, *body_v0; /* [B][12] */
    const double *body_omega;        /* [B][3] angular velocity of kinematic bodies about their centre
                                        of mass (world frame, rad/s), or NULL */
    int32_t n_planes;
    const int32_t *plane_axis;
    const double *plane_sign, *plane_offset;
    double gravity[3];
} orc_scene_desc;

typedef struct {
    double h, dhat, kappa_barrier;   /* kappa_barrier <= 0: 10 * mean dynamic mass * |g| / dhat */
    int32_t rho_adaptive;            /* 0 fixed rho = beta m, 1 residual-driven */
    double beta, tau, mu, sigma_min, sigma_max, theta;
    double newton_tol;               /* epsilon_N on |dq|_inf / (h l) */
    int32_t max_admm, max_newton, max_halvings;
    double accd_s, accd_c;
    /* partition (Sec. 4, Fig. 2): slabs along `axis` */
    int32_t n_slabs, axis;
    const double *planes;            /* n_slabs-1 offsets, or NULL: equal widths over the dynamic AABB */
    double alpha_w, w_min;           /* w = max(alpha_w v_max h, w_min); w_min <= 0: smallest body AABB diagonal */
    int32_t dt_split_max;            /* blocked merge: retake the step as two h/2 steps, this deep (0: off, at most 16) */
} orc_params;

typedef struct {
    int32_t status, admm_iters, newton_iters, n_shared, n_slots, merge_ok;
    int64_t n_candidates_peak, n_active_peak;
    double r_inf, s_inf, delta_inf, min_distance, l, kappa_barrier, w;
} orc_stats;

typedef struct orc_scene orc_scene;

/* scene */
int  orc_scene_create(const orc_scene_desc *d, orc_scene **out);
void orc_scene_destroy(orc_scene *s);
int  orc_scene_counts(const orc_scene *s, int64_t out[4]); /* bodies, verts, tris, edges */
int  orc_state_get(const orc_scene *s, double *q, double *v);
int  orc_state_set(orc_scene *s, const double *q, const double *v);
int  orc_body_props(const orc_scene *s, int b, double *m, double *com, double *S9, double *V);
int  orc_edges(const orc_scene *s, int32_t *edges /* [E][2] global vertex ids */);
int  orc_vertices(const orc_scene *s, const double *q, double *x /* [V][3] */);
int  orc_step(orc_scene *s, const orc_params *p, orc_stats *st);
int  orc_partition(orc_scene *s, const orc_params *p, uint64_t *mask /* [B] */, double *w_out);
int  orc_objective(orc_scene *s, const orc_params *p, const double *q, const double *qtil, double *E, double *g,
                   double *Hdense);
/* per-partition objectives F_i (Eq. 3) at a consensus point and the sums of
 * their gradients and projected Hessians; returns the partition count */
int  orc_local_objectives(orc_scene *s, const orc_params *p, const double *q, const double *qtil, double *E_parts,
                          int cap, double *g_sum, double *H_sum);

/* gradient (and value) of one partition's F_i (Eq. 3, no consensus term) at a
 * replica configuration q ([n_dof][12]); g gets [n_dof][12] */
int  orc_local_gradient(orc_scene *s, const orc_params *p, int part, const double *q, const double *qtil, double *E,
                        double *g);

/* ADMM trace: while set, every round k >= 2 that continues to a penalty
 * update (Sec. 4.3) appends records of ORC_TRACE_REC doubles: one per replica
 * of each shared body, then one per internal slot of each partition:
 *   [0] k  [1] body  [2] partition  [3] 1 shared, 0 internal
 *   [4] rho used by the last local solves  [5] rho after the update
 *   [6] r_b (Eq. 9)  [7] s_b (Eq. 10)  [8..19] the replica's q
 *   [20..31] z_b of round k-1  [32..43] z_b (Eq. 6)
 *   [44..55] u after the dual update (Eq. 7)  [56..67] u after the rescale
 * (fields 4..7 and 20..67 are 0 for internal slots).  Records beyond cap are
 * counted, not written.  buf NULL, cap 0: off. */
#define ORC_TRACE_REC 68
int  orc_admm_trace(orc_scene *s, double *buf, int64_t cap);
int64_t orc_admm_trace_count(const orc_scene *s);

/* building blocks, exposed for the pins */
/* residual-driven penalty of one shared body (Sec. 4.3); *u_scale = rho / rho_new */
double orc_rho_update(double r, double s, double rho, double rho0, double tau, double mu, double sigma_min,
                      double sigma_max, double *u_scale);
int    orc_mass_properties(int nv, const double *xbar, int nt, const int32_t *tris, double density,
                           double *m, double *com, double *S9, double *V);
double orc_orth(const double *q12, double kappa, double V, double *g12, double *H144);
void   orc_barrier(double d, double dhat, double out[3]);
double orc_pair(int is_ee, const double X[12], double dhat, double kB, double eps_x,
                double *E, double *g12, double *H144, int *type);
double orc_dist_type(int is_ee, const double X[12], int *type, double beta[2]);
void   orc_psd_project(int n, double *A);
double orc_ccd(int is_ee, const double X[12], const double dX[12], double s, double c);
double orc_ccd_plane(double d0, double dd, double s);
int64_t orc_candidates(const orc_scene *s, const double *x0, const double *x1, double dhat,
                       int32_t *out /* [cap][3]: type(0 PT,1 EE), i, j */, int64_t cap);
double orc_mollifier(const double X[12], double eps_x, double *g12, double *H144);

#ifdef __cplusplus
}
#endif
#endif
