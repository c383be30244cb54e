/*
 * abd_oracle.c -- FP64, single-threaded CPU oracle of distributed ABD-IPC.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU baseline, never by the product path.  Plain loops, dense
 * linear algebra, brute-force candidates; no blocking, fusion or reordering
 * beyond what each definition states.  Shares no code with the CUDA library.
 *
 * Section map (paper: "Distributed Affine Body Dynamics with Adaptive
 * Consensus"):
 *   O1 affine bodies and mass matrix ............ Sec. 3 (Eq. 1), ABD DoFs
 *   O2 predicted state q~ ........................ Sec. 3, below Eq. 1
 *   O3 energies: inertia, orthogonality, barrier . Eq. 1, Eq. 3
 *   O4 broad-phase candidates (brute force) ...... Sec. 6 (candidate pairs)
 *   O5 additive CCD ............................... Sec. 4.2, linear trajectories
 *   O6 local Newton solve ......................... Eq. 5
 *   O7 partition, consensus ADMM, merge ........... Sec. 4, Eq. 2-10, Alg. 1
 * Parity status of each function is stated where it is defined; every
 * function below is pinned by a CPU test except the full contact-rich
 * trajectories, whose parity is unpinned beyond invariants.
 */
#include "abd_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF (1.0 / 0.0)

/* Kinematic bodies (reading: the paper's turntables have prescribed motion
 * and no stated treatment).  A kinematic body stays a DOF of the solve like a
 * dynamic one, but its predicted state q~ is its prescribed pose -- p moved by
 * its linear velocity, A rotated by R(omega h) about the centre of mass, no
 * gravity -- and its inertia term is weighted by ORC_KIN_WEIGHT, so contacts
 * cannot move it measurably off the prescription while barrier and CCD keep
 * every step penetration-free. */
#define ORC_KIN_WEIGHT 1e6

static int is_dof(int kind) { return kind != ORC_STATIC; }

/* Prescribed pose after h: p + h v_p, and A rotated by the angle |omega| h
 * about the axis omega (Rodrigues' formula R = I + sin t K + (1 - cos t) K^2,
 * K the cross-product matrix of the unit axis), A' = R A. */
static void kinematic_pose(const double *q, const double *v, const double *w, double h, double *out) {
    for (int k = 0; k < 3; ++k) out[k] = q[k] + h * v[k];
    double n = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]), R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (n > 0.0) {
        double u[3] = {w[0] / n, w[1] / n, w[2] / n}, t = n * h, sn = sin(t), c1 = 1.0 - cos(t);
        double K[9] = {0, -u[2], u[1], u[2], 0, -u[0], -u[1], u[0], 0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double k2 = 0.0;
                for (int l = 0; l < 3; ++l) k2 += K[3 * i + l] * K[3 * l + j];
                R[3 * i + j] += sn * K[3 * i + j] + c1 * k2;
            }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            out[3 + 3 * i + j] = R[3 * i] * q[3 + j] + R[3 * i + 1] * q[6 + j] + R[3 * i + 2] * q[9 + j];
}

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(double *o, const double *a, const double *b) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void cross3(double *o, const double *a, const double *b) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static int popcount64(uint64_t m) { int c = 0; while (m) { m &= m - 1; ++c; } return c; }

/* q index of the (component k, xi index a) entry: xi = (1, xbar0, xbar1, xbar2). */
static int qidx(int k, int a) { return a == 0 ? k : 3 + 3 * k + (a - 1); }

/* ------------------------------------------------------------------------ */
/* dense symmetric eigen-decomposition (cyclic Jacobi) and PSD projection    */
/* ------------------------------------------------------------------------ */

/* Cyclic Jacobi rotations on a symmetric n x n matrix (n <= 12).  On return A
 * is (numerically) diagonal and V holds the eigenvectors as columns. */
static void jacobi_eigen(int n, double *A, double *V) {
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double a2 = A[i * n + j] * A[i * n + j];
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* A <- A J */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* A <- J^T A */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) { /* V <- V J */
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

/* Projection to the nearest PSD matrix: negative eigenvalues are clamped to
 * zero (projected Newton, as in IPC/ABD).  A matrix without negative
 * eigenvalues is returned unchanged.  Pinned: PSD input unchanged, output
 * eigenvalues >= 0, agreement with numpy eigh clamping. */
void orc_psd_project(int n, double *A) {
    double E[144], V[144];
    memcpy(E, A, sizeof(double) * n * n);
    jacobi_eigen(n, E, V);
    int neg = 0;
    for (int i = 0; i < n; ++i) if (E[i * n + i] < 0.0) neg = 1;
    if (!neg) return;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) {
                double lam = E[k * n + k];
                if (lam > 0.0) s += V[i * n + k] * lam * V[j * n + k];
            }
            A[i * n + j] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* O1: mass properties of a closed mesh (signed tetrahedra to the origin)    */
/* ------------------------------------------------------------------------ */

/* Volume V, centre of mass and second moment S = rho * int (x-c)(x-c)^T dV of a
 * closed, outward-oriented triangle mesh.  The affine mass matrix is then
 * M = diag(m I3, S, S, S) in q order once xbar is recentred at c (ABD DoFs,
 * Sec. 3).  Pinned: unit cube m = rho, S = rho/12 I; icosphere volume. */
int orc_mass_properties(int nv, const double *xbar, int nt, const int32_t *tris, double density,
                        double *m, double *com, double *S9, double *V) {
    double vol = 0.0, fm[3] = {0, 0, 0};
    for (int t = 0; t < nt; ++t) {
        const double *a = xbar + 3 * tris[3 * t], *b = xbar + 3 * tris[3 * t + 1], *c = xbar + 3 * tris[3 * t + 2];
        double bc[3];
        cross3(bc, b, c);
        double vt = dot3(a, bc) / 6.0;
        vol += vt;
        for (int k = 0; k < 3; ++k) fm[k] += vt * (a[k] + b[k] + c[k]) / 4.0;
    }
    if (!(vol > 0.0) || nv <= 0) return ORC_E_INVALID;
    double cc[3] = {fm[0] / vol, fm[1] / vol, fm[2] / vol};
    double S[9] = {0};
    for (int t = 0; t < nt; ++t) {
        double w[3][3], s[3], bc[3];
        for (int i = 0; i < 3; ++i) sub3(w[i], xbar + 3 * tris[3 * t + i], cc);
        cross3(bc, w[1], w[2]);
        double vt = dot3(w[0], bc) / 6.0;
        for (int k = 0; k < 3; ++k) s[k] = w[0][k] + w[1][k] + w[2][k];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = s[i] * s[j];
                for (int v = 0; v < 3; ++v) acc += w[v][i] * w[v][j];
                S[3 * i + j] += vt / 20.0 * acc;
            }
    }
    *m = density * vol;
    if (V) *V = vol;
    if (com) memcpy(com, cc, sizeof cc);
    if (S9) for (int i = 0; i < 9; ++i) S9[i] = density * S[i];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* O3: orthogonality potential kappa V ||A A^T - I||_F^2                     */
/* ------------------------------------------------------------------------ */

/* Energy, gradient (12, zero in p) and raw Hessian (12x12) of the ABD
 * orthogonality potential (the elastic term of Eq. 1 under the reading in the
 * design notes).  With rows a_k of A and C = A A^T - I:
 *   dE/da_k = 4 kappa V sum_l C_kl a_l,
 *   d2E/da_k da_l = 4 kappa V (delta_kl A^T A + a_l a_k^T + C_kl I).
 * Pinned by central finite differences and by E = grad = 0 at any rotation. */
double orc_orth(const double *q12, double kappa, double V, double *g12, double *H144) {
    const double *a[3] = {q12 + 3, q12 + 6, q12 + 9};
    double C[3][3], E = 0.0, kv = kappa * V;
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            C[k][l] = dot3(a[k], a[l]) - (k == l ? 1.0 : 0.0);
            E += C[k][l] * C[k][l];
        }
    if (g12) {
        for (int i = 0; i < 12; ++i) g12[i] = 0.0;
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int l = 0; l < 3; ++l) s += C[k][l] * a[l][j];
                g12[3 + 3 * k + j] = 4.0 * kv * s;
            }
    }
    if (H144) {
        double AtA[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) AtA[i][j] = a[0][i] * a[0][j] + a[1][i] * a[1][j] + a[2][i] * a[2][j];
        for (int i = 0; i < 144; ++i) H144[i] = 0.0;
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double v = a[l][i] * a[k][j] + (i == j ? C[k][l] : 0.0);
                        if (k == l) v += AtA[i][j];
                        H144[(3 + 3 * k + i) * 12 + 3 + 3 * l + j] = 4.0 * kv * v;
                    }
    }
    return kv * E;
}

/* ------------------------------------------------------------------------ */
/* O3: IPC log barrier on the unsquared distance                             */
/* ------------------------------------------------------------------------ */

/* b(d) = -(d - dhat)^2 ln(d / dhat) on 0 < d < dhat, 0 beyond; out = (b, b', b'').
 * Pinned by finite differences and b(dhat) = b'(dhat) = 0. */
void orc_barrier(double d, double dhat, double out[3]) {
    if (d >= dhat) { out[0] = out[1] = out[2] = 0.0; return; }
    if (d <= 0.0) { out[0] = ORC_INF; out[1] = -ORC_INF; out[2] = ORC_INF; return; }
    double e = d - dhat, L = log(d / dhat);
    out[0] = -e * e * L;
    out[1] = -2.0 * e * L - e * e / d;
    out[2] = -2.0 * L - 4.0 * e / d + e * e / (d * d);
}

/* ------------------------------------------------------------------------ */
/* O3: distance types and their derivatives                                  */
/* ------------------------------------------------------------------------ */
/*
 * Every point-triangle (PT) and edge-edge (EE) distance type is a closest-
 * point problem d^2(x) = min_beta |r(x, beta)|^2 with r = sum_v w_v(beta) x_v,
 * w affine in beta.  Type codes:
 *   PT (X0 = point, X1..X3 = triangle):  0..2 point-vertex t_m, 3..5 point-edge
 *     (t0t1, t1t2, t2t0), 6 point-face.
 *   EE (X0,X1 = edge a, X2,X3 = edge b): 0..3 vertex-vertex (a_i, b_j) = 2i+j,
 *     4..5 a_i to edge b, 6..7 b_j to edge a, 8 edge-edge interior.
 * The type is the feature of the exact closest points: the unconstrained
 * minimiser when it lies inside the parameter domain, otherwise the best of the
 * boundary sub-problems (the objective is a convex quadratic, so its constrained
 * minimum lies on the boundary).  Edges with sin^2(angle) <= 1e-10 are treated
 * as parallel and use the boundary sub-problems (a reading; the mollifier below
 * makes their barrier vanish).  Pinned against dense sampling of the
 * parameter domain.
 */
typedef struct { int k; double w0[4]; double c[2][4]; } feature_t;

static double seg_param(const double *p, const double *a, const double *b) {
    double ab[3], ap[3];
    sub3(ab, b, a);
    sub3(ap, p, a);
    double L = dot3(ab, ab);
    double t = L > 0.0 ? dot3(ap, ab) / L : 0.0;
    return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}

static double seg_dist2(const double *p, const double *a, const double *b, double t) {
    double c[3], r[3];
    for (int k = 0; k < 3; ++k) c[k] = a[k] + t * (b[k] - a[k]);
    sub3(r, p, c);
    return dot3(r, r);
}

static void feature_of(int is_ee, int type, feature_t *f) {
    memset(f, 0, sizeof *f);
    if (!is_ee) {
        static const int em[3] = {0, 1, 2}, en[3] = {1, 2, 0};
        if (type <= 2) { f->k = 0; f->w0[0] = 1; f->w0[1 + type] = -1; }
        else if (type <= 5) {
            int m = em[type - 3], n = en[type - 3];
            f->k = 1; f->w0[0] = 1; f->w0[1 + m] = -1; f->c[0][1 + m] = 1; f->c[0][1 + n] = -1;
        } else {
            f->k = 2; f->w0[0] = 1; f->w0[1] = -1;
            f->c[0][1] = 1; f->c[0][2] = -1; f->c[1][1] = 1; f->c[1][3] = -1;
        }
    } else {
        if (type <= 3) { int i = type >> 1, j = type & 1; f->k = 0; f->w0[i] = 1; f->w0[2 + j] = -1; }
        else if (type <= 5) { int i = type - 4; f->k = 1; f->w0[i] = 1; f->w0[2] = -1; f->c[0][2] = 1; f->c[0][3] = -1; }
        else if (type <= 7) { int j = type - 6; f->k = 1; f->w0[2 + j] = 1; f->w0[0] = -1; f->c[0][0] = 1; f->c[0][1] = -1; }
        else { f->k = 2; f->w0[0] = 1; f->w0[2] = -1; f->c[0][0] = -1; f->c[0][1] = 1; f->c[1][2] = 1; f->c[1][3] = -1; }
    }
}

/* Classify the closest features and return the squared distance. */
double orc_dist_type(int is_ee, const double X[12], int *type, double beta[2]) {
    beta[0] = beta[1] = 0.0;
    if (!is_ee) {
        const double *p = X, *t0 = X + 3, *t1 = X + 6, *t2 = X + 9;
        double e1[3], e2[3], ap[3];
        sub3(e1, t1, t0); sub3(e2, t2, t0); sub3(ap, p, t0);
        double G00 = dot3(e1, e1), G01 = dot3(e1, e2), G11 = dot3(e2, e2);
        double r0 = dot3(ap, e1), r1 = dot3(ap, e2);
        double det = G00 * G11 - G01 * G01;
        if (det > 0.0) {
            double u = (r0 * G11 - r1 * G01) / det, v = (G00 * r1 - G01 * r0) / det;
            if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) {
                double c[3], r[3];
                for (int k = 0; k < 3; ++k) c[k] = t0[k] + u * e1[k] + v * e2[k];
                sub3(r, p, c);
                *type = 6; beta[0] = u; beta[1] = v;
                return dot3(r, r);
            }
        }
        const double *tv[3] = {t0, t1, t2};
        double best = ORC_INF;
        for (int e = 0; e < 3; ++e) {
            int m = e, n = (e + 1) % 3;
            double t = seg_param(p, tv[m], tv[n]);
            double d2 = seg_dist2(p, tv[m], tv[n], t);
            if (d2 < best) {
                best = d2;
                if (t == 0.0) { *type = m; beta[0] = 0.0; }
                else if (t == 1.0) { *type = n; beta[0] = 0.0; }
                else { *type = 3 + e; beta[0] = t; }
            }
        }
        return best;
    }
    const double *a0 = X, *a1 = X + 3, *b0 = X + 6, *b1 = X + 9;
    double ea[3], eb[3], w[3];
    sub3(ea, a1, a0); sub3(eb, b1, b0); sub3(w, a0, b0);
    double A = dot3(ea, ea), B = dot3(ea, eb), C = dot3(eb, eb), D = dot3(ea, w), E = dot3(eb, w);
    double den = A * C - B * B;
    if (den > 1e-10 * A * C) {
        double s = (B * E - C * D) / den, t = (A * E - B * D) / den;
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
            double r[3];
            for (int k = 0; k < 3; ++k) r[k] = w[k] + s * ea[k] - t * eb[k];
            *type = 8; beta[0] = s; beta[1] = t;
            return dot3(r, r);
        }
    }
    double best = ORC_INF;
    const double *av[2] = {a0, a1}, *bv[2] = {b0, b1};
    for (int i = 0; i < 2; ++i) { /* a_i against edge b */
        double t = seg_param(av[i], b0, b1), d2 = seg_dist2(av[i], b0, b1, t);
        if (d2 < best) {
            best = d2;
            if (t == 0.0) { *type = 2 * i; beta[0] = 0.0; }
            else if (t == 1.0) { *type = 2 * i + 1; beta[0] = 0.0; }
            else { *type = 4 + i; beta[0] = t; }
        }
    }
    for (int j = 0; j < 2; ++j) { /* b_j against edge a */
        double t = seg_param(bv[j], a0, a1), d2 = seg_dist2(bv[j], a0, a1, t);
        if (d2 < best) {
            best = d2;
            if (t == 0.0) { *type = j; beta[0] = 0.0; }
            else if (t == 1.0) { *type = 2 + j; beta[0] = 0.0; }
            else { *type = 6 + j; beta[0] = t; }
        }
    }
    return best;
}

/* Squared distance s = |r|^2 at the stationary beta of the type, its gradient
 * and Hessian by the envelope theorem:
 *   grad s = 2 w (x) r,
 *   hess s = 2 (w w^T (x) I3) - 2 sum_ij Ginv_ij g_i g_j^T,
 * with D_j = sum_v c_jv x_v, G_ij = D_i . D_j, g_j[v] = w_v D_j + c_jv r. */
static double dist2_derivs(const double X[12], const feature_t *f, const double beta[2], double *gs, double *Hs) {
    double w[4], r[3] = {0, 0, 0}, D[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int v = 0; v < 4; ++v) {
        w[v] = f->w0[v];
        for (int j = 0; j < f->k; ++j) w[v] += beta[j] * f->c[j][v];
    }
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) {
            r[a] += w[v] * X[3 * v + a];
            for (int j = 0; j < f->k; ++j) D[j][a] += f->c[j][v] * X[3 * v + a];
        }
    double s = dot3(r, r);
    if (gs)
        for (int v = 0; v < 4; ++v)
            for (int a = 0; a < 3; ++a) gs[3 * v + a] = 2.0 * w[v] * r[a];
    if (Hs) {
        for (int i = 0; i < 144; ++i) Hs[i] = 0.0;
        for (int v = 0; v < 4; ++v)
            for (int u = 0; u < 4; ++u)
                for (int a = 0; a < 3; ++a) Hs[(3 * v + a) * 12 + 3 * u + a] = 2.0 * w[v] * w[u];
        if (f->k > 0) {
            double G[2][2], Gi[2][2], g[2][12];
            for (int i = 0; i < f->k; ++i)
                for (int j = 0; j < f->k; ++j) G[i][j] = dot3(D[i], D[j]);
            if (f->k == 1) Gi[0][0] = 1.0 / G[0][0];
            else {
                double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
                Gi[0][0] = G[1][1] / det; Gi[1][1] = G[0][0] / det;
                Gi[0][1] = -G[0][1] / det; Gi[1][0] = -G[1][0] / det;
            }
            for (int j = 0; j < f->k; ++j)
                for (int v = 0; v < 4; ++v)
                    for (int a = 0; a < 3; ++a) g[j][3 * v + a] = w[v] * D[j][a] + f->c[j][v] * r[a];
            for (int i = 0; i < f->k; ++i)
                for (int j = 0; j < f->k; ++j)
                    for (int m = 0; m < 12; ++m)
                        for (int n = 0; n < 12; ++n) Hs[m * 12 + n] -= 2.0 * Gi[i][j] * g[i][m] * g[j][n];
        }
    }
    return s;
}

/* IPC edge-edge mollifier m(c) with c = |(a1-a0) x (b1-b0)|^2:
 * m = (c/eps)(2 - c/eps) for c < eps, else 1; eps = 1e-3 |ea_rest|^2 |eb_rest|^2.
 * Returns m, its gradient and Hessian in the 12 vertex coordinates.
 * Pinned by finite differences. */
double orc_mollifier(const double X[12], double eps_x, double *g12, double *H144) {
    double ea[3], eb[3], cr[3];
    sub3(ea, X + 3, X);
    sub3(eb, X + 9, X + 6);
    cross3(cr, ea, eb);
    double c = dot3(cr, cr);
    if (g12) for (int i = 0; i < 12; ++i) g12[i] = 0.0;
    if (H144) for (int i = 0; i < 144; ++i) H144[i] = 0.0;
    if (c >= eps_x) return 1.0;
    double rr = c / eps_x, m = rr * (2.0 - rr), m1 = (2.0 - 2.0 * rr) / eps_x, m2 = -2.0 / (eps_x * eps_x);
    /* gradient of c in (ea, eb) */
    double ge[6];
    { double t[3]; cross3(t, eb, cr); for (int k = 0; k < 3; ++k) ge[k] = 2.0 * t[k]; }
    { double t[3]; cross3(t, cr, ea); for (int k = 0; k < 3; ++k) ge[3 + k] = 2.0 * t[k]; }
    /* Hessian of c in (ea, eb): 2 J^T J + 2 sum_i cr_i hess(cr_i) */
    double J[3][6];
    /* d cr / d ea = -[eb]x ; d cr / d eb = [ea]x ; [v]x w = v x w */
    double ebx[3][3] = {{0, -eb[2], eb[1]}, {eb[2], 0, -eb[0]}, {-eb[1], eb[0], 0}};
    double eax[3][3] = {{0, -ea[2], ea[1]}, {ea[2], 0, -ea[0]}, {-ea[1], ea[0], 0}};
    double crx[3][3] = {{0, -cr[2], cr[1]}, {cr[2], 0, -cr[0]}, {-cr[1], cr[0], 0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { J[i][j] = -ebx[i][j]; J[i][3 + j] = eax[i][j]; }
    double He[6][6];
    for (int m_ = 0; m_ < 6; ++m_)
        for (int n = 0; n < 6; ++n) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i) s += J[i][m_] * J[i][n];
            He[m_][n] = 2.0 * s;
        }
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            He[j][3 + k] += -2.0 * crx[j][k];
            He[3 + j][k] += 2.0 * crx[j][k];
        }
    /* map (ea, eb) -> (a0, a1, b0, b1) */
    static const int ev[4] = {0, 0, 1, 1};
    static const double sg[4] = {-1.0, 1.0, -1.0, 1.0};
    double gc[12], Hc[144];
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) gc[3 * v + a] = sg[v] * ge[3 * ev[v] + a];
    for (int v = 0; v < 4; ++v)
        for (int u = 0; u < 4; ++u)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    Hc[(3 * v + a) * 12 + 3 * u + b] = sg[v] * sg[u] * He[3 * ev[v] + a][3 * ev[u] + b];
    if (g12) for (int i = 0; i < 12; ++i) g12[i] = m1 * gc[i];
    if (H144)
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) H144[i * 12 + j] = m2 * gc[i] * gc[j] + m1 * Hc[i * 12 + j];
    return m;
}

/* Barrier energy of one PT or EE pair (without the h^2 / kappa_c weight):
 * kB * b(d) for PT, kB * m(c) * b(d) for EE, with gradient and raw (unprojected)
 * Hessian in the 12 vertex coordinates.  Returns the unsigned distance d.
 * Pinned by finite differences for every distance type. */
double orc_pair(int is_ee, const double X[12], double dhat, double kB, double eps_x,
                double *E, double *g12, double *H144, int *type) {
    int ty = 0;
    double beta[2];
    orc_dist_type(is_ee, X, &ty, beta);
    if (type) *type = ty;
    feature_t f;
    feature_of(is_ee, ty, &f);
    double gs[12], Hs[144];
    double s = dist2_derivs(X, &f, beta, gs, Hs);
    double d = sqrt(s);
    if (g12) for (int i = 0; i < 12; ++i) g12[i] = 0.0;
    if (H144) for (int i = 0; i < 144; ++i) H144[i] = 0.0;
    if (E) *E = 0.0;
    if (d >= dhat) return d;
    double bb[3];
    orc_barrier(d, dhat, bb);
    if (d <= 0.0) { if (E) *E = ORC_INF; return d; }
    double gd[12], Hd[144], gb[12], Hb[144];
    for (int i = 0; i < 12; ++i) gd[i] = gs[i] / (2.0 * d);
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) Hd[i * 12 + j] = Hs[i * 12 + j] / (2.0 * d) - gs[i] * gs[j] / (4.0 * d * d * d);
    for (int i = 0; i < 12; ++i) gb[i] = bb[1] * gd[i];
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) Hb[i * 12 + j] = bb[2] * gd[i] * gd[j] + bb[1] * Hd[i * 12 + j];
    if (!is_ee) {
        if (E) *E = kB * bb[0];
        if (g12) for (int i = 0; i < 12; ++i) g12[i] = kB * gb[i];
        if (H144) for (int i = 0; i < 144; ++i) H144[i] = kB * Hb[i];
        return d;
    }
    double gm[12], Hm[144];
    double m = orc_mollifier(X, eps_x, gm, Hm);
    if (E) *E = kB * m * bb[0];
    if (g12) for (int i = 0; i < 12; ++i) g12[i] = kB * (gm[i] * bb[0] + m * gb[i]);
    if (H144)
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j)
                H144[i * 12 + j] = kB * (Hm[i * 12 + j] * bb[0] + gm[i] * gb[j] + gb[i] * gm[j] + m * Hb[i * 12 + j]);
    return d;
}

/* ------------------------------------------------------------------------ */
/* O5: additive CCD along linear vertex trajectories                         */
/* ------------------------------------------------------------------------ */

/* Conservative advancement (additive CCD, Li et al. 2021) for vertices moving
 * from X to X + dX over t in [0, 1].  Displacements are shifted to zero mean;
 * l_p = largest displacement norm on each side, summed, bounds the rate at
 * which the distance can shrink.  The first advance (1-s) d0 / l_p keeps the
 * distance >= g = s d0 and is always taken; later advances c d / l_p keep it
 * above (1-c) d.  An advance that reaches t = 1 certifies the rest of the path
 * (returns exactly 1).  Once the distance after a later advance falls below g,
 * the time before that advance is returned.  Constants s, c are readings
 * (0.1, 0.9).  Pinned: never beyond the exact time of impact, distance at the
 * returned time >= s d0 (up to rounding), 1 for separating or parallel
 * motion. */
double orc_ccd(int is_ee, const double X[12], const double dX[12], double s, double c) {
    double P[12], mean[3] = {0, 0, 0};
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) mean[a] += 0.25 * dX[3 * v + a];
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) P[3 * v + a] = dX[3 * v + a] - mean[a];
    double n[4];
    for (int v = 0; v < 4; ++v) n[v] = sqrt(dot3(P + 3 * v, P + 3 * v));
    double lp = is_ee ? dmax(n[0], n[1]) + dmax(n[2], n[3]) : n[0] + dmax(n[1], dmax(n[2], n[3]));
    if (lp == 0.0) return 1.0;
    int ty;
    double beta[2];
    double d = sqrt(orc_dist_type(is_ee, X, &ty, beta));
    if (!(d > 0.0)) return 0.0;
    double g = s * d, t = 0.0, step = (1.0 - s) * d / lp;
    for (int it = 0; it < 1000000; ++it) {
        if (t + step >= 1.0) return 1.0;
        double tn = t + step, Xn[12];
        for (int i = 0; i < 12; ++i) Xn[i] = X[i] + tn * dX[i];
        double dn = sqrt(orc_dist_type(is_ee, Xn, &ty, beta));
        if (t > 0.0 && dn < g) return t;
        t = tn;
        d = dn;
        step = c * d / lp;
    }
    return t;
}

/* Vertex against an axis-aligned plane: the distance d0 + t*dd is linear in t;
 * the time of impact is when it reaches s*d0 (closed form), capped at 1. */
double orc_ccd_plane(double d0, double dd, double s) {
    if (!(d0 > 0.0)) return 0.0;
    if (dd >= 0.0) return 1.0;
    double t = (1.0 - s) * d0 / (-dd);
    return t < 1.0 ? t : 1.0;
}

/* ------------------------------------------------------------------------ */
/* scene                                                                     */
/* ------------------------------------------------------------------------ */

struct orc_scene {
    int nb, np;
    int *kind, *voff, *nv, *toff, *nt, *eoff, *ne;
    double *mass, *S, *vol, *kappa, *com;
    double *xbar, *erest2;
    int *tri, *edge;
    double *q, *v;
    double *omega;   /* [B][3] kinematic angular velocity */
    int *pax;
    double *psg, *poff;
    double g[3];
    int64_t V, T, E;
    /* optional ADMM trace (orc_admm_trace): ORC_TRACE_REC doubles per record */
    double *trace;
    int64_t trace_cap, trace_n;
};

static int cmp_edge(const void *a, const void *b) {
    const int *x = (const int *)a, *y = (const int *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

/* Unique undirected edges of a triangle list, sorted by (min, max) vertex. */
static int build_edges(int nt, const int32_t *tris, int **out) {
    int *e = (int *)malloc(sizeof(int) * 6 * (size_t)(nt > 0 ? nt : 1));
    if (!e) return -1;
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
            e[6 * t + 2 * k] = a < b ? a : b;
            e[6 * t + 2 * k + 1] = a < b ? b : a;
        }
    qsort(e, (size_t)3 * nt, 2 * sizeof(int), cmp_edge);
    int n = 0;
    for (int i = 0; i < 3 * nt; ++i)
        if (n == 0 || e[2 * i] != e[2 * (n - 1)] || e[2 * i + 1] != e[2 * (n - 1) + 1]) {
            e[2 * n] = e[2 * i];
            e[2 * n + 1] = e[2 * i + 1];
            ++n;
        }
    *out = e;
    return n;
}

void orc_scene_destroy(orc_scene *s) {
    if (!s) return;
    free(s->kind); free(s->voff); free(s->nv); free(s->toff); free(s->nt); free(s->eoff); free(s->ne);
    free(s->mass); free(s->S); free(s->vol); free(s->kappa); free(s->com);
    free(s->xbar); free(s->erest2); free(s->tri); free(s->edge); free(s->q); free(s->v); free(s->omega);
    free(s->pax); free(s->psg); free(s->poff);
    free(s);
}

int orc_scene_create(const orc_scene_desc *d, orc_scene **out) {
    if (!d || !out || d->n_bodies <= 0 || d->n_meshes <= 0) return ORC_E_INVALID;
    int nm = d->n_meshes, nb = d->n_bodies;
    int *mvo = (int *)calloc(nm + 1, sizeof(int)), *mto = (int *)calloc(nm + 1, sizeof(int));
    int **medge = (int **)calloc(nm, sizeof(int *)), *mne = (int *)calloc(nm, sizeof(int));
    orc_scene *s = (orc_scene *)calloc(1, sizeof(orc_scene));
    int rc = ORC_OK;
    if (!mvo || !mto || !medge || !mne || !s) { rc = ORC_E_OOM; goto fail; }
    for (int m = 0; m < nm; ++m) {
        mvo[m + 1] = mvo[m] + d->mesh_n_verts[m];
        mto[m + 1] = mto[m] + d->mesh_n_tris[m];
        mne[m] = build_edges(d->mesh_n_tris[m], d->mesh_tris + 3 * (size_t)mto[m], &medge[m]);
        if (mne[m] < 0) { rc = ORC_E_OOM; goto fail; }
    }
    s->nb = nb;
    s->kind = (int *)malloc(sizeof(int) * nb); s->voff = (int *)malloc(sizeof(int) * (nb + 1));
    s->nv = (int *)malloc(sizeof(int) * nb); s->toff = (int *)malloc(sizeof(int) * (nb + 1));
    s->nt = (int *)malloc(sizeof(int) * nb); s->eoff = (int *)malloc(sizeof(int) * (nb + 1));
    s->ne = (int *)malloc(sizeof(int) * nb);
    s->mass = (double *)calloc(nb, sizeof(double)); s->S = (double *)calloc(9 * (size_t)nb, sizeof(double));
    s->vol = (double *)calloc(nb, sizeof(double)); s->kappa = (double *)calloc(nb, sizeof(double));
    s->com = (double *)calloc(3 * (size_t)nb, sizeof(double));
    s->q = (double *)malloc(sizeof(double) * 12 * nb); s->v = (double *)malloc(sizeof(double) * 12 * nb);
    s->omega = (double *)calloc(3 * (size_t)nb, sizeof(double));
    if (!s->kind || !s->voff || !s->nv || !s->toff || !s->nt || !s->eoff || !s->ne || !s->mass || !s->S ||
        !s->vol || !s->kappa || !s->com || !s->q || !s->v || !s->omega) { rc = ORC_E_OOM; goto fail; }
    s->voff[0] = s->toff[0] = s->eoff[0] = 0;
    for (int b = 0; b < nb; ++b) {
        int m = d->body_mesh[b];
        if (m < 0 || m >= nm) { rc = ORC_E_INVALID; goto fail; }
        s->nv[b] = d->mesh_n_verts[m]; s->nt[b] = d->mesh_n_tris[m]; s->ne[b] = mne[m];
        s->voff[b + 1] = s->voff[b] + s->nv[b];
        s->toff[b + 1] = s->toff[b] + s->nt[b];
        s->eoff[b + 1] = s->eoff[b] + s->ne[b];
    }
    s->V = s->voff[nb]; s->T = s->toff[nb]; s->E = s->eoff[nb];
    s->xbar = (double *)malloc(sizeof(double) * 3 * (s->V ? s->V : 1));
    s->tri = (int *)malloc(sizeof(int) * 3 * (s->T ? s->T : 1));
    s->edge = (int *)malloc(sizeof(int) * 2 * (s->E ? s->E : 1));
    s->erest2 = (double *)malloc(sizeof(double) * (s->E ? s->E : 1));
    if (!s->xbar || !s->tri || !s->edge || !s->erest2) { rc = ORC_E_OOM; goto fail; }
    for (int b = 0; b < nb; ++b) {
        int m = d->body_mesh[b];
        const double *mx = d->mesh_xbar + 3 * (size_t)mvo[m];
        const int32_t *mt = d->mesh_tris + 3 * (size_t)mto[m];
        s->kind[b] = d->body_kind[b];
        s->kappa[b] = d->body_kappa[b];
        memcpy(s->q + 12 * b, d->body_q0 + 12 * b, sizeof(double) * 12);
        if (d->body_v0) memcpy(s->v + 12 * b, d->body_v0 + 12 * b, sizeof(double) * 12);
        else memset(s->v + 12 * b, 0, sizeof(double) * 12);
        double com[3] = {0, 0, 0};
        if (s->kind[b] != ORC_DYNAMIC && s->kind[b] != ORC_STATIC && s->kind[b] != ORC_KINEMATIC) {
            rc = ORC_E_INVALID;
            goto fail;
        }
        if (is_dof(s->kind[b])) {
            if (orc_mass_properties(s->nv[b], mx, s->nt[b], mt, d->body_density[b], &s->mass[b], com,
                                    s->S + 9 * b, &s->vol[b]) != ORC_OK) { rc = ORC_E_INVALID; goto fail; }
        }
        if (s->kind[b] == ORC_KINEMATIC) {
            s->mass[b] *= ORC_KIN_WEIGHT;
            for (int i = 0; i < 9; ++i) s->S[9 * b + i] *= ORC_KIN_WEIGHT;
            if (d->body_omega)
                for (int k = 0; k < 3; ++k) s->omega[3 * b + k] = d->body_omega[3 * b + k];
        }
        memcpy(s->com + 3 * b, com, sizeof com);
        /* recentre xbar at the centre of mass and move p so x is unchanged */
        for (int v = 0; v < s->nv[b]; ++v)
            for (int k = 0; k < 3; ++k) s->xbar[3 * (s->voff[b] + v) + k] = mx[3 * v + k] - com[k];
        const double *A = s->q + 12 * b + 3;
        for (int k = 0; k < 3; ++k) s->q[12 * b + k] += A[3 * k] * com[0] + A[3 * k + 1] * com[1] + A[3 * k + 2] * com[2];
        for (int t = 0; t < s->nt[b]; ++t)
            for (int k = 0; k < 3; ++k) s->tri[3 * (s->toff[b] + t) + k] = mt[3 * t + k];
        for (int e = 0; e < s->ne[b]; ++e) {
            int a = medge[m][2 * e], c = medge[m][2 * e + 1];
            s->edge[2 * (s->eoff[b] + e)] = a;
            s->edge[2 * (s->eoff[b] + e) + 1] = c;
            double r[3];
            sub3(r, mx + 3 * a, mx + 3 * c);
            s->erest2[s->eoff[b] + e] = dot3(r, r);
        }
    }
    s->np = d->n_planes;
    s->pax = (int *)malloc(sizeof(int) * (s->np ? s->np : 1));
    s->psg = (double *)malloc(sizeof(double) * (s->np ? s->np : 1));
    s->poff = (double *)malloc(sizeof(double) * (s->np ? s->np : 1));
    if (!s->pax || !s->psg || !s->poff) { rc = ORC_E_OOM; goto fail; }
    for (int i = 0; i < s->np; ++i) {
        s->pax[i] = d->plane_axis[i]; s->psg[i] = d->plane_sign[i]; s->poff[i] = d->plane_offset[i];
        if (s->pax[i] < 0 || s->pax[i] > 2) { rc = ORC_E_INVALID; goto fail; }
    }
    for (int k = 0; k < 3; ++k) s->g[k] = d->gravity[k];
    for (int m = 0; m < nm; ++m) free(medge[m]);
    free(medge); free(mne); free(mvo); free(mto);
    *out = s;
    return ORC_OK;
fail:
    if (medge) for (int m = 0; m < nm; ++m) free(medge[m]);
    free(medge); free(mne); free(mvo); free(mto);
    orc_scene_destroy(s);
    return rc;
}

int orc_scene_counts(const orc_scene *s, int64_t out[4]) {
    out[0] = s->nb; out[1] = s->V; out[2] = s->T; out[3] = s->E;
    return ORC_OK;
}

int orc_state_get(const orc_scene *s, double *q, double *v) {
    if (q) memcpy(q, s->q, sizeof(double) * 12 * s->nb);
    if (v) memcpy(v, s->v, sizeof(double) * 12 * s->nb);
    return ORC_OK;
}

int orc_state_set(orc_scene *s, const double *q, const double *v) {
    if (q) memcpy(s->q, q, sizeof(double) * 12 * s->nb);
    if (v) memcpy(s->v, v, sizeof(double) * 12 * s->nb);
    return ORC_OK;
}

int orc_body_props(const orc_scene *s, int b, double *m, double *com, double *S9, double *V) {
    if (b < 0 || b >= s->nb) return ORC_E_INVALID;
    if (m) *m = s->mass[b];
    if (com) memcpy(com, s->com + 3 * b, sizeof(double) * 3);
    if (S9) memcpy(S9, s->S + 9 * b, sizeof(double) * 9);
    if (V) *V = s->vol[b];
    return ORC_OK;
}

int orc_edges(const orc_scene *s, int32_t *edges) {
    for (int b = 0; b < s->nb; ++b)
        for (int e = 0; e < s->ne[b]; ++e) {
            edges[2 * (s->eoff[b] + e)] = s->voff[b] + s->edge[2 * (s->eoff[b] + e)];
            edges[2 * (s->eoff[b] + e) + 1] = s->voff[b] + s->edge[2 * (s->eoff[b] + e) + 1];
        }
    return ORC_OK;
}

/* x = A xbar + p for the vertices of body b, written into the global array. */
static void body_positions(const orc_scene *s, int b, const double *q12, double *x) {
    const double *p = q12, *A = q12 + 3;
    for (int v = 0; v < s->nv[b]; ++v) {
        const double *xb = s->xbar + 3 * (s->voff[b] + v);
        double *o = x + 3 * (s->voff[b] + v);
        for (int k = 0; k < 3; ++k) o[k] = p[k] + (A[3 * k] * xb[0] + A[3 * k + 1] * xb[1] + A[3 * k + 2] * xb[2]);
    }
}

int orc_vertices(const orc_scene *s, const double *q, double *x) {
    for (int b = 0; b < s->nb; ++b) body_positions(s, b, (q ? q : s->q) + 12 * b, x);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* O4: broad-phase candidates                                                */
/* ------------------------------------------------------------------------ */

typedef struct { int type, bi, li, bj, lj; } pair_t; /* type 0 PT (vertex, tri), 1 EE */
typedef struct { pair_t *a; int64_t n, cap; } pairvec;

static int pv_push(pairvec *v, pair_t p) {
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 1024;
        pair_t *na = (pair_t *)realloc(v->a, sizeof(pair_t) * nc);
        if (!na) return -1;
        v->a = na;
        v->cap = nc;
    }
    v->a[v->n++] = p;
    return 0;
}

typedef struct { double lo[3], hi[3]; } box_t;

/* Box of a set of vertices of body b, over x0 and (if given) x1, inflated by
 * half on every side.  min/max are exact; +/- half is one rounding. */
static void prim_box(const double *x0, const double *x1, const int *gv, int n, double half, box_t *B) {
    for (int a = 0; a < 3; ++a) {
        double lo = x0[3 * gv[0] + a], hi = lo;
        for (int i = 0; i < n; ++i) {
            lo = dmin(lo, x0[3 * gv[i] + a]); hi = dmax(hi, x0[3 * gv[i] + a]);
            if (x1) { lo = dmin(lo, x1[3 * gv[i] + a]); hi = dmax(hi, x1[3 * gv[i] + a]); }
        }
        B->lo[a] = lo - half;
        B->hi[a] = hi + half;
    }
}

static int box_overlap(const box_t *a, const box_t *b) {
    for (int k = 0; k < 3; ++k)
        if (a->lo[k] > b->hi[k] || b->lo[k] > a->hi[k]) return 0;
    return 1;
}

static void body_box(const orc_scene *s, int b, const double *x0, const double *x1, double half, box_t *B) {
    for (int a = 0; a < 3; ++a) {
        double lo = x0[3 * s->voff[b] + a], hi = lo;
        for (int v = 0; v < s->nv[b]; ++v) {
            int g = s->voff[b] + v;
            lo = dmin(lo, x0[3 * g + a]); hi = dmax(hi, x0[3 * g + a]);
            if (x1) { lo = dmin(lo, x1[3 * g + a]); hi = dmax(hi, x1[3 * g + a]); }
        }
        B->lo[a] = lo - half;
        B->hi[a] = hi + half;
    }
}

/* Candidates among the listed bodies: all (vertex, triangle) pairs in both
 * directions and (edge, edge) pairs from two different bodies, not both
 * non-dynamic, whose boxes (dhat/2-inflated; over both configurations when x1
 * is given) overlap.  Two exact filters keep this brute force tractable
 * without changing the set: a primitive's box lies inside its body's box, so
 * body pairs with disjoint boxes and primitives disjoint from the other
 * body's box cannot contribute. */
static int enumerate_pairs(const orc_scene *s, const int *bodies, int nbod, const double *x0, const double *x1,
                           double dhat, pairvec *out) {
    double half = 0.5 * dhat;
    box_t *bb = (box_t *)malloc(sizeof(box_t) * (nbod ? nbod : 1));
    if (!bb) return -1;
    for (int i = 0; i < nbod; ++i) body_box(s, bodies[i], x0, x1, half, &bb[i]);
    int cap = 0;
    for (int i = 0; i < nbod; ++i) {
        int b = bodies[i];
        int m = s->nv[b];
        if (s->nt[b] > m) m = s->nt[b];
        if (s->ne[b] > m) m = s->ne[b];
        if (m > cap) cap = m;
    }
    int *fa = (int *)malloc(sizeof(int) * 6 * (cap + 1));
    box_t *fb = (box_t *)malloc(sizeof(box_t) * 6 * (cap + 1));
    if (!fa || !fb) { free(bb); free(fa); free(fb); return -1; }
    int *Va = fa, *Ta = fa + cap + 1, *Ea = fa + 2 * (cap + 1), *Vb = fa + 3 * (cap + 1), *Tb = fa + 4 * (cap + 1),
        *Eb = fa + 5 * (cap + 1);
    box_t *BVa = fb, *BTa = fb + cap + 1, *BEa = fb + 2 * (cap + 1), *BVb = fb + 3 * (cap + 1),
          *BTb = fb + 4 * (cap + 1), *BEb = fb + 5 * (cap + 1);
    int rc = 0;
    for (int i = 0; i < nbod && !rc; ++i)
        for (int j = i + 1; j < nbod && !rc; ++j) {
            int a = bodies[i], b = bodies[j];
            if (!is_dof(s->kind[a]) && !is_dof(s->kind[b])) continue;
            if (!box_overlap(&bb[i], &bb[j])) continue;
            int nVa = 0, nTa = 0, nEa = 0, nVb = 0, nTb = 0, nEb = 0;
            for (int pass = 0; pass < 2; ++pass) {
                int me = pass ? b : a;
                const box_t *other = pass ? &bb[i] : &bb[j];
                int *V = pass ? Vb : Va, *T = pass ? Tb : Ta, *E = pass ? Eb : Ea;
                box_t *BV = pass ? BVb : BVa, *BT = pass ? BTb : BTa, *BE = pass ? BEb : BEa;
                int nV = 0, nT = 0, nE = 0;
                for (int v = 0; v < s->nv[me]; ++v) {
                    int gv = s->voff[me] + v;
                    box_t B;
                    prim_box(x0, x1, &gv, 1, half, &B);
                    if (box_overlap(&B, other)) { V[nV] = v; BV[nV++] = B; }
                }
                for (int t = 0; t < s->nt[me]; ++t) {
                    int gv[3];
                    for (int k = 0; k < 3; ++k) gv[k] = s->voff[me] + s->tri[3 * (s->toff[me] + t) + k];
                    box_t B;
                    prim_box(x0, x1, gv, 3, half, &B);
                    if (box_overlap(&B, other)) { T[nT] = t; BT[nT++] = B; }
                }
                for (int e = 0; e < s->ne[me]; ++e) {
                    int gv[2];
                    for (int k = 0; k < 2; ++k) gv[k] = s->voff[me] + s->edge[2 * (s->eoff[me] + e) + k];
                    box_t B;
                    prim_box(x0, x1, gv, 2, half, &B);
                    if (box_overlap(&B, other)) { E[nE] = e; BE[nE++] = B; }
                }
                if (pass) { nVb = nV; nTb = nT; nEb = nE; } else { nVa = nV; nTa = nT; nEa = nE; }
            }
            for (int p = 0; p < nVa && !rc; ++p)
                for (int t = 0; t < nTb && !rc; ++t)
                    if (box_overlap(&BVa[p], &BTb[t])) rc = pv_push(out, (pair_t){0, a, Va[p], b, Tb[t]});
            for (int p = 0; p < nVb && !rc; ++p)
                for (int t = 0; t < nTa && !rc; ++t)
                    if (box_overlap(&BVb[p], &BTa[t])) rc = pv_push(out, (pair_t){0, b, Vb[p], a, Ta[t]});
            for (int p = 0; p < nEa && !rc; ++p)
                for (int q = 0; q < nEb && !rc; ++q)
                    if (box_overlap(&BEa[p], &BEb[q])) rc = pv_push(out, (pair_t){1, a, Ea[p], b, Eb[q]});
        }
    free(bb); free(fa); free(fb);
    return rc;
}

static int cmp_trip(const void *a, const void *b) {
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    for (int k = 0; k < 3; ++k)
        if (x[k] != y[k]) return x[k] < y[k] ? -1 : 1;
    return 0;
}

/* Candidate set of the whole scene at x0 (and swept to x1 when given), as
 * sorted (type, i, j) global ids: PT (vertex, triangle), EE (edge, edge) with
 * i < j.  Returns the count (entries beyond cap are counted, not written), or
 * -1 on allocation failure.  Pinned against an O(n^2) all-primitive scan. */
int64_t orc_candidates(const orc_scene *s, const double *x0, const double *x1, double dhat, int32_t *out, int64_t cap) {
    int *all = (int *)malloc(sizeof(int) * s->nb);
    pairvec pv = {0, 0, 0};
    if (!all) return -1;
    for (int b = 0; b < s->nb; ++b) all[b] = b;
    if (enumerate_pairs(s, all, s->nb, x0, x1, dhat, &pv)) { free(all); free(pv.a); return -1; }
    free(all);
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * 3 * (pv.n ? pv.n : 1));
    if (!tmp) { free(pv.a); return -1; }
    for (int64_t k = 0; k < pv.n; ++k) {
        pair_t p = pv.a[k];
        int32_t i, j;
        if (p.type == 0) { i = s->voff[p.bi] + p.li; j = s->toff[p.bj] + p.lj; }
        else {
            i = s->eoff[p.bi] + p.li; j = s->eoff[p.bj] + p.lj;
            if (i > j) { int32_t t = i; i = j; j = t; }
        }
        tmp[3 * k] = p.type; tmp[3 * k + 1] = i; tmp[3 * k + 2] = j;
    }
    qsort(tmp, (size_t)pv.n, 3 * sizeof(int32_t), cmp_trip);
    int64_t n = pv.n;
    if (out) memcpy(out, tmp, sizeof(int32_t) * 3 * (n < cap ? n : cap));
    free(tmp); free(pv.a);
    return n;
}

/* ------------------------------------------------------------------------ */
/* O6: the local problem of one partition (Eq. 5) and its Newton solve       */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_scene *s;
    int ns;            /* dynamic slots */
    int *body;         /* slot -> body */
    int *sob;          /* body -> slot or -1 */
    const uint64_t *mask; /* per body: partitions holding it */
    int *objs, nobj;   /* slot bodies, then colliders */
    double *q, *qtil, *z, *u, *rho; /* per slot */
    int *shared;
    double h, dhat, kB, epsN, l, accd_s, accd_c;
    int max_newton, max_halv;
    double *x0, *x1;   /* [V][3] scratch */
    int newton_iters;
    int maxed;          /* some solve ran max_newton iterations without meeting eps_N */
    int64_t cand_peak, act_peak;
} local_t;

static double kappa_b(const local_t *L, int b) { return (double)popcount64(L->mask[b]); }

static double kappa_c(const local_t *L, int a, int b) {
    const orc_scene *s = L->s;
    if (!is_dof(s->kind[a])) return (double)popcount64(L->mask[b]);
    if (!is_dof(s->kind[b])) return (double)popcount64(L->mask[a]);
    return (double)popcount64(L->mask[a] & L->mask[b]);
}

static void local_positions(local_t *L, const double *qs, double *x) {
    for (int i = 0; i < L->nobj; ++i) {
        int b = L->objs[i];
        int sl = L->sob[b];
        body_positions(L->s, b, sl >= 0 ? qs + 12 * sl : L->s->q + 12 * b, x);
    }
}

/* Gather the 12 coordinates of a pair's four vertices and their global ids. */
static void pair_vertices(const orc_scene *s, const pair_t *p, const double *x, double X[12], int gv[4], double *eps_x) {
    if (p->type == 0) {
        gv[0] = s->voff[p->bi] + p->li;
        for (int k = 0; k < 3; ++k) gv[1 + k] = s->voff[p->bj] + s->tri[3 * (s->toff[p->bj] + p->lj) + k];
        *eps_x = 0.0;
    } else {
        for (int k = 0; k < 2; ++k) {
            gv[k] = s->voff[p->bi] + s->edge[2 * (s->eoff[p->bi] + p->li) + k];
            gv[2 + k] = s->voff[p->bj] + s->edge[2 * (s->eoff[p->bj] + p->lj) + k];
        }
        *eps_x = 1e-3 * s->erest2[s->eoff[p->bi] + p->li] * s->erest2[s->eoff[p->bj] + p->lj];
    }
    for (int v = 0; v < 4; ++v)
        for (int k = 0; k < 3; ++k) X[3 * v + k] = x[3 * gv[v] + k];
}

static void pair_bodies(const pair_t *p, int bod[4]) {
    if (p->type == 0) { bod[0] = p->bi; bod[1] = bod[2] = bod[3] = p->bj; }
    else { bod[0] = bod[1] = p->bi; bod[2] = bod[3] = p->bj; }
}

/* Inertia + orthogonality of one slot: (1/kappa_b)(1/2 |q - q~|_M^2 + h^2 E_orth). */
static double slot_energy(const local_t *L, int sl, const double *q12) {
    const orc_scene *s = L->s;
    int b = L->body[sl];
    const double *S = s->S + 9 * b, *qt = L->qtil + 12 * sl;
    double d[12];
    for (int i = 0; i < 12; ++i) d[i] = q12[i] - qt[i];
    double E = 0.5 * s->mass[b] * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) {
        const double *a = d + 3 + 3 * k;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) E += 0.5 * a[i] * S[3 * i + j] * a[j];
    }
    E += L->h * L->h * orc_orth(q12, s->kappa[b], s->vol[b], NULL, NULL);
    E /= kappa_b(L, b);
    if (L->shared[sl]) {
        double acc = 0.0;
        for (int i = 0; i < 12; ++i) {
            double r = q12[i] - L->z[12 * sl + i] + L->u[12 * sl + i];
            acc += r * r;
        }
        E += 0.5 * L->rho[sl] * acc;
    }
    return E;
}

/* Objective of Eq. 5 at the slot configuration qs (constant -rho/2|u|^2 term
 * dropped).  The barrier sum runs over every pair closer than dhat: the
 * candidates at qs, then the distance test.  +inf when any pair touches. */
static double local_energy(local_t *L, const double *qs) {
    orc_scene *s = L->s;
    double E = 0.0, h2 = L->h * L->h;
    for (int sl = 0; sl < L->ns; ++sl) E += slot_energy(L, sl, qs + 12 * sl);
    local_positions(L, qs, L->x0);
    pairvec pv = {0, 0, 0};
    if (enumerate_pairs(s, L->objs, L->nobj, L->x0, NULL, L->dhat, &pv)) { free(pv.a); return ORC_INF; }
    for (int64_t k = 0; k < pv.n; ++k) {
        double X[12], eps_x, e;
        int gv[4];
        pair_vertices(s, &pv.a[k], L->x0, X, gv, &eps_x);
        double d = orc_pair(pv.a[k].type, X, L->dhat, L->kB, eps_x, &e, NULL, NULL, NULL);
        if (!(d > 0.0)) { free(pv.a); return ORC_INF; }
        if (d < L->dhat) E += h2 / kappa_c(L, pv.a[k].bi, pv.a[k].bj) * e;
    }
    free(pv.a);
    for (int sl = 0; sl < L->ns; ++sl) {
        int b = L->body[sl];
        for (int v = 0; v < s->nv[b]; ++v)
            for (int pl = 0; pl < s->np; ++pl) {
                double d = s->psg[pl] * L->x0[3 * (s->voff[b] + v) + s->pax[pl]] - s->poff[pl];
                if (!(d > 0.0)) return ORC_INF;
                if (d < L->dhat) {
                    double bb[3];
                    orc_barrier(d, L->dhat, bb);
                    E += h2 / kappa_b(L, b) * L->kB * bb[0];
                }
            }
    }
    return E;
}

/* block-sparse symmetric Hessian: diagonal blocks per slot + upper blocks */
typedef struct { int a, b; double blk[144]; } offblk_t;
typedef struct { double *diag; offblk_t *off; int noff, capoff; int *rowhead; int *next; } bsr_t;

static double *bsr_block(bsr_t *H, int a, int b) {
    if (a == b) return H->diag + 144 * (size_t)a;
    for (int k = H->rowhead[a]; k >= 0; k = H->next[k])
        if (H->off[k].b == b) return H->off[k].blk;
    if (H->noff == H->capoff) {
        int nc = H->capoff ? 2 * H->capoff : 256;
        offblk_t *no = (offblk_t *)realloc(H->off, sizeof(offblk_t) * nc);
        int *nn = (int *)realloc(H->next, sizeof(int) * nc);
        if (!no || !nn) { if (no) H->off = no; if (nn) H->next = nn; return NULL; }
        H->off = no; H->next = nn; H->capoff = nc;
    }
    int k = H->noff++;
    H->off[k].a = a; H->off[k].b = b;
    memset(H->off[k].blk, 0, sizeof(double) * 144);
    H->next[k] = H->rowhead[a];
    H->rowhead[a] = k;
    return H->off[k].blk;
}

/* Add J_v^T Hx J_u (weighted) for the vertex pairs of a contact to the slot
 * blocks; J_v = I3 (x) (1, xbar_v^T) in q order. */
static int scatter_pair(local_t *L, bsr_t *H, double *g, const int gv[4], const int bod[4], const double gx[12],
                        const double Hx[144]) {
    const orc_scene *s = L->s;
    int sl[4];
    double xi[4][4];
    for (int v = 0; v < 4; ++v) {
        sl[v] = L->sob[bod[v]];
        const double *xb = s->xbar + 3 * gv[v];
        xi[v][0] = 1.0; xi[v][1] = xb[0]; xi[v][2] = xb[1]; xi[v][3] = xb[2];
    }
    for (int v = 0; v < 4; ++v) {
        if (sl[v] < 0) continue;
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 4; ++a) g[12 * sl[v] + qidx(k, a)] += gx[3 * v + k] * xi[v][a];
    }
    for (int v = 0; v < 4; ++v)
        for (int u = 0; u < 4; ++u) {
            /* upper blocks only: the (u, v) ordering of a cross-slot pair is the
             * transpose of (v, u) and is represented by the same stored block */
            if (sl[v] < 0 || sl[u] < 0 || sl[v] > sl[u]) continue;
            double *B = bsr_block(H, sl[v], sl[u]);
            if (!B) return -1;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double h = Hx[(3 * v + k) * 12 + 3 * u + l];
                    if (h == 0.0) continue;
                    for (int a = 0; a < 4; ++a)
                        for (int c = 0; c < 4; ++c) {
                            B[qidx(k, a) * 12 + qidx(l, c)] += h * xi[v][a] * xi[u][c];
                        }
                }
        }
    return 0;
}

/* Gradient and projected Hessian of the local objective at qs. */
static int local_assemble(local_t *L, const double *qs, double *g, bsr_t *H) {
    orc_scene *s = L->s;
    double h2 = L->h * L->h;
    int n = 12 * L->ns;
    for (int i = 0; i < n; ++i) g[i] = 0.0;
    memset(H->diag, 0, sizeof(double) * 144 * (size_t)L->ns);
    H->noff = 0;
    for (int i = 0; i < L->ns; ++i) H->rowhead[i] = -1;
    for (int sl = 0; sl < L->ns; ++sl) {
        int b = L->body[sl];
        double kw = 1.0 / kappa_b(L, b);
        const double *q = qs + 12 * sl, *qt = L->qtil + 12 * sl, *S = s->S + 9 * b;
        double *D = H->diag + 144 * sl, *gg = g + 12 * sl;
        for (int k = 0; k < 3; ++k) { gg[k] += kw * s->mass[b] * (q[k] - qt[k]); D[k * 12 + k] += kw * s->mass[b]; }
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i) {
                int r = 3 + 3 * k + i;
                for (int j = 0; j < 3; ++j) {
                    gg[r] += kw * S[3 * i + j] * (q[3 + 3 * k + j] - qt[3 + 3 * k + j]);
                    D[r * 12 + 3 + 3 * k + j] += kw * S[3 * i + j];
                }
            }
        double go[12], Ho[144], H9[81];
        orc_orth(q, s->kappa[b], s->vol[b], go, Ho);
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) H9[i * 9 + j] = Ho[(3 + i) * 12 + 3 + j];
        orc_psd_project(9, H9);
        for (int i = 0; i < 12; ++i) gg[i] += kw * h2 * go[i];
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) D[(3 + i) * 12 + 3 + j] += kw * h2 * H9[i * 9 + j];
        if (L->shared[sl]) {
            for (int i = 0; i < 12; ++i) {
                gg[i] += L->rho[sl] * (q[i] - L->z[12 * sl + i] + L->u[12 * sl + i]);
                D[i * 12 + i] += L->rho[sl];
            }
        }
    }
    local_positions(L, qs, L->x0);
    pairvec pv = {0, 0, 0};
    if (enumerate_pairs(s, L->objs, L->nobj, L->x0, NULL, L->dhat, &pv)) { free(pv.a); return ORC_E_OOM; }
    if (pv.n > L->cand_peak) L->cand_peak = pv.n;
    int64_t nact = 0;
    for (int64_t k = 0; k < pv.n; ++k) {
        double X[12], eps_x, e, gx[12], Hx[144];
        int gv[4], bod[4];
        pair_vertices(s, &pv.a[k], L->x0, X, gv, &eps_x);
        double d = orc_pair(pv.a[k].type, X, L->dhat, L->kB, eps_x, &e, gx, Hx, NULL);
        if (!(d < L->dhat)) continue;
        ++nact;
        double w = h2 / kappa_c(L, pv.a[k].bi, pv.a[k].bj);
        orc_psd_project(12, Hx);
        for (int i = 0; i < 12; ++i) gx[i] *= w;
        for (int i = 0; i < 144; ++i) Hx[i] *= w;
        pair_bodies(&pv.a[k], bod);
        if (scatter_pair(L, H, g, gv, bod, gx, Hx)) { free(pv.a); return ORC_E_OOM; }
    }
    free(pv.a);
    for (int sl = 0; sl < L->ns; ++sl) {
        int b = L->body[sl];
        for (int v = 0; v < s->nv[b]; ++v)
            for (int pl = 0; pl < s->np; ++pl) {
                int gvx = s->voff[b] + v, ax = s->pax[pl];
                double d = s->psg[pl] * L->x0[3 * gvx + ax] - s->poff[pl];
                if (!(d < L->dhat)) continue;
                ++nact;
                double bb[3];
                orc_barrier(d, L->dhat, bb);
                /* d = sign * x[axis] - offset: gradient sign * e_axis, Hessian b'' e e^T (PSD) */
                double w = h2 / kappa_b(L, b) * L->kB;
                double gax = w * bb[1] * s->psg[pl], hax = w * bb[2];
                double xi[4] = {1.0, s->xbar[3 * gvx], s->xbar[3 * gvx + 1], s->xbar[3 * gvx + 2]};
                double *D = H->diag + 144 * sl;
                for (int a = 0; a < 4; ++a) g[12 * sl + qidx(ax, a)] += gax * xi[a];
                for (int a = 0; a < 4; ++a)
                    for (int c = 0; c < 4; ++c) D[qidx(ax, a) * 12 + qidx(ax, c)] += hax * xi[a] * xi[c];
            }
    }
    if (nact > L->act_peak) L->act_peak = nact;
    return ORC_OK;
}

/* dense Cholesky solve of H x = rhs (H n x n, overwritten) */
static int cholesky_solve(int n, double *H, double *x) {
    for (int j = 0; j < n; ++j) {
        double s = H[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= H[(size_t)j * n + k] * H[(size_t)j * n + k];
        if (!(s > 0.0)) return ORC_E_NOT_SPD;
        double ljj = sqrt(s);
        H[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = H[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= H[(size_t)i * n + k] * H[(size_t)j * n + k];
            H[(size_t)i * n + j] = t / ljj;
        }
    }
    for (int i = 0; i < n; ++i) {
        double t = x[i];
        for (int k = 0; k < i; ++k) t -= H[(size_t)i * n + k] * x[k];
        x[i] = t / H[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = x[i];
        for (int k = i + 1; k < n; ++k) t -= H[(size_t)k * n + i] * x[k];
        x[i] = t / H[(size_t)i * n + i];
    }
    return ORC_OK;
}

static void bsr_matvec(const bsr_t *H, int ns, const double *x, double *y) {
    for (int i = 0; i < 12 * ns; ++i) y[i] = 0.0;
    for (int a = 0; a < ns; ++a) {
        const double *D = H->diag + 144 * (size_t)a;
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) y[12 * a + i] += D[i * 12 + j] * x[12 * a + j];
    }
    for (int k = 0; k < H->noff; ++k) {
        int a = H->off[k].a, b = H->off[k].b;
        const double *B = H->off[k].blk;
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) {
                y[12 * a + i] += B[i * 12 + j] * x[12 * b + j];
                y[12 * b + j] += B[i * 12 + j] * x[12 * a + i];
            }
    }
}

/* Solve H dx = -g: dense Cholesky up to 2000 unknowns, otherwise block-Jacobi
 * preconditioned CG to a relative residual of 1e-12. */
static int local_linear_solve(int ns, bsr_t *H, const double *g, double *dx) {
    int n = 12 * ns;
    if (n <= 2000) {
        double *M = (double *)calloc((size_t)n * n, sizeof(double));
        if (!M) return ORC_E_OOM;
        for (int a = 0; a < ns; ++a)
            for (int i = 0; i < 12; ++i)
                for (int j = 0; j < 12; ++j) M[(size_t)(12 * a + i) * n + 12 * a + j] = H->diag[144 * (size_t)a + i * 12 + j];
        for (int k = 0; k < H->noff; ++k) {
            int a = H->off[k].a, b = H->off[k].b;
            for (int i = 0; i < 12; ++i)
                for (int j = 0; j < 12; ++j) {
                    M[(size_t)(12 * a + i) * n + 12 * b + j] += H->off[k].blk[i * 12 + j];
                    M[(size_t)(12 * b + j) * n + 12 * a + i] += H->off[k].blk[i * 12 + j];
                }
        }
        for (int i = 0; i < n; ++i) dx[i] = -g[i];
        int rc = cholesky_solve(n, M, dx);
        free(M);
        return rc;
    }
    double *Pinv = (double *)malloc(sizeof(double) * 144 * (size_t)ns);
    double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *Ap = (double *)malloc(sizeof(double) * n);
    if (!Pinv || !r || !z || !p || !Ap) { free(Pinv); free(r); free(z); free(p); free(Ap); return ORC_E_OOM; }
    int rc = ORC_OK;
    for (int a = 0; a < ns && rc == ORC_OK; ++a) { /* invert each diagonal block by Cholesky */
        double B[144];
        for (int c = 0; c < 12; ++c) {
            memcpy(B, H->diag + 144 * (size_t)a, sizeof B);
            double e[12] = {0};
            e[c] = 1.0;
            rc = cholesky_solve(12, B, e);
            for (int i = 0; i < 12; ++i) Pinv[144 * (size_t)a + i * 12 + c] = e[i];
        }
    }
    double r0 = 0.0, rz = 0.0;
    for (int i = 0; i < n; ++i) { dx[i] = 0.0; r[i] = -g[i]; r0 += r[i] * r[i]; }
    for (int a = 0; a < ns; ++a)
        for (int i = 0; i < 12; ++i) {
            double t = 0.0;
            for (int j = 0; j < 12; ++j) t += Pinv[144 * (size_t)a + i * 12 + j] * r[12 * a + j];
            z[12 * a + i] = t;
        }
    for (int i = 0; i < n; ++i) { p[i] = z[i]; rz += r[i] * z[i]; }
    for (int it = 0; it < 20000 && rc == ORC_OK && r0 > 0.0; ++it) {
        bsr_matvec(H, ns, p, Ap);
        double pAp = 0.0;
        for (int i = 0; i < n; ++i) pAp += p[i] * Ap[i];
        double alpha = rz / pAp, rr = 0.0;
        for (int i = 0; i < n; ++i) { dx[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; rr += r[i] * r[i]; }
        if (rr <= 1e-24 * r0) break;
        for (int a = 0; a < ns; ++a)
            for (int i = 0; i < 12; ++i) {
                double t = 0.0;
                for (int j = 0; j < 12; ++j) t += Pinv[144 * (size_t)a + i * 12 + j] * r[12 * a + j];
                z[12 * a + i] = t;
            }
        double rzn = 0.0;
        for (int i = 0; i < n; ++i) rzn += r[i] * z[i];
        double beta = rzn / rz;
        rz = rzn;
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    free(Pinv); free(r); free(z); free(p); free(Ap);
    return rc;
}

/* Smallest time of impact along x0 -> x1 over the swept candidates of the
 * local problem and the vertex-plane pairs. */
static double local_toi(local_t *L, const double *x0, const double *x1, int64_t *nswept) {
    orc_scene *s = L->s;
    pairvec pv = {0, 0, 0};
    if (enumerate_pairs(s, L->objs, L->nobj, x0, x1, L->dhat, &pv)) { free(pv.a); return 0.0; }
    if (nswept) *nswept = pv.n;
    double toi = 1.0;
    for (int64_t k = 0; k < pv.n; ++k) {
        double X[12], X1[12], dX[12], eps_x;
        int gv[4];
        pair_vertices(s, &pv.a[k], x0, X, gv, &eps_x);
        pair_vertices(s, &pv.a[k], x1, X1, gv, &eps_x);
        for (int i = 0; i < 12; ++i) dX[i] = X1[i] - X[i];
        double t = orc_ccd(pv.a[k].type, X, dX, L->accd_s, L->accd_c);
        if (t < toi) toi = t;
    }
    free(pv.a);
    for (int sl = 0; sl < L->ns; ++sl) {
        int b = L->body[sl];
        for (int v = 0; v < s->nv[b]; ++v)
            for (int pl = 0; pl < s->np; ++pl) {
                int g = s->voff[b] + v, ax = s->pax[pl];
                double d0 = s->psg[pl] * x0[3 * g + ax] - s->poff[pl];
                double dd = s->psg[pl] * (x1[3 * g + ax] - x0[3 * g + ax]);
                double t = orc_ccd_plane(d0, dd, L->accd_s);
                if (t < toi) toi = t;
            }
    }
    return toi;
}

/* Projected Newton on Eq. 5 from L->q (feasible):
 *   active set at q, g and PSD-projected H, solve H dq = -g;
 *   stop when |dq|_inf / (h l) < eps_N (before the line search);
 *   alpha = min(1, TOI along q -> q + dq); halve while E(q + alpha dq) > E(q);
 *   q <- q + alpha dq.
 * A solve that spends max_newton iterations without meeting eps_N marks the
 * partition (the step then reports ORC_NEWTON_MAXITER unless a worse status
 * applies). */
static int local_solve(local_t *L) {
    int n = 12 * L->ns, rc = ORC_OK, converged = 0;
    if (n == 0) return ORC_OK;
    double *g = (double *)malloc(sizeof(double) * n), *dq = (double *)malloc(sizeof(double) * n);
    double *qn = (double *)malloc(sizeof(double) * n);
    bsr_t H = {0};
    H.diag = (double *)malloc(sizeof(double) * 144 * (size_t)L->ns);
    H.rowhead = (int *)malloc(sizeof(int) * L->ns);
    if (!g || !dq || !qn || !H.diag || !H.rowhead) { rc = ORC_E_OOM; goto done; }
    for (int it = 0; it < L->max_newton; ++it) {
        rc = local_assemble(L, L->q, g, &H);
        if (rc) break;
        rc = local_linear_solve(L->ns, &H, g, dq);
        if (rc) break;
        L->newton_iters++;
        double dmax_ = 0.0;
        for (int i = 0; i < n; ++i) dmax_ = dmax(dmax_, fabs(dq[i]));
        if (dmax_ / (L->h * L->l) < L->epsN) { converged = 1; break; }
        for (int i = 0; i < n; ++i) qn[i] = L->q[i] + dq[i];
        local_positions(L, L->q, L->x0);
        local_positions(L, qn, L->x1);
        double alpha = local_toi(L, L->x0, L->x1, NULL);
        double E0 = local_energy(L, L->q);
        for (int nh = 0;; ++nh) {
            for (int i = 0; i < n; ++i) qn[i] = L->q[i] + alpha * dq[i];
            double E1 = local_energy(L, qn);
            if (E1 <= E0 || nh >= L->max_halv) break;
            alpha *= 0.5;
        }
        memcpy(L->q, qn, sizeof(double) * n);
    }
    if (rc == ORC_OK && !converged) L->maxed = 1;
done:
    free(g); free(dq); free(qn); free(H.diag); free(H.rowhead); free(H.off); free(H.next);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* O7: partition, consensus ADMM, merge                                      */
/* ------------------------------------------------------------------------ */

static void body_aabb(const orc_scene *s, int b, const double *q12, double lo[3], double hi[3]) {
    const double *p = q12, *A = q12 + 3;
    for (int k = 0; k < 3; ++k) { lo[k] = ORC_INF; hi[k] = -ORC_INF; }
    for (int v = 0; v < s->nv[b]; ++v) {
        const double *xb = s->xbar + 3 * (s->voff[b] + v);
        for (int k = 0; k < 3; ++k) {
            double x = p[k] + (A[3 * k] * xb[0] + A[3 * k + 1] * xb[1] + A[3 * k + 2] * xb[2]);
            lo[k] = dmin(lo[k], x);
            hi[k] = dmax(hi[k], x);
        }
    }
}

/* Slab partition of Fig. 2 / Sec. 4: planes gamma_1..gamma_{N-1} along the
 * axis; overlap width w = max(alpha v_max h, w_min) (v_max = largest |dp/dt|
 * over dynamic bodies, w_min = smallest dynamic body AABB diagonal unless
 * given); body b is held by slab i iff its AABB along the axis meets
 * [gamma_i - w/2, gamma_{i+1} + w/2] (outer slabs unbounded). */
int orc_partition(orc_scene *s, const orc_params *P, uint64_t *mask, double *w_out) {
    int N = P->n_slabs < 1 ? 1 : P->n_slabs, ax = P->axis;
    if (N > 64 || ax < 0 || ax > 2) return ORC_E_INVALID;
    if (N == 1) {
        for (int b = 0; b < s->nb; ++b) mask[b] = 1;
        if (w_out) *w_out = 0.0;
        return ORC_OK;
    }
    double Lo = ORC_INF, Hi = -ORC_INF, vmax = 0.0, wmin = ORC_INF;
    double *lo = (double *)malloc(sizeof(double) * s->nb), *hi = (double *)malloc(sizeof(double) * s->nb);
    if (!lo || !hi) { free(lo); free(hi); return ORC_E_OOM; }
    for (int b = 0; b < s->nb; ++b) {
        if (!is_dof(s->kind[b])) continue;
        double l3[3], h3[3];
        body_aabb(s, b, s->q + 12 * b, l3, h3);
        lo[b] = l3[ax]; hi[b] = h3[ax];
        Lo = dmin(Lo, lo[b]); Hi = dmax(Hi, hi[b]);
        double dg[3] = {h3[0] - l3[0], h3[1] - l3[1], h3[2] - l3[2]};
        wmin = dmin(wmin, sqrt(dot3(dg, dg)));
        const double *vp = s->v + 12 * b;
        vmax = dmax(vmax, sqrt(dot3(vp, vp)));
    }
    double gam[65];
    for (int i = 1; i < N; ++i) gam[i] = P->planes ? P->planes[i - 1] : Lo + (Hi - Lo) * (double)i / (double)N;
    if (P->w_min > 0.0) wmin = P->w_min;
    double w = dmax(P->alpha_w * vmax * P->h, wmin);
    for (int b = 0; b < s->nb; ++b) {
        mask[b] = 0;
        if (!is_dof(s->kind[b])) continue;
        for (int i = 0; i < N; ++i) {
            double rlo = i == 0 ? -ORC_INF : gam[i] - 0.5 * w;
            double rhi = i == N - 1 ? ORC_INF : gam[i + 1] + 0.5 * w;
            if (lo[b] <= rhi && hi[b] >= rlo) mask[b] |= (uint64_t)1 << i;
        }
    }
    free(lo); free(hi);
    if (w_out) *w_out = w;
    return ORC_OK;
}

static void local_free(local_t *L) {
    free(L->body); free(L->sob); free(L->objs); free(L->q); free(L->qtil); free(L->z); free(L->u); free(L->rho);
    free(L->shared); free(L->x0); free(L->x1);
}

/* Build the local problem of partition `part` (slots = dynamic bodies whose
 * mask has the bit), starting from the state array q_all. */
static int local_init(local_t *L, orc_scene *s, const uint64_t *mask, int part, const double *q_all,
                      const double *qtil_all, const orc_params *P, double kB, double l) {
    memset(L, 0, sizeof *L);
    L->s = s; L->mask = mask;
    L->h = P->h; L->dhat = P->dhat; L->kB = kB; L->epsN = P->newton_tol; L->l = l;
    L->accd_s = P->accd_s; L->accd_c = P->accd_c; L->max_newton = P->max_newton; L->max_halv = P->max_halvings;
    int ns = 0;
    for (int b = 0; b < s->nb; ++b)
        if (is_dof(s->kind[b]) && (mask[b] >> part & 1)) ++ns;
    L->ns = ns;
    L->body = (int *)malloc(sizeof(int) * (ns + 1));
    L->sob = (int *)malloc(sizeof(int) * s->nb);
    L->objs = (int *)malloc(sizeof(int) * s->nb);
    L->q = (double *)calloc(12 * (size_t)(ns + 1), sizeof(double));
    L->qtil = (double *)calloc(12 * (size_t)(ns + 1), sizeof(double));
    L->z = (double *)calloc(12 * (size_t)(ns + 1), sizeof(double));
    L->u = (double *)calloc(12 * (size_t)(ns + 1), sizeof(double));
    L->rho = (double *)calloc((size_t)(ns + 1), sizeof(double));
    L->shared = (int *)calloc((size_t)(ns + 1), sizeof(int));
    L->x0 = (double *)malloc(sizeof(double) * 3 * (s->V ? s->V : 1));
    L->x1 = (double *)malloc(sizeof(double) * 3 * (s->V ? s->V : 1));
    if (!L->body || !L->sob || !L->objs || !L->q || !L->qtil || !L->z || !L->u || !L->rho || !L->shared || !L->x0 ||
        !L->x1) return ORC_E_OOM;
    int k = 0;
    for (int b = 0; b < s->nb; ++b) {
        L->sob[b] = -1;
        if (is_dof(s->kind[b]) && (mask[b] >> part & 1)) {
            L->sob[b] = k;
            L->body[k] = b;
            memcpy(L->q + 12 * k, q_all + 12 * b, sizeof(double) * 12);
            memcpy(L->qtil + 12 * k, qtil_all + 12 * b, sizeof(double) * 12);
            L->shared[k] = popcount64(mask[b]) >= 2;
            ++k;
        }
    }
    L->nobj = 0;
    for (int i = 0; i < ns; ++i) L->objs[L->nobj++] = L->body[i];
    for (int b = 0; b < s->nb; ++b)
        if (!is_dof(s->kind[b])) L->objs[L->nobj++] = b;
    return ORC_OK;
}

static double scene_scale(const orc_scene *s) {
    double lo[3] = {ORC_INF, ORC_INF, ORC_INF}, hi[3] = {-ORC_INF, -ORC_INF, -ORC_INF};
    for (int b = 0; b < s->nb; ++b) {
        double l3[3], h3[3];
        body_aabb(s, b, s->q + 12 * b, l3, h3);
        for (int k = 0; k < 3; ++k) { lo[k] = dmin(lo[k], l3[k]); hi[k] = dmax(hi[k], h3[k]); }
    }
    double d[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    return sqrt(dot3(d, d));
}

/* Minimum distance over all candidate pairs and vertex-plane pairs within
 * dhat at the scene's current state (dhat when none is that close). */
static double scene_min_distance(orc_scene *s, double dhat) {
    double *x = (double *)malloc(sizeof(double) * 3 * (s->V ? s->V : 1));
    int *all = (int *)malloc(sizeof(int) * s->nb);
    pairvec pv = {0, 0, 0};
    double md = dhat;
    if (!x || !all) { free(x); free(all); return -1.0; }
    orc_vertices(s, NULL, x);
    for (int b = 0; b < s->nb; ++b) all[b] = b;
    if (!enumerate_pairs(s, all, s->nb, x, NULL, dhat, &pv)) {
        for (int64_t k = 0; k < pv.n; ++k) {
            double X[12], eps_x;
            int gv[4], ty;
            double beta[2];
            pair_vertices(s, &pv.a[k], x, X, gv, &eps_x);
            md = dmin(md, sqrt(orc_dist_type(pv.a[k].type, X, &ty, beta)));
        }
    }
    for (int b = 0; b < s->nb; ++b) {
        if (!is_dof(s->kind[b])) continue;
        for (int v = 0; v < s->nv[b]; ++v)
            for (int pl = 0; pl < s->np; ++pl)
                md = dmin(md, s->psg[pl] * x[3 * (s->voff[b] + v) + s->pax[pl]] - s->poff[pl]);
    }
    free(pv.a); free(x); free(all);
    return md;
}

/* Residual-driven penalty of one shared body (Sec. 4.3).  r is its primal
 * residual (Eq. 9) and s its dual residual (Eq. 10): rho grows by the factor
 * tau when r > mu s, shrinks by tau when s > mu r, and stays otherwise (the
 * equality cases included); the result is clamped to
 * [sigma_min rho0, sigma_max rho0], rho0 = beta m being the body's initial
 * penalty.  The scaled dual u = y / rho must carry the unscaled dual y across
 * the change (Boyd et al. 2011, Sec. 3.4.1), so the caller multiplies every
 * replica's u by *u_scale = rho / rho_new. */
double orc_rho_update(double r, double s, double rho, double rho0, double tau, double mu, double sigma_min,
                      double sigma_max, double *u_scale) {
    double nw = rho;
    if (r > mu * s) nw = rho * tau;
    else if (s > mu * r) nw = rho / tau;
    nw = dmin(dmax(nw, sigma_min * rho0), sigma_max * rho0);
    if (u_scale) *u_scale = rho / nw;
    return nw;
}

int orc_admm_trace(orc_scene *s, double *buf, int64_t cap) {
    if (!s || cap < 0 || (cap > 0 && !buf)) return ORC_E_INVALID;
    s->trace = buf;
    s->trace_cap = cap;
    s->trace_n = 0;
    return ORC_OK;
}

int64_t orc_admm_trace_count(const orc_scene *s) { return s ? s->trace_n : 0; }

/* Trace records of one round (see orc_admm_trace): with b >= 0 one record
 * per replica of shared body b (its residuals, the penalty before and after
 * the update, its z of this and the previous round, u before and after the
 * rescale); with b < 0 one record per internal slot of every partition (q
 * only), so that a record set holds each partition's whole configuration. */
static void admm_trace_round(orc_scene *s, local_t *parts, int N, int k, int b, double r, double sb, double nw,
                             double scale, const double *zprev, const double *z) {
    for (int i = 0; i < N; ++i)
        for (int sl = 0; sl < parts[i].ns; ++sl) {
            int body = parts[i].body[sl];
            if (b >= 0 ? body != b : parts[i].shared[sl]) continue;
            if (s->trace_n < s->trace_cap) {
                double *rec = s->trace + ORC_TRACE_REC * s->trace_n;
                memset(rec, 0, sizeof(double) * ORC_TRACE_REC);
                rec[0] = k; rec[1] = body; rec[2] = i; rec[3] = b >= 0;
                memcpy(rec + 8, parts[i].q + 12 * sl, sizeof(double) * 12);
                if (b >= 0) {
                    const double *u = parts[i].u + 12 * sl;
                    rec[4] = parts[i].rho[sl]; rec[5] = nw; rec[6] = r; rec[7] = sb;
                    memcpy(rec + 20, zprev + 12 * b, sizeof(double) * 12);
                    memcpy(rec + 32, z + 12 * b, sizeof(double) * 12);
                    memcpy(rec + 44, u, sizeof(double) * 12);
                    for (int j = 0; j < 12; ++j) rec[56 + j] = u[j] * scale;
                }
            }
            ++s->trace_n;
        }
}

/* One time step (Alg. 1 with every partition on this thread):
 *   q~ (O2); partition (O7); z = q~, u = 0, rho = beta m;
 *   k = 1..K+1: for k > 1 consensus z (Eq. 6), dual u (Eq. 7), residuals
 *   r, s (Eq. 9-10), Delta_i = |q_i^k - q_i^{k-1}|_inf, merge check (CCD from
 *   q_i to q^_i, Sec. 4.2); stop when all three are below theta h l and every
 *   TOI is 1; else rho update (Sec. 4.3, u rescaled by rho_old/rho_new);
 *   local solves (Eq. 5).  Without shared bodies each partition solves once.
 *   After K rounds: accept z when the merge check passes (ADMM_MAXITER), else
 *   re-solve the step on one partition (FELL_BACK). */
#define ORC_SPLIT_REQUEST 100 /* internal: the step is to be retaken as two half steps */

static int step_once(orc_scene *s, const orc_params *P, orc_stats *st) {
    int nb = s->nb, rc = ORC_OK;
    orc_stats zero;
    memset(&zero, 0, sizeof zero);
    if (st) *st = zero;
    double *qt = (double *)malloc(sizeof(double) * 12 * nb), *qtil = (double *)malloc(sizeof(double) * 12 * nb);
    double *qnew = (double *)malloc(sizeof(double) * 12 * nb), *z = (double *)calloc(12 * (size_t)nb, sizeof(double));
    double *zprev = (double *)calloc(12 * (size_t)nb, sizeof(double)), *rho0 = (double *)calloc(nb, sizeof(double));
    double *rhob = (double *)calloc(nb, sizeof(double)), *sbody = (double *)calloc(nb, sizeof(double));
    uint64_t *mask = (uint64_t *)calloc(nb, sizeof(uint64_t)), *ones = (uint64_t *)calloc(nb, sizeof(uint64_t));
    local_t *parts = NULL;
    double **qprev = NULL;
    int N = P->n_slabs < 1 ? 1 : P->n_slabs;
    if (!qt || !qtil || !qnew || !z || !zprev || !rho0 || !rhob || !sbody || !mask || !ones) { rc = ORC_E_OOM; goto out; }
    memcpy(qt, s->q, sizeof(double) * 12 * nb);
    /* O2: q~ = q + h qdot + h^2 M^-1 f_ext; gravity only, xbar centred -> (g, 0) */
    for (int b = 0; b < nb; ++b) {
        for (int i = 0; i < 12; ++i) qtil[12 * b + i] = qt[12 * b + i] + P->h * s->v[12 * b + i];
        if (s->kind[b] == ORC_DYNAMIC)
            for (int k = 0; k < 3; ++k) qtil[12 * b + k] += P->h * P->h * s->g[k];
        else if (s->kind[b] == ORC_KINEMATIC)
            kinematic_pose(qt + 12 * b, s->v + 12 * b, s->omega + 3 * b, P->h, qtil + 12 * b);
        else memcpy(qtil + 12 * b, qt + 12 * b, sizeof(double) * 12);
        ones[b] = 1;
    }
    double l = scene_scale(s), kB = P->kappa_barrier;
    if (!(kB > 0.0)) {
        double msum = 0.0;
        int nd = 0;
        for (int b = 0; b < nb; ++b)
            if (s->kind[b] == ORC_DYNAMIC) { msum += s->mass[b]; ++nd; }
        kB = 10.0 * (nd ? msum / nd : 1.0) * sqrt(dot3(s->g, s->g)) / P->dhat;
    }
    double w = 0.0;
    rc = orc_partition(s, P, mask, &w);
    if (rc) goto out;
    int nshared = 0, nslots = 0;
    for (int b = 0; b < nb; ++b) {
        if (!is_dof(s->kind[b])) continue;
        int c = popcount64(mask[b]);
        nslots += c;
        if (c >= 2) ++nshared;
    }
    parts = (local_t *)calloc(N, sizeof(local_t));
    qprev = (double **)calloc(N, sizeof(double *));
    if (!parts || !qprev) { rc = ORC_E_OOM; goto out; }
    for (int i = 0; i < N; ++i) {
        rc = local_init(&parts[i], s, mask, i, qt, qtil, P, kB, l);
        if (rc) goto out;
        qprev[i] = (double *)malloc(sizeof(double) * 12 * (parts[i].ns + 1));
        if (!qprev[i]) { rc = ORC_E_OOM; goto out; }
    }
    for (int b = 0; b < nb; ++b) {
        memcpy(z + 12 * b, qtil + 12 * b, sizeof(double) * 12);
        rho0[b] = rhob[b] = P->beta * s->mass[b];
    }
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < parts[i].ns; ++k) {
            int b = parts[i].body[k];
            memcpy(parts[i].z + 12 * k, z + 12 * b, sizeof(double) * 12);
            parts[i].rho[k] = rhob[b];
        }
    int status = ORC_OK, admm = 0, converged = 0, merge_ok = 1;
    double rinf = 0.0, sinf = 0.0, dinf = 0.0;
    if (nshared == 0) {
        for (int i = 0; i < N; ++i) {
            rc = local_solve(&parts[i]);
            if (rc) goto out;
        }
        admm = 1;
        converged = 1;
    } else {
        int K = P->max_admm < 1 ? 1 : P->max_admm;
        for (int k = 1; k <= K + 1; ++k) {
            if (k > 1) {
                rinf = sinf = dinf = 0.0;
                memcpy(zprev, z, sizeof(double) * 12 * nb);
                double *rb = (double *)calloc(nb, sizeof(double));
                if (!rb) { rc = ORC_E_OOM; goto out; }
                for (int b = 0; b < nb; ++b) {
                    if (!is_dof(s->kind[b]) || popcount64(mask[b]) < 2) continue;
                    double num[12] = {0}, den = 0.0;
                    for (int i = 0; i < N; ++i) {
                        int sl = parts[i].sob[b];
                        if (sl < 0) continue;
                        for (int j = 0; j < 12; ++j) num[j] += parts[i].rho[sl] * (parts[i].q[12 * sl + j] + parts[i].u[12 * sl + j]);
                        den += parts[i].rho[sl];
                    }
                    double sb = 0.0;
                    for (int j = 0; j < 12; ++j) {
                        z[12 * b + j] = num[j] / den;
                        sb = dmax(sb, fabs(z[12 * b + j] - zprev[12 * b + j]));
                    }
                    double r = 0.0;
                    for (int i = 0; i < N; ++i) {
                        int sl = parts[i].sob[b];
                        if (sl < 0) continue;
                        for (int j = 0; j < 12; ++j) {
                            double ri = parts[i].q[12 * sl + j] - z[12 * b + j];
                            parts[i].u[12 * sl + j] += ri;
                            r = dmax(r, fabs(ri));
                        }
                    }
                    rb[b] = r;
                    sbody[b] = sb;
                    rinf = dmax(rinf, r);
                    sinf = dmax(sinf, sb);
                }
                for (int i = 0; i < N; ++i)
                    for (int j = 0; j < 12 * parts[i].ns; ++j) dinf = dmax(dinf, fabs(parts[i].q[j] - qprev[i][j]));
                /* merge check: CCD from q_i to q^_i (shared slots moved to z) */
                merge_ok = 1;
                for (int i = 0; i < N && merge_ok; ++i) {
                    local_t *L = &parts[i];
                    double *qh = (double *)malloc(sizeof(double) * 12 * (L->ns + 1));
                    if (!qh) { free(rb); rc = ORC_E_OOM; goto out; }
                    memcpy(qh, L->q, sizeof(double) * 12 * L->ns);
                    for (int sl = 0; sl < L->ns; ++sl)
                        if (L->shared[sl]) memcpy(qh + 12 * sl, z + 12 * L->body[sl], sizeof(double) * 12);
                    local_positions(L, L->q, L->x0);
                    local_positions(L, qh, L->x1);
                    double toi = local_toi(L, L->x0, L->x1, NULL);
                    if (toi != 1.0) merge_ok = 0;
                    free(qh);
                }
                double tol = P->theta * P->h * l;
                if (dinf < tol && rinf < tol && sinf < tol && merge_ok) { converged = 1; free(rb); break; }
                if (k == K + 1) { free(rb); break; }
                /* rho update (Sec. 4.3) per shared body, recorded first when tracing */
                for (int b = 0; b < nb; ++b) {
                    if (!is_dof(s->kind[b]) || popcount64(mask[b]) < 2) continue;
                    double scale = 1.0;
                    double nw = P->rho_adaptive ? orc_rho_update(rb[b], sbody[b], rhob[b], rho0[b], P->tau, P->mu,
                                                                 P->sigma_min, P->sigma_max, &scale)
                                                : rhob[b];
                    if (s->trace) admm_trace_round(s, parts, N, k, b, rb[b], sbody[b], nw, scale, zprev, z);
                    rhob[b] = nw;
                    for (int i = 0; i < N; ++i) {
                        int sl = parts[i].sob[b];
                        if (sl < 0) continue;
                        for (int j = 0; j < 12; ++j) parts[i].u[12 * sl + j] *= scale;
                        parts[i].rho[sl] = nw;
                    }
                }
                if (s->trace) admm_trace_round(s, parts, N, k, -1, 0.0, 0.0, 0.0, 1.0, zprev, z);
                free(rb);
                for (int i = 0; i < N; ++i)
                    for (int sl = 0; sl < parts[i].ns; ++sl)
                        memcpy(parts[i].z + 12 * sl, z + 12 * parts[i].body[sl], sizeof(double) * 12);
            }
            for (int i = 0; i < N; ++i) {
                memcpy(qprev[i], parts[i].q, sizeof(double) * 12 * parts[i].ns);
                rc = local_solve(&parts[i]);
                if (rc) goto out;
            }
            ++admm;
        }
        if (!converged) status = merge_ok ? ORC_ADMM_MAXITER : ORC_FELL_BACK;
    }
    /* merge (Alg. 1 end of frame): shared bodies take z, internal ones their
     * only replica; colliders keep their state */
    memcpy(qnew, qt, sizeof(double) * 12 * nb);
    for (int i = 0; i < N; ++i)
        for (int sl = 0; sl < parts[i].ns; ++sl) {
            int b = parts[i].body[sl];
            if (parts[i].shared[sl]) memcpy(qnew + 12 * b, z + 12 * b, sizeof(double) * 12);
            else memcpy(qnew + 12 * b, parts[i].q + 12 * sl, sizeof(double) * 12);
        }
    int newton = 0, maxed = 0;
    int64_t cpk = 0, apk = 0;
    for (int i = 0; i < N; ++i) {
        newton += parts[i].newton_iters;
        maxed |= parts[i].maxed;
        if (parts[i].cand_peak > cpk) cpk = parts[i].cand_peak;
        if (parts[i].act_peak > apk) apk = parts[i].act_peak;
    }
    if (status == ORC_FELL_BACK && P->dt_split_max > 0) {
        /* adaptive time stepping on a blocked merge (reading of Sec. 4.2, Fig. 4:
         * a smaller step lets the replicas merge): leave the state untouched and
         * let orc_step retake the step as two steps of h/2 */
        if (st) {
            st->status = status; st->admm_iters = admm; st->n_shared = nshared; st->n_slots = nslots;
            st->merge_ok = merge_ok; st->l = l; st->kappa_barrier = kB; st->w = w;
            int nt = 0;
            for (int i = 0; i < N; ++i) nt += parts[i].newton_iters;
            st->newton_iters = nt;
        }
        rc = ORC_SPLIT_REQUEST;
        goto out;
    }
    if (status == ORC_FELL_BACK) {
        local_t M;
        rc = local_init(&M, s, ones, 0, qt, qtil, P, kB, l);
        if (!rc) rc = local_solve(&M);
        if (!rc)
            for (int sl = 0; sl < M.ns; ++sl) memcpy(qnew + 12 * M.body[sl], M.q + 12 * sl, sizeof(double) * 12);
        newton += M.newton_iters;
        local_free(&M);
        if (rc) goto out;
    }
    for (int b = 0; b < nb; ++b)
        if (is_dof(s->kind[b]))
            for (int i = 0; i < 12; ++i) s->v[12 * b + i] = (qnew[12 * b + i] - qt[12 * b + i]) / P->h;
    memcpy(s->q, qnew, sizeof(double) * 12 * nb);
    double md = scene_min_distance(s, P->dhat);
    if (maxed && status == ORC_OK) status = ORC_NEWTON_MAXITER;
    if (st) {
        st->status = status; st->admm_iters = admm; st->newton_iters = newton; st->n_shared = nshared;
        st->n_slots = nslots; st->merge_ok = merge_ok; st->n_candidates_peak = cpk; st->n_active_peak = apk;
        st->r_inf = rinf; st->s_inf = sinf; st->delta_inf = dinf; st->min_distance = md; st->l = l;
        st->kappa_barrier = kB; st->w = w;
    }
    rc = md > 0.0 ? status : ORC_E_PENETRATION;
out:
    if (parts) for (int i = 0; i < N; ++i) local_free(&parts[i]);
    if (qprev) for (int i = 0; i < N; ++i) free(qprev[i]);
    free(parts); free(qprev);
    free(qt); free(qtil); free(qnew); free(z); free(zprev); free(rho0); free(rhob); free(sbody); free(mask); free(ones);
    return rc;
}

int orc_step(orc_scene *s, const orc_params *P, orc_stats *st) {
    if (!s || !P || P->dt_split_max < 0 || P->dt_split_max > 16) return ORC_E_INVALID;
    orc_stats first;
    int rc = step_once(s, P, &first);
    if (rc != ORC_SPLIT_REQUEST) {
        if (st) *st = first;
        return rc;
    }
    orc_params H = *P;
    H.h = 0.5 * P->h;
    H.dt_split_max = P->dt_split_max - 1;
    orc_stats a, b;
    rc = orc_step(s, &H, &a);
    if (rc < 0) return rc;
    rc = orc_step(s, &H, &b);
    if (rc < 0) return rc;
    if (st) {
        *st = b;
        st->status = ORC_DT_SPLIT;
        st->admm_iters = first.admm_iters + a.admm_iters + b.admm_iters;
        st->newton_iters = first.newton_iters + a.newton_iters + b.newton_iters;
        if (a.n_candidates_peak > st->n_candidates_peak) st->n_candidates_peak = a.n_candidates_peak;
        if (a.n_active_peak > st->n_active_peak) st->n_active_peak = a.n_active_peak;
    }
    return ORC_DT_SPLIT;
}

/* Monolithic objective of Eq. 1 (one partition, kappa = 1, no consensus term)
 * at the dynamic-body configuration q (body order, dynamic bodies only) with
 * predicted state qtil: energy, gradient and PSD-projected Hessian (dense,
 * n x n with n = 12 * #dynamic).  Exposed for the finite-difference pins. */
int orc_objective(orc_scene *s, const orc_params *P, const double *q, const double *qtil, double *E, double *g,
                  double *Hdense) {
    uint64_t *ones = (uint64_t *)malloc(sizeof(uint64_t) * s->nb);
    if (!ones) return ORC_E_OOM;
    for (int b = 0; b < s->nb; ++b) ones[b] = 1;
    double *qa = (double *)calloc(12 * (size_t)s->nb, sizeof(double)), *qt = (double *)calloc(12 * (size_t)s->nb, sizeof(double));
    local_t L;
    int rc = (!qa || !qt) ? ORC_E_OOM : ORC_OK, k = 0;
    if (!rc) {
        memcpy(qa, s->q, sizeof(double) * 12 * s->nb);
        memcpy(qt, s->q, sizeof(double) * 12 * s->nb);
        for (int b = 0; b < s->nb; ++b)
            if (is_dof(s->kind[b])) {
                memcpy(qa + 12 * b, q + 12 * k, sizeof(double) * 12);
                memcpy(qt + 12 * b, qtil + 12 * k, sizeof(double) * 12);
                ++k;
            }
        double kB = P->kappa_barrier;
        rc = local_init(&L, s, ones, 0, qa, qt, P, kB, 1.0);
        if (!rc) {
            if (E) *E = local_energy(&L, L.q);
            if (g || Hdense) {
                int n = 12 * L.ns;
                double *gg = (double *)malloc(sizeof(double) * (n ? n : 1));
                bsr_t H = {0};
                H.diag = (double *)malloc(sizeof(double) * 144 * (size_t)(L.ns ? L.ns : 1));
                H.rowhead = (int *)malloc(sizeof(int) * (L.ns ? L.ns : 1));
                rc = (!gg || !H.diag || !H.rowhead) ? ORC_E_OOM : local_assemble(&L, L.q, gg, &H);
                if (!rc && g) memcpy(g, gg, sizeof(double) * n);
                if (!rc && Hdense) {
                    memset(Hdense, 0, sizeof(double) * (size_t)n * n);
                    for (int a = 0; a < L.ns; ++a)
                        for (int i = 0; i < 12; ++i)
                            for (int j = 0; j < 12; ++j) Hdense[(size_t)(12 * a + i) * n + 12 * a + j] = H.diag[144 * a + i * 12 + j];
                    for (int o = 0; o < H.noff; ++o)
                        for (int i = 0; i < 12; ++i)
                            for (int j = 0; j < 12; ++j) {
                                int a = H.off[o].a, b = H.off[o].b;
                                Hdense[(size_t)(12 * a + i) * n + 12 * b + j] += H.off[o].blk[i * 12 + j];
                                Hdense[(size_t)(12 * b + j) * n + 12 * a + i] += H.off[o].blk[i * 12 + j];
                            }
                }
                free(gg); free(H.diag); free(H.rowhead); free(H.off); free(H.next);
            }
        }
        local_free(&L);
    }
    free(ones); free(qa); free(qt);
    return rc;
}

/* The local objectives F_i of Eq. 3 (partition i's share of Eq. 1: inertia and
 * orthogonality of each slot weighted 1/kappa_b, each contact 1/kappa_c, each
 * plane contact 1/kappa_b) at a consensus point, where every replica sits at
 * the body's own q (z = q, u = 0: the augmented term of Eq. 5 vanishes).
 * Partition membership is the slab rule at the scene's current state; q and
 * qtil give every DOF body ([n_dof][12], body order); barrier stiffness
 * P->kappa_barrier.  E_parts[i] receives F_i (up to cap partitions),
 * g_sum[n_dof][12] the sum over partitions of the gradients of F_i scattered
 * to the bodies, H_sum (dense, 12 n_dof square, or NULL) the sum of their
 * projected Hessians (rho = 0 here, so the augmented term adds nothing to
 * any of them).  Returns the number of partitions, or a negative status. */
int orc_local_objectives(orc_scene *s, const orc_params *P, const double *q, const double *qtil, double *E_parts,
                         int cap, double *g_sum, double *H_sum) {
    int N = P->n_slabs < 1 ? 1 : P->n_slabs;
    uint64_t *mask = (uint64_t *)malloc(sizeof(uint64_t) * s->nb);
    int *dof = (int *)malloc(sizeof(int) * s->nb);
    double *qa = (double *)calloc(12 * (size_t)s->nb, sizeof(double)), *qt = (double *)calloc(12 * (size_t)s->nb, sizeof(double));
    int rc = (!mask || !dof || !qa || !qt) ? ORC_E_OOM : ORC_OK, k = 0;
    if (!rc) rc = orc_partition(s, P, mask, NULL);
    if (!rc) {
        memcpy(qa, s->q, sizeof(double) * 12 * s->nb);
        memcpy(qt, s->q, sizeof(double) * 12 * s->nb);
        for (int b = 0; b < s->nb; ++b) {
            dof[b] = -1;
            if (is_dof(s->kind[b])) {
                memcpy(qa + 12 * b, q + 12 * k, sizeof(double) * 12);
                memcpy(qt + 12 * b, qtil + 12 * k, sizeof(double) * 12);
                dof[b] = k++;
            }
        }
        if (g_sum) memset(g_sum, 0, sizeof(double) * 12 * (size_t)k);
        if (H_sum) memset(H_sum, 0, sizeof(double) * 144 * (size_t)k * k);
    }
    size_t nd = 12 * (size_t)k;
    for (int i = 0; !rc && i < N; ++i) {
        local_t L;
        rc = local_init(&L, s, mask, i, qa, qt, P, P->kappa_barrier, 1.0);
        if (!rc) {
            memcpy(L.z, L.q, sizeof(double) * 12 * (size_t)L.ns);
            for (int sl = 0; sl < L.ns; ++sl) L.rho[sl] = 0.0;
            if (i < cap && E_parts) E_parts[i] = local_energy(&L, L.q);
            if (g_sum || H_sum) {
                int n = 12 * L.ns;
                double *gg = (double *)malloc(sizeof(double) * (n ? n : 1));
                bsr_t H = {0};
                H.diag = (double *)malloc(sizeof(double) * 144 * (size_t)(L.ns ? L.ns : 1));
                H.rowhead = (int *)malloc(sizeof(int) * (L.ns ? L.ns : 1));
                rc = (!gg || !H.diag || !H.rowhead) ? ORC_E_OOM : local_assemble(&L, L.q, gg, &H);
                for (int sl = 0; !rc && g_sum && sl < L.ns; ++sl)
                    for (int j = 0; j < 12; ++j) g_sum[12 * dof[L.body[sl]] + j] += gg[12 * sl + j];
                if (!rc && H_sum) {
                    for (int sl = 0; sl < L.ns; ++sl) {
                        size_t r0 = 12 * (size_t)dof[L.body[sl]];
                        for (int a = 0; a < 12; ++a)
                            for (int c = 0; c < 12; ++c) H_sum[(r0 + a) * nd + r0 + c] += H.diag[144 * sl + 12 * a + c];
                    }
                    for (int o = 0; o < H.noff; ++o) {
                        size_t ra = 12 * (size_t)dof[L.body[H.off[o].a]], rb = 12 * (size_t)dof[L.body[H.off[o].b]];
                        for (int a = 0; a < 12; ++a)
                            for (int c = 0; c < 12; ++c) {
                                H_sum[(ra + a) * nd + rb + c] += H.off[o].blk[12 * a + c];
                                H_sum[(rb + c) * nd + ra + a] += H.off[o].blk[12 * a + c];
                            }
                    }
                }
                free(gg); free(H.diag); free(H.rowhead); free(H.off); free(H.next);
            }
        }
        local_free(&L);
    }
    free(mask); free(dof); free(qa); free(qt);
    return rc ? rc : N;
}

/* Gradient of partition `part`'s local objective F_i (Eq. 3: inertia and
 * orthogonality of each of its slots weighted 1/kappa_b, contacts 1/kappa_c,
 * plane contacts 1/kappa_b; no consensus term) at the replica configuration
 * q ([n_dof][12], body order: bodies of the partition take their rows, the
 * others are ignored), with predicted state qtil and barrier stiffness
 * P->kappa_barrier.  Membership is the slab rule at the scene's current
 * state.  g receives [n_dof][12], zero rows for bodies outside the partition;
 * *E the value of F_i (either may be NULL). */
int orc_local_gradient(orc_scene *s, const orc_params *P, int part, const double *q, const double *qtil, double *E,
                       double *g) {
    int N = P->n_slabs < 1 ? 1 : P->n_slabs;
    if (part < 0 || part >= N) return ORC_E_INVALID;
    uint64_t *mask = (uint64_t *)malloc(sizeof(uint64_t) * s->nb);
    int *dof = (int *)malloc(sizeof(int) * s->nb);
    double *qa = (double *)calloc(12 * (size_t)s->nb, sizeof(double)), *qt = (double *)calloc(12 * (size_t)s->nb, sizeof(double));
    int rc = (!mask || !dof || !qa || !qt) ? ORC_E_OOM : ORC_OK, k = 0;
    if (!rc) rc = orc_partition(s, P, mask, NULL);
    if (!rc) {
        memcpy(qa, s->q, sizeof(double) * 12 * s->nb);
        memcpy(qt, s->q, sizeof(double) * 12 * s->nb);
        for (int b = 0; b < s->nb; ++b) {
            dof[b] = -1;
            if (is_dof(s->kind[b])) {
                memcpy(qa + 12 * b, q + 12 * k, sizeof(double) * 12);
                memcpy(qt + 12 * b, qtil + 12 * k, sizeof(double) * 12);
                dof[b] = k++;
            }
        }
        if (g) memset(g, 0, sizeof(double) * 12 * (size_t)k);
        local_t L;
        rc = local_init(&L, s, mask, part, qa, qt, P, P->kappa_barrier, 1.0);
        if (!rc) {
            for (int sl = 0; sl < L.ns; ++sl) L.rho[sl] = 0.0;
            if (E) *E = local_energy(&L, L.q);
            if (g) {
                int n = 12 * L.ns;
                double *gg = (double *)malloc(sizeof(double) * (n ? n : 1));
                bsr_t H = {0};
                H.diag = (double *)malloc(sizeof(double) * 144 * (size_t)(L.ns ? L.ns : 1));
                H.rowhead = (int *)malloc(sizeof(int) * (L.ns ? L.ns : 1));
                rc = (!gg || !H.diag || !H.rowhead) ? ORC_E_OOM : local_assemble(&L, L.q, gg, &H);
                for (int sl = 0; !rc && sl < L.ns; ++sl)
                    for (int j = 0; j < 12; ++j) g[12 * dof[L.body[sl]] + j] = gg[12 * sl + j];
                free(gg); free(H.diag); free(H.rowhead); free(H.off); free(H.next);
            }
        }
        local_free(&L);
    }
    free(mask); free(dof); free(qa); free(qt);
    return rc;
}
