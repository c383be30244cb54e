// abd_device.cuh -- per-primitive math of ABD-IPC on sm_103a.
//
// Distance types, distance derivatives, the IPC log barrier, the edge-edge
// mollifier, PSD projection and additive CCD, written for one thread per
// primitive pair.  Templated on the assembly precision T (double for the FP64
// path, float for the mixed path); positions always arrive in FP64 and are
// shifted to a pair-local origin in FP64 before any rounding to T, so FP32
// assembly keeps the relative precision of the short difference vectors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace abd {

template <class T> __device__ __forceinline__ T tsqrt(T x);
template <> __device__ __forceinline__ double tsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float tsqrt<float>(float x) { return sqrtf(x); }
template <class T> __device__ __forceinline__ T tlog(T x);
template <> __device__ __forceinline__ double tlog<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float tlog<float>(float x) { return logf(x); }
template <class T> __device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

template <class T> __device__ __forceinline__ T dot3(const T *a, const T *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class T> __device__ __forceinline__ void cross3(T *o, const T *a, const T *b) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// ---------------------------------------------------------------------------
// Closest features.  PT: X0 point, X1..X3 triangle.  Codes 0..2 point-vertex,
// 3..5 point-edge (t0t1, t1t2, t2t0), 6 point-face.  EE: X0X1 edge a, X2X3
// edge b.  Codes 0..3 vertex-vertex (a_i, b_j) = 2i + j, 4..5 a_i to edge b,
// 6..7 b_j to edge a, 8 edge-edge interior.  The feature is the one holding
// the exact closest points: the unconstrained minimiser if it lies inside the
// parameter domain, else the best boundary sub-problem, scanned in a fixed
// order with strict improvement.  Nearly parallel edges (sin^2 <= 1e-10) use
// the boundary sub-problems.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T seg_closest(const T *p, const T *a, const T *b, T &t) {
    T ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    T ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    T L = dot3(ab, ab);
    t = L > T(0) ? dot3(ap, ab) / L : T(0);
    t = t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
    T r[3] = {ap[0] - t * ab[0], ap[1] - t * ab[1], ap[2] - t * ab[2]};
    return dot3(r, r);
}

template <class T>
__device__ T classify(bool ee, const T *X, int &type, T &b0, T &b1) {
    b0 = b1 = T(0);
    if (!ee) {
        const T *p = X, *t0 = X + 3;
        T e1[3] = {X[6] - X[3], X[7] - X[4], X[8] - X[5]};
        T e2[3] = {X[9] - X[3], X[10] - X[4], X[11] - X[5]};
        T ap[3] = {p[0] - t0[0], p[1] - t0[1], p[2] - t0[2]};
        T G00 = dot3(e1, e1), G01 = dot3(e1, e2), G11 = dot3(e2, e2);
        T r0 = dot3(ap, e1), r1 = dot3(ap, e2);
        T det = G00 * G11 - G01 * G01;
        if (det > T(0)) {
            T idet = T(1) / det;
            T u = (r0 * G11 - r1 * G01) * idet, v = (G00 * r1 - G01 * r0) * idet;
            if (u >= T(0) && v >= T(0) && u + v <= T(1)) {
                T r[3];
                for (int k = 0; k < 3; ++k) r[k] = ap[k] - u * e1[k] - v * e2[k];
                type = 6; b0 = u; b1 = v;
                return dot3(r, r);
            }
        }
        T best = sizeof(T) == 8 ? T(1e300) : T(3e38);
        for (int e = 0; e < 3; ++e) {
            int m = e, n = e == 2 ? 0 : e + 1;
            T t;
            T d2 = seg_closest(p, X + 3 + 3 * m, X + 3 + 3 * n, t);
            if (d2 < best) {
                best = d2;
                if (t == T(0)) { type = m; b0 = T(0); }
                else if (t == T(1)) { type = n; b0 = T(0); }
                else { type = 3 + e; b0 = t; }
            }
        }
        return best;
    }
    const T *a0 = X, *a1 = X + 3, *bb0 = X + 6, *bb1 = X + 9;
    T ea[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
    T eb[3] = {bb1[0] - bb0[0], bb1[1] - bb0[1], bb1[2] - bb0[2]};
    T w[3] = {a0[0] - bb0[0], a0[1] - bb0[1], a0[2] - bb0[2]};
    T A = dot3(ea, ea), B = dot3(ea, eb), C = dot3(eb, eb), D = dot3(ea, w), E = dot3(eb, w);
    T den = A * C - B * B;
    if (den > T(1e-10) * A * C) {
        T iden = T(1) / den;
        T s = (B * E - C * D) * iden, t = (A * E - B * D) * iden;
        if (s >= T(0) && s <= T(1) && t >= T(0) && t <= T(1)) {
            T r[3];
            for (int k = 0; k < 3; ++k) r[k] = w[k] + s * ea[k] - t * eb[k];
            type = 8; b0 = s; b1 = t;
            return dot3(r, r);
        }
    }
    T best = sizeof(T) == 8 ? T(1e300) : T(3e38);
    for (int i = 0; i < 2; ++i) {
        T t;
        T d2 = seg_closest(X + 3 * i, bb0, bb1, t);
        if (d2 < best) {
            best = d2;
            if (t == T(0)) { type = 2 * i; b0 = T(0); }
            else if (t == T(1)) { type = 2 * i + 1; b0 = T(0); }
            else { type = 4 + i; b0 = t; }
        }
    }
    for (int j = 0; j < 2; ++j) {
        T t;
        T d2 = seg_closest(X + 6 + 3 * j, a0, a1, t);
        if (d2 < best) {
            best = d2;
            if (t == T(0)) { type = j; b0 = T(0); }
            else if (t == T(1)) { type = 2 + j; b0 = T(0); }
            else { type = 6 + j; b0 = t; }
        }
    }
    return best;
}

// Closest-point parametrisation of a feature: r = sum_v (w0_v + sum_j beta_j c_jv) x_v.
struct Feature {
    int k;
    float w0[4];
    float c[2][4];
};

__device__ __forceinline__ Feature feature_of(bool ee, int type) {
    Feature f;
    f.k = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v) { f.w0[v] = 0.f; f.c[0][v] = 0.f; f.c[1][v] = 0.f; }
    if (!ee) {
        f.w0[0] = 1.f;
        if (type <= 2) f.w0[1 + type] = -1.f;
        else if (type <= 5) {
            int m = type - 3, n = m == 2 ? 0 : m + 1;
            f.k = 1; f.w0[1 + m] = -1.f; f.c[0][1 + m] = 1.f; f.c[0][1 + n] = -1.f;
        } else {
            f.k = 2; f.w0[1] = -1.f; f.c[0][1] = 1.f; f.c[0][2] = -1.f; f.c[1][1] = 1.f; f.c[1][3] = -1.f;
        }
    } else {
        if (type <= 3) { f.w0[type >> 1] = 1.f; f.w0[2 + (type & 1)] = -1.f; }
        else if (type <= 5) { f.k = 1; f.w0[type - 4] = 1.f; f.w0[2] = -1.f; f.c[0][2] = 1.f; f.c[0][3] = -1.f; }
        else if (type <= 7) { f.k = 1; f.w0[2 + type - 6] = 1.f; f.w0[0] = -1.f; f.c[0][0] = 1.f; f.c[0][1] = -1.f; }
        else { f.k = 2; f.w0[0] = 1.f; f.w0[2] = -1.f; f.c[0][0] = -1.f; f.c[0][1] = 1.f; f.c[1][2] = 1.f; f.c[1][3] = -1.f; }
    }
    return f;
}

// IPC log barrier on the unsquared distance: b = -(d - dhat)^2 ln(d / dhat) on (0, dhat).
template <class T>
__device__ __forceinline__ void barrier3(T d, T dhat, T &b, T &b1, T &b2) {
    if (d >= dhat) { b = b1 = b2 = T(0); return; }
    T e = d - dhat, L = tlog(d / dhat), id = T(1) / d, eid = e * id;
    b = -e * e * L;
    b1 = T(-2) * e * L - e * eid;
    b2 = T(-2) * L - T(4) * eid + eid * eid;
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix in place;
// V receives the eigenvectors as columns.
template <class T, int N>
__device__ void jacobi(T *A, T *V) {
    for (int i = 0; i < N * N; ++i) V[i] = T(0);
    for (int i = 0; i < N; ++i) V[i * N + i] = T(1);
    const T tol = sizeof(T) == 8 ? T(1e-30) : T(1e-10);
    for (int sweep = 0; sweep < (sizeof(T) == 8 ? 30 : 10); ++sweep) {
        T off = T(0), tot = T(0);
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                T a2 = A[i * N + j] * A[i * N + j];
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= tol * tot || off == T(0)) break;
        for (int p = 0; p < N - 1; ++p)
            for (int q = p + 1; q < N; ++q) {
                T apq = A[p * N + q];
                if (apq == T(0)) continue;
                T theta = (A[q * N + q] - A[p * N + p]) / (T(2) * apq);
                T t = (theta >= T(0) ? T(1) : T(-1)) / (tabs(theta) + tsqrt(theta * theta + T(1)));
                T c = T(1) / tsqrt(t * t + T(1)), s = t * c;
                for (int k = 0; k < N; ++k) {
                    T akp = A[k * N + p], akq = A[k * N + q];
                    A[k * N + p] = c * akp - s * akq;
                    A[k * N + q] = s * akp + c * akq;
                }
                for (int k = 0; k < N; ++k) {
                    T apk = A[p * N + k], aqk = A[q * N + k];
                    A[p * N + k] = c * apk - s * aqk;
                    A[q * N + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < N; ++k) {
                    T vkp = V[k * N + p], vkq = V[k * N + q];
                    V[k * N + p] = c * vkp - s * vkq;
                    V[k * N + q] = s * vkp + c * vkq;
                }
            }
    }
}

// Nearest PSD matrix (negative eigenvalues clamped to zero); a matrix without
// negative eigenvalues is left unchanged.
template <class T, int N>
__device__ void psd_project(T *H) {
    T E[N * N], V[N * N];
    for (int i = 0; i < N * N; ++i) E[i] = H[i];
    jacobi<T, N>(E, V);
    bool neg = false;
    for (int i = 0; i < N; ++i) neg |= E[i * N + i] < T(0);
    if (!neg) return;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            T s = T(0);
            for (int k = 0; k < N; ++k) {
                T lam = E[k * N + k];
                if (lam > T(0)) s += V[i * N + k] * lam * V[j * N + k];
            }
            H[i * N + j] = s;
        }
}

// |ea x eb|^2 of an edge-edge pair in pair-local coordinates (edge a = X0 X1,
// edge b = X2 X3), the quantity whose comparison with eps_x switches the
// mollifier on.  Every operation is rounded on its own (no contraction into
// fused multiply-adds), so the kernels that split the pairs by this test
// (mollified or not) and the kernel that evaluates them take the same
// decision for every pair.
__device__ __forceinline__ double ee_cross2(const double *X) {
    double a[3], b[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = __dsub_rn(X[3 + k], X[k]);
        b[k] = __dsub_rn(X[9 + k], X[6 + k]);
    }
    double c0 = __dsub_rn(__dmul_rn(a[1], b[2]), __dmul_rn(a[2], b[1]));
    double c1 = __dsub_rn(__dmul_rn(a[2], b[0]), __dmul_rn(a[0], b[2]));
    double c2 = __dsub_rn(__dmul_rn(a[0], b[1]), __dmul_rn(a[1], b[0]));
    return __dadd_rn(__dadd_rn(__dmul_rn(c0, c0), __dmul_rn(c1, c1)), __dmul_rn(c2, c2));
}

// FP64 gradient of one PT/EE pair's barrier energy kB * [m(c)] * b(d) in
// pair-local coordinates X.  Returns d; fills the feature (type, beta) and the
// scalars the Hessian needs.  When d >= dhat or d <= 0 nothing else is written.
struct PairGrad {
    int type;
    double b0, b1;       // beta of the feature
    double b, bp, bpp;   // barrier and its derivatives at d
    double m;            // mollifier value (1 for PT or inactive)
    bool moll;           // mollifier active
};

__device__ inline double pair_gradient(bool ee, const double *X, double dhat, double kB, double eps_x, PairGrad &P,
                                       double *g) {
    double s2 = classify<double>(ee, X, P.type, P.b0, P.b1);
    double d = sqrt(s2);
    if (!(d < dhat) || !(d > 0.0)) return d;
    Feature f = feature_of(ee, P.type);
    double w[4], r[3] = {0, 0, 0};
    for (int v = 0; v < 4; ++v) w[v] = double(f.w0[v]) + P.b0 * double(f.c[0][v]) + P.b1 * double(f.c[1][v]);
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) r[a] += w[v] * X[3 * v + a];
    barrier3<double>(d, dhat, P.b, P.bp, P.bpp);
    // grad b = b' grad d, grad d = grad s / 2d = w (x) r / d (one reciprocal:
    // FP64 division is a long instruction sequence on this GPU)
    const double bpd = P.bp / d;
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) g[3 * v + a] = bpd * w[v] * r[a];
    P.m = 1.0;
    P.moll = false;
    if (ee) {
        double ea[3] = {X[3] - X[0], X[4] - X[1], X[5] - X[2]};
        double eb[3] = {X[9] - X[6], X[10] - X[7], X[11] - X[8]};
        double cr[3], t[3];
        cross3(cr, ea, eb);
        double c = ee_cross2(X);
        if (c < eps_x) {
            double rr = c / eps_x;
            P.m = rr * (2.0 - rr);
            P.moll = true;
            double m1 = (2.0 - 2.0 * rr) / eps_x;
            double ge[6];
            cross3(t, eb, cr);
            ge[0] = 2 * t[0]; ge[1] = 2 * t[1]; ge[2] = 2 * t[2];
            cross3(t, cr, ea);
            ge[3] = 2 * t[0]; ge[4] = 2 * t[1]; ge[5] = 2 * t[2];
            const double sg[4] = {-1, 1, -1, 1};
            for (int v = 0; v < 4; ++v)
                for (int a = 0; a < 3; ++a) g[3 * v + a] = m1 * sg[v] * ge[3 * (v >> 1) + a] * P.b + P.m * g[3 * v + a];
        }
    }
    for (int i = 0; i < 12; ++i) g[i] *= kB;
    return d;
}

// Cyclic Jacobi + clamp for a symmetric n x n matrix, n <= 5, in registers
// (row stride 5).  Leaves K unchanged when it has no negative eigenvalue.
template <class T>
__device__ __forceinline__ void psd_small(T *K, int n) {
    T A[25], V[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) { A[i] = K[i]; V[i] = (i % 6 == 0) ? T(1) : T(0); }
    const T tol = sizeof(T) == 8 ? T(1e-30) : T(1e-10);
    for (int sweep = 0; sweep < 12; ++sweep) {
        T off = T(0), tot = T(0);
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (i < n && j < n) {
                    T a2 = A[i * 5 + j] * A[i * 5 + j];
                    tot += a2;
                    if (i != j) off += a2;
                }
        if (off <= tol * tot || off == T(0)) break;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = p + 1; q < 5; ++q) {
                if (q >= n) continue;
                T apq = A[p * 5 + q];
                if (apq == T(0)) continue;
                T theta = (A[q * 5 + q] - A[p * 5 + p]) / (T(2) * apq);
                T t = (theta >= T(0) ? T(1) : T(-1)) / (tabs(theta) + tsqrt(theta * theta + T(1)));
                T c = T(1) / tsqrt(t * t + T(1)), sn = t * c;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    T akp = A[k * 5 + p], akq = A[k * 5 + q];
                    A[k * 5 + p] = c * akp - sn * akq;
                    A[k * 5 + q] = sn * akp + c * akq;
                }
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    T apk = A[p * 5 + k], aqk = A[q * 5 + k];
                    A[p * 5 + k] = c * apk - sn * aqk;
                    A[q * 5 + k] = sn * apk + c * aqk;
                }
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    T vkp = V[k * 5 + p], vkq = V[k * 5 + q];
                    V[k * 5 + p] = c * vkp - sn * vkq;
                    V[k * 5 + q] = sn * vkp + c * vkq;
                }
            }
    }
    bool neg = false;
#pragma unroll
    for (int i = 0; i < 5; ++i) neg |= (i < n) && A[i * 6] < T(0);
    if (!neg) return;
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (k < n && A[k * 6] > T(0)) acc += V[i * 5 + k] * A[k * 6] * V[j * 5 + k];
            K[i * 5 + j] = (i < n && j < n) ? acc : T(0);
        }
}

// Low-rank form of one unmollified pair's barrier Hessian.  Its range lies in
// span{w (x) e_a, c_j_perp (x) r} (w: closest-point weights, c_j: feature
// parameter directions orthogonalised against w, r: closest-point
// difference), at most 5-dimensional, so H = B K B^T with B orthonormal:
// B = [w^ (x) e_1..3, c^_j (x) r^] and K = B^T H B (n x n, n = 3 + k).
// PSD(H) = B PSD(K) B^T exactly.  Returns n and fills K (row stride 5, kB
// included), the unit weights wh[4], the unit feature directions ch[2][4]
// and r^.
//
// The geometric inputs -- r (length d, a few 1e-4 m) and the feature edges D_j
// (up to metres for a large static triangle) as weighted sums of the pair's
// coordinates, and their Gram matrix -- come from the FP64 coordinates Xd
// and are rounded to T only once formed: in FP32 the sum for r loses about
// eps_32 |X| / d of its direction (1e-3 for a vertex a few metres from the
// far corner of a floor triangle), and the misdirected normal stiffness then
// stiffens the body's tangential and rotational modes enough to end its
// Newton solve early.
template <class T>
__device__ int pair_hessian_lowrank(bool ee, const double *Xd, const PairGrad &P, T d, T kB, T *K, T *wh,
                                    T ch[2][4], T *rh) {
    Feature f = feature_of(ee, P.type);
    T w[4], r[3], D[2][3];
    {
        double wd[4], rd[3] = {0, 0, 0}, Dd[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int v = 0; v < 4; ++v) wd[v] = f.w0[v] + P.b0 * f.c[0][v] + P.b1 * f.c[1][v];
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                rd[a] += wd[v] * Xd[3 * v + a];
                Dd[0][a] += f.c[0][v] * Xd[3 * v + a];
                Dd[1][a] += f.c[1][v] * Xd[3 * v + a];
            }
#pragma unroll
        for (int v = 0; v < 4; ++v) w[v] = T(wd[v]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r[a] = T(rd[a]);
            D[0][a] = T(Dd[0][a]);
            D[1][a] = T(Dd[1][a]);
        }
    }
    const int k = f.k, n = 3 + k;
    T wn2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3], wn = tsqrt(wn2);
#pragma unroll
    for (int v = 0; v < 4; ++v) wh[v] = w[v] / wn;
    T rn = tsqrt(dot3(r, r));
#pragma unroll
    for (int a = 0; a < 3; ++a) rh[a] = r[a] / rn;
    // c^_j: Gram-Schmidt of the feature directions against w^ and each other;
    // cc[j][l] = c_j . c^_l
    T cc[2][2] = {{0, 0}, {0, 0}}, wc[2] = {0, 0};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        T cj[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) cj[v] = T(f.c[j][v]);
        wc[j] = cj[0] * w[0] + cj[1] * w[1] + cj[2] * w[2] + cj[3] * w[3];
        if (j >= k) {
#pragma unroll
            for (int v = 0; v < 4; ++v) ch[j][v] = T(0);
            continue;
        }
        T u[4];
        T pw = wc[j] / wn2;
#pragma unroll
        for (int v = 0; v < 4; ++v) u[v] = cj[v] - pw * w[v];
        if (j == 1) {
            T p0 = u[0] * ch[0][0] + u[1] * ch[0][1] + u[2] * ch[0][2] + u[3] * ch[0][3];
#pragma unroll
            for (int v = 0; v < 4; ++v) u[v] -= p0 * ch[0][v];
        }
        T un = tsqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
#pragma unroll
        for (int v = 0; v < 4; ++v) ch[j][v] = u[v] / un;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int l = 0; l < 2; ++l)
            cc[j][l] = (j < k && l < k)
                           ? T(f.c[j][0]) * ch[l][0] + T(f.c[j][1]) * ch[l][1] + T(f.c[j][2]) * ch[l][2] +
                                 T(f.c[j][3]) * ch[l][3]
                           : T(0);
    T bp = T(P.bp), cg = T(P.bpp) - bp / d, chs = bp / (T(2) * d);
#pragma unroll
    for (int i = 0; i < 25; ++i) K[i] = T(0);
    // cg (B^T gd)(B^T gd)^T, B^T gd = (|w| r / d, 0, 0)
    T gdb[3] = {wn * r[0] / d, wn * r[1] / d, wn * r[2] / d};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) K[a * 5 + b] = cg * gdb[a] * gdb[b];
    // + 2 ch |w|^2 on the first three
#pragma unroll
    for (int a = 0; a < 3; ++a) K[a * 6] += T(2) * chs * wn2;
    // - 2 ch sum_ij Ginv_ij (B^T g_i)(B^T g_j)^T, B^T g_j = (|w| D_j + (w.c_j/|w|) r, (c_j.c^_l)|r|)
    if (k > 0) {
        T G00 = dot3(D[0], D[0]), G01 = dot3(D[0], D[1]), G11 = dot3(D[1], D[1]);
        T i00, i01, i11;
        if (k == 1) { i00 = T(1) / G00; i01 = T(0); i11 = T(0); }
        else {
            T det = G00 * G11 - G01 * G01;
            i00 = G11 / det; i11 = G00 / det; i01 = -G01 / det;
        }
        T gb[2][5];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int a = 0; a < 3; ++a) gb[j][a] = wn * D[j][a] + wc[j] / wn * r[a];
            gb[j][3] = cc[j][0] * rn;
            gb[j][4] = cc[j][1] * rn;
        }
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int b = 0; b < 5; ++b)
                K[a * 5 + b] -= T(2) * chs *
                                (i00 * gb[0][a] * gb[0][b] + i01 * (gb[0][a] * gb[1][b] + gb[1][a] * gb[0][b]) +
                                 i11 * gb[1][a] * gb[1][b]);
    }
#pragma unroll
    for (int i = 0; i < 25; ++i) K[i] *= kB;
    return n;
}

// Barrier energy only (no derivatives), FP64.
__device__ __forceinline__ double pair_energy(bool ee, const double *X, double dhat, double kB, double eps_x, double &d) {
    int type;
    double b0, b1;
    d = sqrt(classify<double>(ee, X, type, b0, b1));
    if (!(d > 0.0)) return 1.0 / 0.0;
    if (!(d < dhat)) return 0.0;
    double b, bp, bpp;
    barrier3<double>(d, dhat, b, bp, bpp);
    if (ee) {
        double ea[3] = {X[3] - X[0], X[4] - X[1], X[5] - X[2]};
        double eb[3] = {X[9] - X[6], X[10] - X[7], X[11] - X[8]};
        double cr[3];
        cross3(cr, ea, eb);
        double c = dot3(cr, cr);
        if (c < eps_x) {
            double rr = c / eps_x;
            b *= rr * (2.0 - rr);
        }
    }
    return kB * b;
}

// Additive CCD (Li et al. 2021) along X -> X + dX, t in [0, 1], FP64.
// Displacements shifted to zero mean; l_p = max displacement norm per side,
// summed.  First advance (1 - s) d0 / l_p, later c d / l_p; an advance
// reaching t = 1 certifies the path (exactly 1); once the distance after a
// later advance drops below s d0, the previous time is returned.
// With d0_out, the distance at t = 0 (computed once for both uses).
__device__ inline double accd(bool ee, const double *X, const double *dX, double s, double c, int max_iter,
                              double *d0_out = nullptr) {
    double mean[3] = {0, 0, 0};
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) mean[a] += 0.25 * dX[3 * v + a];
    double n[4];
    for (int v = 0; v < 4; ++v) {
        double p0 = dX[3 * v] - mean[0], p1 = dX[3 * v + 1] - mean[1], p2 = dX[3 * v + 2] - mean[2];
        n[v] = sqrt(p0 * p0 + p1 * p1 + p2 * p2);
    }
    double lp = ee ? fmax(n[0], n[1]) + fmax(n[2], n[3]) : n[0] + fmax(n[1], fmax(n[2], n[3]));
    if (lp == 0.0 && !d0_out) return 1.0;
    int ty;
    double b0, b1;
    double d = sqrt(classify<double>(ee, X, ty, b0, b1));
    if (d0_out) *d0_out = d;
    if (lp == 0.0) return 1.0;
    if (!(d > 0.0)) return 0.0;
    double g = s * d, t = 0.0, step = (1.0 - s) * d / lp;
    for (int it = 0; it < max_iter; ++it) {
        if (t + step >= 1.0) return 1.0;
        double tn = t + step, Xn[12];
        for (int i = 0; i < 12; ++i) Xn[i] = X[i] + tn * dX[i];
        double dn = sqrt(classify<double>(ee, Xn, ty, b0, b1));
        if (t > 0.0 && dn < g) return t;
        t = tn;
        d = dn;
        step = c * d / lp;
    }
    return t;
}

__device__ __forceinline__ double accd_plane(double d0, double dd, double s) {
    if (!(d0 > 0.0)) return 0.0;
    if (dd >= 0.0) return 1.0;
    double t = (1.0 - s) * d0 / (-dd);
    return t < 1.0 ? t : 1.0;
}

// Order-preserving map of non-negative doubles to uint64 (for atomicMin/Max).
__device__ __forceinline__ unsigned long long ord(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double unord(unsigned long long u) { return __longlong_as_double((long long)u); }

}  // namespace abd
