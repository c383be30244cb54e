// abd_assemble.cu -- narrow phase, Newton assembly, CCD and line-search energies.
//
// Per slot: inertia (1/kappa_b) M (q - q~), orthogonality (1/kappa_b) h^2 kappa V
// ||A A^T - I||^2 with its 9x9 Hessian projected to PSD, and the consensus
// penalty rho (q - z + u) for shared replicas (Eq. 3, Eq. 5).  Per active
// pair: (h^2 / kappa_c) kB b(d) [m(c)] with its 12x12 vertex Hessian projected
// to PSD before the J^T H J map onto the slot blocks (12x12, J_v = I3 (x)
// (1, xbar_v^T)).  CCD and energies are FP64; assembly runs in T.
#include <cfloat>

#include "abd_device.cuh"
#include "abd_internal.h"

namespace abd {

__device__ __forceinline__ int qidx(int k, int a) { return a == 0 ? k : 3 + 3 * k + (a - 1); }

__device__ __forceinline__ int pair_slots(const PairRec &r, const int *sv_slot, int &sa, int &sb) {
    sa = sv_slot[r.v[0]];
    sb = sv_slot[r.v[(r.flags & 1) ? 2 : 1]];
    return 0;
}

__device__ __forceinline__ double pair_kappa(int sa, int sb, int S_dyn, const unsigned long long *mask) {
    if (sa >= S_dyn) return (double)__popcll(mask[sb]);
    if (sb >= S_dyn) return (double)__popcll(mask[sa]);
    return (double)__popcll(mask[sa] & mask[sb]);
}

__device__ __forceinline__ int pair_part(int sa, int sb, int S_dyn, const int *slot_part) {
    return sa < S_dyn ? slot_part[sa] : slot_part[sb];
}

// Warp-aggregated append of `rec` when `keep`.
__device__ __forceinline__ void append(bool keep, const PairRec &rec, PairRec *out, int64_t cap,
                                       unsigned long long *count) {
    int lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) return;
    unsigned long long pos = 0;
    int leader = __ffs(m) - 1;
    if (lane == leader) pos = atomicAdd(count, (unsigned long long)__popc(m));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (keep) {
        unsigned long long my = pos + __popc(m & ((1u << lane) - 1));
        if ((int64_t)my < cap) out[my] = rec;
    }
}

// Narrow phase: keep candidates with 0 < d < dhat.
__global__ void k_narrow(const PairRec *__restrict__ cand, int64_t n, const unsigned long long *__restrict__ n_dev,
                         const double *__restrict__ x, double dhat, PairRec *__restrict__ act, int64_t cap,
                         unsigned long long *__restrict__ count) {
    if (n_dev) n = min((int64_t)*n_dev, n);
    for (int64_t base = spread_base(); base < n; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = base + (threadIdx.x & 31);
        bool keep = false;
        PairRec r;
        if (i < n) {
            r = cand[i];
            double X[12];
            for (int v = 0; v < 4; ++v)
                for (int k = 0; k < 3; ++k) X[3 * v + k] = x[3 * (int64_t)r.v[v] + k];
            int ty;
            double b0, b1;
            double d = sqrt(classify<double>(r.flags & 1, X, ty, b0, b1));
            keep = d < dhat;
        }
        append(keep, r, act, cap, count);
    }
}

struct AsmArgs {
    int S_dyn;
    const int *slot_body, *slot_part, *slot_rep, *sv_slot;
    const unsigned long long *slot_mask;
    const double *slot_kw;
    const int *voff;
    const double *xbar, *mass, *S, *vol, *kappa;
    const double *q, *qtil, *z, *u, *rho;
    const double *x;
    const PartState *part;  // per partition: active flag, barrier stiffness kB
    double h, dhat;
    Planes planes;
    const int64_t *slot_voff;
    double *g;
    int *rowcnt;  // per dynamic slot: number of distinct off-diagonal blocks in its row
};

// Per dynamic slot of an active partition: write g and the diagonal block.
template <class T>
__global__ void k_slot_assemble(AsmArgs A, T *__restrict__ diag) {
    for (int64_t sb = spread_base(); sb < A.S_dyn; sb += (int64_t)gridDim.x * blockDim.x) {
        int s = (int)(sb + (threadIdx.x & 31));
        if (s >= A.S_dyn || !A.part[A.slot_part[s]].active) continue;
        int b = A.slot_body[s];
        double kw = A.slot_kw[s], h2 = A.h * A.h;
        const double *q = A.q + 12 * (int64_t)s, *qt = A.qtil + 12 * (int64_t)s;
        const double *S = A.S + 9 * (int64_t)b;
        double m = A.mass[b];
        double g[12];
        T D[144];
        for (int i = 0; i < 144; ++i) D[i] = T(0);
        for (int k = 0; k < 3; ++k) {
            g[k] = kw * m * (q[k] - qt[k]);
            D[k * 12 + k] = T(kw * m);
        }
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i) {
                double acc = 0.0;
                for (int j = 0; j < 3; ++j) {
                    acc += S[3 * i + j] * (q[3 + 3 * k + j] - qt[3 + 3 * k + j]);
                    D[(3 + 3 * k + i) * 12 + 3 + 3 * k + j] = T(kw * S[3 * i + j]);
                }
                g[3 + 3 * k + i] = kw * acc;
            }
        // orthogonality potential: rows a_k, C = A A^T - I
        double a[3][3], C[3][3];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) a[k][j] = q[3 + 3 * k + j];
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) C[k][l] = a[k][0] * a[l][0] + a[k][1] * a[l][1] + a[k][2] * a[l][2] - (k == l);
        double kv = A.kappa[b] * A.vol[b], c4 = 4.0 * kv * kw * h2;
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) g[3 + 3 * k + j] += c4 * (C[k][0] * a[0][j] + C[k][1] * a[1][j] + C[k][2] * a[2][j]);
        // Hessian of the orthogonality term in the block type T (the
        // gradient above stays FP64)
        T H9[81], at[3][3], Ct[3][3], AtA[3][3];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) { at[k][j] = T(a[k][j]); Ct[k][j] = T(C[k][j]); }
        const T kvT = T(kv);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) AtA[i][j] = at[0][i] * at[0][j] + at[1][i] * at[1][j] + at[2][i] * at[2][j];
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        T v = at[l][i] * at[k][j] + (i == j ? Ct[k][l] : T(0)) + (k == l ? AtA[i][j] : T(0));
                        H9[(3 * k + i) * 9 + 3 * l + j] = T(4) * kvT * v;
                    }
        // PSD projection through the analytic eigensystem of the isotropic
        // energy kappa V sum_k (sigma_k^2 - 1)^2: with A = U diag(sigma) V^T and
        // every sigma_k^2 >= 1/3, only the three twist modes
        // (u_i v_j^T - u_j v_i^T)/sqrt2, eigenvalue 4 kappa V (s_i^2 - s_i s_j +
        // s_j^2 - 1), can be negative; they are removed from H9.  Otherwise the
        // 9x9 Jacobi projection is used.
        {
            T M3[9], V3[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) M3[3 * i + j] = AtA[i][j];
            jacobi<T, 3>(M3, V3);
            T sg[3] = {M3[0], M3[4], M3[8]};
            if (min(sg[0], min(sg[1], sg[2])) < T(1.0 / 3.0 + 1e-3)) {
                psd_project<T, 9>(H9);
            } else {
                T sv[3], U3[3][3];
                for (int k = 0; k < 3; ++k) sv[k] = tsqrt(sg[k]);
                for (int r = 0; r < 3; ++r)
                    for (int k = 0; k < 3; ++k)
                        U3[r][k] = (at[r][0] * V3[0 * 3 + k] + at[r][1] * V3[1 * 3 + k] + at[r][2] * V3[2 * 3 + k]) / sv[k];
                const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
                for (int t = 0; t < 3; ++t) {
                    int i = pi[t], j = pj[t];
                    T lam = T(4) * kvT * (sg[i] - sv[i] * sv[j] + sg[j] - T(1));
                    if (!(lam < T(0))) continue;
                    T v[9];
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c)
                            v[3 * r + c] = (U3[r][i] * V3[c * 3 + j] - U3[r][j] * V3[c * 3 + i]) * T(0.70710678118654752);
                    for (int e = 0; e < 9; ++e)
                        for (int f = 0; f < 9; ++f) H9[e * 9 + f] -= lam * v[e] * v[f];
                }
            }
        }
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) D[(3 + i) * 12 + 3 + j] += T(kw * h2) * H9[i * 9 + j];
        if (A.slot_rep[s] >= 0) {
            double r = A.rho[s];
            for (int i = 0; i < 12; ++i) {
                g[i] += r * (q[i] - A.z[12 * (int64_t)s + i] + A.u[12 * (int64_t)s + i]);
                D[i * 12 + i] += T(r);
            }
        }
        for (int i = 0; i < 12; ++i) A.g[12 * (int64_t)s + i] = g[i];
        T *o = diag + 144 * (int64_t)s;
        for (int i = 0; i < 144; ++i) o[i] = D[i];
    }
}

template <class T> __device__ __forceinline__ void atomic_addT(T *a, T v) { atomicAdd(a, v); }

// Per active pair: barrier gradient and projected Hessian scattered to slots.
// Edge-edge pairs whose mollifier is on (ee_cross2 < eps_x) are skipped: they
// belong to k_pair_moll (full 12x12 projection), which runs beside this kernel
// and picks them out with the same test.
template <class T>
__global__ void k_pair_assemble(AsmArgs A, const PairRec *__restrict__ act, int64_t n, const int2 *__restrict__ l1,
                                T *__restrict__ diag, T *__restrict__ off, int *__restrict__ offflag,
                                const unsigned long long *__restrict__ n_dev) {
    if (n_dev) n = min((int64_t)*n_dev, n);
    for (int64_t ib = spread_base(); ib < n; ib += (int64_t)gridDim.x * blockDim.x) {
        int64_t ii = ib + (threadIdx.x & 31);
        if (ii >= n) continue;
        const int64_t i = ii;
        PairRec r = act[i];
        int sa, sb;
        pair_slots(r, A.sv_slot, sa, sb);
        int part = pair_part(sa, sb, A.S_dyn, A.slot_part);
        if (!A.part[part].active) continue;
        bool ee = r.flags & 1;
        // pair-local coordinates in FP64; gradient in FP64, Hessian in T
        double Xd[12];
        for (int v = 0; v < 4; ++v)
            for (int k = 0; k < 3; ++k) Xd[3 * v + k] = A.x[3 * (int64_t)r.v[v] + k] - A.x[3 * (int64_t)r.v[0] + k];
        if (ee && ee_cross2(Xd) < r.eps) continue;  // mollified: k_pair_moll
        PairGrad PG;
        double gx[12];
        const double kB = A.part[part].kB;  // the barrier stiffness of the pair's partition
        double d = pair_gradient(ee, Xd, A.dhat, kB, r.eps, PG, gx);
        if (!(d < A.dhat) || !(d > 0.0)) continue;
        double w = A.h * A.h / pair_kappa(sa, sb, A.S_dyn, A.slot_mask);
        int sl[4];
        T xi[4][4];
        double xbv[4][4];
        for (int v = 0; v < 4; ++v) {
            int s = A.sv_slot[r.v[v]];
            sl[v] = s < A.S_dyn ? s : -1;
            int b = A.slot_body[s];
            const double *xb = A.xbar + 3 * ((int64_t)A.voff[b] + (r.v[v] - A.slot_voff[s]));
            xbv[v][0] = 1.0; xbv[v][1] = xb[0]; xbv[v][2] = xb[1]; xbv[v][3] = xb[2];
            for (int a = 0; a < 4; ++a) xi[v][a] = T(xbv[v][a]);
        }
        for (int v = 0; v < 4; ++v) {
            if (sl[v] < 0) continue;
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 4; ++a)
                    atomicAdd(A.g + 12 * (int64_t)sl[v] + qidx(k, a), w * gx[3 * v + k] * xbv[v][a]);
        }
        // slot sides: PT = {point} | {triangle}, EE = {edge a} | {edge b}
        const int nA = ee ? 2 : 1;
        int ss[2] = {sa < A.S_dyn ? sa : -1, sb < A.S_dyn ? sb : -1};
        {
            // exact low-rank projection: PSD(H) = B PSD(K) B^T, J^T PSD(H) J = P_s K+ P_t^T
            T K[25], wh[4], chat[2][4], rh[3];
            int n = pair_hessian_lowrank<T>(ee, Xd, PG, T(d), T(kB), K, wh, chat, rh);
            psd_small<T>(K, n);
            // pull-backs of the basis to each side: om[a] = sum_v w^_v xi_v, ga[j] = sum_v c^_jv xi_v
            T om[2][4], ga[2][2][4];
            for (int sd = 0; sd < 2; ++sd)
                for (int a = 0; a < 4; ++a) {
                    om[sd][a] = T(0); ga[sd][0][a] = T(0); ga[sd][1][a] = T(0);
                    for (int v = sd ? nA : 0; v < (sd ? 4 : nA); ++v) {
                        om[sd][a] += wh[v] * xi[v][a];
                        ga[sd][0][a] += chat[0][v] * xi[v][a];
                        ga[sd][1][a] += chat[1][v] * xi[v][a];
                    }
                }
            for (int bi = 0; bi < 2; ++bi)
                for (int bj = bi; bj < 2; ++bj) {
                    int s1 = ss[bi], s2 = ss[bj];
                    if (s1 < 0 || s2 < 0) continue;
                    T *dst;
                    bool tr = false;
                    if (bi == bj) dst = diag + 144 * (int64_t)s1;
                    else {
                        int2 lp = l1[r.l1];
                        dst = off + 144 * (int64_t)r.l1;
                        tr = (lp.x != s1);
                        if (atomicExch(&offflag[r.l1], 1) == 0) {
                            atomicAdd(&A.rowcnt[lp.x], 1);
                            atomicAdd(&A.rowcnt[lp.y], 1);
                        }
                    }
                    // column by column: m = K P_t^T e_col, then the 12 rows P_s m
                    for (int l = 0; l < 3; ++l)
                        for (int be = 0; be < 4; ++be) {
                            int col = qidx(l, be);
                            T mc[5];
                            for (int c = 0; c < 5; ++c) {
                                T acc = c < n ? K[c * 5 + l] * om[bj][be] : T(0);
                                for (int j = 0; j < 2; ++j)
                                    if (3 + j < n && c < n) acc += K[c * 5 + 3 + j] * rh[l] * ga[bj][j][be];
                                mc[c] = acc;
                            }
                            for (int kk = 0; kk < 3; ++kk)
                                for (int al = 0; al < 4; ++al) {
                                    int row = qidx(kk, al);
                                    T v = om[bi][al] * mc[kk];
                                    for (int j = 0; j < 2; ++j)
                                        if (3 + j < n) v += rh[kk] * ga[bi][j][al] * mc[3 + j];
                                    v *= T(w);
                                    if (v != T(0)) atomic_addT(dst + (tr ? col * 12 + row : row * 12 + col), v);
                                }
                        }
                }
        }
    }
}

// Pair k (0..5) of round rd (0..10) of the round-robin ordering on 12
// indices: (rd, 11) for k = 0, ((rd + k) mod 11, (rd - k) mod 11) otherwise,
// returned with p < q.
__device__ __forceinline__ void rr_pair(int rd, int k, int &p, int &q) {
    if (k == 0) { p = rd; q = 11; return; }
    int a = rd + k, b = rd - k;
    a = a >= 11 ? a - 11 : a;
    b = b < 0 ? b + 11 : b;
    p = a < b ? a : b;
    q = a < b ? b : a;
}

// Warp-cooperative PSD projection of a symmetric 12x12 matrix H (shared
// memory): eigen-decomposition by parallel cyclic Jacobi -- per sweep 11
// rounds of 6 disjoint rotations in round-robin order, every rotation angle
// of a round computed from the same matrix, columns then rows then the
// eigenvectors updated by all lanes -- then H = V max(L, 0) V^T if any
// eigenvalue is negative (H unchanged otherwise).  W, V: [144] scratch,
// R: [12] scratch for the round's cosines and sines.  Each lane's tasks
// (which pair slot, row or column) are fixed for the whole decomposition and
// set up once; only the pair indices change with the round.
template <class T>
__device__ void warp_psd12(T *H, T *W, T *V, T *R, int lane) {
    for (int i = lane; i < 144; i += 32) {
        W[i] = H[i];
        V[i] = (i % 13 == 0) ? T(1) : T(0);
    }
    // this lane's tasks, the same in every round: column updates (matrix,
    // pair slot, row) for tk = lane + 32 i < 144 (W for tk < 72, else V), row
    // updates (pair slot, column) for tk = lane + 32 i < 72
    int ck[5], crow[5], rk[3], rcol[3];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int tk = lane + 32 * i, t = tk < 72 ? tk : tk - 72;
        ck[i] = t / 12;
        crow[i] = (tk < 72 ? 0 : 144) + t % 12;  // offset of the matrix + row
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int tk = lane + 32 * i;
        rk[i] = tk / 12;
        rcol[i] = tk % 12;
    }
    __syncwarp();
    const T tol = sizeof(T) == 8 ? T(1e-30) : T(1e-10);
    for (int sweep = 0; sweep < (sizeof(T) == 8 ? 30 : 10); ++sweep) {
        T off = T(0), tot = T(0);
        for (int i = lane; i < 144; i += 32) {
            T a2 = W[i] * W[i];
            tot += a2;
            if (i / 12 != i % 12) off += a2;
        }
        for (int o = 16; o; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (off <= tol * tot || off == T(0)) break;
        for (int rd = 0; rd < 11; ++rd) {
            if (lane < 6) {
                int p, q;
                rr_pair(rd, lane, p, q);
                T apq = W[p * 12 + q], c = T(1), sn = T(0);
                if (apq != T(0)) {
                    T theta = (W[q * 12 + q] - W[p * 12 + p]) / (T(2) * apq);
                    T t = (theta >= T(0) ? T(1) : T(-1)) / (tabs(theta) + tsqrt(theta * theta + T(1)));
                    c = T(1) / tsqrt(t * t + T(1));
                    sn = t * c;
                }
                R[2 * lane] = c;
                R[2 * lane + 1] = sn;
            }
            __syncwarp();
            // columns p, q of W and V
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                if (lane + 32 * i >= 144) continue;
                int p, q;
                rr_pair(rd, ck[i], p, q);
                const T c = R[2 * ck[i]], sn = R[2 * ck[i] + 1];
                T *M = crow[i] >= 144 ? V : W;
                const int row = crow[i] >= 144 ? crow[i] - 144 : crow[i];
                const T mp = M[row * 12 + p], mq = M[row * 12 + q];
                M[row * 12 + p] = c * mp - sn * mq;
                M[row * 12 + q] = sn * mp + c * mq;
            }
            __syncwarp();
            // rows p, q of W
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (lane + 32 * i >= 72) continue;
                int p, q;
                rr_pair(rd, rk[i], p, q);
                const T c = R[2 * rk[i]], sn = R[2 * rk[i] + 1];
                const int col = rcol[i];
                const T mp = W[p * 12 + col], mq = W[q * 12 + col];
                W[p * 12 + col] = c * mp - sn * mq;
                W[q * 12 + col] = sn * mp + c * mq;
            }
            __syncwarp();
        }
    }
    bool neg = __any_sync(0xffffffffu, lane < 12 && W[lane * 13] < T(0));
    if (!neg) return;
    __syncwarp();
    for (int i = lane; i < 144; i += 32) {
        int r = i / 12, c = i % 12;
        T acc = T(0);
        for (int k = 0; k < 12; ++k) {
            T lam = W[k * 13];
            if (lam > T(0)) acc += V[r * 12 + k] * lam * V[c * 12 + k];
        }
        H[i] = acc;
    }
    __syncwarp();
}

// The raw (unprojected) Hessian of a mollified edge-edge pair's barrier
// energy, kB [m hess b + b hess m + grad m grad b^T + grad b grad m^T], in
// closed form: every entry (v a, u c) is a short expression of per-pair
// vectors, so lane 0 forms those (MollTerms, from the FP64 coordinates and the
// FP64 feature and barrier scalars of pair_gradient) and every lane then
// writes its entries.
//   s = |r|^2 at the stationary beta of the feature, r = sum_v w_v x_v; by the
//   envelope theorem grad s = 2 w (x) r and
//   hess s = 2 w_v w_u d_ac - 2 sum_ij Ginv_ij g_i g_j^T,
//   D_j = sum_v c_jv x_v, G_ij = D_i . D_j, g_j[v] = w_v D_j + c_jv r;
//   hess b = cg gd gd^T + ch hess s,  gd = grad s / 2d, cg = b'' - b'/d, ch = b'/2d;
//   m(c) = (c/eps)(2 - c/eps), c = |ea x eb|^2 (below eps_x: the pair is
//   mollified), hess m = m'' gc gc^T + m' sg_v sg_u He, gc = grad c,
//   He = the 6x6 Hessian of c in the edge vectors.
// r, D_j, the edge vectors and their cross product (short for nearly
// parallel edges) are formed from the FP64 coordinates and rounded to T once
// formed, as in pair_hessian_lowrank.
template <class T>
struct MollTerms {
    T gd[12], g0[12], g1[12], gc[12], He[36], w[4];
    T i00, i01, i11, cg, ch, m, m1, m2, b, bp, kB;
};

template <class T>
__device__ void moll_terms(const double *Xd, const PairGrad &P, double d, double kB, T eps, MollTerms<T> &M) {
    Feature f = feature_of(true, P.type);
    T r[3], D[2][3];
    {
        double wd[4], rd[3] = {0, 0, 0}, Dd[2][3] = {{0, 0, 0}, {0, 0, 0}};
        for (int v = 0; v < 4; ++v) wd[v] = f.w0[v] + P.b0 * f.c[0][v] + P.b1 * f.c[1][v];
        for (int v = 0; v < 4; ++v)
            for (int a = 0; a < 3; ++a) {
                rd[a] += wd[v] * Xd[3 * v + a];
                Dd[0][a] += f.c[0][v] * Xd[3 * v + a];
                Dd[1][a] += f.c[1][v] * Xd[3 * v + a];
            }
        for (int v = 0; v < 4; ++v) M.w[v] = T(wd[v]);
        for (int a = 0; a < 3; ++a) {
            r[a] = T(rd[a]);
            D[0][a] = T(Dd[0][a]);
            D[1][a] = T(Dd[1][a]);
        }
    }
    const T dT = T(d), inv2d = T(1) / (T(2) * dT);
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) M.gd[3 * v + a] = T(2) * M.w[v] * r[a] * inv2d;
    M.i00 = M.i01 = M.i11 = T(0);
    if (f.k > 0) {
        T G00 = dot3(D[0], D[0]), G01 = dot3(D[0], D[1]), G11 = dot3(D[1], D[1]);
        if (f.k == 1) M.i00 = T(1) / G00;
        else {
            T det = G00 * G11 - G01 * G01;
            M.i00 = G11 / det; M.i11 = G00 / det; M.i01 = -G01 / det;
        }
    }
    for (int v = 0; v < 4; ++v)
        for (int a = 0; a < 3; ++a) {
            M.g0[3 * v + a] = M.w[v] * D[0][a] + T(f.c[0][v]) * r[a];
            M.g1[3 * v + a] = M.w[v] * D[1][a] + T(f.c[1][v]) * r[a];
        }
    M.bp = T(P.bp);
    M.cg = T(P.bpp) - M.bp / dT;
    M.ch = M.bp * inv2d;
    M.b = T(P.b);
    M.kB = T(kB);
    // mollifier: edge vectors and their cross product formed in FP64
    T ea[3], eb[3], cr[3], c;
    {
        double ead[3] = {Xd[3] - Xd[0], Xd[4] - Xd[1], Xd[5] - Xd[2]};
        double ebd[3] = {Xd[9] - Xd[6], Xd[10] - Xd[7], Xd[11] - Xd[8]};
        double crd[3] = {ead[1] * ebd[2] - ead[2] * ebd[1], ead[2] * ebd[0] - ead[0] * ebd[2],
                         ead[0] * ebd[1] - ead[1] * ebd[0]};
        for (int k = 0; k < 3; ++k) { ea[k] = T(ead[k]); eb[k] = T(ebd[k]); cr[k] = T(crd[k]); }
        c = T(crd[0] * crd[0] + crd[1] * crd[1] + crd[2] * crd[2]);
    }
    const T rr = c / eps;
    M.m = rr * (T(2) - rr);
    M.m1 = (T(2) - T(2) * rr) / eps;
    M.m2 = T(-2) / (eps * eps);
    T t[3];
    cross3(t, eb, cr);
    for (int k = 0; k < 3; ++k) { M.gc[k] = -T(2) * t[k]; M.gc[3 + k] = T(2) * t[k]; }
    cross3(t, cr, ea);
    for (int k = 0; k < 3; ++k) { M.gc[6 + k] = -T(2) * t[k]; M.gc[9 + k] = T(2) * t[k]; }
    // He = 2 J^T J + the cross-product coupling, J = [-[eb]x, [ea]x]
    const T J[3][6] = {{0, eb[2], -eb[1], 0, -ea[2], ea[1]},
                       {-eb[2], 0, eb[0], ea[2], 0, -ea[0]},
                       {eb[1], -eb[0], 0, -ea[1], ea[0], 0}};
    const T crx[3][3] = {{0, -cr[2], cr[1]}, {cr[2], 0, -cr[0]}, {-cr[1], cr[0], 0}};
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) M.He[6 * a + b] = T(2) * (J[0][a] * J[0][b] + J[1][a] * J[1][b] + J[2][a] * J[2][b]);
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            M.He[6 * j + 3 + k] -= T(2) * crx[j][k];
            M.He[6 * (3 + j) + k] += T(2) * crx[j][k];
        }
}

template <class T>
__device__ __forceinline__ void moll_entries(const MollTerms<T> &M, T *H, int lane) {
    for (int e = lane; e < 144; e += 32) {
        const int i = e / 12, j = e % 12, v = i / 3, a = i % 3, u = j / 3, c = j % 3;
        T hs = a == c ? T(2) * M.w[v] * M.w[u] : T(0);
        hs -= T(2) * (M.i00 * M.g0[i] * M.g0[j] + M.i01 * (M.g0[i] * M.g1[j] + M.g1[i] * M.g0[j]) +
                      M.i11 * M.g1[i] * M.g1[j]);
        const T hb = M.cg * M.gd[i] * M.gd[j] + M.ch * hs;
        const T sv = (v & 1) ? T(1) : T(-1), su = (u & 1) ? T(1) : T(-1);
        const T hm = M.m2 * M.gc[i] * M.gc[j] + M.m1 * sv * su * M.He[6 * (3 * (v >> 1) + a) + 3 * (u >> 1) + c];
        const T gmi = M.m1 * M.gc[i], gmj = M.m1 * M.gc[j], gbi = M.bp * M.gd[i], gbj = M.bp * M.gd[j];
        H[e] = M.kB * (hm * M.b + gmi * gbj + gbi * gmj + M.m * hb);
    }
}

// The mollified edge-edge pairs of the active list (ee_cross2 < eps_x: the
// pairs k_pair_assemble skips, in partitions still iterating), compacted into
// mlist[0 .. *mcount) so that k_pair_moll can give every one its own warp.
__global__ void k_moll_scan(AsmArgs A, const PairRec *__restrict__ act, const unsigned long long *__restrict__ n_dev,
                            int64_t cap, int64_t *__restrict__ mlist, unsigned long long *__restrict__ mcount) {
    const int64_t n = min((int64_t)*n_dev, cap);
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + lane;
        bool found = false;
        if (i < n) {
            const PairRec r = act[i];
            if (r.flags & 1) {
                int sa, sb;
                pair_slots(r, A.sv_slot, sa, sb);
                if (A.part[pair_part(sa, sb, A.S_dyn, A.slot_part)].active) {
                    double Xd[12];
                    for (int v = 0; v < 4; ++v)
                        for (int k = 0; k < 3; ++k)
                            Xd[3 * v + k] = A.x[3 * (int64_t)r.v[v] + k] - A.x[3 * (int64_t)r.v[0] + k];
                    found = ee_cross2(Xd) < r.eps;
                }
            }
        }
        const unsigned M = __ballot_sync(0xffffffffu, found);
        if (!M) continue;
        const int leader = __ffs(M) - 1;
        unsigned long long pos = 0;
        if (lane == leader) pos = atomicAdd(mcount, (unsigned long long)__popc(M));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (found) mlist[pos + __popc(M & ((1u << lane) - 1))] = i;
    }
}

// The mollified edge-edge pairs listed by k_moll_scan, one warp per pair
// (warps dealt over SMs, then SM sub-partitions, as in spread_base); it runs
// beside k_pair_assemble.  For each pair, lane 0 evaluates the FP64 gradient
// and the per-pair terms of the raw 12x12 Hessian (T), the lanes write its
// entries, the warp projects it to PSD and scatters J^T H J and the gradient
// onto the slots.  n_moll counts the pairs assembled.
template <class T>
__global__ void __launch_bounds__(128) k_pair_moll(AsmArgs A, const PairRec *__restrict__ act,
                                                   const int64_t *__restrict__ mlist,
                                                   const unsigned long long *__restrict__ mcount, int64_t cap,
                                                   const int2 *__restrict__ l1, T *__restrict__ diag,
                                                   T *__restrict__ off, int *__restrict__ offflag,
                                                   unsigned long long *__restrict__ n_moll) {
    __shared__ T sH[4][144], sW[4][144], sV[4][144], sR[4][12];
    __shared__ double sg[4][12], sw[4];
    __shared__ T sxi[4][4][4];
    __shared__ int ssl[4][4], sok[4];
    __shared__ MollTerms<T> smt[4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t n = min((int64_t)*mcount, cap), nw = (int64_t)gridDim.x * 4;
    for (int64_t t = spread_slot(); t < n; t += nw) {
        const PairRec r = act[mlist[t]];
        if (lane == 0) {
            int sa, sb;
            pair_slots(r, A.sv_slot, sa, sb);
            bool ee = r.flags & 1;
            double Xd[12];
            for (int v = 0; v < 4; ++v)
                for (int k = 0; k < 3; ++k) Xd[3 * v + k] = A.x[3 * (int64_t)r.v[v] + k] - A.x[3 * (int64_t)r.v[0] + k];
            PairGrad PG;
            const double kB = A.part[pair_part(sa, sb, A.S_dyn, A.slot_part)].kB;
            double d = pair_gradient(ee, Xd, A.dhat, kB, r.eps, PG, sg[wib]);
            sok[wib] = (d < A.dhat) && (d > 0.0);
            if (sok[wib]) {
                atomicAdd(n_moll, 1ull);
                moll_terms<T>(Xd, PG, d, kB, T(r.eps), smt[wib]);
                sw[wib] = A.h * A.h / pair_kappa(sa, sb, A.S_dyn, A.slot_mask);
                for (int v = 0; v < 4; ++v) {
                    int s = A.sv_slot[r.v[v]];
                    ssl[wib][v] = s < A.S_dyn ? s : -1;
                    int b = A.slot_body[s];
                    const double *xb = A.xbar + 3 * ((int64_t)A.voff[b] + (r.v[v] - A.slot_voff[s]));
                    sxi[wib][v][0] = T(1); sxi[wib][v][1] = T(xb[0]); sxi[wib][v][2] = T(xb[1]); sxi[wib][v][3] = T(xb[2]);
                }
            }
        }
        __syncwarp();
        const bool ok = sok[wib];
        __syncwarp();
        if (!ok) continue;
        moll_entries<T>(smt[wib], sH[wib], lane);
        __syncwarp();
        warp_psd12<T>(sH[wib], sW[wib], sV[wib], sR[wib], lane);
        const double w = sw[wib];
        const int *sl = ssl[wib];
        // gradient: 4 vertices x 3 components x 4 xi entries
        for (int e = lane; e < 48; e += 32) {
            int v = e / 12, k = (e / 4) % 3, a = e % 4;
            if (sl[v] < 0) continue;
            double xa = a == 0 ? 1.0 : (double)sxi[wib][v][a];
            atomicAdd(A.g + 12 * (int64_t)sl[v] + qidx(k, a), w * sg[wib][3 * v + k] * xa);
        }
        int sa = sl[0] >= 0 ? sl[0] : -1;
        int sb = sl[(r.flags & 1) ? 2 : 1];
        int ss[2] = {sa, sb};
        for (int bi = 0; bi < 2; ++bi)
            for (int bj = bi; bj < 2; ++bj) {
                int s1 = ss[bi], s2 = ss[bj];
                if (s1 < 0 || s2 < 0 || (bi != bj && s1 == s2)) continue;
                T *dst;
                bool tr = false;
                if (bi == bj) dst = diag + 144 * (int64_t)s1;
                else {
                    int2 lp = l1[r.l1];
                    dst = off + 144 * (int64_t)r.l1;
                    tr = (lp.x != s1);
                    if (lane == 0 && atomicExch(&offflag[r.l1], 1) == 0) {
                        atomicAdd(&A.rowcnt[lp.x], 1);
                        atomicAdd(&A.rowcnt[lp.y], 1);
                    }
                }
                for (int e = lane; e < 144; e += 32) {
                    int row = e / 12, col = e % 12;
                    int k = row < 3 ? row : (row - 3) / 3, a = row < 3 ? 0 : 1 + (row - 3) % 3;
                    int l = col < 3 ? col : (col - 3) / 3, c = col < 3 ? 0 : 1 + (col - 3) % 3;
                    T acc = T(0);
                    for (int v = 0; v < 4; ++v) {
                        if (sl[v] != s1) continue;
                        for (int u = 0; u < 4; ++u) {
                            if (sl[u] != s2) continue;
                            acc += sH[wib][(3 * v + k) * 12 + 3 * u + l] * sxi[wib][v][a] * sxi[wib][u][c];
                        }
                    }
                    T val = T(w) * acc;
                    if (val != T(0)) atomic_addT(dst + (tr ? col * 12 + row : row * 12 + col), val);
                }
            }
        __syncwarp();
    }
}

// Zero the off-diagonal blocks and flags of the first min(count, cap) level-1 pairs.
template <class T>
__global__ void k_zero_off(T *__restrict__ off, int *__restrict__ flag, const unsigned long long *__restrict__ n_dev,
                           int64_t cap) {
    int64_t n = min((int64_t)*n_dev, cap);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 144 * n; e += (int64_t)gridDim.x * blockDim.x) {
        off[e] = T(0);
        if (e % 144 == 0) flag[e / 144] = 0;
    }
}

// Exclusive scan of the per-slot block counts (one block of 1024 threads).
__global__ void k_csr_scan(int n, const int *__restrict__ cnt, int *__restrict__ off) {
    __shared__ int part[1024];
    int t = threadIdx.x, per = (n + 1023) / 1024, b = t * per, e = min(n, b + per);
    int loc = 0;
    for (int i = b; i < e; ++i) loc += cnt[i];
    part[t] = loc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - loc;
    for (int i = b; i < e; ++i) {
        off[i] = run;
        run += cnt[i];
    }
    if (t == 1023) off[n] = part[1023];
}

// Row CSR of the off-diagonal blocks: each flagged level-1 pair (a, b) is an
// entry (b, k) of row a and (a, k | transposed) of row b.
__global__ void k_csr_fill(const unsigned long long *__restrict__ n_dev, int64_t cap, const int2 *__restrict__ l1,
                           const int *__restrict__ flag, const int *__restrict__ off, int *__restrict__ cur,
                           int2 *__restrict__ ent) {
    int64_t n = min((int64_t)*n_dev, cap);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[k]) continue;
        int2 lp = l1[k];
        int pa = off[lp.x] + atomicAdd(&cur[lp.x], 1);
        ent[pa] = make_int2(lp.y, (int)k);
        int pb = off[lp.y] + atomicAdd(&cur[lp.y], 1);
        ent[pb] = make_int2(lp.x, (int)k | (int)0x80000000);
    }
}

// Vertex-plane barrier of dynamic slot vertices.
template <class T>
__global__ void k_vp_assemble(AsmArgs A, int64_t SVd, T *__restrict__ diag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < SVd; i += (int64_t)gridDim.x * blockDim.x) {
        int s = A.sv_slot[i];
        if (!A.part[A.slot_part[s]].active) continue;
        for (int pl = 0; pl < A.planes.n; ++pl) {
            int ax = A.planes.axis[pl];
            double d = A.planes.sign[pl] * A.x[3 * i + ax] - A.planes.offset[pl];
            if (!(d < A.dhat) || !(d > 0.0)) continue;
            double bb, b1, b2;
            barrier3<double>(d, A.dhat, bb, b1, b2);
            double w = A.h * A.h / (double)__popcll(A.slot_mask[s]) * A.part[A.slot_part[s]].kB;
            int b = A.slot_body[s];
            const double *xb = A.xbar + 3 * ((int64_t)A.voff[b] + (i - A.slot_voff[s]));
            double xi[4] = {1.0, xb[0], xb[1], xb[2]};
            double ga = w * b1 * A.planes.sign[pl], ha = w * b2;
            for (int a = 0; a < 4; ++a) atomicAdd(A.g + 12 * (int64_t)s + qidx(ax, a), ga * xi[a]);
            T *D = diag + 144 * (int64_t)s;
            for (int a = 0; a < 4; ++a)
                for (int c = 0; c < 4; ++c) atomic_addT(D + qidx(ax, a) * 12 + qidx(ax, c), T(ha * xi[a] * xi[c]));
        }
    }
}

// CCD over swept candidates: min TOI per partition; pairs that can come within
// dhat somewhere on the path (d0 - l_p < dhat, l_p bounding the distance
// change) go to the line-search list.
__global__ void k_ccd(const PairRec *__restrict__ cand, int64_t n, const unsigned long long *__restrict__ n_dev,
                      const double *__restrict__ x0,
                      const double *__restrict__ x1, const int *__restrict__ sv_slot, const int *__restrict__ slot_part,
                      int S_dyn, double dhat, double s_, double c_, PartState *__restrict__ part,
                      PairRec *__restrict__ ls, int64_t cap, unsigned long long *__restrict__ count, int want_ls) {
    if (n_dev) n = min((int64_t)*n_dev, n);
    for (int64_t base = spread_base(); base < n; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = base + (threadIdx.x & 31);
        bool keep = false;
        PairRec r;
        if (i < n) {
            r = cand[i];
            bool ee = r.flags & 1;
            double X[12], dX[12];
            for (int v = 0; v < 4; ++v)
                for (int k = 0; k < 3; ++k) {
                    double a = x0[3 * (int64_t)r.v[v] + k];
                    X[3 * v + k] = a;
                    dX[3 * v + k] = x1[3 * (int64_t)r.v[v] + k] - a;
                }
            int sa, sb;
            pair_slots(r, sv_slot, sa, sb);
            int p = pair_part(sa, sb, S_dyn, slot_part);
            double d0 = 0.0;
            double t = accd(ee, X, dX, s_, c_, 1000000, want_ls ? &d0 : nullptr);
            if (t < 1.0) atomicMin(&part[p].toi, ord(t));
            if (want_ls) {
                double mean[3] = {0, 0, 0}, nn[4];
                for (int v = 0; v < 4; ++v)
                    for (int k = 0; k < 3; ++k) mean[k] += 0.25 * dX[3 * v + k];
                for (int v = 0; v < 4; ++v) {
                    double a0 = dX[3 * v] - mean[0], a1 = dX[3 * v + 1] - mean[1], a2 = dX[3 * v + 2] - mean[2];
                    nn[v] = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
                }
                double lp = ee ? fmax(nn[0], nn[1]) + fmax(nn[2], nn[3]) : nn[0] + fmax(nn[1], fmax(nn[2], nn[3]));
                keep = d0 - lp < dhat;
            }
        }
        if (want_ls) append(keep, r, ls, cap, count);
    }
}

__global__ void k_vp_ccd(int64_t SVd, const double *__restrict__ x0, const double *__restrict__ x1,
                         const int *__restrict__ sv_slot, const int *__restrict__ slot_part, Planes pl, double s_,
                         PartState *__restrict__ part) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < SVd; i += (int64_t)gridDim.x * blockDim.x) {
        int p = slot_part[sv_slot[i]];
        if (!part[p].active) continue;
        for (int k = 0; k < pl.n; ++k) {
            int ax = pl.axis[k];
            double d0 = pl.sign[k] * x0[3 * i + ax] - pl.offset[k];
            double dd = pl.sign[k] * (x1[3 * i + ax] - x0[3 * i + ax]);
            double t = accd_plane(d0, dd, s_);
            if (t < 1.0) atomicMin(&part[p].toi, ord(t));
        }
    }
}

// Accumulate v into part[p].E[j].  Called by all 32 lanes with a uniform j;
// lanes with nothing to add pass p < 0.  One atomic per warp when every
// contributing lane has the same partition, else one per lane.
__device__ __forceinline__ void add_energy(PartState *part, int p, int j, double v) {
    const unsigned full = 0xffffffffu;
    int pmax = __reduce_max_sync(full, p);
    int pmin = __reduce_min_sync(full, p < 0 ? 0x7fffffff : p);
    if (pmax < 0) return;
    if (pmin == pmax) {
        double t = p < 0 ? 0.0 : v;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(full, t, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&part[pmax].E[j], t);
    } else if (p >= 0) {
        atomicAdd(&part[p].E[j], v);
    }
}

struct EnArgs {
    int S_dyn;
    const int *slot_body, *slot_part, *slot_rep, *sv_slot;
    const unsigned long long *slot_mask;
    const double *slot_kw, *mass, *S, *vol, *kappa;
    const double *q, *dq, *qtil, *z, *u, *rho;
    const double *x0, *x1;
    const double *alphas;  // [NP][kLS+1], alphas[.][0] = 0
    const int *live;       // 0: no partition has a trial step in this pass (every thread returns)
    PartState *part;  // per partition: active flag, trial-step energies, barrier stiffness kB
    double h, dhat;
    Planes planes;
};

__device__ double slot_energy(const EnArgs &A, int s, double al) {
    int b = A.slot_body[s];
    double q[12], d[12];
    for (int i = 0; i < 12; ++i) {
        q[i] = A.q[12 * (int64_t)s + i] + al * A.dq[12 * (int64_t)s + i];
        d[i] = q[i] - A.qtil[12 * (int64_t)s + i];
    }
    const double *S = A.S + 9 * (int64_t)b;
    double E = 0.5 * A.mass[b] * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) {
        const double *a = d + 3 + 3 * k;
        for (int i = 0; i < 3; ++i) E += 0.5 * a[i] * (S[3 * i] * a[0] + S[3 * i + 1] * a[1] + S[3 * i + 2] * a[2]);
    }
    double orth = 0.0;
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double c = q[3 + 3 * k] * q[3 + 3 * l] + q[4 + 3 * k] * q[4 + 3 * l] + q[5 + 3 * k] * q[5 + 3 * l] - (k == l);
            orth += c * c;
        }
    E += A.h * A.h * A.kappa[b] * A.vol[b] * orth;
    E *= A.slot_kw[s];
    if (A.slot_rep[s] >= 0) {
        double acc = 0.0;
        for (int i = 0; i < 12; ++i) {
            double r = q[i] - A.z[12 * (int64_t)s + i] + A.u[12 * (int64_t)s + i];
            acc += r * r;
        }
        E += 0.5 * A.rho[s] * acc;
    }
    return E;
}

// The line-search energy kernels give every (item, trial step j) its own lane
// when the list is short: the items are padded to whole warps for each j,
// t in [0, (kLS + 1) npad), j = t / npad, item t - j npad, so the lanes of a
// warp share j (add_energy sums a warp into one partition's E[j]) and a warp
// carries one FP64 chain instead of kLS + 1 in a row.  A long list (more
// than about two warps per SM sub-partition that way) keeps one lane per
// item looping over j, which loads each item once.  ls_range gives the
// iteration space and, per warp, the item offset and the steps [j0, j1).
constexpr int64_t kLsSplitItems = 32 * 152 * 8;
__device__ __forceinline__ int64_t ls_pad(int64_t n) { return (n + 31) & ~(int64_t)31; }
__device__ __forceinline__ int64_t ls_total(int64_t n) {
    const int64_t npad = ls_pad(n);
    return (kLS + 1) * npad <= kLsSplitItems ? (kLS + 1) * npad : npad;
}
__device__ __forceinline__ void ls_range(int64_t n, int64_t base, int64_t &first, int &j0, int &j1) {
    const int64_t npad = ls_pad(n);
    if ((kLS + 1) * npad <= kLsSplitItems) {
        j0 = (int)(base / npad);
        j1 = j0 + 1;
        first = base - (int64_t)j0 * npad;
    } else {
        j0 = 0;
        j1 = kLS + 1;
        first = base;
    }
}

__global__ void k_energy_slots(EnArgs A) {
    if (!*A.live) return;
    const int64_t total = ls_total(A.S_dyn);
    for (int64_t base = spread_base(); base < total; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t first;
        int j0, j1;
        ls_range(A.S_dyn, base, first, j0, j1);
        const int s = (int)(first + (threadIdx.x & 31));
        int p = s < A.S_dyn ? A.slot_part[s] : -1;
        if (p >= 0 && !A.part[p].active) p = -1;
        if (p >= 0 && A.alphas[(kLS + 1) * p] < 0.0) p = -1;  // partition already decided
        for (int j = j0; j < j1; ++j) {
            const double al = p >= 0 ? A.alphas[(kLS + 1) * p + j] : -1.0;
            const bool use = p >= 0 && (j == 0 || al >= 0.0);
            const double v = use ? slot_energy(A, s, al) : 0.0;
            add_energy(A.part, use ? p : -1, j, v);
        }
    }
}

__global__ void k_energy_pairs(EnArgs A, const PairRec *__restrict__ ls, int64_t n,
                               const unsigned long long *__restrict__ n_dev) {
    if (!*A.live) return;
    if (n_dev) n = min((int64_t)*n_dev, n);
    const int64_t total = ls_total(n);
    for (int64_t base = spread_base(); base < total; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t first;
        int j0, j1;
        ls_range(n, base, first, j0, j1);
        const int64_t i = first + (threadIdx.x & 31);
        int p = -1;
        PairRec r;
        double w = 0.0, kB = 0.0, X0[12], DX[12];
        if (i < n) {
            r = ls[i];
            int sa, sb;
            pair_slots(r, A.sv_slot, sa, sb);
            p = pair_part(sa, sb, A.S_dyn, A.slot_part);
            kB = A.part[p].kB;
            if (!A.part[p].active || A.alphas[(kLS + 1) * p] < 0.0) p = -1;
            w = A.h * A.h / pair_kappa(sa, sb, A.S_dyn, A.slot_mask);
            for (int v = 0; v < 4; ++v)
                for (int k = 0; k < 3; ++k) {
                    double a = A.x0[3 * (int64_t)r.v[v] + k];
                    X0[3 * v + k] = a;
                    DX[3 * v + k] = A.x1[3 * (int64_t)r.v[v] + k] - a;
                }
        }
        for (int j = j0; j < j1; ++j) {
            double al = p >= 0 ? A.alphas[(kLS + 1) * p + j] : -1.0;
            bool use = p >= 0 && (j == 0 || al >= 0.0);
            double e = 0.0;
            if (use) {
                double X[12], d;
                for (int q = 0; q < 12; ++q) X[q] = X0[q] + al * DX[q];
                e = w * pair_energy(r.flags & 1, X, A.dhat, kB, r.eps, d);
            }
            add_energy(A.part, use ? p : -1, j, e);
        }
    }
}

__global__ void k_energy_vp(EnArgs A, int64_t SVd) {
    if (!*A.live) return;
    const int64_t total = ls_total(SVd);
    for (int64_t base = spread_base(); base < total; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t first;
        int j0, j1;
        ls_range(SVd, base, first, j0, j1);
        const int64_t i = first + (threadIdx.x & 31);
        int p = -1, s = 0;
        if (i < SVd) {
            s = A.sv_slot[i];
            p = A.slot_part[s];
            if (!A.part[p].active || A.alphas[(kLS + 1) * p] < 0.0) p = -1;
        }
        const double w = p >= 0 ? A.h * A.h / (double)__popcll(A.slot_mask[s]) * A.part[p].kB : 0.0;
        for (int j = j0; j < j1; ++j) {
            const double al = p >= 0 ? A.alphas[(kLS + 1) * p + j] : -1.0;
            const bool use = p >= 0 && (j == 0 || al >= 0.0);
            double e = 0.0;
            if (use)
                for (int k = 0; k < A.planes.n; ++k) {
                    const int ax = A.planes.axis[k];
                    const double xa = A.x0[3 * i + ax] + al * (A.x1[3 * i + ax] - A.x0[3 * i + ax]);
                    const double d = A.planes.sign[k] * xa - A.planes.offset[k];
                    if (!(d > 0.0)) e += 1.0 / 0.0;
                    else if (d < A.dhat) {
                        double bb, b1, b2;
                        barrier3<double>(d, A.dhat, bb, b1, b2);
                        e += w * bb;
                    }
                }
            add_energy(A.part, use && e != 0.0 ? p : -1, j, e);
        }
    }
}

}  // namespace abd

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
namespace abd {

static AsmArgs make_asm(abd_scene *s, const abd_step_params *p) {
    World &w = s->w;
    AsmArgs A = {};
    A.S_dyn = w.S_dyn;
    A.slot_body = P<int>(w.slot_body); A.slot_part = P<int>(w.slot_part); A.slot_rep = P<int>(w.slot_rep);
    A.sv_slot = P<int>(w.sv_slot); A.slot_mask = P<unsigned long long>(w.slot_mask); A.slot_kw = P<double>(w.slot_kw);
    A.voff = P<int>(s->dev.voff); A.xbar = P<double>(s->dev.xbar); A.mass = P<double>(s->dev.mass);
    A.S = P<double>(s->dev.S); A.vol = P<double>(s->dev.vol); A.kappa = P<double>(s->dev.kappa);
    A.q = P<double>(w.q); A.qtil = P<double>(w.qtil); A.z = P<double>(w.z); A.u = P<double>(w.u);
    A.rho = P<double>(w.rho); A.x = P<double>(w.x); A.part = P<PartState>(w.part);
    A.h = p->h; A.dhat = p->dhat; A.planes = s->planes;
    A.slot_voff = P<int64_t>(w.slot_voff);
    A.g = P<double>(w.g);
    A.rowcnt = P<int>(w.rowcnt);
    return A;
}

// ---------------------------------------------------------------------------
// Asynchronous launchers (device counts, capacity-clamped; see abd_broad.cu).
// ---------------------------------------------------------------------------
int launch_narrow_async(abd_scene *s, const PairRec *src, const unsigned long long *src_n, int64_t src_cap,
                        double dhat) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    cudaMemsetAsync(&c->act, 0, 8, s->stream);
    ABD_LAUNCH(s, k_narrow, grid_for(src_cap, 256, 152 * 8), 256, 0, s->stream, src, src_cap, src_n, P<double>(w.x),
               dhat, P<PairRec>(w.act), w.cap_act, &c->act);
    return cuda_check(s, cudaGetLastError(), "k_narrow");
}

template <class T>
static int assemble_async_T(abd_scene *s, const abd_step_params *p) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    AsmArgs A = make_asm(s, p);
    cudaMemsetAsync(w.rowcnt.p, 0, sizeof(int) * (size_t)(w.S_dyn + 1), s->stream);
    cudaMemsetAsync(w.rowcur.p, 0, sizeof(int) * (size_t)(w.S_dyn + 1), s->stream);
    ABD_LAUNCH(s, k_zero_off<T>, grid_for(144 * w.cap_l1, 256, 152 * 8), 256, 0, s->stream, P<T>(w.off),
               P<int>(w.offflag), &c->l1, w.cap_l1);
    cudaEvent_t ea, eb;
    if (w.S_dyn > 0) {
        prof_begin(s, "slot_assemble", (double)w.S_dyn * (4 * 96 + 72 + 96 + 144.0 * sizeof(T)), &ea, &eb);
        ABD_LAUNCH(s, k_slot_assemble<T>, grid_for(w.S_dyn, 32, 152 * 8), 128, 0, s->stream, A, P<T>(w.diag));
        prof_end(s, ea, eb, prof_index(s, "slot_assemble"));
    }
    // w.nmoll: [0] pairs assembled, [1] pairs listed, the list from byte 64
    unsigned long long *nmoll = P<unsigned long long>(w.nmoll);
    int64_t *mlist = (int64_t *)((char *)w.nmoll.p + 64);
    cudaMemsetAsync(nmoll, 0, 16, s->stream);
    // the mollified pairs (one warp each, the longest chain) on the side
    // branch, beside the other pairs and the vertex-plane terms; both only
    // add onto what k_slot_assemble stored
    cudaStream_t side = fork_side(s);
    cudaEvent_t ma, mb;
    prof_begin(s, "pair_moll", 0.0, &ma, &mb, side);
    ABD_LAUNCH(s, k_moll_scan, grid_for(w.cap_act, 256, 152 * 8), 256, 0, side, A, P<PairRec>(w.act), &c->act,
               w.cap_act, mlist, nmoll + 1);
    ABD_LAUNCH(s, k_pair_moll<T>, 152 * 4, 128, 0, side, A, P<PairRec>(w.act), mlist, nmoll + 1, w.cap_act,
               P<int2>(w.l1), P<T>(w.diag), P<T>(w.off), P<int>(w.offflag), nmoll);
    prof_end(s, ma, mb, prof_index(s, "pair_moll"), side);
    prof_begin(s, "pair_assemble", 0.0, &ea, &eb);
    ABD_LAUNCH(s, k_pair_assemble<T>, grid_for(w.cap_act, 128, 152 * 8), 128, 0, s->stream, A,
               P<PairRec>(w.act), w.cap_act, P<int2>(w.l1), P<T>(w.diag), P<T>(w.off), P<int>(w.offflag), &c->act);
    prof_end(s, ea, eb, prof_index(s, "pair_assemble"));
    int64_t SVd = w.S_dyn > 0 ? w.h_slot_voff[w.S_dyn] : 0;
    if (s->planes.n > 0 && SVd > 0)
        ABD_LAUNCH(s, k_vp_assemble<T>, grid_for(SVd, 256), 256, 0, s->stream, A, SVd, P<T>(w.diag));
    join_side(s, side);
    ABD_LAUNCH(s, k_csr_scan, 1, 1024, 0, s->stream, w.S_dyn, P<int>(w.rowcnt), P<int>(w.rowoff));
    ABD_LAUNCH(s, k_csr_fill, grid_for(w.cap_l1, 256, 152 * 8), 256, 0, s->stream, &c->l1, w.cap_l1, P<int2>(w.l1),
               P<int>(w.offflag), P<int>(w.rowoff), P<int>(w.rowcur), P<int2>(w.ent));
    return cuda_check(s, cudaGetLastError(), "assemble");
}

int launch_assemble_async(abd_scene *s, int precision, const abd_step_params *p) {
    return precision == ABD_MIXED ? assemble_async_T<float>(s, p) : assemble_async_T<double>(s, p);
}

int launch_ccd_async(abd_scene *s, const abd_step_params *p, bool want_ls) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    int64_t SVd = w.S_dyn > 0 ? w.h_slot_voff[w.S_dyn] : 0;
    cudaMemsetAsync(&c->ls, 0, 8, s->stream);
    cudaEvent_t ea, eb;
    // pair CCD on the side branch, vertex-plane CCD beside it (both only
    // lower the partitions' TOI)
    cudaStream_t side = fork_side(s);
    prof_begin(s, "ccd", 0.0, &ea, &eb, side);
    ABD_LAUNCH(s, k_ccd, grid_for(w.cap_cand, 128, 152 * 8), 128, 0, side, P<PairRec>(w.cand), w.cap_cand, &c->cand,
               P<double>(w.x), P<double>(w.x1), P<int>(w.sv_slot), P<int>(w.slot_part), w.S_dyn, p->dhat, p->accd_s,
               p->accd_c, P<PartState>(w.part), P<PairRec>(w.ls), w.cap_ls, &c->ls, want_ls ? 1 : 0);
    prof_end(s, ea, eb, prof_index(s, "ccd"), side);
    if (s->planes.n > 0 && SVd > 0)
        ABD_LAUNCH(s, k_vp_ccd, grid_for(SVd, 256), 256, 0, s->stream, SVd, P<double>(w.x), P<double>(w.x1),
                   P<int>(w.sv_slot), P<int>(w.slot_part), s->planes, p->accd_s, P<PartState>(w.part));
    join_side(s, side);
    return cuda_check(s, cudaGetLastError(), "k_ccd");
}

int launch_energy_async(abd_scene *s, const abd_step_params *p, const double *alphas_dev) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    EnArgs A = {};
    A.S_dyn = w.S_dyn;
    A.slot_body = P<int>(w.slot_body); A.slot_part = P<int>(w.slot_part); A.slot_rep = P<int>(w.slot_rep);
    A.sv_slot = P<int>(w.sv_slot); A.slot_mask = P<unsigned long long>(w.slot_mask); A.slot_kw = P<double>(w.slot_kw);
    A.mass = P<double>(s->dev.mass); A.S = P<double>(s->dev.S); A.vol = P<double>(s->dev.vol);
    A.kappa = P<double>(s->dev.kappa);
    A.q = P<double>(w.q); A.dq = P<double>(w.dq); A.qtil = P<double>(w.qtil); A.z = P<double>(w.z);
    A.u = P<double>(w.u); A.rho = P<double>(w.rho); A.x0 = P<double>(w.x); A.x1 = P<double>(w.x1);
    A.alphas = alphas_dev; A.part = P<PartState>(w.part);
    A.live = &c->ls_live;
    A.h = p->h; A.dhat = p->dhat; A.planes = s->planes;
    int64_t SVd = w.S_dyn > 0 ? w.h_slot_voff[w.S_dyn] : 0;
    cudaEvent_t ea, eb;
    // the three sums are independent (each adds into the partitions' trial
    // energies): pairs on the side branch, slots then vertex-plane terms beside
    // them; the timed span covers both branches
    prof_begin(s, "energy", 0.0, &ea, &eb);
    cudaStream_t side = fork_side(s);
    ABD_LAUNCH(s, k_energy_pairs, grid_for(w.cap_ls, 128, 152 * 8), 128, 0, side, A, P<PairRec>(w.ls), w.cap_ls,
               &c->ls);
    if (w.S_dyn > 0)
        ABD_LAUNCH(s, k_energy_slots, grid_for((kLS + 1) * (int64_t)w.S_dyn, 32, 152 * 8), 128, 0, s->stream, A);
    if (s->planes.n > 0 && SVd > 0)
        ABD_LAUNCH(s, k_energy_vp, grid_for((kLS + 1) * SVd, 32, 152 * 8), 128, 0, s->stream, A, SVd);
    join_side(s, side);
    prof_end(s, ea, eb, prof_index(s, "energy"));
    return cuda_check(s, cudaGetLastError(), "energy");
}

// Final-state check: minimum distance over the candidate pairs (FP64
// closest-feature distance) and over dynamic vertices against the planes.
__global__ void k_min_dist(const PairRec *__restrict__ cand, int64_t cap, const unsigned long long *__restrict__ n_dev,
                           const double *__restrict__ x, unsigned long long *__restrict__ out) {
    int64_t n = min((int64_t)*n_dev, cap);
    for (int64_t base = spread_base(); base < n; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = base + (threadIdx.x & 31);
        if (i >= n) continue;
        PairRec r = cand[i];
        double X[12];
        for (int v = 0; v < 4; ++v)
            for (int k = 0; k < 3; ++k) X[3 * v + k] = x[3 * (int64_t)r.v[v] + k];
        int ty;
        double b0, b1;
        double d = sqrt(classify<double>(r.flags & 1, X, ty, b0, b1));
        atomicMin(out, ord(d));
    }
}

__global__ void k_min_dist_vp(int64_t SVd, const double *__restrict__ x, Planes planes,
                              unsigned long long *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < SVd; i += (int64_t)gridDim.x * blockDim.x) {
        double m = 1e300;
        for (int pl = 0; pl < planes.n; ++pl) {
            double d = planes.sign[pl] * x[3 * i + planes.axis[pl]] - planes.offset[pl];
            m = fmin(m, d > 0.0 ? d : 0.0);
        }
        if (m < 1e300) atomicMin(out, ord(m));
    }
}

int launch_min_dist_async(abd_scene *s) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    ABD_LAUNCH(s, k_min_dist, grid_for(w.cap_cand, 32, 152 * 8), 128, 0, s->stream, P<PairRec>(w.cand), w.cap_cand,
               &c->cand, P<double>(w.x), &c->mind);
    int64_t SVd = w.S_dyn > 0 ? w.h_slot_voff[w.S_dyn] : 0;
    if (s->planes.n > 0 && SVd > 0)
        ABD_LAUNCH(s, k_min_dist_vp, grid_for(SVd, 256), 256, 0, s->stream, SVd, P<double>(w.x), s->planes, &c->mind);
    return cuda_check(s, cudaGetLastError(), "min distance");
}

}  // namespace abd
