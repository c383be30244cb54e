// abd_broad.cu -- vertex transform and two-level broad phase on sm_103a.
//
// Level 1: slot boxes (dhat/2-inflated AABB of a replica's vertices, static or
// swept) and all overlapping slot pairs (same partition, or a slot against a
// static collider).  Level 2: one warp per level-1 pair streams the
// primitives of both slots, keeps those whose box meets the other slot's box
// (an exact filter: a primitive's box lies inside its slot's box), stages one
// side in shared memory and tests the other side against it; hits are
// compacted with warp ballots into the global list.  The resulting set is the
// plain definition -- every PT (both directions) and EE pair of different
// slots, not both static, whose dhat/2-inflated boxes overlap -- evaluated
// with exact FP64 min/max and one rounding per bound.
#include "abd_broad.cuh"

namespace abd {

// ---------------------------------------------------------------------------
// x = A xbar + p per slot vertex.  mode 0: slot q; mode 1: q + dq (dynamic
// slots); mode 2: shared dynamic slots take the consensus z, others q.
// ---------------------------------------------------------------------------
__global__ void k_transform(int64_t SV, const int *__restrict__ sv_slot, const int *__restrict__ slot_body,
                            const int64_t *__restrict__ slot_voff, const int *__restrict__ voff,
                            const double *__restrict__ xbar, const double *__restrict__ q,
                            const double *__restrict__ alt, const int *__restrict__ slot_rep, int S_dyn, int mode,
                            double *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < SV; i += (int64_t)gridDim.x * blockDim.x) {
        int s = sv_slot[i];
        int b = slot_body[s];
        const double *xb = xbar + 3 * ((int64_t)voff[b] + (i - slot_voff[s]));
        const double *qs = q + 12 * (int64_t)s;
        double qq[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) qq[k] = qs[k];
        if (s < S_dyn) {
            if (mode == 1) {
#pragma unroll
                for (int k = 0; k < 12; ++k) qq[k] += alt[12 * (int64_t)s + k];
            } else if (mode == 2 && slot_rep[s] >= 0) {
#pragma unroll
                for (int k = 0; k < 12; ++k) qq[k] = alt[12 * (int64_t)s + k];
            }
        }
        double x0 = xb[0], x1 = xb[1], x2 = xb[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) x[3 * i + k] = qq[k] + (qq[3 + 3 * k] * x0 + qq[4 + 3 * k] * x1 + qq[5 + 3 * k] * x2);
    }
}

// One warp per slot: inflated AABB of its vertices (over x0 and x1 if given).
__global__ void k_boxes(int S, const int64_t *__restrict__ slot_voff, const double *__restrict__ x0,
                        const double *__restrict__ x1, double half, double *__restrict__ box) {
    int lane = threadIdx.x & 31;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += (gridDim.x * blockDim.x) >> 5) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int64_t v = slot_voff[s] + lane; v < slot_voff[s + 1]; v += 32)
            for (int k = 0; k < 3; ++k) {
                double a = x0[3 * v + k];
                lo[k] = fmin(lo[k], a);
                hi[k] = fmax(hi[k], a);
                if (x1) {
                    double c = x1[3 * v + k];
                    lo[k] = fmin(lo[k], c);
                    hi[k] = fmax(hi[k], c);
                }
            }
        for (int o = 16; o; o >>= 1)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        if (lane < 3) box[6 * (int64_t)s + lane] = lo[lane] - half;
        else if (lane < 6) box[6 * (int64_t)s + lane] = hi[lane - 3] + half;
    }
}

__device__ __forceinline__ bool overlap6(const double *a, const double *b) {
    return !(a[0] > b[3] || b[0] > a[3] || a[1] > b[4] || b[1] > a[4] || a[2] > b[5] || b[2] > a[5]);
}

// Level 1: slot pairs (a < b) with overlapping boxes, in the same partition or
// against a static collider (slot_part < 0); partitions not marked active are
// skipped.  Thread per (a, tile of 32 b's).
__global__ void k_l1(int S_all, const int *__restrict__ slot_part, const double *__restrict__ box,
                     const PartState *__restrict__ part, int2 *__restrict__ out, int64_t cap,
                     unsigned long long *__restrict__ count) {
    int64_t ntile = (S_all + 31) / 32;
    int64_t total = (int64_t)S_all * ntile;
    int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += (int64_t)gridDim.x * blockDim.x) {
        int64_t idx = base + threadIdx.x;
        int a = -1, b0 = 0, b1 = 0;
        if (idx < total) {
            a = (int)(idx / ntile);
            b0 = (int)(idx % ntile) * 32;
            b1 = min(S_all, b0 + 32);
            if (b1 <= a + 1) a = -1;
            b0 = max(b0, a + 1);
        }
        int pa = a >= 0 ? slot_part[a] : -2;
        bool act_a = a >= 0 && (pa < 0 || part[pa].active);
        double ba[6];
        if (act_a)
            for (int k = 0; k < 6; ++k) ba[k] = box[6 * (int64_t)a + k];
        for (int j = 0; j < 32; ++j) {
            int b = b0 + j;
            bool hit = false;
            if (act_a && b < b1) {
                int pb = slot_part[b];
                bool ok = (pa >= 0 && pb >= 0) ? (pa == pb) : (pa >= 0 || pb >= 0);
                if (ok && pb >= 0 && !part[pb].active) ok = false;
                if (ok) {
                    double bb[6];
                    for (int k = 0; k < 6; ++k) bb[k] = box[6 * (int64_t)b + k];
                    hit = overlap6(ba, bb);
                }
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) {
                unsigned long long pos = 0;
                int leader = __ffs(m) - 1;
                if (lane == leader) pos = atomicAdd(count, (unsigned long long)__popc(m));
                pos = __shfl_sync(0xffffffffu, pos, leader);
                if (hit) {
                    unsigned long long my = pos + __popc(m & ((1u << lane) - 1));
                    if ((int64_t)my < cap) out[my] = make_int2(a, b);
                }
            }
        }
    }
}



// Primitive kind: 0 vertex, 1 triangle, 2 edge.  Fills the slot-vertex ids and
// returns the number of vertices.
__device__ __forceinline__ int prim_verts(const L2Args &A, int kind, int slot, int idx, int sv[3]) {
    int b = A.slot_body[slot];
    int64_t base = A.slot_voff[slot];
    if (kind == 0) { sv[0] = (int)(base + idx); return 1; }
    if (kind == 1) {
        const int *t = A.tri + 3 * ((int64_t)A.toff[b] + idx);
        sv[0] = (int)(base + t[0]); sv[1] = (int)(base + t[1]); sv[2] = (int)(base + t[2]);
        return 3;
    }
    const int *e = A.edge + 2 * ((int64_t)A.eoff[b] + idx);
    sv[0] = (int)(base + e[0]); sv[1] = (int)(base + e[1]);
    return 2;
}

__device__ __forceinline__ void prim_box(const L2Args &A, const int *sv, int n, double *bx) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            double a = A.x0[3 * (int64_t)sv[i] + k];
            lo[k] = fmin(lo[k], a);
            hi[k] = fmax(hi[k], a);
            if (A.x1) {
                double c = A.x1[3 * (int64_t)sv[i] + k];
                lo[k] = fmin(lo[k], c);
                hi[k] = fmax(hi[k], c);
            }
        }
    for (int k = 0; k < 3; ++k) { bx[k] = lo[k] - A.half; bx[3 + k] = hi[k] + A.half; }
}

__device__ __forceinline__ int prim_count(const L2Args &A, int kind, int slot) {
    int b = A.slot_body[slot];
    return kind == 0 ? A.nv[b] : (kind == 1 ? A.nt[b] : A.ne[b]);
}

constexpr int kStage = 64;

__global__ void __launch_bounds__(32 * kL2Warps) k_l2(L2Args A) {
    __shared__ double st_box[kL2Warps][kStage][6];
    __shared__ int st_idx[kL2Warps][kStage];
    int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int gw = blockIdx.x * kL2Warps + wib, nw = gridDim.x * kL2Warps;
    int64_t npairs = A.n_l1;
    if (A.n_l1_dev) npairs = min((int64_t)*A.n_l1_dev, A.n_l1);
    for (int64_t p = gw; p < npairs; p += nw) {
        int2 pr = A.l1[p];
        double boxS[2][6];
        for (int k = 0; k < 6; ++k) { boxS[0][k] = A.box[6 * (int64_t)pr.x + k]; boxS[1][k] = A.box[6 * (int64_t)pr.y + k]; }
        for (int job = 0; job < 3; ++job) {
            // job 0: vertices of x vs triangles of y; 1: vertices of y vs triangles of x; 2: edges x vs edges y
            int s1 = job == 1 ? pr.y : pr.x, s2 = job == 1 ? pr.x : pr.y;
            int k1 = job == 2 ? 2 : 0, k2 = job == 2 ? 2 : 1;
            const double *box1 = boxS[job == 1 ? 1 : 0], *box2 = boxS[job == 1 ? 0 : 1];
            int n1 = prim_count(A, k1, s1), n2 = prim_count(A, k2, s2);
            int i = 0;
            while (i < n1) {
                int nst = 0;
                for (; i < n1 && nst + 32 <= kStage; i += 32) {
                    int idx = i + lane;
                    bool keep = false;
                    double bx[6];
                    if (idx < n1) {
                        int sv[3];
                        int nvx = prim_verts(A, k1, s1, idx, sv);
                        prim_box(A, sv, nvx, bx);
                        keep = overlap6(bx, box2);
                    }
                    unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (keep) {
                        int pos = nst + __popc(m & ((1u << lane) - 1));
                        st_idx[wib][pos] = idx;
                        for (int k = 0; k < 6; ++k) st_box[wib][pos][k] = bx[k];
                    }
                    nst += __popc(m);
                }
                __syncwarp();
                if (nst == 0) continue;
                for (int j = 0; j < n2; j += 32) {
                    int idx2 = j + lane;
                    bool keep = false;
                    double bx[6];
                    int sv2[3];
                    int nv2 = 0;
                    if (idx2 < n2) {
                        nv2 = prim_verts(A, k2, s2, idx2, sv2);
                        prim_box(A, sv2, nv2, bx);
                        keep = overlap6(bx, box1);
                    }
                    if (!__any_sync(0xffffffffu, keep)) continue;
                    for (int k = 0; k < nst; ++k) {
                        bool hit = keep && overlap6(bx, st_box[wib][k]);
                        unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (!m) continue;
                        unsigned long long pos = 0;
                        int leader = __ffs(m) - 1;
                        if (lane == leader) pos = atomicAdd(A.count, (unsigned long long)__popc(m));
                        pos = __shfl_sync(0xffffffffu, pos, leader);
                        if (!hit) continue;
                        unsigned long long my = pos + __popc(m & ((1u << lane) - 1));
                        if ((int64_t)my >= A.cap) continue;
                        int idx1 = st_idx[wib][k];
                        int sv1[3];
                        prim_verts(A, k1, s1, idx1, sv1);
                        int b1 = A.slot_body[s1], b2 = A.slot_body[s2];
                        if (A.mode == 0) {
                            int32_t *o = A.out3 + 3 * my;
                            if (job < 2) {
                                o[0] = 0;
                                o[1] = A.voff[b1] + idx1;
                                o[2] = A.toff[b2] + idx2;
                            } else {
                                int ea = A.eoff[b1] + idx1, eb = A.eoff[b2] + idx2;
                                o[0] = 1;
                                o[1] = min(ea, eb);
                                o[2] = max(ea, eb);
                            }
                        } else {
                            PairRec r;
                            r.l1 = (int)p;
                            if (job < 2) {
                                r.v[0] = sv1[0]; r.v[1] = sv2[0]; r.v[2] = sv2[1]; r.v[3] = sv2[2];
                                r.flags = 0;
                                r.eps = 0.0;
                            } else {
                                r.v[0] = sv1[0]; r.v[1] = sv1[1]; r.v[2] = sv2[0]; r.v[3] = sv2[1];
                                r.flags = 1;
                                r.eps = 1e-3 * A.erest2[A.eoff[b1] + idx1] * A.erest2[A.eoff[b2] + idx2];
                            }
                            A.recs[my] = r;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

// One warp per primitive cluster: box of its (up to 32) primitives' vertices
// over x0 (and x1), inflated by half.  It contains every primitive box of the
// cluster, so it filters exactly.
__global__ void k_cluster_boxes(int64_t C, const int2 *__restrict__ cl_info, const int *__restrict__ slot_body,
                                const int64_t *__restrict__ slot_voff, const int *__restrict__ nv,
                                const int *__restrict__ toff, const int *__restrict__ nt, const int *__restrict__ eoff,
                                const int *__restrict__ ne, const int *__restrict__ voff, const int *__restrict__ tri,
                                const int *__restrict__ edge, const int *__restrict__ vperm,
                                const int *__restrict__ tperm, const int *__restrict__ eperm,
                                const double *__restrict__ x0, const double *__restrict__ x1, double half,
                                double *__restrict__ cbox) {
    int lane = threadIdx.x & 31;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < C;
         c += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int2 info = cl_info[c];
        int slot = info.x, kind = info.y >> 24, j = info.y & 0xffffff;
        int b = slot_body[slot];
        int64_t base = slot_voff[slot];
        int n = kind == 0 ? nv[b] : (kind == 1 ? nt[b] : ne[b]);
        int i = kClusterSize * j + lane;
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        if (i < n) {
            int sv[3], k = 0;
            if (kind == 0) sv[k++] = (int)(base + vperm[voff[b] + i]);
            else if (kind == 1) {
                const int *t = tri + 3 * ((int64_t)toff[b] + tperm[toff[b] + i]);
                sv[0] = (int)(base + t[0]); sv[1] = (int)(base + t[1]); sv[2] = (int)(base + t[2]);
                k = 3;
            } else {
                const int *e = edge + 2 * ((int64_t)eoff[b] + eperm[eoff[b] + i]);
                sv[0] = (int)(base + e[0]); sv[1] = (int)(base + e[1]);
                k = 2;
            }
            for (int q = 0; q < k; ++q)
                for (int a = 0; a < 3; ++a) {
                    double v = x0[3 * (int64_t)sv[q] + a];
                    lo[a] = fmin(lo[a], v);
                    hi[a] = fmax(hi[a], v);
                    if (x1) {
                        double u = x1[3 * (int64_t)sv[q] + a];
                        lo[a] = fmin(lo[a], u);
                        hi[a] = fmax(hi[a], u);
                    }
                }
        }
        for (int o = 16; o; o >>= 1)
            for (int a = 0; a < 3; ++a) {
                lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
                hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
            }
        if (lane < 3) cbox[6 * c + lane] = lo[lane] - half;
        else if (lane < 6) cbox[6 * c + lane] = hi[lane - 3] + half;
    }
}

__device__ __forceinline__ int cl_count(const L2Args &A, int kind, int body) {
    int n = kind == 0 ? A.nv[body] : (kind == 1 ? A.nt[body] : A.ne[body]);
    return (n + kClusterSize - 1) / kClusterSize;
}

__device__ __forceinline__ int cl_first(const L2cArgs &A, int kind, int slot, int body) {
    int c = A.slot_cbase[slot];
    if (kind >= 1) c += cl_count(A.a, 0, body);
    if (kind >= 2) c += cl_count(A.a, 1, body);
    return c;
}

__device__ __forceinline__ int cl_prim(const L2cArgs &A, int kind, int body, int i) {
    return kind == 0 ? A.vperm[A.a.voff[body] + i] : (kind == 1 ? A.tperm[A.a.toff[body] + i] : A.eperm[A.a.eoff[body] + i]);
}

// Test the staged side-1 primitives against every side-2 primitive of the
// side-2 clusters that meet both the side-1 slot box and the staged set's box;
// emit the hits (ballot-compacted).
__device__ void l2c_flush(const L2cArgs &A, int64_t p, int job, int s1, int s2, int k1, int k2, int b2,
                          const double *box1, const double *stbox, const double (*st_box)[6], const int *st_idx,
                          int nst, int lane) {
    const L2Args &B = A.a;
    int n2 = k2 == 0 ? B.nv[b2] : (k2 == 1 ? B.nt[b2] : B.ne[b2]);
    int nc2 = (n2 + kClusterSize - 1) / kClusterSize, cb2 = cl_first(A, k2, s2, b2);
    for (int cbk = 0; cbk < nc2; cbk += 32) {
        int c = cbk + lane;
        bool ok = false;
        if (c < nc2) {
            const double *cbx = A.cbox + 6 * (int64_t)(cb2 + c);
            ok = overlap6(cbx, box1) && overlap6(cbx, stbox);
        }
        unsigned m = __ballot_sync(0xffffffffu, ok);
        while (m) {
            int cc = cbk + __ffs(m) - 1;
            m &= m - 1;
            int i2 = kClusterSize * cc + lane;
            bool keep = false;
            double bx[6];
            int idx2 = -1, sv2[3];
            if (i2 < n2) {
                idx2 = cl_prim(A, k2, b2, i2);
                int nv2 = prim_verts(B, k2, s2, idx2, sv2);
                prim_box(B, sv2, nv2, bx);
                keep = overlap6(bx, box1) && overlap6(bx, stbox);
            }
            if (!__any_sync(0xffffffffu, keep)) continue;
            for (int k = 0; k < nst; ++k) {
                bool hit = keep && overlap6(bx, st_box[k]);
                unsigned hm = __ballot_sync(0xffffffffu, hit);
                if (!hm) continue;
                unsigned long long pos = 0;
                int leader = __ffs(hm) - 1;
                if (lane == leader) pos = atomicAdd(B.count, (unsigned long long)__popc(hm));
                pos = __shfl_sync(0xffffffffu, pos, leader);
                if (!hit) continue;
                unsigned long long my = pos + __popc(hm & ((1u << lane) - 1));
                if ((int64_t)my >= B.cap) continue;
                int idx1 = st_idx[k];
                int sv1[3];
                prim_verts(B, k1, s1, idx1, sv1);
                int b1 = B.slot_body[s1];
                if (B.mode == 0) {
                    int32_t *o = B.out3 + 3 * my;
                    if (job < 2) {
                        o[0] = 0;
                        o[1] = B.voff[b1] + idx1;
                        o[2] = B.toff[b2] + idx2;
                    } else {
                        int ea = B.eoff[b1] + idx1, eb = B.eoff[b2] + idx2;
                        o[0] = 1;
                        o[1] = min(ea, eb);
                        o[2] = max(ea, eb);
                    }
                } else {
                    PairRec r;
                    r.l1 = (int)p;
                    if (job < 2) {
                        r.v[0] = sv1[0]; r.v[1] = sv2[0]; r.v[2] = sv2[1]; r.v[3] = sv2[2];
                        r.flags = 0;
                        r.eps = 0.0;
                    } else {
                        r.v[0] = sv1[0]; r.v[1] = sv1[1]; r.v[2] = sv2[0]; r.v[3] = sv2[1];
                        r.flags = 1;
                        r.eps = 1e-3 * B.erest2[B.eoff[b1] + idx1] * B.erest2[B.eoff[b2] + idx2];
                    }
                    B.recs[my] = r;
                }
            }
        }
    }
}

// Level 2 with primitive clusters: one warp per level-1 slot pair.  Side-1
// clusters meeting the side-2 slot box are opened and their primitives that
// meet the side-2 box are staged; each full stage is flushed against the
// side-2 clusters (see l2c_flush).  Same set as k_l2.
__global__ void __launch_bounds__(32 * kL2Warps) k_l2c(L2cArgs A) {
    __shared__ double st_box[kL2Warps][kStage][6];
    __shared__ int st_idx[kL2Warps][kStage];
    const L2Args &B = A.a;
    int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int gw = blockIdx.x * kL2Warps + wib, nw = gridDim.x * kL2Warps;
    int64_t npairs = B.n_l1;
    if (B.n_l1_dev) npairs = min((int64_t)*B.n_l1_dev, B.n_l1);
    for (int64_t p = gw; p < npairs; p += nw) {
        int2 pr = B.l1[p];
        double boxS[2][6];
        for (int k = 0; k < 6; ++k) { boxS[0][k] = B.box[6 * (int64_t)pr.x + k]; boxS[1][k] = B.box[6 * (int64_t)pr.y + k]; }
        for (int job = 0; job < 3; ++job) {
            int s1 = job == 1 ? pr.y : pr.x, s2 = job == 1 ? pr.x : pr.y;
            int k1 = job == 2 ? 2 : 0, k2 = job == 2 ? 2 : 1;
            const double *box1 = boxS[job == 1 ? 1 : 0], *box2 = boxS[job == 1 ? 0 : 1];
            int b1 = B.slot_body[s1], b2 = B.slot_body[s2];
            int n1 = k1 == 0 ? B.nv[b1] : (k1 == 1 ? B.nt[b1] : B.ne[b1]);
            int nc1 = (n1 + kClusterSize - 1) / kClusterSize, cb1 = cl_first(A, k1, s1, b1);
            int nst = 0;
            double stbox[6] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300};
            for (int cbk = 0; cbk < nc1; cbk += 32) {
                int c = cbk + lane;
                bool ok = c < nc1 && overlap6(A.cbox + 6 * (int64_t)(cb1 + c), box2);
                unsigned m = __ballot_sync(0xffffffffu, ok);
                while (m) {
                    int cc = cbk + __ffs(m) - 1;
                    m &= m - 1;
                    int i1 = kClusterSize * cc + lane;
                    bool keep = false;
                    double bx[6];
                    int idx1 = -1;
                    if (i1 < n1) {
                        int sv[3];
                        idx1 = cl_prim(A, k1, b1, i1);
                        int nvx = prim_verts(B, k1, s1, idx1, sv);
                        prim_box(B, sv, nvx, bx);
                        keep = overlap6(bx, box2);
                    }
                    unsigned km = __ballot_sync(0xffffffffu, keep);
                    int cnt = __popc(km);
                    if (cnt == 0) continue;
                    if (nst + cnt > kStage) {
                        __syncwarp();
                        l2c_flush(A, p, job, s1, s2, k1, k2, b2, box1, stbox, st_box[wib], st_idx[wib], nst, lane);
                        nst = 0;
                        for (int a = 0; a < 3; ++a) { stbox[a] = 1e300; stbox[3 + a] = -1e300; }
                        __syncwarp();
                    }
                    if (keep) {
                        int pos = nst + __popc(km & ((1u << lane) - 1));
                        st_idx[wib][pos] = idx1;
                        for (int k = 0; k < 6; ++k) st_box[wib][pos][k] = bx[k];
                    }
                    nst += cnt;
                    for (int a = 0; a < 3; ++a) {
                        double l = keep ? bx[a] : 1e300, h = keep ? bx[3 + a] : -1e300;
                        for (int o = 16; o; o >>= 1) {
                            l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
                            h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
                        }
                        stbox[a] = fmin(stbox[a], l);
                        stbox[3 + a] = fmax(stbox[3 + a], h);
                    }
                }
            }
            if (nst > 0) {
                __syncwarp();
                l2c_flush(A, p, job, s1, s2, k1, k2, b2, box1, stbox, st_box[wib], st_idx[wib], nst, lane);
                __syncwarp();
            }
        }
    }
}

}  // namespace abd

using namespace abd;

namespace abd {

int launch_transform(abd_scene *s, const double *q_slots, double *x, const double *alt, int mode) {
    World &w = s->w;
    if (w.SV == 0) return ABD_OK;
    ABD_LAUNCH(s, k_transform, grid_for(w.SV, 256), 256, 0, s->stream, w.SV, P<int>(w.sv_slot), P<int>(w.slot_body),
                                                           P<int64_t>(w.slot_voff), P<int>(s->dev.voff),
                                                           P<double>(s->dev.xbar), q_slots, alt, P<int>(w.slot_rep),
                                                           w.S_dyn, mode, x);
    return cuda_check(s, cudaGetLastError(), "k_transform");
}

int launch_boxes(abd_scene *s, const double *x0, const double *x1, double half, double *box) {
    World &w = s->w;
    if (w.S_all == 0) return ABD_OK;
    ABD_LAUNCH(s, k_boxes, grid_for((int64_t)w.S_all * 32, 256), 256, 0, s->stream, w.S_all, P<int64_t>(w.slot_voff), x0, x1,
                                                                          half, box);
    // primitive-cluster boxes for the level-2 pass (static or swept set)
    if (w.C > 0)
        ABD_LAUNCH(s, k_cluster_boxes, grid_for(w.C * 32, 256), 256, 0, s->stream, w.C, P<int2>(w.cl_info),
                   P<int>(w.slot_body), P<int64_t>(w.slot_voff), P<int>(s->dev.nv), P<int>(s->dev.toff),
                   P<int>(s->dev.nt), P<int>(s->dev.eoff), P<int>(s->dev.ne), P<int>(s->dev.voff), P<int>(s->dev.tri),
                   P<int>(s->dev.edge), P<int>(s->dev.vperm), P<int>(s->dev.tperm), P<int>(s->dev.eperm), x0, x1, half,
                   x1 ? P<double>(w.cbox1) : P<double>(w.cbox));
    return cuda_check(s, cudaGetLastError(), "k_boxes");
}

static L2cArgs cluster_args(abd_scene *s, const L2Args &a, bool swept) {
    L2cArgs C;
    C.a = a;
    C.vperm = P<int>(s->dev.vperm);
    C.tperm = P<int>(s->dev.tperm);
    C.eperm = P<int>(s->dev.eperm);
    C.slot_cbase = P<int>(s->w.slot_cbase);
    C.cbox = swept ? P<double>(s->w.cbox1) : P<double>(s->w.cbox);
    return C;
}

// Read a device counter (synchronises the stream).
static int read_counter(abd_scene *s, unsigned long long *dptr, unsigned long long *h) {
    cudaError_t e = cudaMemcpyAsync(h, dptr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_check(s, e, "read counter");
}

int launch_l1(abd_scene *s, const double *box, int64_t *count) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    if (w.cap_l1 == 0) {
        w.cap_l1 = 4 * (int64_t)w.S_all + 1024;
        if (!dbuf_ensure(w.l1, 8 * w.cap_l1)) return set_err(s, ABD_E_OOM, "l1 list");
    }
    for (;;) {
        cudaMemsetAsync(&c->l1, 0, sizeof(unsigned long long), s->stream);
        int64_t ntile = (w.S_all + 31) / 32;
        ABD_LAUNCH(s, k_l1, grid_for((int64_t)w.S_all * ntile, 256), 256, 0, s->stream, w.S_all, P<int>(w.slot_part), box,
                                                                             P<PartState>(w.part), P<int2>(w.l1),
                                                                             w.cap_l1, &c->l1);
        int rc = cuda_check(s, cudaGetLastError(), "k_l1");
        if (rc) return rc;
        unsigned long long n = 0;
        if ((rc = read_counter(s, &c->l1, &n))) return rc;
        if ((int64_t)n <= w.cap_l1) {
            *count = (int64_t)n;
            return ABD_OK;
        }
        w.cap_l1 = (int64_t)n + n / 2 + 1024;
        if (!dbuf_ensure(w.l1, 8 * w.cap_l1)) return set_err(s, ABD_E_OOM, "l1 list");
    }
}

int launch_l2(abd_scene *s, int mode, const double *x0, const double *x1, double half, int64_t n_l1, int32_t *out3,
              int64_t cap, int64_t *count) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    L2Args A = {};
    A.slot_body = P<int>(w.slot_body);
    A.slot_voff = P<int64_t>(w.slot_voff);
    A.voff = P<int>(s->dev.voff); A.nv = P<int>(s->dev.nv); A.toff = P<int>(s->dev.toff); A.nt = P<int>(s->dev.nt);
    A.eoff = P<int>(s->dev.eoff); A.ne = P<int>(s->dev.ne); A.tri = P<int>(s->dev.tri); A.edge = P<int>(s->dev.edge);
    A.erest2 = P<double>(s->dev.erest2);
    A.x0 = x0; A.x1 = x1; A.box = x1 ? P<double>(w.box1) : P<double>(w.box);
    A.half = half;
    A.l1 = P<int2>(w.l1);
    A.n_l1 = n_l1;
    A.n_l1_dev = nullptr;
    A.mode = mode;
    A.out3 = out3;
    A.count = &c->cand;
    if (mode == 1 && w.cap_cand == 0) {
        w.cap_cand = 1 << 16;
        if (!dbuf_ensure(w.cand, sizeof(PairRec) * w.cap_cand)) return set_err(s, ABD_E_OOM, "candidate list");
    }
    for (;;) {
        A.recs = P<PairRec>(w.cand);
        A.cap = mode == 1 ? w.cap_cand : cap;
        cudaMemsetAsync(&c->cand, 0, sizeof(unsigned long long), s->stream);
        if (n_l1 > 0) {
            cudaEvent_t ea, eb;
            // compulsory unique bytes: slot-vertex positions (one or two
            // configurations), triangle and edge indices of the slots' bodies,
            // the level-1 list and the emitted records
            double bytes = 0.0;
            if (s->prof) {
                double tri_e = 0.0;
                for (int sl = 0; sl < w.S_all; ++sl) {
                    int b = w.h_slot_body[sl];
                    tri_e += 12.0 * s->nt[b] + 8.0 * s->ne[b];
                }
                bytes = (x1 ? 48.0 : 24.0) * (double)w.SV + tri_e + 8.0 * (double)n_l1;
            }
            prof_begin(s, x1 ? "l2_swept" : "l2_static", bytes, &ea, &eb);
            ABD_LAUNCH(s, k_l2c, grid_for(n_l1, kL2Warps, 152 * 16), 32 * kL2Warps, 0, s->stream,
                       cluster_args(s, A, x1 != nullptr));
            prof_end(s, ea, eb, prof_index(s, x1 ? "l2_swept" : "l2_static"));
        }
        int rc = cuda_check(s, cudaGetLastError(), "k_l2");
        if (rc) return rc;
        unsigned long long n = 0;
        if ((rc = read_counter(s, &c->cand, &n))) return rc;
        *count = (int64_t)n;
        if (s->prof && n_l1 > 0) prof_add_bytes(s, x1 ? "l2_swept" : "l2_static", (double)sizeof(PairRec) * (double)n);
        if (mode == 0 || (int64_t)n <= w.cap_cand) return ABD_OK;
        w.cap_cand = (int64_t)n + n / 2 + 1024;
        if (!dbuf_ensure(w.cand, sizeof(PairRec) * w.cap_cand)) return set_err(s, ABD_E_OOM, "candidate list");
    }
}

// ---------------------------------------------------------------------------
// Asynchronous variants for the Newton loop: counts stay on the device, the
// kernels clamp to the buffer capacity, and the host checks counts against
// capacities once per iteration (a count above its capacity means the
// iteration is redone with larger buffers).
// ---------------------------------------------------------------------------
int launch_l1_async(abd_scene *s, const double *box) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    cudaMemsetAsync(&c->l1, 0, sizeof(unsigned long long), s->stream);
    int64_t ntile = (w.S_all + 31) / 32;
    ABD_LAUNCH(s, k_l1, grid_for((int64_t)w.S_all * ntile, 256), 256, 0, s->stream, w.S_all, P<int>(w.slot_part), box,
               P<PartState>(w.part), P<int2>(w.l1), w.cap_l1, &c->l1);
    return cuda_check(s, cudaGetLastError(), "k_l1");
}

int launch_l2_async(abd_scene *s, const double *x0, const double *x1, double half) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    L2Args A = {};
    A.slot_body = P<int>(w.slot_body);
    A.slot_voff = P<int64_t>(w.slot_voff);
    A.voff = P<int>(s->dev.voff); A.nv = P<int>(s->dev.nv); A.toff = P<int>(s->dev.toff); A.nt = P<int>(s->dev.nt);
    A.eoff = P<int>(s->dev.eoff); A.ne = P<int>(s->dev.ne); A.tri = P<int>(s->dev.tri); A.edge = P<int>(s->dev.edge);
    A.erest2 = P<double>(s->dev.erest2);
    A.x0 = x0; A.x1 = x1; A.box = x1 ? P<double>(w.box1) : P<double>(w.box);
    A.half = half;
    A.l1 = P<int2>(w.l1);
    A.n_l1 = w.cap_l1;
    A.n_l1_dev = &c->l1;
    A.mode = 1;
    A.out3 = nullptr;
    A.recs = P<PairRec>(w.cand);
    A.cap = w.cap_cand;
    A.count = &c->cand;
    cudaMemsetAsync(&c->cand, 0, sizeof(unsigned long long), s->stream);
    cudaEvent_t ea, eb;
    double bytes = 0.0;
    if (s->prof) {
        double tri_e = 0.0;
        for (int sl = 0; sl < w.S_all; ++sl) {
            int b = w.h_slot_body[sl];
            tri_e += 12.0 * s->nt[b] + 8.0 * s->ne[b];
        }
        bytes = (x1 ? 48.0 : 24.0) * (double)w.SV + tri_e;
    }
    prof_begin(s, x1 ? "l2_swept" : "l2_static", bytes, &ea, &eb);
    ABD_LAUNCH(s, k_l2c, grid_for(w.cap_l1, kL2Warps, 152 * 16), 32 * kL2Warps, 0, s->stream,
               cluster_args(s, A, x1 != nullptr));
    prof_end(s, ea, eb, prof_index(s, x1 ? "l2_swept" : "l2_static"));
    return cuda_check(s, cudaGetLastError(), "k_l2");
}

}  // namespace abd
