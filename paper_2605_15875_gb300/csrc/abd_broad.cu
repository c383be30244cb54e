// abd_broad.cu -- vertex transform and broad phase on sm_103a.
//
// Level 1: slot boxes (dhat/2-inflated AABB of a replica's vertices, static or
// swept) and all overlapping slot pairs (same partition, or a slot against a
// static collider).  Level 2, solver path: stage A lists, per slot pair, the
// pairs of primitive clusters (32 Morton-ordered primitives of one kind)
// whose boxes overlap; stage B takes one warp per cluster pair, lane i holding
// primitive i of each cluster, filters both sides against the other slot's
// and cluster's box (exact filters: a primitive's box lies inside both),
// stages the smaller kept set in shared memory and tests the other set
// against it; hits are compacted with warp ballots.  The no-allocation query
// keeps the older one-warp-per-slot-pair pass (k_l2) on FP64 boxes.  The
// resulting set is the plain definition -- every PT (both directions) and EE
// pair of different slots, not both static, whose dhat/2-inflated boxes
// overlap -- evaluated with exact FP64 min/max and one rounding per bound.
//
// FP64 instructions are scarce on this GPU, so the solver's broad phase
// filters in FP32: every vertex coordinate carries FP32 bounds rounded
// outward (down and up), and every slot, cluster and primitive box built from
// them is rounded outward as well, so it contains the FP64 box.  Only pairs
// whose FP32 primitive boxes overlap are tested again with the FP64 boxes,
// which decide; the list is the same set as the FP64-only pass.
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
                            double *__restrict__ x, float *__restrict__ xb) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < SV; i += (int64_t)gridDim.x * blockDim.x) {
        int s = sv_slot[i];
        int b = slot_body[s];
        const double *xr = xbar + 3 * ((int64_t)voff[b] + (i - slot_voff[s]));
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
        double x0 = xr[0], x1 = xr[1], x2 = xr[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v = qq[k] + (qq[3 + 3 * k] * x0 + qq[4 + 3 * k] * x1 + qq[5 + 3 * k] * x2);
            x[3 * i + k] = v;
            if (xb) {
                xb[6 * i + k] = __double2float_rd(v);
                xb[6 * i + 3 + k] = __double2float_ru(v);
            }
        }
    }
}

// FP32 bounds (rounded down, rounded up) of caller-given FP64 positions.
__global__ void k_vert_bounds(int64_t SV, const double *__restrict__ x, float *__restrict__ xb) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * SV; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = i / 3;
        int k = (int)(i - 3 * v);
        xb[6 * v + k] = __double2float_rd(x[i]);
        xb[6 * v + 3 + k] = __double2float_ru(x[i]);
    }
}

// One warp per slot: FP32 box of its vertex bounds (over both configurations
// when xb1 is given), inflated outward by halfu >= dhat / 2.
__global__ void k_boxes32(int S, const int64_t *__restrict__ slot_voff, const float *__restrict__ xb0,
                          const float *__restrict__ xb1, float halfu, float *__restrict__ box) {
    int lane = threadIdx.x & 31;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += (gridDim.x * blockDim.x) >> 5) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t v = slot_voff[s] + lane; v < slot_voff[s + 1]; v += 32)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], xb0[6 * v + k]);
                hi[k] = fmaxf(hi[k], xb0[6 * v + 3 + k]);
                if (xb1) {
                    lo[k] = fminf(lo[k], xb1[6 * v + k]);
                    hi[k] = fmaxf(hi[k], xb1[6 * v + 3 + k]);
                }
            }
        for (int o = 16; o; o >>= 1)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        if (lane < 3) box[6 * (int64_t)s + lane] = __fsub_rd(lo[lane], halfu);
        else if (lane < 6) box[6 * (int64_t)s + lane] = __fadd_ru(hi[lane - 3], halfu);
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



__device__ __forceinline__ bool overlapf(const float *a, const float *b) {
    return !(a[0] > b[3] || b[0] > a[3] || a[1] > b[4] || b[1] > a[4] || a[2] > b[5] || b[2] > a[5]);
}

// Level 1 on FP32 boxes (same pairing rules as k_l1).  `cross` instead pairs
// slots of different bodies across partitions too (not two static slots): the
// whole-scene check of the final state.
__global__ void k_l1f(int S_all, const int *__restrict__ slot_part, const float *__restrict__ box,
                     const PartState *__restrict__ part, int2 *__restrict__ out, int64_t cap,
                     unsigned long long *__restrict__ count, const int *__restrict__ slot_body, int cross) {
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
        float ba[6];
        if (act_a)
            for (int k = 0; k < 6; ++k) ba[k] = box[6 * (int64_t)a + k];
        for (int j = 0; j < 32; ++j) {
            int b = b0 + j;
            bool hit = false;
            if (act_a && b < b1) {
                int pb = slot_part[b];
                bool ok = cross ? ((pa >= 0 || pb >= 0) && slot_body[a] != slot_body[b])
                               : ((pa >= 0 && pb >= 0) ? (pa == pb) : (pa >= 0 || pb >= 0));
                if (ok && pb >= 0 && !part[pb].active) ok = false;
                if (ok) {
                    float bb[6];
                    for (int k = 0; k < 6; ++k) bb[k] = box[6 * (int64_t)b + k];
                    hit = overlapf(ba, bb);
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



// Level 1 within partitions: one warp per dynamic slot a of an active
// partition tests the later slots of its own partition (slots are sorted by
// partition) and the static colliders that serve it (static_grp -1: every
// partition), with ballot compaction of the hits (a, b), a < b.  The set is
// k_l1f's non-cross set; the work is the sum over partitions of n_p^2 / 2
// instead of S^2 / 2, so the scenes of a batched world never meet.
__global__ void k_l1_part(int S_dyn, int S_all, const int *__restrict__ slot_part, const int *__restrict__ part_off,
                          const int *__restrict__ static_grp, const float *__restrict__ box,
                          const PartState *__restrict__ part, int2 *__restrict__ out, int64_t cap,
                          unsigned long long *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int n_static = S_all - S_dyn;
    for (int a = blockIdx.x + gridDim.x * (threadIdx.x >> 5); a < S_dyn; a += nw) {
        const int pa = slot_part[a];
        if (!part[pa].active) continue;  // warp-uniform
        float ba[6];
        for (int k = 0; k < 6; ++k) ba[k] = box[6 * (int64_t)a + k];
        const int n1 = part_off[pa + 1] - (a + 1), tot = n1 + n_static;
        for (int j0 = 0; j0 < tot; j0 += 32) {
            const int j = j0 + lane;
            int b = -1;
            if (j < n1) b = a + 1 + j;
            else if (j < tot) {
                const int g = static_grp[j - n1];
                if (g < 0 || g == pa) b = S_dyn + (j - n1);
            }
            bool hit = false;
            if (b >= 0) {
                float bb[6];
                for (int k = 0; k < 6; ++k) bb[k] = box[6 * (int64_t)b + k];
                hit = overlapf(ba, bb);
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

// FP32 outward box of a primitive from its vertices' bounds (contains the
// FP64 box of prim_box).
__device__ __forceinline__ void prim_boxf(const L2Args &A, const int *sv, int n, float *bx) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], A.xb0[6 * (int64_t)sv[i] + k]);
            hi[k] = fmaxf(hi[k], A.xb0[6 * (int64_t)sv[i] + 3 + k]);
            if (A.xb1) {
                lo[k] = fminf(lo[k], A.xb1[6 * (int64_t)sv[i] + k]);
                hi[k] = fmaxf(hi[k], A.xb1[6 * (int64_t)sv[i] + 3 + k]);
            }
        }
    for (int k = 0; k < 3; ++k) { bx[k] = __fsub_rd(lo[k], A.halfu); bx[3 + k] = __fadd_ru(hi[k], A.halfu); }
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

// One warp per primitive cluster: FP32 box of its (up to 32) primitives'
// vertex bounds over xb0 (and xb1), inflated outward by halfu.  It contains
// every primitive box of the cluster.
__global__ void k_cluster_boxes(int64_t C, const int2 *__restrict__ cl_info, const int *__restrict__ slot_body,
                                const int64_t *__restrict__ slot_voff, const int *__restrict__ nv,
                                const int *__restrict__ toff, const int *__restrict__ nt, const int *__restrict__ eoff,
                                const int *__restrict__ ne, const int *__restrict__ voff, const int *__restrict__ tri,
                                const int *__restrict__ edge, const int *__restrict__ vperm,
                                const int *__restrict__ tperm, const int *__restrict__ eperm,
                                const float *__restrict__ xb0, const float *__restrict__ xb1, float halfu,
                                float *__restrict__ cbox) {
    int lane = threadIdx.x & 31;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < C;
         c += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int2 info = cl_info[c];
        int slot = info.x, kind = info.y >> 24, j = info.y & 0xffffff;
        int b = slot_body[slot];
        int64_t base = slot_voff[slot];
        int n = kind == 0 ? nv[b] : (kind == 1 ? nt[b] : ne[b]);
        int i = kClusterSize * j + lane;
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
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
                    lo[a] = fminf(lo[a], xb0[6 * (int64_t)sv[q] + a]);
                    hi[a] = fmaxf(hi[a], xb0[6 * (int64_t)sv[q] + 3 + a]);
                    if (xb1) {
                        lo[a] = fminf(lo[a], xb1[6 * (int64_t)sv[q] + a]);
                        hi[a] = fmaxf(hi[a], xb1[6 * (int64_t)sv[q] + 3 + a]);
                    }
                }
        }
        for (int o = 16; o; o >>= 1)
            for (int a = 0; a < 3; ++a) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
            }
        if (lane < 3) cbox[6 * c + lane] = __fsub_rd(lo[lane], halfu);
        else if (lane < 6) cbox[6 * c + lane] = __fadd_ru(hi[lane - 3], halfu);
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

// Emit one primitive pair (side-1 primitive idx1 with slot vertices sv1,
// side-2 primitive idx2 with sv2) at list position `my`.
__device__ __forceinline__ void l2_emit(const L2Args &B, unsigned long long my, int p, int job, int b1, int b2,
                                        int idx1, const int *sv1, int idx2, const int *sv2) {
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
        return;
    }
    PairRec r;
    r.l1 = p;
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

// Stage A of level 2: one warp per level-1 slot pair lists the cluster pairs
// (c1, c2) of its three jobs whose boxes overlap, c1 meeting the side-2 slot
// box and c2 the side-1 slot box.  Lanes hold side-2 cluster boxes; side-1
// cluster boxes are broadcast by shuffles.
__global__ void __launch_bounds__(32 * kL2Warps) k_cpairs(L2cArgs A) {
    const L2Args &B = A.a;
    int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int gw = blockIdx.x * kL2Warps + wib, nw = gridDim.x * kL2Warps;
    int64_t npairs = B.n_l1;
    if (B.n_l1_dev) npairs = min((int64_t)*B.n_l1_dev, B.n_l1);
    for (int64_t p = gw; p < npairs; p += nw) {
        int2 pr = B.l1[p];
        float boxS[2][6];
        for (int k = 0; k < 6; ++k) { boxS[0][k] = B.boxf[6 * (int64_t)pr.x + k]; boxS[1][k] = B.boxf[6 * (int64_t)pr.y + k]; }
        for (int job = 0; job < 3; ++job) {
            // job 0: vertices of x vs triangles of y; 1: vertices of y vs triangles of x; 2: edges x vs edges y
            int s1 = job == 1 ? pr.y : pr.x, s2 = job == 1 ? pr.x : pr.y;
            int k1 = job == 2 ? 2 : 0, k2 = job == 2 ? 2 : 1;
            const float *box1 = boxS[job == 1 ? 1 : 0], *box2 = boxS[job == 1 ? 0 : 1];
            int b1 = B.slot_body[s1], b2 = B.slot_body[s2];
            int nc1 = cl_count(B, k1, b1), cb1 = cl_first(A, k1, s1, b1);
            int nc2 = cl_count(B, k2, b2), cb2 = cl_first(A, k2, s2, b2);
            for (int c2b = 0; c2b < nc2; c2b += 32) {
                float m2[6];
                bool v2 = false;
                if (c2b + lane < nc2) {
                    const float *cb = A.cbox + 6 * (int64_t)(cb2 + c2b + lane);
                    for (int k = 0; k < 6; ++k) m2[k] = cb[k];
                    v2 = overlapf(m2, box1);
                }
                if (!__any_sync(0xffffffffu, v2)) continue;
                for (int c1b = 0; c1b < nc1; c1b += 32) {
                    float m1[6];
                    bool v1 = false;
                    if (c1b + lane < nc1) {
                        const float *cb = A.cbox + 6 * (int64_t)(cb1 + c1b + lane);
                        for (int k = 0; k < 6; ++k) m1[k] = cb[k];
                        v1 = overlapf(m1, box2);
                    }
                    unsigned M1 = __ballot_sync(0xffffffffu, v1);
                    while (M1) {
                        int src = __ffs(M1) - 1;
                        M1 &= M1 - 1;
                        float o[6];
                        for (int k = 0; k < 6; ++k) o[k] = __shfl_sync(0xffffffffu, m1[k], src);
                        bool hit = v2 && overlapf(m2, o);
                        unsigned hm = __ballot_sync(0xffffffffu, hit);
                        if (!hm) continue;
                        unsigned long long pos = 0;
                        int leader = __ffs(hm) - 1;
                        if (lane == leader) pos = atomicAdd(A.n_cp, (unsigned long long)__popc(hm));
                        pos = __shfl_sync(0xffffffffu, pos, leader);
                        if (!hit) continue;
                        unsigned long long my = pos + __popc(hm & ((1u << lane) - 1));
                        if ((int64_t)my < A.cap_cp) A.cp[my] = make_int4(cb1 + c1b + src, cb2 + c2b + lane, (int)p, job);
                    }
                }
            }
        }
    }
}

// Stage B of level 2: one warp per cluster pair.  Lane i takes primitive i of
// each cluster; a side-1 primitive is kept when its FP32 box meets the side-2
// slot box and cluster box, a side-2 primitive likewise.  The smaller kept set
// is staged in shared memory and every lane of the other set tests its
// primitive against each staged one, in FP32 and, where that overlaps, again
// with the FP64 boxes, which decide.  A pair of primitives is tested in
// exactly one cluster pair, so the list has no duplicates; every filter box
// contains the FP64 primitive boxes, so the list is the full set.
__global__ void __launch_bounds__(32 * kL2Warps, 6) k_l2p(L2cArgs A) {
    __shared__ float st_box[kL2Warps][32][6];
    __shared__ int st_sv[kL2Warps][32][3];
    __shared__ int st_idx[kL2Warps][32];
    const L2Args &B = A.a;
    int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int gw = blockIdx.x * kL2Warps + wib, nw = gridDim.x * kL2Warps;
    int64_t n = min((int64_t)*A.n_cp, A.cap_cp);
    for (int64_t t = gw; t < n; t += nw) {
        int4 r = A.cp[t];
        int2 i1 = A.cl_info[r.x], i2 = A.cl_info[r.y];
        int s1 = i1.x, k1 = i1.y >> 24, j1 = i1.y & 0xffffff;
        int s2 = i2.x, k2 = i2.y >> 24, j2 = i2.y & 0xffffff;
        int b1 = B.slot_body[s1], b2 = B.slot_body[s2];
        const float *box1 = B.boxf + 6 * (int64_t)s1, *box2 = B.boxf + 6 * (int64_t)s2;
        const float *cbx1 = A.cbox + 6 * (int64_t)r.x, *cbx2 = A.cbox + 6 * (int64_t)r.y;
        int n1 = k1 == 0 ? B.nv[b1] : (k1 == 1 ? B.nt[b1] : B.ne[b1]);
        int n2 = k2 == 0 ? B.nv[b2] : (k2 == 1 ? B.nt[b2] : B.ne[b2]);
        int nv1 = k1 == 0 ? 1 : (k1 == 1 ? 3 : 2), nv2 = k2 == 0 ? 1 : (k2 == 1 ? 3 : 2);
        int ia = kClusterSize * j1 + lane, ib = kClusterSize * j2 + lane;
        bool keep1 = false, keep2 = false;
        float bx1[6], bx2[6];
        int sv1[3] = {0, 0, 0}, sv2[3] = {0, 0, 0}, idx1 = -1, idx2 = -1;
        if (ia < n1) {
            idx1 = cl_prim(A, k1, b1, ia);
            prim_boxf(B, sv1, prim_verts(B, k1, s1, idx1, sv1), bx1);
            keep1 = overlapf(bx1, box2) && overlapf(bx1, cbx2);
        }
        if (ib < n2) {
            idx2 = cl_prim(A, k2, b2, ib);
            prim_boxf(B, sv2, prim_verts(B, k2, s2, idx2, sv2), bx2);
            keep2 = overlapf(bx2, box1) && overlapf(bx2, cbx1);
        }
        unsigned K1 = __ballot_sync(0xffffffffu, keep1), K2 = __ballot_sync(0xffffffffu, keep2);
        if (!K1 || !K2) continue;
        // stage the smaller set (side 1 when `one`), loop over it
        bool one = __popc(K1) <= __popc(K2);
        if (one ? keep1 : keep2) {
            const float *bx = one ? bx1 : bx2;
            const int *sv = one ? sv1 : sv2;
            for (int k = 0; k < 6; ++k) st_box[wib][lane][k] = bx[k];
            st_sv[wib][lane][0] = sv[0]; st_sv[wib][lane][1] = sv[1]; st_sv[wib][lane][2] = sv[2];
            st_idx[wib][lane] = one ? idx1 : idx2;
        }
        __syncwarp();
        bool other = one ? keep2 : keep1;
        const float *obx = one ? bx2 : bx1;
        const int *osv = one ? sv2 : sv1;
        int onv = one ? nv2 : nv1, snv = one ? nv1 : nv2;
        double ob64[6];
        bool have64 = false;
        unsigned M = one ? K1 : K2;
        while (M) {
            int k = __ffs(M) - 1;
            M &= M - 1;
            bool hit = other && overlapf(obx, st_box[wib][k]);
            if (hit) {
                // FP64 boxes decide
                if (!have64) { prim_box(B, osv, onv, ob64); have64 = true; }
                double sb64[6];
                prim_box(B, st_sv[wib][k], snv, sb64);
                hit = overlap6(ob64, sb64);
            }
            unsigned hm = __ballot_sync(0xffffffffu, hit);
            if (!hm) continue;
            unsigned long long pos = 0;
            int leader = __ffs(hm) - 1;
            if (lane == leader) pos = atomicAdd(B.count, (unsigned long long)__popc(hm));
            pos = __shfl_sync(0xffffffffu, pos, leader);
            if (!hit) continue;
            unsigned long long my = pos + __popc(hm & ((1u << lane) - 1));
            if ((int64_t)my >= B.cap) continue;
            if (one)
                l2_emit(B, my, r.z, r.w, b1, b2, st_idx[wib][k], st_sv[wib][k], idx2, sv2);
            else
                l2_emit(B, my, r.z, r.w, b1, b2, idx1, sv1, st_idx[wib][k], st_sv[wib][k]);
        }
        __syncwarp();
    }
}

// Cluster boxes straight from the affine DOFs.  A cluster's vertices satisfy
// xbar = c + d with |d| <= e (its rest-frame box), so x = A xbar + p lies in
// the box with centre A c + p and half extent |A| e.  Both configurations
// (q, and the mode's second one) are covered.  The arithmetic is FP32; the
// box is padded by 1e-5 of the magnitudes involved (FP32 rounding of the
// inputs and of these few operations is below 1e-6 of them), so it contains
// every FP64 primitive box of the cluster.
__global__ void k_cluster_boxes_q(int64_t C, const int2 *__restrict__ cl_info, const int *__restrict__ slot_cbase,
                                  const int *__restrict__ slot_body, const int *__restrict__ cbody_off,
                                  const float *__restrict__ crest, const double *__restrict__ q,
                                  const double *__restrict__ alt, const int *__restrict__ slot_rep, int S_dyn,
                                  int mode, float halfu, float *__restrict__ cbox) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        int slot = cl_info[c].x;
        int b = slot_body[slot];
        const float *rb = crest + 6 * ((int64_t)cbody_off[b] + (c - slot_cbase[slot]));
        float ce[3] = {rb[0], rb[1], rb[2]}, he[3] = {rb[3], rb[4], rb[5]};
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        int ncfg = mode < 0 ? 1 : 2;
        for (int cfg = 0; cfg < ncfg; ++cfg) {
            const double *qs = q + 12 * (int64_t)slot;
            bool add = false;
            if (cfg == 1 && slot < S_dyn) {
                if (mode == 1) add = true;
                else if (mode == 2 && slot_rep[slot] >= 0) qs = alt + 12 * (int64_t)slot;
            }
            float qq[12];
            for (int k = 0; k < 12; ++k) qq[k] = (float)(add ? qs[k] + alt[12 * (int64_t)slot + k] : qs[k]);
            for (int k = 0; k < 3; ++k) {
                const float *Ak = qq + 3 + 3 * k;
                float m = qq[k] + (Ak[0] * ce[0] + Ak[1] * ce[1] + Ak[2] * ce[2]);
                float r = fabsf(Ak[0]) * he[0] + fabsf(Ak[1]) * he[1] + fabsf(Ak[2]) * he[2];
                float pad = 1e-5f * (fabsf(qq[k]) + fabsf(Ak[0]) * (fabsf(ce[0]) + he[0]) +
                                     fabsf(Ak[1]) * (fabsf(ce[1]) + he[1]) + fabsf(Ak[2]) * (fabsf(ce[2]) + he[2])) +
                            1e-30f;
                lo[k] = fminf(lo[k], m - r - pad);
                hi[k] = fmaxf(hi[k], m + r + pad);
            }
        }
        for (int k = 0; k < 3; ++k) {
            cbox[6 * c + k] = __fsub_rd(lo[k], halfu);
            cbox[6 * c + 3 + k] = __fadd_ru(hi[k], halfu);
        }
    }
}

}  // namespace abd

using namespace abd;

namespace abd {

// dhat / 2 rounded up to FP32.
static float half_up(double half) {
    float h = (float)half;
    if ((double)h < half) h = std::nextafter(h, INFINITY);
    return h;
}

int launch_transform(abd_scene *s, const double *q_slots, double *x, const double *alt, int mode) {
    World &w = s->w;
    if (w.SV == 0) return ABD_OK;
    float *xb = x == P<double>(w.x) ? P<float>(w.xb) : (x == P<double>(w.x1) ? P<float>(w.xb1) : nullptr);
    ABD_LAUNCH(s, k_transform, grid_for(w.SV, 256), 256, 0, s->stream, w.SV, P<int>(w.sv_slot), P<int>(w.slot_body),
               P<int64_t>(w.slot_voff), P<int>(s->dev.voff), P<double>(s->dev.xbar), q_slots, alt, P<int>(w.slot_rep),
               w.S_dyn, mode, x, xb);
    return cuda_check(s, cudaGetLastError(), "k_transform");
}

int launch_vert_bounds(abd_scene *s, bool swept) {
    World &w = s->w;
    if (w.SV == 0) return ABD_OK;
    ABD_LAUNCH(s, k_vert_bounds, grid_for(3 * w.SV, 256), 256, 0, s->stream, w.SV, P<double>(w.x), P<float>(w.xb));
    if (swept)
        ABD_LAUNCH(s, k_vert_bounds, grid_for(3 * w.SV, 256), 256, 0, s->stream, w.SV, P<double>(w.x1),
                   P<float>(w.xb1));
    return cuda_check(s, cudaGetLastError(), "k_vert_bounds");
}

int launch_boxes(abd_scene *s, bool swept, double half, int cmode, const double *alt) {
    World &w = s->w;
    if (w.S_all == 0) return ABD_OK;
    float hu = half_up(half);
    const float *xb1 = swept ? P<float>(w.xb1) : nullptr;
    ABD_LAUNCH(s, k_boxes32, grid_for((int64_t)w.S_all * 32, 256), 256, 0, s->stream, w.S_all, P<int64_t>(w.slot_voff),
               P<float>(w.xb), xb1, hu, swept ? P<float>(w.box1) : P<float>(w.box));
    // primitive-cluster boxes for the level-2 pass (static or swept set)
    float *cb = swept ? P<float>(w.cbox1) : P<float>(w.cbox);
    if (w.C > 0 && cmode == -2)
        ABD_LAUNCH(s, k_cluster_boxes, grid_for(w.C * 32, 256), 256, 0, s->stream, w.C, P<int2>(w.cl_info),
                   P<int>(w.slot_body), P<int64_t>(w.slot_voff), P<int>(s->dev.nv), P<int>(s->dev.toff),
                   P<int>(s->dev.nt), P<int>(s->dev.eoff), P<int>(s->dev.ne), P<int>(s->dev.voff), P<int>(s->dev.tri),
                   P<int>(s->dev.edge), P<int>(s->dev.vperm), P<int>(s->dev.tperm), P<int>(s->dev.eperm),
                   P<float>(w.xb), xb1, hu, cb);
    else if (w.C > 0)
        ABD_LAUNCH(s, k_cluster_boxes_q, grid_for(w.C, 128), 128, 0, s->stream, w.C, P<int2>(w.cl_info),
                   P<int>(w.slot_cbase), P<int>(w.slot_body), P<int>(s->dev.cbody_off), P<float>(s->dev.crest),
                   P<double>(w.q), alt, P<int>(w.slot_rep), w.S_dyn, swept ? cmode : -1, hu, cb);
    return cuda_check(s, cudaGetLastError(), "k_boxes");
}

// Level-2 arguments for the solver's lists over w.x (and w.x1 when swept).
static L2Args l2_args(abd_scene *s, bool swept, double half) {
    World &w = s->w;
    L2Args A = {};
    A.slot_body = P<int>(w.slot_body);
    A.slot_voff = P<int64_t>(w.slot_voff);
    A.voff = P<int>(s->dev.voff); A.nv = P<int>(s->dev.nv); A.toff = P<int>(s->dev.toff); A.nt = P<int>(s->dev.nt);
    A.eoff = P<int>(s->dev.eoff); A.ne = P<int>(s->dev.ne); A.tri = P<int>(s->dev.tri); A.edge = P<int>(s->dev.edge);
    A.erest2 = P<double>(s->dev.erest2);
    A.x0 = P<double>(w.x);
    A.x1 = swept ? P<double>(w.x1) : nullptr;
    A.box = nullptr;
    A.half = half;
    A.xb0 = P<float>(w.xb);
    A.xb1 = swept ? P<float>(w.xb1) : nullptr;
    A.boxf = swept ? P<float>(w.box1) : P<float>(w.box);
    A.halfu = half_up(half);
    A.l1 = P<int2>(w.l1);
    return A;
}

static L2cArgs cluster_args(abd_scene *s, const L2Args &a, bool swept) {
    L2cArgs C = {};
    C.a = a;
    C.vperm = P<int>(s->dev.vperm);
    C.tperm = P<int>(s->dev.tperm);
    C.eperm = P<int>(s->dev.eperm);
    C.slot_cbase = P<int>(s->w.slot_cbase);
    C.cl_info = P<int2>(s->w.cl_info);
    C.cbox = swept ? P<float>(s->w.cbox1) : P<float>(s->w.cbox);
    C.cp = P<int4>(s->w.cp);
    C.cap_cp = s->w.cap_cp;
    C.n_cp = &P<Counters>(s->w.ctr)->cp;
    return C;
}

// The two level-2 stages; counts stay on the device (grids sized for the
// capacities, kernels clamp to them).
static void launch_l2_stages(abd_scene *s, const L2cArgs &C, int64_t l1_cap) {
    cudaMemsetAsync(C.n_cp, 0, sizeof(unsigned long long), s->stream);
    ABD_LAUNCH(s, k_cpairs, grid_for(l1_cap, kL2Warps, 152 * 16), 32 * kL2Warps, 0, s->stream, C);
    ABD_LAUNCH(s, k_l2p, grid_for(C.cap_cp, kL2Warps, 152 * 16), 32 * kL2Warps, 0, s->stream, C);
}

// Read a device counter (synchronises the stream).
static int read_counter(abd_scene *s, unsigned long long *dptr, unsigned long long *h) {
    cudaError_t e = cudaMemcpyAsync(h, dptr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_check(s, e, "read counter");
}

// Level 1 within partitions (k_l1_part, or the spatial hash of abd_hash.cu
// when the world uses it) into w.l1, counting into Counters::l1.
static void launch_l1_part(abd_scene *s, bool swept) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    if (w.S_dyn == 0) return;
    if (w.use_hash) {
        launch_l1_hash(s, swept);
        return;
    }
    ABD_LAUNCH(s, k_l1_part, grid_for((int64_t)w.S_dyn * 32, 256), 256, 0, s->stream, w.S_dyn, w.S_all,
               P<int>(w.slot_part), P<int>(w.part_off), P<int>(w.static_grp),
               swept ? P<float>(w.box1) : P<float>(w.box), P<PartState>(w.part), P<int2>(w.l1), w.cap_l1, &c->l1);
}

int launch_l1(abd_scene *s, bool swept, int64_t *count) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    if (w.cap_l1 == 0) {
        w.cap_l1 = 4 * (int64_t)w.S_all + 1024;
        if (!dbuf_ensure(w.l1, 8 * w.cap_l1)) return set_err(s, ABD_E_OOM, "l1 list");
    }
    for (;;) {
        cudaMemsetAsync(&c->l1, 0, sizeof(unsigned long long), s->stream);
        launch_l1_part(s, swept);
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

int launch_l2(abd_scene *s, int mode, bool swept, double half, int64_t n_l1, int32_t *out3, int64_t cap,
              int64_t *count) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    L2Args A = l2_args(s, swept, half);
    A.n_l1 = n_l1;
    A.n_l1_dev = nullptr;
    A.mode = mode;
    A.out3 = out3;
    A.count = &c->cand;
    if (mode == 1 && w.cap_cand == 0) {
        w.cap_cand = 1 << 16;
        if (!dbuf_ensure(w.cand, sizeof(PairRec) * w.cap_cand)) return set_err(s, ABD_E_OOM, "candidate list");
    }
    if (w.cap_cp == 0) {
        w.cap_cp = 1 << 18;
        if (!dbuf_ensure(w.cp, sizeof(int4) * w.cap_cp)) return set_err(s, ABD_E_OOM, "cluster-pair list");
    }
    for (;;) {
        A.recs = P<PairRec>(w.cand);
        A.cap = mode == 1 ? w.cap_cand : cap;
        cudaMemsetAsync(&c->cand, 0, sizeof(unsigned long long), s->stream);
        cudaMemsetAsync(&c->cp, 0, sizeof(unsigned long long), s->stream);
        if (n_l1 > 0) launch_l2_stages(s, cluster_args(s, A, swept), n_l1);
        int rc = cuda_check(s, cudaGetLastError(), "k_l2");
        if (rc) return rc;
        unsigned long long n = 0, ncp = 0;
        if ((rc = read_counter(s, &c->cand, &n)) || (rc = read_counter(s, &c->cp, &ncp))) return rc;
        if ((int64_t)ncp > w.cap_cp) {
            w.cap_cp = (int64_t)ncp + ncp / 2 + 1024;
            if (!dbuf_ensure(w.cp, sizeof(int4) * w.cap_cp)) return set_err(s, ABD_E_OOM, "cluster-pair list");
            continue;
        }
        *count = (int64_t)n;
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
int launch_l1_async(abd_scene *s, bool swept, int cross) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    cudaMemsetAsync(&c->l1, 0, sizeof(unsigned long long), s->stream);
    if (cross && s->group.empty()) {
        // whole-scene check across slab partitions (replicas of different
        // bodies on different slabs); a batched world's scenes never meet,
        // so its partitions are checked one by one
        int64_t ntile = (w.S_all + 31) / 32;
        ABD_LAUNCH(s, k_l1f, grid_for((int64_t)w.S_all * ntile, 256), 256, 0, s->stream, w.S_all,
                   P<int>(w.slot_part), swept ? P<float>(w.box1) : P<float>(w.box), P<PartState>(w.part),
                   P<int2>(w.l1), w.cap_l1, &c->l1, P<int>(w.slot_body), cross);
    } else {
        launch_l1_part(s, swept);
    }
    return cuda_check(s, cudaGetLastError(), "k_l1");
}

int launch_l2_async(abd_scene *s, bool swept, double half) {
    World &w = s->w;
    Counters *c = P<Counters>(w.ctr);
    L2Args A = l2_args(s, swept, half);
    A.n_l1 = w.cap_l1;
    A.n_l1_dev = &c->l1;
    A.mode = 1;
    A.out3 = nullptr;
    A.recs = P<PairRec>(w.cand);
    A.cap = w.cap_cand;
    A.count = &c->cand;
    cudaMemsetAsync(&c->cand, 0, sizeof(unsigned long long), s->stream);
    cudaEvent_t ea, eb;
    // compulsory unique bytes: slot-vertex positions (one or two
    // configurations) and the triangle and edge indices of the slots' bodies
    // algorithmic bytes are added after the iteration's status read, from
    // the number of level-1 pairs the pass processed (l2_bytes_per_pair)
    prof_begin(s, swept ? "l2_swept" : "l2_static", 0.0, &ea, &eb);
    launch_l2_stages(s, cluster_args(s, A, swept), w.cap_l1);
    prof_end(s, ea, eb, prof_index(s, swept ? "l2_swept" : "l2_static"));
    return cuda_check(s, cudaGetLastError(), "k_l2");
}

}  // namespace abd

namespace abd {
// Algorithmic bytes of the level-2 pass per level-1 slot pair: both slots'
// vertex positions (one or two configurations) and their triangle and edge
// indices, each read once, at the world's mean slot size.
double l2_bytes_per_pair(const abd_scene *s, bool swept) {
    const World &w = s->w;
    if (w.S_all == 0) return 0.0;
    double tri_e = 0.0;
    for (int sl = 0; sl < w.S_all; ++sl) {
        int b = w.h_slot_body[sl];
        tri_e += 12.0 * s->nt[b] + 8.0 * s->ne[b];
    }
    return 2.0 * ((swept ? 48.0 : 24.0) * (double)w.SV + tri_e) / (double)w.S_all;
}
}  // namespace abd
