// abd_pcg.cu -- block-Jacobi preconditioned CG on thread-block clusters.
//
// One cluster per partition solves H dq = -g of that partition's Newton step
// (Eq. 5).  The partition's slots are split evenly over the cluster's CTAs;
// each CTA keeps its rows of p, Ap, r, z, x in shared memory together with
// its diagonal, preconditioner and off-diagonal blocks and a copy of the
// neighbours' p for its off-diagonal entries.  An iteration has two cluster
// barriers: after each dot product every CTA pushes its partial into every
// CTA's shared memory (DSMEM stores), the barrier publishes them, and each CTA
// adds the partials in rank order, so all CTAs take bit-identical step sizes
// and the same termination decision.  The neighbours' new p is rebuilt
// locally as z + beta p from their z, which the second barrier has already
// published, so no third barrier is needed (unless some entries did not fit
// in shared memory and are read from the owner's p directly).  Cluster
// barriers are hardware barriers; there is no spin-wait in this file.
//
// The block type T is also the type of every scalar and of x: the mixed path
// runs the whole solve in FP32 (FP64 instructions are scarce on this GPU and
// the Newton direction only needs the PCG tolerance); the FP64 path is FP64
// throughout.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "abd_internal.h"

namespace cg = cooperative_groups;

namespace abd {

struct PcgClArgs {
    const int *part_off;  // [NP + 1] dynamic-slot range of each partition
    const PartState *part;
    const void *diag, *off;
    const int *rowoff;                   // [S_dyn + 1] row CSR of the off-diagonal blocks
    const int2 *ent;                     // (neighbour slot, block index | bit 31 = transposed)
    const double *g;
    double *x;
    void *pinv;           // non-null: blocks stay in global memory, preconditioner blocks inverted here
                          // ([S_dyn][144]), for partitions whose blocks do not fit in shared memory
    double tol, tol2;
    int zrel;             // 1: stop on the preconditioned residual (see k_pcg_cluster), 0: on |r|_2
    int max_it;
    int *iters;           // PCG status words (kPcg* layout): iterations per partition, flags, entries
};

// Dynamic shared memory of one CTA owning m slots: p, Ap, r, z, x (all T)
// for 12 m rows, 64 partial words, 32 reduction words, m + 1 row
// offsets, its diagonal and preconditioner blocks (unless they stay in global
// memory: pcg_vec_bytes), then (as far as the budget goes) per off-diagonal
// entry of its rows the neighbour id, the block (staged row-major in the
// orientation the row needs) and the neighbour's p.
template <class T>
inline size_t pcg_vec_bytes(int m) {
    size_t rows = 12 * (size_t)m;
    return rows * 5 * sizeof(T) + 16 + 112 * sizeof(T) + 4 * ((size_t)m + 1) + 16;
}
template <class T>
inline size_t pcg_base_bytes(int m) {
    return pcg_vec_bytes<T>(m) + 2 * 144 * sizeof(T) * (size_t)m;
}

// Block-wide sums of two values (every thread gets both).  Callers separate
// consecutive calls by a barrier, which protects the scratch words.
template <class R>
__device__ __forceinline__ void block_sum2(R &a, R &b, R *scratch) {
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { scratch[2 * w] = a; scratch[2 * w + 1] = b; }
    __syncthreads();
    a = R(0);
    b = R(0);
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += scratch[2 * i]; b += scratch[2 * i + 1]; }
}

// Block-wide maximum of a non-negative value (every thread gets it), through
// words [16, 24) of the scratch (block_sum2 uses [0, 16) for 256 threads), so
// it may follow block_sum2 without a barrier in between.
template <class R>
__device__ __forceinline__ R block_max(R a, R *scratch) {
    for (int o = 16; o; o >>= 1) {
        R b = __shfl_xor_sync(0xffffffffu, a, o);
        a = b > a ? b : a;
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) scratch[16 + w] = a;
    __syncthreads();
    a = R(0);
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a = scratch[16 + i] > a ? scratch[16 + i] : a;
    return a;
}

// Thread q < CS stores this CTA's values v[0..nk) at words base + nk * rank + k
// of CTA q's partial array.
template <class R>
__device__ __forceinline__ void push_partials(cg::cluster_group &cl, R *red, int base, const R *v, int nk, int rank,
                                              int CS) {
    if ((int)threadIdx.x < CS) {
        R *dst = cl.map_shared_rank(red, (int)threadIdx.x) + base + nk * rank;
        for (int k = 0; k < nk; ++k) dst[k] = v[k];
    }
}

// Block-Jacobi preconditioner: invert the n 12x12 diagonal blocks in M (in
// place, shared memory) by Gauss-Jordan elimination without pivoting (the
// blocks are symmetric positive definite).  16 threads per block, each owning
// 9 entries; step k reads the old entries, then writes
//   M[k][k] = 1/p, M[k][j] = M[k][j]/p, M[i][k] = -M[i][k]/p,
//   M[i][j] -= M[i][k] M[k][j] / p      (p = M[k][k]).
// Every thread of the CTA takes part in each step (blockDim.x a multiple of 32).
template <class T>
__device__ void invert_blocks(T *M, int n) {
    const int grp = threadIdx.x >> 4, sub = threadIdx.x & 15, ngrp = blockDim.x >> 4;
    for (int b0 = 0; b0 < n; b0 += ngrp) {
        const int b = b0 + grp;
        const bool own = b < n;
        T *B = M + 144 * (int64_t)(own ? b : 0);
        for (int k = 0; k < 12; ++k) {
            T nv[9];
            if (own) {
                T ip = T(1) / B[13 * k];
                for (int t = 0; t < 9; ++t) {
                    int e = sub + 16 * t, i = e / 12, j = e % 12;
                    T mij = B[e], mik = B[12 * i + k], mkj = B[12 * k + j];
                    if (i == k && j == k) nv[t] = ip;
                    else if (i == k) nv[t] = mkj * ip;
                    else if (j == k) nv[t] = -mik * ip;
                    else nv[t] = mij - mik * (mkj * ip);
                }
            }
            __syncwarp();
            if (own)
                for (int t = 0; t < 9; ++t) B[sub + 16 * t] = nv[t];
            __syncwarp();
        }
    }
    __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(256) k_pcg_cluster(PcgClArgs A, int smem_bytes) {
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int part = blockIdx.x / CS;
    const int s0 = A.part_off[part], s1 = A.part_off[part + 1], n = s1 - s0;
    const int m = (n + CS - 1) / CS;
    const int my0 = min(s1, s0 + rank * m), my1 = min(s1, my0 + m), mine = my1 - my0;
    const T *diag = (const T *)A.diag, *off = (const T *)A.off;
    using R = T;  // scalars and x: FP32 in the mixed path, FP64 otherwise

    extern __shared__ __align__(16) unsigned char smem[];
    const int rows = 12 * m;
    T *p = (T *)smem, *Ap = p + rows, *r = Ap + rows, *z = r + rows;
    R *x = (R *)(((uintptr_t)(z + rows) + 15) & ~uintptr_t(15));
    R *red = x + rows;      // [80] partials: [0,16) p.Ap, [16,48) (r.r, r.z), [48,64) flags, [64,80) max |z|
    R *scratch = red + 80;  // [32] block reduction
    int *rofs = (int *)(scratch + 32);                                  // [m + 1] my entry ranges
    T *blk = (T *)(((uintptr_t)(rofs + m + 1) + 15) & ~uintptr_t(15));
    // diagonal and preconditioner blocks: staged in shared memory, or (a
    // partition too large for that) read from global memory, the
    // preconditioner inverted in A.pinv
    const bool gblk = A.pinv != nullptr;
    T *Ds = gblk ? nullptr : blk;                                      // [m][144] diagonal blocks
    const T *Dr = gblk ? diag + 144 * (int64_t)my0 : Ds;
    T *Ps = gblk ? (T *)A.pinv + 144 * (int64_t)my0 : blk + 144 * m;   // [m][144] preconditioner blocks
    unsigned char *tail = (unsigned char *)(gblk ? blk : blk + 2 * 144 * m);

    const bool active = A.part[part].active != 0 && n > 0;
    if (rank == 0 && threadIdx.x == 0) A.iters[kPcgNent + part] = active ? A.rowoff[s1] - A.rowoff[s0] : 0;
    if (!active) {
        for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) A.x[12 * (int64_t)my0 + e] = 0.0;
        if (rank == 0 && threadIdx.x == 0) A.iters[part] = 0;
        return;  // uniform over the cluster: every CTA reads the same flag
    }
    // entries of my rows; how many fit in shared memory with block and p
    const int e0 = A.rowoff[my0], ne = A.rowoff[my0 + mine] - e0;
    const size_t per_e = sizeof(int) + sizeof(T) * (144 + 12);
    const int left = max(0, smem_bytes - (int)(tail - smem) - 16);  // 16: alignment slack
    const int es = min(ne, (int)(left / per_e));  // staged entries
    int *enb = (int *)tail;                        // [es] neighbour slot
    T *Bs = (T *)(((uintptr_t)(enb + es) + 15) & ~uintptr_t(15));  // [es][144]
    T *gp = Bs + 144 * (size_t)es;                                 // [es][12] neighbours' p
    for (int e = threadIdx.x; e < 144 * mine; e += blockDim.x) {
        T v = diag[144 * (int64_t)my0 + e];
        if (!gblk) Ds[e] = v;
        Ps[e] = v;
    }
    for (int sl = threadIdx.x; sl <= mine; sl += blockDim.x) rofs[sl] = A.rowoff[my0 + sl] - e0;
    for (int j = threadIdx.x; j < es; j += blockDim.x) enb[j] = A.ent[e0 + j].x;
    for (int64_t e = threadIdx.x; e < 144 * (int64_t)es; e += blockDim.x) {
        int j = (int)(e / 144), q = (int)(e % 144), i = q / 12, c = q % 12;
        int2 en = A.ent[e0 + j];
        const T *B = off + 144 * (int64_t)(en.y & 0x7fffffff);
        Bs[e] = en.y < 0 ? B[12 * c + i] : B[12 * i + c];  // row i of the block as row slot sees it
    }
    __syncthreads();
    invert_blocks(Ps, mine);
    // r = -g, x = 0, z = P r, p = z
    for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
        r[e] = T(-A.g[12 * (int64_t)my0 + e]);
        x[e] = R(0);
    }
    __syncthreads();
    R rr0 = R(0), rz = R(0), zm = R(0);
    for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
        int sl = e / 12, i = e % 12;
        const T *M = Ps + 144 * sl + 12 * i;
        T t = T(0);
        for (int j = 0; j < 12; ++j) t += M[j] * r[12 * sl + j];
        z[e] = t;
        p[e] = t;
        rr0 += r[e] * r[e];
        rz += r[e] * t;
        zm = fabs(t) > zm ? R(fabs(t)) : zm;
    }
    block_sum2(rr0, rz, scratch);
    zm = block_max(zm, scratch);
    cl.sync();  // every CTA of the cluster has started before any DSMEM access
    {
        R v[2] = {rr0, rz}, f = es < ne ? R(1) : R(0);
        push_partials(cl, red, 16, v, 2, rank, CS);
        push_partials(cl, red, 48, &f, 1, rank, CS);
        push_partials(cl, red, 64, &zm, 1, rank, CS);
    }
    cl.sync();
    R r0 = R(0), unstaged = R(0), zm0 = R(0);
    rz = R(0);
    for (int q = 0; q < CS; ++q) {
        r0 += red[16 + 2 * q];
        rz += red[17 + 2 * q];
        unstaged += red[48 + q];
        zm0 = red[64 + q] > zm0 ? red[64 + q] : zm0;
    }
    const bool need_sync3 = unstaged > R(0);  // some CTA reads owners' p directly
    if (need_sync3 && rank == 0 && threadIdx.x == 0) A.iters[kPcgUnstaged] = 1;
    // neighbours' p (= z) of the staged entries
    for (int e = threadIdx.x; e < 12 * es; e += blockDim.x) {
        int j = e / 12, i = e % 12, nb = enb[j];
        int o = (nb - s0) / m, lo = (nb - s0) - o * m;
        gp[e] = (o == rank ? p : cl.map_shared_rank(p, o))[12 * lo + i];
    }
    __syncthreads();
    int it = 0;
    bool done = !(r0 > R(0));  // identical in every CTA of the cluster
    while (!done && it < A.max_it) {
        // Ap = H p over my rows, p . Ap
        R pap = R(0), unused = R(0);
        for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
            int sl = e / 12, i = e % 12;
            const T *D = Dr + 144 * sl + 12 * i;
            T acc = T(0);
            for (int j = 0; j < 12; ++j) acc += D[j] * p[12 * sl + j];
            for (int jj = rofs[sl]; jj < rofs[sl + 1]; ++jj) {
                if (jj < es) {
                    const T *B = Bs + 144 * jj + 12 * i;
                    const T *pn = gp + 12 * jj;
                    for (int c = 0; c < 12; ++c) acc += B[c] * pn[c];
                } else {
                    int2 en = A.ent[e0 + jj];
                    int nb = en.x, bi = en.y;
                    const T *B = off + 144 * (int64_t)(bi & 0x7fffffff);
                    int o = (nb - s0) / m, lo = (nb - s0) - o * m;
                    const T *pn = (o == rank ? p : cl.map_shared_rank(p, o)) + 12 * lo;
                    if (bi >= 0)
                        for (int c = 0; c < 12; ++c) acc += B[12 * i + c] * pn[c];
                    else
                        for (int c = 0; c < 12; ++c) acc += B[12 * c + i] * pn[c];
                }
            }
            Ap[e] = acc;
            pap += p[e] * acc;
        }
        block_sum2(pap, unused, scratch);
        push_partials(cl, red, 0, &pap, 1, rank, CS);
        cl.sync();
        R papt = R(0);
        for (int q = 0; q < CS; ++q) papt += red[q];
        R alpha = rz / papt;
        for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
            x[e] += alpha * p[e];
            r[e] = r[e] - alpha * Ap[e];
        }
        __syncthreads();
        R rrl = R(0), rzl = R(0), zml = R(0);
        for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
            int sl = e / 12, i = e % 12;
            const T *M = Ps + 144 * sl + 12 * i;
            T t = T(0);
            for (int j = 0; j < 12; ++j) t += M[j] * r[12 * sl + j];
            z[e] = t;
            rrl += r[e] * r[e];
            rzl += r[e] * t;
            zml = fabs(t) > zml ? R(fabs(t)) : zml;
        }
        block_sum2(rrl, rzl, scratch);
        zml = block_max(zml, scratch);
        {
            R v[2] = {rrl, rzl};
            push_partials(cl, red, 16, v, 2, rank, CS);
            push_partials(cl, red, 64, &zml, 1, rank, CS);
        }
        cl.sync();  // partials and every CTA's z published
        R rrt = R(0), rzn = R(0), zmt = R(0);
        for (int q = 0; q < CS; ++q) {
            rrt += red[16 + 2 * q];
            rzn += red[17 + 2 * q];
            zmt = red[64 + q] > zmt ? red[64 + q] : zmt;
        }
        ++it;
        // FP64: |r|_2 <= rtol |r0|_2.  Mixed: the block-Jacobi preconditioned
        // residual z = P r is in the units of q, body by body, so its largest
        // entry bounds how far each body's step is from the exact Newton step
        // (|r|_2 is dominated by the stiff orthogonality and barrier rows and
        // can stop while a body's nearly free rotation is still unresolved):
        // |z|_inf <= rtol |z0|_inf
        done = A.zrel ? zmt <= R(A.tol) * zm0 : rrt <= R(A.tol2) * r0;
        if (!done) {
            R beta = rzn / rz;
            rz = rzn;
            for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) p[e] = z[e] + beta * p[e];
            // the same update of the neighbours' copies, from their published z
            for (int e = threadIdx.x; e < 12 * es; e += blockDim.x) {
                int j = e / 12, i = e % 12, nb = enb[j];
                int o = (nb - s0) / m, lo = (nb - s0) - o * m;
                T zn = (o == rank ? z : cl.map_shared_rank(z, o))[12 * lo + i];
                gp[e] = zn + beta * gp[e];
            }
            if (need_sync3) cl.sync();  // owners' new p visible to direct readers
            else __syncthreads();
        }
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
    for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) A.x[12 * (int64_t)my0 + e] = (double)x[e];
    if (rank == 0 && threadIdx.x == 0) A.iters[part] = it;
}

template <class T>
static int launch_T(abd_scene *s, const abd_step_params *p) {
    World &w = s->w;
    // device limits and kernel attributes, set once (thread-safe static init)
    struct Limits {
        int max_cluster;
        size_t max_smem;
    };
    static const Limits lim = [] {
        Limits L;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        L.max_smem = (size_t)optin;
        cudaFuncSetAttribute(k_pcg_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        L.max_cluster =
            cudaFuncSetAttribute(k_pcg_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess
                ? 16
                : 8;
        cudaGetLastError();
        return L;
    }();
    const int max_cluster = lim.max_cluster;
    const size_t max_smem = lim.max_smem;
    int maxn = 0;
    for (int q = 0; q < w.NP; ++q) maxn = std::max(maxn, w.h_part_off[q + 1] - w.h_part_off[q]);
    // default cluster size: up to 16 CTAs, about 16 owned slots each
    int CS = std::min(max_cluster, std::max(2, (maxn + 15) / 16));
    if (CS > 8 && max_cluster < 16) CS = 8;
    // shared memory of a CTA for cluster size cs; the blocks stay in global
    // memory (gblk) when the largest partition's do not fit
    auto smem_for = [&](int cs, size_t &smem, bool &gblk) {
        int m = std::max(1, (maxn + cs - 1) / cs);
        size_t base = pcg_base_bytes<T>(m);
        gblk = base + 1024 > max_smem;
        if (gblk) base = pcg_vec_bytes<T>(m);
        smem = std::max(base + 1024, std::min(max_smem, base + (size_t)m * 12 * (144 + 12 + 4) * sizeof(T)));
        return base + 1024 <= max_smem;
    };
    auto config = [&](int cs, size_t smem, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at) {
        cfg = cudaLaunchConfig_t{};
        cfg.gridDim = dim3(w.NP * cs);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s->stream;
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    };
    // cluster-size autotuner: directly launched solves (not graph captures)
    // try each schedulable candidate twice, timed per PCG iteration; the
    // fastest is kept for this partition-size bucket and the iteration graph
    // is re-captured with it
    PcgTune &tu = s->pcg_tune[sizeof(T) == 8 ? 1 : 0];
    int key = 32 - __builtin_clz((unsigned)std::max(1, maxn));
    const bool cap = stream_capturing(s);  // no occupancy queries or timing inside a capture
    if (tu.key != key && !cap) {
        cudaEvent_t ea0 = tu.a, eb0 = tu.b;
        tu = PcgTune();
        tu.a = ea0;
        tu.b = eb0;
        tu.key = key;
        const int cands[4] = {CS, 4, 8, 16};
        for (int c : cands) {
            if (c < 2 || c > max_cluster || c > std::max(2, maxn)) continue;
            bool dup = false;
            for (int i = 0; i < tu.ncand; ++i) dup |= tu.cand[i] == c;
            size_t sm = 0;
            bool gb = false;
            if (dup || !smem_for(c, sm, gb)) continue;
            cudaLaunchConfig_t cf;
            cudaLaunchAttribute at[1];
            config(c, sm, cf, at);
            int nclu = 0;
            if (cudaOccupancyMaxActiveClusters(&nclu, k_pcg_cluster<T>, &cf) != cudaSuccess || nclu < 1) {
                cudaGetLastError();
                continue;
            }
            tu.cand[tu.ncand++] = c;
        }
        if (tu.ncand <= 1) tu.best = CS;
    }
    bool timed = false;
    if (tu.key != key) {
        // partition-size bucket not tuned yet (inside a capture): default size
    } else if (tu.best) {
        CS = tu.best;
    } else if (tu.pending < 0 && !cap) {
        tu.pending = tu.next % tu.ncand;
        CS = tu.cand[tu.pending];
        timed = true;
    }
    size_t smem = 0;
    bool gblk = false;
    if (!smem_for(CS, smem, gblk)) return set_err(s, ABD_E_UNSUPPORTED, "pcg: partition too large for the cluster");
    if (gblk && !dbuf_ensure(w.pinv, 144 * sizeof(T) * (size_t)std::max(1, w.S_dyn)))
        return set_err(s, ABD_E_OOM, "pcg preconditioner blocks");
    PcgClArgs A = {};
    A.part_off = P<int>(w.part_off); A.part = P<PartState>(w.part);
    A.diag = w.diag.p; A.off = w.off.p;
    A.rowoff = P<int>(w.rowoff); A.ent = P<int2>(w.ent);
    A.g = P<double>(w.g); A.x = P<double>(w.dq);
    A.pinv = gblk ? w.pinv.p : nullptr;
    A.tol = p->pcg_rtol; A.tol2 = p->pcg_rtol * p->pcg_rtol; A.max_it = p->pcg_max;
    A.zrel = sizeof(T) == 4;
    A.iters = P<int>(w.pcg_sc);
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    config(CS, smem, cfg, at);
    if (timed && !tu.a) {
        cudaEventCreate(&tu.a);
        cudaEventCreate(&tu.b);
    }
    s->pcg_cs_last = CS;
    cudaEvent_t ea, eb;
    prof_begin(s, "pcg", 0, &ea, &eb);
    if (timed) cudaEventRecord(tu.a, s->stream);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_pcg_cluster<T>, A, (int)smem);
    if (timed) cudaEventRecord(tu.b, s->stream);
    prof_end(s, ea, eb, prof_index(s, "pcg"));
    ++s->n_launches;
    return cuda_check(s, e, "pcg cluster launch");
}

void pcg_tune_observe(abd_scene *s, int64_t iterations) {
    for (PcgTune &tu : s->pcg_tune) {
        if (tu.pending < 0) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, tu.a, tu.b) == cudaSuccess && iterations > 0) {
            tu.sum[tu.pending] += ms / (double)iterations;
            tu.cnt[tu.pending] += 1;
            tu.next = tu.pending + 1;
        }
        cudaGetLastError();
        tu.pending = -1;
        bool done = tu.ncand > 0;
        for (int i = 0; i < tu.ncand; ++i) done &= tu.cnt[i] >= 2;
        if (done) {
            int bi = 0;
            for (int i = 1; i < tu.ncand; ++i)
                if (tu.sum[i] / tu.cnt[i] < tu.sum[bi] / tu.cnt[bi]) bi = i;
            tu.best = tu.cand[bi];
            ++s->w.gen;  // re-capture the iteration graph with the chosen size
        }
    }
}

// Iterations and CSR entries per partition land in w.pcg_sc (kPcg* layout)
// for the caller's per-iteration status read.
int launch_pcg_async(abd_scene *s, int precision, const abd_step_params *p) {
    return precision == ABD_MIXED ? launch_T<float>(s, p) : launch_T<double>(s, p);
}

}  // namespace abd
