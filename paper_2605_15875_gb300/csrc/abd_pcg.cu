// abd_pcg.cu -- block-Jacobi preconditioned CG on thread-block clusters.
//
// One cluster per partition solves H dq = -g of that partition's Newton step
// (Eq. 5).  The partition's slots are split evenly over the cluster's CTAs;
// each CTA keeps its rows of p, Ap, r, z, x in shared memory, reads the
// neighbours' p through distributed shared memory (DSMEM), and the three dot
// products of an iteration are reduced first inside the CTA, then across the
// cluster by reading every CTA's partial in rank order, so all CTAs take
// identical step sizes and the same termination decision.  Cluster barriers
// are hardware barriers; there is no spin-wait in this file.
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
    const void *diag, *pinv, *off;
    const int *rowoff;                   // [S_dyn + 1] row CSR of the off-diagonal blocks
    const int2 *ent;                     // (neighbour slot, block index | bit 31 = transposed)
    const double *g;
    double *x;
    double tol2;
    int max_it;
    int *iters;           // [NP] iterations used
};

// Dynamic shared memory of one CTA owning m slots: p, Ap, r, z (T), x
// (double) for 12 m rows, reduction words, then (as far as the budget goes)
// its diagonal and preconditioner blocks and, per off-diagonal entry of its
// rows, the neighbour id, the block (staged row-major in the orientation the
// row needs) and the neighbour's gathered p.
template <class T>
__host__ __device__ inline size_t pcg_base_bytes(int m) {
    size_t rows = 12 * (size_t)m;
    return rows * (4 * sizeof(T) + sizeof(double)) + 64 * sizeof(double) + 16 + 2 * 144 * sizeof(T) * (size_t)m;
}

__device__ __forceinline__ double block_sum(double v, double *scratch) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += scratch[i];
    return t;
}

// Sum of word `k` of every CTA's partials across the cluster: lane q of warp
// 0 reads CTA q's value through DSMEM, a fixed shuffle tree adds them (the
// same order in every CTA, so every CTA gets bit-identical sums), and the
// result is broadcast through local shared memory.  nk <= 3 words at a time.
__device__ __forceinline__ void cluster_sum(cg::cluster_group &cl, double *red, double *out, int k0, int nk, int CS) {
    if (threadIdx.x < 32) {
        int lane = threadIdx.x;
        for (int k = 0; k < nk; ++k) {
            double v = lane < CS ? cl.map_shared_rank(red, lane)[k0 + k] : 0.0;
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) out[k] = v;
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
    const int my0 = s0 + rank * m, my1 = min(s1, my0 + m), mine = max(0, my1 - my0);
    const T *diag = (const T *)A.diag, *pinv = (const T *)A.pinv, *off = (const T *)A.off;

    extern __shared__ __align__(16) unsigned char smem[];
    const int rows = 12 * m;
    T *p = (T *)smem, *Ap = p + rows, *r = Ap + rows, *z = r + rows;
    double *x = (double *)(((uintptr_t)(z + rows) + 15) & ~uintptr_t(15));
    double *red = x + rows;      // [8] partials
    double *scratch = red + 8;   // [<= 32] block reduction
    T *Ds = (T *)(scratch + 48); // [m][144] diagonal blocks
    T *Ps = Ds + 144 * m;        // [m][144] preconditioner blocks
    unsigned char *tail = (unsigned char *)(Ps + 144 * m);

    const bool active = A.part[part].active != 0 && n > 0;
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
    T *gp = Bs + 144 * (size_t)es;                                 // [es][12]
    for (int e = threadIdx.x; e < 144 * mine; e += blockDim.x) {
        Ds[e] = diag[144 * (int64_t)my0 + e];
        Ps[e] = pinv[144 * (int64_t)my0 + e];
    }
    for (int sl = 0; sl < mine; ++sl)
        for (int k = A.rowoff[my0 + sl] + threadIdx.x; k < A.rowoff[my0 + sl + 1]; k += blockDim.x) {
            int j = k - e0;
            if (j >= es) continue;
            enb[j] = A.ent[k].x;
        }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < 144 * (int64_t)es; e += blockDim.x) {
        int j = (int)(e / 144), q = (int)(e % 144), i = q / 12, c = q % 12;
        int2 en = A.ent[e0 + j];
        const T *B = off + 144 * (int64_t)(en.y & 0x7fffffff);
        Bs[e] = en.y < 0 ? B[12 * c + i] : B[12 * i + c];  // row i of the block as row slot sees it
    }
    // r = -g, x = 0, z = P r, p = z
    double rr0 = 0.0, rz_loc = 0.0;
    for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
        r[e] = T(-A.g[12 * (int64_t)my0 + e]);
        x[e] = 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
        int sl = e / 12, i = e % 12;
        const T *M = Ps + 144 * sl + 12 * i;
        T t = T(0);
        for (int j = 0; j < 12; ++j) t += M[j] * r[12 * sl + j];
        z[e] = t;
        p[e] = t;
        rr0 += (double)r[e] * (double)r[e];
        rz_loc += (double)r[e] * (double)t;
    }
    rr0 = block_sum(rr0, scratch);
    rz_loc = block_sum(rz_loc, scratch);
    double *tot = scratch + 40;  // cluster sums, local copy
    if (threadIdx.x == 0) { red[0] = rr0; red[1] = rz_loc; }
    cl.sync();
    cluster_sum(cl, red, tot, 0, 2, CS);
    double r0 = tot[0], rz = tot[1];
    int it = 0;
    bool done = !(r0 > 0.0);  // identical in every CTA of the cluster
    cl.sync();  // partials read before they are overwritten
    while (!done && it < A.max_it) {
        // gather the neighbours' p of the staged entries (local or DSMEM)
        for (int e = threadIdx.x; e < 12 * es; e += blockDim.x) {
            int j = e / 12, i = e % 12, nb = enb[j];
            int o = (nb - s0) / m, lo = (nb - s0) - o * m;
            const T *pn = (o == rank ? p : cl.map_shared_rank(p, o)) + 12 * lo;
            gp[e] = pn[i];
        }
        __syncthreads();
        // Ap = H p over my rows, p . Ap
        double pap = 0.0;
        for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
            int sl = e / 12, i = e % 12;
            const T *D = Ds + 144 * sl + 12 * i;
            T acc = T(0);
            for (int j = 0; j < 12; ++j) acc += D[j] * p[12 * sl + j];
            for (int k = A.rowoff[my0 + sl]; k < A.rowoff[my0 + sl + 1]; ++k) {
                int jj = k - e0;
                if (jj < es) {
                    const T *B = Bs + 144 * jj + 12 * i;
                    const T *pn = gp + 12 * jj;
                    for (int c = 0; c < 12; ++c) acc += B[c] * pn[c];
                } else {
                    int2 en = A.ent[k];
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
            pap += (double)p[e] * (double)acc;
        }
        pap = block_sum(pap, scratch);
        if (threadIdx.x == 0) red[2] = pap;
        cl.sync();
        cluster_sum(cl, red, tot, 2, 1, CS);
        double alpha = rz / tot[0];
        for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
            x[e] += alpha * (double)p[e];
            r[e] = T((double)r[e] - alpha * (double)Ap[e]);
        }
        __syncthreads();
        double rrl = 0.0, rzl = 0.0;
        for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) {
            int sl = e / 12, i = e % 12;
            const T *M = Ps + 144 * sl + 12 * i;
            T t = T(0);
            for (int j = 0; j < 12; ++j) t += M[j] * r[12 * sl + j];
            z[e] = t;
            rrl += (double)r[e] * (double)r[e];
            rzl += (double)r[e] * (double)t;
        }
        rrl = block_sum(rrl, scratch);
        rzl = block_sum(rzl, scratch);
        if (threadIdx.x == 0) { red[3] = rrl; red[4] = rzl; }
        cl.sync();
        cluster_sum(cl, red, tot, 3, 2, CS);
        double rrt = tot[0], rzn = tot[1];
        ++it;
        done = rrt <= A.tol2 * r0;
        if (!done) {
            double beta = rzn / rz;
            rz = rzn;
            for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) p[e] = T((double)z[e] + beta * (double)p[e]);
        }
        cl.sync();  // new p visible to the cluster; partials free for reuse
    }
    for (int e = threadIdx.x; e < 12 * mine; e += blockDim.x) A.x[12 * (int64_t)my0 + e] = x[e];
    if (rank == 0 && threadIdx.x == 0) A.iters[part] = it;
}

template <class T>
static int launch_T(abd_scene *s, const abd_step_params *p) {
    World &w = s->w;
    static int max_cluster = -1;
    static size_t max_smem = 0;
    if (max_cluster < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        max_smem = (size_t)optin;
        cudaFuncSetAttribute(k_pcg_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (cudaFuncSetAttribute(k_pcg_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)
            max_cluster = 16;
        else
            max_cluster = 8;
        cudaGetLastError();
    }
    int maxn = 0;
    for (int q = 0; q < w.NP; ++q) maxn = std::max(maxn, w.h_part_off[q + 1] - w.h_part_off[q]);
    // cluster size: up to 16 CTAs, about 16 owned slots each
    int CS = std::min(max_cluster, std::max(2, (maxn + 15) / 16));
    if (CS > 8 && max_cluster < 16) CS = 8;
    int m = std::max(1, (maxn + CS - 1) / CS);
    size_t base = pcg_base_bytes<T>(m);
    if (base > max_smem) return set_err(s, ABD_E_UNSUPPORTED, "pcg: partition too large for the cluster");
    size_t smem = std::max(base + 1024, std::min(max_smem, base + (size_t)m * 12 * (144 + 12 + 4) * sizeof(T)));
    PcgClArgs A = {};
    A.part_off = P<int>(w.part_off); A.part = P<PartState>(w.part);
    A.diag = w.diag.p; A.pinv = w.pinv.p; A.off = w.off.p;
    A.rowoff = P<int>(w.rowoff); A.ent = P<int2>(w.ent);
    A.g = P<double>(w.g); A.x = P<double>(w.dq);
    A.tol2 = p->pcg_rtol * p->pcg_rtol; A.max_it = p->pcg_max;
    A.iters = P<int>(w.pcg_sc);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(w.NP * CS);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaEvent_t ea, eb;
    prof_begin(s, "pcg", 0, &ea, &eb);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_pcg_cluster<T>, A, (int)smem);
    prof_end(s, ea, eb, prof_index(s, "pcg"));
    ++s->n_launches;
    return cuda_check(s, e, "pcg cluster launch");
}

// Iterations per partition land in w.pcg_sc ([kMaxParts] ints) for the
// caller's per-iteration status read.
int launch_pcg_async(abd_scene *s, int precision, const abd_step_params *p) {
    return precision == ABD_MIXED ? launch_T<float>(s, p) : launch_T<double>(s, p);
}

}  // namespace abd
