// abd_broad.cuh -- declarations of the broad-phase kernels (abd_broad.cu).
#pragma once
#include "abd_internal.h"

namespace abd {

struct L2Args {
    const int *slot_body;
    const int64_t *slot_voff;
    const int *voff, *nv, *toff, *nt, *eoff, *ne, *tri, *edge;
    const double *erest2;
    const double *x0, *x1, *box;
    double half;
    const float *xb0, *xb1;  // FP32 vertex bounds [SV][6] (lo, hi) of x0, x1
    const float *boxf;       // FP32 slot boxes (outward)
    float halfu;             // dhat / 2 rounded up to FP32
    const int2 *l1;
    int64_t n_l1;                          // used when n_l1_dev is null
    const unsigned long long *n_l1_dev;    // device count of level-1 pairs (clamped to n_l1)
    int mode;          // 0: (type, gid_i, gid_j) triples; 1: PairRec
    int32_t *out3;
    PairRec *recs;
    int64_t cap;
    unsigned long long *count;
};

constexpr int kL2Warps = 4;

// Level-2 pass over primitive clusters: the L2Args fields plus the cluster
// orders, the cluster table, the per-slot cluster boxes and the cluster-pair
// list that links its two stages.
struct L2cArgs {
    L2Args a;
    const int *vperm, *tperm, *eperm;
    const int *slot_cbase;
    const int2 *cl_info;     // [C] (slot, kind << 24 | cluster index within the kind)
    const float *cbox;       // [C][6] inflated FP32 cluster boxes (outward)
    int4 *cp;                // cluster pairs (c1, c2, level-1 pair, job)
    int64_t cap_cp;
    unsigned long long *n_cp;
};

__global__ void __launch_bounds__(32 * kL2Warps) k_cpairs(L2cArgs A);
__global__ void __launch_bounds__(32 * kL2Warps, 6) k_l2p(L2cArgs A);

__global__ void k_boxes(int S, const int64_t *__restrict__ slot_voff, const double *__restrict__ x0,
                        const double *__restrict__ x1, double half, double *__restrict__ box);
__global__ void k_l1(int S_all, const int *__restrict__ slot_part, const double *__restrict__ box,
                     const PartState *__restrict__ part, int2 *__restrict__ out, int64_t cap,
                     unsigned long long *__restrict__ count);
__global__ void __launch_bounds__(32 * kL2Warps) k_l2(L2Args A);

}  // namespace abd
