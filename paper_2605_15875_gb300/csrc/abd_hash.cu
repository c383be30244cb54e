// abd_hash.cu -- spatial-hash level 1 of the broad phase (slot pairs).
//
// Uniform grid with cell size c = 1.01 x the largest slot-box extent of the
// active partitions (computed on the device every launch, so a captured
// iteration keeps working as boxes change).  Every dynamic slot is entered
// in the cell of its box's lower corner, cell (partition, floor(lo / c)),
// hashed into a table of T = 2^k >= 2 S_dyn buckets by a counting sort
// (count, exclusive scan, scatter).  A slot whose box has extent <= c / 1.01
// can overlap slot a only if its lower corner lies in
// [a.lo - c / 1.01, a.hi], i.e. in cells floor(a.lo / c) - 1 .. floor(a.hi / c)
// along every axis (at most 3, the 1 % margin absorbing the rounding of the
// divisions), so one warp per slot a visits at most 27 cells, and a lane per
// bucket entry b keeps b when it is a later slot of a's partition whose home
// cell is the visited cell (a bucket may hold other cells' slots) and whose
// box overlaps a's; static colliders are tested as in k_l1_part.  Hits are
// compacted with warp ballots.  The pair set equals k_l1_part's; the work is
// about 27 x (slots per cell) per slot instead of the partition's size.
#include "abd_broad.cuh"

namespace abd {

namespace {

constexpr float kCellMargin = 1.01f;

__device__ __forceinline__ int cell_coord(float x, float c) {
    float f = floorf(x / c);
    return (int)fminf(fmaxf(f, -1.0e9f), 1.0e9f);
}

__device__ __forceinline__ unsigned hash_cell(int part, int ix, int iy, int iz) {
    unsigned h = (unsigned)part * 0x9E3779B1u;
    h ^= (unsigned)ix * 0x85EBCA77u + (h << 6) + (h >> 2);
    h ^= (unsigned)iy * 0xC2B2AE3Du + (h << 6) + (h >> 2);
    h ^= (unsigned)iz * 0x27D4EB2Fu + (h << 6) + (h >> 2);
    return h;
}

// Largest box extent over the dynamic slots of active partitions, as the bit
// pattern of a non-negative float (integer order = float order).
__global__ void k_hash_extent(int S_dyn, const int *__restrict__ slot_part, const float *__restrict__ box,
                              const PartState *__restrict__ part, int *__restrict__ ext_bits) {
    float m = 0.f;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < S_dyn; a += gridDim.x * blockDim.x) {
        if (!part[slot_part[a]].active) continue;
        const float *b = box + 6 * (int64_t)a;
        m = fmaxf(m, fmaxf(b[3] - b[0], fmaxf(b[4] - b[1], b[5] - b[2])));
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(ext_bits, __float_as_int(m));
}

__device__ __forceinline__ float cell_size(const int *ext_bits) {
    return __int_as_float(*ext_bits) * kCellMargin;
}

__global__ void k_hash_count(int S_dyn, const int *__restrict__ slot_part, const float *__restrict__ box,
                             const PartState *__restrict__ part, const int *__restrict__ ext_bits, unsigned mask,
                             int *__restrict__ cnt) {
    const float c = cell_size(ext_bits);
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < S_dyn; a += gridDim.x * blockDim.x) {
        const int p = slot_part[a];
        if (!part[p].active) continue;
        const float *b = box + 6 * (int64_t)a;
        unsigned key = hash_cell(p, cell_coord(b[0], c), cell_coord(b[1], c), cell_coord(b[2], c)) & mask;
        atomicAdd(&cnt[key], 1);
    }
}

// Exclusive scan of a block's 1024 counts (one per thread) into out; the
// block's total into bsum[blockIdx.x].
__device__ __forceinline__ int block_scan_excl(int v, int *warp_tot, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive prefix of the warp totals
    }
    __syncthreads();
    total = warp_tot[(blockDim.x >> 5) - 1];
    return x - v + (w > 0 ? warp_tot[w - 1] : 0);
}

__global__ void __launch_bounds__(1024) k_scan_blocks(int n, const int *__restrict__ cnt, int *__restrict__ start,
                                                      int *__restrict__ bsum) {
    __shared__ int wt[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int total = 0;
    int e = block_scan_excl(i < n ? cnt[i] : 0, wt, total);
    if (i < n) start[i] = e;
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(int nb, int *__restrict__ bsum) {
    __shared__ int wt[32];
    int total = 0;
    int v = (int)threadIdx.x < nb ? bsum[threadIdx.x] : 0;
    int e = block_scan_excl(v, wt, total);
    if ((int)threadIdx.x < nb) bsum[threadIdx.x] = e;
}

__global__ void k_scan_add(int n, int *__restrict__ start, const int *__restrict__ bsum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) start[i] += bsum[blockIdx.x];
}

__global__ void k_hash_scatter(int S_dyn, const int *__restrict__ slot_part, const float *__restrict__ box,
                               const PartState *__restrict__ part, const int *__restrict__ ext_bits, unsigned mask,
                               const int *__restrict__ start, int *__restrict__ cur, int *__restrict__ sorted) {
    const float c = cell_size(ext_bits);
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < S_dyn; a += gridDim.x * blockDim.x) {
        const int p = slot_part[a];
        if (!part[p].active) continue;
        const float *b = box + 6 * (int64_t)a;
        unsigned key = hash_cell(p, cell_coord(b[0], c), cell_coord(b[1], c), cell_coord(b[2], c)) & mask;
        sorted[start[key] + atomicAdd(&cur[key], 1)] = a;
    }
}

__device__ __forceinline__ bool overlap_f(const float *a, const float *b) {
    return !(a[0] > b[3] || b[0] > a[3] || a[1] > b[4] || b[1] > a[4] || a[2] > b[5] || b[2] > a[5]);
}

// Ballot-compacted append of (a, b) for the lanes with hit set.
__device__ __forceinline__ void emit_pair(bool hit, int a, int b, int2 *out, int64_t cap, unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (!m) return;
    unsigned long long pos = 0;
    int leader = __ffs(m) - 1;
    if (lane == leader) pos = atomicAdd(count, (unsigned long long)__popc(m));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (hit) {
        unsigned long long my = pos + __popc(m & ((1u << lane) - 1));
        if ((int64_t)my < cap) out[my] = make_int2(a, b);
    }
}

__global__ void k_l1_hash(int S_dyn, int S_all, const int *__restrict__ slot_part, const int *__restrict__ static_grp,
                          const float *__restrict__ box, const PartState *__restrict__ part,
                          const int *__restrict__ ext_bits, unsigned mask, const int *__restrict__ start,
                          const int *__restrict__ cnt, const int *__restrict__ sorted, int2 *__restrict__ out,
                          int64_t cap, unsigned long long *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int n_static = S_all - S_dyn;
    const float c = cell_size(ext_bits);
    for (int a = blockIdx.x + gridDim.x * (threadIdx.x >> 5); a < S_dyn; a += nw) {
        const int pa = slot_part[a];
        if (!part[pa].active) continue;  // warp-uniform
        float ba[6];
        for (int k = 0; k < 6; ++k) ba[k] = box[6 * (int64_t)a + k];
        int lo[3], hi[3];
        for (int k = 0; k < 3; ++k) {
            lo[k] = cell_coord(ba[k], c) - 1;
            hi[k] = cell_coord(ba[3 + k], c);
        }
        for (int ix = lo[0]; ix <= hi[0]; ++ix)
            for (int iy = lo[1]; iy <= hi[1]; ++iy)
                for (int iz = lo[2]; iz <= hi[2]; ++iz) {
                    const unsigned key = hash_cell(pa, ix, iy, iz) & mask;
                    const int s0 = start[key], n = cnt[key];
                    for (int j0 = 0; j0 < n; j0 += 32) {
                        bool hit = false;
                        int b = -1;
                        if (j0 + lane < n) {
                            b = sorted[s0 + j0 + lane];
                            if (b > a && slot_part[b] == pa) {
                                float bb[6];
                                for (int k = 0; k < 6; ++k) bb[k] = box[6 * (int64_t)b + k];
                                hit = cell_coord(bb[0], c) == ix && cell_coord(bb[1], c) == iy &&
                                      cell_coord(bb[2], c) == iz && overlap_f(ba, bb);
                            }
                        }
                        emit_pair(hit, a, b, out, cap, count);
                    }
                }
        for (int j0 = 0; j0 < n_static; j0 += 32) {
            const int j = j0 + lane;
            bool hit = false;
            int b = -1;
            if (j < n_static) {
                const int g = static_grp[j];
                if (g < 0 || g == pa) {
                    b = S_dyn + j;
                    float bb[6];
                    for (int k = 0; k < 6; ++k) bb[k] = box[6 * (int64_t)b + k];
                    hit = overlap_f(ba, bb);
                }
            }
            emit_pair(hit, a, b, out, cap, count);
        }
    }
}

}  // namespace

// Table size of the hash for S dynamic slots: the smallest power of two >= 2 S
// (at least 1024, at most 2^20; more slots share buckets).
int hash_table_size(int S) {
    int T = 1024;
    while (T < 2 * S && T < (1 << 20)) T <<= 1;
    return T;
}

bool hash_ensure(abd_scene *s) {
    World &w = s->w;
    const int T = hash_table_size(w.S_dyn);
    return dbuf_ensure(w.hash_cnt, 4 * (size_t)T) && dbuf_ensure(w.hash_cur, 4 * (size_t)T) &&
           dbuf_ensure(w.hash_start, 4 * (size_t)T) && dbuf_ensure(w.hash_bsum, 4 * 1024 + 64) &&
           dbuf_ensure(w.hash_sorted, 4 * (size_t)std::max(1, w.S_dyn));
}

// Level-1 pairs of the solver's lists through the hash (into w.l1, counting
// into Counters::l1, which the caller has zeroed).  Buffers from hash_ensure.
void launch_l1_hash(abd_scene *s, bool swept) {
    World &w = s->w;
    if (w.S_dyn == 0) return;
    Counters *c = P<Counters>(w.ctr);
    const int T = hash_table_size(w.S_dyn), nb = T / 1024;
    const unsigned mask = (unsigned)(T - 1);
    const float *box = swept ? P<float>(w.box1) : P<float>(w.box);
    int *ext = P<int>(w.hash_bsum) + 1024;  // one word after the block sums
    cudaMemsetAsync(P<int>(w.hash_cnt), 0, 4 * (size_t)T, s->stream);
    cudaMemsetAsync(P<int>(w.hash_cur), 0, 4 * (size_t)T, s->stream);
    cudaMemsetAsync(ext, 0, 4, s->stream);
    const int g = grid_for(w.S_dyn, 256);
    ABD_LAUNCH(s, k_hash_extent, g, 256, 0, s->stream, w.S_dyn, P<int>(w.slot_part), box, P<PartState>(w.part), ext);
    ABD_LAUNCH(s, k_hash_count, g, 256, 0, s->stream, w.S_dyn, P<int>(w.slot_part), box, P<PartState>(w.part), ext,
               mask, P<int>(w.hash_cnt));
    ABD_LAUNCH(s, k_scan_blocks, nb, 1024, 0, s->stream, T, P<int>(w.hash_cnt), P<int>(w.hash_start),
               P<int>(w.hash_bsum));
    ABD_LAUNCH(s, k_scan_top, 1, 1024, 0, s->stream, nb, P<int>(w.hash_bsum));
    ABD_LAUNCH(s, k_scan_add, nb, 1024, 0, s->stream, T, P<int>(w.hash_start), P<int>(w.hash_bsum));
    ABD_LAUNCH(s, k_hash_scatter, g, 256, 0, s->stream, w.S_dyn, P<int>(w.slot_part), box, P<PartState>(w.part), ext,
               mask, P<int>(w.hash_start), P<int>(w.hash_cur), P<int>(w.hash_sorted));
    ABD_LAUNCH(s, k_l1_hash, grid_for((int64_t)w.S_dyn * 32, 256), 256, 0, s->stream, w.S_dyn, w.S_all,
               P<int>(w.slot_part), P<int>(w.static_grp), box, P<PartState>(w.part), ext, mask,
               P<int>(w.hash_start), P<int>(w.hash_cnt), P<int>(w.hash_sorted), P<int2>(w.l1), w.cap_l1, &c->l1);
}

}  // namespace abd
