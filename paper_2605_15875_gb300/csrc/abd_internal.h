// abd_internal.h -- host/device data layout of the GB300 ABD-IPC library.
//
// Layout in HBM (all device arrays, FP64 unless noted):
//   per body (persistent):  q, v [B][12]; mass, vol, kappa [B]; S [B][9];
//                           xbar [V][3] (centred), tri [T][3], edge [E][2]
//                           (body-local vertex ids), erest2 [E].
//   per slot (one per (partition, dynamic body) replica, then one per static
//   collider, rebuilt every step):  q, qprev, qtil, z, u, dq, g [S][12];
//   rho, kw [S]; diag Hessian block [S][144] (T = assembly type).
//   per slot vertex: x, x1 [SV][3] (positions at q and at the swept end).
//   pair lists: level-1 slot pairs [L1][2], candidates / active / line-search
//   pair records (PairRec, 32 B), off-diagonal blocks [L1][144] (T).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/abd.h"

namespace abd {

constexpr int kMaxPlanes = 8;
// Partitions of one world: up to 64 slabs (membership masks are 64-bit), or
// up to kMaxParts groups of a batched world (independent scenes, one
// partition each).
constexpr int kMaxSlabs = 64;
constexpr int kMaxParts = 256;
// Layout of the PCG status words (w.pcg_sc, ints): iterations per partition,
// the overflow word, a flag set when some CTA read off-diagonal entries that
// did not fit in its shared memory, then the off-diagonal CSR entries of each
// partition (twice its off-diagonal blocks).
constexpr int kPcgOver = kMaxParts, kPcgUnstaged = kMaxParts + 1, kPcgNent = kMaxParts + 2;
constexpr int kPcgWords = 2 * kMaxParts + 2;
constexpr int kLS = 4;  // trial step sizes evaluated per line-search pass

struct Planes {
    int n;
    int axis[kMaxPlanes];
    double sign[kMaxPlanes], offset[kMaxPlanes];
};

// A PT or EE primitive pair between two slots.  v = slot-vertex ids (PT: point,
// t0, t1, t2; EE: a0, a1, b0, b1); l1 = index of its level-1 slot pair;
// flags bit 0 = edge-edge; eps = mollifier threshold (EE).
struct PairRec {
    int v[4];
    int l1;
    int flags;
    double eps;
};

// Growable device buffer.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
};
bool dbuf_ensure(DBuf &b, size_t bytes);  // keeps no contents
void dbuf_free(DBuf &b);

template <class X> inline X *P(const DBuf &b) { return (X *)b.p; }

// Persistent device copy of a scene.
struct SceneDev {
    int nb = 0;
    int64_t V = 0, T = 0, E = 0;
    DBuf q, v, mass, S, vol, kappa, kind, voff, nv, toff, nt, eoff, ne, xbar, tri, edge, erest2;
    // primitive clusters: per body, vertices / triangles / edges in a
    // rest-frame Morton order (body-local ids), chunked by 32
    DBuf vperm, tperm, eperm;
    DBuf cbody_off;  // [B + 1] first cluster of each body (vertices, triangles, edges)
    DBuf omega;      // [B][3] angular velocity of kinematic bodies
    DBuf crest;      // [clusters][6] FP32 rest-frame box of each cluster's vertices (centre, half extent)
};

constexpr int kClusterSize = 32;
// Partition size from which the automatic level 1 switches to the spatial hash.
constexpr int kHashMinSlots = 1024;
// Deepest adaptive time-step split a step may request (2^16 sub-steps).
constexpr int kMaxDtSplit = 16;
// Inertia weight of kinematic bodies (prescribed motion through their
// predicted state, see include/abd.h).
constexpr double kKinematicWeight = 1e6;

// Per-step workspace of the consensus solve.
struct World {
    int NP = 0, S_dyn = 0, S_all = 0, nsh = 0, R = 0;
    int64_t gen = 0;  // bumped whenever slot tables or list buffers change (captured graphs go stale)
    int64_t SV = 0;
    DBuf slot_body, slot_part, slot_voff, slot_mask, slot_rep, slot_kw, sv_slot;
    DBuf q, qprev, qtil, z, u, rho, dq, g;
    DBuf x, x1, dx, box, box1;  // box, box1: [S][6] FP32 slot boxes (outward)
    DBuf xb, xb1;               // [SV][6] FP32 bounds (rounded down, up) of x, x1
    DBuf rep_off, rep_slot, zb, rho0, rhob, rb, sb, body_rep, body_slot;
    DBuf l1, cand, act, ls, diag, off, offflag;
    DBuf pcg_sc;  // PCG iteration counts per partition and the overflow word
    DBuf part;   // per-partition scalars (PartState)
    DBuf ctr;    // counters
    DBuf aabb;   // body AABBs at the step start
    DBuf part_off;  // [NP + 1] dynamic-slot range of each partition
    DBuf nmoll;     // mollified edge-edge pairs: counts (assembled, listed), then their list
    DBuf rowcnt, rowoff, rowcur, ent;  // row CSR of the off-diagonal blocks
    DBuf slot_cbase;   // [S_all + 1] first cluster of each slot
    DBuf cl_info;      // [C] (slot, kind << 24 | cluster index)
    DBuf cbox, cbox1;  // [C][6] cluster boxes (static, swept)
    DBuf cp;           // [cap_cp] int4 cluster pairs of the level-2 pass
    DBuf static_grp;   // [S_all - S_dyn] partition a static slot serves (-1: every partition)
    DBuf pinv;         // [S_dyn][144] preconditioner blocks when a partition is too large to stage them
    // spatial-hash level 1 (abd_hash.cu): bucket counts, cursors, starts, block
    // sums (+ the cell-size word), slots sorted by bucket
    DBuf hash_cnt, hash_cur, hash_start, hash_bsum, hash_sorted;
    bool use_hash = false;  // level 1 through the spatial hash (else partition-local all pairs)
    int64_t C = 0;
    int64_t cap_l1 = 0, cap_cand = 0, cap_act = 0, cap_ls = 0, cap_cp = 0;
    int ecap_mult = 16;  // PCG neighbour-list capacity per owned slot
    // host mirrors
    std::vector<int> h_slot_body, h_slot_part;
    std::vector<int64_t> h_slot_voff;
    std::vector<uint64_t> h_slot_mask;
    std::vector<int> h_rep_off, h_rep_slot, h_body_rep, h_body_slot, h_part_off, h_slot_cbase;
};

// Per-partition scalars, device resident.
struct PartState {
    int active;        // local solve still running
    int newton_it;
    unsigned long long dqmax;   // ordered-double max |dq|
    unsigned long long toi;     // ordered-double min TOI
    double alpha;
    double E[kLS + 1];          // E(q) and E(q + alpha_j dq)
    double rz, rz_new, r0, rr, pap;
    int pcg_done, pcg_it;
    double kB;      // barrier stiffness of the partition (its scene's, in a batched world)
    double inv_hl;  // 1 / (h l), l the scale of the partition's scene (Eq. 8's normalisation)
};

struct Counters {
    unsigned long long l1, cand, act, ls, cp;
    unsigned long long rinf, sinf, dinf;  // ordered doubles
    unsigned long long mind;              // ordered double: minimum distance of the final-state check
    int overflow;
    int timeout;
    unsigned long long pcg_total;
    int pending;  // line-search passes still undecided
    int ls_live;  // some partition has trial steps to evaluate in this line-search pass
    int bad;      // a list outgrew its buffer in this iteration
};

struct KStat {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0, bytes = 0.0;
};

}  // namespace abd

// Captured steady-state Newton iteration (see iteration_graph).
struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t gen = -1;
    int kernels = 0;
    bool disabled = false;
    // profiling event pairs recorded as graph nodes: (kstat index, bytes, begin, end)
    struct Ev {
        int idx;
        double bytes;
        cudaEvent_t a, b;
    };
    std::vector<Ev> ev;
};

// Cluster-size autotuner of the PCG (abd_pcg.cu), one per block precision.
struct PcgTune {
    int key = -1;             // partition-size bucket the result belongs to
    int best = 0;             // chosen cluster size, 0 while tuning
    int ncand = 0, cand[4] = {0, 0, 0, 0};
    double sum[4] = {0, 0, 0, 0};  // ms per PCG iteration, summed over trials
    int cnt[4] = {0, 0, 0, 0};
    int next = 0;             // next candidate to try
    int pending = -1;         // candidate whose timed launch awaits the status read
    cudaEvent_t a = nullptr, b = nullptr;
};

struct abd_scene {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;  // second branch of an iteration's independent kernels
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // no side branch: the serving runtime's scenes, whose workers' streams
    // already keep the GPU busy side by side (forks there only add joins)
    bool no_side = false;
    std::string err;
    // host copy of constants
    int nb = 0;
    int64_t V = 0, T = 0, E = 0;
    std::vector<int> kind, voff, nv, toff, nt, eoff, ne;
    std::vector<double> mass, S, vol, kappa, com, xbar, erest2;
    std::vector<int> tri, edge;
    std::vector<int> vperm, tperm, eperm, cbody_off;
    std::vector<double> crest;
    abd::Planes planes{};
    double g[3] = {0, 0, 0};
    // batched world (abd_scene_create_batch): group of every body (its
    // scene), body offsets of the groups; empty for an ordinary scene
    std::vector<int> group;
    std::vector<int64_t> group_off;
    std::vector<int64_t> last_part_newton;  // Newton iterations per partition in the last step
    int bp_mode = 0;  // level 1: 0 hash when a partition has >= kHashMinSlots slots, 1 all pairs, 2 hash
    // partition
    int axis = 0, n_slabs = 1;
    std::vector<double> slab_planes;
    double alpha_w = 2.0, w_min = 0.0;
    // control-based load balancing (Sec. 5.2)
    double pd_kp = 0.0, pd_kd = 0.0, pd_smooth = 0.0;
    std::vector<double> pd_tau, pd_T;   // smoothed work and last imbalance per plane
    std::vector<double> last_planes;    // planes the last step used
    // device
    abd::SceneDev dev;
    abd::World w;
    // pinned host staging
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
    IterGraph ig;
    PcgTune pcg_tune[2];  // [0] FP32 blocks, [1] FP64 blocks
    int pcg_cs_last = 0;  // cluster size of the last PCG launch (captured or direct)
    // profiling
    bool prof = false;
    int64_t n_launches = 0;
    std::vector<abd::KStat> kstats;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
};

namespace abd {

// ---- launchers (abd_broad.cu) ----
int launch_transform(abd_scene *s, const double *q_slots, double *x, const double *qalt, int use_alt_shared);
// FP32 bounds of caller positions already in w.x (and w.x1 when swept).
int launch_vert_bounds(abd_scene *s, bool swept);
// FP32 slot boxes of w.xb (and w.xb1 when swept) and the matching cluster
// boxes: cmode -2 gathers the vertex bounds; otherwise they come from the slot
// DOFs w.q with the second configuration of k_transform's mode cmode (1: q +
// alt, 2: shared slots at alt).
int launch_boxes(abd_scene *s, bool swept, double half, int cmode, const double *alt);
// Level-1 slot pairs (synchronous, with capacity growth)
int launch_l1(abd_scene *s, bool swept, int64_t *count);
// Level-2 candidates over w.x (and w.x1): mode 0 writes triples to out3, mode
// 1 PairRecs to w.cand (synchronous, with capacity growth)
int launch_l2(abd_scene *s, int mode, bool swept, double half, int64_t n_l1, int32_t *out3, int64_t cap,
              int64_t *count);
int launch_l1_async(abd_scene *s, bool swept, int cross = 0);
double l2_bytes_per_pair(const abd_scene *s, bool swept);
// ---- (abd_hash.cu) ----
int hash_table_size(int S);
bool hash_ensure(abd_scene *s);
void launch_l1_hash(abd_scene *s, bool swept);
int launch_l2_async(abd_scene *s, bool swept, double half);
// ---- (abd_assemble.cu) ----
int launch_narrow_async(abd_scene *s, const PairRec *src, const unsigned long long *src_n, int64_t src_cap,
                        double dhat);
// barrier stiffness per partition from PartState::kB
int launch_assemble_async(abd_scene *s, int precision, const abd_step_params *p);
int launch_ccd_async(abd_scene *s, const abd_step_params *p, bool want_ls);
int launch_energy_async(abd_scene *s, const abd_step_params *p, const double *alphas_dev);
// minimum unsigned distance over w.cand at w.x and vertex-plane distances of
// dynamic slot vertices (negative plane distances count as 0) into Counters::mind
int launch_min_dist_async(abd_scene *s);
int launch_pcg_async(abd_scene *s, int precision, const abd_step_params *p);
// ---- (abd_solve.cu) ----

// profiling helpers (abd_scene.cu)
// The events go on stream `st` (nullptr: the scene's stream).
void prof_begin(abd_scene *s, const char *name, double bytes, cudaEvent_t *a, cudaEvent_t *b,
                cudaStream_t st = nullptr);
void prof_end(abd_scene *s, cudaEvent_t a, cudaEvent_t b, int idx, cudaStream_t st = nullptr);
void prof_flush(abd_scene *s);
void prof_add_bytes(abd_scene *s, const char *name, double bytes);
int prof_index(abd_scene *s, const char *name);
void prof_graph_replayed(abd_scene *s);
bool stream_capturing(abd_scene *s);
// Two independent branches of an iteration: fork_side returns the scene's
// side stream, made to wait for everything enqueued on the scene's stream so
// far (or the scene's stream itself when there is no side stream, e.g. on the
// legacy default stream); join_side makes the scene's stream wait for what
// was enqueued on the branch.  Works the same under graph capture, where the
// branch becomes a parallel path of the graph.  ensure_side creates the side
// stream and its events (outside any capture).
void ensure_side(abd_scene *s);
void scene_no_side(abd_scene *s);  // never fork this scene's iterations
cudaStream_t fork_side(abd_scene *s);
void join_side(abd_scene *s, cudaStream_t side);
// After the status read of a Newton iteration: account the timed PCG launch
// of the cluster-size autotuner (iterations = largest partition's count).
void pcg_tune_observe(abd_scene *s, int64_t iterations);
void prof_graph_release(abd_scene *s);

int set_err(abd_scene *s, int code, const std::string &msg);
int cuda_check(abd_scene *s, cudaError_t e, const char *what);

// Every kernel launch goes through this macro so the scene can report how
// many of the library's kernels a step launched.
#define ABD_LAUNCH(S, K, G, B, SM, ST, ...)      \
    do {                                         \
        K<<<G, B, SM, ST>>>(__VA_ARGS__);        \
        ++(S)->n_launches;                       \
    } while (0)

// First item of this thread's warp in a "spread" grid-stride loop: the warp
// slots are dealt out so that a short list puts one warp on each of many SMs
// (blocks 152 k .. 152 k + 151 are taken to sit on distinct SMs), then one on
// each further SM sub-partition of those SMs (warp w of a block runs on
// sub-partition w mod 4), before any sub-partition gets a second warp.  FP64
// work in particular is limited by each sub-partition's FP64 pipe, which takes
// a warp instruction at a time however few of its lanes are active.  Slot of
// warp w of block b (G blocks of W warps, F = 152 floor(G / 152)):
//   b < F:  152 W floor(b / 152) + 152 w + b mod 152;   else  F W + (G - F) w + b - F,
// a bijection onto [0, G W).  Loop as
//   for (int64_t wb = spread_base(); wb < n; wb += gridDim.x * blockDim.x)
// with item wb + lane; the trip count is warp-uniform.
#ifdef __CUDACC__
__device__ __forceinline__ int64_t spread_slot() {
    constexpr int64_t kSM = 152;
    const int64_t G = gridDim.x, W = blockDim.x >> 5, b = blockIdx.x, w = threadIdx.x >> 5;
    const int64_t F = G / kSM * kSM;
    return b < F ? (b / kSM) * (kSM * W) + w * kSM + b % kSM : F * W + (G - F) * w + (b - F);
}
__device__ __forceinline__ int64_t spread_base() { return spread_slot() * 32; }
#endif

inline int grid_for(int64_t n, int block, int maxb = 152 * 32) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > maxb) g = maxb;
    return (int)g;
}

}  // namespace abd
