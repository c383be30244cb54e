// abd_noalloc.cu -- broad-phase candidate query that allocates no device memory.
//
// abd_candidates() builds per-call work buffers with cudaMalloc.  Some callers
// cannot do that: code embedded in a host framework that owns the GPU's
// memory budget (a serving process or training job whose caching allocator
// has reserved the free memory, so a cudaMalloc from a plugin fails or
// bypasses the framework's accounting), and latency-critical loops that
// cannot afford the implicit device-wide synchronisation cudaMalloc and
// cudaFree may perform.  abd_candidates_noalloc() serves them: the caller
// passes device buffers for the input positions and the output triples, and
// every intermediate (slot tables, slot boxes, the level-1 pair list,
// counters) lives in one file-scope __device__ array of fixed size.
#include <cstring>
#include <mutex>

#include "abd_broad.cuh"

namespace {

using namespace abd;

// 32 MiB of scratch.  Every GPU on which this library's module is loaded holds
// it until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Fixed per-body tables take 64 B per body; the rest holds level-1 pairs.
constexpr int kNoAllocMaxBodies = 131072;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];  // device address of g_scratch, per device

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// One-time set-up per device (with that device current): the host-side name
// g_scratch is only a stand-in, so kernels get the address the runtime reports.
int scratch_address(abd_scene *s, int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return set_err(s, ABD_E_INVALID, "candidates_noalloc: device index too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_err(s, ABD_E_CUDA,
                           std::string("candidates_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ABD_OK;
}

// Slot tables for "every body is one slot of one partition" and the zeroed
// counters; the scratch keeps the previous call's contents, so everything the
// query reads is rewritten here.
__global__ void k_noalloc_tables(int nb, const int *__restrict__ kind, const int *__restrict__ voff,
                                 int *__restrict__ slot_body, int *__restrict__ slot_part,
                                 int64_t *__restrict__ slot_voff, PartState *__restrict__ part,
                                 unsigned long long *__restrict__ ctr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nb; i += gridDim.x * blockDim.x) {
        slot_voff[i] = voff[i];
        if (i == nb) continue;
        slot_body[i] = i;
        slot_part[i] = kind[i] != ABD_STATIC ? 0 : -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        PartState p = {};
        p.active = 1;
        *part = p;
        ctr[0] = 0;
        ctr[1] = 0;
    }
}

int read_count(abd_scene *s, const unsigned long long *d, unsigned long long *h) {
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(*h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_check(s, e, "candidates_noalloc");
}

}  // namespace

extern "C" int abd_candidates_noalloc(abd_scene *s, const double *x0, const double *x1, double dhat, int32_t *out,
                                      int64_t cap, int64_t *n_out) {
    if (!s || !x0 || !n_out || !(dhat > 0) || cap < 0 || (cap > 0 && !out)) return ABD_E_INVALID;
    if (s->nb > kNoAllocMaxBodies)
        return set_err(s, ABD_E_INVALID,
                       "candidates_noalloc: " + std::to_string(s->nb) + " bodies exceed the no-allocation limit of " +
                           std::to_string(kNoAllocMaxBodies));
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    void *base = nullptr;
    int rc = scratch_address(s, s->device, &base);
    if (rc) {
        if (prev != s->device) cudaSetDevice(prev);
        return rc;
    }
    int nb = s->nb;
    char *p = (char *)base;
    size_t off = 0;
    int *slot_body = (int *)(p + off); off = align256(off + 4 * (size_t)nb);
    int *slot_part = (int *)(p + off); off = align256(off + 4 * (size_t)nb);
    int64_t *slot_voff = (int64_t *)(p + off); off = align256(off + 8 * (size_t)(nb + 1));
    double *box = (double *)(p + off); off = align256(off + 48 * (size_t)nb);
    PartState *part = (PartState *)(p + off); off = align256(off + sizeof(PartState));
    unsigned long long *ctr = (unsigned long long *)(p + off); off = align256(off + 2 * sizeof(unsigned long long));
    int2 *l1 = (int2 *)(p + off);
    int64_t cap_l1 = (int64_t)((kScratchBytes - off) / sizeof(int2));

    ABD_LAUNCH(s, k_noalloc_tables, grid_for(nb + 1, 256), 256, 0, s->stream, nb, P<int>(s->dev.kind),
               P<int>(s->dev.voff), slot_body, slot_part, slot_voff, part, ctr);
    double half = 0.5 * dhat;
    ABD_LAUNCH(s, k_boxes, grid_for((int64_t)nb * 32, 256), 256, 0, s->stream, nb, slot_voff, x0, x1, half, box);
    int64_t ntile = (nb + 31) / 32;
    ABD_LAUNCH(s, k_l1, grid_for((int64_t)nb * ntile, 256), 256, 0, s->stream, nb, slot_part, box, part, l1, cap_l1,
               &ctr[0]);
    unsigned long long n_l1 = 0;
    if ((rc = cuda_check(s, cudaGetLastError(), "candidates_noalloc")) || (rc = read_count(s, &ctr[0], &n_l1))) {
        if (prev != s->device) cudaSetDevice(prev);
        return rc;
    }
    if ((int64_t)n_l1 > cap_l1) {
        if (prev != s->device) cudaSetDevice(prev);
        return set_err(s, ABD_E_PAIR_OVERFLOW,
                       "candidates_noalloc: " + std::to_string(n_l1) + " overlapping body pairs exceed the scratch limit of " +
                           std::to_string(cap_l1));
    }
    L2Args A = {};
    A.slot_body = slot_body;
    A.slot_voff = slot_voff;
    A.voff = P<int>(s->dev.voff); A.nv = P<int>(s->dev.nv); A.toff = P<int>(s->dev.toff); A.nt = P<int>(s->dev.nt);
    A.eoff = P<int>(s->dev.eoff); A.ne = P<int>(s->dev.ne); A.tri = P<int>(s->dev.tri); A.edge = P<int>(s->dev.edge);
    A.erest2 = P<double>(s->dev.erest2);
    A.x0 = x0; A.x1 = x1; A.box = box; A.half = half;
    A.l1 = l1; A.n_l1 = (int64_t)n_l1; A.n_l1_dev = nullptr;
    A.mode = 0; A.out3 = out; A.recs = nullptr; A.cap = cap; A.count = &ctr[1];
    if (n_l1 > 0)
        ABD_LAUNCH(s, k_l2, grid_for((int64_t)n_l1, kL2Warps, 152 * 16), 32 * kL2Warps, 0, s->stream, A);
    unsigned long long n = 0;
    if (!(rc = cuda_check(s, cudaGetLastError(), "candidates_noalloc"))) rc = read_count(s, &ctr[1], &n);
    if (!rc) *n_out = (int64_t)n;
    if (prev != s->device) cudaSetDevice(prev);
    return rc;
}
