// abd_solve.cu -- one time step of distributed ABD on one GPU.
//
// Host driver of Alg. 1 with every partition's local solve batched into the
// same launches: partition membership (Sec. 4), slot tables, projected Newton
// on Eq. 5 (block-Jacobi PCG, CCD-filtered backtracking), consensus (Eq. 6),
// dual update (Eq. 7), stopping metrics (Eq. 8-10), the CCD merge check
// (Sec. 4.2) and the rho adaptation (Sec. 4.3).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "abd_device.cuh"
#include "abd_internal.h"

namespace abd {

void prof_flush(abd_scene *s);

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

// One warp per body: AABB of its vertices at the persistent state q.
__global__ void k_body_aabb(int nb, const int *__restrict__ voff, const double *__restrict__ xbar,
                            const double *__restrict__ q, double *__restrict__ out) {
    int lane = threadIdx.x & 31;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += (gridDim.x * blockDim.x) >> 5) {
        const double *qb = q + 12 * (int64_t)b;
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int v = voff[b] + lane; v < voff[b + 1]; v += 32) {
            const double *xb = xbar + 3 * (int64_t)v;
            for (int k = 0; k < 3; ++k) {
                double x = qb[k] + (qb[3 + 3 * k] * xb[0] + qb[4 + 3 * k] * xb[1] + qb[5 + 3 * k] * xb[2]);
                lo[k] = fmin(lo[k], x);
                hi[k] = fmax(hi[k], x);
            }
        }
        for (int o = 16; o; o >>= 1)
            for (int k = 0; k < 3; ++k) {
                lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        if (lane < 3) out[6 * (int64_t)b + lane] = lo[lane];
        else if (lane < 6) out[6 * (int64_t)b + lane] = hi[lane - 3];
    }
}

__global__ void k_fill_sv_slot(int S, const int64_t *__restrict__ slot_voff, int *__restrict__ sv_slot) {
    for (int s = blockIdx.x; s < S; s += gridDim.x)
        for (int64_t v = slot_voff[s] + threadIdx.x; v < slot_voff[s + 1]; v += blockDim.x) sv_slot[v] = s;
}

// Prescribed pose of a kinematic body after h: p + h v_p, and A rotated by the
// angle |omega| h about the axis omega (Rodrigues' formula
// R = I + sin t K + (1 - cos t) K^2, K the cross-product matrix of the unit
// axis), A' = R A.
__device__ void kinematic_pose(const double *q, const double *v, const double *w, double h, double *out) {
    for (int k = 0; k < 3; ++k) out[k] = q[k] + h * v[k];
    double n = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]), R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (n > 0.0) {
        double u[3] = {w[0] / n, w[1] / n, w[2] / n}, t = n * h, sn = sin(t), c1 = 1.0 - cos(t);
        double K[9] = {0, -u[2], u[1], u[2], 0, -u[0], -u[1], u[0], 0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double k2 = 0.0;
                for (int l = 0; l < 3; ++l) k2 += K[3 * i + l] * K[3 * l + j];
                R[3 * i + j] += sn * K[3 * i + j] + c1 * k2;
            }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            out[3 + 3 * i + j] = R[3 * i] * q[3 + j] + R[3 * i + 1] * q[6 + j] + R[3 * i + 2] * q[9 + j];
}

// q^t, q~ (gravity only for dynamic bodies, Sec. 3; the prescribed pose for
// kinematic ones), z = q~, u = 0, rho = beta m per slot.
__global__ void k_slot_init(int S_all, int S_dyn, const int *__restrict__ slot_body, const int *__restrict__ slot_rep,
                            const double *__restrict__ qb, const double *__restrict__ vb, const double *__restrict__ mass,
                            const int *__restrict__ kind, const double *__restrict__ omega, double h, double gx,
                            double gy, double gz, double beta, double *__restrict__ q, double *__restrict__ qtil,
                            double *__restrict__ z, double *__restrict__ u, double *__restrict__ rho) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S_all; s += gridDim.x * blockDim.x) {
        int b = slot_body[s];
        for (int i = 0; i < 12; ++i) q[12 * (int64_t)s + i] = qb[12 * (int64_t)b + i];
        if (s >= S_dyn) continue;
        double t12[12];
        if (kind[b] == ABD_KINEMATIC) {
            kinematic_pose(qb + 12 * (int64_t)b, vb + 12 * (int64_t)b, omega + 3 * (int64_t)b, h, t12);
        } else {
            double gg[3] = {gx, gy, gz};
            for (int i = 0; i < 12; ++i) {
                t12[i] = qb[12 * (int64_t)b + i] + h * vb[12 * (int64_t)b + i];
                if (i < 3) t12[i] += h * h * gg[i];
            }
        }
        for (int i = 0; i < 12; ++i) {
            qtil[12 * (int64_t)s + i] = t12[i];
            z[12 * (int64_t)s + i] = t12[i];
            u[12 * (int64_t)s + i] = 0.0;
        }
        rho[s] = beta * mass[b];
    }
}

__global__ void k_shared_init(int nsh, const int *__restrict__ rep_off, const int *__restrict__ rep_slot,
                              const double *__restrict__ qtil, const double *__restrict__ rho, double *__restrict__ zb,
                              double *__restrict__ rho0, double *__restrict__ rhob) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nsh; j += gridDim.x * blockDim.x) {
        int s = rep_slot[rep_off[j]];
        for (int i = 0; i < 12; ++i) zb[12 * (int64_t)j + i] = qtil[12 * (int64_t)s + i];
        rho0[j] = rhob[j] = rho[s];
    }
}

// max |dq| per partition (ordered-double atomics).
__global__ void k_dqmax(int S_dyn, const int *__restrict__ slot_part, const double *__restrict__ dq,
                        PartState *__restrict__ part) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S_dyn; s += gridDim.x * blockDim.x) {
        int p = slot_part[s];
        if (!part[p].active) continue;
        double m = 0.0;
        for (int i = 0; i < 12; ++i) m = fmax(m, fabs(dq[12 * (int64_t)s + i]));
        atomicMax(&part[p].dqmax, ord(m));
    }
}

// Newton stopping test of every active partition, before its line search:
// |dq|_inf / (h l) < eps_N ends the local solve (l the scale of the
// partition's scene, PartState::inv_hl = 1 / (h l)).  Resets the
// per-iteration TOI and |dq| accumulators.
__global__ void k_newton_decide(int NP, PartState *part, double tol) {
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        if (part[p].active) {
            part[p].newton_it++;
            if (unord(part[p].dqmax) * part[p].inv_hl < tol) part[p].active = 0;
        }
        part[p].dqmax = 0ull;
        part[p].toi = ord(1.0);
    }
}

__global__ void k_ls_reset(int NP, int *nh0, int *decided) {
    for (int p = threadIdx.x; p < NP; p += blockDim.x) { nh0[p] = 0; decided[p] = 0; }
}

// Line search bookkeeping: trial steps alpha_j = toi 2^-(nh0 + j - 1);
// alphas[p][0] = -1 marks a partition with nothing left to evaluate.
__global__ void k_ls_alphas(int NP, PartState *part, const int *nh0, const int *decided, double *alphas,
                            int max_halv, int *live) {
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        for (int j = 0; j <= kLS; ++j) part[p].E[j] = 0.0;
        double toi = unord(part[p].toi);
        bool skip = !part[p].active || decided[p];
        alphas[(kLS + 1) * p] = skip ? -1.0 : 0.0;
        if (!skip) *live = 1;
        for (int j = 1; j <= kLS; ++j) {
            int nh = nh0[p] + j - 1;
            alphas[(kLS + 1) * p + j] = (!skip && nh <= max_halv) ? ldexp(toi < 1.0 ? toi : 1.0, -nh) : -1.0;
        }
    }
}

// Accept the first trial with E <= E(q); after max_halv halvings accept the
// last trial.  decided[p] = 1 when settled; nh0 advances otherwise.
__global__ void k_ls_select(int NP, PartState *part, int *nh0, int *decided, const double *alphas, int max_halv,
                            int *pending) {
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        if (!part[p].active || decided[p]) continue;
        double E0 = part[p].E[0];
        int pick = -1;
        for (int j = 1; j <= kLS; ++j) {
            if (alphas[(kLS + 1) * p + j] < 0.0) break;
            if (part[p].E[j] <= E0) { pick = j; break; }
            if (nh0[p] + j - 1 == max_halv) { pick = j; break; }
        }
        if (pick > 0) {
            part[p].alpha = alphas[(kLS + 1) * p + pick];
            decided[p] = 1;
        } else {
            nh0[p] += kLS;
            atomicAdd(pending, 1);
        }
    }
}

// Flag an iteration whose lists outgrew their buffers (its results are void).
// The swept lists contain the static ones, so their counts bound both passes.
__global__ void k_check_bad(Counters *c, int64_t cap_l1, int64_t cap_cand, int64_t cap_act, int64_t cap_ls,
                            int64_t cap_cp, const int *pcg_over) {
    c->bad = ((int64_t)c->l1 > cap_l1 || (int64_t)c->cand > cap_cand || (int64_t)c->act > cap_act ||
              (int64_t)c->ls > cap_ls || (int64_t)c->cp > cap_cp || *pcg_over)
                 ? 1
                 : c->bad;
}

// q += alpha dq for partitions whose line search just settled.
__global__ void k_update_q(int S_dyn, const int *__restrict__ slot_part, const PartState *__restrict__ part,
                           const int *__restrict__ decided, const Counters *__restrict__ c,
                           const double *__restrict__ dq, double *__restrict__ q) {
    if (c->bad) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 12 * (int64_t)S_dyn;
         e += (int64_t)gridDim.x * blockDim.x) {
        int p = slot_part[e / 12];
        if (!part[p].active || decided[p] != 1) continue;
        q[e] += part[p].alpha * dq[e];
    }
}

__global__ void k_mark_updated(int NP, int *decided, const Counters *c) {
    if (c->bad) return;
    for (int p = threadIdx.x; p < NP; p += blockDim.x)
        if (decided[p] == 1) decided[p] = 2;
}

// Consensus (Eq. 6), dual update (Eq. 7), per-body residuals (Eq. 9-10).
__global__ void k_consensus(int nsh, const int *__restrict__ rep_off, const int *__restrict__ rep_slot,
                            const double *__restrict__ q, double *__restrict__ u, const double *__restrict__ rho,
                            double *__restrict__ zb, double *__restrict__ rb, double *__restrict__ sb,
                            Counters *__restrict__ c) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nsh; j += gridDim.x * blockDim.x) {
        double num[12], den = 0.0;
        for (int i = 0; i < 12; ++i) num[i] = 0.0;
        for (int k = rep_off[j]; k < rep_off[j + 1]; ++k) {
            int s = rep_slot[k];
            for (int i = 0; i < 12; ++i) num[i] += rho[s] * (q[12 * (int64_t)s + i] + u[12 * (int64_t)s + i]);
            den += rho[s];
        }
        double sv = 0.0, rv = 0.0, zn[12];
        for (int i = 0; i < 12; ++i) {
            zn[i] = num[i] / den;
            sv = fmax(sv, fabs(zn[i] - zb[12 * (int64_t)j + i]));
            zb[12 * (int64_t)j + i] = zn[i];
        }
        for (int k = rep_off[j]; k < rep_off[j + 1]; ++k) {
            int s = rep_slot[k];
            for (int i = 0; i < 12; ++i) {
                double ri = q[12 * (int64_t)s + i] - zn[i];
                u[12 * (int64_t)s + i] += ri;
                rv = fmax(rv, fabs(ri));
            }
        }
        rb[j] = rv;
        sb[j] = sv;
        atomicMax(&c->rinf, ord(rv));
        atomicMax(&c->sinf, ord(sv));
    }
}

__global__ void k_delta(int S_dyn, const double *__restrict__ q, const double *__restrict__ qprev, Counters *c) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 12 * (int64_t)S_dyn;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicMax(&c->dinf, ord(fabs(q[e] - qprev[e])));
}

// Per-slot copy of z for the local solves and the merge-check targets.
__global__ void k_scatter_z(int S_dyn, const int *__restrict__ slot_rep, const double *__restrict__ zb,
                            double *__restrict__ z) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 12 * (int64_t)S_dyn;
         e += (int64_t)gridDim.x * blockDim.x) {
        int j = slot_rep[e / 12];
        if (j >= 0) z[e] = zb[12 * (int64_t)j + e % 12];
    }
}

// Residual-driven rho (Sec. 4.3) with clamp and scaled-dual rescale.
__global__ void k_rho_update(int nsh, const int *__restrict__ rep_off, const int *__restrict__ rep_slot,
                             const double *__restrict__ rb, const double *__restrict__ sb,
                             const double *__restrict__ rho0, double *__restrict__ rhob, double *__restrict__ rho,
                             double *__restrict__ u, double tau, double mu, double smin, double smax) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nsh; j += gridDim.x * blockDim.x) {
        double old = rhob[j], nw = old;
        if (rb[j] > mu * sb[j]) nw = old * tau;
        else if (sb[j] > mu * rb[j]) nw = old / tau;
        nw = fmin(fmax(nw, smin * rho0[j]), smax * rho0[j]);
        rhob[j] = nw;
        for (int k = rep_off[j]; k < rep_off[j + 1]; ++k) {
            int s = rep_slot[k];
            for (int i = 0; i < 12; ++i) u[12 * (int64_t)s + i] *= old / nw;
            rho[s] = nw;
        }
    }
}

// Merge (Alg. 1 end of frame) and velocity update.
__global__ void k_merge(int nb, const int *__restrict__ kind, const int *__restrict__ body_rep,
                        const int *__restrict__ body_slot, const double *__restrict__ zb, const double *__restrict__ q,
                        double h, double *__restrict__ qbody, double *__restrict__ vbody) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        if (kind[b] == ABD_STATIC || (body_rep[b] < 0 && body_slot[b] < 0)) continue;
        const double *src = body_rep[b] >= 0 ? zb + 12 * (int64_t)body_rep[b] : q + 12 * (int64_t)body_slot[b];
        for (int i = 0; i < 12; ++i) {
            double qn = src[i];
            vbody[12 * (int64_t)b + i] = (qn - qbody[12 * (int64_t)b + i]) / h;
            qbody[12 * (int64_t)b + i] = qn;
        }
    }
}

}  // namespace abd

using namespace abd;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

struct Ctx {
    abd_scene *s;
    const abd_step_params *p;
    double kB, l, half;          // the whole scene's (slab partitions) or the largest over scenes (batched)
    std::vector<double> kBp, lp;  // per partition: barrier stiffness and scene scale
    abd_step_stats *st;
    int precision;
    int it_prec = 0;  // precision of the blocks and PCG of the last enqueued iteration
    DBuf alphas, nh0, decided, pending;
    double t_coll = 0, t_solve = 0, t_sync = 0;
    std::vector<int64_t> part_newton;  // Newton iterations per partition over the step
};

double u2d(unsigned long long u) {
    double d;
    memcpy(&d, &u, sizeof d);
    return d;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <class X> int h2d(abd_scene *s, DBuf &b, const std::vector<X> &v) {
    if (!dbuf_ensure(b, sizeof(X) * (v.size() ? v.size() : 1))) return set_err(s, ABD_E_OOM, "upload");
    if (v.empty()) return ABD_OK;
    return cuda_check(s, cudaMemcpyAsync(b.p, v.data(), sizeof(X) * v.size(), cudaMemcpyHostToDevice, s->stream),
                      "upload");
}

int sync(abd_scene *s) { return cuda_check(s, cudaStreamSynchronize(s->stream), "sync"); }

// Body AABBs at the persistent state (device) -> host.
int body_aabbs(abd_scene *s, std::vector<double> &box) {
    DBuf &tmp = s->w.aabb;
    if (!dbuf_ensure(tmp, 48 * (size_t)s->nb)) return set_err(s, ABD_E_OOM, "aabb");
    ABD_LAUNCH(s, k_body_aabb, grid_for((int64_t)s->nb * 32, 256), 256, 0, s->stream, s->nb, P<int>(s->dev.voff),
                                                                          P<double>(s->dev.xbar),
                                                                          P<double>(s->dev.q), P<double>(tmp));
    box.resize(6 * (size_t)s->nb);
    int rc = cuda_check(s, cudaMemcpyAsync(box.data(), tmp.p, 48 * (size_t)s->nb, cudaMemcpyDeviceToHost, s->stream),
                        "aabb");
    return rc ? rc : sync(s);
}

// Slab membership (Sec. 4): w = max(alpha v_max h, w_min); body b on slab i iff
// its AABB along the axis meets [gamma_i - w/2, gamma_{i+1} + w/2].
int compute_masks(abd_scene *s, double h, const std::vector<double> &box, const std::vector<double> &v,
                  std::vector<uint64_t> &mask, double &w_out) {
    int N = s->n_slabs, ax = s->axis;
    mask.assign(s->nb, 0);
    if (N <= 1) {
        for (int b = 0; b < s->nb; ++b) mask[b] = s->kind[b] != ABD_STATIC ? 1 : 0;
        w_out = 0.0;
        return ABD_OK;
    }
    double Lo = INFINITY, Hi = -INFINITY, vmax = 0.0, wmin = INFINITY;
    for (int b = 0; b < s->nb; ++b) {
        if (s->kind[b] == ABD_STATIC) continue;
        const double *bx = &box[6 * (size_t)b];
        Lo = std::min(Lo, bx[ax]);
        Hi = std::max(Hi, bx[3 + ax]);
        double dx = bx[3] - bx[0], dy = bx[4] - bx[1], dz = bx[5] - bx[2];
        wmin = std::min(wmin, std::sqrt(dx * dx + dy * dy + dz * dz));
        const double *vb = &v[12 * (size_t)b];
        vmax = std::max(vmax, std::sqrt(vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]));
    }
    std::vector<double> gam(N + 1);
    for (int i = 1; i < N; ++i)
        gam[i] = s->slab_planes.size() == (size_t)(N - 1) ? s->slab_planes[i - 1] : Lo + (Hi - Lo) * (double)i / (double)N;
    s->last_planes.assign(gam.begin() + 1, gam.begin() + N);
    if (s->w_min > 0.0) wmin = s->w_min;
    double w = std::max(s->alpha_w * vmax * h, wmin);
    for (int b = 0; b < s->nb; ++b) {
        if (s->kind[b] == ABD_STATIC) continue;
        double lo = box[6 * (size_t)b + ax], hi = box[6 * (size_t)b + 3 + ax];
        for (int i = 0; i < N; ++i) {
            double rlo = i == 0 ? -INFINITY : gam[i] - 0.5 * w;
            double rhi = i == N - 1 ? INFINITY : gam[i + 1] + 0.5 * w;
            if (lo <= rhi && hi >= rlo) mask[b] |= (uint64_t)1 << i;
        }
    }
    w_out = w;
    return ABD_OK;
}

// Build the slot tables of one step from the body masks (nparts partitions).
// In a batched world (s->group non-empty) partition p holds the dynamic and
// kinematic bodies of scene p (masks then have one bit), and a static body
// serves only its own scene's partition.
int build_world(abd_scene *s, const std::vector<uint64_t> &mask, int nparts) {
    const bool batched = !s->group.empty() && nparts > 1;
    ++s->w.gen;
    World &w = s->w;
    w.NP = nparts;
    w.h_slot_body.clear(); w.h_slot_part.clear(); w.h_slot_mask.clear();
    std::vector<int> slot_rep;
    std::vector<double> slot_kw;
    w.h_body_rep.assign(s->nb, -1);
    w.h_body_slot.assign(s->nb, -1);
    int nsh = 0;
    for (int b = 0; b < s->nb; ++b)
        if (s->kind[b] != ABD_STATIC && __builtin_popcountll(mask[b]) >= 2) w.h_body_rep[b] = nsh++;
    std::vector<std::vector<int>> reps(nsh);
    for (int p = 0; p < nparts; ++p)
        for (int b = 0; b < s->nb; ++b) {
            if (s->kind[b] == ABD_STATIC || !(batched ? s->group[b] == p && mask[b] : (mask[b] >> p) & 1)) continue;
            int sl = (int)w.h_slot_body.size();
            w.h_slot_body.push_back(b);
            w.h_slot_part.push_back(p);
            w.h_slot_mask.push_back(mask[b]);
            slot_rep.push_back(w.h_body_rep[b]);
            slot_kw.push_back(1.0 / (double)__builtin_popcountll(mask[b]));
            if (w.h_body_slot[b] < 0) w.h_body_slot[b] = sl;
            if (w.h_body_rep[b] >= 0) reps[w.h_body_rep[b]].push_back(sl);
        }
    w.S_dyn = (int)w.h_slot_body.size();
    w.h_part_off.assign(nparts + 1, 0);
    for (int i = 0; i < w.S_dyn; ++i) w.h_part_off[w.h_slot_part[i] + 1]++;
    int maxn = 0;
    for (int p = 0; p < nparts; ++p) maxn = std::max(maxn, w.h_part_off[p + 1]);
    for (int p = 0; p < nparts; ++p) w.h_part_off[p + 1] += w.h_part_off[p];
    // level 1 through the spatial hash for large partitions (or as asked)
    w.use_hash = s->bp_mode == 2 || (s->bp_mode == 0 && maxn >= kHashMinSlots);
    std::vector<int> static_grp;
    for (int b = 0; b < s->nb; ++b)
        if (s->kind[b] == ABD_STATIC) {
            w.h_slot_body.push_back(b);
            w.h_slot_part.push_back(-1);
            w.h_slot_mask.push_back(0);
            static_grp.push_back(batched ? s->group[b] : -1);
        }
    w.S_all = (int)w.h_slot_body.size();
    w.h_slot_voff.assign(w.S_all + 1, 0);
    for (int i = 0; i < w.S_all; ++i) w.h_slot_voff[i + 1] = w.h_slot_voff[i] + s->nv[w.h_slot_body[i]];
    // primitive clusters of every slot: vertices, then triangles, then edges
    auto ncl = [](int n) { return (n + kClusterSize - 1) / kClusterSize; };
    w.h_slot_cbase.assign(w.S_all + 1, 0);
    std::vector<int2> cl_info;
    for (int i = 0; i < w.S_all; ++i) {
        int b = w.h_slot_body[i];
        int nc[3] = {ncl(s->nv[b]), ncl(s->nt[b]), ncl(s->ne[b])};
        w.h_slot_cbase[i + 1] = w.h_slot_cbase[i] + nc[0] + nc[1] + nc[2];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < nc[k]; ++j) cl_info.push_back(make_int2(i, (k << 24) | j));
    }
    w.C = (int64_t)cl_info.size();
    w.SV = w.h_slot_voff[w.S_all];
    w.nsh = nsh;
    w.h_rep_off.assign(nsh + 1, 0);
    w.h_rep_slot.clear();
    for (int j = 0; j < nsh; ++j) {
        w.h_rep_off[j + 1] = w.h_rep_off[j] + (int)reps[j].size();
        for (int sl : reps[j]) w.h_rep_slot.push_back(sl);
    }
    w.R = (int)w.h_rep_slot.size();
    int rc;
    if ((rc = h2d(s, w.slot_body, w.h_slot_body)) || (rc = h2d(s, w.slot_part, w.h_slot_part)) ||
        (rc = h2d(s, w.slot_voff, w.h_slot_voff)) || (rc = h2d(s, w.slot_mask, w.h_slot_mask)) ||
        (rc = h2d(s, w.slot_rep, slot_rep)) || (rc = h2d(s, w.slot_kw, slot_kw)) ||
        (rc = h2d(s, w.rep_off, w.h_rep_off)) || (rc = h2d(s, w.rep_slot, w.h_rep_slot)) ||
        (rc = h2d(s, w.body_rep, w.h_body_rep)) || (rc = h2d(s, w.body_slot, w.h_body_slot)) ||
        (rc = h2d(s, w.part_off, w.h_part_off)) || (rc = h2d(s, w.slot_cbase, w.h_slot_cbase)) ||
        (rc = h2d(s, w.cl_info, cl_info)) || (rc = h2d(s, w.static_grp, static_grp)))
        return rc;
    size_t S = (size_t)(w.S_all ? w.S_all : 1), Sd = (size_t)(w.S_dyn ? w.S_dyn : 1);
    size_t SV = (size_t)(w.SV ? w.SV : 1), NS = (size_t)(nsh ? nsh : 1);
    bool ok = dbuf_ensure(w.sv_slot, 4 * SV) && dbuf_ensure(w.q, 96 * S) && dbuf_ensure(w.qprev, 96 * Sd) &&
              dbuf_ensure(w.qtil, 96 * Sd) && dbuf_ensure(w.z, 96 * Sd) && dbuf_ensure(w.u, 96 * Sd) &&
              dbuf_ensure(w.rho, 8 * Sd) && dbuf_ensure(w.dq, 96 * Sd) && dbuf_ensure(w.g, 96 * Sd) &&
              dbuf_ensure(w.x, 24 * SV) && dbuf_ensure(w.x1, 24 * SV) && dbuf_ensure(w.box, 48 * S) &&
              dbuf_ensure(w.xb, 24 * SV) && dbuf_ensure(w.xb1, 24 * SV) &&
              dbuf_ensure(w.box1, 48 * S) && dbuf_ensure(w.zb, 96 * NS) && dbuf_ensure(w.rho0, 8 * NS) &&
              dbuf_ensure(w.rhob, 8 * NS) && dbuf_ensure(w.rb, 8 * NS) && dbuf_ensure(w.sb, 8 * NS) &&
              dbuf_ensure(w.part, sizeof(PartState) * kMaxParts) && dbuf_ensure(w.ctr, sizeof(Counters)) &&
              dbuf_ensure(w.cbox, 48 * (size_t)(w.C ? w.C : 1)) && dbuf_ensure(w.cbox1, 48 * (size_t)(w.C ? w.C : 1));
    if (!ok) return set_err(s, ABD_E_OOM, "world buffers");
    if (w.use_hash && !hash_ensure(s)) return set_err(s, ABD_E_OOM, "spatial hash");
    if (w.S_all > 0) ABD_LAUNCH(s, k_fill_sv_slot, std::min(w.S_all, 152 * 8), 256, 0, s->stream, w.S_all, P<int64_t>(w.slot_voff), P<int>(w.sv_slot));
    return cuda_check(s, cudaGetLastError(), "build world");
}

int read_parts(abd_scene *s, std::vector<PartState> &ps) {
    ps.resize(s->w.NP);
    int rc = cuda_check(s, cudaMemcpyAsync(ps.data(), s->w.part.p, sizeof(PartState) * s->w.NP,
                                           cudaMemcpyDeviceToHost, s->stream), "read parts");
    return rc ? rc : sync(s);
}

int write_parts(abd_scene *s, const std::vector<PartState> &ps) {
    return cuda_check(s, cudaMemcpyAsync(s->w.part.p, ps.data(), sizeof(PartState) * s->w.NP, cudaMemcpyHostToDevice,
                                         s->stream), "write parts");
}


// Pinned host mirror of the per-iteration status: counters, per-partition
// state, PCG iterations and flags.
struct Status {
    Counters c;
    int pcg_iters[kMaxParts];
    int pcg_over, pcg_unstaged;
    int pcg_nent[kMaxParts];  // off-diagonal CSR entries of each partition
    int csr_total;  // entries of the off-diagonal row CSR (twice the blocks)
    unsigned long long n_moll;  // mollified edge-edge pairs assembled by the warp kernel
    PartState part[kMaxParts];
};

Status *pinned_status(abd_scene *s) {
    if (!s->pinned) {
        if (cudaHostAlloc(&s->pinned, sizeof(Status), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            s->pinned = nullptr;
            return nullptr;
        }
        s->pinned_bytes = sizeof(Status);
    }
    return (Status *)s->pinned;
}

int enqueue_status(abd_scene *s, Status *h) {
    World &w = s->w;
    cudaMemcpyAsync(&h->c, w.ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream);
    cudaMemcpyAsync(h->pcg_iters, w.pcg_sc.p, sizeof(int) * kPcgWords, cudaMemcpyDeviceToHost, s->stream);
    cudaMemcpyAsync(h->part, w.part.p, sizeof(PartState) * w.NP, cudaMemcpyDeviceToHost, s->stream);
    if (s->prof && w.S_dyn > 0) {
        cudaMemcpyAsync(&h->csr_total, P<int>(w.rowoff) + w.S_dyn, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
        cudaMemcpyAsync(&h->n_moll, w.nmoll.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream);
    }
    return cuda_check(s, cudaGetLastError(), "status");
}

// Capacities of the pair lists and the buffers that depend on them.
int ensure_lists(Ctx &C) {
    abd_scene *s = C.s;
    World &w = s->w;
    if (w.cap_l1 == 0) w.cap_l1 = 8 * (int64_t)w.S_all + 4096;
    if (w.cap_cand == 0) w.cap_cand = 1 << 16;
    if (w.cap_act == 0) w.cap_act = 1 << 15;
    if (w.cap_ls == 0) w.cap_ls = 1 << 16;
    if (w.cap_cp == 0) w.cap_cp = 1 << 18;
    // block storage: FP32 in the mixed path, unless its first Newton
    // iterations assemble FP64 blocks into the same buffers
    size_t tb = C.precision == ABD_MIXED && !C.p->mixed_fp64_first ? 4 : 8;
    bool ok = dbuf_ensure(w.l1, 8 * (size_t)w.cap_l1) && dbuf_ensure(w.cand, sizeof(PairRec) * (size_t)w.cap_cand) &&
              dbuf_ensure(w.act, sizeof(PairRec) * (size_t)w.cap_act) &&
              dbuf_ensure(w.ls, sizeof(PairRec) * (size_t)w.cap_ls) && dbuf_ensure(w.cp, sizeof(int4) * (size_t)w.cap_cp) &&
              dbuf_ensure(w.off, tb * 144 * (size_t)w.cap_l1) && dbuf_ensure(w.offflag, 4 * (size_t)w.cap_l1) &&
              dbuf_ensure(w.nmoll, 64 + 8 * (size_t)w.cap_act) &&
              dbuf_ensure(w.rowcnt, 4 * (size_t)(w.S_dyn + 2)) && dbuf_ensure(w.rowoff, 4 * (size_t)(w.S_dyn + 2)) &&
              dbuf_ensure(w.rowcur, 4 * (size_t)(w.S_dyn + 2)) && dbuf_ensure(w.ent, 16 * (size_t)w.cap_l1) &&
              dbuf_ensure(w.diag, tb * 144 * (size_t)(w.S_dyn ? w.S_dyn : 1)) &&
              dbuf_ensure(w.pcg_sc, 4 * (size_t)kPcgWords) && dbuf_ensure(C.alphas, 8 * (kLS + 1) * kMaxParts) &&
              dbuf_ensure(C.nh0, 4 * kMaxParts) && dbuf_ensure(C.decided, 4 * kMaxParts);
    return ok ? ABD_OK : set_err(s, ABD_E_OOM, "pair lists");
}

// Grow every list whose count exceeded its capacity (counts from the status).
void grow_lists(World &w, const Counters &c, bool pcg_over) {
    auto g = [](int64_t &cap, unsigned long long n) {
        if ((int64_t)n > cap) cap = (int64_t)n + (int64_t)n / 2 + 1024;
    };
    g(w.cap_l1, c.l1); g(w.cap_cand, c.cand); g(w.cap_act, c.act); g(w.cap_ls, c.ls); g(w.cap_cp, c.cp);
    if (pcg_over) w.ecap_mult *= 2;
    ++w.gen;
}


// Enqueue one Newton iteration of every active partition (no host round
// trip): broad phase (static on the first iteration, else the previous
// line-search list), assembly, PCG, stopping test, CCD, two line-search
// passes, update, and the status copy into pinned memory.
int enqueue_iteration(Ctx &C, bool static_bp, Status *hs) {
    abd_scene *s = C.s;
    World &w = s->w;
    const abd_step_params *p = C.p;
    Counters *dc = P<Counters>(w.ctr);
    int *d_iters = P<int>(w.pcg_sc);
    int rc;
    cudaMemsetAsync(&dc->bad, 0, sizeof(int), s->stream);
    cudaMemsetAsync(d_iters, 0, sizeof(int) * kPcgWords, s->stream);
    // active set at q: static broad phase on the first iteration, then the
    // previous line-search list (q lies on that swept path)
    if ((rc = launch_transform(s, P<double>(w.q), P<double>(w.x), nullptr, 0))) return rc;
    if (static_bp) {
        if ((rc = launch_boxes(s, false, C.half, -1, nullptr)) || (rc = launch_l1_async(s, false)) ||
            (rc = launch_l2_async(s, false, C.half)) ||
            (rc = launch_narrow_async(s, P<PairRec>(w.cand), &dc->cand, w.cap_cand, p->dhat)))
            return rc;
    } else if ((rc = launch_narrow_async(s, P<PairRec>(w.ls), &dc->ls, w.cap_ls, p->dhat))) {
        return rc;
    }
    // assemble, precondition, solve
    // the first (directly launched) iteration of a local solve in FP64 when
    // the mixed path asks for it; the captured steady-state iterations in
    // the path's own precision
    const int prec = static_bp && C.precision == ABD_MIXED && p->mixed_fp64_first ? ABD_FP64 : C.precision;
    C.it_prec = prec;
    if ((rc = launch_assemble_async(s, prec, p))) return rc;
    if ((rc = launch_pcg_async(s, prec, p))) return rc;
    // Newton stopping test before the line search
    ABD_LAUNCH(s, k_dqmax, grid_for(w.S_dyn, 128), 128, 0, s->stream, w.S_dyn, P<int>(w.slot_part), P<double>(w.dq),
               P<PartState>(w.part));
    ABD_LAUNCH(s, k_newton_decide, 1, 256, 0, s->stream, w.NP, P<PartState>(w.part), p->newton_tol);
    // CCD along q -> q + dq over the swept candidates; line-search list
    if ((rc = launch_transform(s, P<double>(w.q), P<double>(w.x1), P<double>(w.dq), 1)) ||
        (rc = launch_boxes(s, true, C.half, 1, P<double>(w.dq))) || (rc = launch_l1_async(s, true)) ||
        (rc = launch_l2_async(s, true, C.half)) || (rc = launch_ccd_async(s, p, true)))
        return rc;
    // backtracking on the FP64 energy: two passes of kLS trial steps
    ABD_LAUNCH(s, k_ls_reset, 1, 256, 0, s->stream, w.NP, P<int>(C.nh0), P<int>(C.decided));
    for (int pass = 0; pass < 2; ++pass) {
        cudaMemsetAsync(&dc->pending, 0, sizeof(int), s->stream);
        cudaMemsetAsync(&dc->ls_live, 0, sizeof(int), s->stream);
        ABD_LAUNCH(s, k_ls_alphas, 1, 256, 0, s->stream, w.NP, P<PartState>(w.part), P<int>(C.nh0),
                   P<int>(C.decided), P<double>(C.alphas), p->max_halvings, &dc->ls_live);
        if ((rc = launch_energy_async(s, p, P<double>(C.alphas)))) return rc;
        ABD_LAUNCH(s, k_ls_select, 1, 256, 0, s->stream, w.NP, P<PartState>(w.part), P<int>(C.nh0),
                   P<int>(C.decided), P<double>(C.alphas), p->max_halvings, &dc->pending);
    }
    ABD_LAUNCH(s, k_check_bad, 1, 1, 0, s->stream, dc, w.cap_l1, w.cap_cand, w.cap_act, w.cap_ls, w.cap_cp,
               d_iters + kPcgOver);
    ABD_LAUNCH(s, k_update_q, grid_for(12 * (int64_t)w.S_dyn, 256), 256, 0, s->stream, w.S_dyn,
               P<int>(w.slot_part), P<PartState>(w.part), P<int>(C.decided), dc, P<double>(w.dq), P<double>(w.q));
    ABD_LAUNCH(s, k_mark_updated, 1, 256, 0, s->stream, w.NP, P<int>(C.decided), dc);
    return enqueue_status(s, hs);
}

// The steady-state iteration (static_bp false) as a CUDA graph: captured on
// the scene's stream, re-captured when the world or a list buffer changed
// (w.gen) and instantiated afresh.  Profiling
// events become graph nodes.  Returns false when capture is not possible
// (the legacy default stream cannot be captured).
bool iteration_graph(Ctx &C, Status *hs) {
    abd_scene *s = C.s;
    IterGraph &g = s->ig;
    if (g.disabled || !s->stream) return false;
    if (g.exec && g.gen == s->w.gen && (s->prof == !g.ev.empty() || !s->prof)) return true;
    prof_graph_release(s);
    int64_t L0 = s->n_launches;
    if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        g.disabled = true;
        return false;
    }
    int rc = enqueue_iteration(C, false, hs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->stream, &graph);
    int kernels = (int)(s->n_launches - L0);
    s->n_launches = L0;
    if (rc || e != cudaSuccess || !graph) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        g.disabled = true;
        return false;
    }
    // always a fresh instantiation (the stream is idle here): an in-place
    // update would have to carry the PCG node's cluster shape along with its
    // grid, which change together when the cluster size changes
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    if (cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        g.exec = nullptr;
        cudaGraphDestroy(graph);
        g.disabled = true;
        return false;
    }
    cudaGraphDestroy(graph);
    g.gen = s->w.gen;
    g.kernels = kernels;
    return true;
}

// Projected Newton on Eq. 5 for every partition whose `run` flag is set.  One
// iteration is enqueued without host round trips (list sizes stay on the
// device, decisions are made by small kernels) and ends with one status read;
// an iteration whose lists overflowed is redone with larger buffers.
int newton_solve(Ctx &C, const std::vector<int> &run, int &newton_total, int &maxed) {
    abd_scene *s = C.s;
    World &w = s->w;
    const abd_step_params *p = C.p;
    int rc = ensure_lists(C);
    if (rc) return rc;
    ensure_side(s);
    Status *hs = pinned_status(s);
    if (!hs) return set_err(s, ABD_E_OOM, "pinned status");
    std::vector<PartState> ps(w.NP);
    for (int i = 0; i < w.NP; ++i) {
        memset(&ps[i], 0, sizeof(PartState));
        ps[i].active = run[i];
        ps[i].toi = 0x3FF0000000000000ull;
        ps[i].kB = C.kBp[i];
        ps[i].inv_hl = 1.0 / (p->h * C.lp[i]);
    }
    if ((rc = write_parts(s, ps))) return rc;
    Counters *dc = P<Counters>(w.ctr);
    int *d_iters = P<int>(w.pcg_sc);
    bool static_bp = true, any = false;
    for (int i = 0; i < w.NP; ++i) any |= run[i] != 0;
    int it = 0;
    while (any && it < p->max_newton) {
        double t0 = now_ms();
        bool graphed = !static_bp && iteration_graph(C, hs);
        if (graphed) {
            C.it_prec = C.precision;  // the captured iteration runs in the path's own precision
            if ((rc = cuda_check(s, cudaGraphLaunch(s->ig.exec, s->stream), "graph launch"))) return rc;
            s->n_launches += s->ig.kernels;
        } else if ((rc = enqueue_iteration(C, static_bp, hs))) {
            return rc;
        }
        if ((rc = sync(s))) return rc;
        if (graphed) prof_graph_replayed(s);
        if (hs->c.bad) {
            // lists outgrew their buffers: grow, restore the partition state, redo
            ++C.st->list_redo;
            grow_lists(w, hs->c, hs->pcg_over != 0);
            if ((rc = ensure_lists(C)) || (rc = write_parts(s, ps))) return rc;
            static_bp = true;
            continue;
        }
        // rare: line searches still undecided after 2 * kLS halvings
        for (int guard = 0; hs->c.pending > 0 && guard < 64; ++guard) {
            cudaMemsetAsync(&dc->pending, 0, sizeof(int), s->stream);
            cudaMemsetAsync(&dc->ls_live, 0, sizeof(int), s->stream);
            ABD_LAUNCH(s, k_ls_alphas, 1, 256, 0, s->stream, w.NP, P<PartState>(w.part), P<int>(C.nh0),
                       P<int>(C.decided), P<double>(C.alphas), p->max_halvings, &dc->ls_live);
            if ((rc = launch_energy_async(s, p, P<double>(C.alphas)))) return rc;
            ABD_LAUNCH(s, k_ls_select, 1, 256, 0, s->stream, w.NP, P<PartState>(w.part), P<int>(C.nh0),
                       P<int>(C.decided), P<double>(C.alphas), p->max_halvings, &dc->pending);
            ABD_LAUNCH(s, k_update_q, grid_for(12 * (int64_t)w.S_dyn, 256), 256, 0, s->stream, w.S_dyn,
                       P<int>(w.slot_part), P<PartState>(w.part), P<int>(C.decided), dc, P<double>(w.dq),
                       P<double>(w.q));
            ABD_LAUNCH(s, k_mark_updated, 1, 256, 0, s->stream, w.NP, P<int>(C.decided), dc);
            if ((rc = enqueue_status(s, hs)) || (rc = sync(s))) return rc;
        }
        static_bp = false;
        ++it;
        C.st->n_active_peak = std::max<int64_t>(C.st->n_active_peak, (int64_t)hs->c.act);
        C.st->n_candidates_peak = std::max<int64_t>(C.st->n_candidates_peak, (int64_t)hs->c.cand);
        int64_t pmax = 0;
        for (int i = 0; i < w.NP; ++i) pmax = std::max<int64_t>(pmax, hs->pcg_iters[i]);
        C.st->pcg_iters += pmax;
        C.st->pcg_cluster = std::max(C.st->pcg_cluster, s->pcg_cs_last);
        C.st->pcg_unstaged |= hs->pcg_unstaged != 0;
        pcg_tune_observe(s, pmax);
        if (s->prof) {
            double tb = C.it_prec == ABD_MIXED ? 4.0 : 8.0;
            // algorithmic bytes of one PCG launch, counted per iteration: each
            // iteration of partition i reads its blocks (diagonal and
            // off-diagonal, 144 entries each) and seven 12-vectors per slot
            // (p, Ap, r, z, x and the preconditioner's input and output)
            double pb = 0.0;
            for (int i = 0; i < w.NP; ++i) {
                double S_i = (double)(w.h_part_off[i + 1] - w.h_part_off[i]);
                pb += (double)hs->pcg_iters[i] * (144.0 * tb * (S_i + 0.5 * hs->pcg_nent[i]) + 7.0 * 12.0 * tb * S_i);
            }
            prof_add_bytes(s, "pcg", pb);
            // the swept pass's level-1 count is the one left in the counters
            prof_add_bytes(s, "l2_swept", (double)std::min<int64_t>((int64_t)hs->c.l1, w.cap_l1) *
                                              l2_bytes_per_pair(s, true));
            // one pair assembly: record, four FP64 positions, gradient and
            // three 12x12 blocks accumulated
            prof_add_bytes(s, "pair_assemble", (double)hs->c.act * (sizeof(PairRec) + 96.0 + 96.0 + 3.0 * 144.0 * tb));
            prof_add_bytes(s, "pair_moll", (double)hs->n_moll * (sizeof(PairRec) + 8.0 + 96.0 + 96.0 + 3.0 * 144.0 * tb));
            // energies: the line-search list and its positions at two
            // configurations, per pass
            prof_add_bytes(s, "energy", 2.0 * (double)hs->c.ls * (sizeof(PairRec) + 192.0));
        }
        any = false;
        for (int i = 0; i < w.NP; ++i) {
            ps[i] = hs->part[i];
            any |= ps[i].active != 0;
        }
        C.t_solve += now_ms() - t0;
    }
    for (int i = 0; i < w.NP; ++i) newton_total += ps[i].newton_it;
    if ((int)C.part_newton.size() < w.NP) C.part_newton.resize(w.NP, 0);
    for (int i = 0; i < w.NP; ++i) C.part_newton[i] += ps[i].newton_it;
    if (any) maxed = 1;
    return ABD_OK;
}

// TOI of the merge path q_i -> q^_i for every partition; true when all are 1.
int merge_check(Ctx &C, bool &ok) {
    abd_scene *s = C.s;
    World &w = s->w;
    int rc = ensure_lists(C);
    if (rc) return rc;
    Status *hs = pinned_status(s);
    if (!hs) return set_err(s, ABD_E_OOM, "pinned status");
    std::vector<PartState> ps(w.NP);
    for (int i = 0; i < w.NP; ++i) {
        memset(&ps[i], 0, sizeof(PartState));
        ps[i].active = 1;
        ps[i].toi = 0x3FF0000000000000ull;
    }
    for (int attempt = 0; attempt < 8; ++attempt) {
        if ((rc = write_parts(s, ps))) return rc;
        if ((rc = launch_transform(s, P<double>(w.q), P<double>(w.x), nullptr, 0)) ||
            (rc = launch_transform(s, P<double>(w.q), P<double>(w.x1), P<double>(w.z), 2)) ||
            (rc = launch_boxes(s, true, C.half, 2, P<double>(w.z))) || (rc = launch_l1_async(s, true)) ||
            (rc = launch_l2_async(s, true, C.half)) || (rc = launch_ccd_async(s, C.p, false)))
            return rc;
        if ((rc = enqueue_status(s, hs)) || (rc = sync(s))) return rc;
        if ((int64_t)hs->c.l1 > w.cap_l1 || (int64_t)hs->c.cand > w.cap_cand || (int64_t)hs->c.cp > w.cap_cp) {
            grow_lists(w, hs->c, false);
            if ((rc = ensure_lists(C))) return rc;
            continue;
        }
        ok = true;
        for (int i = 0; i < w.NP; ++i) ok &= hs->part[i].toi == 0x3FF0000000000000ull;
        return ABD_OK;
    }
    return set_err(s, ABD_E_PAIR_OVERFLOW, "merge check: lists keep overflowing");
}

// Minimum distance of the final state (shared bodies at z), over every pair
// of different bodies whose boxes overlap -- across partitions too -- and the
// vertex-plane distances; 0 means touching or penetrating.
int final_min_distance(Ctx &C, double &out) {
    abd_scene *s = C.s;
    World &w = s->w;
    int rc = ensure_lists(C);
    if (rc) return rc;
    Status *hs = pinned_status(s);
    if (!hs) return set_err(s, ABD_E_OOM, "pinned status");
    std::vector<PartState> ps(w.NP);
    for (int i = 0; i < w.NP; ++i) {
        memset(&ps[i], 0, sizeof(PartState));
        ps[i].active = 1;
    }
    Counters *dc = P<Counters>(w.ctr);
    for (int attempt = 0; attempt < 8; ++attempt) {
        if ((rc = write_parts(s, ps))) return rc;
        const unsigned long long big = 0x7FEFFFFFFFFFFFFFull;  // largest finite double
        cudaMemcpyAsync(&dc->mind, &big, sizeof big, cudaMemcpyHostToDevice, s->stream);
        if ((rc = launch_transform(s, P<double>(w.q), P<double>(w.x), P<double>(w.z), 2)) ||
            (rc = launch_boxes(s, false, C.half, -2, nullptr)) || (rc = launch_l1_async(s, false, 1)) ||
            (rc = launch_l2_async(s, false, C.half)) || (rc = launch_min_dist_async(s)) ||
            (rc = enqueue_status(s, hs)) || (rc = sync(s)))
            return rc;
        if ((int64_t)hs->c.l1 > w.cap_l1 || (int64_t)hs->c.cand > w.cap_cand || (int64_t)hs->c.cp > w.cap_cp) {
            grow_lists(w, hs->c, false);
            if ((rc = ensure_lists(C))) return rc;
            continue;
        }
        uint64_t bits = hs->c.mind;
        memcpy(&out, &bits, sizeof out);
        return ABD_OK;
    }
    return set_err(s, ABD_E_PAIR_OVERFLOW, "final check: lists keep overflowing");
}

// Control-based load balancing (Sec. 5.2) after a step on N slabs: work of
// a slab = its Newton iterations x its slots, smoothed; every plane moves by
// abd_pd_update's shift (the slower slab shrinks); planes stay ordered.
void pd_balance(abd_scene *s, const Ctx &C, int N) {
    World &w = s->w;
    if (N < 2 || w.NP != N || (int)s->last_planes.size() != N - 1) return;
    std::vector<double> tau(N);
    for (int i = 0; i < N; ++i) {
        double slots = (double)(w.h_part_off[i + 1] - w.h_part_off[i]);
        double nit = i < (int)C.part_newton.size() ? (double)C.part_newton[i] : 0.0;
        tau[i] = nit * slots;
    }
    if ((int)s->pd_tau.size() != N) s->pd_tau = tau;
    else
        for (int i = 0; i < N; ++i) s->pd_tau[i] = s->pd_smooth * s->pd_tau[i] + (1.0 - s->pd_smooth) * tau[i];
    std::vector<double> delta(N - 1), T(N - 1);
    abd_pd_update(N, s->pd_tau.data(), (int)s->pd_T.size() == N - 1 ? s->pd_T.data() : nullptr, s->pd_kp, s->pd_kd,
                  delta.data(), T.data());
    std::vector<double> planes = s->last_planes;
    for (int i = 0; i < N - 1; ++i) planes[i] += delta[i];
    for (int i = 1; i < N - 1; ++i) planes[i] = std::max(planes[i], planes[i - 1] + 1e-6);
    s->slab_planes = planes;
    s->pd_T = T;
}

int step_impl(abd_scene *s, const abd_step_params *p, abd_step_stats *st, bool force_mono) {
    double T0 = now_ms();
    int64_t L0 = s->n_launches;
    World &w = s->w;
    Ctx C;
    C.s = s; C.p = p; C.st = st; C.precision = p->precision; C.half = 0.5 * p->dhat;
    std::vector<double> box, vh(12 * (size_t)s->nb);
    int rc = body_aabbs(s, box);
    if (rc) return rc;
    if ((rc = cuda_check(s, cudaMemcpyAsync(vh.data(), s->dev.v.p, 96 * (size_t)s->nb, cudaMemcpyDeviceToHost,
                                            s->stream), "v")) || (rc = sync(s)))
        return rc;
    // scene scale l (diagonal of the AABB of every body at the step start,
    // Eq. 8's normalisation) and barrier stiffness (explicit, else 10 x mean
    // dynamic mass x |g| / dhat) over the bodies [b0, b1)
    const double gn = std::sqrt(s->g[0] * s->g[0] + s->g[1] * s->g[1] + s->g[2] * s->g[2]);
    auto scale_of = [&](int64_t b0, int64_t b1, double &l, double &kB) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, msum = 0.0;
        int nd = 0, ndof = 0;
        for (int64_t b = b0; b < b1; ++b) {
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], box[6 * (size_t)b + k]);
                hi[k] = std::max(hi[k], box[6 * (size_t)b + 3 + k]);
            }
            if (s->kind[b] == ABD_DYNAMIC) { msum += s->mass[b]; ++nd; }
            if (s->kind[b] != ABD_STATIC) ++ndof;
        }
        l = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                      (hi[2] - lo[2]) * (hi[2] - lo[2]));
        kB = p->kappa_barrier > 0.0 ? p->kappa_barrier : 10.0 * (nd ? msum / nd : 1.0) * gn / p->dhat;
        return ndof;
    };
    const bool batched = !s->group.empty();
    const int NG = batched ? (int)s->group_off.size() - 1 : 0;
    int ndof = scale_of(0, s->nb, C.l, C.kB);
    if (batched) {
        // every scene of a batched world keeps its own scale and stiffness,
        // so its step is the one it would take alone
        C.lp.resize(NG);
        C.kBp.resize(NG);
        C.l = C.kB = 0.0;
        for (int g = 0; g < NG; ++g) {
            scale_of(s->group_off[g], s->group_off[g + 1], C.lp[g], C.kBp[g]);
            C.l = std::max(C.l, C.lp[g]);
            C.kB = std::max(C.kB, C.kBp[g]);
        }
    }
    if (ndof == 0) {
        // every body is static: the step has no unknowns and nothing moves
        st->l = C.l; st->kappa_barrier = C.kB; st->n_partitions = 1;
        st->admm_iters = 1;
        st->status = ABD_OK;
        st->t_total_ms = now_ms() - T0;
        st->kernel_launches = s->n_launches - L0;
        return ABD_OK;
    }
    std::vector<uint64_t> mask;
    double wov = 0.0;
    int N = 1;
    if (batched) {
        mask.assign(s->nb, 0);
        for (int b = 0; b < s->nb; ++b) mask[b] = s->kind[b] != ABD_STATIC ? 1 : 0;
        N = NG;
    } else {
        int saved = s->n_slabs;
        if (force_mono) s->n_slabs = 1;
        rc = compute_masks(s, p->h, box, vh, mask, wov);
        N = s->n_slabs;
        s->n_slabs = saved;
        if (rc) return rc;
        C.lp.assign(N, C.l);
        C.kBp.assign(N, C.kB);
    }
    if ((rc = build_world(s, mask, N))) return rc;
    st->l = C.l; st->kappa_barrier = C.kB; st->w = wov;
    st->n_partitions = N; st->n_shared = w.nsh; st->n_slots = w.S_dyn;
    ABD_LAUNCH(s, k_slot_init, grid_for(w.S_all, 128), 128, 0, s->stream, w.S_all, w.S_dyn, P<int>(w.slot_body), P<int>(w.slot_rep),
                                                              P<double>(s->dev.q), P<double>(s->dev.v),
                                                              P<double>(s->dev.mass), P<int>(s->dev.kind),
                                                              P<double>(s->dev.omega), p->h, s->g[0], s->g[1], s->g[2],
                                                              p->beta, P<double>(w.q), P<double>(w.qtil),
                                                              P<double>(w.z), P<double>(w.u), P<double>(w.rho));
    if (w.nsh > 0)
        ABD_LAUNCH(s, k_shared_init, grid_for(w.nsh, 128), 128, 0, s->stream, w.nsh, P<int>(w.rep_off), P<int>(w.rep_slot),
                                                                  P<double>(w.qtil), P<double>(w.rho), P<double>(w.zb),
                                                                  P<double>(w.rho0), P<double>(w.rhob));
    cudaMemsetAsync(w.ctr.p, 0, sizeof(Counters), s->stream);
    if ((rc = cuda_check(s, cudaGetLastError(), "step init"))) return rc;
    std::vector<int> run(N, 1);
    int newton = 0, maxed = 0, status = ABD_OK, admm = 0;
    bool converged = false, merge_ok = true;
    double rinf = 0, sinf = 0, dinf = 0;
    if (w.nsh == 0) {
        if ((rc = newton_solve(C, run, newton, maxed))) return rc;
        admm = 1;
        converged = true;
    } else {
        int K = std::max(1, p->max_admm);
        Counters *dc = P<Counters>(w.ctr);
        for (int k = 1; k <= K + 1; ++k) {
            if (k > 1) {
                double ts = now_ms();
                cudaMemsetAsync(&dc->rinf, 0, 24, s->stream);
                ABD_LAUNCH(s, k_consensus, grid_for(w.nsh, 128), 128, 0, s->stream, w.nsh, P<int>(w.rep_off), P<int>(w.rep_slot),
                                                                        P<double>(w.q), P<double>(w.u),
                                                                        P<double>(w.rho), P<double>(w.zb),
                                                                        P<double>(w.rb), P<double>(w.sb), dc);
                ABD_LAUNCH(s, k_delta, grid_for(12 * (int64_t)w.S_dyn, 256), 256, 0, s->stream, w.S_dyn, P<double>(w.q),
                                                                                    P<double>(w.qprev), dc);
                ABD_LAUNCH(s, k_scatter_z, grid_for(12 * (int64_t)w.S_dyn, 256), 256, 0, s->stream, 
                    w.S_dyn, P<int>(w.slot_rep), P<double>(w.zb), P<double>(w.z));
                if ((rc = cuda_check(s, cudaGetLastError(), "consensus"))) return rc;
                if ((rc = merge_check(C, merge_ok))) return rc;
                Counters hc;
                if ((rc = cuda_check(s, cudaMemcpyAsync(&hc, dc, sizeof hc, cudaMemcpyDeviceToHost, s->stream),
                                     "status")) || (rc = sync(s)))
                    return rc;
                rinf = u2d(hc.rinf);
                sinf = u2d(hc.sinf);
                dinf = u2d(hc.dinf);
                double tol = p->theta * p->h * C.l;
                C.t_sync += now_ms() - ts;
                if (dinf < tol && rinf < tol && sinf < tol && merge_ok) { converged = true; break; }
                if (k == K + 1) break;
                if (p->rho_mode == ABD_RHO_ADAPTIVE) {
                    ABD_LAUNCH(s, k_rho_update, grid_for(w.nsh, 128), 128, 0, s->stream, 
                        w.nsh, P<int>(w.rep_off), P<int>(w.rep_slot), P<double>(w.rb), P<double>(w.sb),
                        P<double>(w.rho0), P<double>(w.rhob), P<double>(w.rho), P<double>(w.u), p->tau, p->mu,
                        p->sigma_min, p->sigma_max);
                }
            }
            cudaMemcpyAsync(w.qprev.p, w.q.p, 96 * (size_t)w.S_dyn, cudaMemcpyDeviceToDevice, s->stream);
            if ((rc = newton_solve(C, run, newton, maxed))) return rc;
            ++admm;
        }
        if (!converged) status = merge_ok ? ABD_ADMM_MAXITER : ABD_FELL_BACK_MONOLITHIC;
    }
    if (status == ABD_FELL_BACK_MONOLITHIC && p->dt_split_max > 0) {
        // adaptive time stepping on a blocked merge (reading of Sec. 4.2,
        // Fig. 4: a smaller step lets the replicas merge): the body state is
        // still that of the step start, so retake it as two steps of h/2
        abd_step_params hp = *p;
        hp.h = 0.5 * p->h;
        hp.dt_split_max = p->dt_split_max - 1;
        abd_step_stats a, b;
        memset(&a, 0, sizeof a);
        memset(&b, 0, sizeof b);
        if ((rc = step_impl(s, &hp, &a, false)) < 0) return rc;
        if ((rc = step_impl(s, &hp, &b, false)) < 0) return rc;
        const abd_step_stats first = *st;
        *st = b;
        st->status = ABD_DT_SPLIT;
        st->admm_iters = admm + a.admm_iters + b.admm_iters;
        st->newton_iters = newton + a.newton_iters + b.newton_iters;
        st->pcg_iters = first.pcg_iters + a.pcg_iters + b.pcg_iters;
        st->pcg_cluster = std::max({first.pcg_cluster, a.pcg_cluster, b.pcg_cluster});
        st->pcg_unstaged = first.pcg_unstaged | a.pcg_unstaged | b.pcg_unstaged;
        st->list_redo = first.list_redo + a.list_redo + b.list_redo;
        st->n_candidates_peak = std::max(st->n_candidates_peak, first.n_candidates_peak);
        st->n_active_peak = std::max(st->n_active_peak, first.n_active_peak);
        st->n_candidates_peak = std::max(st->n_candidates_peak, a.n_candidates_peak);
        st->n_active_peak = std::max(st->n_active_peak, a.n_active_peak);
        st->kernel_launches = s->n_launches - L0;
        return ABD_DT_SPLIT;
    }
    if (status == ABD_FELL_BACK_MONOLITHIC) {
        abd_step_stats st2;
        memset(&st2, 0, sizeof st2);
        rc = step_impl(s, p, &st2, true);
        if (rc < 0) return rc;
        st->newton_iters = newton + st2.newton_iters;
        st->admm_iters = admm;
        st->status = status;
        st->pcg_iters += st2.pcg_iters;
        st->pcg_cluster = std::max(st->pcg_cluster, st2.pcg_cluster);
        st->pcg_unstaged |= st2.pcg_unstaged;
        st->list_redo += st2.list_redo;
        st->min_distance = st2.min_distance;
        return status;
    }
    ABD_LAUNCH(s, k_merge, grid_for(s->nb, 128), 128, 0, s->stream, s->nb, P<int>(s->dev.kind), P<int>(w.body_rep),
                                                        P<int>(w.body_slot), P<double>(w.zb), P<double>(w.q), p->h,
                                                        P<double>(s->dev.q), P<double>(s->dev.v));
    if ((rc = cuda_check(s, cudaGetLastError(), "merge")) || (rc = sync(s))) return rc;
    prof_flush(s);
    double mind = 0.0;
    if ((rc = final_min_distance(C, mind))) return rc;
    st->min_distance = mind;
    if (maxed && status == ABD_OK) status = ABD_NEWTON_MAXITER;
    if (mind <= 0.0) status = set_err(s, ABD_E_PENETRATION, "a contact pair or plane is at distance <= 0 after the step");
    st->status = status;
    st->admm_iters = admm;
    st->newton_iters = newton;
    st->r_inf = rinf; st->s_inf = sinf; st->delta_inf = dinf;
    st->t_coll_ms = C.t_coll; st->t_solve_ms = C.t_solve; st->t_sync_ms = C.t_sync;
    st->t_total_ms = now_ms() - T0;
    st->kernel_launches = s->n_launches - L0;
    if (!force_mono && (s->pd_kp != 0.0 || s->pd_kd != 0.0)) pd_balance(s, C, N);
    s->last_part_newton = C.part_newton;
    return status;
}

}  // namespace

extern "C" int abd_step(abd_scene *s, const abd_step_params *p, abd_step_stats *st) {
    if (!s || !p || p->h <= 0 || p->dhat <= 0 || p->dt_split_max < 0 || p->dt_split_max > kMaxDtSplit)
        return ABD_E_INVALID;
    abd_step_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof *st);
    st->min_distance = p->dhat;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != s->device) cudaSetDevice(s->device);
    int rc = step_impl(s, p, st, false);
    if (dev != s->device) cudaSetDevice(dev);
    st->status = rc;
    return rc;
}

extern "C" int abd_partition_masks(abd_scene *s, double h, uint64_t *mask, double *w_out) {
    if (!s || !mask) return ABD_E_INVALID;
    std::vector<double> box, vh(12 * (size_t)s->nb);
    int rc = body_aabbs(s, box);
    if (rc) return rc;
    if ((rc = cuda_check(s, cudaMemcpy(vh.data(), s->dev.v.p, 96 * (size_t)s->nb, cudaMemcpyDeviceToHost), "v")))
        return rc;
    std::vector<uint64_t> m;
    double w = 0;
    if ((rc = compute_masks(s, h, box, vh, m, w))) return rc;
    for (int b = 0; b < s->nb; ++b) mask[b] = m[b];
    if (w_out) *w_out = w;
    return ABD_OK;
}

extern "C" int abd_candidates(abd_scene *s, const double *x0, const double *x1, double dhat, int32_t *out, int64_t cap,
                              int64_t *n_out) {
    if (!s || !x0 || dhat <= 0 || !n_out) return ABD_E_INVALID;
    std::vector<uint64_t> mask(s->nb);
    for (int b = 0; b < s->nb; ++b) mask[b] = s->kind[b] != ABD_STATIC ? 1 : 0;
    int rc = build_world(s, mask, 1);
    if (rc) return rc;
    World &w = s->w;
    std::vector<PartState> ps(1);
    memset(&ps[0], 0, sizeof(PartState));
    ps[0].active = 1;
    if ((rc = write_parts(s, ps))) return rc;
    // caller positions are in global vertex order; slot-vertex order differs
    std::vector<double> xs(3 * (size_t)w.SV), xs1(x1 ? 3 * (size_t)w.SV : 0);
    for (int sl = 0; sl < w.S_all; ++sl) {
        int b = w.h_slot_body[sl];
        for (int v = 0; v < s->nv[b]; ++v)
            for (int k = 0; k < 3; ++k) {
                xs[3 * (w.h_slot_voff[sl] + v) + k] = x0[3 * ((size_t)s->voff[b] + v) + k];
                if (x1) xs1[3 * (w.h_slot_voff[sl] + v) + k] = x1[3 * ((size_t)s->voff[b] + v) + k];
            }
    }
    if ((rc = h2d(s, w.x, xs))) return rc;
    if (x1 && (rc = h2d(s, w.x1, xs1))) return rc;
    double half = 0.5 * dhat;
    if ((rc = launch_vert_bounds(s, x1 != nullptr)) || (rc = launch_boxes(s, x1 != nullptr, half, -2, nullptr)))
        return rc;
    int64_t n_l1 = 0, n = 0;
    if ((rc = launch_l1(s, x1 != nullptr, &n_l1))) return rc;
    DBuf tmp;
    int64_t c = std::max<int64_t>(cap, 1);
    if (!dbuf_ensure(tmp, 12 * (size_t)c)) return set_err(s, ABD_E_OOM, "candidates");
    rc = launch_l2(s, 0, x1 != nullptr, half, n_l1, P<int32_t>(tmp), c, &n);
    if (!rc && out && cap > 0)
        rc = cuda_check(s, cudaMemcpy(out, tmp.p, 12 * (size_t)std::min(n, cap), cudaMemcpyDeviceToHost), "candidates");
    dbuf_free(tmp);
    *n_out = n;
    return rc;
}

extern "C" int abd_partition_get(const abd_scene *s, int32_t part, int32_t *bodies, int32_t cap, int32_t *n,
                                 int32_t *shared, int32_t cap_shared, int32_t *n_shared) {
    if (!s || !n || !n_shared || cap < 0 || cap_shared < 0) return ABD_E_INVALID;
    const World &w = s->w;
    if (part < 0 || part >= w.NP || (int)w.h_part_off.size() < w.NP + 1) return ABD_E_INVALID;
    int cnt = 0, cs = 0;
    for (int sl = w.h_part_off[part]; sl < w.h_part_off[part + 1]; ++sl) {
        int b = w.h_slot_body[sl];
        if (bodies && cnt < cap) bodies[cnt] = b;
        ++cnt;
        if (__builtin_popcountll(w.h_slot_mask[sl]) > 1) {
            if (shared && cs < cap_shared) shared[cs] = b;
            ++cs;
        }
    }
    *n = cnt;
    *n_shared = cs;
    return ABD_OK;
}

extern "C" int abd_partition_newton(const abd_scene *s, int32_t *iters, int32_t cap, int32_t *n) {
    if (!s || !n || cap < 0) return ABD_E_INVALID;
    *n = (int32_t)s->last_part_newton.size();
    if (iters)
        for (int i = 0; i < std::min<int>(*n, cap); ++i) iters[i] = (int32_t)s->last_part_newton[i];
    return ABD_OK;
}
