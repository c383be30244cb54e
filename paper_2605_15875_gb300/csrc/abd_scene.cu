// abd_scene.cu -- scene lifetime, per-body constants, partition membership,
// state transfer, diagnostics and profiling for the GB300 ABD-IPC library.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "abd_internal.h"

using namespace abd;

namespace abd {

bool dbuf_ensure(DBuf &b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return true;
    dbuf_free(b);
    size_t nb = bytes < 256 ? 256 : bytes + bytes / 4;
    if (cudaMalloc(&b.p, nb) != cudaSuccess) {
        b.p = nullptr;
        b.bytes = 0;
        cudaGetLastError();
        return false;
    }
    b.bytes = nb;
    return true;
}

void dbuf_free(DBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int set_err(abd_scene *s, int code, const std::string &msg) {
    if (s) s->err = msg;
    return code;
}

int cuda_check(abd_scene *s, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return ABD_OK;
    cudaGetLastError();
    return set_err(s, e == cudaErrorMemoryAllocation ? ABD_E_OOM : ABD_E_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

int prof_index(abd_scene *s, const char *name) {
    for (size_t i = 0; i < s->kstats.size(); ++i)
        if (s->kstats[i].name == name) return (int)i;
    KStat k;
    k.name = name;
    s->kstats.push_back(k);
    return (int)s->kstats.size() - 1;
}

bool stream_capturing(abd_scene *s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!s->stream || cudaStreamIsCapturing(s->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusActive;
}

// While the stream is being captured into the iteration graph, the events
// become graph nodes (external records) and the pair is kept with the graph;
// its bytes are added on every replay (prof_graph_replayed).
void prof_begin(abd_scene *s, const char *name, double bytes, cudaEvent_t *a, cudaEvent_t *b, cudaStream_t st) {
    *a = *b = nullptr;
    if (!s->prof) return;
    if (!st) st = s->stream;
    for (int k = 0; k < 2; ++k) {
        cudaEvent_t e;
        if (!s->ev_pool.empty()) {
            e = s->ev_pool.back();
            s->ev_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            return;
        }
        (k ? *b : *a) = e;
    }
    int idx = prof_index(s, name);
    if (stream_capturing(s)) {
        s->ig.ev.push_back({idx, bytes, *a, *b});
        cudaEventRecordWithFlags(*a, st, cudaEventRecordExternal);
        return;
    }
    s->kstats[idx].bytes += bytes;
    cudaEventRecord(*a, st);
}

void prof_add_bytes(abd_scene *s, const char *name, double bytes) {
    if (s->prof) s->kstats[prof_index(s, name)].bytes += bytes;
}

void prof_end(abd_scene *s, cudaEvent_t a, cudaEvent_t b, int idx, cudaStream_t st) {
    if (!a || !b) return;
    if (!st) st = s->stream;
    if (stream_capturing(s)) {
        cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
        return;
    }
    cudaEventRecord(b, st);
    s->ev_pending.push_back({idx, {a, b}});
}

void ensure_side(abd_scene *s) {
    if (s->side || !s->stream || s->no_side) return;
    if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) == cudaSuccess)
        return;
    cudaGetLastError();  // no side stream: both branches run on the scene's stream
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->side) cudaStreamDestroy(s->side);
    s->side = nullptr;
    s->ev_fork = s->ev_join = nullptr;
}

void scene_no_side(abd_scene *s) { s->no_side = true; }

cudaStream_t fork_side(abd_scene *s) {
    if (!s->side || !s->ev_join) return s->stream;
    cudaEventRecord(s->ev_fork, s->stream);
    cudaStreamWaitEvent(s->side, s->ev_fork, 0);
    return s->side;
}

void join_side(abd_scene *s, cudaStream_t side) {
    if (side == s->stream) return;
    cudaEventRecord(s->ev_join, side);
    cudaStreamWaitEvent(s->stream, s->ev_join, 0);
}

// After a replay of the iteration graph has completed: accumulate its event
// pairs (they are overwritten by the next replay).
void prof_graph_replayed(abd_scene *s) {
    if (!s->prof) return;
    for (auto &e : s->ig.ev) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
            s->kstats[e.idx].ms += ms;
            s->kstats[e.idx].launches += 1;
            s->kstats[e.idx].bytes += e.bytes;
        }
        cudaGetLastError();
    }
}

// Return the graph's event pairs to the pool (graph re-captured or freed).
void prof_graph_release(abd_scene *s) {
    for (auto &e : s->ig.ev) {
        s->ev_pool.push_back(e.a);
        s->ev_pool.push_back(e.b);
    }
    s->ig.ev.clear();
}

// Resolve recorded event pairs (call after a stream synchronisation).
void prof_flush(abd_scene *s) {
    for (auto &pe : s->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
            s->kstats[pe.first].ms += ms;
            s->kstats[pe.first].launches += 1;
        }
        cudaGetLastError();
        s->ev_pool.push_back(pe.second.first);
        s->ev_pool.push_back(pe.second.second);
    }
    s->ev_pending.clear();
}

}  // namespace abd

// Volume, centre of mass and second moment about the centre of mass of a
// closed outward mesh, by the divergence theorem over the tetrahedra
// (origin, v0, v1, v2): per tetrahedron V_t = det/6, first moment V_t * sum/4,
// second moment about the origin (V_t/20)(sum v v^T + s s^T); the moment about
// the centre follows from the parallel-axis shift.
static bool mesh_mass(const double *xb, int nv, const int32_t *tri, int nt, double rho, double &m, double com[3],
                      double S[9], double &vol) {
    double V = 0, F[3] = {0, 0, 0}, M2[9] = {0};
    for (int t = 0; t < nt; ++t) {
        int i0 = tri[3 * t], i1 = tri[3 * t + 1], i2 = tri[3 * t + 2];
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) return false;
        const double *a = xb + 3 * i0, *b = xb + 3 * i1, *c = xb + 3 * i2;
        double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                     a[2] * (b[0] * c[1] - b[1] * c[0]);
        double vt = det / 6.0;
        V += vt;
        double sm[3] = {a[0] + b[0] + c[0], a[1] + b[1] + c[1], a[2] + b[2] + c[2]};
        for (int k = 0; k < 3; ++k) F[k] += vt * sm[k] * 0.25;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                M2[3 * i + j] += vt / 20.0 * (a[i] * a[j] + b[i] * b[j] + c[i] * c[j] + sm[i] * sm[j]);
    }
    if (!(V > 0.0)) return false;
    for (int k = 0; k < 3; ++k) com[k] = F[k] / V;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[3 * i + j] = rho * (M2[3 * i + j] - V * com[i] * com[j]);
    m = rho * V;
    vol = V;
    return true;
}

// Order of n primitives along a Morton curve of their rest-frame centres
// (10 bits per axis over the body's box); chunks of 32 consecutive entries
// form the clusters the broad phase filters before it looks at primitives.
static void morton_order(const std::vector<double> &c, int n, int *out) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], c[3 * i + k]);
            hi[k] = std::max(hi[k], c[3 * i + k]);
        }
    std::vector<std::pair<uint64_t, int>> key(n);
    for (int i = 0; i < n; ++i) {
        uint64_t code = 0;
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            double t = hi[k] > lo[k] ? (c[3 * i + k] - lo[k]) / (hi[k] - lo[k]) : 0.0;
            q[k] = (uint32_t)std::min(1023.0, std::max(0.0, t * 1023.0));
        }
        for (int bit = 9; bit >= 0; --bit)
            for (int k = 0; k < 3; ++k) code = (code << 1) | ((q[k] >> bit) & 1u);
        key[i] = {code, i};
    }
    std::sort(key.begin(), key.end());
    for (int i = 0; i < n; ++i) out[i] = key[i].second;
}

static bool upload(abd_scene *s, DBuf &b, const void *h, size_t bytes) {
    if (!dbuf_ensure(b, bytes ? bytes : 8)) return false;
    if (bytes && cudaMemcpy(b.p, h, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return false;
    (void)s;
    return true;
}

extern "C" int abd_scene_create(const abd_scene_desc *d, void *stream, abd_scene **out) {
    if (!d || !out || d->n_bodies <= 0 || d->n_meshes <= 0 || d->n_planes < 0 || d->n_planes > kMaxPlanes)
        return ABD_E_INVALID;
    *out = nullptr;
    abd_scene *s = new abd_scene();
    cudaGetDevice(&s->device);
    s->stream = (cudaStream_t)stream;
    int nm = d->n_meshes, nb = d->n_bodies;
    std::vector<int64_t> mvo(nm + 1, 0), mto(nm + 1, 0);
    for (int m = 0; m < nm; ++m) {
        if (d->mesh_n_verts[m] <= 0 || d->mesh_n_tris[m] < 0) { delete s; return ABD_E_INVALID; }
        mvo[m + 1] = mvo[m] + d->mesh_n_verts[m];
        mto[m + 1] = mto[m] + d->mesh_n_tris[m];
    }
    for (int m = 0; m < nm; ++m)
        for (int64_t i = 3 * mto[m]; i < 3 * mto[m + 1]; ++i)
            if (d->mesh_tris[i] < 0 || d->mesh_tris[i] >= d->mesh_n_verts[m]) { delete s; return ABD_E_INVALID; }
    // unique sorted edges per mesh
    std::vector<std::vector<int>> medges(nm);
    for (int m = 0; m < nm; ++m) {
        std::vector<std::pair<int, int>> e;
        e.reserve(3 * d->mesh_n_tris[m]);
        for (int t = 0; t < d->mesh_n_tris[m]; ++t)
            for (int k = 0; k < 3; ++k) {
                int a = d->mesh_tris[3 * (mto[m] + t) + k], b = d->mesh_tris[3 * (mto[m] + t) + (k + 1) % 3];
                e.push_back({std::min(a, b), std::max(a, b)});
            }
        std::sort(e.begin(), e.end());
        e.erase(std::unique(e.begin(), e.end()), e.end());
        for (auto &p : e) {
            medges[m].push_back(p.first);
            medges[m].push_back(p.second);
        }
    }
    s->nb = nb;
    s->kind.resize(nb); s->voff.resize(nb + 1); s->nv.resize(nb); s->toff.resize(nb + 1); s->nt.resize(nb);
    s->eoff.resize(nb + 1); s->ne.resize(nb);
    s->mass.assign(nb, 0.0); s->S.assign(9 * (size_t)nb, 0.0); s->vol.assign(nb, 0.0); s->kappa.assign(nb, 0.0);
    s->com.assign(3 * (size_t)nb, 0.0);
    s->voff[0] = s->toff[0] = s->eoff[0] = 0;
    for (int b = 0; b < nb; ++b) {
        int m = d->body_mesh[b];
        if (m < 0 || m >= nm) { delete s; return ABD_E_INVALID; }
        s->nv[b] = d->mesh_n_verts[m];
        s->nt[b] = d->mesh_n_tris[m];
        s->ne[b] = (int)medges[m].size() / 2;
        s->voff[b + 1] = s->voff[b] + s->nv[b];
        s->toff[b + 1] = s->toff[b] + s->nt[b];
        s->eoff[b + 1] = s->eoff[b] + s->ne[b];
    }
    s->V = s->voff[nb]; s->T = s->toff[nb]; s->E = s->eoff[nb];
    if (s->V >= (1ll << 31) || s->T >= (1ll << 31) || s->E >= (1ll << 31)) { delete s; return ABD_E_INVALID; }
    s->xbar.resize(3 * (size_t)s->V); s->tri.resize(3 * (size_t)s->T); s->edge.resize(2 * (size_t)s->E);
    s->erest2.resize((size_t)s->E);
    std::vector<double> q(12 * (size_t)nb), v(12 * (size_t)nb, 0.0), omega(3 * (size_t)nb, 0.0);
    for (int b = 0; b < nb; ++b) {
        int m = d->body_mesh[b];
        s->kind[b] = d->body_kind[b];
        s->kappa[b] = d->body_kappa[b];
        if (s->kind[b] != ABD_DYNAMIC && s->kind[b] != ABD_STATIC && s->kind[b] != ABD_KINEMATIC) {
            delete s;
            return ABD_E_INVALID;
        }
        const double *mx = d->mesh_xbar + 3 * mvo[m];
        const int32_t *mt = d->mesh_tris + 3 * mto[m];
        double com[3] = {0, 0, 0};
        if (s->kind[b] != ABD_STATIC) {
            if (!mesh_mass(mx, s->nv[b], mt, s->nt[b], d->body_density[b], s->mass[b], com, &s->S[9 * (size_t)b],
                           s->vol[b])) {
                delete s;
                return ABD_E_INVALID;
            }
        }
        if (s->kind[b] == ABD_KINEMATIC) {
            // prescribed motion: inertia weighted so that contacts cannot
            // move the body measurably off its predicted (prescribed) pose
            s->mass[b] *= kKinematicWeight;
            for (int i = 0; i < 9; ++i) s->S[9 * (size_t)b + i] *= kKinematicWeight;
            if (d->body_omega)
                for (int k = 0; k < 3; ++k) omega[3 * (size_t)b + k] = d->body_omega[3 * (size_t)b + k];
        }
        for (int k = 0; k < 3; ++k) s->com[3 * (size_t)b + k] = com[k];
        for (int i = 0; i < s->nv[b]; ++i)
            for (int k = 0; k < 3; ++k) s->xbar[3 * ((size_t)s->voff[b] + i) + k] = mx[3 * i + k] - com[k];
        for (int i = 0; i < 3 * s->nt[b]; ++i) s->tri[3 * (size_t)s->toff[b] + i] = mt[i];
        for (int e = 0; e < s->ne[b]; ++e) {
            int a = medges[m][2 * e], c = medges[m][2 * e + 1];
            s->edge[2 * ((size_t)s->eoff[b] + e)] = a;
            s->edge[2 * ((size_t)s->eoff[b] + e) + 1] = c;
            double dx = mx[3 * a] - mx[3 * c], dy = mx[3 * a + 1] - mx[3 * c + 1], dz = mx[3 * a + 2] - mx[3 * c + 2];
            s->erest2[(size_t)s->eoff[b] + e] = dx * dx + dy * dy + dz * dz;
        }
        const double *q0 = d->body_q0 + 12 * (size_t)b;
        for (int i = 0; i < 12; ++i) q[12 * (size_t)b + i] = q0[i];
        for (int k = 0; k < 3; ++k)
            q[12 * (size_t)b + k] += q0[3 + 3 * k] * com[0] + q0[4 + 3 * k] * com[1] + q0[5 + 3 * k] * com[2];
        if (d->body_v0)
            for (int i = 0; i < 12; ++i) v[12 * (size_t)b + i] = d->body_v0[12 * (size_t)b + i];
    }
    // primitive cluster orders (rest frame, per body)
    s->vperm.resize((size_t)s->V);
    s->tperm.resize((size_t)s->T);
    s->eperm.resize((size_t)s->E);
    for (int b = 0; b < nb; ++b) {
        const double *xb = s->xbar.data() + 3 * (size_t)s->voff[b];
        std::vector<double> c(3 * (size_t)std::max(s->nv[b], std::max(s->nt[b], s->ne[b])));
        morton_order(std::vector<double>(xb, xb + 3 * (size_t)s->nv[b]), s->nv[b], s->vperm.data() + s->voff[b]);
        for (int t = 0; t < s->nt[b]; ++t)
            for (int k = 0; k < 3; ++k) {
                const int *tr = s->tri.data() + 3 * ((size_t)s->toff[b] + t);
                c[3 * t + k] = (xb[3 * tr[0] + k] + xb[3 * tr[1] + k] + xb[3 * tr[2] + k]) / 3.0;
            }
        morton_order(c, s->nt[b], s->tperm.data() + s->toff[b]);
        for (int e = 0; e < s->ne[b]; ++e)
            for (int k = 0; k < 3; ++k) {
                const int *ed = s->edge.data() + 2 * ((size_t)s->eoff[b] + e);
                c[3 * e + k] = 0.5 * (xb[3 * ed[0] + k] + xb[3 * ed[1] + k]);
            }
        morton_order(c, s->ne[b], s->eperm.data() + s->eoff[b]);
    }
    // rest-frame boxes of the clusters (centre, half extent of their vertices)
    s->cbody_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        int nc = (s->nv[b] + kClusterSize - 1) / kClusterSize + (s->nt[b] + kClusterSize - 1) / kClusterSize +
                 (s->ne[b] + kClusterSize - 1) / kClusterSize;
        s->cbody_off[b + 1] = s->cbody_off[b] + nc;
    }
    s->crest.assign(6 * (size_t)s->cbody_off[nb], 0.0);
    for (int b = 0; b < nb; ++b) {
        const double *xb = s->xbar.data() + 3 * (size_t)s->voff[b];
        int c = s->cbody_off[b];
        for (int kind = 0; kind < 3; ++kind) {
            int n = kind == 0 ? s->nv[b] : (kind == 1 ? s->nt[b] : s->ne[b]);
            for (int j = 0; j * kClusterSize < n; ++j, ++c) {
                double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
                for (int i = j * kClusterSize; i < std::min(n, (j + 1) * kClusterSize); ++i) {
                    int vs[3], k = 0;
                    if (kind == 0) vs[k++] = s->vperm[s->voff[b] + i];
                    else if (kind == 1) {
                        const int *t = s->tri.data() + 3 * ((size_t)s->toff[b] + s->tperm[s->toff[b] + i]);
                        vs[0] = t[0]; vs[1] = t[1]; vs[2] = t[2]; k = 3;
                    } else {
                        const int *e = s->edge.data() + 2 * ((size_t)s->eoff[b] + s->eperm[s->eoff[b] + i]);
                        vs[0] = e[0]; vs[1] = e[1]; k = 2;
                    }
                    for (int q = 0; q < k; ++q)
                        for (int a = 0; a < 3; ++a) {
                            lo[a] = std::min(lo[a], xb[3 * vs[q] + a]);
                            hi[a] = std::max(hi[a], xb[3 * vs[q] + a]);
                        }
                }
                for (int a = 0; a < 3; ++a) {
                    s->crest[6 * (size_t)c + a] = 0.5 * (lo[a] + hi[a]);
                    s->crest[6 * (size_t)c + 3 + a] = 0.5 * (hi[a] - lo[a]);
                }
            }
        }
    }
    s->planes.n = d->n_planes;
    for (int i = 0; i < d->n_planes; ++i) {
        if (d->plane_axis[i] < 0 || d->plane_axis[i] > 2) { delete s; return ABD_E_INVALID; }
        s->planes.axis[i] = d->plane_axis[i];
        s->planes.sign[i] = d->plane_sign[i];
        s->planes.offset[i] = d->plane_offset[i];
    }
    for (int k = 0; k < 3; ++k) s->g[k] = d->gravity[k];
    SceneDev &D = s->dev;
    D.nb = nb; D.V = s->V; D.T = s->T; D.E = s->E;
    bool ok = upload(s, D.q, q.data(), q.size() * 8) && upload(s, D.v, v.data(), v.size() * 8) &&
              upload(s, D.mass, s->mass.data(), nb * 8) && upload(s, D.S, s->S.data(), s->S.size() * 8) &&
              upload(s, D.vol, s->vol.data(), nb * 8) && upload(s, D.kappa, s->kappa.data(), nb * 8) &&
              upload(s, D.kind, s->kind.data(), nb * 4) && upload(s, D.voff, s->voff.data(), (nb + 1) * 4) &&
              upload(s, D.nv, s->nv.data(), nb * 4) && upload(s, D.toff, s->toff.data(), (nb + 1) * 4) &&
              upload(s, D.nt, s->nt.data(), nb * 4) && upload(s, D.eoff, s->eoff.data(), (nb + 1) * 4) &&
              upload(s, D.ne, s->ne.data(), nb * 4) && upload(s, D.xbar, s->xbar.data(), s->xbar.size() * 8) &&
              upload(s, D.tri, s->tri.data(), s->tri.size() * 4) &&
              upload(s, D.edge, s->edge.data(), s->edge.size() * 4) &&
              upload(s, D.erest2, s->erest2.data(), s->erest2.size() * 8) &&
              upload(s, D.vperm, s->vperm.data(), s->vperm.size() * 4) &&
              upload(s, D.tperm, s->tperm.data(), s->tperm.size() * 4) &&
              upload(s, D.eperm, s->eperm.data(), s->eperm.size() * 4) &&
              upload(s, D.cbody_off, s->cbody_off.data(), s->cbody_off.size() * 4) &&
              upload(s, D.omega, omega.data(), omega.size() * 8) &&
              upload(s, D.crest, std::vector<float>(s->crest.begin(), s->crest.end()).data(), s->crest.size() * 4);
    if (!ok) {
        abd_scene_destroy(s);
        cudaGetLastError();
        return ABD_E_OOM;
    }
    *out = s;
    return ABD_OK;
}

extern "C" void abd_scene_destroy(abd_scene *s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    if (s->side) cudaStreamSynchronize(s->side);
    if (s->ig.exec) cudaGraphExecDestroy(s->ig.exec);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->side) cudaStreamDestroy(s->side);
    prof_graph_release(s);
    for (auto &t : s->pcg_tune) {
        if (t.a) cudaEventDestroy(t.a);
        if (t.b) cudaEventDestroy(t.b);
    }
    SceneDev &D = s->dev;
    DBuf *bufs[] = {&D.q, &D.v, &D.mass, &D.S, &D.vol, &D.kappa, &D.kind, &D.voff, &D.nv, &D.toff, &D.nt,
                    &D.eoff, &D.ne, &D.xbar, &D.tri, &D.edge, &D.erest2, &D.vperm, &D.tperm, &D.eperm, &D.cbody_off, &D.crest, &D.omega};
    for (DBuf *b : bufs) dbuf_free(*b);
    World &w = s->w;
    DBuf *wb[] = {&w.slot_body, &w.slot_part, &w.slot_voff, &w.slot_mask, &w.slot_rep, &w.slot_kw, &w.sv_slot,
                  &w.q, &w.qprev, &w.qtil, &w.z, &w.u, &w.rho, &w.dq, &w.g, &w.x, &w.x1, &w.dx, &w.box, &w.box1,
                  &w.rep_off, &w.rep_slot, &w.zb, &w.rho0, &w.rhob, &w.rb, &w.sb, &w.body_rep, &w.body_slot,
                  &w.l1, &w.cand, &w.act, &w.ls, &w.diag, &w.off, &w.offflag,
                  &w.pcg_sc, &w.part, &w.ctr, &w.aabb, &w.part_off, &w.nmoll, &w.rowcnt, &w.rowoff, &w.rowcur, &w.ent, &w.slot_cbase, &w.cl_info, &w.cbox, &w.cbox1, &w.cp, &w.xb, &w.xb1};
    for (DBuf *b : wb) dbuf_free(*b);
    if (s->pinned) cudaFreeHost(s->pinned);
    for (auto &pe : s->ev_pending) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (auto e : s->ev_pool) cudaEventDestroy(e);
    delete s;
}

extern "C" int abd_scene_counts(const abd_scene *s, int64_t c[4]) {
    if (!s || !c) return ABD_E_INVALID;
    c[0] = s->nb; c[1] = s->V; c[2] = s->T; c[3] = s->E;
    return ABD_OK;
}

extern "C" int abd_body_props(const abd_scene *s, int32_t b, double *m, double com[3], double S[9], double *V) {
    if (!s || b < 0 || b >= s->nb) return ABD_E_INVALID;
    if (m) *m = s->mass[b];
    if (com) for (int k = 0; k < 3; ++k) com[k] = s->com[3 * (size_t)b + k];
    if (S) for (int k = 0; k < 9; ++k) S[k] = s->S[9 * (size_t)b + k];
    if (V) *V = s->vol[b];
    return ABD_OK;
}

extern "C" int abd_partition(abd_scene *s, const abd_partition_desc *d) {
    if (!s || !d || d->n_slabs < 1 || d->n_slabs > kMaxSlabs || d->axis < 0 || d->axis > 2)
        return set_err(s, ABD_E_INVALID, "abd_partition: n_slabs must be 1..64 and axis 0..2");
    if (!s->group.empty())
        return set_err(s, ABD_E_INVALID, "abd_partition: a batched world is partitioned by its scenes");
    s->axis = d->axis;
    s->n_slabs = d->n_slabs;
    s->slab_planes.clear();
    if (d->planes)
        for (int i = 0; i + 1 < d->n_slabs; ++i) s->slab_planes.push_back(d->planes[i]);
    s->alpha_w = d->alpha;
    s->w_min = d->w_min;
    s->pd_kp = d->pd_kp;
    s->pd_kd = d->pd_kd;
    s->pd_smooth = d->pd_smooth;
    s->pd_tau.clear();
    s->pd_T.clear();
    s->last_planes.clear();
    return ABD_OK;
}

extern "C" int abd_scene_broadphase(abd_scene *s, int32_t mode) {
    if (!s || mode < 0 || mode > 2) return ABD_E_INVALID;
    s->bp_mode = mode;
    ++s->w.gen;  // the next world picks its level-1 pass anew
    return ABD_OK;
}

extern "C" int abd_scene_reserve(abd_scene *s, int64_t pairs) {
    if (!s || pairs < 0) return ABD_E_INVALID;
    int64_t n = std::max<int64_t>(pairs, 16);
    World &w = s->w;
    w.cap_cand = w.cap_act = w.cap_ls = n;
    w.cap_cp = 4 * n;
    ++w.gen;  // buffers are re-sized at the next step; captured graphs go stale
    return ABD_OK;
}

extern "C" int abd_partition_planes(const abd_scene *s, double *planes, int32_t cap, int32_t *n) {
    if (!s || !n || cap < 0) return ABD_E_INVALID;
    const std::vector<double> &src = s->slab_planes.size() == (size_t)std::max(0, s->n_slabs - 1) && s->n_slabs > 1
                                         ? s->slab_planes
                                         : s->last_planes;
    *n = (int32_t)src.size();
    if (planes)
        for (int i = 0; i < std::min((int)src.size(), (int)cap); ++i) planes[i] = src[i];
    return ABD_OK;
}

extern "C" int abd_pd_update(int32_t n_slabs, const double *tau, const double *T_prev, double kp, double kd,
                             double *delta, double *T) {
    if (n_slabs < 1 || !tau || (n_slabs > 1 && (!delta || !T))) return ABD_E_INVALID;
    for (int i = 0; i + 1 < n_slabs; ++i) {
        // (eta - 1) / (eta + 1) with eta = tau_i / tau_{i+1}, written without the quotient
        double sum = tau[i] + tau[i + 1];
        T[i] = sum > 0.0 ? (tau[i] - tau[i + 1]) / sum : 0.0;
        double tp = T_prev ? T_prev[i] : 0.0;
        delta[i] = -(kp * T[i] + kd * (T[i] - tp));
    }
    return ABD_OK;
}

extern "C" int abd_state_get(const abd_scene *s, double *q, double *v, int64_t n) {
    if (!s || n != s->nb) return ABD_E_INVALID;
    abd_scene *ms = const_cast<abd_scene *>(s);
    if (q && cudaMemcpyAsync(q, s->dev.q.p, 96 * (size_t)n, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
        return cuda_check(ms, cudaGetLastError(), "state_get");
    if (v && cudaMemcpyAsync(v, s->dev.v.p, 96 * (size_t)n, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
        return cuda_check(ms, cudaGetLastError(), "state_get");
    return cuda_check(ms, cudaStreamSynchronize(s->stream), "state_get");
}

extern "C" int abd_state_set(abd_scene *s, const double *q, const double *v, int64_t n) {
    if (!s || n != s->nb) return ABD_E_INVALID;
    if (q && cudaMemcpyAsync(s->dev.q.p, q, 96 * (size_t)n, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return cuda_check(s, cudaGetLastError(), "state_set");
    if (v && cudaMemcpyAsync(s->dev.v.p, v, 96 * (size_t)n, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return cuda_check(s, cudaGetLastError(), "state_set");
    return cuda_check(s, cudaStreamSynchronize(s->stream), "state_set");
}

extern "C" int abd_state_device(abd_scene *s, double **q, double **v) {
    if (!s) return ABD_E_INVALID;
    if (q) *q = (double *)s->dev.q.p;
    if (v) *v = (double *)s->dev.v.p;
    return ABD_OK;
}

extern "C" int abd_profile(abd_scene *s, int32_t enable) {
    if (!s) return ABD_E_INVALID;
    s->prof = enable != 0;
    if (!enable) s->kstats.clear();
    return ABD_OK;
}

extern "C" int abd_kernel_stats(const abd_scene *s, const char *name, int64_t *launches, double *ms, double *bytes) {
    if (!s || !name) return ABD_E_INVALID;
    for (auto &k : s->kstats)
        if (k.name == name) {
            if (launches) *launches = k.launches;
            if (ms) *ms = k.ms;
            if (bytes) *bytes = k.bytes;
            return ABD_OK;
        }
    if (launches) *launches = 0;
    if (ms) *ms = 0;
    if (bytes) *bytes = 0;
    return ABD_OK;
}

extern "C" abd_step_params abd_step_params_default(void) {
    abd_step_params p;
    p.h = 1e-2; p.dhat = 1e-3; p.kappa_barrier = 0.0;
    p.precision = ABD_FP64; p.rho_mode = ABD_RHO_ADAPTIVE;
    p.beta = 1.0; p.tau = 2.0; p.mu = 5.0; p.sigma_min = 1e-3; p.sigma_max = 1e3;
    p.theta = 1e-3; p.newton_tol = 1e-6;
    p.max_admm = 200; p.max_newton = 100; p.max_halvings = 40;
    p.pcg_rtol = 1e-12; p.pcg_max = 5000;
    p.accd_s = 0.1; p.accd_c = 0.9;
    p.dt_split_max = 0;
    p.mixed_fp64_first = 1;
    return p;
}

extern "C" const char *abd_status_string(int c) {
    switch (c) {
        case ABD_OK: return "ok";
        case ABD_ADMM_MAXITER: return "ADMM reached max_admm; merge check passed";
        case ABD_NEWTON_MAXITER: return "a local solve reached max_newton";
        case ABD_FELL_BACK_MONOLITHIC: return "ADMM did not converge; step re-solved on one partition";
        case ABD_DT_SPLIT: return "merge blocked; step taken as two half steps";
        case ABD_E_INVALID: return "invalid argument";
        case ABD_E_OOM: return "out of device memory";
        case ABD_E_CUDA: return "CUDA error";
        case ABD_E_PAIR_OVERFLOW: return "pair buffer overflow";
        case ABD_E_DEVICE_TIMEOUT: return "device-side wait timed out";
        case ABD_E_PENETRATION: return "penetration detected";
        case ABD_E_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

extern "C" const char *abd_last_error(const abd_scene *s) { return s ? s->err.c_str() : "null scene"; }

// ---------------------------------------------------------------------------
// Batched world: many independent scenes in one scene object, one partition
// per scene, every Newton phase of every scene in the same launches.
// ---------------------------------------------------------------------------
extern "C" int abd_scene_create_batch(const abd_scene_desc *descs, int32_t n, void *stream, abd_scene **out) {
    if (!descs || !out || n < 1 || n > kMaxParts) return ABD_E_INVALID;
    *out = nullptr;
    const abd_scene_desc &d0 = descs[0];
    std::vector<int32_t> mnv, mnt, bmesh, bkind, tris;
    std::vector<double> xbar, dens, kap, q0, v0, om;
    std::vector<int> group;
    std::vector<int64_t> goff(1, 0);
    int64_t nbt = 0;
    for (int i = 0; i < n; ++i) {
        const abd_scene_desc &d = descs[i];
        if (d.n_bodies <= 0 || d.n_meshes <= 0 || !d.mesh_n_verts || !d.mesh_n_tris || !d.mesh_xbar ||
            !d.mesh_tris || !d.body_mesh || !d.body_density || !d.body_kappa || !d.body_kind || !d.body_q0)
            return ABD_E_INVALID;
        // one set of ground planes and one gravity for the whole world
        if (d.n_planes != d0.n_planes) return ABD_E_INVALID;
        for (int k = 0; k < d.n_planes; ++k)
            if (d.plane_axis[k] != d0.plane_axis[k] || d.plane_sign[k] != d0.plane_sign[k] ||
                d.plane_offset[k] != d0.plane_offset[k])
                return ABD_E_INVALID;
        for (int k = 0; k < 3; ++k)
            if (d.gravity[k] != d0.gravity[k]) return ABD_E_INVALID;
        const int mesh_base = (int)mnv.size();
        int64_t nvt = 0, ntt = 0;
        for (int m = 0; m < d.n_meshes; ++m) {
            if (d.mesh_n_verts[m] <= 0 || d.mesh_n_tris[m] < 0) return ABD_E_INVALID;
            mnv.push_back(d.mesh_n_verts[m]);
            mnt.push_back(d.mesh_n_tris[m]);
            nvt += d.mesh_n_verts[m];
            ntt += d.mesh_n_tris[m];
        }
        xbar.insert(xbar.end(), d.mesh_xbar, d.mesh_xbar + 3 * nvt);
        tris.insert(tris.end(), d.mesh_tris, d.mesh_tris + 3 * ntt);
        for (int b = 0; b < d.n_bodies; ++b) {
            if (d.body_mesh[b] < 0 || d.body_mesh[b] >= d.n_meshes) return ABD_E_INVALID;
            bmesh.push_back(mesh_base + d.body_mesh[b]);
            bkind.push_back(d.body_kind[b]);
            dens.push_back(d.body_density[b]);
            kap.push_back(d.body_kappa[b]);
            for (int k = 0; k < 12; ++k) {
                q0.push_back(d.body_q0[12 * (size_t)b + k]);
                v0.push_back(d.body_v0 ? d.body_v0[12 * (size_t)b + k] : 0.0);
            }
            for (int k = 0; k < 3; ++k) om.push_back(d.body_omega ? d.body_omega[3 * (size_t)b + k] : 0.0);
            group.push_back(i);
        }
        nbt += d.n_bodies;
        if (nbt >= (1ll << 31)) return ABD_E_INVALID;
        goff.push_back(nbt);
    }
    abd_scene_desc D = d0;
    D.n_meshes = (int32_t)mnv.size();
    D.mesh_n_verts = mnv.data();
    D.mesh_n_tris = mnt.data();
    D.mesh_xbar = xbar.data();
    D.mesh_tris = tris.data();
    D.n_bodies = (int32_t)nbt;
    D.body_mesh = bmesh.data();
    D.body_density = dens.data();
    D.body_kappa = kap.data();
    D.body_kind = bkind.data();
    D.body_q0 = q0.data();
    D.body_v0 = v0.data();
    D.body_omega = om.data();
    int rc = abd_scene_create(&D, stream, out);
    if (rc) return rc;
    (*out)->group = std::move(group);
    (*out)->group_off = std::move(goff);
    return ABD_OK;
}

extern "C" int abd_batch_layout(const abd_scene *s, int64_t *body_off, int32_t cap, int32_t *n) {
    if (!s || !n || cap < 0) return ABD_E_INVALID;
    if (s->group.empty()) {
        *n = 1;
        if (body_off && cap >= 2) { body_off[0] = 0; body_off[1] = s->nb; }
        return ABD_OK;
    }
    *n = (int32_t)s->group_off.size() - 1;
    if (body_off)
        for (int i = 0; i < std::min<int>((int)s->group_off.size(), cap); ++i) body_off[i] = s->group_off[i];
    return ABD_OK;
}
