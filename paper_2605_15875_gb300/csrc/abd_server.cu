// abd_server.cu -- serving many independent scenes on one GPU.
//
// A fixed pool of worker threads, each with its own CUDA stream, takes
// requests in FIFO order.  A request is admitted when its estimated device
// memory fits what is left of the HBM budget (the first admissible request
// waits rather than being overtaken, so a large scene is not starved; a
// request larger than the whole budget runs once nothing else holds memory).
// An ephemeral request's worker creates the scene on its stream, partitions
// it, advances it with abd_step, reads the final state into server-owned host
// memory and frees the scene.  A keyed request advances a resident scene
// instead: the scene (its state and its device workspace and contact lists)
// stays on the device between the requests of its key, on a stream of its
// own, until it is released or evicted to make room (its state then waits in
// host memory and the scene is rebuilt at its next request).  Work of
// different workers overlaps on the device; each request's arithmetic is
// exactly abd_step's on its own scene.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/abd.h"

namespace abd {
// abd_scene.cu: run the scene's iterations on its own stream only (no side
// branch for independent kernels)
void scene_no_side(abd_scene *s);
}  // namespace abd

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Deep copy of a scene description and its partition (the caller's arrays
// may be freed once submit returns).
struct OwnedScene {
    std::vector<int32_t> mesh_n_verts, mesh_n_tris, mesh_tris, body_mesh, body_kind, plane_axis;
    std::vector<double> mesh_xbar, body_density, body_kappa, body_q0, body_v0, body_omega, plane_sign, plane_offset,
        planes;
    abd_scene_desc d{};
    abd_partition_desc p{};
    bool has_part = false;

    template <class T>
    static void take(std::vector<T> &dst, const T *src, size_t n) {
        if (src) dst.assign(src, src + n);
        else dst.clear();
    }

    int copy(const abd_scene_desc *s, const abd_partition_desc *part) {
        if (!s || s->n_meshes < 1 || s->n_bodies < 1 || !s->mesh_n_verts || !s->mesh_n_tris || !s->mesh_xbar ||
            !s->mesh_tris || !s->body_mesh || !s->body_density || !s->body_kappa || !s->body_kind || !s->body_q0 ||
            s->n_planes < 0)
            return ABD_E_INVALID;
        size_t V = 0, T = 0;
        for (int m = 0; m < s->n_meshes; ++m) {
            if (s->mesh_n_verts[m] < 0 || s->mesh_n_tris[m] < 0) return ABD_E_INVALID;
            V += (size_t)s->mesh_n_verts[m];
            T += (size_t)s->mesh_n_tris[m];
        }
        size_t B = (size_t)s->n_bodies, P = (size_t)s->n_planes;
        for (size_t b = 0; b < B; ++b)
            if (s->body_mesh[b] < 0 || s->body_mesh[b] >= s->n_meshes) return ABD_E_INVALID;
        take(mesh_n_verts, s->mesh_n_verts, s->n_meshes);
        take(mesh_n_tris, s->mesh_n_tris, s->n_meshes);
        take(mesh_xbar, s->mesh_xbar, 3 * V);
        take(mesh_tris, s->mesh_tris, 3 * T);
        take(body_mesh, s->body_mesh, B);
        take(body_density, s->body_density, B);
        take(body_kappa, s->body_kappa, B);
        take(body_kind, s->body_kind, B);
        take(body_q0, s->body_q0, 12 * B);
        take(body_v0, s->body_v0, 12 * B);
        take(body_omega, s->body_omega, 3 * B);
        if (P && (!s->plane_axis || !s->plane_sign || !s->plane_offset)) return ABD_E_INVALID;
        take(plane_axis, s->plane_axis, P);
        take(plane_sign, s->plane_sign, P);
        take(plane_offset, s->plane_offset, P);
        d = *s;
        d.mesh_n_verts = mesh_n_verts.data();
        d.mesh_n_tris = mesh_n_tris.data();
        d.mesh_xbar = mesh_xbar.data();
        d.mesh_tris = mesh_tris.data();
        d.body_mesh = body_mesh.data();
        d.body_density = body_density.data();
        d.body_kappa = body_kappa.data();
        d.body_kind = body_kind.data();
        d.body_q0 = body_q0.data();
        d.body_v0 = body_v0.empty() ? nullptr : body_v0.data();
        d.body_omega = body_omega.empty() ? nullptr : body_omega.data();
        d.plane_axis = P ? plane_axis.data() : nullptr;
        d.plane_sign = P ? plane_sign.data() : nullptr;
        d.plane_offset = P ? plane_offset.data() : nullptr;
        if (part) {
            if (part->n_slabs < 1) return ABD_E_INVALID;
            has_part = true;
            p = *part;
            if (part->planes && part->n_slabs > 1) {
                planes.assign(part->planes, part->planes + (part->n_slabs - 1));
                p.planes = planes.data();
            } else {
                p.planes = nullptr;
            }
        }
        return ABD_OK;
    }

    // Device memory estimate used for admission: per-vertex positions and
    // bounds (two configurations), per-body and per-slot state, and the
    // initial pair-list capacities.
    int64_t estimate() const {
        int64_t V = 0, T = 0;
        for (int32_t b : body_mesh) {
            V += mesh_n_verts[b];
            T += mesh_n_tris[b];
        }
        int64_t B = (int64_t)body_mesh.size();
        int slabs = has_part ? p.n_slabs : 1;
        return (int64_t(48) << 20) + 160 * V + 80 * T + 4096 * B * (slabs > 1 ? 2 : 1);
    }
};

// A scene kept on the device across the requests of one key.
struct Resident {
    int64_t key = 0;
    OwnedScene scene;            // description, for rebuilding after an eviction
    abd_scene *sc = nullptr;     // null while evicted (or before the first request)
    cudaStream_t st = nullptr;
    std::vector<double> q, v;    // host state while evicted
    int64_t est = 0;             // admission estimate, held while resident
    bool busy = false;           // a request of the key is running
    int pending = 0;             // requests of the key queued or running
    bool released = false;       // release asked: freed once the last request is done
    double last_used = 0.0;
};

struct Request {
    int64_t ticket = 0;
    int64_t key = 0;             // 0: ephemeral scene
    OwnedScene scene;
    abd_step_params params{};
    int n_steps = 0;
    abd_request_info info{};
    double t_submit = 0.0, t_admit = 0.0;
    std::vector<double> q, v, lat;
    std::string err;
};

}  // namespace

struct abd_server {
    abd_server_desc desc{};
    int64_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::map<int64_t, std::unique_ptr<Resident>> residents;
    std::vector<std::thread> workers;
    int64_t next_ticket = 1;
    int running = 0;
    bool stop = false;

    // Evict the least recently used idle resident scene other than `keep`
    // (its state goes to host memory, the scene is freed).  Under the lock.
    bool evict_one(const Resident *keep) {
        Resident *v = nullptr;
        for (auto &kv : residents) {
            Resident *c = kv.second.get();
            if (c == keep || c->busy || !c->sc) continue;
            if (!v || c->last_used < v->last_used) v = c;
        }
        if (!v) return false;
        size_t B = v->scene.body_mesh.size();
        v->q.assign(12 * B, 0.0);
        v->v.assign(12 * B, 0.0);
        if (abd_state_get(v->sc, v->q.data(), v->v.data(), (int64_t)B) < 0) v->q.clear();
        abd_scene_destroy(v->sc);
        v->sc = nullptr;
        used -= v->est;
        return true;
    }

    // Free a released resident scene once nothing of its key is pending.  Under the lock.
    void reap(int64_t key) {
        auto it = residents.find(key);
        if (it == residents.end()) return;
        Resident *res = it->second.get();
        if (!res->released || res->pending > 0 || res->busy) return;
        if (res->sc) {
            abd_scene_destroy(res->sc);
            used -= res->est;
        }
        if (res->st) cudaStreamDestroy(res->st);
        residents.erase(it);
    }

    // Admission under the lock: the first queued request whose key has no
    // request running runs when its memory fits the budget -- after evicting
    // idle resident scenes, least recently used first, if that makes room --
    // or when nothing else holds memory; otherwise it waits, and so does
    // everything behind it.  A resident scene on the device needs nothing.
    Request *admit(int64_t &held) {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            Request *h = reqs[*it].get();
            Resident *res = h->key ? residents[h->key].get() : nullptr;
            if (res && res->busy) continue;
            int64_t need = res ? (res->sc ? 0 : res->est) : h->info.est_bytes;
            while (used + need > budget && evict_one(res)) {
            }
            if (used + need > budget && used > 0) return nullptr;
            queue.erase(it);
            used += need;
            held = need;
            ++running;
            if (res) res->busy = true;
            h->info.state = ABD_REQ_RUNNING;
            h->t_admit = now_ms();
            h->info.queue_ms = h->t_admit - h->t_submit;
            return h;
        }
        return nullptr;
    }

    void worker_main() {
        cudaSetDevice(desc.device);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        for (;;) {
            Request *r = nullptr;
            Resident *res = nullptr;
            abd_request_info inf{};
            int64_t held = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    r = admit(held);
                    if (r || (stop && queue.empty())) break;
                    cv_work.wait(lk);
                }
                if (!r) break;
                inf = r->info;
                if (r->key) res = residents[r->key].get();
            }
            if (res) run_resident(r, res, inf);
            else run(r, st, inf);
            {
                std::lock_guard<std::mutex> lk(mu);
                if (res) {
                    if (!res->sc) used -= held;  // the scene could not be built: nothing stays resident
                    res->busy = false;
                    res->last_used = now_ms();
                    --res->pending;
                    reap(r->key);
                } else {
                    used -= held;
                }
                --running;
                inf.state = ABD_REQ_DONE;
                r->info = inf;
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
        if (st) cudaStreamDestroy(st);
    }

    // Steps, state read-back and latency percentiles of a request on scene sc.
    static void steps_on(Request *r, abd_scene *sc, abd_request_info &inf) {
        r->lat.reserve(r->n_steps);
        for (int k = 0; k < r->n_steps; ++k) {
            double t0 = now_ms();
            abd_step_stats stats{};
            int s = abd_step(sc, &r->params, &stats);
            r->lat.push_back(now_ms() - t0);
            inf.last = stats;
            if (s < 0) {
                inf.status = s;
                r->err = abd_last_error(sc);
                break;
            }
            if (s > inf.status) inf.status = s;
            ++inf.steps_done;
        }
        size_t B = (size_t)inf.n_bodies;
        r->q.assign(12 * B, 0.0);
        r->v.assign(12 * B, 0.0);
        int g = abd_state_get(sc, r->q.data(), r->v.data(), (int64_t)B);
        if (g < 0 && inf.status >= 0) {
            inf.status = g;
            r->err = abd_last_error(sc);
        }
    }

    static void finish(Request *r, abd_request_info &inf) {
        if (!r->lat.empty()) {
            std::vector<double> t = r->lat;
            std::sort(t.begin(), t.end());
            auto pct = [&](double f) { return t[std::min(t.size() - 1, (size_t)(f * (t.size() - 1) + 0.5))]; };
            inf.step_ms_p50 = pct(0.50);
            inf.step_ms_p99 = pct(0.99);
        }
        inf.run_ms = now_ms() - r->t_admit;
    }

    // Runs without the lock: works on `inf` (published when done) and on the
    // request's result vectors, which readers touch only once it is done.
    static void run(Request *r, cudaStream_t st, abd_request_info &inf) {
        abd_scene *sc = nullptr;
        int rc = abd_scene_create(&r->scene.d, (void *)st, &sc);
        if (rc < 0) {
            inf.status = rc;
            r->err = "scene create failed";
        } else {
            abd::scene_no_side(sc);  // the workers' streams already run side by side
        }
        if (rc >= 0 && r->scene.has_part) {
            rc = abd_partition(sc, &r->scene.p);
            if (rc < 0) {
                inf.status = rc;
                r->err = abd_last_error(sc);
            }
        }
        if (rc >= 0) steps_on(r, sc, inf);
        if (sc) abd_scene_destroy(sc);
        finish(r, inf);
    }

    // A keyed request: the resident scene is built on first use (or after an
    // eviction, from its description and the state kept on the host) on a
    // stream of its own, advanced, and left on the device.  Only this worker
    // touches `res` while its busy flag is set.
    static void run_resident(Request *r, Resident *res, abd_request_info &inf) {
        int rc = ABD_OK;
        if (!res->sc) {
            if (!res->st && cudaStreamCreateWithFlags(&res->st, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                res->st = nullptr;
            }
            rc = abd_scene_create(&res->scene.d, (void *)res->st, &res->sc);
            if (rc < 0) {
                res->sc = nullptr;
                r->err = "scene create failed";
            } else {
                abd::scene_no_side(res->sc);
            }
            if (rc >= 0 && res->scene.has_part && (rc = abd_partition(res->sc, &res->scene.p)) < 0)
                r->err = abd_last_error(res->sc);
            if (rc >= 0 && !res->q.empty()) {
                rc = abd_state_set(res->sc, res->q.data(), res->v.data(), (int64_t)res->scene.body_mesh.size());
                if (rc < 0) r->err = abd_last_error(res->sc);
            }
            if (rc < 0) {
                inf.status = rc;
                if (res->sc) abd_scene_destroy(res->sc);
                res->sc = nullptr;
            }
        }
        if (rc >= 0) steps_on(r, res->sc, inf);
        finish(r, inf);
    }
};

extern "C" int abd_server_create(const abd_server_desc *desc, abd_server **out) {
    if (!desc || !out || desc->n_streams < 1 || desc->hbm_budget_bytes < 0) return ABD_E_INVALID;
    *out = nullptr;
    if (cudaSetDevice(desc->device) != cudaSuccess) {
        cudaGetLastError();
        return ABD_E_CUDA;
    }
    auto *s = new abd_server();
    s->desc = *desc;
    s->budget = desc->hbm_budget_bytes;
    if (s->budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return ABD_E_CUDA;
        }
        s->budget = (int64_t)(0.8 * (double)fr);
    }
    for (int i = 0; i < desc->n_streams; ++i) s->workers.emplace_back([s] { s->worker_main(); });
    *out = s;
    return ABD_OK;
}

extern "C" int abd_server_submit(abd_server *srv, const abd_scene_desc *scene, const abd_partition_desc *part,
                                 const abd_step_params *params, int32_t n_steps, int64_t *ticket) {
    if (!srv || !scene || !ticket || n_steps < 0) return ABD_E_INVALID;
    auto r = std::make_unique<Request>();
    int rc = r->scene.copy(scene, part);
    if (rc) return rc;
    r->params = params ? *params : abd_step_params_default();
    r->n_steps = n_steps;
    r->info.state = ABD_REQ_QUEUED;
    r->info.n_bodies = scene->n_bodies;
    r->info.est_bytes = r->scene.estimate();
    r->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return ABD_E_INVALID;
        r->ticket = srv->next_ticket++;
        *ticket = r->ticket;
        srv->queue.push_back(r->ticket);
        srv->reqs[r->ticket] = std::move(r);
    }
    srv->cv_work.notify_one();
    return ABD_OK;
}

extern "C" int abd_server_submit_keyed(abd_server *srv, int64_t key, const abd_scene_desc *scene,
                                       const abd_partition_desc *part, const abd_step_params *params, int32_t n_steps,
                                       int64_t *ticket) {
    if (!srv || !ticket || n_steps < 0 || key == 0) return ABD_E_INVALID;
    auto r = std::make_unique<Request>();
    r->key = key;
    std::unique_ptr<Resident> fresh;
    if (scene) {
        fresh = std::make_unique<Resident>();
        fresh->key = key;
        int rc = fresh->scene.copy(scene, part);
        if (rc) return rc;
        fresh->est = fresh->scene.estimate();
    }
    r->params = params ? *params : abd_step_params_default();
    r->n_steps = n_steps;
    r->info.state = ABD_REQ_QUEUED;
    r->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return ABD_E_INVALID;
        auto it = srv->residents.find(key);
        if (it == srv->residents.end()) {
            if (!fresh) return ABD_E_INVALID;  // the first request of a key describes its scene
            it = srv->residents.emplace(key, std::move(fresh)).first;
        } else if (fresh || it->second->released) {
            return ABD_E_INVALID;  // a key names one scene until it is released and freed
        }
        Resident *res = it->second.get();
        ++res->pending;
        r->info.n_bodies = (int32_t)res->scene.body_mesh.size();
        r->info.est_bytes = res->est;
        r->ticket = srv->next_ticket++;
        *ticket = r->ticket;
        srv->queue.push_back(r->ticket);
        srv->reqs[r->ticket] = std::move(r);
    }
    srv->cv_work.notify_one();
    return ABD_OK;
}

extern "C" int abd_server_release(abd_server *srv, int64_t key) {
    if (!srv) return ABD_E_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->residents.find(key);
    if (it == srv->residents.end() || it->second->released) return ABD_E_INVALID;
    it->second->released = true;
    srv->reap(key);
    return ABD_OK;
}

extern "C" int abd_server_poll(abd_server *srv, int64_t ticket, abd_request_info *info) {
    if (!srv || !info) return ABD_E_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return ABD_E_INVALID;
    *info = it->second->info;
    return ABD_OK;
}

extern "C" int abd_server_wait(abd_server *srv, int64_t ticket, abd_request_info *info) {
    if (!srv || !info) return ABD_E_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return ABD_E_INVALID;
    Request *r = it->second.get();
    srv->cv_done.wait(lk, [r] { return r->info.state == ABD_REQ_DONE; });
    *info = r->info;
    return ABD_OK;
}

extern "C" int abd_server_result(abd_server *srv, int64_t ticket, double *q, double *v, int64_t n_bodies) {
    if (!srv) return ABD_E_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return ABD_E_INVALID;
    Request *r = it->second.get();
    if (r->info.state != ABD_REQ_DONE) return ABD_E_INVALID;
    if (r->info.status < 0 && r->q.empty()) return r->info.status;
    if (n_bodies != (int64_t)r->info.n_bodies) return ABD_E_INVALID;
    if (q) std::memcpy(q, r->q.data(), sizeof(double) * r->q.size());
    if (v) std::memcpy(v, r->v.data(), sizeof(double) * r->v.size());
    return r->info.status < 0 ? r->info.status : ABD_OK;
}

extern "C" int abd_server_latencies(abd_server *srv, int64_t ticket, double *ms, int32_t cap, int32_t *n) {
    if (!srv || !n || cap < 0) return ABD_E_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return ABD_E_INVALID;
    Request *r = it->second.get();
    if (r->info.state != ABD_REQ_DONE) return ABD_E_INVALID;
    int k = (int)r->lat.size();
    if (ms)
        for (int i = 0; i < std::min(k, (int)cap); ++i) ms[i] = r->lat[i];
    *n = k;
    return ABD_OK;
}

extern "C" const char *abd_server_error(abd_server *srv, int64_t ticket) {
    if (!srv) return "";
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return "unknown ticket";
    if (it->second->info.state != ABD_REQ_DONE) return "";
    return it->second->err.c_str();
}

extern "C" void abd_server_destroy(abd_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->workers) t.join();
    cudaSetDevice(srv->desc.device);
    for (auto &kv : srv->residents) {
        if (kv.second->sc) abd_scene_destroy(kv.second->sc);
        if (kv.second->st) cudaStreamDestroy(kv.second->st);
    }
    delete srv;
}
