"""Python binding of the C ABI in include/abd.h (argument marshalling only).

Every step of the method runs inside libabd.so's CUDA kernels; this module
only converts numpy arrays and Python values to the C structs.  It raises
when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libabd.so")

DYNAMIC, STATIC, KINEMATIC = 0, 1, 2
FP64, MIXED = 0, 1
RHO_FIXED, RHO_ADAPTIVE = 0, 1
OK, ADMM_MAXITER, NEWTON_MAXITER, FELL_BACK_MONOLITHIC, DT_SPLIT = 0, 1, 2, 3, 4


class SceneDesc(C.Structure):
    _fields_ = [("n_meshes", C.c_int32), ("mesh_n_verts", C.c_void_p), ("mesh_n_tris", C.c_void_p),
                ("mesh_xbar", C.c_void_p), ("mesh_tris", C.c_void_p), ("n_bodies", C.c_int32),
                ("body_mesh", C.c_void_p), ("body_density", C.c_void_p), ("body_kappa", C.c_void_p),
                ("body_kind", C.c_void_p), ("body_q0", C.c_void_p), ("body_v0", C.c_void_p),
                ("body_omega", C.c_void_p),
                ("n_planes", C.c_int32), ("plane_axis", C.c_void_p), ("plane_sign", C.c_void_p),
                ("plane_offset", C.c_void_p), ("gravity", C.c_double * 3)]


class PartitionDesc(C.Structure):
    _fields_ = [("axis", C.c_int32), ("n_slabs", C.c_int32), ("planes", C.c_void_p), ("alpha", C.c_double),
                ("w_min", C.c_double), ("pd_kp", C.c_double), ("pd_kd", C.c_double), ("pd_smooth", C.c_double)]


class StepParams(C.Structure):
    _fields_ = [("h", C.c_double), ("dhat", C.c_double), ("kappa_barrier", C.c_double),
                ("precision", C.c_int32), ("rho_mode", C.c_int32), ("beta", C.c_double), ("tau", C.c_double),
                ("mu", C.c_double), ("sigma_min", C.c_double), ("sigma_max", C.c_double), ("theta", C.c_double),
                ("newton_tol", C.c_double), ("max_admm", C.c_int32), ("max_newton", C.c_int32),
                ("max_halvings", C.c_int32), ("pcg_rtol", C.c_double), ("pcg_max", C.c_int32),
                ("accd_s", C.c_double), ("accd_c", C.c_double), ("dt_split_max", C.c_int32),
                ("mixed_fp64_first", C.c_int32)]


class StepStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("admm_iters", C.c_int32), ("newton_iters", C.c_int32),
                ("n_partitions", C.c_int32), ("n_shared", C.c_int32), ("n_slots", C.c_int32),
                ("pcg_iters", C.c_int64), ("n_candidates_peak", C.c_int64), ("n_active_peak", C.c_int64),
                ("r_inf", C.c_double), ("s_inf", C.c_double), ("delta_inf", C.c_double),
                ("min_distance", C.c_double), ("l", C.c_double), ("kappa_barrier", C.c_double), ("w", C.c_double),
                ("t_solve_ms", C.c_double), ("t_coll_ms", C.c_double), ("t_sync_ms", C.c_double),
                ("t_total_ms", C.c_double), ("kernel_launches", C.c_int64), ("pcg_cluster", C.c_int32),
                ("pcg_unstaged", C.c_int32), ("list_redo", C.c_int32), ("reserved0", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerDesc(C.Structure):
    _fields_ = [("device", C.c_int32), ("n_streams", C.c_int32), ("hbm_budget_bytes", C.c_int64)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE = 0, 1, 2


class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("steps_done", C.c_int32), ("n_bodies", C.c_int32),
                ("est_bytes", C.c_int64), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("step_ms_p50", C.c_double), ("step_ms_p99", C.c_double), ("last", StepStats)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "last"}
        d["last"] = self.last.as_dict()
        return d


# every symbol declared in include/abd.h
EXPORTS = ["abd_scene_create", "abd_scene_destroy", "abd_scene_counts", "abd_body_props", "abd_partition",
           "abd_partition_masks", "abd_step", "abd_state_get", "abd_state_set", "abd_state_device",
           "abd_candidates", "abd_profile", "abd_kernel_stats", "abd_step_params_default", "abd_status_string",
           "abd_last_error", "abd_candidates_noalloc", "abd_partition_get", "abd_server_create",
           "abd_server_submit", "abd_server_poll", "abd_server_wait", "abd_server_result", "abd_server_latencies",
           "abd_server_error", "abd_server_destroy", "abd_partition_planes", "abd_pd_update", "abd_scene_reserve",
           "abd_scene_create_batch", "abd_batch_layout", "abd_partition_newton",
           "abd_server_submit_keyed", "abd_server_release", "abd_scene_broadphase"]

_lib = None


def load(path: Optional[str] = None):
    """Load libabd.so (raises when it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libabd.so not found at {p}: build it with paper_2605_15875_gb300.build.build()")
    L = C.CDLL(p)
    vp, i64 = C.c_void_p, C.c_int64
    L.abd_scene_create.argtypes = [C.POINTER(SceneDesc), vp, C.POINTER(vp)]
    L.abd_scene_destroy.argtypes = [vp]
    L.abd_scene_destroy.restype = None
    L.abd_scene_counts.argtypes = [vp, vp]
    L.abd_body_props.argtypes = [vp, C.c_int32, vp, vp, vp, vp]
    L.abd_partition.argtypes = [vp, C.POINTER(PartitionDesc)]
    L.abd_partition_masks.argtypes = [vp, C.c_double, vp, vp]
    L.abd_step.argtypes = [vp, C.POINTER(StepParams), C.POINTER(StepStats)]
    L.abd_state_get.argtypes = [vp, vp, vp, i64]
    L.abd_state_set.argtypes = [vp, vp, vp, i64]
    L.abd_state_device.argtypes = [vp, C.POINTER(vp), C.POINTER(vp)]
    L.abd_candidates.argtypes = [vp, vp, vp, C.c_double, vp, i64, C.POINTER(i64)]
    L.abd_candidates_noalloc.argtypes = [vp, vp, vp, C.c_double, vp, i64, C.POINTER(i64)]
    L.abd_profile.argtypes = [vp, C.c_int32]
    L.abd_kernel_stats.argtypes = [vp, C.c_char_p, C.POINTER(i64), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.abd_step_params_default.argtypes = []
    L.abd_step_params_default.restype = StepParams
    L.abd_status_string.argtypes = [C.c_int]
    L.abd_status_string.restype = C.c_char_p
    L.abd_last_error.argtypes = [vp]
    L.abd_last_error.restype = C.c_char_p
    i32p = C.POINTER(C.c_int32)
    L.abd_partition_get.argtypes = [vp, C.c_int32, vp, C.c_int32, i32p, vp, C.c_int32, i32p]
    L.abd_partition_planes.argtypes = [vp, vp, C.c_int32, i32p]
    L.abd_scene_reserve.argtypes = [vp, i64]
    L.abd_scene_broadphase.argtypes = [vp, C.c_int32]
    L.abd_scene_create_batch.argtypes = [vp, C.c_int32, vp, C.POINTER(vp)]
    L.abd_batch_layout.argtypes = [vp, vp, C.c_int32, i32p]
    L.abd_partition_newton.argtypes = [vp, vp, C.c_int32, i32p]
    L.abd_pd_update.argtypes = [C.c_int32, vp, vp, C.c_double, C.c_double, vp, vp]
    L.abd_server_create.argtypes = [C.POINTER(ServerDesc), C.POINTER(vp)]
    L.abd_server_submit.argtypes = [vp, C.POINTER(SceneDesc), vp, vp, C.c_int32, C.POINTER(i64)]
    L.abd_server_submit_keyed.argtypes = [vp, i64, vp, vp, vp, C.c_int32, C.POINTER(i64)]
    L.abd_server_release.argtypes = [vp, i64]
    L.abd_server_poll.argtypes = [vp, i64, C.POINTER(RequestInfo)]
    L.abd_server_wait.argtypes = [vp, i64, C.POINTER(RequestInfo)]
    L.abd_server_result.argtypes = [vp, i64, vp, vp, i64]
    L.abd_server_latencies.argtypes = [vp, i64, vp, C.c_int32, i32p]
    L.abd_server_error.argtypes = [vp, i64]
    L.abd_server_error.restype = C.c_char_p
    L.abd_server_destroy.argtypes = [vp]
    L.abd_server_destroy.restype = None
    if path is None:
        _lib = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data


def default_params(**kw) -> StepParams:
    p = load().abd_step_params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class AbdError(RuntimeError):
    pass


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def scene_desc(sa) -> SceneDesc:
    """SceneDesc pointing into the arrays of `sa` (keep `sa` alive while the
    descriptor is in use)."""
    d = SceneDesc()
    d.n_meshes = len(sa.mesh_n_verts)
    d.mesh_n_verts, d.mesh_n_tris = _p(sa.mesh_n_verts), _p(sa.mesh_n_tris)
    d.mesh_xbar, d.mesh_tris = _p(sa.mesh_xbar), _p(sa.mesh_tris)
    d.n_bodies = sa.n_bodies
    d.body_mesh, d.body_density, d.body_kappa = _p(sa.body_mesh), _p(sa.body_density), _p(sa.body_kappa)
    d.body_kind, d.body_q0, d.body_v0 = _p(sa.body_kind), _p(sa.body_q0), _p(sa.body_v0)
    d.body_omega = _p(getattr(sa, "body_omega", None))
    d.n_planes = len(sa.plane_axis)
    d.plane_axis, d.plane_sign, d.plane_offset = _p(sa.plane_axis), _p(sa.plane_sign), _p(sa.plane_offset)
    for k in range(3):
        d.gravity[k] = float(sa.gravity[k])
    return d


class Scene:
    """A scene resident on the current CUDA device (C ABI handle).  Given a
    list of scene arrays, a batched world of those scenes
    (abd_scene_create_batch): one partition per scene, all stepped in the same
    launches; its state is the concatenation of the scenes' states."""

    def __init__(self, sa, stream: Optional[int] = None):
        L = load()
        self._keep = [sa]
        h = C.c_void_p()
        self.stream = _current_stream() if stream is None else stream
        if isinstance(sa, (list, tuple)):
            descs = (SceneDesc * len(sa))(*[scene_desc(x) for x in sa])
            self._keep.append(descs)
            rc = L.abd_scene_create_batch(C.cast(descs, C.c_void_p), len(sa), self.stream, C.byref(h))
        else:
            d = scene_desc(sa)
            rc = L.abd_scene_create(C.byref(d), self.stream, C.byref(h))
        if rc != 0:
            raise AbdError(f"abd_scene_create failed: {L.abd_status_string(rc).decode()} ({rc})")
        self.h = h
        self.L = L
        cnt = np.zeros(4, dtype=np.int64)
        L.abd_scene_counts(self.h, _p(cnt))
        self.n_bodies, self.n_verts, self.n_tris, self.n_edges = (int(c) for c in cnt)

    def close(self):
        if getattr(self, "h", None) is not None:
            self.L.abd_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc < 0:
            raise AbdError(f"{what}: {self.L.abd_status_string(rc).decode()} ({rc}): "
                           f"{self.L.abd_last_error(self.h).decode()}")
        return rc

    def partition(self, n_slabs=1, axis=0, planes=None, alpha=2.0, w_min=0.0, pd_kp=0.0, pd_kd=0.0, pd_smooth=0.0):
        d = PartitionDesc(axis=axis, n_slabs=n_slabs, planes=None, alpha=alpha, w_min=w_min, pd_kp=pd_kp,
                          pd_kd=pd_kd, pd_smooth=pd_smooth)
        arr = None
        if planes is not None:
            arr = np.ascontiguousarray(planes, dtype=np.float64)
            d.planes = arr.ctypes.data
        self._check(self.L.abd_partition(self.h, C.byref(d)), "abd_partition")

    def partition_masks(self, h=1e-2):
        m = np.zeros(self.n_bodies, dtype=np.uint64)
        w = C.c_double()
        self._check(self.L.abd_partition_masks(self.h, h, _p(m), C.byref(w)), "abd_partition_masks")
        return m, w.value

    def partition_planes(self):
        n = C.c_int32()
        out = np.zeros(64)
        self._check(self.L.abd_partition_planes(self.h, _p(out), 64, C.byref(n)), "abd_partition_planes")
        return out[:n.value].copy()

    def partition_get(self, part):
        n, ns = C.c_int32(), C.c_int32()
        self._check(self.L.abd_partition_get(self.h, part, None, 0, C.byref(n), None, 0, C.byref(ns)),
                    "abd_partition_get")
        b = np.zeros(max(1, n.value), dtype=np.int32)
        sh = np.zeros(max(1, ns.value), dtype=np.int32)
        self._check(self.L.abd_partition_get(self.h, part, _p(b), n.value, C.byref(n), _p(sh), ns.value,
                                             C.byref(ns)), "abd_partition_get")
        return b[:n.value], sh[:ns.value]

    def layout(self):
        """Body offsets of the scenes of a batched world ([n + 1])."""
        n = C.c_int32()
        self._check(self.L.abd_batch_layout(self.h, None, 0, C.byref(n)), "abd_batch_layout")
        off = np.zeros(n.value + 1, dtype=np.int64)
        self._check(self.L.abd_batch_layout(self.h, _p(off), n.value + 1, C.byref(n)), "abd_batch_layout")
        return off

    def partition_newton(self):
        """Newton iterations of each partition (scene of a batched world) in the last step."""
        n = C.c_int32()
        self._check(self.L.abd_partition_newton(self.h, None, 0, C.byref(n)), "abd_partition_newton")
        it = np.zeros(max(1, n.value), dtype=np.int32)
        self._check(self.L.abd_partition_newton(self.h, _p(it), n.value, C.byref(n)), "abd_partition_newton")
        return it[:n.value]

    def broadphase(self, mode):
        """Level-1 pass of later steps: 0 automatic, 1 all pairs per partition, 2 spatial hash."""
        self._check(self.L.abd_scene_broadphase(self.h, int(mode)), "abd_scene_broadphase")

    def reserve(self, pairs):
        self._check(self.L.abd_scene_reserve(self.h, int(pairs)), "abd_scene_reserve")

    def step(self, params: Optional[StepParams] = None) -> dict:
        params = default_params() if params is None else params
        st = StepStats()
        rc = self.L.abd_step(self.h, C.byref(params), C.byref(st))
        self._check(rc, "abd_step")
        return st.as_dict()

    def state(self):
        q, v = np.zeros((self.n_bodies, 12)), np.zeros((self.n_bodies, 12))
        self._check(self.L.abd_state_get(self.h, _p(q), _p(v), self.n_bodies), "abd_state_get")
        return q, v

    def set_state(self, q, v):
        q = np.ascontiguousarray(q, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        self._check(self.L.abd_state_set(self.h, _p(q), _p(v), self.n_bodies), "abd_state_set")

    def device_state(self):
        q, v = C.c_void_p(), C.c_void_p()
        self._check(self.L.abd_state_device(self.h, C.byref(q), C.byref(v)), "abd_state_device")
        return q.value, v.value

    def body_props(self, b):
        m, V = C.c_double(), C.c_double()
        com, S = np.zeros(3), np.zeros(9)
        self._check(self.L.abd_body_props(self.h, b, C.byref(m), _p(com), _p(S), C.byref(V)), "abd_body_props")
        return m.value, com, S.reshape(3, 3), V.value

    def candidates(self, x0, x1=None, dhat=1e-3, cap=None):
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        x1 = None if x1 is None else np.ascontiguousarray(x1, dtype=np.float64)
        n = C.c_int64()
        self._check(self.L.abd_candidates(self.h, _p(x0), _p(x1), dhat, None, 0, C.byref(n)), "abd_candidates")
        cnt = n.value
        out = np.zeros((max(cnt, 1), 3), dtype=np.int32)
        self._check(self.L.abd_candidates(self.h, _p(x0), _p(x1), dhat, _p(out), cnt, C.byref(n)), "abd_candidates")
        return out[:cnt]

    def profile(self, enable=True):
        self._check(self.L.abd_profile(self.h, 1 if enable else 0), "abd_profile")

    def kernel_stats(self, name):
        n, ms, b = C.c_int64(), C.c_double(), C.c_double()
        self._check(self.L.abd_kernel_stats(self.h, name.encode(), C.byref(n), C.byref(ms), C.byref(b)),
                    "abd_kernel_stats")
        return n.value, ms.value, b.value


class Server:
    """Serving runtime (C ABI): worker threads with one CUDA stream each run
    submitted scenes concurrently under an HBM admission budget."""

    def __init__(self, n_streams=4, hbm_budget_bytes=0, device=None):
        L = load()
        if device is None:
            try:
                import torch
                device = torch.cuda.current_device()
            except Exception:
                device = 0
        d = ServerDesc(device=device, n_streams=n_streams, hbm_budget_bytes=hbm_budget_bytes)
        h = C.c_void_p()
        rc = L.abd_server_create(C.byref(d), C.byref(h))
        if rc != 0:
            raise AbdError(f"abd_server_create failed: {L.abd_status_string(rc).decode()} ({rc})")
        self.L, self.h, self._n, self._nb_key = L, h, {}, {}

    def submit(self, sa, n_steps, params: Optional[StepParams] = None, n_slabs=1, axis=0, planes=None,
               alpha=2.0, w_min=0.0, key: Optional[int] = None) -> int:
        """Queue `n_steps` steps of scene `sa`.  With `key`, the scene stays
        resident under that key (abd_server_submit_keyed): give `sa` on the
        key's first request and None on later ones, which continue from the
        state the previous request left."""
        pr = default_params() if params is None else params
        t = C.c_int64()
        if sa is None and key is None:
            raise AbdError("a request without a scene needs the key of a resident scene")
        d = None if sa is None else scene_desc(sa)
        arr = None if planes is None else np.ascontiguousarray(planes, dtype=np.float64)
        pd = PartitionDesc(axis=axis, n_slabs=n_slabs, planes=None if arr is None else arr.ctypes.data,
                           alpha=alpha, w_min=w_min)
        dp = None if d is None else C.cast(C.pointer(d), C.c_void_p)
        if key is None:
            rc = self.L.abd_server_submit(self.h, C.byref(d), C.cast(C.pointer(pd), C.c_void_p),
                                          C.cast(C.pointer(pr), C.c_void_p), n_steps, C.byref(t))
        else:
            rc = self.L.abd_server_submit_keyed(self.h, int(key), dp, C.cast(C.pointer(pd), C.c_void_p),
                                                C.cast(C.pointer(pr), C.c_void_p), n_steps, C.byref(t))
        if rc != 0:
            raise AbdError(f"abd_server_submit: {self.L.abd_status_string(rc).decode()} ({rc})")
        if sa is not None:
            self._nb_key[key] = sa.n_bodies
        self._n[t.value] = sa.n_bodies if sa is not None else self._nb_key[key]
        return t.value

    def release(self, key):
        rc = self.L.abd_server_release(self.h, int(key))
        if rc != 0:
            raise AbdError(f"abd_server_release: {rc}")

    def poll(self, ticket) -> dict:
        info = RequestInfo()
        rc = self.L.abd_server_poll(self.h, ticket, C.byref(info))
        if rc != 0:
            raise AbdError(f"abd_server_poll: {rc}")
        return info.as_dict()

    def wait(self, ticket) -> dict:
        info = RequestInfo()
        rc = self.L.abd_server_wait(self.h, ticket, C.byref(info))
        if rc != 0:
            raise AbdError(f"abd_server_wait: {rc}")
        return info.as_dict()

    def result(self, ticket):
        n = self._n[ticket]
        q, v = np.zeros((n, 12)), np.zeros((n, 12))
        rc = self.L.abd_server_result(self.h, ticket, _p(q), _p(v), n)
        if rc < 0:
            raise AbdError(f"abd_server_result: {self.L.abd_status_string(rc).decode()} ({rc}): "
                           f"{self.L.abd_server_error(self.h, ticket).decode()}")
        return q, v

    def latencies(self, ticket):
        n = C.c_int32()
        self.L.abd_server_latencies(self.h, ticket, None, 0, C.byref(n))
        ms = np.zeros(max(1, n.value))
        self.L.abd_server_latencies(self.h, ticket, _p(ms), n.value, C.byref(n))
        return ms[:n.value]

    def close(self):
        if getattr(self, "h", None) is not None:
            self.L.abd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_update(tau, T_prev=None, kp=0.0, kd=0.0):
    """The load-balancing law of abd_pd_update: (plane shifts, T)."""
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    n = len(tau)
    Tp = None if T_prev is None else np.ascontiguousarray(T_prev, dtype=np.float64)
    delta, T = np.zeros(max(1, n - 1)), np.zeros(max(1, n - 1))
    rc = load().abd_pd_update(n, _p(tau), _p(Tp), kp, kd, _p(delta), _p(T))
    if rc != 0:
        raise AbdError(f"abd_pd_update: {rc}")
    return delta[:n - 1], T[:n - 1]
