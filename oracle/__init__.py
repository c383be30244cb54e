"""FP64 single-threaded CPU oracle of distributed ABD-IPC (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by `tests/`, by `__graft_entry__.smoke()`
and by the benchmark's CPU baseline, never by the product package.  The C
library `libabd_oracle.so` is built from `abd_oracle.c` with the host C
compiler (`build()`); it shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libabd_oracle.so")
_SRC = os.path.join(_HERE, "abd_oracle.c")

DYNAMIC, STATIC, KINEMATIC = 0, 1, 2
OK, ADMM_MAXITER, NEWTON_MAXITER, FELL_BACK, DT_SPLIT = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no -march, no intrinsics)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "abd_oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Desc(C.Structure):
    _fields_ = [("n_meshes", C.c_int32), ("mesh_n_verts", C.c_void_p), ("mesh_n_tris", C.c_void_p),
                ("mesh_xbar", C.c_void_p), ("mesh_tris", C.c_void_p), ("n_bodies", C.c_int32),
                ("body_mesh", C.c_void_p), ("body_density", C.c_void_p), ("body_kappa", C.c_void_p),
                ("body_kind", C.c_void_p), ("body_q0", C.c_void_p), ("body_v0", C.c_void_p), ("body_omega", C.c_void_p),
                ("n_planes", C.c_int32), ("plane_axis", C.c_void_p), ("plane_sign", C.c_void_p),
                ("plane_offset", C.c_void_p), ("gravity", C.c_double * 3)]


class Params(C.Structure):
    _fields_ = [("h", C.c_double), ("dhat", C.c_double), ("kappa_barrier", C.c_double),
                ("rho_adaptive", C.c_int32), ("beta", C.c_double), ("tau", C.c_double),
                ("mu", C.c_double), ("sigma_min", C.c_double), ("sigma_max", C.c_double),
                ("theta", C.c_double), ("newton_tol", C.c_double), ("max_admm", C.c_int32),
                ("max_newton", C.c_int32), ("max_halvings", C.c_int32), ("accd_s", C.c_double),
                ("accd_c", C.c_double), ("n_slabs", C.c_int32), ("axis", C.c_int32),
                ("planes", C.c_void_p), ("alpha_w", C.c_double), ("w_min", C.c_double),
                ("dt_split_max", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("admm_iters", C.c_int32), ("newton_iters", C.c_int32),
                ("n_shared", C.c_int32), ("n_slots", C.c_int32), ("merge_ok", C.c_int32),
                ("n_candidates_peak", C.c_int64), ("n_active_peak", C.c_int64),
                ("r_inf", C.c_double), ("s_inf", C.c_double), ("delta_inf", C.c_double),
                ("min_distance", C.c_double), ("l", C.c_double), ("kappa_barrier", C.c_double),
                ("w", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.orc_scene_create.argtypes = [C.POINTER(_Desc), C.POINTER(C.c_void_p)]
        L.orc_scene_destroy.argtypes = [C.c_void_p]
        L.orc_scene_counts.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_state_get.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_state_set.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_body_props.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_edges.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_vertices.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.POINTER(Params), C.POINTER(Stats)]
        L.orc_partition.argtypes = [C.c_void_p, C.POINTER(Params), C.c_void_p, dp]
        L.orc_mass_properties.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_double, dp,
                                          C.c_void_p, C.c_void_p, dp]
        L.orc_orth.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        L.orc_orth.restype = C.c_double
        L.orc_barrier.argtypes = [C.c_double, C.c_double, C.c_void_p]
        L.orc_pair.argtypes = [C.c_int, C.c_void_p, C.c_double, C.c_double, C.c_double, dp, C.c_void_p,
                               C.c_void_p, ip]
        L.orc_pair.restype = C.c_double
        L.orc_dist_type.argtypes = [C.c_int, C.c_void_p, ip, C.c_void_p]
        L.orc_dist_type.restype = C.c_double
        L.orc_psd_project.argtypes = [C.c_int, C.c_void_p]
        L.orc_ccd.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_double]
        L.orc_ccd.restype = C.c_double
        L.orc_ccd_plane.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_ccd_plane.restype = C.c_double
        L.orc_candidates.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_int64]
        L.orc_candidates.restype = C.c_int64
        L.orc_objective.argtypes = [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_void_p, dp, C.c_void_p, C.c_void_p]
        L.orc_local_objectives.argtypes = [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_int, C.c_void_p, C.c_void_p]
        L.orc_mollifier.argtypes = [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
        L.orc_mollifier.restype = C.c_double
        L.orc_rho_update.argtypes = [C.c_double] * 8 + [dp]
        L.orc_rho_update.restype = C.c_double
        L.orc_local_gradient.argtypes = [C.c_void_p, C.POINTER(Params), C.c_int, C.c_void_p, C.c_void_p, dp,
                                         C.c_void_p]
        L.orc_admm_trace.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        L.orc_admm_trace_count.argtypes = [C.c_void_p]
        L.orc_admm_trace_count.restype = C.c_int64
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- building blocks

def mass_properties(xbar, tris, density):
    xbar, tris = _f64(xbar), np.ascontiguousarray(tris, dtype=np.int32)
    m, V = C.c_double(), C.c_double()
    com, S = np.zeros(3), np.zeros(9)
    rc = lib().orc_mass_properties(xbar.shape[0], _p(xbar), tris.shape[0], _p(tris), density,
                                   C.byref(m), _p(com), _p(S), C.byref(V))
    if rc != 0:
        raise ValueError(f"mass properties failed: {rc}")
    return m.value, com, S.reshape(3, 3), V.value


def orth(q12, kappa, V):
    q = _f64(q12)
    g, H = np.zeros(12), np.zeros(144)
    E = lib().orc_orth(_p(q), kappa, V, _p(g), _p(H))
    return E, g, H.reshape(12, 12)


def barrier(d, dhat):
    out = np.zeros(3)
    lib().orc_barrier(d, dhat, _p(out))
    return out


def pair(is_ee, X, dhat, kB, eps_x=0.0):
    X = _f64(X).reshape(12)
    E, t = C.c_double(), C.c_int()
    g, H = np.zeros(12), np.zeros(144)
    d = lib().orc_pair(int(is_ee), _p(X), dhat, kB, eps_x, C.byref(E), _p(g), _p(H), C.byref(t))
    return d, E.value, g, H.reshape(12, 12), t.value


def dist_type(is_ee, X):
    X = _f64(X).reshape(12)
    t = C.c_int()
    beta = np.zeros(2)
    d2 = lib().orc_dist_type(int(is_ee), _p(X), C.byref(t), _p(beta))
    return d2, t.value, beta


def mollifier(X, eps_x):
    X = _f64(X).reshape(12)
    g, H = np.zeros(12), np.zeros(144)
    m = lib().orc_mollifier(_p(X), eps_x, _p(g), _p(H))
    return m, g, H.reshape(12, 12)


def psd_project(A):
    A = _f64(A).copy()
    n = A.shape[0]
    lib().orc_psd_project(n, _p(A))
    return A


def ccd(is_ee, X, dX, s=0.1, c=0.9):
    X, dX = _f64(X).reshape(12), _f64(dX).reshape(12)
    return lib().orc_ccd(int(is_ee), _p(X), _p(dX), s, c)


def ccd_plane(d0, dd, s=0.1):
    return lib().orc_ccd_plane(d0, dd, s)


def rho_update(r, s, rho, rho0, tau=2.0, mu=5.0, sigma_min=1e-3, sigma_max=1e3):
    """Residual-driven penalty of one shared body (Sec. 4.3): (rho_new,
    u_scale), u_scale = rho / rho_new being the factor of the scaled dual."""
    sc = C.c_double()
    nw = lib().orc_rho_update(r, s, rho, rho0, tau, mu, sigma_min, sigma_max, C.byref(sc))
    return nw, sc.value


TRACE_REC = 68  # doubles per ADMM trace record (oracle/abd_oracle.h)


# ---------------------------------------------------------------- scene + step

def default_params(**kw) -> Params:
    p = Params(h=1e-2, dhat=1e-3, kappa_barrier=0.0, rho_adaptive=1, beta=1.0, tau=2.0, mu=5.0,
               sigma_min=1e-3, sigma_max=1e3, theta=1e-3, newton_tol=1e-6, max_admm=200,
               max_newton=100, max_halvings=40, accd_s=0.1, accd_c=0.9, n_slabs=1, axis=0,
               planes=None, alpha_w=2.0, w_min=0.0, dt_split_max=0)
    planes = kw.pop("planes", None)
    for k, v in kw.items():
        setattr(p, k, v)
    if planes is not None:
        arr = _f64(planes)
        p._planes_keepalive = arr
        p.planes = arr.ctypes.data
    return p


class Scene:
    """Oracle scene built from `scenes.SceneArrays`."""

    def __init__(self, sa):
        self._keep = [sa]
        d = _Desc()
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
        h = C.c_void_p()
        rc = lib().orc_scene_create(C.byref(d), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle scene create failed: {rc}")
        self.h = h
        cnt = np.zeros(4, dtype=np.int64)
        lib().orc_scene_counts(self.h, _p(cnt))
        self.n_bodies, self.n_verts, self.n_tris, self.n_edges = (int(c) for c in cnt)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.orc_scene_destroy(self.h)
            self.h = None

    def state(self):
        q, v = np.zeros((self.n_bodies, 12)), np.zeros((self.n_bodies, 12))
        lib().orc_state_get(self.h, _p(q), _p(v))
        return q, v

    def set_state(self, q, v):
        q, v = _f64(q), _f64(v)
        lib().orc_state_set(self.h, _p(q), _p(v))

    def body_props(self, b):
        m, V = C.c_double(), C.c_double()
        com, S = np.zeros(3), np.zeros(9)
        lib().orc_body_props(self.h, b, C.byref(m), _p(com), _p(S), C.byref(V))
        return m.value, com, S.reshape(3, 3), V.value

    def edges(self):
        e = np.zeros((self.n_edges, 2), dtype=np.int32)
        lib().orc_edges(self.h, _p(e))
        return e

    def vertices(self, q=None):
        x = np.zeros((self.n_verts, 3))
        lib().orc_vertices(self.h, _p(None if q is None else _f64(q)), _p(x))
        return x

    def candidates(self, x0, x1=None, dhat=1e-3):
        x0 = _f64(x0)
        x1 = None if x1 is None else _f64(x1)
        n = lib().orc_candidates(self.h, _p(x0), _p(x1), dhat, None, 0)
        if n < 0:
            raise MemoryError("oracle candidates")
        out = np.zeros((max(n, 1), 3), dtype=np.int32)
        lib().orc_candidates(self.h, _p(x0), _p(x1), dhat, _p(out), n)
        return out[:n]

    def partition(self, params: Params):
        m = np.zeros(self.n_bodies, dtype=np.uint64)
        w = C.c_double()
        rc = lib().orc_partition(self.h, C.byref(params), _p(m), C.byref(w))
        if rc != 0:
            raise ValueError(f"partition failed: {rc}")
        return m, w.value

    def objective(self, params: Params, q_dyn, qtil_dyn, want_hess=True):
        """Monolithic objective (energy, gradient, projected Hessian) at the
        dynamic-body configuration q_dyn [n_dyn, 12]."""
        q, qt = _f64(q_dyn), _f64(qtil_dyn)
        n = q.size
        E = C.c_double()
        g = np.zeros(n)
        H = np.zeros((n, n)) if want_hess else None
        rc = lib().orc_objective(self.h, C.byref(params), _p(q), _p(qt), C.byref(E), _p(g), _p(H))
        if rc != 0:
            raise RuntimeError(f"objective failed: {rc}")
        return E.value, g, H

    def local_objectives(self, params: Params, q_dyn, qtil_dyn, want_hess=False):
        """Per-partition objectives F_i of Eq. 3 at the consensus point where
        every replica equals q_dyn (membership from the slab rule at the
        scene's current state), the sum of their gradients scattered to the
        bodies and, with want_hess, the sum of their projected Hessians.
        Returns (E_parts [N], g_sum [n_dof, 12], H_sum [12 n_dof]^2 or None)."""
        q, qt = _f64(q_dyn), _f64(qtil_dyn)
        E = np.zeros(64)
        g = np.zeros(q.shape)
        H = np.zeros((q.size, q.size)) if want_hess else None
        n = lib().orc_local_objectives(self.h, C.byref(params), _p(q), _p(qt), _p(E), 64, _p(g), _p(H))
        if n < 0:
            raise RuntimeError(f"local objectives failed: {n}")
        return E[:n], g, H

    def local_gradient(self, params: Params, part, q_dyn, qtil_dyn):
        """(F_i, dF_i/dq [n_dof, 12]) of partition `part` (Eq. 3, no consensus
        term) at the replica configuration q_dyn; barrier stiffness
        params.kappa_barrier, membership from the slab rule at the current
        state."""
        q, qt = _f64(q_dyn), _f64(qtil_dyn)
        E = C.c_double()
        g = np.zeros(q.shape)
        rc = lib().orc_local_gradient(self.h, C.byref(params), int(part), _p(q), _p(qt), C.byref(E), _p(g))
        if rc != 0:
            raise RuntimeError(f"local gradient failed: {rc}")
        return E.value, g

    def step_traced(self, params: Params, cap: int = 20000):
        """One step with the ADMM trace on: (stats, records [n, TRACE_REC]),
        one record per (continuing round, shared body, replica)."""
        buf = np.zeros((cap, TRACE_REC))
        lib().orc_admm_trace(self.h, _p(buf), cap)
        try:
            st = self.step(params)
            n = lib().orc_admm_trace_count(self.h)
        finally:
            lib().orc_admm_trace(self.h, None, 0)
        if n > cap:
            raise RuntimeError(f"trace of {n} records exceeds cap {cap}")
        return st, buf[:n].copy()

    def step(self, params: Params):
        st = Stats()
        rc = lib().orc_step(self.h, C.byref(params), C.byref(st))
        if rc < 0:
            raise RuntimeError(f"oracle step failed: {rc} {st.as_dict()}")
        return st.as_dict()
