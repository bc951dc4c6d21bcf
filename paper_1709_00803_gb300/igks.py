"""Thin ctypes binding of libigks (include/igks.h). Argument marshalling only: every step
of the IGKS iteration runs in the library's CUDA kernels. There is no CPU fallback: if the
shared library cannot be built or loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, CONVERGED = 0, 1
EINVAL, EMESH, ENOMEM, ECUDA, DIVERGED, TIMEOUT, EBUSY, MAXITER = -1, -2, -3, -4, -5, -6, -7, -8
PREC_FP64, PREC_MIXED, PREC_DF64 = 0, 1, 2
ARR = dict(grad=1, phi=2, lambda_f=3, lambda_c=4, flux=5, res=6, dwstar=7, dw=8, ghost=9,
           geom_cell=10, geom_face=11)


class IgksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libigks error {code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("stream", C.c_void_p),
                ("check_every", C.c_int32), ("use_graph", C.c_int32), ("sweep_threads", C.c_int32),
                ("timing", C.c_int32), ("sweep_mode", C.c_int32), ("sweep_cluster", C.c_int32),
                ("groups", C.c_int32), ("wait_limit", C.c_int32), ("starve_test", C.c_int32),
                ("reserved", C.c_int32 * 1)]


class Flow(C.Structure):
    _fields_ = [("mach", C.c_double), ("reynolds", C.c_double), ("aoa_deg", C.c_double),
                ("prandtl", C.c_double), ("t_ref", C.c_double), ("s_suth", C.c_double),
                ("sa_on", C.c_int32), ("limiter", C.c_int32), ("nut_ratio_inf", C.c_double),
                ("cfl_exp", C.c_double), ("cfl_init", C.c_double), ("cfl_min", C.c_double),
                ("cfl_max", C.c_double), ("res_target", C.c_double), ("venkat_k", C.c_double),
                ("c_num", C.c_double), ("visc_sr", C.c_int32), ("scheme", C.c_int32),
                ("eq40_target", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("sweep_threads", C.c_int32), ("flux_block", C.c_int32), ("sweep_mode", C.c_int32),
                ("sweep_cluster", C.c_int32), ("ms_per_iter", C.c_float), ("groups", C.c_int32)]


class Status(C.Structure):
    _fields_ = [("iters", C.c_int32), ("state", C.c_int32), ("res_l2_rho", C.c_double),
                ("res_l2_rel", C.c_double), ("res_inf", C.c_double), ("eq40_ratio", C.c_double),
                ("cfl", C.c_double), ("dt", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("max_slots", C.c_int32),
                ("max_cohort", C.c_int32), ("iters_per_step", C.c_int32), ("max_iters", C.c_int32),
                ("hbm_budget", C.c_int64), ("repack_fraction", C.c_double), ("keep_fields", C.c_int32),
                ("reserved", C.c_int32 * 7)]


class Request(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("xy", C.c_void_p), ("n_cells", C.c_int32), ("cell_ptr", C.c_void_p),
                ("cell_nodes", C.c_void_p), ("n_faces", C.c_int32), ("face_nodes", C.c_void_p),
                ("face_cells", C.c_void_p), ("face_bc", C.c_void_p), ("flow", Flow), ("tag", C.c_int64),
                ("W0", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("id", C.c_int64), ("tag", C.c_int64), ("state", C.c_int32), ("iters", C.c_int32),
                ("n_cells", C.c_int32), ("cohort", C.c_int32), ("res_l2_rel", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_finish", C.c_double),
                ("forces", C.c_double * 3), ("footprint", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "forces"}
        d["forces"] = tuple(self.forces)
        return d


class ServerStatus(C.Structure):
    _fields_ = [("queued", C.c_int32), ("live", C.c_int32), ("cohorts", C.c_int32), ("finished", C.c_int32),
                ("bytes", C.c_int64), ("budget", C.c_int64), ("admitted", C.c_int32), ("repacked", C.c_int32),
                ("step_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load (building first if needed) the in-tree libigks.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P, i32, d = C.POINTER, C.c_int32, C.c_double
        ip, dp, vp = P(C.c_int32), P(C.c_double), C.c_void_p
        L.igks_create.argtypes = [P(Options), P(vp)]
        L.igks_mesh_upload.argtypes = [vp, i32, dp, i32, ip, ip, i32, ip, ip, ip, ip]
        L.igks_set_flow.argtypes = [vp, i32, P(Flow)]
        L.igks_init_freestream.argtypes = [vp, i32]
        L.igks_iterate.argtypes = [vp, i32, P(Status)]
        L.igks_get_fields.argtypes = [vp, i32, dp]
        L.igks_set_fields.argtypes = [vp, i32, dp]
        L.igks_get_fields_all.argtypes = [vp, dp]
        L.igks_set_fields_all.argtypes = [vp, dp]
        L.igks_get_scalars.argtypes = [vp, i32, dp]
        L.igks_set_scalars.argtypes = [vp, i32, dp]
        L.igks_get_array.argtypes = [vp, i32, i32, dp]
        L.igks_mesh_info.argtypes = [vp, i32, ip]
        L.igks_get_forces.argtypes = [vp, i32, i32, dp]
        L.igks_launches_per_iteration.argtypes = [vp, ip]
        L.igks_destroy.argtypes = [vp]
        L.igks_last_error.argtypes = [vp]
        L.igks_last_error.restype = C.c_char_p
        L.igks_enqueue.argtypes = [vp, i32]
        L.igks_kernel_times.argtypes = [vp, i32, P(C.c_float), ip]
        L.igks_kernel_name.argtypes = [i32]
        L.igks_kernel_name.restype = C.c_char_p
        L.igks_residual_norms_noalloc.argtypes = [vp, vp, i32, vp, vp]
        L.igks_residual_norms_noalloc.restype = C.c_int32
        L.igks_fp64_probe.argtypes = [i32, dp]
        L.igks_autotune.argtypes = [vp, i32, P(Tuning)]
        L.igks_set_launch.argtypes = [vp, P(Tuning)]
        L.igks_get_history.argtypes = [vp, i32, i32, dp, ip]
        L.igks_autotune.restype = C.c_int32
        L.igks_order_cells.argtypes = [i32, i32, ip, i32, ip, ip]
        L.igks_order_cells.restype = C.c_int32
        i64p = P(C.c_int64)
        L.igks_footprint_bytes.argtypes = [i32, i32, i32, i32, i64p]
        L.igks_device_bytes.argtypes = [vp, i64p]
        L.igks_server_create.argtypes = [P(ServerOptions), P(vp)]
        L.igks_server_submit.argtypes = [vp, P(Request), i64p]
        L.igks_server_step.argtypes = [vp, P(ServerStatus)]
        L.igks_server_poll.argtypes = [vp, P(Result), i32, ip]
        L.igks_server_take_fields.argtypes = [vp, C.c_int64, dp]
        L.igks_server_now.argtypes = [vp, dp]
        L.igks_server_get_status.argtypes = [vp, P(ServerStatus)]
        L.igks_server_destroy.argtypes = [vp]
        L.igks_server_last_error.argtypes = [vp]
        L.igks_server_last_error.restype = C.c_char_p
        for name in ("igks_footprint_bytes", "igks_device_bytes", "igks_server_create", "igks_server_submit",
                     "igks_server_step", "igks_server_poll", "igks_server_take_fields", "igks_server_now",
                     "igks_server_get_status", "igks_server_destroy"):
            getattr(L, name).restype = C.c_int32
        for name in ("igks_create", "igks_mesh_upload", "igks_set_flow", "igks_init_freestream",
                     "igks_iterate", "igks_get_fields", "igks_set_fields", "igks_get_scalars",
                     "igks_set_scalars", "igks_get_array", "igks_mesh_info", "igks_get_forces",
                     "igks_launches_per_iteration", "igks_destroy", "igks_enqueue", "igks_kernel_times"):
            getattr(L, name).restype = C.c_int32
        _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


NOALLOC_MAX_CELLS = 1 << 20


def fp64_probe(device: int = 0) -> float:
    """Measured FP64 rate of the device in TFLOP/s (igks_fp64_probe)."""
    t = C.c_double()
    rc = lib().igks_fp64_probe(device, C.byref(t))
    if rc != OK:
        raise IgksError(rc, "igks_fp64_probe failed")
    return t.value


def residual_norms_noalloc(m_rho_ptr: int, area_ptr: int, n_cells: int, out_ptr: int, stream: int = 0) -> int:
    """igks_residual_norms_noalloc: DEVICE pointers in and out (e.g. tensor.data_ptr());
    the library allocates nothing for it. Returns the status code; raises on error."""
    L = lib()
    rc = L.igks_residual_norms_noalloc(C.c_void_p(m_rho_ptr), C.c_void_p(area_ptr), n_cells,
                                       C.c_void_p(out_ptr), C.c_void_p(stream))
    if rc != OK:
        raise IgksError(rc, L.igks_last_error(None).decode())
    return rc


ORDER_AS_GIVEN, ORDER_MULTICOLOR = 0, 1


def order_cells(mesh, mode=ORDER_MULTICOLOR):
    """igks_order_cells: a cell permutation (perm[k] = old index at position k) and the
    number of colours. Apply it with mesh.renumbered(perm) before upload."""
    fc = np.ascontiguousarray(mesh.face_cells, dtype=np.int32).ravel()
    perm = np.zeros(mesh.n_cells, dtype=np.int32)
    nc = C.c_int32()
    rc = lib().igks_order_cells(mesh.n_cells, mesh.n_faces, _ip(fc), mode, _ip(perm), C.byref(nc))
    if rc != OK:
        raise IgksError(rc, "igks_order_cells failed")
    return perm, nc.value


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def to_flow(flow) -> Flow:
    d = flow.as_dict() if hasattr(flow, "as_dict") else dict(flow)
    f = Flow()
    for name, _ in Flow._fields_:
        if name in d:
            setattr(f, name, d[name])
    return f


class Context:
    """One igks_ctx: a set of steady solves resident on one GPU."""

    def __init__(self, precision=PREC_FP64, device=0, stream=None, check_every=20, use_graph=1,
                 sweep_threads=0, timing=0, sweep_mode=0, sweep_cluster=0, groups=0, wait_limit=0,
                 starve_test=0):
        o = Options(precision=precision, device=device, stream=stream, check_every=check_every,
                    use_graph=use_graph, sweep_threads=sweep_threads, timing=timing, sweep_mode=sweep_mode,
                    sweep_cluster=sweep_cluster, groups=groups, wait_limit=wait_limit, starve_test=starve_test)
        h = C.c_void_p()
        rc = lib().igks_create(C.byref(o), C.byref(h))
        if rc:
            raise IgksError(rc, "igks_create failed")
        self.h = h
        self.meshes = []
        self.precision = precision

    def _check(self, rc, ok=(OK,)):
        if rc not in ok:
            raise IgksError(rc, lib().igks_last_error(self.h).decode())
        return rc

    # --- C ABI, same names ---
    def mesh_upload(self, mesh) -> int:
        xy = np.ascontiguousarray(mesh.xy, dtype=np.float64).ravel()
        cp = np.ascontiguousarray(mesh.cell_ptr, dtype=np.int32)
        cn = np.ascontiguousarray(mesh.cell_nodes, dtype=np.int32)
        fn = np.ascontiguousarray(mesh.face_nodes, dtype=np.int32).ravel()
        fc = np.ascontiguousarray(mesh.face_cells, dtype=np.int32).ravel()
        fb = np.ascontiguousarray(mesh.face_bc, dtype=np.int32)
        sid = C.c_int32()
        self._check(lib().igks_mesh_upload(self.h, mesh.n_nodes, _dp(xy), mesh.n_cells, _ip(cp), _ip(cn),
                                           mesh.n_faces, _ip(fn), _ip(fc), _ip(fb), C.byref(sid)))
        self.meshes.append(mesh)
        return sid.value

    def set_flow(self, solve, flow):
        f = to_flow(flow)
        self._check(lib().igks_set_flow(self.h, solve, C.byref(f)))

    def init_freestream(self, solve):
        self._check(lib().igks_init_freestream(self.h, solve))

    def iterate(self, max_iters):
        st = (Status * len(self.meshes))()
        rc = self._check(lib().igks_iterate(self.h, max_iters, st), ok=(OK, CONVERGED, DIVERGED, TIMEOUT))
        return rc, [s.as_dict() for s in st]

    def enqueue(self, n_iters):
        self._check(lib().igks_enqueue(self.h, n_iters))

    def autotune(self, iters_per_trial=3):
        t = Tuning()
        self._check(lib().igks_autotune(self.h, iters_per_trial, C.byref(t)))
        return {k: getattr(t, k) for k, _ in t._fields_}

    def set_launch(self, tuning):
        """Apply a launch configuration (a dict as autotune() returns)."""
        t = Tuning(**{k: tuning[k] for k, _ in Tuning._fields_ if k in tuning})
        self._check(lib().igks_set_launch(self.h, C.byref(t)))

    def kernel_times(self):
        ms = (C.c_float * 32)()
        n = C.c_int32()
        self._check(lib().igks_kernel_times(self.h, 32, ms, C.byref(n)))
        return {lib().igks_kernel_name(k).decode(): float(ms[k]) for k in range(n.value)}

    def get_fields(self, solve, out=None):
        shape = (5, self.meshes[solve].n_cells)
        W = np.zeros(shape) if out is None else out
        assert W.shape == shape and W.dtype == np.float64 and W.flags.c_contiguous
        self._check(lib().igks_get_fields(self.h, solve, _dp(W)))
        return W

    def set_fields(self, solve, W):
        if not (isinstance(W, np.ndarray) and W.dtype == np.float64 and W.flags.c_contiguous):
            W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == (5, self.meshes[solve].n_cells)
        self._check(lib().igks_set_fields(self.h, solve, _dp(W)))

    def get_fields_all(self, out=None):
        """The state of every solve: [5, N] with the solves' cells side by side in upload order."""
        shape = (5, sum(m.n_cells for m in self.meshes))
        W = np.zeros(shape) if out is None else out
        assert W.shape == shape and W.dtype == np.float64 and W.flags.c_contiguous
        self._check(lib().igks_get_fields_all(self.h, _dp(W)))
        return W

    def set_fields_all(self, W):
        if not (isinstance(W, np.ndarray) and W.dtype == np.float64 and W.flags.c_contiguous):
            W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == (5, sum(m.n_cells for m in self.meshes))
        self._check(lib().igks_set_fields_all(self.h, _dp(W)))

    def get_scalars(self, solve):
        o = np.zeros(5)
        self._check(lib().igks_get_scalars(self.h, solve, _dp(o)))
        return dict(iter=int(o[0]), cfl=o[1], res_inf_prev=o[2], res_l2_first=o[3], state=int(o[4]))

    def set_scalars(self, solve, sc):
        o = np.array([sc["iter"], sc["cfl"], sc["res_inf_prev"], sc["res_l2_first"], sc["state"]], dtype=np.float64)
        self._check(lib().igks_set_scalars(self.h, solve, _dp(o)))

    def get_array(self, solve, which):
        m = self.meshes[solve]
        n, nf = m.n_cells, m.n_faces
        shapes = dict(grad=(4, 2, n), phi=(4, n), lambda_f=(nf,), lambda_c=(n,), flux=(6, nf), res=(5, n),
                      dwstar=(5, n), dw=(5, n), ghost=(5, nf), geom_cell=(4, n), geom_face=(5, nf))
        out = np.zeros(shapes[which])
        self._check(lib().igks_get_array(self.h, solve, ARR[which], _dp(out)))
        return out

    def get_history(self, solve, cap=1024):
        """Residual history of a solve: array [n, 3] of (iteration, RMS M_rho/Omega, max |M_rho|)."""
        out = np.zeros((cap, 3))
        n = C.c_int32()
        self._check(lib().igks_get_history(self.h, solve, cap, _dp(out), C.byref(n)))
        return out[:n.value].copy()

    def mesh_info(self, solve):
        o = np.zeros(5, dtype=np.int32)
        self._check(lib().igks_mesh_info(self.h, solve, _ip(o)))
        return dict(n_cells=int(o[0]), n_faces=int(o[1]), levels_fwd=int(o[2]), levels_bwd=int(o[3]),
                    n_boundary=int(o[4]))

    def get_forces(self, solve, bc_tag=3):
        o = np.zeros(3)
        self._check(lib().igks_get_forces(self.h, solve, bc_tag, _dp(o)))
        return dict(cl=o[0], cd=o[1], cd_viscous=o[2])

    def device_bytes(self):
        o = C.c_int64()
        self._check(lib().igks_device_bytes(self.h, C.byref(o)))
        return o.value

    def launches_per_iteration(self):
        o = C.c_int32()
        self._check(lib().igks_launches_per_iteration(self.h, C.byref(o)))
        return o.value

    def destroy(self):
        if getattr(self, "h", None):
            lib().igks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def footprint_bytes(mesh) -> int:
    """igks_footprint_bytes: upper bound of the device bytes of one solve of this mesh."""
    o = C.c_int64()
    rc = lib().igks_footprint_bytes(mesh.n_nodes, mesh.n_cells, mesh.n_faces, int(mesh.cell_ptr[-1]), C.byref(o))
    if rc != OK:
        raise IgksError(rc, "igks_footprint_bytes failed")
    return o.value


class Server:
    """One igks_server: continuous batching of steady solves on one GPU."""

    def __init__(self, precision=PREC_MIXED, device=0, max_slots=64, max_cohort=64, iters_per_step=20,
                 max_iters=50000, hbm_budget=0, repack_fraction=0.5, keep_fields=1):
        o = ServerOptions(precision=precision, device=device, max_slots=max_slots, max_cohort=max_cohort,
                          iters_per_step=iters_per_step, max_iters=max_iters, hbm_budget=hbm_budget,
                          repack_fraction=repack_fraction, keep_fields=keep_fields)
        h = C.c_void_p()
        rc = lib().igks_server_create(C.byref(o), C.byref(h))
        if rc:
            raise IgksError(rc, "igks_server_create failed")
        self.h = h
        self._keep = {}

    def _check(self, rc):
        if rc != OK:
            raise IgksError(rc, lib().igks_server_last_error(self.h).decode())
        return rc

    def submit(self, mesh, flow, tag=0, W0=None) -> int:
        """Queue one steady solve; W0 (optional, [5, n_cells]) is its starting state."""
        w0 = None if W0 is None else np.ascontiguousarray(W0, dtype=np.float64).reshape(5, mesh.n_cells)
        arrs = (np.ascontiguousarray(mesh.xy, dtype=np.float64).ravel(),
                np.ascontiguousarray(mesh.cell_ptr, dtype=np.int32),
                np.ascontiguousarray(mesh.cell_nodes, dtype=np.int32),
                np.ascontiguousarray(mesh.face_nodes, dtype=np.int32).ravel(),
                np.ascontiguousarray(mesh.face_cells, dtype=np.int32).ravel(),
                np.ascontiguousarray(mesh.face_bc, dtype=np.int32))
        xy, cp, cn, fn, fc, fb = (a.ctypes.data for a in arrs)
        r = Request(n_nodes=mesh.n_nodes, xy=xy, n_cells=mesh.n_cells, cell_ptr=cp, cell_nodes=cn,
                    n_faces=mesh.n_faces, face_nodes=fn, face_cells=fc, face_bc=fb, flow=to_flow(flow), tag=tag,
                    W0=None if w0 is None else w0.ctypes.data)
        rid = C.c_int64()
        self._check(lib().igks_server_submit(self.h, C.byref(r), C.byref(rid)))
        self._keep[rid.value] = mesh.n_cells
        return rid.value

    def step(self):
        st = ServerStatus()
        self._check(lib().igks_server_step(self.h, C.byref(st)))
        return st.as_dict()

    def status(self):
        st = ServerStatus()
        self._check(lib().igks_server_get_status(self.h, C.byref(st)))
        return st.as_dict()

    def poll(self, cap=256):
        out = (Result * cap)()
        n = C.c_int32()
        self._check(lib().igks_server_poll(self.h, out, cap, C.byref(n)))
        return [out[k].as_dict() for k in range(n.value)]

    def take_fields(self, rid):
        W = np.zeros((5, self._keep[rid]))
        self._check(lib().igks_server_take_fields(self.h, rid, _dp(W)))
        return W

    def now(self):
        t = C.c_double()
        self._check(lib().igks_server_now(self.h, C.byref(t)))
        return t.value

    def destroy(self):
        if getattr(self, "h", None):
            lib().igks_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
