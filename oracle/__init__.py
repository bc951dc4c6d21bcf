"""CPU oracle of the implicit gas-kinetic scheme -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded FP64 C restatement of one IGKS iteration (Pan, Zhong &
Zhuo, arXiv:1709.00803, Sections II.A-II.E), loaded through ctypes. Only the test-suite,
the smoke check and the CPU-baseline leg of the benchmark may import this package; the
CUDA library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "igks_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ORA_W, ORA_GRAD, ORA_PHI, ORA_LAMBDA_F, ORA_LAMBDA_C, ORA_FLUX, ORA_RES, ORA_DWSTAR, \
    ORA_DW, ORA_GHOST, ORA_GEOM_CELL, ORA_GEOM_FACE = range(12)
SCALARS = ["dt", "cfl", "res_inf", "res_l2", "res_l2_first", "eq40", "iter", "status",
           "res_inf_prev"]


class OraFlow(C.Structure):
    _fields_ = [("mach", C.c_double), ("reynolds", C.c_double), ("aoa_deg", C.c_double),
                ("prandtl", C.c_double), ("t_ref", C.c_double), ("s_suth", C.c_double),
                ("sa_on", C.c_int), ("limiter", C.c_int),
                ("nut_ratio_inf", C.c_double), ("cfl_exp", C.c_double), ("cfl_init", C.c_double),
                ("cfl_min", C.c_double), ("cfl_max", C.c_double), ("res_target", C.c_double),
                ("venkat_k", C.c_double), ("c_num", C.c_double),
                ("visc_sr", C.c_int), ("scheme", C.c_int), ("eq40_target", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, -ffp-contract=off so every product is rounded)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(os.path.dirname(_LIB), exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        d, i, P = C.c_double, C.c_int, C.POINTER
        dp, ip = P(C.c_double), P(C.c_int)
        L.ora_moments_full.argtypes = [d, d, dp]
        L.ora_moments_half.argtypes = [d, d, i, dp]
        L.ora_moments_xi.argtypes = [d, dp]
        L.ora_moment_matrix.argtypes = [d, d, d, dp]
        L.ora_moment_solve.argtypes = [d, d, d, dp, dp]
        L.ora_moment_solve.restype = i
        L.ora_time_weights.argtypes = [d, d, dp]
        L.ora_viscosity.argtypes = [P(OraFlow), d]
        L.ora_viscosity.restype = d
        L.ora_face_flux.argtypes = [P(OraFlow)] + [dp] * 8 + [d, d, d, d, dp, dp]
        L.ora_face_flux.restype = i
        L.ora_euler_flux.argtypes = [dp, d, d, dp]
        L.ora_sa_source.argtypes = [d, d, d, d, dp]
        L.ora_create.argtypes = [i, dp, i, ip, ip, i, ip, ip, ip, P(OraFlow)]
        L.ora_create.restype = C.c_void_p
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_init_freestream.argtypes = [C.c_void_p]
        L.ora_set_W.argtypes = [C.c_void_p, dp]
        L.ora_iterate.argtypes = [C.c_void_p, i]
        L.ora_iterate.restype = i
        L.ora_get.argtypes = [C.c_void_p, i, dp]
        L.ora_get.restype = i
        L.ora_get_scalars.argtypes = [C.c_void_p, dp]
        L.ora_set_scalars.argtypes = [C.c_void_p, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def to_flow(flow) -> OraFlow:
    d = flow.as_dict() if hasattr(flow, "as_dict") else dict(flow)
    f = OraFlow()
    for name, _ in OraFlow._fields_:
        if name in d:
            setattr(f, name, d[name])
    return f


# ---- building blocks --------------------------------------------------------------------

def moments_full(U, lam):
    m = np.zeros(10); lib().ora_moments_full(U, lam, _dp(m)); return m


def moments_half(U, lam, side):
    m = np.zeros(10); lib().ora_moments_half(U, lam, side, _dp(m)); return m


def moments_xi(lam):
    m = np.zeros(4); lib().ora_moments_xi(lam, _dp(m)); return m


def moment_matrix(U, V, lam):
    M = np.zeros(16); lib().ora_moment_matrix(U, V, lam, _dp(M)); return M.reshape(4, 4)


def moment_solve(U, V, lam, b):
    b = np.ascontiguousarray(b, dtype=np.float64); a = np.zeros(4)
    if lib().ora_moment_solve(U, V, lam, _dp(b), _dp(a)):
        raise ArithmeticError("singular moment matrix")
    return a


def time_weights(dt, tau):
    q = np.zeros(6); lib().ora_time_weights(dt, tau, _dp(q)); return q


def viscosity(flow, lam):
    f = to_flow(flow)
    return lib().ora_viscosity(C.byref(f), lam)


def euler_flux(W, nx, ny):
    W = np.ascontiguousarray(W[:4], dtype=np.float64); F = np.zeros(4)
    lib().ora_euler_flux(_dp(W), nx, ny, _dp(F)); return F


def sa_source(nut, nu, omega, d):
    """Spalart-Allmaras source of Eq. 28a per unit volume and its parts:
    dict(Sr, fw, S_tilde, r, fv1, fv2)."""
    o = np.zeros(6)
    lib().ora_sa_source(nut, nu, omega, d, _dp(o))
    return dict(zip(("Sr", "fw", "S_tilde", "r", "fv1", "fv2"), o.tolist()))


def face_flux(flow, WL, WR, sLn, sLt, sRn, sRt, WcL, WcR, dL, dR, mut, dt):
    """Time-integrated interface flux in the face frame; returns (F[4], heat flux)."""
    f = to_flow(flow)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (WL, WR, sLn, sLt, sRn, sRt, WcL, WcR)]
    F = np.zeros(4); h = np.zeros(1)
    rc = lib().ora_face_flux(C.byref(f), *[_dp(a) for a in arrs], dL, dR, mut, dt, _dp(F), _dp(h))
    if rc:
        raise ArithmeticError(f"face flux failed ({rc})")
    return F, float(h[0])


# ---- whole solver ------------------------------------------------------------------------

class Oracle:
    """One steady solve on one mesh, advanced iteration by iteration in the oracle."""

    def __init__(self, mesh, flow):
        self.mesh = mesh
        self.flow = flow
        self._f = to_flow(flow)
        self._keep = [np.ascontiguousarray(mesh.xy, dtype=np.float64).ravel(),
                      np.ascontiguousarray(mesh.cell_ptr, dtype=np.int32),
                      np.ascontiguousarray(mesh.cell_nodes, dtype=np.int32),
                      np.ascontiguousarray(mesh.face_nodes, dtype=np.int32).ravel(),
                      np.ascontiguousarray(mesh.face_cells, dtype=np.int32).ravel(),
                      np.ascontiguousarray(mesh.face_bc, dtype=np.int32)]
        xy, cp, cn, fn, fc, fb = self._keep
        self.h = lib().ora_create(mesh.n_nodes, _dp(xy), mesh.n_cells, _ip(cp), _ip(cn),
                                  mesh.n_faces, _ip(fn), _ip(fc), _ip(fb), C.byref(self._f))
        if not self.h:
            raise MemoryError("ora_create failed")
        self.N, self.Nf = mesh.n_cells, mesh.n_faces

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().ora_destroy(h)
            self.h = None

    def set_W(self, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == (5, self.N)
        lib().ora_set_W(self.h, _dp(W))

    def iterate(self, n=1):
        return lib().ora_iterate(self.h, n)

    def get(self, which):
        shapes = {ORA_W: (5, self.N), ORA_GRAD: (4, 2, self.N), ORA_PHI: (4, self.N),
                  ORA_LAMBDA_F: (self.Nf,), ORA_LAMBDA_C: (self.N,), ORA_FLUX: (6, self.Nf),
                  ORA_RES: (5, self.N), ORA_DWSTAR: (5, self.N), ORA_DW: (5, self.N),
                  ORA_GHOST: (5, self.Nf), ORA_GEOM_CELL: (4, self.N), ORA_GEOM_FACE: (5, self.Nf)}
        out = np.zeros(shapes[which])
        if lib().ora_get(self.h, which, _dp(out)):
            raise ValueError(which)
        return out

    def scalars(self):
        o = np.zeros(len(SCALARS))
        lib().ora_get_scalars(self.h, _dp(o))
        return dict(zip(SCALARS, o.tolist()))

    def set_scalars(self, d):
        o = np.zeros(len(SCALARS))
        lib().ora_get_scalars(self.h, _dp(o))
        for k, v in d.items():
            o[SCALARS.index(k)] = v
        lib().ora_set_scalars(self.h, _dp(o))
