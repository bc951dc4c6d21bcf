"""Flow conditions and seeded initial fields (inputs shared by the oracle and the CUDA path).

Non-dimensionalisation used throughout (the paper leaves it open): free-stream density 1,
free-stream speed 1, reference length 1, so p_inf = 1/(gamma Ma^2) and mu_inf = 1/Re.
gamma = (K+4)/(K+2) = 1.4 with K = 3 internal degrees of freedom (Eq. 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict

import numpy as np

K_INTERNAL = 3
GAMMA = (K_INTERNAL + 4.0) / (K_INTERNAL + 2.0)

LIMITER_NONE, LIMITER_BJ, LIMITER_VENKAT = 0, 1, 2


@dataclass
class Flow:
    mach: float = 0.15
    reynolds: float = 1e5          # per unit reference length
    aoa_deg: float = 0.0
    prandtl: float = 0.72
    t_ref: float = 288.15          # free-stream temperature [K] for Sutherland's law
    s_suth: float = 110.4          # Sutherland constant [K]
    sa_on: int = 0
    nut_ratio_inf: float = 3.0     # free-stream nu_tilde / nu
    cfl_exp: float = 1.0           # CFL of the flux time step (Eq. 23)
    cfl_init: float = 100.0        # implicit CFL (Eq. 24) at the first iteration
    cfl_min: float = 100.0
    cfl_max: float = 100.0         # Eq. 25 result is clamped to [cfl_min, cfl_max]
    res_target: float = 1e-10      # relative L2 of the density residual
    limiter: int = LIMITER_NONE
    venkat_k: float = 5.0
    c_num: float = 1.0             # numerical collision-time coefficient
    visc_sr: int = 0               # add the viscous spectral radius to lambda_f
    eq40_target: float = 0.0       # if > 0, also stop at the Eq. 40 ratio <= this (paper: 3e-8)
    scheme: int = 0                # 0 implicit (LU-SGS, Eq. 22), 1 explicit (Eq. 15)

    def as_dict(self) -> dict:
        return asdict(self)


def laminar_plate_flow() -> Flow:
    return Flow(mach=0.15, reynolds=1e5, sa_on=0, cfl_init=100.0, cfl_min=100.0,
                cfl_max=100.0, visc_sr=0)


def turbulent_plate_flow() -> Flow:
    return Flow(mach=0.2, reynolds=5e6, sa_on=1, nut_ratio_inf=3.0, cfl_init=10.0,
                cfl_min=10.0, cfl_max=1000.0, visc_sr=1)


def naca_flow(mach: float = 0.15, reynolds: float = 6e6, aoa_deg: float = 10.0) -> Flow:
    # the airfoils use the limiter of Eq. 9 (Barth-Jespersen reading): unlimited, the wall
    # cells at the leading- and trailing-edge stagnation regions of these O-meshes fall
    # into an oscillation below Ma ~0.2 that stops the residual from converging
    return Flow(mach=mach, reynolds=reynolds, aoa_deg=aoa_deg, sa_on=1, nut_ratio_inf=3.0,
                cfl_init=10.0, cfl_min=10.0, cfl_max=1000.0, visc_sr=1, limiter=LIMITER_BJ)


def _node_average_centres(mesh) -> np.ndarray:
    cnt = np.diff(mesh.cell_ptr)
    owner = np.repeat(np.arange(mesh.n_cells), cnt)
    c = np.zeros((mesh.n_cells, 2))
    np.add.at(c, owner, mesh.xy[mesh.cell_nodes])
    return c / cnt[:, None]


def freestream_primitives(flow: Flow):
    a = math.radians(flow.aoa_deg)
    return 1.0, math.cos(a), math.sin(a), 1.0 / (GAMMA * flow.mach ** 2)


def perturbed_state(mesh, flow: Flow, seed: int = 0, amp: float = 0.05) -> np.ndarray:
    """Seeded smooth perturbation of the free stream, as conserved SoA [5, n_cells]
    (rho, rho U, rho V, rho E, nu_tilde). Used as the common start of parity checks so
    that every flux, gradient and sweep term is non-trivial."""
    rng = np.random.default_rng(seed)
    xc = _node_average_centres(mesh)
    x, y = xc[:, 0], xc[:, 1]
    r0, u0, v0, p0 = freestream_primitives(flow)
    modes = rng.uniform(0.5, 3.0, size=(5, 2))
    phase = rng.uniform(0, 2 * math.pi, size=(5,))

    def wave(k):
        return np.sin(modes[k, 0] * 2 * math.pi * x + phase[k]) * np.cos(modes[k, 1] * 2 * math.pi * y)

    rho = r0 * (1.0 + amp * wave(0))
    u = u0 * (1.0 + 2 * amp * wave(1)) + amp * 0.5 * wave(2)
    v = v0 + amp * 0.5 * wave(3)
    p = p0 * (1.0 + amp * wave(4))
    nu_inf = 1.0 / flow.reynolds
    nut = flow.nut_ratio_inf * nu_inf * (1.0 + 0.5 * np.abs(wave(2))) if flow.sa_on else np.zeros_like(x)
    W = np.empty((5, mesh.n_cells))
    W[0] = rho
    W[1] = rho * u
    W[2] = rho * v
    W[3] = p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)
    W[4] = nut
    return W


def uniform_state(mesh, flow: Flow) -> np.ndarray:
    r0, u0, v0, p0 = freestream_primitives(flow)
    W = np.empty((5, mesh.n_cells))
    W[0] = r0
    W[1] = r0 * u0
    W[2] = r0 * v0
    W[3] = p0 / (GAMMA - 1.0) + 0.5 * r0 * (u0 * u0 + v0 * v0)
    W[4] = flow.nut_ratio_inf / flow.reynolds if flow.sa_on else 0.0
    return W


def cavity_flow(scheme: int = 0) -> Flow:
    """Lid-driven cavity of the paper's first test: Re = 1000 on the lid speed and the
    cavity size, Ma = 0.1 sqrt(3), laminar; the lid moves with the free-stream velocity
    (AoA 0: along +x). Implicit CFL from 1000 by Eq. 25 up to 1e6, as the paper reports."""
    return Flow(mach=0.1 * math.sqrt(3.0), reynolds=1000.0, aoa_deg=0.0, sa_on=0, cfl_init=1000.0,
                cfl_min=1000.0, cfl_max=1e6, visc_sr=0, limiter=LIMITER_NONE, scheme=scheme)


def rest_state(mesh, flow: Flow) -> np.ndarray:
    """Fluid at rest with the free-stream density and pressure (the cavity's start)."""
    r0, _, _, p0 = freestream_primitives(flow)
    W = np.zeros((5, mesh.n_cells))
    W[0] = r0
    W[3] = p0 / (GAMMA - 1.0)
    return W
