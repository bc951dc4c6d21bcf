"""Pins of the oracle's Spalart-Allmaras model (Section II.C, Eq. 26-30 and the source of
Eq. 28a) against facts that do not come from the oracle's own formulas:

  * the source alone: in the log layer (nu~ = kappa u_tau d, S~ = u_tau / (kappa d), so
    r = 1) the wall function is fw(1) = 1 and production minus destruction equals minus
    the diffusion, Sr d^2 / nu~^2 = -(1 + cb2) / sigma -- the relation that defines cw1;
    fw saturates at (1 + cw3^6)^(1/6) once r is clipped at 10; fv1(cv1) = 1/2; the 2012
    clipping of S~ is continuous where it switches on and tends to (1 - cv3) omega;
  * the whole discrete residual: on a stretched wall mesh carrying the log-layer profile
    the SA residual M[4] vanishes up to a discretisation error that falls under mesh
    refinement; for nu~ = c y^2 with the source off, M[4] / Omega tends to the analytic
    diffusion (6 + 4 cb2) c^2 y^2 / sigma of Eq. 26's diffusion term, which is where the
    anti-diffusion part of Eq. 30 enters;
  * conservation: the inviscid and viscous SA face fluxes telescope; what is left on a
    face is the anti-diffusion part alone.
"""
import math

import numpy as np
import pytest

import oracle as O
from igks_inputs import fields as F
from igks_inputs import meshgen as G

# the model's published constants (SA-noft2 with the 2012 S~ clipping)
CB1, CB2, SIGMA, KAPPA = 0.1355, 0.622, 2.0 / 3.0, 0.41
CW3, CV1, CV2, CV3 = 2.0, 7.1, 0.7, 0.9


def test_log_layer_balance_of_the_source():
    u_tau = 0.05
    for d in (1e-4, 1e-3, 3e-2):
        nut = KAPPA * u_tau * d
        omega = u_tau / (KAPPA * d)
        s = O.sa_source(nut, 1e-18, omega, d)     # nu -> 0: fv2 -> 0, S~ -> omega
        assert abs(s["r"] - 1.0) <= 1e-11
        assert abs(s["fw"] - 1.0) <= 1e-10
        assert abs(s["Sr"] * d * d / (nut * nut) + (1.0 + CB2) / SIGMA) <= 1e-9 * (1.0 + CB2) / SIGMA


def test_wall_function_saturates_once_r_is_clipped():
    d, nut = 1e-3, 2e-5
    base = nut / (KAPPA ** 2 * d * d)          # omega that makes r = 1 when fv2 -> 0
    fw_sat = (1.0 + CW3 ** 6) ** (1.0 / 6.0)
    clipped = [O.sa_source(nut, 1e-18, base / k, d) for k in (20.0, 200.0, 2e4)]
    for s in clipped:
        assert s["r"] == 10.0
        assert abs(s["fw"] - fw_sat) <= 1e-14
    # below the clip fw rises monotonically with r, from 0 at r = 0
    fws = [O.sa_source(nut, 1e-18, base * k, d)["fw"] for k in (1e6, 4.0, 2.0, 1.0, 0.7, 0.5)]
    assert fws[0] < 1e-5
    assert all(a < b for a, b in zip(fws, fws[1:]))
    assert fws[-1] < fw_sat


def test_fv1_is_one_half_at_cv1_and_limits():
    nu = 1e-5
    assert abs(O.sa_source(CV1 * nu, nu, 1.0, 1.0)["fv1"] - 0.5) <= 1e-15
    s0 = O.sa_source(0.0, nu, 1.0, 1.0)
    assert s0["fv1"] == 0.0 and s0["fv2"] == 1.0
    big = O.sa_source(1e8 * nu, nu, 1.0, 1.0)
    assert abs(big["fv1"] - 1.0) <= 1e-15 and 0.0 < big["fv2"] <= 2e-8


def test_s_tilde_clipping_is_continuous_and_positive():
    nu, d = 1e-5, 1e-3
    nut = 5.0 * nu                                  # chi = 5: fv2 < 0, S-bar < 0
    big = 1e7
    sbar = O.sa_source(nut, nu, big, d)["S_tilde"] - big    # unclipped branch: S~ = omega + S-bar
    assert sbar < 0.0
    w_star = -sbar / CV2                            # the clipping switches on below this omega
    above = O.sa_source(nut, nu, w_star * (1 + 1e-12), d)["S_tilde"]
    below = O.sa_source(nut, nu, w_star * (1 - 1e-12), d)["S_tilde"]
    assert abs(above - below) <= 1e-9 * above
    assert abs(above / w_star - (1.0 - CV2)) <= 1e-9
    # deep in the clipped branch S~ / omega -> 1 - cv3, and S~ stays positive throughout
    tiny = w_star * 1e-9
    assert abs(O.sa_source(nut, nu, tiny, d)["S_tilde"] / tiny - (1.0 - CV3)) <= 1e-8
    for k in np.geomspace(1e-6, 1e2, 60):
        assert O.sa_source(nut, nu, w_star * k, d)["S_tilde"] > 0.0


def _wall_mesh(ratio, first=1e-4, top=0.06, nx=8):
    ny = int(math.ceil(math.log(1.0 + top * (ratio - 1.0) / first) / math.log(ratio)))
    return G.flat_plate_quads(nx, ny, ratio, xmin=0.0, xmax=0.02, height=first * (ratio ** ny - 1) / (ratio - 1)), ny


def _sa_flow(re=1e14):
    fl = F.turbulent_plate_flow()
    fl.reynolds = re
    return fl


def _state(m, fl, U, nut):
    p = 1.0 / (F.GAMMA * fl.mach ** 2)
    W = np.zeros((5, m.n_cells))
    W[0] = 1.0
    W[1] = U
    W[3] = p / (F.GAMMA - 1.0) + 0.5 * U * U
    W[4] = nut
    return W


def _log_layer_error(ratio):
    """max |M[4]| / (Omega cb1 u_tau^2) over the cells clear of the domain edges, for the
    log-layer state U = 1 + (u_tau/kappa) ln(y/y1), nu~ = kappa u_tau y on a wall mesh."""
    m, ny = _wall_mesh(ratio)
    fl = _sa_flow()
    o = O.Oracle(m, fl)
    gc = o.get(O.ORA_GEOM_CELL)
    area, yc, wd = gc[0], gc[2], gc[3]
    assert np.allclose(wd, yc, rtol=1e-12)          # the wall distance of these cells is y
    u_tau = 0.04
    U = 1.0 + u_tau / KAPPA * np.log(yc / yc.min())
    o.set_W(_state(m, fl, U, KAPPA * u_tau * yc))
    o.iterate(1)
    M4 = o.get(O.ORA_RES)[4]
    nx = 8
    j = np.arange(m.n_cells) // nx
    i = np.arange(m.n_cells) % nx
    # the same band of the layer on every mesh, clear of the top rows and the side edges;
    # there the rows grow by about ratio - 1 of their height
    sel = (yc >= 0.01) & (yc <= 0.03) & (i >= 2) & (i <= nx - 3)
    assert sel.sum() >= 4 * 4
    return np.max(np.abs(M4[sel]) / (area[sel] * CB1 * u_tau ** 2))


def test_log_layer_residual_vanishes_under_refinement():
    errs = [_log_layer_error(r) for r in (1.2, 1.1, 1.05)]
    # O((r - 1)^2): the face averages and the least-squares shear on a stretched mesh
    assert errs[0] < 0.5, errs
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 2.5, errs


def _quadratic_diffusion_error(n):
    m = G.tiny_quads(n, n, bcs=("farfield", "farfield"))   # no wall: d = infinity, no source
    fl = _sa_flow()
    o = O.Oracle(m, fl)
    gc = o.get(O.ORA_GEOM_CELL)
    area, yc = gc[0], gc[2]
    c = 1e-3
    o.set_W(_state(m, fl, np.ones(m.n_cells), c * (yc + 0.5) ** 2))   # y + 1/2 > 0 everywhere
    o.iterate(1)
    M4 = o.get(O.ORA_RES)[4]
    j = np.arange(m.n_cells) // n
    i = np.arange(m.n_cells) % n
    sel = (yc >= 0.25) & (yc <= 0.75) & (i >= 1) & (i <= n - 2)    # the same band on every mesh
    exact = (6.0 + 4.0 * CB2) * c * c * (yc + 0.5) ** 2 / SIGMA
    return np.max(np.abs(M4[sel] / area[sel] - exact[sel]) / exact[sel])


def test_quadratic_nu_tilde_diffusion_matches_the_pde():
    e = [_quadratic_diffusion_error(n) for n in (8, 16, 32)]
    assert e[0] < 0.01, e
    assert e[1] < e[0] / 3.5 and e[2] < e[1] / 3.5, e      # second order


@pytest.mark.parametrize("uniform_velocity", [True, False])
def test_sa_face_fluxes_are_conservative_but_for_the_anti_diffusion(uniform_velocity):
    m = G.flat_plate_hybrid(nx=16, nq=6, ntri_rows=5, first=1e-3, seed=2)
    m = G.Mesh(m.xy, m.cell_ptr, m.cell_nodes, m.face_nodes, m.face_cells,
               np.where(m.face_cells[:, 1] < 0, G.BC_FARFIELD, 0).astype(np.int32), m.name)
    fl = _sa_flow(re=2e4)
    o = O.Oracle(m, fl)
    W = F.perturbed_state(m, fl, seed=7, amp=0.1)
    if uniform_velocity:
        W = F.uniform_state(m, fl)
        W[4] = F.perturbed_state(m, fl, seed=7, amp=0.1)[4] * (1.0 + 0.5 * np.sin(3.0 * np.arange(m.n_cells)))
    o.set_W(W)
    o.iterate(1)
    Fx = o.get(O.ORA_FLUX)
    M4 = o.get(O.ORA_RES)[4]
    gc = o.get(O.ORA_GEOM_CELL)
    gf = o.get(O.ORA_GEOM_FACE)
    inner = m.face_cells[:, 1] >= 0
    l, r = m.face_cells[inner, 0], m.face_cells[inner, 1]
    S, nx, ny = gf[0, inner], gf[1, inner], gf[2, inner]
    dn = np.abs((gc[1, r] - gc[1, l]) * nx + (gc[2, r] - gc[2, l]) * ny)
    dnu = W[4, r] - W[4, l]
    # Eq. 30: anti-diffusion -cb2/sigma nu~_i grad_n nu~ to each side, gradient taken from
    # that side; inviscid and viscous parts are equal and opposite on the two sides
    ad_sum = -CB2 / SIGMA * (W[4, l] * dnu / dn + W[4, r] * (-dnu) / dn) * S
    left = Fx[4, inner] + Fx[5, inner] - ad_sum
    scale = np.abs(Fx[4:6, inner]).max()
    assert np.abs(left).max() <= 1e-12 * scale
    if uniform_velocity:
        # no shear and no wall: the source vanishes, and the gathered residual is the sum of
        # the face terms each cell receives
        tot = M4.sum()
        ref = Fx[4].sum() + Fx[5, inner].sum()
        assert abs(tot - ref) <= 1e-12 * np.abs(Fx[4:6]).sum()
