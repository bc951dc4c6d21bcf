"""Pins of the oracle's whole iteration against invariants and independent solves.

  * geometry: cells close (sum n S = 0), areas add up to the domain,
  * free stream is preserved to round-off on a mesh closed by free-stream faces (Section II.E),
  * discrete conservation: interior face fluxes telescope (Eq. 15-16),
  * the two LU-SGS sweeps equal a dense direct solve of the factored system
    (L + D) D^-1 (D + U) dW = M of Eq. 22, the blocks built from the textbook Euler
    Jacobian, in the linear regime (mean flow) and exactly (SA scalar system),
  * rotating mesh and free stream leaves every scalar field unchanged,
  * the Barth-Jespersen reading of Eq. 9 keeps reconstructed vertex values inside the
    neighbourhood's range.
"""
import math

import numpy as np
import pytest

import oracle as O
from igks_inputs import fields as F
from igks_inputs import meshgen as G

GAM = 1.4


def _all_farfield(mesh):
    m = G.Mesh(mesh.xy, mesh.cell_ptr, mesh.cell_nodes, mesh.face_nodes, mesh.face_cells,
               np.where(mesh.face_cells[:, 1] < 0, G.BC_FARFIELD, 0).astype(np.int32), mesh.name)
    return m


def test_geometry_closes():
    m = G.flat_plate_hybrid(nx=16, nq=6, ntri_rows=5, first=1e-3, seed=2)
    o = O.Oracle(m, F.laminar_plate_flow())
    gc = o.get(O.ORA_GEOM_CELL)
    gf = o.get(O.ORA_GEOM_FACE)
    assert abs(gc[0].sum() - 1.5) < 1e-13
    S, nx, ny = gf[0], gf[1], gf[2]
    sx = np.zeros(m.n_cells); sy = np.zeros(m.n_cells)
    np.add.at(sx, m.face_cells[:, 0], nx * S); np.add.at(sy, m.face_cells[:, 0], ny * S)
    inner = m.face_cells[:, 1] >= 0
    np.add.at(sx, m.face_cells[inner, 1], -nx[inner] * S[inner])
    np.add.at(sy, m.face_cells[inner, 1], -ny[inner] * S[inner])
    assert np.abs(sx).max() < 1e-14 and np.abs(sy).max() < 1e-14
    # normals point out of the left cell
    dx = gf[3] - gc[1][m.face_cells[:, 0]]
    dy = gf[4] - gc[2][m.face_cells[:, 0]]
    assert np.all(dx * nx + dy * ny > 0)


@pytest.mark.parametrize("sa_on", [0, 1])
def test_free_stream_preserved(sa_on):
    m = _all_farfield(G.flat_plate_hybrid(nx=24, nq=8, ntri_rows=8, first=1e-4, seed=5))
    fl = F.turbulent_plate_flow() if sa_on else F.laminar_plate_flow()
    fl.aoa_deg = 17.0
    o = O.Oracle(m, fl)
    o.iterate(1)
    M = o.get(O.ORA_RES)
    Fx = o.get(O.ORA_FLUX)
    dt = o.scalars()["dt"]
    scale = np.abs(Fx[:4]).max(axis=1) / dt
    assert np.all(np.abs(M[:4]).max(axis=1) <= 1e-12 * scale.max())
    if sa_on:
        W = o.get(O.ORA_W)
        assert np.abs(W[4] - fl.nut_ratio_inf / fl.reynolds).max() < 1e-12 * fl.nut_ratio_inf / fl.reynolds
    dW = o.get(O.ORA_DW)
    assert np.abs(dW[:4]).max() < 1e-12


def test_conservation_telescopes():
    m = G.laminar_plate()
    fl = F.laminar_plate_flow()
    o = O.Oracle(m, fl)
    o.set_W(F.perturbed_state(m, fl, seed=3))
    o.iterate(1)
    M = o.get(O.ORA_RES)
    Fx = o.get(O.ORA_FLUX)
    dt = o.scalars()["dt"]
    bnd = m.face_cells[:, 1] < 0
    total = M[:4].sum(axis=1) * dt + Fx[:4, bnd].sum(axis=1)
    scale = np.abs(Fx[:4]).sum(axis=1)
    assert np.all(np.abs(total) <= 1e-13 * scale)


def _euler_jacobian(W, nx, ny):
    """Textbook Jacobian d(F.n)/dW of the 2D Euler flux, W = (rho, rho u, rho v, rho E)."""
    rho, u, v = W[0], W[1] / W[0], W[2] / W[0]
    E = W[3] / rho
    g1 = GAM - 1.0
    q2 = 0.5 * (u * u + v * v)
    vn = u * nx + v * ny
    H = GAM * E - g1 * q2
    return np.array([
        [0.0, nx, ny, 0.0],
        [g1 * q2 * nx - u * vn, vn - (GAM - 2) * u * nx, u * ny - g1 * v * nx, g1 * nx],
        [g1 * q2 * ny - v * vn, v * nx - g1 * u * ny, vn - (GAM - 2) * v * ny, g1 * ny],
        [vn * (g1 * q2 - H), H * nx - g1 * u * vn, H * ny - g1 * v * vn, GAM * vn],
    ])


@pytest.mark.parametrize("mesh_fn", [lambda: G.triangle_fan(5), lambda: G.tiny_quads(3, 2, skew=0.3, seed=4),
                                     lambda: G.mixed_polygons()])
def test_lusgs_equals_dense_factored_solve(mesh_fn):
    m = _all_farfield(mesh_fn())
    fl = F.turbulent_plate_flow()
    fl.reynolds = 500.0
    fl.cfl_init = 7.0
    N = m.n_cells
    errs = []
    for amp in (1e-5, 1e-6):
        o = O.Oracle(m, fl)
        W = F.perturbed_state(m, fl, seed=11, amp=amp)
        W[4] = fl.nut_ratio_inf / fl.reynolds * (1 + 0.3 * np.sin(np.arange(N)))
        o.set_W(W)
        o.iterate(1)
        M = o.get(O.ORA_RES)
        dW = o.get(O.ORA_DW)
        lamf = o.get(O.ORA_LAMBDA_F)
        Lam = o.get(O.ORA_LAMBDA_C)
        gc = o.get(O.ORA_GEOM_CELL)
        gf = o.get(O.ORA_GEOM_FACE)
        cfl = o.scalars()["cfl"]
        area = gc[0]
        D = area / (cfl * area / Lam) + Lam
        Lm = np.zeros((4 * N, 4 * N)); Um = np.zeros((4 * N, 4 * N)); Dm = np.zeros((4 * N, 4 * N))
        for i in range(N):
            Dm[4 * i:4 * i + 4, 4 * i:4 * i + 4] = D[i] * np.eye(4)
        for f in range(m.n_faces):
            l, r = m.face_cells[f]
            if r < 0:
                continue
            S, nx, ny = gf[0, f], gf[1, f], gf[2, f]
            for (i, j, sg) in ((l, r, 1.0), (r, l, -1.0)):
                B = 0.5 * S * (_euler_jacobian(W[:, j], sg * nx, sg * ny) - lamf[f] * np.eye(4))
                (Lm if j < i else Um)[4 * i:4 * i + 4, 4 * j:4 * j + 4] += B
        A = (Lm + Dm) @ np.linalg.inv(Dm) @ (Dm + Um)
        rhs = M[:4].T.ravel()
        x = np.linalg.solve(A, rhs).reshape(N, 4).T
        errs.append(np.abs(x - dW[:4]).max() / np.abs(dW[:4]).max())
        # SA: a linear scalar system with frozen coefficients (reading of Eq. 31-32)
        nu = np.array([O.viscosity(fl, W[0, i] / (2 * (GAM - 1) * (W[3, i] - 0.5 * (W[1, i] ** 2 + W[2, i] ** 2) / W[0, i])))
                       / W[0, i] for i in range(N)])
        a = np.zeros((N, N))
        a[np.arange(N), np.arange(N)] = area / (cfl * area / Lam)
        cb2, sig = 0.622, 2.0 / 3.0
        for f in range(m.n_faces):
            l, r = m.face_cells[f]
            S, nx, ny = gf[0, f], gf[1, f], gf[2, f]
            if r < 0:
                # ghost: far field free stream (its increment is zero in both sweeps)
                Wg = o.get(O.ORA_GHOST)[:, f]
                pairs = ((l, None, 1.0, Wg),)
            else:
                pairs = ((l, r, 1.0, None), (r, l, -1.0, None))
            for (i, j, sg, Wg) in pairs:
                Wj = W[:, j] if j is not None else Wg
                nuj = nu[j] if j is not None else O.viscosity(
                    fl, Wj[0] / (2 * (GAM - 1) * (Wj[3] - 0.5 * (Wj[1] ** 2 + Wj[2] ** 2) / Wj[0]))) / Wj[0]
                cj = gc[1:3, j] if j is not None else None
                if j is None:
                    d = 2 * abs((gf[3, f] - gc[1, i]) * nx + (gf[4, f] - gc[2, i]) * ny)
                else:
                    d = abs((cj[0] - gc[1, i]) * nx + (cj[1] - gc[2, i]) * ny)
                vni = (W[1, i] * sg * nx + W[2, i] * sg * ny) / W[0, i]
                vnj = (Wj[1] * sg * nx + Wj[2] * sg * ny) / Wj[0]
                kap = (nu[i] + nuj + (1 + cb2) * (W[4, i] + Wj[4])) / (2 * sig)
                a[i, i] += S * (max(vni, 0.0) + kap / d)
                if j is not None:
                    a[i, j] += S * (min(vnj, 0.0) - kap / d)
        La = np.tril(a, -1); Ua = np.triu(a, 1); Da = np.diag(np.diag(a))
        xs = np.linalg.solve((La + Da) @ np.linalg.inv(Da) @ (Da + Ua), M[4])
        assert np.allclose(xs, dW[4], rtol=1e-11, atol=1e-12 * np.abs(dW[4]).max())
    # mean flow: the sweeps use nonlinear flux differences, equal to the Jacobian form up
    # to O(dW^2): the mismatch must be small and shrink with the perturbation
    assert errs[0] < 1e-3 and errs[1] < errs[0] / 5, errs


def test_rotational_invariance():
    base = G.flat_plate_hybrid(nx=12, nq=4, ntri_rows=4, first=1e-3, seed=9)
    fl = F.turbulent_plate_flow()
    fl.reynolds = 2e4
    W0 = F.perturbed_state(base, fl, seed=2)
    out = []
    for ang in (0.0, 37.0):
        c, s = math.cos(math.radians(ang)), math.sin(math.radians(ang))
        R = np.array([[c, -s], [s, c]])
        m = G.Mesh(base.xy @ R.T, base.cell_ptr, base.cell_nodes, base.face_nodes, base.face_cells,
                   base.face_bc, base.name)
        f2 = F.turbulent_plate_flow(); f2.reynolds = fl.reynolds; f2.aoa_deg = ang
        W = W0.copy()
        W[1], W[2] = c * W0[1] - s * W0[2], s * W0[1] + c * W0[2]
        o = O.Oracle(m, f2)
        o.set_W(W)
        o.iterate(2)
        Wn = o.get(O.ORA_W)
        out.append(np.stack([Wn[0], Wn[3], np.hypot(Wn[1], Wn[2]), Wn[4]]))
    a, b = out
    scale = np.abs(a).max(axis=1, keepdims=True)
    assert np.all(np.abs(a - b) <= 1e-11 * scale)


def test_barth_jespersen_bounds_vertex_values():
    m = G.flat_plate_hybrid(nx=20, nq=6, ntri_rows=6, first=1e-3, seed=4)
    fl = F.laminar_plate_flow()
    fl.limiter = F.LIMITER_BJ
    o = O.Oracle(m, fl)
    W = F.perturbed_state(m, fl, seed=6, amp=0.2)
    W[0, 50] *= 1.5    # a local extremum: the limiter must flatten that cell
    o.set_W(W)
    o.iterate(1)
    grad = o.get(O.ORA_GRAD)
    phi = o.get(O.ORA_PHI)
    gc = o.get(O.ORA_GEOM_CELL)
    ghost = o.get(O.ORA_GHOST)
    assert phi.min() >= 0.0 and phi.max() <= 1.0
    assert phi[0, 50] == 0.0
    for i in range(m.n_cells):
        faces = np.where((m.face_cells[:, 0] == i) | (m.face_cells[:, 1] == i))[0]
        for v in range(4):
            nb = []
            for f in faces:
                l, r = m.face_cells[f]
                nb.append(W[v, r if l == i else l] if r >= 0 else ghost[v, f])
            lo, hi = min(min(nb), W[v, i]), max(max(nb), W[v, i])
            for nd in m.cell_node_list(i):
                wv = W[v, i] + phi[v, i] * (grad[v, 0, i] * (m.xy[nd, 0] - gc[1, i]) + grad[v, 1, i] * (m.xy[nd, 1] - gc[2, i]))
                tol = 1e-12 * max(abs(hi), abs(lo))
                assert lo - tol <= wv <= hi + tol


def test_wall_ghost_face_velocity_zero():
    m = G.laminar_plate()
    fl = F.laminar_plate_flow()
    o = O.Oracle(m, fl)
    W = F.perturbed_state(m, fl, seed=1)
    o.set_W(W)
    o.iterate(1)
    gh = o.get(O.ORA_GHOST)
    wall = np.where(m.face_bc == G.BC_WALL)[0]
    l = m.face_cells[wall, 0]
    assert np.allclose(gh[1, wall] + W[1, l], 0.0) and np.allclose(gh[2, wall] + W[2, l], 0.0)
    assert np.allclose(gh[0, wall], W[0, l]) and np.allclose(gh[3, wall], W[3, l])
    sym = np.where(m.face_bc == G.BC_SYMMETRY)[0]
    # symmetry faces of the plate are horizontal: normal momentum (y) flips
    ls = m.face_cells[sym, 0]
    assert np.allclose(gh[2, sym], -W[2, ls]) and np.allclose(gh[1, sym], W[1, ls])


def _venkat_phi(k, A=0.06):
    """Density limiter factor of the centre cell of a 3 x 3 box of unit-spaced quads whose
    density columns hold rho0 - A, rho0, rho0 + A/3: the least-squares slope is 2A/3 per
    cell, so the vertex excursions are +-A/3 against a neighbourhood range of +A/3 / -A."""
    m = G.tiny_quads(3, 3, bcs=("symmetry", "symmetry"))
    fl = F.laminar_plate_flow()
    fl.limiter = F.LIMITER_VENKAT
    fl.venkat_k = k
    W = F.uniform_state(m, fl)
    col = np.arange(m.n_cells) % 3
    W[0] = 1.0 + np.array([-A, 0.0, A / 3.0])[col]
    o = O.Oracle(m, fl)
    o.set_W(W)
    o.iterate(1)
    return o.get(O.ORA_PHI)


def test_venkatakrishnan_limiter_values_and_limits():
    """Venkatakrishnan's smooth limiter at the excursion ratio y = range / excursion: with
    K = 0 it is (y^2 + 2y)/(y^2 + y + 2), which is 3/4 at y = 1 and exceeds 1 only for y > 2
    (the factor is capped at 1); as K grows it tends to 1 (no limiting)."""
    phi = _venkat_phi(0.0)
    assert abs(phi[0, 4] - 0.75) <= 1e-14
    assert np.all(phi[1:, 4] == 1.0)               # uniform momentum and energy
    ks = [0.0, 0.5, 1.0, 3.0, 30.0]
    vals = [_venkat_phi(k)[0, 4] for k in ks]
    assert all(a < b for a, b in zip(vals, vals[1:]))
    assert 1.0 - vals[-1] < 1e-4


def test_venkatakrishnan_factors_stay_in_zero_one():
    m = G.flat_plate_hybrid(nx=20, nq=6, ntri_rows=6, first=1e-3, seed=4)
    fl = F.laminar_plate_flow()
    fl.limiter = F.LIMITER_VENKAT
    for k in (0.0, 0.3, 5.0):
        fl.venkat_k = k
        o = O.Oracle(m, fl)
        W = F.perturbed_state(m, fl, seed=6, amp=0.2)
        W[0, 50] *= 1.5
        o.set_W(W)
        o.iterate(1)
        phi = o.get(O.ORA_PHI)
        assert phi.min() >= 0.0 and phi.max() <= 1.0
        if k == 0.0:
            assert phi[0, 50] < 0.5          # the local extremum is limited


def test_viscous_spectral_radius_closed_form():
    """Two cells side by side: lambda_f = |Vbar . n| + cbar + 2 (mubar + mutbar) gamma /
    (rhobar Pr dn), with the means over the two cells (reading (ii) of the spectral radius
    of Eq. 20-21), Sutherland's law for mu and mu_t = rho nu~ fv1."""
    xy = np.array([[0, 0], [1, 0], [2, 0], [0, 0.5], [1, 0.5], [2, 0.5]], dtype=np.float64)
    m = G.build_mesh(xy, [[0, 1, 4, 3], [1, 2, 5, 4]], lambda a, b, xm, ym: G.BC_FARFIELD, name="two_cells")
    fl = F.turbulent_plate_flow()
    fl.reynolds = 300.0
    W = np.zeros((5, 2))
    prim = [(1.1, 0.7, -0.2, 19.0, 0.02), (0.9, 0.4, 0.3, 16.0, 0.05)]
    for c, (r, u, v, p, nut) in enumerate(prim):
        W[:, c] = [r, r * u, r * v, p / (GAM - 1) + 0.5 * r * (u * u + v * v), nut]
    o = O.Oracle(m, fl)
    o.set_W(W)
    o.iterate(1)
    lam = o.get(O.ORA_LAMBDA_F)
    f = int(np.nonzero(m.face_cells[:, 1] >= 0)[0][0])
    n = np.array([1.0, 0.0]) if m.face_cells[f, 0] == 0 else np.array([-1.0, 0.0])
    p_inf = 1 / (GAM * fl.mach ** 2)
    s = fl.s_suth / fl.t_ref
    mus, muts = [], []
    for (r, u, v, p, nut) in prim:
        tr = (p / r) / p_inf                          # T / T_inf
        mu = (1 / fl.reynolds) * tr ** 1.5 * (1 + s) / (tr + s)
        chi3 = (nut * r / mu) ** 3
        mus.append(mu)
        muts.append(r * nut * chi3 / (chi3 + 7.1 ** 3))
    (r0, u0, v0, p0, _), (r1, u1, v1, p1, _) = prim
    vbar = 0.5 * np.array([u0 + u1, v0 + v1])
    cbar = 0.5 * (math.sqrt(GAM * p0 / r0) + math.sqrt(GAM * p1 / r1))
    ref = abs(vbar @ n) + cbar + 2 * (0.5 * sum(mus) + 0.5 * sum(muts)) * GAM / (0.5 * (r0 + r1) * fl.prandtl * 1.0)
    assert abs(lam[f] - ref) <= 1e-13 * ref
    fl.visc_sr = 0
    o2 = O.Oracle(m, fl)
    o2.set_W(W)
    o2.iterate(1)
    assert abs(o2.get(O.ORA_LAMBDA_F)[f] - (abs(vbar @ n) + cbar)) <= 1e-14 * ref


def test_exactly_zero_residual_counts_as_converged():
    """Fluid at rest in a box closed by symmetry planes on an axis-aligned mesh: every face
    carries the pressure alone and each cell's fluxes cancel exactly, so the residual is
    exactly zero. The solve stops at once as converged and the CFL stays finite."""
    m = G.tiny_quads(6, 4, bcs=("symmetry", "symmetry"))
    fl = F.cavity_flow()
    o = O.Oracle(m, fl)
    o.set_W(F.rest_state(m, fl))
    assert o.iterate(5) == 1
    sc = o.scalars()
    assert sc["iter"] == 1 and sc["res_l2"] == 0.0 and sc["res_inf"] == 0.0
    assert math.isfinite(sc["cfl"]) and sc["cfl"] == fl.cfl_init


def test_zero_residual_after_a_nonzero_one_sends_the_cfl_to_its_cap():
    """Eq. 25 with a residual that vanished exactly: the ratio of the norms is infinite, so
    the CFL goes to its cap; after two vanishing residuals in a row it stays put."""
    m = G.tiny_quads(6, 4, bcs=("symmetry", "symmetry"))
    fl = F.cavity_flow()
    for prev, cfl_expected in ((3.5, fl.cfl_max), (0.0, 2345.0)):
        o = O.Oracle(m, fl)
        o.set_W(F.rest_state(m, fl))
        o.set_scalars({"iter": 7, "cfl": 2345.0, "res_inf_prev": prev, "res_l2_first": 1.0})
        assert o.iterate(1) == 1
        sc = o.scalars()
        assert sc["res_inf"] == 0.0 and sc["cfl"] == cfl_expected


def test_venkatakrishnan_epsilon_is_k_h_cubed():
    """Venkatakrishnan's threshold eps^2 = (K h)^3 with h = sqrt(Omega): at the excursion
    ratio y = 1 the factor is (3 d^2 + eps^2) / (4 d^2 + eps^2), d the vertex excursion
    (A/3 = 0.02 here, h = 1/3)."""
    d2 = 0.02 ** 2
    for k in (0.3, 0.5, 1.0):
        e2 = (k / 3.0) ** 3
        assert abs(_venkat_phi(k)[0, 4] - (3 * d2 + e2) / (4 * d2 + e2)) <= 1e-13
