"""Pins of the CPU oracle's building blocks against mathematics independent of it.

Each check below would fail on a plausible slip in the oracle (a dropped term, a wrong
sign or index, a transposed operand):
  * Maxwellian moments (Eq. 2) against high-precision quadrature,
  * the 4x4 moment systems of Eq. 101 against Gauss-Hermite cubature in five dimensions
    (u, v and the K = 3 internal components of xi) and against their closed-form solution,
  * the time weights of Eq. 13-14 against quadrature,
  * the interface flux (Eq. 4-14) in three limits with a textbook answer: uniform flow
    (exact Euler flux), the collisionless limit (kinetic flux-vector splitting) and the
    Navier-Stokes limit (Newtonian shear stress and Fourier heat flux with Pr = 0.72).
"""
import math

import numpy as np
import pytest

import oracle as O
from igks_inputs import fields as F

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40

K = 3
GAM = (K + 4) / (K + 2)


def _maxw_1d(U, lam):
    U = mpmath.mpf(U); lam = mpmath.mpf(lam)
    return lambda u: mpmath.sqrt(lam / mpmath.pi) * mpmath.exp(-lam * (u - U) ** 2)


@pytest.mark.parametrize("U,lam", [(0.0, 1.0), (0.7, 2.3), (-1.3, 0.4), (3.0, 0.035), (-0.2, 40.0)])
def test_moments_full_and_half_vs_quadrature(U, lam):
    g = _maxw_1d(U, lam)
    full = O.moments_full(U, lam)
    pos = O.moments_half(U, lam, +1)
    neg = O.moments_half(U, lam, -1)
    for n in range(10):
        ref_f = mpmath.quad(lambda u: u ** n * g(u), [-mpmath.inf, U, mpmath.inf])
        ref_p = mpmath.quad(lambda u: u ** n * g(u), [0, mpmath.inf])
        ref_n = mpmath.quad(lambda u: u ** n * g(u), [-mpmath.inf, 0])
        scale = float(mpmath.quad(lambda u: abs(u) ** n * g(u), [-mpmath.inf, 0, mpmath.inf]))
        assert abs(full[n] - float(ref_f)) <= 1e-13 * scale, (n, full[n], ref_f)
        assert abs(pos[n] - float(ref_p)) <= 1e-13 * scale, (n, pos[n], ref_p)
        assert abs(neg[n] - float(ref_n)) <= 1e-13 * scale, (n, neg[n], ref_n)
        assert abs(pos[n] + neg[n] - full[n]) <= 2e-14 * scale


@pytest.mark.parametrize("lam", [0.3, 1.0, 17.0])
def test_internal_moments_vs_quadrature(lam):
    # xi^2 = xi_1^2 + xi_2^2 + xi_3^2, each component a zero-mean Gaussian of Eq. 2
    g = _maxw_1d(0.0, lam)
    m = [mpmath.quad(lambda x: x ** (2 * k) * g(x), [-mpmath.inf, 0, mpmath.inf]) for k in range(4)]
    m2, m4, m6 = m[1], m[2], m[3]
    ref = [1.0, K * m2, K * m4 + K * (K - 1) * m2 ** 2,
           K * m6 + 3 * K * (K - 1) * m4 * m2 + K * (K - 1) * (K - 2) * m2 ** 3]
    got = O.moments_xi(lam)
    for k in range(4):
        assert abs(got[k] - float(ref[k])) <= 1e-14 * abs(float(ref[k]))


def _gauss_hermite_5d(U, V, lam, n=8):
    """Cubature nodes/weights for the normalised 5D Maxwellian of Eq. 2 (u, v, xi_1..3)."""
    x, w = np.polynomial.hermite.hermgauss(n)
    s = 1.0 / math.sqrt(lam)
    grids = np.meshgrid(*([x] * 5), indexing="ij")
    wts = np.ones_like(grids[0])
    for d in range(5):
        wts = wts * np.meshgrid(*([w] * 5), indexing="ij")[d]
    wts = wts.ravel() / math.pi ** 2.5
    u = U + s * grids[0].ravel()
    v = V + s * grids[1].ravel()
    xi2 = s * s * (grids[2].ravel() ** 2 + grids[3].ravel() ** 2 + grids[4].ravel() ** 2)
    psi = np.stack([np.ones_like(u), u, v, 0.5 * (u * u + v * v + xi2)])
    return psi, wts


@pytest.mark.parametrize("U,V,lam", [(0.0, 0.0, 1.0), (0.3, -0.8, 2.5), (-1.1, 0.4, 0.6), (0.05, 0.9, 35.0)])
def test_moment_matrix_vs_cubature(U, V, lam):
    psi, wts = _gauss_hermite_5d(U, V, lam)
    ref = (psi * wts) @ psi.T
    got = O.moment_matrix(U, V, lam)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_moment_solve_round_trip_and_closed_form():
    rng = np.random.default_rng(7)
    for _ in range(40):
        U, V = rng.uniform(-1.5, 1.5, 2)
        lam = math.exp(rng.uniform(-2, 4))
        b = rng.normal(size=4)
        a = O.moment_solve(U, V, lam, b)
        # round trip through independent cubature: <(a . psi) psi> = b
        psi, wts = _gauss_hermite_5d(U, V, lam)
        back = (psi * wts) @ (a @ psi)
        assert np.allclose(back, b, rtol=1e-10, atol=1e-11 * np.abs(b).max())
        # closed-form solution of the same Maxwellian moment system
        E2 = U * U + V * V + (K + 2) / (2 * lam)
        R4 = 2 * b[3] - E2 * b[0]
        R2 = b[1] - U * b[0]
        R3 = b[2] - V * b[0]
        a4 = 4 * lam * lam / (K + 2) * (R4 - 2 * U * R2 - 2 * V * R3)
        a3 = 2 * lam * R3 - V * a4
        a2 = 2 * lam * R2 - U * a4
        a1 = b[0] - U * a2 - V * a3 - 0.5 * a4 * E2
        cf = np.array([a1, a2, a3, a4])
        assert np.allclose(a, cf, rtol=1e-10, atol=1e-12 * np.abs(cf).max())


@pytest.mark.parametrize("x", [1e-3, 0.1, 1.0, 7.5, 60.0, 1e3])
def test_time_weights_vs_quadrature(x):
    tau = 1.3e-4
    dt = x * tau
    T = mpmath.mpf(tau)
    ints = [lambda t: 1 - mpmath.exp(-t / T),
            lambda t: T * (-1 + mpmath.exp(-t / T)) + t * mpmath.exp(-t / T),
            lambda t: T * (t / T - 1 + mpmath.exp(-t / T)),
            lambda t: mpmath.exp(-t / T),
            lambda t: -(t + T) * mpmath.exp(-t / T),
            lambda t: -T * mpmath.exp(-t / T)]
    q = O.time_weights(dt, tau)
    # rounding is measured against the size of the terms each closed form combines
    scales = [dt + tau, tau * (dt + tau), (dt + tau) ** 2, dt + tau, tau * (dt + tau), tau * tau]
    for k in range(6):
        ref = float(mpmath.quad(ints[k], [0, dt]))
        assert abs(q[k] - ref) <= 1e-13 * max(abs(ref), 1e-2 * scales[k]), (k, q[k], ref)


# ---------------------------------------------------------------------------------------
# interface flux limits
# ---------------------------------------------------------------------------------------

def _cons(rho, un, ut, p):
    return np.array([rho, rho * un, rho * ut, p / (GAM - 1) + 0.5 * rho * (un * un + ut * ut)])


def _flow(**kw):
    f = F.Flow(mach=0.2, reynolds=1e4, c_num=0.0)
    for k, v in kw.items():
        setattr(f, k, v)
    return f


@pytest.mark.parametrize("un,ut", [(0.3, 0.1), (-0.45, 0.7), (0.0, -0.2), (1.2, 0.0)])
def test_flux_uniform_is_exact_euler(un, ut):
    fl = _flow()
    W = _cons(1.1, un, ut, 20.0)
    z = np.zeros(4)
    dt = 2e-4
    Fx, heat = O.face_flux(fl, W, W, z, z, z, z, W, W, 0.01, 0.012, 0.0, dt)
    p = 20.0
    ref = np.array([1.1 * un, 1.1 * un * un + p, 1.1 * un * ut, (W[3] + p) * un]) * dt
    assert np.allclose(Fx, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())
    assert abs(heat) <= 1e-13 * np.abs(ref).max()


def test_flux_collisionless_limit_is_kfvs():
    """dt << tau, no slopes: f_cf -> g^l H[u] + g^r (1 - H[u]); F/dt is the kinetic
    flux-vector splitting flux, here integrated by quadrature over each half line."""
    fl = _flow(reynolds=1e-6, prandtl=1.0)   # huge collision time; BGK's own Pr = 1
    WL = _cons(1.0, 0.25, 0.3, 17.0)
    WR = _cons(0.8, -0.1, -0.2, 15.0)
    z = np.zeros(4)
    Fx, _ = O.face_flux(fl, WL, WR, z, z, z, z, WL, WR, 0.01, 0.01, 0.0, 1e-9)
    ref = np.zeros(4)
    for W, lo, hi in ((WL, 0, mpmath.inf), (WR, -mpmath.inf, 0)):
        rho, U, V = W[0], W[1] / W[0], W[2] / W[0]
        p = (GAM - 1) * (W[3] - 0.5 * rho * (U * U + V * V))
        lam = rho / (2 * p)
        g = _maxw_1d(U, lam)
        v2 = V * V + 1 / (2 * lam)            # <v^2>
        xi2 = K / (2 * lam)                   # <xi^2>
        ref[0] += rho * float(mpmath.quad(lambda u: u * g(u), [lo, hi]))
        ref[1] += rho * float(mpmath.quad(lambda u: u * u * g(u), [lo, hi]))
        ref[2] += rho * V * float(mpmath.quad(lambda u: u * g(u), [lo, hi]))
        ref[3] += rho * float(mpmath.quad(lambda u: 0.5 * u * (u * u + v2 + xi2) * g(u), [lo, hi]))
    assert np.allclose(Fx / 1e-9, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def _sutherland(fl, lam):
    lam_inf = GAM * fl.mach ** 2 / 2
    tr = lam_inf / lam
    s = fl.s_suth / fl.t_ref
    return (1 / fl.reynolds) * tr ** 1.5 * (1 + s) / (tr + s)


@pytest.mark.parametrize("ratio", [1e3, 1e5])
def test_flux_ns_limit_shear_stress(ratio):
    """Linear shear U_t = a x_n: the tangential momentum flux tends to -mu a dt as
    tau/dt -> 0 (Chapman-Enskog / Newtonian stress), with error O(tau/dt)."""
    fl = _flow(reynolds=1e3)
    rho, p, a = 1.0, 1 / (GAM * fl.mach ** 2), 0.8
    lam = rho / (2 * p)
    mu = _sutherland(fl, lam)
    tau = mu / p
    dt = ratio * tau
    d = 1e-3
    W = _cons(rho, 0.0, 0.0, p)
    sn = np.array([0.0, 0.0, rho * a, 0.0])
    z = np.zeros(4)
    WcL = _cons(rho, 0.0, -a * d, p)
    WcR = _cons(rho, 0.0, a * d, p)
    Fx, _ = O.face_flux(fl, W, W, sn, z, sn, z, WcL, WcR, d, d, 0.0, dt)
    ref = -mu * a * dt
    assert abs(Fx[2] - ref) <= 5.0 / ratio * abs(ref) + 1e-12 * abs(ref)
    # the mass flux stays zero
    assert abs(Fx[0]) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("ratio", [1e3, 1e5])
def test_flux_ns_limit_heat_flux_with_prandtl_fix(ratio):
    """Linear temperature T = T0 (1 + b x_n) at rest and uniform pressure: the energy
    flux tends to -(mu c_p / Pr) dT/dn dt, c_p = (K+4)/2 with R = 1 (lambda = 1/(2T))."""
    fl = _flow(reynolds=1e3, prandtl=0.72)
    p = 1 / (GAM * fl.mach ** 2)
    T0, b, d = p / 1.0, 0.5, 1e-3
    rho0 = p / T0

    def W_at(x):
        T = T0 * (1 + b * x)
        return _cons(p / T, 0.0, 0.0, p)
    W = W_at(0.0)
    # d(rho)/dn = -p T0 b / T0^2 at x=0; energy density is constant (p uniform, at rest)
    sn = np.array([-p * b / T0, 0.0, 0.0, 0.0])
    z = np.zeros(4)
    lam0 = rho0 / (2 * p)
    mu = _sutherland(fl, lam0)
    tau = mu / p
    dt = ratio * tau
    Fx, heat = O.face_flux(fl, W, W, sn, z, sn, z, W_at(-d), W_at(d), d, d, 0.0, dt)
    cp = (K + 4) / 2.0
    ref = -(mu * cp / fl.prandtl) * (T0 * b) * dt
    assert abs(Fx[3] - ref) <= 5.0 / ratio * abs(ref) + 1e-9 * abs(ref)
    # the unfixed (BGK, Pr = 1) heat flux is Pr times smaller
    assert abs(heat - ref * fl.prandtl) <= 5.0 / ratio * abs(ref)


# --- boundary conditions (Section II.E) -------------------------------------------------

def _ghosts_of_uniform(W0, bcs=("wall", "outflow"), flow=None):
    """Ghost states the oracle builds from a uniform interior state W0 on a 2 x 2 quad mesh
    whose bottom is `bcs[0]` and whose other sides are `bcs[1]`."""
    from igks_inputs import meshgen as G
    m = G.tiny_quads(2, 2, bcs=bcs)
    fl = flow or F.laminar_plate_flow()
    o = O.Oracle(m, fl)
    o.set_W(np.repeat(np.asarray(W0, dtype=np.float64)[:, None], m.n_cells, axis=1))
    o.iterate(1)
    return m, fl, o.get(O.ORA_GHOST)


def _conserved(r, u, v, p, nut=0.0):
    return [r, r * u, r * v, p / (F.GAMMA - 1.0) + 0.5 * r * (u * u + v * v), nut]


def _prim(W):
    r, u, v = W[0], W[1] / W[0], W[2] / W[0]
    return r, u, v, (F.GAMMA - 1.0) * (W[3] - 0.5 * r * (u * u + v * v))


def _outflow_faces(m):
    from igks_inputs import meshgen as G
    return np.nonzero((m.face_cells[:, 1] < 0) & (m.face_bc == G.BC_OUTFLOW))[0]


def _face_normal(m, f):
    a, b = m.face_nodes[f]
    d = m.xy[b] - m.xy[a]
    n = np.array([d[1], -d[0]])          # right of a -> b: out of the left cell
    return n / np.linalg.norm(n)


def test_free_stream_ghosts_hold_the_free_stream():
    """Free-stream boundary: the ghost is the free stream whatever the interior holds."""
    fl = F.laminar_plate_flow()
    r, u, v, p = 1.2, 0.6, -0.3, 1.3 / (F.GAMMA * fl.mach ** 2)
    m, fl, gh = _ghosts_of_uniform(_conserved(r, u, v, p), bcs=("wall", "farfield"), flow=fl)
    Winf = F.uniform_state(m, fl)[:, 0]
    far = np.nonzero(m.face_bc == 1)[0]
    assert len(far) > 0
    np.testing.assert_allclose(gh[:, far], np.repeat(Winf[:, None], len(far), axis=1), rtol=0, atol=1e-14 * Winf[3])


def test_outflow_ghost_of_the_free_stream_is_the_free_stream():
    fl = F.laminar_plate_flow()
    from igks_inputs import meshgen as G
    m0 = G.tiny_quads(2, 2, bcs=("wall", "outflow"))
    Winf = F.uniform_state(m0, fl)[:, 0]
    m, fl, gh = _ghosts_of_uniform(Winf, flow=fl)
    out = _outflow_faces(m)
    assert len(out) >= 4
    for f in out:
        np.testing.assert_allclose(gh[:, f], Winf, rtol=1e-14, atol=1e-14)


def test_outflow_ghost_passes_inside_values_and_averages_the_invariants():
    """Outflow boundary: density, pressure (through lambda) and tangential velocity come
    from inside; the normal velocity is the mean of the two Riemann invariants, so it
    moves by half of a change of the inside normal velocity and by 1/(gamma-1) of a change
    of the inside sound speed, and does not depend on the inside tangential velocity."""
    fl = F.laminar_plate_flow()
    g = F.GAMMA
    p_inf = 1.0 / (g * fl.mach ** 2)
    base = dict(r=1.1, u=0.8, v=0.15, p=1.04 * p_inf)

    def ghosts(**kw):
        q = dict(base, **kw)
        m, _, gh = _ghosts_of_uniform(_conserved(q["r"], q["u"], q["v"], q["p"]), flow=fl)
        return m, gh

    m, gh0 = ghosts()
    out = _outflow_faces(m)
    for f in out:
        n = _face_normal(m, f)
        t = np.array([-n[1], n[0]])
        r, u, v, p = _prim(gh0[:, f])
        assert abs(r - base["r"]) <= 1e-14
        assert abs(p - base["p"]) <= 1e-12 * base["p"]
        assert abs((u * t[0] + v * t[1]) - (base["u"] * t[0] + base["v"] * t[1])) <= 1e-13
    # responses of the normal velocity, by finite differences of the inside state
    eps = 1e-6
    for f in out:
        n = _face_normal(m, f)
        t = np.array([-n[1], n[0]])
        un0 = (gh0[1, f] * n[0] + gh0[2, f] * n[1]) / gh0[0, f]
        # inside normal velocity + eps
        m1, gh1 = ghosts(u=base["u"] + eps * n[0], v=base["v"] + eps * n[1])
        un1 = (gh1[1, f] * n[0] + gh1[2, f] * n[1]) / gh1[0, f]
        assert abs((un1 - un0) / eps - 0.5) < 1e-6
        # inside tangential velocity + eps: no change of the normal velocity
        m2, gh2 = ghosts(u=base["u"] + eps * t[0], v=base["v"] + eps * t[1])
        un2 = (gh2[1, f] * n[0] + gh2[2, f] * n[1]) / gh2[0, f]
        assert abs(un2 - un0) < 1e-12
        # inside sound speed c -> c (1 + eps) at fixed density: pressure scales by (1+eps)^2
        c0 = math.sqrt(g * base["p"] / base["r"])
        m3, gh3 = ghosts(p=base["p"] * (1 + eps) ** 2)
        un3 = (gh3[1, f] * n[0] + gh3[2, f] * n[1]) / gh3[0, f]
        assert abs((un3 - un0) / (c0 * eps) - 1.0 / (g - 1.0)) < 1e-5


def test_explicit_scheme_conserves_mass_and_energy_in_a_closed_mirror_box():
    """Eq. 15 is in flux form: on a box closed by symmetry planes (an exact mirror of the
    kinetic problem, so no mass or energy crosses them) total mass and energy stay fixed
    to round-off, step after step."""
    from igks_inputs import meshgen as G
    m = G.tiny_quads(6, 5, skew=0.3, seed=2, bcs=("symmetry", "symmetry"))
    fl = F.cavity_flow(scheme=1)
    o = O.Oracle(m, fl)
    W0 = F.perturbed_state(m, fl, seed=4, amp=0.05)
    o.set_W(W0)
    area = None
    for _ in range(4):
        assert o.iterate(1) == 0
        W = o.get(O.ORA_W)
        area = o.get(O.ORA_GEOM_CELL)[0]
        for v in (0, 3):
            tot0 = (W0[v] * area).sum()
            assert abs((W[v] * area).sum() - tot0) <= 1e-14 * abs(tot0)
    # and it is not a fixed point: the fields did change
    assert np.abs(W - W0).max() > 1e-6


def test_explicit_step_of_a_uniform_state_is_zero():
    from igks_inputs import meshgen as G
    m = G.tiny_quads(3, 3, bcs=("symmetry", "farfield"))
    fl = F.laminar_plate_flow(); fl.scheme = 1
    o = O.Oracle(m, fl)
    W0 = F.uniform_state(m, fl)
    o.set_W(W0)
    o.iterate(2)
    np.testing.assert_allclose(o.get(O.ORA_W), W0, rtol=1e-13, atol=1e-13)


def test_moving_wall_ghost_mirrors_velocity_about_the_lid():
    """A fluid moving with the lid sees itself as the ghost (no slip); a fluid at rest sees
    a ghost at twice the lid velocity; density and internal energy are those inside."""
    from igks_inputs import meshgen as G
    m = G.cavity(3)
    fl = F.cavity_flow()
    p0 = 1.0 / (F.GAMMA * fl.mach ** 2)
    lid = np.nonzero(m.face_bc == G.BC_MOVING_WALL)[0]
    for u_in, u_ghost in ((1.0, 1.0), (0.0, 2.0), (0.4, 1.6)):
        W = np.repeat(np.array(_conserved(1.05, u_in, 0.0, 1.02 * p0))[:, None], m.n_cells, axis=1)
        o = O.Oracle(m, fl)
        o.set_W(W)
        o.iterate(1)
        gh = o.get(O.ORA_GHOST)[:, lid]
        r, u, v, p = _prim(gh)
        np.testing.assert_allclose(r, 1.05, rtol=1e-15)
        np.testing.assert_allclose(u, u_ghost, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(v, 0.0, atol=1e-14)
        np.testing.assert_allclose(p, 1.02 * p0, rtol=1e-13)


@pytest.mark.parametrize("ratio", [1e3, 1e5])
def test_flux_ns_limit_shear_through_the_tangential_slopes(ratio):
    """U_n = a x_t (the normal velocity varies along the face): the shear stress
    mu (dU_t/dn + dU_n/dt) = mu a is carried by the tangential slopes a_t and abar_t of
    Eq. 4-5 alone, so the tangential momentum flux tends to -mu a dt as tau/dt -> 0. The
    flow is divergence free and steady at the face: no other flux changes."""
    fl = _flow(reynolds=1e3)
    rho, p, a = 1.0, 1 / (GAM * fl.mach ** 2), 0.8
    lam = rho / (2 * p)
    mu = _sutherland(fl, lam)
    dt = ratio * mu / p
    W = _cons(rho, 0.0, 0.0, p)
    st = np.array([0.0, rho * a, 0.0, 0.0])     # d(rho U_n)/dt; U_n = 0 at the face
    z = np.zeros(4)
    Fx, _ = O.face_flux(fl, W, W, z, st, z, st, W, W, 1e-3, 1e-3, 0.0, dt)
    ref = -mu * a * dt
    assert abs(Fx[2] - ref) <= 5.0 / ratio * abs(ref) + 1e-12 * abs(ref)
    assert abs(Fx[1] - p * dt) <= 5.0 / ratio * abs(ref) + 1e-13 * p * dt
    assert abs(Fx[0]) <= 1e-10 * abs(ref) and abs(Fx[3]) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("ratio", [1e3, 1e4])
def test_flux_ns_limit_normal_stress(ratio):
    """U_n = a x_n at uniform density and pressure: the BGK normal stress of a gas with
    D = K + 2 energy-carrying degrees of freedom is -2 mu a (D - 1)/D (Chapman-Enskog of
    Eq. 1; 1.6 mu a here), on top of the pressure, which itself evolves by the Euler
    equations, dp/dt = -a p (D + 2)/D at the face, over the step: the normal momentum flux
    tends to p dt - a p (D + 2)/D dt^2/2 - 2 mu a (D - 1)/D dt."""
    fl = _flow(reynolds=1e3)
    rho, p, a = 1.0, 1 / (GAM * fl.mach ** 2), 0.05
    lam = rho / (2 * p)
    mu = _sutherland(fl, lam)
    dt = ratio * mu / p
    D = K + 2
    d = 1e-7          # centre states close to the face: their kinetic energy is O(a^2 d^2)
    W = _cons(rho, 0.0, 0.0, p)
    sn = np.array([0.0, rho * a, 0.0, 0.0])
    z = np.zeros(4)
    Fx, _ = O.face_flux(fl, W, W, sn, z, sn, z, _cons(rho, -a * d, 0.0, p), _cons(rho, a * d, 0.0, p), d, d, 0.0, dt)
    stress = -2.0 * mu * a * (D - 1) / D * dt
    ref = p * dt - a * p * (D + 2) / D * dt * dt / 2 + stress
    assert abs(Fx[1] - ref) <= 10.0 / ratio * abs(stress) + 1e-13 * p * dt, (Fx[1] - ref) / stress
    assert abs(Fx[0]) <= 1e-10 * abs(stress) and abs(Fx[2]) <= 1e-10 * abs(stress)
