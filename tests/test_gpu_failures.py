"""Failure paths of the CUDA path, made on the host (no GPU fault is provoked): a state
with negative pressure or a non-finite nu~ planted through igks_set_fields, or handed to
the server as a request's starting state, must end that solve with IGKS_DIVERGED (the
update's check of density, pressure and finiteness) and leave the context usable; a
state whose residual is exactly zero counts as converged with a finite CFL (Eq. 25 with
a vanishing norm), on both sides."""
import math

import numpy as np
import pytest

import oracle as O
from igks_inputs import fields as F
from igks_inputs import meshgen as G

pytestmark = pytest.mark.gpu


def _negative_pressure(W, cell):
    W = W.copy()
    ke = 0.5 * (W[1, cell] ** 2 + W[2, cell] ** 2) / W[0, cell]
    W[3, cell] = 0.5 * ke            # energy below the kinetic energy: p < 0, rho > 0
    return W


@pytest.mark.parametrize("precision", [0, 1])
def test_planted_negative_pressure_diverges(precision):
    from paper_1709_00803_gb300 import igks
    m = G.flat_plate_hybrid(nx=24, nq=8, ntri_rows=6, first=1e-4, seed=3)
    fl = F.turbulent_plate_flow()
    good = G.laminar_plate()
    ctx = igks.Context(precision=precision, check_every=1)
    bad_id = ctx.mesh_upload(m); ctx.set_flow(bad_id, fl)
    ok_id = ctx.mesh_upload(good); ctx.set_flow(ok_id, F.laminar_plate_flow())
    ctx.init_freestream(bad_id); ctx.init_freestream(ok_id)
    ctx.set_fields(bad_id, _negative_pressure(F.perturbed_state(m, fl, seed=2), 17))
    rc, st = ctx.iterate(3)
    assert rc == igks.DIVERGED
    assert st[bad_id]["state"] == igks.DIVERGED and st[bad_id]["iters"] == 1
    # the other solve of the context is untouched by its neighbour's failure
    assert st[ok_id]["state"] == 0 and st[ok_id]["iters"] == 3
    W = ctx.get_fields(ok_id)
    assert np.all(np.isfinite(W))
    # and it matches the same solve alone
    alone = igks.Context(precision=precision)
    s = alone.mesh_upload(good); alone.set_flow(s, F.laminar_plate_flow()); alone.init_freestream(s)
    alone.iterate(3)
    assert np.array_equal(alone.get_fields(s), W)


def test_planted_nan_nu_tilde_diverges():
    from paper_1709_00803_gb300 import igks
    m = G.flat_plate_hybrid(nx=24, nq=8, ntri_rows=6, first=1e-4, seed=3)
    fl = F.turbulent_plate_flow()
    ctx = igks.Context(check_every=1)
    sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl); ctx.init_freestream(sid)
    W = F.perturbed_state(m, fl, seed=2)
    W[4, 40] = float("nan")
    ctx.set_fields(sid, W)
    rc, st = ctx.iterate(5)
    assert rc == igks.DIVERGED and st[sid]["state"] == igks.DIVERGED
    # a restart from a good state runs again
    ctx.set_fields(sid, F.perturbed_state(m, fl, seed=2))
    ctx.set_scalars(sid, {"iter": 0, "cfl": fl.cfl_init, "res_inf_prev": 0.0, "res_l2_first": 0.0, "state": 0})
    rc, st = ctx.iterate(2)
    assert rc == igks.OK and st[sid]["state"] == 0


def test_set_fields_rejects_non_positive_density():
    from paper_1709_00803_gb300 import igks
    m = G.laminar_plate()
    ctx = igks.Context()
    sid = ctx.mesh_upload(m); ctx.set_flow(sid, F.laminar_plate_flow()); ctx.init_freestream(sid)
    W = F.uniform_state(m, F.laminar_plate_flow())
    W[0, 3] = -1.0
    with pytest.raises(igks.IgksError) as e:
        ctx.set_fields(sid, W)
    assert e.value.code == igks.EINVAL


def test_served_request_that_diverges_is_reported():
    from paper_1709_00803_gb300 import igks
    m = G.flat_plate_hybrid(nx=24, nq=8, ntri_rows=6, first=1e-4, seed=3)
    fl = F.turbulent_plate_flow()
    fl.eq40_target = 3e-8
    good = G.plate_scaled(2000, 5)
    srv = igks.Server(precision=igks.PREC_MIXED, max_slots=4, iters_per_step=10, max_iters=30)
    a = srv.submit(m, fl, tag=1, W0=_negative_pressure(F.perturbed_state(m, fl, seed=2), 5))
    b = srv.submit(good, fl, tag=2)
    res = {}
    for _ in range(20):
        srv.step()
        for r in srv.poll():
            res[r["id"]] = r
        if len(res) == 2:
            break
    srv.destroy()
    assert res[a]["state"] == igks.DIVERGED and res[a]["iters"] == 1
    assert res[b]["state"] in (igks.CONVERGED, igks.MAXITER) and res[b]["iters"] >= 1
    with pytest.raises(igks.IgksError):
        srv2 = igks.Server(precision=igks.PREC_MIXED)
        W = F.uniform_state(m, fl)
        W[0, 0] = 0.0
        try:
            srv2.submit(m, fl, W0=W)
        finally:
            srv2.destroy()


def _one_cell_box():
    """One unit-square cell closed by symmetry planes: its four faces see the same state,
    the same mirror ghost and the same centre-to-face distance (the centroid of the unit
    square is exactly (0.5, 0.5)), so with the fluid at rest their fluxes cancel exactly
    whatever the rounding of the flux algebra."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    return G.build_mesh(xy, [[0, 1, 2, 3]], lambda a, b, xm, ym: G.BC_SYMMETRY, name="one_cell_box")


def test_exactly_zero_residual_converges_with_finite_cfl():
    """A residual that is exactly zero converges at once on both sides, and Eq. 25 after a
    non-zero norm sends the CFL to its cap (never NaN)."""
    from paper_1709_00803_gb300 import igks
    m = _one_cell_box()
    fl = F.cavity_flow()
    ctx = igks.Context(check_every=1)
    sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl); ctx.init_freestream(sid)
    ctx.set_fields(sid, F.rest_state(m, fl))
    rc, st = ctx.iterate(5)
    o = O.Oracle(m, fl)
    o.set_W(F.rest_state(m, fl))
    assert o.iterate(5) == 1
    assert rc == igks.CONVERGED and st[sid]["iters"] == 1 == o.scalars()["iter"]
    assert st[sid]["res_l2_rho"] == 0.0 and st[sid]["res_inf"] == 0.0
    assert math.isfinite(st[sid]["cfl"]) and st[sid]["cfl"] == fl.cfl_init
    # after a non-zero norm: the CFL goes to its cap
    ctx.set_scalars(sid, {"iter": 7, "cfl": 2345.0, "res_inf_prev": 3.5, "res_l2_first": 1.0, "state": 0})
    rc, st = ctx.iterate(1)
    assert rc == igks.CONVERGED and st[sid]["cfl"] == fl.cfl_max


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_sweep_wait_that_runs_out_reports_timeout(precision):
    """The one-block-per-solve sweeps wait on an mbarrier for each level's bulk-copied
    records, at most wait_limit tries. The test hook starve_test makes every forward sweep
    skip the copy of its second level, so that wait runs out (a barrier nothing completes):
    the solve stops with IGKS_TIMEOUT after one iteration, its fields as they were before it,
    the block lets its other copies land before it exits, and the device goes on working (a
    fresh context iterates the same solve as usual)."""
    from paper_1709_00803_gb300 import igks
    m = G.flat_plate_hybrid(nx=24, nq=8, ntri_rows=6, first=1e-4, seed=3)
    fl = F.turbulent_plate_flow()
    W0 = F.perturbed_state(m, fl, seed=2)
    ctx = igks.Context(precision=precision, sweep_mode=1, wait_limit=4096, starve_test=1, check_every=1)
    sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl); ctx.init_freestream(sid)
    ctx.set_fields(sid, W0)
    rc, st = ctx.iterate(3)
    assert rc == igks.TIMEOUT
    assert st[sid]["state"] == igks.TIMEOUT and st[sid]["iters"] == 1
    assert np.array_equal(ctx.get_fields(sid), W0)
    ctx.destroy()
    ok = igks.Context(precision=precision, sweep_mode=1, check_every=1)
    sid = ok.mesh_upload(m); ok.set_flow(sid, fl); ok.init_freestream(sid)
    ok.set_fields(sid, W0)
    rc, st = ok.iterate(3)
    assert rc == igks.OK and st[sid]["state"] == 0 and st[sid]["iters"] == 3
    assert np.all(np.isfinite(ok.get_fields(sid)))
    ok.destroy()


def test_whole_context_state_round_trip_and_rejection():
    """igks_get_fields_all / igks_set_fields_all move every solve's state in one call: the
    round trip equals the per-solve calls bitwise, iterating from a state set all at once
    equals iterating from the same state set solve by solve, and a solve with a
    non-physical state (negative density) is rejected with IGKS_EINVAL and keeps its state
    while the other solves take theirs."""
    from paper_1709_00803_gb300 import igks
    cases = [(G.flat_plate_hybrid(nx=24, nq=8, ntri_rows=6, first=1e-4, seed=3), F.turbulent_plate_flow(), 2),
             (G.laminar_plate(), F.laminar_plate_flow(), 5),
             (G.mixed_polygons(), F.turbulent_plate_flow(), 7)]
    ctxs = []
    for _ in range(2):
        ctx = igks.Context(precision=1, check_every=2)
        for m, fl, _ in cases:
            sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl)
        for k in range(len(cases)):
            ctx.init_freestream(k)
        ctxs.append(ctx)
    a, b = ctxs
    states = [F.perturbed_state(m, fl, seed=sd) for m, fl, sd in cases]
    for k, W in enumerate(states):
        a.set_fields(k, W)
    b.set_fields_all(np.concatenate(states, axis=1))
    assert np.array_equal(b.get_fields_all(), np.concatenate([a.get_fields(k) for k in range(len(cases))], axis=1))
    a.iterate(4); b.iterate(4)
    got = b.get_fields_all()
    off = 0
    for k, (m, _, _) in enumerate(cases):
        assert np.array_equal(got[:, off:off + m.n_cells], a.get_fields(k))
        off += m.n_cells
    # reject one non-physical solve, apply the others
    before = b.get_fields_all()
    bad = np.concatenate(states, axis=1)
    n0 = cases[0][0].n_cells
    bad[0, n0 + 3] = -1.0                      # a negative density in solve 1
    with pytest.raises(igks.IgksError) as e:
        b.set_fields_all(bad)
    assert e.value.code == igks.EINVAL
    after = b.get_fields_all()
    n1 = cases[1][0].n_cells
    assert np.array_equal(after[:, n0:n0 + n1], before[:, n0:n0 + n1])
    assert np.array_equal(after[:, :n0], bad[:, :n0])
    assert np.array_equal(after[:, n0 + n1:], bad[:, n0 + n1:])
    for c in ctxs:
        c.destroy()
