"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element,
from the same seeded states, on meshes that span many thread blocks with ragged tails
(2048, 20480 and 60160 cells; 4192-98240 faces), with and without the SA model, with
each limiter, on general polygons, for one and several iterations, and at the full sizes
the benchmark times. Bar: 1e-12 relative per iteration in FP64 (see _parity.py)."""
import numpy as np
import pytest

import oracle as O
from igks_inputs import fields as F
from igks_inputs import meshgen as G

from _parity import GPU_TO_ORA, assert_close, make_pair, seeded

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _compare_iteration(ctx, sid, ora, tol=TOL, skip=()):
    for name, which in GPU_TO_ORA.items():
        if name in skip:
            continue
        g = ctx.get_array(sid, name)
        r = ora.get(which)
        if name == "grad":
            g = g.reshape(8, -1); r = r.reshape(8, -1)
        if name in ("dwstar", "dw"):
            # The increments are formed differently on the two sides: the oracle differences
            # two Euler fluxes, F(W + dW) - F(W), the CUDA path uses their difference-free
            # form. The two agree to rounding of the state's size, so the bar is 1e-12 of
            # max |W| per component (what the update W + dW sees); against the increments'
            # own, much smaller scale they agree to 1e-9.
            Ws = np.abs(ora.get(O.ORA_W)).max(axis=1)[:, None]
            Ws = np.where(Ws == 0, 1.0, Ws)
            e = np.max(np.abs(g - r) / Ws)
            assert e <= tol, f"{name}: max error {e:.3e} of max |W| > {tol:.1e}"
            assert_close(name, g, r, 1e-9)
            continue
        assert_close(name, g, r, tol)
    Wg = ctx.get_fields(sid)
    Wo = ora.get(O.ORA_W)
    assert_close("W", Wg, Wo, tol)
    so = ora.scalars()
    _, st = ctx.iterate(0)
    assert abs(st[sid]["dt"] - so["dt"]) <= 1e-14 * so["dt"]
    assert abs(st[sid]["cfl"] - so["cfl"]) <= 1e-12 * so["cfl"]
    assert abs(st[sid]["res_inf"] - so["res_inf"]) <= 1e-10 * so["res_inf"]
    assert abs(st[sid]["res_l2_rho"] - so["res_l2"]) <= 1e-10 * so["res_l2"]


def test_laminar_plate_one_iteration():
    m = G.laminar_plate()
    fl = F.laminar_plate_flow()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 1))
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)


def test_turbulent_plate_sa_one_iteration_full_size():
    m = G.turbulent_plate()
    fl = F.turbulent_plate_flow()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 2))
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)


def test_naca0012_sa_one_iteration_full_size():
    m = G.naca0012()
    fl = F.naca_flow()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 3, amp=0.02))
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)


@pytest.mark.parametrize("limiter", [F.LIMITER_BJ, F.LIMITER_VENKAT])
def test_limiters_one_iteration(limiter):
    m = G.flat_plate_hybrid(nx=40, nq=10, ntri_rows=10, first=1e-3, seed=4)
    fl = F.turbulent_plate_flow(); fl.reynolds = 1e5; fl.limiter = limiter
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 5, amp=0.15))
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)


def test_general_polygons_one_iteration():
    m = G.mixed_polygons()
    fl = F.turbulent_plate_flow(); fl.reynolds = 2e3
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 6))
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)


@pytest.mark.parametrize("mk,flow_fn", [(G.laminar_plate, F.laminar_plate_flow),
                                        (lambda: G.flat_plate_hybrid(nx=64, nq=24, ntri_rows=16, first=1e-5, seed=7),
                                         F.turbulent_plate_flow)])
def test_many_iterations_with_cfl_adaptation(mk, flow_fn):
    m = mk()
    fl = flow_fn()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 8), check_every=7)
    for n in (1, 4, 15):
        ctx.iterate(n); ora.iterate(n)
        assert_close(f"W after +{n}", ctx.get_fields(sid), ora.get(O.ORA_W), TOL)
    _, st = ctx.iterate(0)
    so = ora.scalars()
    assert st[sid]["iters"] == so["iter"] == 20
    assert abs(st[sid]["cfl"] - so["cfl"]) <= 1e-10 * so["cfl"]


def test_free_stream_start_matches():
    m = G.laminar_plate()
    fl = F.laminar_plate_flow()
    ctx, sid, ora = make_pair(m, fl)
    ctx.iterate(3); ora.iterate(3)
    assert_close("W", ctx.get_fields(sid), ora.get(O.ORA_W), TOL)


def test_mixed_precision_sweeps_close_to_fp64():
    m = G.flat_plate_hybrid(nx=64, nq=24, ntri_rows=16, first=1e-5, seed=7)
    fl = F.turbulent_plate_flow()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 9), precision=1)
    ctx.iterate(1); ora.iterate(1)
    # flux, residual and state update are FP64 in both modes
    for name in ("flux", "res", "lambda_f", "grad"):
        g = ctx.get_array(sid, name); r = ora.get(GPU_TO_ORA[name])
        assert_close(name, g.reshape(g.shape[0], -1) if g.ndim > 1 else g,
                     r.reshape(r.shape[0], -1) if r.ndim > 1 else r, TOL)
    # FP32 sweeps: increments to single-precision accuracy
    assert_close("dw (fp32 sweeps)", ctx.get_array(sid, "dw")[:4], ora.get(O.ORA_DW)[:4], 2e-5)


def test_batched_solves_equal_alone():
    from paper_1709_00803_gb300 import igks
    cases = [(G.laminar_plate(), F.laminar_plate_flow(), 1),
             (G.flat_plate_hybrid(nx=48, nq=16, ntri_rows=12, first=1e-5, seed=3), F.turbulent_plate_flow(), 2),
             (G.mixed_polygons(), F.turbulent_plate_flow(), 3)]
    alone = []
    for m, fl, seed in cases:
        ctx = igks.Context()
        sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl); ctx.init_freestream(sid)
        ctx.set_fields(sid, seeded(m, fl, seed))
        ctx.iterate(12)
        alone.append(ctx.get_fields(sid))
        ctx.destroy()
    ctx = igks.Context(check_every=5)
    for m, fl, seed in cases:
        sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl)
    for k, (m, fl, seed) in enumerate(cases):
        ctx.init_freestream(k)
        ctx.set_fields(k, seeded(m, fl, seed))
    ctx.iterate(12)
    for k in range(len(cases)):
        assert np.array_equal(ctx.get_fields(k), alone[k]), f"solve {k} differs in the batch"


def test_checkpoint_resume_bitwise():
    from paper_1709_00803_gb300 import igks
    m = G.flat_plate_hybrid(nx=48, nq=16, ntri_rows=12, first=1e-5, seed=3)
    fl = F.turbulent_plate_flow()
    ref = igks.Context(); s = ref.mesh_upload(m); ref.set_flow(s, fl); ref.init_freestream(s)
    ref.iterate(30)
    a = igks.Context(); s = a.mesh_upload(m); a.set_flow(s, fl); a.init_freestream(s)
    a.iterate(13)
    W, sc = a.get_fields(s), a.get_scalars(s)
    a.destroy()
    b = igks.Context(); s = b.mesh_upload(m); b.set_flow(s, fl); b.init_freestream(s)
    b.set_fields(s, W); b.set_scalars(s, sc)
    b.iterate(17)
    assert np.array_equal(b.get_fields(s), ref.get_fields(s))


def test_mesh_errors_are_reported():
    from paper_1709_00803_gb300 import igks
    m = G.tiny_quads(2, 2)
    bad = G.Mesh(m.xy, m.cell_ptr, m.cell_nodes[::-1].copy(), m.face_nodes, m.face_cells, m.face_bc)
    ctx = igks.Context()
    with pytest.raises(igks.IgksError):
        ctx.mesh_upload(bad)     # node lists no longer close the cells through the faces
    fc = m.face_cells.copy(); fc[0, 0] = 99
    with pytest.raises(igks.IgksError) as e:
        ctx.mesh_upload(G.Mesh(m.xy, m.cell_ptr, m.cell_nodes, m.face_nodes, fc, m.face_bc))
    assert e.value.code == igks.EMESH
    # clockwise cells: caught when the geometry is built on the device
    cw = [m.cell_node_list(c)[::-1] for c in range(m.n_cells)]
    flip_nodes = np.concatenate(cw).astype(np.int32)
    fn = m.face_nodes[:, ::-1].copy()
    ctx2 = igks.Context()
    ctx2.mesh_upload(G.Mesh(m.xy, m.cell_ptr, flip_nodes, fn, m.face_cells, m.face_bc))
    with pytest.raises(igks.IgksError) as e:
        ctx2.init_freestream(0)
    assert e.value.code == igks.EMESH


@pytest.mark.parametrize("mk,flow_fn", [(G.laminar_plate, F.laminar_plate_flow),
                                        (G.turbulent_plate, F.turbulent_plate_flow)])
def test_multicolor_order_wide_sweeps_match_oracle(mk, flow_fn):
    """Multicolour numbering (few, wide levels: one launch per level) on both sides."""
    from paper_1709_00803_gb300 import igks
    base = mk()
    perm, ncol = igks.order_cells(base, igks.ORDER_MULTICOLOR)
    m = base.renumbered(perm)
    fl = flow_fn()
    W0 = seeded(base, fl, 12)[:, perm]
    ctx, sid, ora = make_pair(m, fl, W0)
    info = ctx.mesh_info(sid)
    assert info["levels_fwd"] <= ncol
    assert ctx.launches_per_iteration() == 9 + info["levels_fwd"] + info["levels_bwd"]
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)
    ctx.iterate(6); ora.iterate(6)
    assert_close("W after 7", ctx.get_fields(sid), ora.get(O.ORA_W), TOL)


def test_forced_wide_schedule_on_deep_ordering():
    m = G.flat_plate_hybrid(nx=24, nq=8, ntri_rows=6, first=1e-5, seed=11)
    fl = F.turbulent_plate_flow()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 13), sweep_mode=2)
    ctx.iterate(3); ora.iterate(3)
    assert_close("W", ctx.get_fields(sid), ora.get(O.ORA_W), TOL)
    ctx2, sid2, ora2 = make_pair(m, fl, seeded(m, fl, 13), sweep_mode=1, precision=1)
    ctx2.iterate(1); ora2.iterate(1)
    assert_close("dw fp32 narrow", ctx2.get_array(sid2, "dw")[:4], ora2.get(O.ORA_DW)[:4], 2e-5)


def test_autotune_leaves_iterates_unchanged():
    from paper_1709_00803_gb300 import igks
    cases = [(G.flat_plate_hybrid(nx=48, nq=16, ntri_rows=12, first=1e-5, seed=3), F.turbulent_plate_flow()),
             (G.laminar_plate(), F.laminar_plate_flow())]
    results = []
    for tune in (False, True):
        ctx = igks.Context(precision=1)
        for m, fl in cases:
            sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl)
        for k in range(len(cases)):
            ctx.init_freestream(k)
        ctx.iterate(5)
        if tune:
            choice = ctx.autotune(2)
            assert choice["sweep_mode"] in (1, 2) and choice["ms_per_iter"] > 0
        ctx.iterate(10)
        results.append([ctx.get_fields(k) for k in range(len(cases))])
        ctx.destroy()
    for a, b in zip(*results):
        assert np.array_equal(a, b)


def test_moving_wall_cavity_one_iteration():
    m = G.cavity(40)
    fl = F.cavity_flow()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 21, amp=0.05))
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)


@pytest.mark.parametrize("mk,flow_fn", [(lambda: G.cavity(40), lambda: F.cavity_flow(scheme=1)),
                                        (lambda: G.flat_plate_hybrid(nx=48, nq=16, ntri_rows=12, first=1e-5, seed=3),
                                         F.turbulent_plate_flow)])
def test_explicit_scheme_matches_oracle(mk, flow_fn):
    """The explicit gas-kinetic scheme (Eq. 15) on the same kernels: no sweeps, W += dt M / Omega."""
    m = mk()
    fl = flow_fn()
    fl.scheme = 1
    for precision in (0, 1):    # the sweep precision plays no part in the explicit update
        ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 22, amp=0.05), precision=precision)
        ctx.iterate(1); ora.iterate(1)
        _compare_iteration(ctx, sid, ora, skip=("dwstar", "dw"))
        ctx.iterate(6); ora.iterate(6)
        assert_close("W after 7 explicit steps", ctx.get_fields(sid), ora.get(O.ORA_W), TOL)


@pytest.mark.parametrize("precision", [0, 1])
def test_cluster_sweeps_bitwise_equal_one_block(precision):
    """A cluster of C blocks per solve shares every level of the sweeps (distributed shared
    memory, one cluster barrier per level) and does the same arithmetic in the same order:
    the iterates are bitwise those of one block per solve, alone and in a batch."""
    from paper_1709_00803_gb300 import igks
    cases = [(G.flat_plate_hybrid(nx=48, nq=16, ntri_rows=12, first=1e-5, seed=3), F.turbulent_plate_flow(), 1),
             (G.mixed_polygons(), F.turbulent_plate_flow(), 2),
             (G.laminar_plate(), F.laminar_plate_flow(), 3)]
    ref = None
    for cl in (1, 2, 4, 8):
        ctx = igks.Context(precision=precision, sweep_mode=1, sweep_cluster=cl)
        for m, fl, seed in cases:
            sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl)
        for k, (m, fl, seed) in enumerate(cases):
            ctx.init_freestream(k)
            ctx.set_fields(k, seeded(m, fl, seed))
        ctx.iterate(6)
        out = [ctx.get_fields(k) for k in range(len(cases))]
        ctx.destroy()
        if ref is None:
            ref = out
        else:
            for k in range(len(cases)):
                assert np.array_equal(out[k], ref[k]), f"cluster {cl}, solve {k}"


def _sweep_stencil_sizes(m):
    """Per cell: interior neighbours earlier in the numbering (forward-sweep entries) and
    later ones plus wall / symmetry ghosts (backward-sweep entries)."""
    lower = np.zeros(m.n_cells, int)
    upper = np.zeros(m.n_cells, int)
    for f in range(m.n_faces):
        l, r = m.face_cells[f]
        if r < 0:
            if m.face_bc[f] in (G.BC_SYMMETRY, G.BC_WALL, G.BC_MOVING_WALL):
                upper[l] += 1
            continue
        lower[max(l, r)] += 1
        upper[min(l, r)] += 1
    return lower, upper


@pytest.mark.parametrize("permute", [None, 11])
@pytest.mark.parametrize("sweep_mode", [1, 2])
def test_refined_cavity_polygons_fp64(permute, sweep_mode):
    """The adaptively refined cavity (quads, pentagons, hexagons, hanging nodes), 1470
    cells over six blocks: FP64 parity at 1e-12 for three iterations, one block per solve
    walking the levels (1) and one launch per level (2). With the random numbering some
    cells have five lower or upper neighbours: more than the four entries a sweep record
    holds, so the narrow sweeps take the position-ordered stencil for them."""
    m = G.refined_cavity(permute_seed=permute)
    sizes = np.bincount(np.diff(m.cell_ptr))
    assert sizes[5] > 0 and sizes[6] > 0               # pentagons and hexagons
    lower, upper = _sweep_stencil_sizes(m)
    if permute is not None:
        assert lower.max() > 4 and upper.max() > 4
    fl = F.cavity_flow()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 31, amp=0.05), sweep_mode=sweep_mode)
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)
    ctx.iterate(2); ora.iterate(2)
    assert_close("W after 3", ctx.get_fields(sid), ora.get(O.ORA_W), TOL)


@pytest.mark.parametrize("permute", [None, 11])
def test_refined_cavity_polygons_fp32_sweeps(permute):
    """FP32 sweeps on the same meshes: the two schedules apply every stencil entry in the
    same order, so they give the same bits; the increments agree with the FP64 oracle to
    single precision and flux / residual stay at the FP64 bar."""
    m = G.refined_cavity(permute_seed=permute)
    fl = F.cavity_flow()
    W0 = seeded(m, fl, 32, amp=0.05)
    out = []
    for mode in (1, 2):
        ctx, sid, ora = make_pair(m, fl, W0, precision=1, sweep_mode=mode)
        ctx.iterate(1)
        if mode == 1:
            ora.iterate(1)
            for name in ("flux", "res"):
                assert_close(name, ctx.get_array(sid, name), ora.get(GPU_TO_ORA[name]), TOL)
            assert_close("dw (fp32 sweeps)", ctx.get_array(sid, "dw")[:4], ora.get(O.ORA_DW)[:4], 2e-5)
        ctx.iterate(2)
        out.append(ctx.get_fields(sid))
        ctx.destroy()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_groups_of_solves_bitwise_equal_one_group(precision):
    """Solves split into groups that iterate on streams of their own (so one group's sweeps
    run beside another group's flux) do the same arithmetic: the fields are bitwise those of
    one group, for 2 and 3 groups, also after the configuration is switched between runs."""
    from paper_1709_00803_gb300 import igks
    cases = [(G.flat_plate_hybrid(nx=48, nq=16, ntri_rows=12, first=1e-5, seed=3), F.turbulent_plate_flow(), 1),
             (G.mixed_polygons(), F.turbulent_plate_flow(), 2),
             (G.laminar_plate(), F.laminar_plate_flow(), 3),
             (G.refined_cavity(12, band=2), F.cavity_flow(), 4),
             (G.flat_plate_hybrid(nx=32, nq=12, ntri_rows=8, first=1e-4, seed=5), F.turbulent_plate_flow(), 5)]
    ref = None
    for groups in (1, 2, 3):
        ctx = igks.Context(precision=precision, sweep_mode=1, groups=groups, check_every=4)
        for m, fl, seed in cases:
            sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl)
        for k, (m, fl, seed) in enumerate(cases):
            ctx.init_freestream(k)
            ctx.set_fields(k, seeded(m, fl, seed))
        ctx.iterate(5)
        ctx.set_launch(dict(sweep_threads=256, flux_block=128, sweep_mode=1, sweep_cluster=1, groups=4 - groups))
        ctx.iterate(4)
        out = [ctx.get_fields(k) for k in range(len(cases))]
        ctx.destroy()
        if ref is None:
            ref = out
        else:
            for k in range(len(cases)):
                assert np.array_equal(out[k], ref[k]), f"groups {groups}, solve {k}"


def test_residual_history_matches_oracle_norms():
    """The per-iteration residual history kept on the device (Eq. 25's norms) against the
    oracle's norms of the same iterations."""
    m = G.flat_plate_hybrid(nx=48, nq=16, ntri_rows=12, first=1e-5, seed=3)
    fl = F.turbulent_plate_flow()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 41), check_every=6)
    ref = []
    for _ in range(25):
        ora.iterate(1)
        sc = ora.scalars()
        ref.append((sc["iter"], sc["res_l2"], sc["res_inf"]))
    ctx.iterate(25)
    h = ctx.get_history(sid)
    assert h.shape == (25, 3)
    ref = np.array(ref)
    assert np.array_equal(h[:, 0], ref[:, 0])
    assert np.all(np.abs(h[:, 1:] - ref[:, 1:]) <= 1e-10 * np.abs(ref[:, 1:]))
    assert len(ctx.get_history(sid, cap=7)) == 7 and ctx.get_history(sid, cap=7)[-1, 0] == 25


@pytest.mark.parametrize("mk,flow_fn", [(G.laminar_plate, F.laminar_plate_flow),
                                        (G.turbulent_plate, F.turbulent_plate_flow),
                                        (lambda: G.refined_cavity(permute_seed=11), F.cavity_flow)])
def test_double_float_sweeps_meet_the_fp64_bar(mk, flow_fn):
    """Sweeps in double-float (pairs of FP32 numbers, about 48 bits, on the FP32 pipes):
    one iteration compared term by term with the FP64 oracle at the FP64 bar (increments
    within 1e-12 of max |W|, everything else 1e-12 relative), then 6 more iterations."""
    m = mk()
    fl = flow_fn()
    ctx, sid, ora = make_pair(m, fl, seeded(m, fl, 51, amp=0.05), precision=2)
    ctx.iterate(1); ora.iterate(1)
    _compare_iteration(ctx, sid, ora)
    ctx.iterate(6); ora.iterate(6)
    assert_close("W after 7", ctx.get_fields(sid), ora.get(O.ORA_W), TOL)
