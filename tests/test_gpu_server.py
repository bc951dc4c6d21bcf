"""Serving layer (igks_server_*): continuous batching must not change any solve's result.
Each served solve -- admitted at a different step, sharing cohorts with other solves,
moved between cohorts -- ends with bitwise the fields and the stopping iteration of the
same solve run alone in a context of its own. Admission respects the HBM budget and the
slot limit; the iteration cap stops a solve; submit rejects bad requests."""
import numpy as np
import pytest

from igks_inputs import fields as F
from igks_inputs import meshgen as G

pytestmark = pytest.mark.gpu


def _flow(mach, reynolds):
    fl = F.laminar_plate_flow()
    fl.mach, fl.reynolds = mach, reynolds
    fl.cfl_init, fl.cfl_min, fl.cfl_max = 50.0, 50.0, 1e4
    return fl


CASES = [(G.flat_plate_quads(24, 12, 1.15), _flow(0.5, 1e3)),
         (G.flat_plate_quads(24, 12, 1.15), _flow(0.3, 2e3)),
         (G.flat_plate_quads(32, 16, 1.12), _flow(0.4, 1.5e3)),
         (G.flat_plate_hybrid(nx=24, nq=8, ntri_rows=6, first=1e-3, ratio=1.2, seed=2), _flow(0.35, 1e3)),
         (G.flat_plate_quads(20, 10, 1.15), _flow(0.45, 1.2e3))]


@pytest.mark.parametrize("precision", [0, 1])
def test_served_results_equal_alone(precision):
    from paper_1709_00803_gb300 import igks
    alone = []
    for m, fl in CASES:
        ctx = igks.Context(precision=precision, check_every=100)
        sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl); ctx.init_freestream(sid)
        rc, st = ctx.iterate(20000)
        assert rc == igks.CONVERGED
        alone.append((ctx.get_fields(sid), st[sid]["iters"]))
        ctx.destroy()
    # small cohorts and an eager repack threshold: solves are admitted at different
    # steps, share cohorts and are moved while they iterate
    srv = igks.Server(precision=precision, max_slots=3, max_cohort=2, iters_per_step=37,
                      max_iters=20000, repack_fraction=0.9)
    ids = {}
    for k in (0, 1):
        ids[srv.submit(*CASES[k], tag=k)] = k
    results, repacked, max_cohorts, step = [], 0, 0, 0
    while len(results) < len(CASES):
        if step in (3, 5, 9):
            k = {3: 2, 5: 3, 9: 4}[step]
            ids[srv.submit(*CASES[k], tag=k)] = k
        st = srv.step()
        step += 1
        assert st["live"] <= 3
        repacked += st["repacked"]
        max_cohorts = max(max_cohorts, st["cohorts"])
        results += srv.poll()
        assert step < 2000
    assert repacked > 0 and max_cohorts >= 2
    for r in results:
        k = r["tag"]
        assert ids[r["id"]] == k
        assert r["state"] == igks.CONVERGED
        W, iters = alone[k]
        assert r["iters"] == iters, (k, r["iters"], iters)
        assert np.array_equal(srv.take_fields(r["id"]), W), f"served solve {k} differs from alone"
        assert r["t_submit"] <= r["t_admit"] <= r["t_finish"]
    srv.destroy()


def test_admission_respects_budget_and_iteration_cap():
    from paper_1709_00803_gb300 import igks
    m, fl = CASES[2]
    fp = igks.footprint_bytes(m)
    srv = igks.Server(precision=1, max_slots=8, max_cohort=8, iters_per_step=25, max_iters=100,
                      hbm_budget=int(2.5 * fp), repack_fraction=0.0, keep_fields=0)
    for k in range(5):
        srv.submit(m, fl, tag=k)
    results = []
    for _ in range(100):
        st = srv.step()
        assert st["bytes"] <= st["budget"] and st["live"] <= 2
        results += srv.poll()
        if len(results) == 5:
            break
    assert sorted(r["tag"] for r in results) == list(range(5))
    for r in results:
        assert r["state"] == igks.MAXITER and 100 <= r["iters"] < 125
    # FIFO: admission order follows submission order
    admits = [r["t_admit"] for r in sorted(results, key=lambda r: r["id"])]
    assert admits == sorted(admits)
    srv.destroy()


def test_submit_rejects_bad_requests():
    from paper_1709_00803_gb300 import igks
    m, fl = CASES[0]
    srv = igks.Server(hbm_budget=igks.footprint_bytes(m) // 2)
    with pytest.raises(igks.IgksError) as e:
        srv.submit(m, fl)
    assert e.value.code == igks.ENOMEM
    srv.destroy()
    srv = igks.Server()
    fc = m.face_cells.copy(); fc[0, 0] = 10 ** 6
    with pytest.raises(igks.IgksError) as e:
        srv.submit(G.Mesh(m.xy, m.cell_ptr, m.cell_nodes, m.face_nodes, fc, m.face_bc), fl)
    assert e.value.code == igks.EMESH
    bad = _flow(0.3, 1e3); bad.mach = -1.0
    with pytest.raises(igks.IgksError) as e:
        srv.submit(m, bad)
    assert e.value.code == igks.EINVAL
    assert srv.status()["queued"] == 0
    srv.destroy()


def test_footprint_bounds_the_allocation():
    from paper_1709_00803_gb300 import igks
    meshes = [G.laminar_plate(), G.mixed_polygons(), G.flat_plate_hybrid(nx=48, nq=16, ntri_rows=12, seed=3)]
    ctx = igks.Context()
    for m in meshes:
        sid = ctx.mesh_upload(m); ctx.set_flow(sid, F.laminar_plate_flow())
    ctx.init_freestream(0)
    used = ctx.device_bytes()
    bound = sum(igks.footprint_bytes(m) for m in meshes)
    assert used <= bound <= 1.15 * used
    ctx.destroy()
