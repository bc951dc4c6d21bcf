"""Laminar flat plate against the Blasius boundary layer (the similarity solution of the
boundary-layer equations): the verification plate of the laminar workload's generator
(64 x 64 quads, first spacing 1e-4, about 25 cells across the layer at x = 0.5), Ma 0.15,
Re 1e5 per unit length, run with the FP64 path (equal to the oracle iteration by
iteration) to the paper's criterion. The streamwise velocity across the layer at
x = 0.5 is compared with f'(eta), eta = y sqrt(Re / x), from the Blasius equation
f''' + f f'' / 2 = 0 integrated here by RK4 shooting."""
import numpy as np
import pytest

from igks_inputs import fields as F
from igks_inputs import meshgen as G

def blasius(eta_max=10.0, n=4000):
    """f'(eta) on [0, eta_max] by RK4 shooting on f''(0) (bisection until f'(eta_max) = 1)."""
    h = eta_max / n

    def run(s):
        y = np.array([0.0, 0.0, s])
        out = [y[1]]
        rhs = lambda y: np.array([y[1], y[2], -0.5 * y[0] * y[2]])
        for _ in range(n):
            k1 = rhs(y); k2 = rhs(y + 0.5 * h * k1); k3 = rhs(y + 0.5 * h * k2); k4 = rhs(y + h * k3)
            y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            out.append(y[1])
        return np.array(out)

    lo, hi = 0.1, 1.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if run(mid)[-1] < 1.0:
            lo = mid
        else:
            hi = mid
    s = 0.5 * (lo + hi)
    return np.linspace(0.0, eta_max, n + 1), run(s), s


def test_blasius_shooting_gives_the_known_wall_curvature():
    _, _, s = blasius()
    assert abs(s - 0.332057) < 2e-5


def _profile_error(W, xc, yc, nx, ny, re):
    """max |u/U - f'(eta)| across the layer at the cell column nearest x = 0.5."""
    xc, yc = xc.reshape(ny, nx), yc.reshape(ny, nx)
    i = int(np.argmin(np.abs(xc[0] - 0.5)))
    x = xc[0, i]
    u = (W[1] / W[0]).reshape(ny, nx)[:, i]
    eta = yc[:, i] * np.sqrt(re / x)
    et, fp, _ = blasius()
    sel = eta <= 8.0
    return np.abs(u[sel] - np.interp(eta[sel], et, fp)), int(sel.sum()), x


def test_oracle_converged_plate_matches_blasius():
    """The oracle's own fixed point: its converged field on the verification plate (run to
    Eq. 40 <= 3e-8 by tests/golden/make_converged_fields.py, oracle only) has the Blasius
    profile across the layer, and its residual there is at the converged level."""
    import os
    import oracle as O
    d = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "converged_blasius_plate.npz"))
    nx, ny = 64, 64
    m = G.flat_plate_quads(nx, ny, first=1e-4, name="plate_blasius")
    fl = F.laminar_plate_flow()
    o = O.Oracle(m, fl)
    o.set_W(d["W"])
    gc = o.get(O.ORA_GEOM_CELL)
    err, n, x = _profile_error(d["W"], gc[1], gc[2], nx, ny, fl.reynolds)
    assert n >= 20
    assert err.max() <= 0.02, (x, err.max())
    # one more oracle iteration from the stored field changes it by the paper's criterion
    o.iterate(1)
    assert o.scalars()["eq40"] <= 3e-8


@pytest.mark.gpu
def test_laminar_plate_profile_matches_blasius():
    from paper_1709_00803_gb300 import igks
    nx, ny = 64, 64
    m = G.flat_plate_quads(nx, ny, first=1e-4, name="plate_blasius")
    fl = F.laminar_plate_flow()
    fl.eq40_target = 3e-8
    ctx = igks.Context(precision=0, check_every=200)
    sid = ctx.mesh_upload(m); ctx.set_flow(sid, fl); ctx.init_freestream(sid)
    rc, st = ctx.iterate(40000)
    assert rc == igks.CONVERGED, st[sid]
    W = ctx.get_fields(sid)
    geo = ctx.get_array(sid, "geom_cell")
    ctx.destroy()
    xc, yc = geo[1].reshape(ny, nx), geo[2].reshape(ny, nx)
    i = int(np.argmin(np.abs(xc[0] - 0.5)))
    x = xc[0, i]
    u = (W[1] / W[0]).reshape(ny, nx)[:, i]
    eta = yc[:, i] * np.sqrt(fl.reynolds / x)
    et, fp, _ = blasius()
    sel = eta <= 8.0
    assert sel.sum() >= 20                       # the layer is resolved
    err = np.abs(u[sel] - np.interp(eta[sel], et, fp))
    print(f"Blasius: x = {x:.4f}, {int(sel.sum())} cells with eta <= 8, max |u/U - f'| = {err.max():.4f}, "
          f"iterations {st[sid]['iters']}")
    assert err.max() <= 0.02, (x, err.max(), int(np.argmax(err)))
