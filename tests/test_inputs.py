"""The seeded input generators: mesh quality of the airfoil O-meshes (a folded ring
behind the trailing edge once made the solver diverge), sizes of the scaled meshes, and
determinism of the seeded workload specs."""
import numpy as np
import pytest

from igks_inputs import meshgen as G


def _min_angles(m):
    out = np.empty(m.n_cells)
    for c in range(m.n_cells):
        P = m.xy[m.cell_node_list(c)]
        a = []
        for k in range(len(P)):
            u, v = P[k - 1] - P[k], P[(k + 1) % len(P)] - P[k]
            a.append(np.degrees(np.arccos(np.clip(u @ v / np.linalg.norm(u) / np.linalg.norm(v), -1, 1))))
        out[c] = min(a)
    return out


@pytest.mark.parametrize("args", [(0.0, 0.0, 0.12, 8000, 33), (0.06, 0.4, 0.08, 30000, 5)])
def test_airfoil_omesh_triangles_are_not_slivers(args):
    m = G.naca_scaled(*args)
    tri = np.diff(m.cell_ptr) == 3
    ang = _min_angles(m)[tri]
    assert ang.min() > 3.0
    assert np.percentile(ang, 1) > 8.0


def test_scaled_meshes_hit_their_cell_counts():
    for c in (2000, 20480, 60000):
        m = G.plate_scaled(c, 1)
        assert abs(m.n_cells - c) <= 0.05 * c
    for c in (8000, 40000):
        m = G.naca_scaled(0.02, 0.4, 0.12, c, 7)
        assert abs(m.n_cells - c) <= 0.10 * c


def test_seeded_specs_are_deterministic_and_in_range():
    a, b = G.serving_specs(20, 5), G.serving_specs(20, 5)
    assert a == b
    for s in a:
        assert s["kind"] in ("plate", "naca")
        assert 2000 <= s["cells"] <= 250000 and 0.1 <= s["mach"] <= 0.75 and 1e6 <= s["reynolds"] <= 1e7
    c = G.naca_batch_specs(64, 4)
    assert c == G.naca_batch_specs(64, 4) and len(c) == 64
    assert all(8000 <= s["cells"] <= 80000 for s in c)
