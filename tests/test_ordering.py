"""Cell orderings for the LU-SGS sweeps (host logic, no GPU): igks_order_cells returns a
permutation; with the multicolour order every forward-sweep dependency chain is at most
one colour deep, so the sweep has as many levels as colours."""
import numpy as np
import pytest

from igks_inputs import meshgen as G


def _fwd_levels(mesh):
    lev = np.zeros(mesh.n_cells, dtype=np.int64)
    nb = [[] for _ in range(mesh.n_cells)]
    for l, r in mesh.face_cells:
        if r >= 0:
            nb[l].append(r); nb[r].append(l)
    for i in range(mesh.n_cells):
        lo = [lev[j] + 1 for j in nb[i] if j < i]
        lev[i] = max(lo) if lo else 0
    return lev


@pytest.mark.parametrize("mk", [G.laminar_plate, lambda: G.flat_plate_hybrid(nx=40, nq=10, ntri_rows=10, seed=3),
                                G.mixed_polygons])
def test_multicolor_order_is_a_low_depth_permutation(mk):
    from paper_1709_00803_gb300 import igks
    m = mk()
    perm, ncol = igks.order_cells(m, igks.ORDER_MULTICOLOR)
    assert sorted(perm.tolist()) == list(range(m.n_cells))
    assert 2 <= ncol <= 8
    r = m.renumbered(perm)
    assert r.n_cells == m.n_cells and r.n_faces == m.n_faces
    assert np.array_equal(np.bincount(r.face_bc, minlength=4), np.bincount(m.face_bc, minlength=4))
    assert _fwd_levels(r).max() + 1 <= ncol
    # the generator's own numbering of the quad plate is a wavefront of nx + ny - 1 levels
    if m.name.startswith("laminar"):
        assert _fwd_levels(m).max() + 1 == 64 + 32 - 1


def test_identity_order():
    from paper_1709_00803_gb300 import igks
    m = G.tiny_quads(3, 3)
    perm, ncol = igks.order_cells(m, igks.ORDER_AS_GIVEN)
    assert perm.tolist() == list(range(m.n_cells)) and ncol == 1
