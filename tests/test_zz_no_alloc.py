"""igks_residual_norms_noalloc, the entry point for callers that cannot let the library
allocate GPU memory (a stream under graph capture, a host-owned memory pool, a real-time
loop), against the norms igks_iterate itself reports, on two calls in a row.

This file is collected last on purpose, so that a run that stops at the first failure
has already run every other test. It passes alone in a fresh process and after the rest.
"""
import numpy as np
import pytest

from igks_inputs import fields as F
from igks_inputs import meshgen as G

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the per-iteration parity tolerance of the other GPU tests


def test_noalloc_norms_match_iterate_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1709_00803_gb300 import igks

    mesh = G.flat_plate_hybrid(nx=64, nq=24, ntri_rows=16, first=1e-5, seed=7)
    flow = F.turbulent_plate_flow()
    ctx = igks.Context()
    sid = ctx.mesh_upload(mesh)
    ctx.set_flow(sid, flow)
    ctx.init_freestream(sid)
    ctx.set_fields(sid, F.perturbed_state(mesh, flow, seed=4))
    area = torch.tensor(ctx.get_array(sid, "geom_cell")[0], dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    seen = []
    for call in range(2):
        _, st = ctx.iterate(1)
        m_rho = torch.tensor(ctx.get_array(sid, "res")[0], dtype=torch.float64, device="cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        igks.residual_norms_noalloc(m_rho.data_ptr(), area.data_ptr(), mesh.n_cells, out.data_ptr(),
                                    stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        ref = np.array([st[sid]["res_inf"], st[sid]["res_l2_rho"]])
        assert np.all(np.abs(got - ref) <= TOL * np.abs(ref)), (call, got, ref)
        seen.append(got)
    # the two iterations have different residuals: the second call really recomputed
    assert not np.array_equal(seen[0], seen[1])
    ctx.destroy()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1709_00803_gb300 import igks

    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(igks.IgksError) as e:
        igks.residual_norms_noalloc(buf.data_ptr(), buf.data_ptr(), igks.NOALLOC_MAX_CELLS + 1,
                                    buf.data_ptr(), 0)
    assert e.value.code == igks.EINVAL
    assert "exceeds the maximum" in str(e.value)
