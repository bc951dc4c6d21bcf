"""Shared helpers of the parity tests: run the oracle and the CUDA path from the same
seeded state and compare arrays element by element against a per-component scale.

Tolerance: FP64 per-iteration agreement is required to 1e-12 relative. An element's
error is measured against the largest magnitude of its component over the mesh (the
scale of the terms that were summed to form it), because residual-like arrays are
differences of much larger face fluxes and near-zero entries carry rounding of that size.
"""
import numpy as np

import oracle as O
from igks_inputs import fields as F


def rel_err(a, b, axis=-1):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b), axis=axis, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return np.max(np.abs(a - b) / scale)


def assert_close(name, got, ref, tol):
    e = rel_err(got, ref)
    assert e <= tol, f"{name}: max scaled error {e:.3e} > {tol:.1e}"
    return e


GPU_TO_ORA = dict(grad=O.ORA_GRAD, phi=O.ORA_PHI, lambda_f=O.ORA_LAMBDA_F, lambda_c=O.ORA_LAMBDA_C,
                  flux=O.ORA_FLUX, res=O.ORA_RES, dwstar=O.ORA_DWSTAR, dw=O.ORA_DW, ghost=O.ORA_GHOST,
                  geom_cell=O.ORA_GEOM_CELL, geom_face=O.ORA_GEOM_FACE)


def make_pair(mesh, flow, W0=None, precision=0, **ctx_kw):
    from paper_1709_00803_gb300 import igks
    ctx = igks.Context(precision=precision, **ctx_kw)
    sid = ctx.mesh_upload(mesh)
    ctx.set_flow(sid, flow)
    ctx.init_freestream(sid)
    ora = O.Oracle(mesh, flow)
    if W0 is not None:
        ctx.set_fields(sid, W0)
        ora.set_W(W0)
    return ctx, sid, ora


def seeded(mesh, flow, seed=1, amp=0.05):
    return F.perturbed_state(mesh, flow, seed=seed, amp=amp)
