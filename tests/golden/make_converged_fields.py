"""Writes the converged fields that the converged-parity tests compare against.

Every value stored here comes from the CPU oracle alone (`oracle/`): the script runs the
oracle's iteration from the free stream until its own stopping rule fires and saves the
conserved state. Nothing here touches the CUDA library.

  python tests/golden/make_converged_fields.py laminar_plate      (~20 min, one core)
  python tests/golden/make_converged_fields.py blasius_plate      (~35 min, one core)

Cases:
  laminar_plate  the 64 x 32 laminar flat plate (Ma 0.15, Re 1e5, CFL 100) run to density
                 residual 1e-10 relative to its first iteration (the stopping rule of the
                 steady solve, Section III with Eq. 16 residuals);
  blasius_plate  the 64 x 64 verification plate (first spacing 1e-4, same flow) run to the
                 paper's own criterion, Eq. 40 ratio <= 3e-8.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from igks_inputs import fields as F  # noqa: E402
from igks_inputs import meshgen as G  # noqa: E402


def case(name):
    if name == "laminar_plate":
        return G.laminar_plate(), F.laminar_plate_flow(), 40000
    if name == "blasius_plate":
        fl = F.laminar_plate_flow()
        fl.eq40_target = 3e-8
        return G.flat_plate_quads(64, 64, first=1e-4, name="plate_blasius"), fl, 40000
    raise KeyError(name)


def path(name):
    return os.path.join(HERE, f"converged_{name}.npz")


def main(name):
    mesh, flow, cap = case(name)
    o = O.Oracle(mesh, flow)
    t0 = time.time()
    done, st = 0, 0
    while done < cap and st == 0:
        st = o.iterate(500)
        done = int(o.scalars()["iter"])
        print(f"{name}: {done} iterations, {time.time() - t0:.0f} s, res_l2 "
              f"{o.scalars()['res_l2'] / o.scalars()['res_l2_first']:.3e}", flush=True)
    sc = o.scalars()
    if st != 1:
        raise SystemExit(f"{name}: the oracle stopped with status {st} after {done} iterations")
    np.savez_compressed(path(name), W=o.get(O.ORA_W), iters=int(sc["iter"]),
                        res_l2_rel=sc["res_l2"] / sc["res_l2_first"], eq40=sc["eq40"])
    print(f"{name}: converged after {int(sc['iter'])} iterations -> {path(name)}")


if __name__ == "__main__":
    for n in sys.argv[1:] or ["laminar_plate", "blasius_plate"]:
        main(n)
