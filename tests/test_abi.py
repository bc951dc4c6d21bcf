"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/igks.h
declares; the binding's structures match the header's layout. No GPU needed."""
import ctypes as C
import re
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "igks.h")).read()
    return re.findall(r"^(?:int|const char\*)\s+(igks_\w+)\(", src, re.M)


def test_library_exports_every_declared_symbol():
    from paper_1709_00803_gb300 import igks
    L = igks.lib()
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n


def test_struct_layouts_match_header(tmp_path):
    """sizeof and field offsets as the C compiler lays them out, against ctypes."""
    from paper_1709_00803_gb300 import igks
    checks = {"igks_flow": igks.Flow, "igks_status": igks.Status, "igks_options": igks.Options,
              "igks_tuning": igks.Tuning, "igks_server_options": igks.ServerOptions,
              "igks_request": igks.Request, "igks_result": igks.Result,
              "igks_server_status": igks.ServerStatus}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "igks.h"', "int main(void){"]
    for cname, py in checks.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = checks[cname]
        if field == "size":
            assert C.sizeof(py) == int(val), line
        else:
            assert getattr(py, field).offset == int(val), line


def test_oracle_and_library_share_no_code():
    """Neither side includes, imports or links the other."""
    csrc = os.path.join(ROOT, "paper_1709_00803_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    for f in ("igks_oracle.c", "igks_oracle.h", "__init__.py"):
        txt = open(os.path.join(ROOT, "oracle", f)).read()
        assert "paper_1709_00803_gb300" not in txt and "igks_dev" not in txt and "igks.h" not in txt, f


def test_footprint_bound_is_host_only_and_monotone():
    """igks_footprint_bytes runs on the host (no GPU needed) and grows with every size."""
    from paper_1709_00803_gb300 import igks
    from igks_inputs import meshgen as G
    small, big = G.laminar_plate(), G.turbulent_plate()
    a, b = igks.footprint_bytes(small), igks.footprint_bytes(big)
    assert 0 < a < b
    # about 2 kB per cell for these meshes: one 250k-cell solve takes well under 1 GB
    assert 1500 < b / big.n_cells < 2500


@pytest.mark.parametrize("bad", [dict(wait_limit=-1), dict(starve_test=2), dict(sweep_threads=512),
                                 dict(sweep_threads=100), dict(precision=7), dict(sweep_cluster=3)])
def test_create_rejects_bad_options_on_the_host(bad):
    """igks_create checks its options before it touches a device (so this runs without a
    GPU): a negative wait limit, a test hook other than 0/1, more than 256 threads per sweep
    block, a block that is not whole warps, an unknown precision or cluster size."""
    from paper_1709_00803_gb300 import igks
    o = igks.Options(**bad)
    h = C.c_void_p()
    assert igks.lib().igks_create(C.byref(o), C.byref(h)) == igks.EINVAL
    assert not h.value
