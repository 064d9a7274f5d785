"""CPU checks of the C ABI: the library loads, exports every function that
include/droplet.h declares, the ctypes structs match the C layout, and invalid
configurations are rejected before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2005_02867_gb300 import _build, droplet as D, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "droplet.h")


@pytest.fixture(scope="module")
def lib():
    _build.build_library()
    return D.load_library()


def declared_functions():
    src = open(HDR).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(droplet_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(D.EXPORTS)


def test_struct_layout_matches_header(tmp_path):
    fields_c = [f for f, _ in D.DropletConfig._fields_]
    fields_d = [f for f, _ in D.DropletDiag._fields_]
    prog = ['#include <stdio.h>', '#include <stddef.h>', '#include "droplet.h"', "int main(void){"]
    prog.append('printf("%zu %zu\\n", sizeof(droplet_config), sizeof(droplet_diag_t));')
    for f in fields_c:
        prog.append(f'printf("%zu\\n", offsetof(droplet_config, {f}));')
    for f in fields_d:
        prog.append(f'printf("%zu\\n", offsetof(droplet_diag_t, {f}));')
    prog.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(D.DropletConfig)
    assert int(out[1]) == ctypes.sizeof(D.DropletDiag)
    offs = [int(x) for x in out[2:]]
    py = [getattr(D.DropletConfig, f).offset for f in fields_c] + [getattr(D.DropletDiag, f).offset for f in fields_d]
    assert offs == py


@pytest.mark.parametrize("bad", [dict(dt=0.0), dict(n=(2, 128, 1)), dict(D0=-1.0), dict(geom=5), dict(mg_tile=(4, 32)),
                                 dict(mg_tile=(32, 512)),
                                 dict(xc=(1e-3, 4e-3, 0.0)), dict(eq_model=3),
                                 dict(cg_maxit=0), dict(wait_limit=-1), dict(solver_select=2), dict(co_max=-0.1),
                                 dict(co_max=float("nan")), dict(adv_scheme=2), dict(drho_l_dT=float("nan")),
                                 dict(drho_l_dT=-2.0), dict(fiber=2),
                                 dict(fiber=1, adv_scheme=1), dict(fiber=1, drho_l_dT=-0.9),
                                 dict(fiber=1, fiber_radius=0.0)])
def test_invalid_config_rejected_without_device(lib, bad):
    cfg = W.cfg1_axisym_64x128(**bad)
    c = D.make_config(cfg)
    h = ctypes.c_void_p()
    rc = lib.droplet_init(ctypes.byref(c), 1, None, ctypes.byref(h))
    assert rc == -1 and h.value is None
    assert lib.droplet_strerror(rc).decode() == "invalid argument"


def test_null_arguments(lib):
    assert lib.droplet_step(None, 1) == -1
    assert lib.droplet_sync(None) == -1
    lib.droplet_free(None)


def test_status_names(lib):
    names = {rc: lib.droplet_strerror(rc).decode() for rc in range(-9, 1)}
    assert names[-3] == "linear solve not converged"
    assert names[-4] == "non-finite value"
    assert names[-8] == "device wait timed out"
    assert names[-9] == "unknown status"
