"""CPU checks of the C ABI: the library loads, exports every function include/lbm.h declares,
the ctypes mirrors of the structs match the C layout, and argument validation (which runs before
any CUDA call) rejects bad parameters with LBM_ERR_ARG.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2501_00846_b300 import solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    L = solver.load()
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def _c_layout(tmp_path):
    src = tmp_path / "layout.c"
    fields_p = ["struct_size", "nx", "ny", "nz", "wall_z", "rho_l", "rho_g", "mu_l", "mu_g", "sigma",
                "width", "mobility", "gravity", "rho_ref", "body", "storage", "stream"]
    fields_o = [f for f, _ in solver.LbmObs._fields_]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void){",
             'printf("lbm_params %zu\\n", sizeof(lbm_params));',
             'printf("lbm_obs %zu\\n", sizeof(lbm_obs));']
    for f in fields_p:
        lines.append(f'printf("p.{f} %zu\\n", offsetof(lbm_params, {f}));')
    for f in fields_o:
        lines.append(f'printf("o.{f} %zu\\n", offsetof(lbm_obs, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return dict((k, int(v)) for k, v in (ln.split() for ln in out.strip().splitlines()))


def test_struct_layout_matches_header(tmp_path):
    lay = _c_layout(tmp_path)
    assert lay["lbm_params"] == ctypes.sizeof(solver.LbmParams)
    assert lay["lbm_obs"] == ctypes.sizeof(solver.LbmObs)
    for name, _ in solver.LbmParams._fields_:
        assert lay["p." + name] == getattr(solver.LbmParams, name).offset, name
    for name, _ in solver.LbmObs._fields_:
        assert lay["o." + name] == getattr(solver.LbmObs, name).offset, name


def test_status_strings_and_version():
    L = solver.load()
    assert L.lbm_abi_version() == 1
    for code in solver.STATUS:
        assert L.lbm_status_string(code)
    assert L.lbm_status_string(12345) == b"unknown status"


def _create(**kw):
    L = solver.load()
    base = dict(nx=16, ny=16, nz=16)
    base.update(kw)
    p = solver.make_params(**base)
    ctx = ctypes.c_void_p(123)
    st = L.lbm_create(ctypes.byref(p), ctypes.byref(ctx))
    return st, ctx, L.lbm_last_error().decode()


@pytest.mark.parametrize("bad", [
    dict(nx=3), dict(nz=0), dict(nx=2000, ny=2000, nz=1000), dict(ny=70000),
    dict(rho_g=0.0), dict(mu_l=-1.0), dict(width=0.0), dict(sigma=-0.1),
    dict(mobility=0.35), dict(mobility=-0.01), dict(wall_z=2),
    dict(gravity=(0.0, 0.0, float("nan"))), dict(storage=7),
])
def test_invalid_parameters_rejected(bad):
    st, ctx, msg = _create(**bad)
    assert st == -1 and msg
    assert ctx.value is None          # *out = NULL on error


def test_struct_size_checked():
    L = solver.load()
    p = solver.make_params(16, 16, 16)
    p.struct_size = 8
    ctx = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(p), ctypes.byref(ctx)) == -1
    assert b"struct_size" in L.lbm_last_error()


def test_null_handles():
    L = solver.load()
    assert L.lbm_step(None, 1) == -1
    assert L.lbm_observables(None, None) == -1
    assert L.lbm_num_nodes(None) == 0
    assert L.lbm_step_count(None) == 0
    assert L.lbm_set_path(None, 0) == -1
    L.lbm_destroy(None)
    p = solver.make_params(16, 16, 16)
    assert L.lbm_create(ctypes.byref(p), None) == -1
