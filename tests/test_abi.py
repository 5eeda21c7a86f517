"""The C-ABI library loads, exports every declared entry point, matches the header's struct
layout, and rejects invalid arguments before touching a GPU."""
import ctypes as ct
import math
import os
import re
import subprocess

import pytest

from paper_2606_04347_gb300 import abi
from paper_2606_04347_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "etd.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(abi.LIB_PATH):
        from paper_2606_04347_gb300 import build
        build.build()
    return abi.load_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:etd_status|const char \*)\s*(etd_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(abi.SIGNATURES)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    fields = [f for f, _ in abi.etd_params._fields_]
    dfields = [f for f, _ in abi.etd_diag._fields_]
    body = "\n".join(f'printf("p {f} %zu\\n", offsetof(etd_params, {f}));' for f in fields)
    body += "\n" + "\n".join(f'printf("d {f} %zu\\n", offsetof(etd_diag, {f}));' for f in dfields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "etd.h"\nint main(void){\n' + body +
                   '\nprintf("s %zu %zu\\n", sizeof(etd_params), sizeof(etd_diag));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.startswith(("p ", "d ")):
            k, f, off = line.split()
            got[(k, f)] = int(off)
        elif line.startswith("s "):
            _, sp, sd = line.split()
            assert int(sp) == ct.sizeof(abi.etd_params) and int(sd) == ct.sizeof(abi.etd_diag)
    for f in fields:
        assert got[("p", f)] == getattr(abi.etd_params, f).offset, f
    for f in dfields:
        assert got[("d", f)] == getattr(abi.etd_diag, f).offset, f


def _plan_status(lib, p):
    h = ct.c_void_p(123)
    s = abi.params_struct(p)
    code = lib.etd_plan(ct.byref(s), None, ct.byref(h))
    return code, h.value


@pytest.mark.parametrize("change", [
    dict(dim=4), dict(n=(48, 64, 64)), dict(n=(512, 64, 64)), dict(n=(64, 64, 4)), dict(n=(64, 192, 64)),
    dict(half_len=(math.pi, 2.0, math.pi)), dict(tau=0.0), dict(eps_u=-1.0), dict(scheme=3),
    dict(precision=7), dict(cg_maxit=0), dict(band_mask_hi=1.5), dict(model=3),
    dict(model=2, B2=0.0), dict(krylov_tol=-1.0), dict(krylov_tol=1.0),
])
def test_invalid_parameters_rejected_without_gpu(lib, change):
    p = wl.workload("c3", n=64)[0].replace(**change)
    code, h = _plan_status(lib, p)
    assert code == 1 and h is None
    assert lib.etd_last_error().decode() != ""


def test_null_handling(lib):
    assert lib.etd_free(None) == 0
    assert lib.etd_step(None, None, None, 1, None) == 1
    assert lib.etd_plan(None, None, None) == 1


def test_batch_rejects_the_sqrtg_model_without_gpu(lib):
    good = wl.workload("c2", n=32)[0]
    arr = (abi.etd_params * 2)(abi.params_struct(good), abi.params_struct(good.replace(model=2)))
    h = ct.c_void_p(123)
    code = lib.etd_plan_batch(arr, 2, None, 0, ct.byref(h))
    assert code == 1 and h.value is None
    assert "run 1" in lib.etd_last_error().decode()
