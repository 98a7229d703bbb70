"""The C-ABI library builds, loads, and exports every entry point that
include/lb.h declares; the binding's struct layouts match the header.  Only
host-side calls are made (no GPU is needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lb():
    import paper_0807_4471_gb300 as lb
    from paper_0807_4471_gb300 import build
    build.build()
    lb.load()
    return lb


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lb_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lb):
    names = declared_functions()
    assert {"lb_create", "lb_init_seeded", "lb_step", "lb_fields", "lb_stress",
            "lb_destroy"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", lb.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lb_\w+)", out))
    missing = names - exported
    assert not missing, missing
    L = lb.load()
    for n in names:
        assert getattr(L, n) is not None


def test_struct_layout_matches_header(lb, tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lb.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(lb_params),"
        " offsetof(lb_params, stress_t0), offsetof(lb_params, tau_A),"
        " offsetof(lb_params, kolmo_k), sizeof(lb_stress_out),"
        " offsetof(lb_stress_out, samples)); return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    P, S = lb.lb_params, lb.lb_stress_out
    assert got == [C.sizeof(P), P.stress_t0.offset, P.tau_A.offset, P.kolmo_k.offset,
                   C.sizeof(S), S.samples.offset]


def test_defaults_and_status_strings(lb):
    p = lb.lb_params_default()
    assert (p.G_A1, p.G_A2, p.G_B1, p.G_B2, p.G_X, p.rho0) == (-12.55, 11.70, -11.80, 10.95,
                                                               0.58, 0.70)
    assert p.tau_A == 1.0 and p.stress_every == 1
    for s in range(-7, 1):
        assert lb.lb_status_string(s)
    assert lb.lb_status_string(-99) == "unknown status"


def test_host_validation(lb):
    ok = lb.make_params(64, 64)
    assert lb.lb_workspace_size(ok) > 18 * 64 * 64 * 4 * 2
    bad = [dict(nx=4), dict(tau_A=0.5), dict(rho0=0.0), dict(precision=7),
           dict(boundary=3), dict(stress_every=0), dict(init_amp=1.5),
           dict(G_X=float("nan"))]
    for kw in bad:
        p = lb.make_params(64, 64)
        for k, v in kw.items():
            setattr(p, k, v)
        with pytest.raises(lb.LbError) as e:
            lb.lb_workspace_size(p)
        assert e.value.status == lb.LB_ERR_INVALID


def test_workspace_scales_with_precision(lb):
    sizes = [lb.lb_workspace_size(lb.make_params(512, 512, precision=p))
             for p in ("fp64", "fp32", "fp16", "bf16")]
    assert sizes[0] > sizes[1] > sizes[2] == sizes[3]
    assert sizes[1] < 2.2 * 18 * 512 * 512 * 4 + (1 << 20)
