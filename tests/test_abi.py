"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/pss.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(pss_\w+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_boundary():
    d = _declared()
    for name in ["pss_create_grid", "pss_set_state", "pss_step_n", "pss_conserved_quantities",
                 "pss_get_state", "pss_destroy"]:
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing
    assert set(lib.EXPORTED) == set(_declared())


def test_no_device_needed_for_host_only_calls(lib):
    assert lib.pss_version().startswith("pss")
    p = lib.pss_default_params()
    assert p.nx == 64 and p.batch == 1 and p.max_iter == 100


def test_params_layout_matches_header(lib, tmp_path):
    # the ctypes mirror must match the C struct: compile offsetof() probes with gcc
    import subprocess
    P = lib.PssParams
    fields = [f[0] for f in P._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'printf("%zu\\n", offsetof(pss_params, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pss.h"\n'
                   'int main(void){' + body + 'printf("%zu\\n", sizeof(pss_params));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got[:-1] == [getattr(P, f).offset for f in fields]
    assert got[-1] == ctypes.sizeof(P)


def test_bad_arguments_rejected_before_any_device_work(lib):
    import pytest
    bad = [dict(nx=48), dict(ny=8), dict(nx=16384), dict(batch=0), dict(lx=0.0), dict(dt=-1.0),
           dict(eq=7), dict(precision=3)]
    for kw in bad:
        with pytest.raises(lib.PssError) as e:
            lib.pss_create_grid(lib.pss_default_params(**kw))
        assert e.value.code == lib.PSS_E_ARG
