"""The C-ABI library builds, loads and exports every declared entry point
(no GPU needed; no compute call is made)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2009_06725_gb300 import build, scvs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "scvs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(scvs_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    assert scvs.lib() is not None


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 25
    L = scvs.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(scvs.SIGNATURES), set(names) ^ set(scvs.SIGNATURES)


def test_default_options():
    o = scvs.scvs_default_opts()
    assert o.tol == 1e-8 and o.restart == 30 and o.precision == scvs.SCVS_PREC_MIXED
    assert o.cheb_u >= 1 and o.max_cycles >= 1
    assert o.stage == -1 and o.krylov == scvs.SCVS_KRYLOV_FGMRES and o.inner_max == 400
    assert o.lap_size == 0 and o.lap_smooth == 0


@pytest.mark.parametrize("field,value", [("lap_size", -2), ("lap_size", 4097), ("lap_smooth", -1), ("lap_smooth", 65),
                                         ("stage", 3), ("schur_agg", 513)])
def test_invalid_options_are_refused_before_any_device_call(field, value):
    o = scvs.scvs_default_opts()
    setattr(o, field, value)
    with pytest.raises(scvs.ScvsError) as e:
        scvs.scvs_create(o)
    assert e.value.code == scvs.SCVS_ERR_ARG


def test_option_struct_layout_matches_the_header(tmp_path):
    """sizeof and field offsets of scvs_opts as the C compiler lays them out equal the binding's."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in scvs.scvs_opts._fields_]
    body = "".join(f'printf("%s %zu\\n", "{f}", offsetof(scvs_opts, {f}));' for f in fields)
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "scvs.h"\nint main(void) { '
                   + body + ' printf("sizeof %zu\\n", sizeof(scvs_opts)); return 0; }\n')
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for f in fields:
        assert int(out[f]) == getattr(scvs.scvs_opts, f).offset, f
    assert int(out["sizeof"]) == ctypes.sizeof(scvs.scvs_opts)


def test_header_constants_match_binding():
    src = open(os.path.join(ROOT, "include", "scvs.h")).read()
    for name, val in re.findall(r"#define (SCVS_[A-Z0-9_]+) \(?(-?\d+)\)?", src):
        assert getattr(scvs, name) == int(val), name


def test_header_is_plain_c(tmp_path):
    """include/scvs.h compiles on its own as C99 (no C++ or torch types in the ABI)."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "scvs.h"\nint main(void) { scvs_opts o; scvs_ckpt_header h; scvs_mode_report r;'
                   ' (void)o; (void)h; (void)r; return 0; }\n')
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
