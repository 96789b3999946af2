"""The C-ABI library loads, exports every entry point of include/dd.h and
rejects invalid arguments before touching the GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2001_10986_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2001_10986_gb300 import dd
    return dd


def _declared():
    txt = open(os.path.join(ROOT, "include", "dd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("dd_create", "dd_sweep", "dd_get_plan", "dd_cost", "dd_half_sweep",
              "dd_set_state", "dd_destroy", "dd_last_error"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(lib.LIB)
    for name in _declared():
        assert hasattr(so, name), name
    assert set(_declared()) == set(lib.EXPORTED)


def _create(lib, mu, nu, n=16, levels=1, b=4, sched=((0.01, 1, 0),)):
    return lib.dd_create(mu, nu, n, levels, b, sched)


def test_create_rejects_bad_arguments(lib):
    n = 16
    mu = np.full((n, n), 1.0 / n**2)
    nu = mu.copy()
    bad = mu.copy(); bad[3, 4] = np.nan
    with pytest.raises(lib.DDError) as e:
        _create(lib, bad, nu)
    assert e.value.status == lib.DD_ERR_ARG
    neg = mu.copy(); neg[0, 0] = -1e-3
    with pytest.raises(lib.DDError):
        _create(lib, neg, nu)
    with pytest.raises(lib.DDError):
        _create(lib, mu, nu * 2.0)                     # masses differ
    with pytest.raises(lib.DDError):
        _create(lib, mu, nu, b=3)                       # b not in {2,4,8}
    with pytest.raises(lib.DDError):
        _create(lib, mu, nu, levels=3)                  # coarsest 4 < 2b
    with pytest.raises(lib.DDError):
        _create(lib, mu, nu, sched=((0.01, 1, 1),))     # level out of range
    with pytest.raises(lib.DDError):
        _create(lib, mu, nu, sched=((-1.0, 1, 0),))     # eps <= 0
    zero = mu.copy(); zero[:4, :4] = 0.0; zero /= zero.sum()
    with pytest.raises(lib.DDError) as e:
        _create(lib, zero, nu)                          # empty basic cell (Def. 3.1)
    assert "basic cell" in str(e.value)


def test_options_default(lib):
    o = lib.dd_options_default()
    assert o.err_tol == 1e-6 and o.trunc == 1e-15 and o.max_iter == 2000
    assert o.x_newton == 1 and o.max_cluster_cells == -1 and o.threads_per_cell == 0
    assert o.dual_refine == 0
    with pytest.raises(TypeError):
        lib.dd_options_default(no_such_option=1)


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: include/dd.h compiles as C99 without warnings
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "dd.h"\nint main(void) { dd_options o; dd_options_default(&o); return o.mode; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_struct_layouts_match_the_binding(tmp_path, lib):
    # the ctypes mirrors of dd_options, dd_profile and dd_sweep_stats have the
    # C layout (sizes and every field offset)
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"dd_options": lib.dd_options, "dd_profile": lib.dd_profile, "dd_sweep_stats": lib.dd_sweep_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dd.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'  printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            parts = ln.split()
            got[tuple(parts[:-1])] = int(parts[-1])
    for sname, cls in structs.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)


def test_load_rejects_files_that_are_not_checkpoints(tmp_path, lib):
    # dd_load checks the file before it touches the device
    bad = tmp_path / "not_a_checkpoint.bin"
    bad.write_bytes(b"hello, this is not a checkpoint" * 4)
    with pytest.raises(lib.DDError) as e:
        lib.dd_load(str(bad))
    assert e.value.status == lib.DD_ERR_ARG and "checkpoint" in str(e.value)
    short = tmp_path / "truncated.bin"
    short.write_bytes(b"DDCKPT01" + b"\x00" * 6)
    with pytest.raises(lib.DDError) as e:
        lib.dd_load(str(short))
    assert e.value.status == lib.DD_ERR_ARG
    with pytest.raises(lib.DDError) as e:
        lib.dd_load(str(tmp_path / "missing.bin"))
    assert e.value.status == lib.DD_ERR_ARG


def test_safeguard_is_on_by_default(lib):
    assert lib.dd_options_default().safeguard == 1
