"""The C-ABI library loads without a GPU and exports every function that
include/*.h declares; host-side argument validation needs no device."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT
from paper_2101_11157_gb300 import wv


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(wv_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("wv_sieve", "wv_bernoulli_pm3", "wv_euler_pm3", "wv_search"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(wv.load()._name)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = [n for n in declared_functions() if not hasattr(wv, n)]
    assert not missing, missing


def test_version_and_errors_without_gpu():
    assert "wv" in wv.wv_version()
    with pytest.raises(wv.WvError) as e:
        wv.wv_congruence_info(99)
    assert e.value.status == wv.WV_EINVAL
    assert "congruence" in wv.wv_last_error()


def test_host_validation_without_gpu():
    lib = wv.load()
    n = ctypes.c_size_t(0)
    # lo > hi and hi > 2^37 are rejected before any device work
    assert lib.wv_sieve(10, 5, None, 0, ctypes.byref(n), None) == wv.WV_EINVAL
    assert lib.wv_search(0, (1 << 37) + 1, None, 0, ctypes.byref(n), None) == wv.WV_EINVAL
    assert lib.wv_sieve(0, 10, None, 0, None, None) == wv.WV_EINVAL
    # n == 0 is a no-op that touches nothing
    assert lib.wv_residues_pm3(None, 0, None, None, None) == wv.WV_OK
    # the formulation and launch options are checked before any device work
    for bad in ({"arith": 24}, {"arith": 53}, {"arith": 3}, {"arith": 10}, {"arith": 19},
                {"arith": 25, "ilp": 4}, {"arith": 31, "ilp": 4}, {"arith": 2, "ilp": 4},
                {"ilp": 4}, {"ilp": 3}, {"block": 48}, {"tiling": 3}, {"tiling": -1}):
        assert lib.wv_residues_ex(None, 0, None, None, wv._options(bad), None) == wv.WV_EINVAL, bad
    for good in ({"arith": 23}, {"arith": 25}, {"arith": 28, "ilp": 1}, {"arith": 9, "ilp": 4},
                 {"arith": 32}, {"arith": 37}, {"arith": 38}, {"arith": 39, "ilp": 1}, {"arith": 21, "ilp": 4},
                 {"check_primes": 1}, {"tiling": 1}, {"tiling": 2, "ilp": 1},
                 {"uform_min31": 1, "uform_min64": 1 << 30}):
        assert lib.wv_residues_ex(None, 0, None, None, wv._options(good), None) == wv.WV_OK, good


def test_every_tuning_grid_passes_option_validation():
    # each option set a tuning grid times must be one the library accepts
    # (n == 0: validated, then nothing runs)
    from paper_2101_11157_gb300 import tune
    lib = wv.load()
    grids = dict(tune.GRIDS)
    grids["batch"] = tune.BATCH_GRID
    for name, grid in grids.items():
        for opt in grid:
            st = lib.wv_residues_ex(None, 0, None, None, wv._options(opt), None)
            assert st == wv.WV_OK, (name, opt, wv.wv_last_error())


def test_binding_structs_match_the_headers(tmp_path):
    """Every struct the binding passes across the boundary has the size and
    field offsets the C headers give it (a C program built with the host
    compiler prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = [s for s in ("wv_options", "wv_hit", "wv_request", "wv_server_config", "wv_query_info")
               if hasattr(wv, s)]
    headers = sorted(os.path.basename(h) for h in glob.glob(os.path.join(ROOT, "include", "*.h")))
    lines = ['#include <stdio.h>', '#include <stddef.h>'] + [f'#include "{h}"' for h in headers]
    lines.append("int main(void) {")
    for s in structs:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(wv, s)._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            s, f, v = line.split()
            got[(s, f)] = int(v)
    for s in structs:
        cls = getattr(wv, s)
        assert got[(s, "size")] == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert got[(s, f)] == getattr(cls, f).offset, (s, f)
