"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/claire.h; argument validation that needs no
device (NULL handles)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "claire.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(claire_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire
    return claire.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("claire_create", "claire_transport", "claire_objective_gradient",
                     "claire_hessian_matvec", "claire_solve", "claire_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2401_17493_b300 import claire
    assert sorted(claire.EXPORTED) == _declared()


def test_null_arguments_are_rejected_without_a_device(lib):
    from paper_2401_17493_b300 import claire
    assert lib.claire_default_options(None) == claire.EINVAL
    assert lib.claire_create(64, 64, 64, 4, 1e-2, 1.0, None) == claire.EINVAL
    h = ctypes.c_void_p()
    # invalid shapes are rejected before any CUDA call
    assert lib.claire_create(15, 64, 64, 4, 1e-2, 1.0, ctypes.byref(h)) == claire.EINVAL
    assert lib.claire_create(64, 8, 64, 4, 1e-2, 1.0, ctypes.byref(h)) == claire.EINVAL
    assert lib.claire_create(64, 64, 64, 0, 1e-2, 1.0, ctypes.byref(h)) == claire.EINVAL
    assert lib.claire_create(64, 64, 64, 4, 0.0, 1.0, ctypes.byref(h)) == claire.EINVAL
    # largest grid: 3 N must fit the 32-bit element counts of the kernels (N < 2^31 / 3)
    assert lib.claire_create(1024, 1024, 1024, 4, 1e-2, 1.0, ctypes.byref(h)) == claire.EINVAL
    assert lib.claire_create(896, 896, 896, 4, 1e-2, 1.0, ctypes.byref(h)) == claire.EINVAL
    assert h.value is None
    assert lib.claire_destroy(None) == claire.OK
    assert lib.claire_set_tuning(None, 0, 8, 32) == claire.EINVAL
    assert lib.claire_get_tuning(None, None, None, None) == claire.EINVAL
    assert lib.claire_last_error(None) == b"null context"
    # a wait budget outside 1 .. 2^20 polls is rejected before any launch
    assert lib.claire_wait_selftest(0, 0, None) == claire.EINVAL
    assert lib.claire_wait_selftest((1 << 20) + 1, 1, None) == claire.EINVAL
    o = claire.Options()
    assert lib.claire_default_options(ctypes.byref(o)) == claire.OK
    assert abs(o.eps_opt - 5e-2) < 1e-15 and o.max_pcg == 100 and o.hessian == 0
    assert o.precond == 2 and o.warm_check == 0


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of claire_options, claire_stats and claire_kernel_stat
    have the header's size and field offsets (a C program compiled with gcc
    against include/claire.h prints them)."""
    import shutil
    import subprocess
    from paper_2401_17493_b300 import claire
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    mirrors = {"claire_options": claire.Options, "claire_stats": claire.Stats,
               "claire_kernel_stat": claire.KernelStat}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "claire.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
