"""The C ABI library loads without a GPU and exports every function that
include/dynot.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dynot.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(ot_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_04840_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("ot_plan", "ot_solve", "ot_path", "ot_destroy", "ot_last_error", "ot_project", "ot_prox"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version_and_error_string_without_gpu(lib):
    lib.ot_abi_version.restype = ctypes.c_int
    assert lib.ot_abi_version() == 2
    lib.ot_last_error.restype = ctypes.c_char_p
    assert lib.ot_last_error() == b""


def test_grid_defaults(lib):
    from paper_1501_04840_gb300 import binding as b
    g = b.rgb_grid(256, 256, 32)
    assert (g.ndim, list(g.n), list(g.bc), g.P) == (3, [256, 256, 3], [1, 1, 0], 32)
    assert g.sigma == pytest.approx(0.3) and g.tau * g.sigma == pytest.approx(0.99)
    h = b.hue_grid(360, 64)
    assert (h.ndim, h.n[0], h.bc[0]) == (1, 360, 0)


def test_invalid_grids_are_rejected_before_any_device_work(lib):
    """ot_plan validates the grid before it touches CUDA."""
    from paper_1501_04840_gb300 import binding as b
    for P, kw in ((1, {}), (65, {}), (16, {"sigma": -1.0}), (16, {"tau": 10.0})):
        g = b.rgb_grid(32, 32, P, **kw)
        with pytest.raises(b.OTError) as ei:
            b.Plan(g)
        assert ei.value.status in (b.OT_EINVAL, b.OT_EUNSUPPORTED)
    g = b.grid([32, 32, 5], ["neumann", "neumann", "periodic"], 8)   # colour axis longer than the kernels' 4
    with pytest.raises(b.OTError) as ei:
        b.Plan(g)
    assert ei.value.status == b.OT_EUNSUPPORTED


def test_sizes_beyond_the_kernels_index_range_are_rejected(lib):
    """Problems of 2^31 cells or more (32-bit in-problem offsets) and batches whose problems x time
    steps exceed a grid dimension (65535) are refused before any device work."""
    from paper_1501_04840_gb300 import binding as b
    g = b.grid([4096, 4096, 4], ["neumann", "neumann", "periodic"], 32)      # 2^31 cells
    with pytest.raises(b.OTError) as ei:
        b.Plan(g)
    assert ei.value.status == b.OT_EUNSUPPORTED
    with pytest.raises(b.OTError) as ei:
        b.Plan(b.hue_grid(64, 64), batch=1024)                               # 1024 * 64 > 65535
    assert ei.value.status == b.OT_EUNSUPPORTED


def test_product_code_never_reaches_the_oracle():
    """The package and its CUDA sources neither import nor include anything from oracle/ (the oracle is
    test infrastructure; the product path has no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_1501_04840_gb300")
    offenders = []
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if not name.endswith((".py", ".cu", ".cuh", ".h")):
                continue
            path = os.path.join(dirpath, name)
            src = open(path).read()
            if re.search(r"^\s*(import\s+oracle|from\s+oracle\b|from\s+\.\.\s*import\s+oracle)", src, flags=re.M) or \
                    re.search(r'#include\s+"[^"]*oracle/', src):
                offenders.append(os.path.relpath(path, ROOT))
    assert not offenders, offenders


def test_header_and_library_from_plain_c(lib, tmp_path):
    """include/dynot.h is plain C99 (pedantic, no warnings), and a C program links against libdynot.so and
    calls host-only entry points: the ABI version, the grid defaults and an invalid plan's status and
    message."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    from paper_1501_04840_gb300 import _build
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "dynot.h"
int main(void) {
  ot_grid g;
  ot_plan_t p = 0;
  if (ot_abi_version() != OT_ABI_VERSION) return 1;
  ot_grid_rgb(&g, 64, 48, 16);
  if (g.ndim != 3 || g.n[0] != 64 || g.n[1] != 48 || g.n[2] != 3 || g.P != 16) return 2;
  g.P = 1;                                   /* below the supported range */
  if (ot_plan(&g, 1, NULL, &p) != OT_EUNSUPPORTED || p != NULL) return 3;
  if (strlen(ot_last_error()) == 0) return 4;
  puts(ot_last_error());
  return 0;
}
''')
    exe = tmp_path / "abi"
    libdir = os.path.dirname(_build.LIB)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-ldynot", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert "P must be" in run.stdout
