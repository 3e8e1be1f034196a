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
    assert lib.ot_abi_version() == 1
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
