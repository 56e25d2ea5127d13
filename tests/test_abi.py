"""The C-ABI library loads, exports every entry point include/*.h declares, and
rejects bad configurations on the host (no GPU work in this file)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b((?:lbm|fem|fsi|mlp|batch)_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_02375_gb300 import lbm
    return lbm.load()


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ("lbm_create", "lbm_step", "lbm_get_macros", "lbm_destroy", "lbm_workspace_size"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_bad_configs_rejected_on_host(lib):
    from paper_1710_02375_gb300 import lbm
    bad = [
        lbm.make_config(10, 8, 8, 8, 0.9),                # unknown lattice
        lbm.make_config(9, 8, 8, 2, 0.9),                 # D2Q9 with nz > 1
        lbm.make_config(27, 8, 8, 8, 1.5),                # beta outside (0,1)
        lbm.make_config(27, 0, 8, 8, 0.9),                # empty lattice
        lbm.make_config(27, 8, 8, 8, 0.9, storage=7),     # unknown storage
        lbm.make_config(27, 8, 8, 8, 0.9, storage=3),     # FP64 storage is D2Q9 only
        lbm.make_config(27, 8, 8, 8, 0.9, bc=(0, 1, 0, 0, 0, 0)),  # unpaired periodic face
    ]
    for cfg in bad:
        n = ctypes.c_size_t()
        assert lib.lbm_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == lbm.LBM_EINVAL
        out = ctypes.c_void_p()
        assert lib.lbm_create(ctypes.byref(cfg), None, 0, ctypes.byref(out)) == lbm.LBM_EINVAL
        assert out.value is None
        assert len(lib.lbm_last_error(None)) > 0


def test_workspace_size_counts_populations(lib):
    from paper_1710_02375_gb300 import lbm
    a = lbm.lbm_workspace_size(lbm.make_config(27, 64, 64, 64, 0.9))
    b = lbm.lbm_workspace_size(lbm.make_config(27, 64, 64, 64, 0.9, storage=lbm.LBM_STORE_F16))
    c = lbm.lbm_workspace_size(lbm.make_config(27, 64, 64, 64, 0.9, storage=lbm.LBM_STORE_F16N))
    pops = 2 * 27 * 64 ** 3
    assert a - b == pops * 2
    assert b == c
    assert a >= pops * 4
    d9 = lbm.lbm_workspace_size(lbm.make_config(9, 64, 64, 1, 0.9, storage=lbm.LBM_STORE_F64))
    f9 = lbm.lbm_workspace_size(lbm.make_config(9, 64, 64, 1, 0.9))
    assert d9 - f9 >= 2 * 9 * 64 * 64 * 4


def test_null_context_calls_fail_cleanly(lib):
    from paper_1710_02375_gb300 import lbm
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_check(None) == lbm.LBM_EINVAL
    lib.lbm_destroy(None)
