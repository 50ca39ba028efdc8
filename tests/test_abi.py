"""Host-side checks of the C-ABI library (no GPU needed, no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2209_13049_b300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lqmpc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lqmpc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lqmpc_setup", "lqmpc_solve", "lqmpc_solve_batch", "lqmpc_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(lqmpc_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    assert sorted(binding.EXPORTS) == sorted(declared_functions())


def test_default_options_and_status_strings(lib):
    o = lib.lqmpc_default_options()
    assert o.tol == 1e-8 and o.max_iter == 100 and o.precision == 0
    assert o.tau == 0.995 and o.fallback == 1 and o.refine_max >= 1
    for code in range(10):
        assert lib.lqmpc_status_str(code).decode() == binding.STATUS[code]
    assert lib.lqmpc_status_str(99).decode() == "unknown status"


def test_setup_rejects_bad_arguments_without_device_work(lib):
    h = ctypes.c_void_p()
    # ns = 0 is rejected before any CUDA call
    code = lib.lqmpc_setup(ctypes.byref(h), 0, 1, 1, None, None, None, None, None, None, None, None, None,
                           None, None, None, None, None, None, None, None)
    assert code == 1 and not h.value
    assert lib.lqmpc_solve(None, None, None, None) == 1
    assert lib.lqmpc_solve_batch(None, 0, None, None, None) == 1
    assert lib.lqmpc_solve_batch_warm(None, 0, None, None, 0.0, None, None) == 1
    # general data: rows without their arrays, crossed row bounds
    import numpy as np
    from paper_2209_13049_b300 import inputs
    p = inputs.heat1d(6, 2, 3)
    a = [np.ascontiguousarray(v) for v in (p.A.indptr.astype(np.int32), p.A.indices.astype(np.int32), p.A.data)]
    B = np.asfortranarray(p.B)
    R = np.asfortranarray(p.R)
    ptr = lambda v: v.ctypes.data_as(ctypes.c_void_p)
    gl, gu = np.array([1.0]), np.array([0.0])
    E, F = np.asfortranarray(np.ones((1, 6))), np.asfortranarray(np.ones((1, 2)))
    for g in (binding.General(None, None, 1, None, None, None, None, None),
              binding.General(None, None, 1, ptr(E), ptr(F), ptr(gl), ptr(gu), None)):
        code = lib.lqmpc_setup_general(ctypes.byref(h), 6, 2, 3, ptr(a[0]), ptr(a[1]), ptr(a[2]), ptr(B),
                                       ptr(a[0]), ptr(a[1]), ptr(a[2]), None, None, None, ptr(R),
                                       ptr(p.xl), ptr(p.xu), ptr(p.ul), ptr(p.uu), ctypes.byref(g), None, None)
        assert code == 1 and not h.value
    lib.lqmpc_free(None)


def test_binding_fails_loudly_without_library(tmp_path):
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved


def test_no_oracle_in_product_path():
    """The CUDA package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2209_13049_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text
                assert "import baseline" not in text and "from baseline" not in text
                assert "liboracle" not in text and "oracle.h" not in text
