"""The C-ABI library builds, loads and exports every function the public
headers declare (no device calls: runs without a GPU)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2312_11740_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_2312_11740_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    declared = declared_functions()
    assert declared, "no declarations found"
    missing = declared - exported
    assert not missing, "declared but not exported: %s" % sorted(missing)
    for name in declared:
        assert hasattr(lib, name)


def test_binding_covers_declared_symbols():
    from paper_2312_11740_gb300 import _lib
    assert declared_functions() <= set(_lib.SIGNATURES)


def test_host_only_calls(lib):
    """Calls that touch no device memory: defaults and status strings."""
    from paper_2312_11740_gb300 import _lib
    import ctypes
    o = _lib.mp_opts()
    lib.mp_opts_default(ctypes.byref(o))
    assert (o.precision, o.method, o.nu1, o.nu2, o.max_iters) == (0, 0, 2, 2, 200)
    assert lib.mp_status_str(0) == b"ok"
    assert b"invalid" in lib.mp_status_str(1)
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    bc = (ctypes.c_int * 3)(0, 0, 1)
    st = lib.mp_poisson_setup(ctypes.byref(h), _lib.mp_grid(8, 8, 8), 1.0 / 8, bc, None, 1.0,
                              1e-3, 0.0, None)
    assert st == _lib.MP_ERR_INVALID_ARG
    lib.mp_poisson_destroy(None)
