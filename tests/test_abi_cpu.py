"""CPU checks of the C-ABI boundary: the library builds, loads, and exports
exactly the entry points include/tde.h declares (no compute call: no GPU here)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "tde.h")).read()
    return sorted(set(re.findall(r"^TDE_API\s+(?:const\s+char\s+\*|int\s+)(tde_\w+)\(", src, re.M)))


def test_header_declares_the_boundary_calls():
    names = declared()
    for core in ("tde_eos_load_table", "tde_mesh_create", "tde_hydro_stage", "tde_dual_energy_sync"):
        assert core in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol():
    from paper_2609_37859_gb300 import build, tde
    build.build()
    L = tde.lib()
    for n in declared():
        assert hasattr(L, n), n
    assert sorted(declared()) == tde.exported_symbols()
    syms = os.popen("nm -D --defined-only %s" % build.LIB).read()
    exported = sorted(set(re.findall(r" T (tde_\w+)", syms)))
    assert exported == declared()


def test_init_without_gpu_fails_cleanly():
    """No CUDA device in this container: tde_init returns an error code, no crash."""
    import ctypes as C
    from paper_2609_37859_gb300 import tde
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert tde.lib().tde_init(C.byref(h), 0, None) == tde.TDE_ECUDA
    assert tde.lib().tde_last_error(None) == b"null context"


def test_stored_table_is_the_oracle_table():
    """The data file the benchmark reads equals a fresh oracle build (libm may
    differ across machines by an ulp)."""
    import sys
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    from oracle import make_saha_table
    d = np.load(os.path.join(ROOT, "paper_2609_37859_gb300", "data", "eos_saha_hhe_256.npz"))
    fresh = make_saha_table.make()
    for k in ("log10_e", "log10_P", "log10_cs2"):
        assert np.allclose(d[k], fresh[k], rtol=0, atol=1e-12), k
