"""The C-ABI library builds, loads and exports every entry point declared in include/sph.h
(no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

from paper_2405_05155_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2405_05155_gb300 import build
        build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    # and the Python binding declares a signature for each of them
    assert set(names) <= set(_lib._SIGNATURES)


def test_status_strings_and_argument_checks(lib):
    assert lib.sph_status_string(0).decode() == "SPH_OK"
    assert b"CAPACITY" in lib.sph_status_string(2)
    # argument validation happens on the host, before any device work
    assert lib.sph_kernel_eval(7, 3, 1.0, 2.0, 0, None, None, None, 0, None) == _lib.SPH_ERR_ARG
    assert lib.sph_kernel_eval(0, 4, 1.0, 2.0, 0, None, None, None, 0, None) == _lib.SPH_ERR_ARG
    assert lib.sph_kernel_eval(0, 3, -1.0, 2.0, 0, None, None, None, 0, None) == _lib.SPH_ERR_ARG
    assert lib.sph_kernel_eval(0, 3, 1.0, 2.5, 0, None, None, None, 0, None) == _lib.SPH_ERR_ARG
    assert lib.sph_cell_order(None, None, None, None, None) == _lib.SPH_ERR_ARG
    # the context settings refuse a null context or an unknown value before touching it
    assert lib.sph_set_l2_persist(None, 1) == _lib.SPH_ERR_ARG
    assert lib.sph_set_entry_ring(None, _lib.SPH_RING_AUTO) == _lib.SPH_ERR_ARG
    d = _lib.SphDomain()
    d.dim, d.n, d.h, d.kappa = 3, 10, 0.1, 2.0
    for k in range(3):
        d.len[k] = 0.3           # periodic box shorter than 2 kappa h = 0.4
    d.periodic_mask = 7
    nnz = ctypes.c_int64()
    assert lib.sph_build_neighbors(ctypes.c_void_p(1), ctypes.byref(d), ctypes.c_void_p(1), ctypes.c_void_p(1),
                                   ctypes.c_void_p(1), 10, ctypes.byref(nnz), None) == _lib.SPH_ERR_ARG


def test_struct_layouts_match_header():
    # sph_domain: int32, uint32, int64, 2 doubles, 2 x 3 doubles = 80 bytes
    assert ctypes.sizeof(_lib.SphDomain) == 80
    assert ctypes.sizeof(_lib.EulerianParams) == 80 + 5 * 8 + 8
    assert ctypes.sizeof(_lib.EulerianState) == 12 * 8 + 2 * 8 + 2 * 4
    assert ctypes.sizeof(_lib.TLParams) == 80 + 4 * 8 + 8
    assert ctypes.sizeof(_lib.TLState) == 16 * 8 + 2 * 8 + 2 * 4
    assert ctypes.sizeof(_lib.BatchCase) == 96 + 8 + 8 + 2 * 4
    assert ctypes.sizeof(_lib.BatchState) == 4 * 8
    assert ctypes.sizeof(_lib.RelaxParams) == 80 + 3 * 8 + 16 + 64 * 8


def test_header_constants_match_the_binding():
    import re
    from paper_2405_05155_gb300 import _lib
    hdr = open(os.path.join(ROOT, "include", "sph.h")).read()
    defs = dict(re.findall(r"^#define\s+(SPH_[A-Z0-9_]+)\s+(-?\d+)\b", hdr, flags=re.M))
    checked = 0
    for name, val in defs.items():
        if hasattr(_lib, name):
            assert getattr(_lib, name) == int(val), name
            checked += 1
    for name in ("SPH_PIPE_STREAM", "SPH_PIPE_PERSISTENT", "SPH_PIPE_BULK", "SPH_PIPE_GEOM", "SPH_PASS_RELAX", "SPH_PASS_COMPRESSIBLE", "SPH_TIMER_NEIGHBORS"):
        assert name in defs and hasattr(_lib, name), name
    assert checked >= 10


def test_host_alloc_argument_checks(lib):
    h, d = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.sph_host_alloc(ctypes.c_size_t(0), ctypes.byref(h), ctypes.byref(d)) == _lib.SPH_ERR_ARG
    assert lib.sph_host_alloc(ctypes.c_size_t(64), None, ctypes.byref(d)) == _lib.SPH_ERR_ARG
    assert lib.sph_host_free(None) == _lib.SPH_ERR_ARG


def test_binding_refuses_strided_tensors():
    import torch
    from paper_2405_05155_gb300 import api
    a = torch.zeros((2, 3), dtype=torch.float64)
    assert api._p(a) is not None and api._p(None) is None
    with pytest.raises(ValueError):
        api._p(a.t())
    import numpy as np
    with pytest.raises(ValueError):
        api._p(torch.tensor(np.asfortranarray(np.zeros((2, 3)))))
