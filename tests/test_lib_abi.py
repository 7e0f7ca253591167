"""The C-ABI library builds, loads without a GPU and exports every entry point of the header."""
import ctypes
import subprocess

import pytest

import paper_1805_10638_gb300 as km
from paper_1805_10638_gb300 import _lib


def test_library_exports_every_declared_symbol():
    L = km.load()
    names = _lib.exported_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_path()], capture_output=True, text=True)
    if out.returncode == 0:
        defined = {ln.split()[-1] for ln in out.stdout.splitlines() if ln.strip()}
        for n in names:
            assert n in defined, n


def test_defaults_and_status_strings_without_gpu():
    p = km.default_params()
    assert (p.m_max, p.m_init, p.max_iter, p.lloyd_only, p.fixed_m) == (10, 2, 1000, 0, 0)
    assert (p.eps1, p.eps2, p.tol, p.rank_tol) == (0.02, 0.5, 0.0, 1e-12)
    assert km.default_params(fixed_m=1, m_init=5).fixed_m == 1
    with pytest.raises(KeyError):
        km.default_params(no_such_field=1)
    # the structs the Python side uses have the header's fields in the header's order
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(_lib._build.PKG), "include", "kmeans_aa.h")).read()
    for name, cls in (("kmeans_params", _lib.kmeans_params), ("kmeans_info", _lib.kmeans_info),
                      ("kmeans_data", _lib.kmeans_data), ("kmeans_problem", _lib.kmeans_problem),
                      ("kmeans_server_stats", _lib.kmeans_server_stats), ("kmeans_state", _lib.kmeans_state)):
        body = re.search(r"typedef struct \{([^}]*)\} " + name + ";", hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = [f for decl in body.split(";") for f in re.findall(r"(\w+)(?:\[\d+\])?\s*(?:,|$)", decl.strip())]
        assert [f for f, _ in cls._fields_] == fields, name
    L = km.load()
    assert L.kmeans_status_string(1) == b"KM_EINVAL"
    assert L.kmeans_status_string(5) == b"KM_ENONFINITE"
    assert L.kmeans_last_error(None) == b""


def test_null_arguments_rejected_before_any_cuda_call():
    L = km.load()
    assert L.kmeans_create(None, 0, 0, None) == _lib.KM_EINVAL
    assert L.kmeans_destroy(None) == _lib.KM_OK
    data = _lib.kmeans_data(None, None, 10, 2, 0)
    assert L.kmeans_assign(None, ctypes.byref(data), None, 1, None, None, None, None) == _lib.KM_EINVAL

    u = (ctypes.c_double * 2)(0.1, 0.2)
    assert L.kmeans_seed_pp(None, ctypes.byref(data), 2, u, None, None) == _lib.KM_EINVAL
