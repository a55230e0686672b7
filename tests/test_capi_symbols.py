"""The C-ABI library loads on a machine without a GPU and exports every function the
public headers declare, with matching ctypes signatures in the binding."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\*]+\s+\**(pfmp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared()
    for n in ["pfmp_ctx_create", "pfmp_dslash", "pfmp_mhat", "pfmp_kop", "pfmp_solve"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1609_02652_gb300 import build, capi

    if not os.path.exists(capi.LIB_PATH):
        build.build()
    L = capi.lib()
    for n in declared():
        assert hasattr(L, n), n
        assert n in capi.SIGNATURES, f"{n} missing from the ctypes binding"
    assert L.pfmp_version() >= 100
    assert L.pfmp_strerror(capi.PFMP_E_NOT_CONVERGED) == b"solver did not converge"
