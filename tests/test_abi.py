"""The C ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

from conftest import ROOT


def declared_symbols():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            names += re.findall(r"SFAIRSC_API\s+[\w\s\*]+?\b(sfairsc_\w+)\s*\(", text)
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for want in ["sfairsc_create", "sfairsc_solve", "sfairsc_apply_operator", "sfairsc_backward", "sfairsc_kmeans",
                 "sfairsc_destroy", "sfairsc_strerror", "sfairsc_opts_default"]:
        assert want in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_no_gpu_calls_that_need_a_device(built_lib):
    from paper_2210_16435_gb300 import binding as B

    o = B.sfairsc_opts_default()
    assert o.tol == 1e-6 and o.block == 1 and o.prec == B.SFAIRSC_PREC_MIXED
    assert B.sfairsc_strerror(-7) == "eigensolver did not converge"
    assert B.load().sfairsc_opts_default(None) == -1
