"""The C-ABI library loads and exports every symbol include/qxd.h declares,
and host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

import __graft_entry__ as ge
from paper_1710_08839_gb300 import build as B
from paper_1710_08839_gb300 import qxd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    ge.build()


def declared_symbols():
    syms = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            syms |= set(re.findall(r"\b(qxd_\w+)\s*\(", txt))
    return syms


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["qxd_lattice_create", "qxd_lattice_destroy", "qxd_set_gauge", "qxd_set_params",
                 "qxd_sw_build", "qxd_Dw", "qxd_last_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.library_path())
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() <= set(qxd.SIGNATURES), declared_symbols() - set(qxd.SIGNATURES)


@pytest.mark.parametrize("dims,mask", [((3, 4, 4, 4), 14), ((4, 4, 4, 5), 14), ((4, 4, 4, 4), 4),
                                        ((4, 0, 4, 4), 14), ((4, 4, 4, 4), 1)])
def test_create_rejects_bad_geometry(dims, mask):
    with pytest.raises(qxd.QxdError) as e:
        qxd.qxd_lattice_create(*dims, mask, 0)
    assert e.value.code == qxd.QXD_ERR_ARG


def test_null_arguments_are_errors():
    lib = qxd.lib()
    assert lib.qxd_Dw(None, None, None, 0, None) == qxd.QXD_ERR_ARG
    assert lib.qxd_set_params(None, 0.0, 0.0, 0.0, 0) == qxd.QXD_ERR_ARG
    assert lib.qxd_sw_build(None) == qxd.QXD_ERR_ARG
    assert lib.qxd_sap_multi(None, 1, None, None, 5, 5, None) == qxd.QXD_ERR_ARG
    assert lib.qxd_lattice_destroy(None) == qxd.QXD_OK
    assert "NULL" in qxd.qxd_last_error() or qxd.qxd_last_error() != ""


def test_pseudofermion_entry_points_check_arguments():
    lib = qxd.lib()
    out = ctypes.c_double()
    assert lib.qxd_sw_logdet(None, qxd.QXD_SITES_ODD, ctypes.byref(out)) == qxd.QXD_ERR_ARG
    p = qxd.qxd_mscg_defaults()
    assert (p.tol, p.max_iter, p.flags, p.prec, p.delta) == (1e-10, 10000, 0, 0, 0.01)
    info = qxd.qxd_mscg_info()
    sig = (ctypes.c_double * 1)(0.1)
    xs = (ctypes.c_void_p * 1)(None)
    assert lib.qxd_mscg(None, 1, sig, xs, None, ctypes.byref(p), ctypes.byref(info), None, None) == \
        qxd.QXD_ERR_ARG
    assert info.status == qxd.QXD_ERR_ARG
    assert lib.qxd_rational_apply(None, 1, sig, sig, None, None, ctypes.byref(p), ctypes.byref(info),
                                  None) == qxd.QXD_ERR_ARG


def test_engine_entry_points_check_arguments():
    lib = qxd.lib()
    c, r = ctypes.c_longlong(), ctypes.c_longlong()
    assert lib.qxd_engine_graph_stats(None, ctypes.byref(c), ctypes.byref(r)) == qxd.QXD_ERR_ARG
    a, h, s = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_longlong()
    assert lib.qxd_engine_stats(None, ctypes.byref(a), ctypes.byref(h), ctypes.byref(s)) == qxd.QXD_ERR_ARG
    assert lib.qxd_engine_create(None, 0, 1, None) == qxd.QXD_ERR_ARG
    e = ctypes.c_void_p()
    assert lib.qxd_engine_create(ctypes.byref(e), 0, 0, None) == qxd.QXD_ERR_ARG
    assert lib.qxd_engine_destroy(None) == qxd.QXD_OK


def test_tuning_entry_points_without_a_gpu():
    lib = qxd.lib()
    prev = lib.qxd_set_autotune(0)
    assert lib.qxd_set_autotune(prev) == 0
    need = ctypes.c_size_t()
    assert lib.qxd_tune_report(None, 0, ctypes.byref(need)) == qxd.QXD_OK and need.value >= 1
    assert lib.qxd_dw_shape(None, qxd.QXD_FP32, None, None, None, None) == qxd.QXD_ERR_ARG
    assert lib.qxd_dw_set_shape(None, qxd.QXD_FP32, 1, 128, 2) == qxd.QXD_ERR_ARG
