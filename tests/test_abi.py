"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "frsvt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1509_00296_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("frsvt_create", "frsvt_destroy", "frsvt_svt", "rpca_init", "rpca_ialm_step",
                     "frsvt_get_info", "frsvt_spectral_norm"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    from paper_1509_00296_gb300 import frsvt
    L = frsvt.lib()
    assert L.frsvt_status_string(0) == b"ok"
    assert L.frsvt_status_string(2) == b"unsupported"
    assert L.frsvt_last_error(None) == b"null handle"


def test_invalid_arguments_rejected_on_host(libpath):
    """Host-side validation answers before any device work (no GPU needed)."""
    from paper_1509_00296_gb300 import frsvt
    L = frsvt.lib()
    h = ctypes.c_void_p()
    bad = frsvt.Config(0, 10, 8, 1, 1, 0, 0, 30, 0, 1e-10)           # m_max = 0
    assert L.frsvt_create(ctypes.byref(h), ctypes.byref(bad), None) == 1
    bad = frsvt.Config(10, 10, 129, 1, 1, 0, 0, 30, 0, 1e-10)        # l_max > 128
    assert L.frsvt_create(ctypes.byref(h), ctypes.byref(bad), None) == 1
    bad = frsvt.Config(10, 10, 33, 1, 0, 0, 0, 30, 1, 1e-10)         # wide basis with the adjoint workspace
    assert L.frsvt_create(ctypes.byref(h), ctypes.byref(bad), None) == 2
    bad = frsvt.Config(10, 10, 8, 1, 1, 7, 0, 30, 0, 1e-10)          # unknown precision
    assert L.frsvt_create(ctypes.byref(h), ctypes.byref(bad), None) == 2
    bad = frsvt.Config(10, 10, 8, 1, 1, 0, 0, 30, 4, 1e-10)          # unknown flag bit
    assert L.frsvt_create(ctypes.byref(h), ctypes.byref(bad), None) == 1
    bad = frsvt.Config(10, 10, 8, 1, 0, 0, 0, 30, 0, 1e-10, 4)       # child streams without the adjoint
    assert L.frsvt_create(ctypes.byref(h), ctypes.byref(bad), None) == 1
    bad = frsvt.Config(10, 10, 8, 1, 0, 0, 0, 30, 1, 1e-10, 17)      # more than 16 child streams
    assert L.frsvt_create(ctypes.byref(h), ctypes.byref(bad), None) == 1
    assert L.frsvt_create(None, None, None) == 1
    assert L.frsvt_svt(None, None, 1, 1, 4, ctypes.c_float(1.0), 1, None, 4) == 1


def test_product_path_has_no_oracle_dependency():
    """The package never imports the oracle (the oracle is test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_1509_00296_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, flags=re.M), f


def _header_text():
    return re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)


def _struct_fields(name):
    """(type, field) pairs of `typedef struct name { ... } name;` in the header."""
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), _header_text(), flags=re.S).group(1)
    return re.findall(r"^\s*([a-z0-9_]+)\s+([a-z0-9_]+)\s*;", body, flags=re.M)


_CTYPES = {"int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32, "int64_t": ctypes.c_int64,
           "uint64_t": ctypes.c_uint64, "double": ctypes.c_double, "float": ctypes.c_float}


@pytest.mark.parametrize("cname,pyname", [("frsvt_config", "Config"), ("frsvt_info", "Info")])
def test_binding_structs_match_header(cname, pyname):
    """The ctypes structures of the binding list the header's fields in order with the same types."""
    from paper_1509_00296_gb300 import frsvt
    want = [(f, _CTYPES[t]) for t, f in _struct_fields(cname)]
    got = list(getattr(frsvt, pyname)._fields_)
    assert got == want


def test_binding_constants_match_header():
    """Status codes, device status bits, configuration flags, precisions, phases and WSVT variants."""
    from paper_1509_00296_gb300 import frsvt
    src = _header_text()
    macros = {k: v for k, v in re.findall(r"#define (FRSVT_\w+)\s+\(?([0-9]+u?(?:\s*<<\s*[0-9]+)?)\)?", src)}
    val = lambda k: eval(macros[k].replace("u", ""))
    assert frsvt.CFG_ADJOINT == val("FRSVT_CFG_ADJOINT") and frsvt.CFG_ORTH_LAST == val("FRSVT_CFG_ORTH_LAST")
    assert (frsvt.DEV_RANK_DEFICIENT, frsvt.DEV_NOT_CONVERGED, frsvt.DEV_NONFINITE, frsvt.DEV_TIMEOUT,
            frsvt.DEV_BAD_PROBLEM) == tuple(val("FRSVT_DEV_" + k) for k in
                                            ("RANK_DEFICIENT", "NOT_CONVERGED", "NONFINITE", "TIMEOUT", "BAD_PROBLEM"))
    assert (frsvt.WSVT_EXACT, frsvt.WSVT_FRSVT) == (val("FRSVT_WSVT_EXACT"), val("FRSVT_WSVT_FRSVT"))
    assert frsvt.NPHASE == val("FRSVT_NPHASE")
    enums = dict((k, int(v)) for k, v in re.findall(r"(FRSVT_(?:ERR_\w+|OK|PREC_\w+))\s*=\s*([0-9]+)", src))
    assert {v: k for k, v in frsvt.STATUS_NAMES.items()} == {k: v for k, v in enums.items()
                                                           if k == "FRSVT_OK" or k.startswith("FRSVT_ERR_")}
    assert (frsvt.PREC_FP32, frsvt.PREC_BF16, frsvt.PREC_FP8) == (enums["FRSVT_PREC_FP32"], enums["FRSVT_PREC_BF16"],
                                                                 enums["FRSVT_PREC_FP8"])
