"""The C ABI library loads without a GPU and exports every function include/*.h declares."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gdm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_api():
    names = declared_functions()
    for required in ("gdm_init", "gdm_set_overlap", "gdm_set_hamiltonian", "gdm_solve_dm",
                     "gdm_reinit", "gdm_finalize", "gdm_op_product"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1912_13403_gb300 as g
    lib = ctypes.CDLL(g.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_null_handle_paths():
    import paper_1912_13403_gb300 as g
    assert g.status_name(g.GDM_OK) == "GDM_OK"
    assert g.status_name(g.GDM_ERR_CUDA) == "GDM_ERR_CUDA"
    assert g.gdm_last_error(None) == b"null handle"
    assert g.gdm_finalize(None) == g.GDM_OK
    assert g.gdm_set_precision(None, 0) == g.GDM_ERR_ARG
    h = ctypes.c_void_p()
    assert g.gdm_init(None, 10, 5, 0) == g.GDM_ERR_ARG
    assert g.gdm_init(ctypes.byref(h), 10, 0, 0) == g.GDM_ERR_ARG
    assert g.gdm_init(ctypes.byref(h), 10, 10, 0) == g.GDM_ERR_ARG
    assert not h.value
