"""The C ABI library loads and exports every entry point that include/dsm.h
declares (no GPU needed: nothing here launches device work)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dsm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dsm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2308_10896_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_2308_10896_b300 import dsm
    assert sorted(dsm.EXPORTED) == _declared()


def test_null_context_is_rejected_without_device_work():
    from paper_2308_10896_b300 import dsm
    lib = dsm.load_library()
    assert lib.dsm_render(None, None, None, None, 0, None, None, None) == dsm.DSM_ERR_INVALID_ARG
    assert lib.dsm_render_backward(None, None, None, None, None) == dsm.DSM_ERR_INVALID_ARG
    assert lib.dsm_sync(None) == dsm.DSM_ERR_INVALID_ARG
    assert lib.dsm_last_error(None) == b"null context"
    assert lib.dsm_create(None) == dsm.DSM_ERR_INVALID_ARG
