"""CPU checks of the C ABI: the library builds, loads and exports every symbol
that include/pf.h declares; host-side argument validation needs no GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpf():
    from paper_2601_06079_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(libpf):
    names = _declared()
    assert len(names) >= 7
    for n in names:
        assert hasattr(libpf, n), n


def test_binding_covers_header():
    from paper_2601_06079_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared()


def test_create_mesh_validates_on_host(libpf):
    from paper_2601_06079_gb300 import _lib
    _lib.lib()
    ok, ctx, ws = _lib.pf_create_mesh(2, [64, 64], [1.0, 1.0], _lib.PF_MODEL_CH, 1, 0)
    assert ok == 0 and ws >= 2 * 64 * 64 * 4
    # no workspace bound -> PF_ERR_STATE without touching the device
    assert _lib.pf_step_explicit(ctx, 0x1000, 1) == _lib.PF_ERR_STATE
    assert "workspace" in _lib.pf_last_error(ctx)
    assert _lib.pf_bind_workspace(ctx, 0x1001, ws) == _lib.PF_ERR_ARG  # misaligned
    assert _lib.pf_bind_workspace(ctx, 0x1000, ws - 1) == _lib.PF_ERR_ARG  # too small
    _lib.pf_destroy(ctx)
    for bad in ([1, 64], [64, 0]):
        st, _, _ = _lib.pf_create_mesh(2, bad, [1.0, 1.0], _lib.PF_MODEL_AC, 1, 0)
        assert st == _lib.PF_ERR_ARG
    st, _, _ = _lib.pf_create_mesh(2, [2, 8], [1.0, 1.0], _lib.PF_MODEL_CH, 1, 0)
    assert st == _lib.PF_ERR_ARG
    st, _, _ = _lib.pf_create_mesh(2, [8, 8], [1.0, -1.0], _lib.PF_MODEL_AC, 1, 0)
    assert st == _lib.PF_ERR_ARG
    _lib.pf_destroy(None)
