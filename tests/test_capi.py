"""The C-ABI library loads and exports every entry point include/tdgl.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tdgl.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdgl_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_28800_b300 import build as pb
    path = pb.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = declared()
    for must in ("tdgl_ctx_create", "tdgl_sim_create", "tdgl_material_define", "tdgl_set_layers",
                 "tdgl_set_temperature", "tdgl_set_field", "tdgl_step", "tdgl_energy", "tdgl_get_P",
                 "tdgl_relax", "tdgl_batch_create", "tdgl_batch_relax"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2605_28800_b300 import tdgl
    assert sorted(tdgl.EXPORTED) == declared()


def test_library_reports_errors_without_device(lib):
    # without a GPU the context cannot be created; the call must fail with a status, not crash
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    rc = lib.tdgl_ctx_create(ctypes.byref(h), 0, None)
    assert rc != 0


def test_binding_constants_match_the_header():
    # every #define of the header that the binding mirrors has the same value there
    from paper_2605_28800_b300 import tdgl
    defs = dict(re.findall(r"#define\s+TDGL_([A-Z0-9_]+)\s+\(?(-?\d+)", open(HEADER).read()))
    pairs = {"ZPASS_VARIANTS": tdgl.ZPASS_VARIANTS, "ROW_CANDIDATES": tdgl.ROW_CANDIDATES, "EULER": tdgl.EULER, "HEUN": tdgl.HEUN, "RK45": tdgl.RK45,
             "AB3M2": tdgl.AB3M2, "K_STEP": tdgl.K_STEP, "K_ZCONV": tdgl.K_ZCONV, "K_UNET": tdgl.K_UNET,
             "EINVAL": tdgl.EINVAL, "ECUDA": tdgl.ECUDA, "EDIVERGED": tdgl.EDIVERGED, "ETIMEOUT": tdgl.ETIMEOUT}
    for name, value in pairs.items():
        assert name in defs, name
        assert int(defs[name]) == value, name
