"""The C-ABI library builds, loads and exports every entry point declared in include/loss.h; host-side argument
and shape validation (no GPU needed: validation happens before any CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2301_05127_gb300 import build

    build.build()
    import paper_2301_05127_gb300 as p

    return p


def _declared():
    text = open(os.path.join(ROOT, "include", "loss.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(loss_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("loss_create_grid", "loss_set_model", "loss_step", "loss_record", "loss_derivative"):
        assert want in names


def test_library_exports_every_declared_symbol(pkg):
    L = ctypes.CDLL(pkg.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert set(pkg._PROTOS) == set(_declared())


def test_status_strings_and_version(pkg):
    L = pkg.lib()
    assert L.loss_version().startswith(b"loss-gb300")
    assert L.loss_status_str(pkg.LOSS_E_SHAPE) == b"LOSS_E_SHAPE"
    assert L.loss_status_str(99) == b"LOSS_E_UNKNOWN"


def _create(pkg, **kw):
    base = dict(dim=2, physics=pkg.LOSS_ACOUSTIC, precision=pkg.LOSS_FP64, n_nb=8, n=(32, 32), p=(2, 2),
                h=(1.0, 1.0), dt=1e-3)
    base.update(kw)
    d = pkg.make_desc(**base)
    h = ctypes.c_void_p()
    st = pkg.lib().loss_create_grid(ctypes.byref(d), 1, None, None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,status", [
    (dict(dim=4), "LOSS_E_SHAPE"),
    (dict(n=(30, 32)), "LOSS_E_SHAPE"),          # 30 % 4 != 0 with p = 4 below
    (dict(p=(4, 2), n=(30, 32)), "LOSS_E_SHAPE"),
    (dict(n_nb=17), "LOSS_E_SHAPE"),             # n_nb > M = 16
    (dict(n_nb=0), "LOSS_E_SHAPE"),
    (dict(dt=0.0), "LOSS_E_SHAPE"),
    (dict(h=(1.0, -1.0)), "LOSS_E_SHAPE"),
    (dict(physics=1), "LOSS_E_SHAPE"),            # elastic needs dim 3
    (dict(precision=7), "LOSS_E_ARG"),
    (dict(p=(32, 2)), "LOSS_E_SHAPE"),            # M = 1
])
def test_shape_validation(pkg, kw, status):
    if kw == dict(n=(30, 32)):
        kw = dict(n=(30, 32), p=(4, 2))
    st, h = _create(pkg, **kw)
    assert pkg.lib().loss_status_str(st).decode() == status
    assert not h.value


def test_null_arguments(pkg):
    L = pkg.lib()
    assert L.loss_create_grid(None, 1, None, None, None) == pkg.LOSS_E_ARG
    h = ctypes.c_void_p()
    assert L.loss_create_grid(None, 1, None, None, ctypes.byref(h)) == pkg.LOSS_E_ARG
    assert L.loss_step(None, 1) == pkg.LOSS_E_ARG
    assert L.loss_destroy(None) == pkg.LOSS_OK


def test_binding_fails_loudly_without_library(pkg, monkeypatch, tmp_path):
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(ImportError):
        pkg.lib()


def test_binding_refuses_buffers_of_the_wrong_size(pkg):
    """The library reads and writes a field's whole dense extent behind a plain pointer, so the binding refuses an
    array or tensor with another element count or element size before it calls the library."""
    import numpy as np
    import torch

    from paper_2301_05127_gb300 import _expect_buffer

    _expect_buffer(np.zeros((3, 4), np.float32), (3, 4), 4, "sigma")
    _expect_buffer(torch.zeros(12, dtype=torch.float64), (3, 4), 8, "sigma")
    for a, esize in ((np.zeros((3, 3), np.float32), 4), (np.zeros((3, 4), np.float64), 4),
                     (torch.zeros(12, dtype=torch.float32), 8), (torch.zeros(13, dtype=torch.float64), 8)):
        with pytest.raises(ValueError):
            _expect_buffer(a, (3, 4), esize, "sigma")
