"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/lbp.h declares, and rejects invalid arguments before any CUDA work."""
import os
import re

import pytest

from paper_1909_13412_gb300 import build as lbp_build
from paper_1909_13412_gb300 import lbp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lbp_build.build()
    return lbp.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "lbp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("lbp_create", "lbp_step", "lbp_read_fields", "lbp_particles_add",
                     "lbp_particles_read", "lbp_destroy", "lbp_vacf_read"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(header_functions()) == set(lbp.exported_symbols())


def test_version(lib):
    assert lbp.lbp_version() >= 100


@pytest.mark.parametrize("args", [
    (0, 4, 4, 0.8), (4, -1, 4, 0.8), (4, 4, 4, 0.5), (4, 4, 4, 0.3), (4, 4, 4, float("nan")),
    (2048, 2048, 1024, 0.8),
])
def test_create_rejects_invalid_boxes_before_touching_the_gpu(lib, args):
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_create(*args)
    assert ei.value.status == lbp.LBP_EINVAL
    assert lbp.lbp_last_error()


def test_create_rejects_unknown_precision(lib):
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_create(4, 4, 4, 0.8, precision=9)
    assert ei.value.status == lbp.LBP_EINVAL


def test_null_handle_is_rejected(lib):
    import ctypes as C
    st = lib.lbp_step(C.c_void_p(0), 1)
    assert st == lbp.LBP_EINVAL
    assert lib.lbp_destroy(C.c_void_p(0)) == lbp.LBP_OK
    phi = C.c_double(-1.0)
    assert lib.lbp_volume_fraction(C.c_void_p(0), -1, C.byref(phi)) == lbp.LBP_EINVAL
    assert phi.value == -1.0


def test_binding_warns_when_a_dense_suspension_is_added(monkeypatch):
    """Section 2.2: the method was checked below a volume fraction of 0.1; the
    binding warns after an add that takes a box beyond it (host logic only: the
    fraction itself comes from lbp_volume_fraction)."""
    import warnings
    monkeypatch.setattr(lbp, "lbp_volume_fraction", lambda h, replica=-1: 0.125)
    with pytest.warns(RuntimeWarning, match="volume fraction 0.125 exceeds 0.1"):
        lbp._warn_if_dense(None)
    for phi in (0.0, 0.05, 0.1):
        monkeypatch.setattr(lbp, "lbp_volume_fraction", lambda h, replica=-1, p=phi: p)
        with warnings.catch_warnings(record=True) as seen:
            warnings.simplefilter("always")
            lbp._warn_if_dense(None)
        assert not seen, phi


@pytest.mark.parametrize("boxes,prec", [
    ([(4, 4, 4, 0.8)] * 257, 0),                       # more than 256 boxes
    ([(4, 4, 4, 0.8), (4, 4, 0, 0.8)], 0),             # one empty box
    ([(4, 4, 4, 0.8), (4, 4, 4, 0.5)], 0),             # one box with nu = 0
    ([(1024, 1024, 1024, 0.8), (1024, 1024, 1024, 0.8)], 0),  # 2^31 nodes in all
    ([], 0),                                           # no box
])
def test_create_batch_rejects_invalid_ensembles_before_touching_the_gpu(lib, boxes, prec):
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_create_batch(boxes, precision=prec)
    assert ei.value.status == lbp.LBP_EINVAL
    assert lbp.lbp_last_error()


def test_create_batch_rejects_mixed_storage(lib):
    import ctypes as C
    descs = (lbp.lbp_lattice_desc * 2)(lbp.lbp_lattice_desc(4, 4, 4, 0.8, lbp.LBP_F32),
                                       lbp.lbp_lattice_desc(4, 4, 4, 0.8, lbp.LBP_BF16))
    out = C.c_void_p()
    st = lib.lbp_create_batch(C.cast(descs, C.c_void_p), 2, C.c_void_p(0), C.byref(out))
    assert st == lbp.LBP_EINVAL and not out.value
    assert "precision" in lbp.lbp_last_error()


def test_autotune_candidate_tables_agree():
    """The header's candidate count, the binding's (variant, rows) table and the
    bench's shape names describe the same ten kernel shapes."""
    text = open(os.path.join(ROOT, "include", "lbp.h")).read()
    m = re.search(r"#define\s+LBP_AUTOTUNE_CANDIDATES\s+(\d+)", text)
    assert m and int(m.group(1)) == len(lbp.AUTOTUNE_SHAPES)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_shapes", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert len(bench.SHAPE_NAMES) == len(set(bench.SHAPE_NAMES)) == len(lbp.AUTOTUNE_SHAPES)
    assert bench.SHAPES["4nodes_1row"] == (3, 1) and bench.SHAPES["bulk_staged"] == (2, 1)
