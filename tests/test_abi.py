"""CPU checks of the C ABI boundary: the library builds, loads without a GPU
and exports every entry point that include/pcg_beta.h declares; the binding
rejects bad arguments before any device call."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcg_beta.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pcg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12437_gb300 import build
    build.build()
    import paper_1810_12437_gb300 as pb
    return pb.load_library()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("pcg_draw_beta", "pcg_draw_beta_batched", "pcg_draw_beta_uneven", "pcg_adjoint",
                 "pcg_ctx_create", "pcg_ctx_destroy", "pcg_build_rhs", "pcg_phi_mul"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    import paper_1810_12437_gb300 as pb
    assert sorted(pb.exported_symbols()) == declared_functions()
    for name in declared_functions():
        if name != "pcg_options_default":
            assert hasattr(pb, name), name


def test_options_default(lib):
    import ctypes
    from paper_1810_12437_gb300._native import _Options
    o = _Options()
    assert lib.pcg_options_default(ctypes.byref(o)) == 0
    assert (o.precision, o.reliable_k, o.stop_rule, o.use_graph) == (3, 50, 0, 1)   # PCG_PREC_DF32
    assert lib.pcg_options_default(None) == 4


def test_null_context_is_badarg(lib):
    import ctypes
    i, d = ctypes.c_int(), ctypes.c_double()
    assert lib.pcg_draw_beta(None, None, None, None, None, None, 1.0, None, None, 1e-6, 10, None,
                             ctypes.byref(i), ctypes.byref(d)) == 4
    assert lib.pcg_last_error(None) == b"NULL context"
    lib.pcg_ctx_destroy(None)


def test_ctx_create_without_gpu_fails_cleanly(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.pcg_ctx_create(ctypes.byref(h), None, None)
    assert st == 6 and not h.value


def test_build_script_targets_sm103a():
    from paper_1810_12437_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    for src in build.SOURCES:
        assert os.path.exists(os.path.join(build.CSRC, src))


def test_precision_names_match_header():
    """The binding's precision names carry the header's PCG_PREC_* values."""
    import os
    import re
    from paper_1810_12437_gb300._native import PREC
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "pcg_beta.h")).read()
    enum = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"PCG_PREC_(\w+)\s*=\s*(\d+)", hdr)}
    assert enum == PREC


def test_tiled_geometry_and_size_guard(lib):
    """pcg_tiled_plan_applies (host arithmetic): the bench workload's tile and
    strip counts, and the size guard on the plan's 32-bit padded positions
    and int segment counts.  n = 1e8 rows with p = 5e4 and 1e9 nonzeros
    passes the former test nnz + 32 (n + p) < 2^32; with one double-float
    right-hand side per group it has 2 column tiles and fits, but with 4 its
    CSR side has 8 column tiles, 8e8 (tile, row) segments, and 7 pad slots
    for each of them overflow 32-bit positions: the untiled products must
    take it."""
    import paper_1810_12437_gb300 as pb
    assert pb.pcg_tiled_plan_applies(500_000, 50_000, 114_693_671, "df32", 2) == (4, 36)
    assert pb.pcg_tiled_plan_applies(500_000, 50_000, 114_693_671, "df32", 1) == (2, 18)
    assert pb.pcg_tiled_plan_applies(500_000, 50_000, 114_693_671, "fp32", 1) == (1, 9)
    n, p, nnz = 100_000_000, 50_000, 1_000_000_000
    assert nnz + 32 * (n + p) < 2 ** 32
    assert pb.pcg_tiled_plan_applies(n, p, nnz, "df32", 1) == (2, 3553)
    assert pb.pcg_tiled_plan_applies(n, p, nnz, "df32", 4) is None
    assert pb.pcg_tiled_plan_applies(0, 10, 0, "df32", 1) is None
    assert pb.pcg_tiled_plan_applies(10, 10, 5, "df32", 0) is None
