"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/lindblad.h declares.  No compute calls (no GPU here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


HEADER = os.path.join(ROOT, "include", "lindblad.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2608_30860_b300.build import build
    path = build(verbose=False)
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lindblad_setup", "phi_apply", "jump_apply", "steady_state", "low_spectrum", "lindblad_destroy",
                     "steady_state_adjoint",
                     "lindblad_workspace_bytes", "resolvent_apply", "lindbladian_apply"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_opts_struct_layout_and_defaults(lib):
    from paper_2608_30860_b300 import lindblad as B
    o = B.default_opts()
    assert o.tol == 1e-10 and o.krylov_m == 20 and o.gmres_m == 40 and o.eta == 1.0 and o.precision == B.LB_PREC_FP64
    assert o.route == B.LB_ROUTE_SCHUR and o.eig_cond_max == 1e3
    assert o.schur_tol == 1e-12 and o.recycle_k == 8 and not o.gauge_c and not o.batched_tiles
    assert ctypes.sizeof(B.LbOpts) == 104  # C layout: 5 doubles, 9 ints, two pointers, natural padding
    assert ctypes.sizeof(B.LbInfo) == 96


def test_invalid_sizes_rejected_on_host(lib):
    from paper_2608_30860_b300 import lindblad as B
    assert B.lindblad_workspace_bytes(1, 1) == 0
    assert B.lindblad_workspace_bytes(8, 0) == 0
    o = B.default_opts(krylov_m=200)
    assert B.lindblad_workspace_bytes(8, 2, o) == 0


def test_status_strings(lib):
    lib.lb_status_string.restype = ctypes.c_char_p
    assert lib.lb_status_string(-3) == b"LB_ETA_EXCLUDED"
    assert lib.lb_status_string(2) == b"LB_S_SINGULAR"


def test_batched_workspace_query_host_logic():
    """Workspace sizing of the batched engine is host arithmetic: positive and growing with the
    sizes, zero for a size outside [2, 256] or an empty batch."""
    import ctypes

    import paper_2608_30860_b300 as B
    small = B.lindblad_batched_workspace_bytes([16, 40], 2)
    big = B.lindblad_batched_workspace_bytes([16, 40, 160], 2)
    assert 0 < small < big
    assert big % 256 == 0
    assert B.lindblad_batched_workspace_bytes([16, 257], 2) == 0
    assert B.lindblad_batched_workspace_bytes([1], 2) == 0
    lib = B.load_library()
    assert lib.lindblad_batched_workspace_bytes(0, (ctypes.c_int * 1)(16), 2, None) == 0


def test_tuner_and_test_hook_arguments_rejected_on_host():
    """Argument checks that return before any CUDA call: the batched tile autotuner's workspace query and
    entry point, and the bounded-wait test hook."""
    import paper_2608_30860_b300 as B
    lib = B.load_library()
    assert lib.lindblad_batched_tune_workspace_bytes(0, 100) == 0      # d < 1
    assert lib.lindblad_batched_tune_workspace_bytes(2, 1) == 0        # nmax < 2
    assert lib.lindblad_batched_tune_workspace_bytes(2, 300) == 0      # nmax > 256
    tiles = (ctypes.c_int * B.LB_TILE_BUCKETS)()
    assert lib.lindblad_batched_tune(0, 100, None, 0, tiles, None, None) == -1
    assert lib.lindblad_batched_tune(2, 100, None, 0, tiles, None, None) == -1   # null workspace
    assert lib.lb_test_bounded_wait(None, 0, 10.0) == -1
    assert B.LB_TILE_BUCKETS == 16 and B.LB_TILE_SHAPES == len(B.TILE_NAMES) == 4
    src = open(HEADER).read()
    assert "#define LB_TILE_BUCKETS 16" in src and "#define LB_TILE_SHAPES 4" in src
