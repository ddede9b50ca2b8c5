"""Host-side checks of the C ABI boundary: the library builds, loads and
exports every function include/sph.h declares.  No compute call is made
(none of these needs a GPU)."""
import ctypes

import pytest

from paper_2107_01276_gb300 import build as B
from paper_2107_01276_gb300 import sph


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    L = ctypes.CDLL(path)
    names = sph.declared_functions()
    assert "sph_create" in names and "sph_step" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_abi_covers_the_core_entry_points():
    names = set(sph.declared_functions())
    for n in ("sph_create", "sph_load_particles", "sph_rhs", "sph_step",
              "sph_adapt", "sph_background", "sph_forces", "sph_read",
              "sph_batch_step", "sph_batch_adapt", "sph_destroy",
              "sph_last_error"):
        assert n in names


def test_default_params_are_the_papers():
    P = sph.Params()
    sph.lib().sph_default_params(ctypes.byref(P))
    assert P.dim == 2
    assert P.alpha_e == 1.5
    assert P.split_alpha == 0.9 and P.split_eps == 0.4
    assert P.merge_iters == 3 and P.shift_iters == 3
    assert P.Cr == 1.08
    assert P.pavg_mode == 0 and P.edac_diff_denominator == 1 \
        and P.edac_rho_factor == 1


def test_params_struct_layout_matches_header():
    """Field order and count of the ctypes mirror follow include/sph.h."""
    import os
    import re
    txt = open(os.path.join(B.INCLUDE, "sph.h")).read()
    body = txt[txt.index("typedef struct {\n    int dim;"):]
    body = body[:body.index("} sph_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"([a-zA-Z_0-9]+)(?:\[2\])?\s*[,;]", body)
    assert names == [f for f, _ in sph.Params._fields_]


def test_null_and_invalid_arguments_rejected_without_gpu():
    L = sph.lib()
    out = ctypes.c_void_p()
    assert L.sph_create(None, None, ctypes.byref(out)) == sph.SPH_EINVAL
    P = sph.Params()
    L.sph_default_params(ctypes.byref(P))
    P.capacity = 0                       # invalid: rejected before any CUDA call
    assert L.sph_create(ctypes.byref(P), None, ctypes.byref(out)) == \
        sph.SPH_EINVAL
    assert b"capacity" in L.sph_last_error(None)
    P.capacity = 10
    P.dim = 3
    assert L.sph_create(ctypes.byref(P), None, ctypes.byref(out)) == \
        sph.SPH_EINVAL
    assert L.sph_rhs(None) == sph.SPH_EINVAL
    assert L.sph_destroy(None) == sph.SPH_EINVAL


def test_batch_arguments_rejected_without_gpu():
    """The batched step's argument checks come before any CUDA call."""
    L = sph.lib()
    out = ctypes.c_void_p(123)
    assert L.sph_batch_create(0, None, ctypes.byref(out)) == sph.SPH_EINVAL
    assert out.value is None                     # *out cleared on error
    assert L.sph_batch_create(1 << 21, None, ctypes.byref(out)) == sph.SPH_EINVAL
    assert L.sph_batch_create(4, None, None) == sph.SPH_EINVAL
    failed = ctypes.c_int(7)
    arr = (ctypes.c_void_p * 1)(None)
    assert L.sph_batch_step(None, arr, 1, None, ctypes.byref(failed)) == sph.SPH_EINVAL
    assert failed.value == -1
    assert L.sph_batch_destroy(None) == sph.SPH_EINVAL
    assert L.sph_batch_launches(None) == -1
    assert L.sph_batch_graph_steps(None) == -1
    assert L.sph_batch_set_graphs(None, 1) == sph.SPH_EINVAL
