"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/cyq.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cyq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(cyq_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cyq_create", "cyq_factor", "cyq_solve", "cyq_solve_adjoint", "cyq_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2512_09058_gb300 import build, cyq
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(cyq.EXPORTS) == declared_functions()


def test_host_logic_without_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    L = cyq.load()
    assert L.cyq_status_string(2) == b"matrix not positive definite"
    N = (ctypes.c_int32 * 1)(4)
    d = cyq.cyq_desc(1, N, N, N, 0, 0, None, 1, 0, 0.0, -1, -1)
    h = ctypes.c_void_p()
    assert L.cyq_create(ctypes.byref(d), ctypes.byref(h)) == 8     # CYQ_ERR_NO_DEVICE
    bad = cyq.cyq_desc(0, N, N, N, 0, 0, None, 1, 0, 0.0, -1, -1)
    assert L.cyq_create(ctypes.byref(bad), ctypes.byref(h)) == 1   # CYQ_ERR_INVALID_ARG


def test_new_entry_points_reject_bad_arguments_without_a_device():
    """Host-side argument checks of the coupling-tail and Newton-assembly entry
    points (no device work: a null handle is refused before anything runs)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    L = cyq.load()
    INVALID = 1
    assert L.cyq_set_pcr_tail(None, 2) == INVALID
    v = ctypes.c_int32(-1)
    assert L.cyq_get_pcr_tail(None, ctypes.byref(v)) == INVALID
    a, o = cyq.cyq_newton_in(), cyq.cyq_newton_out()
    assert L.cyq_assemble_newton(None, ctypes.byref(a), ctypes.byref(o), None) == INVALID


def test_every_entry_point_refuses_a_null_handle_without_device_work():
    """The error behaviour include/cyq.h states for missing arguments: every
    entry point that takes a handle returns CYQ_ERR_INVALID_ARG for NULL (the
    size queries -1, cyq_destroy nothing) before any device call, so this runs
    on a host without a GPU as well."""
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    L = cyq.load()
    INVALID = 1
    one = ctypes.c_int32(1)
    calls = {
        "cyq_factor": (None,) * 8,
        "cyq_solve": (None, None, None, 1, None),
        "cyq_apply_factor": (None, None, None, 1, None),
        "cyq_update_factor": (None,) * 6 + (1, None),
        "cyq_build_rhs": (None,) * 7,
        "cyq_residual": (None,) * 6,
        "cyq_residual_compensated": (None,) * 6,
        "cyq_solve_adjoint": (None,) * 16,
        "cyq_get_instance_status": (None, None, None),
        "cyq_get_stats": (None, None, None),
        "cyq_get_segments": (None, None),
        "cyq_get_escalation_segments": (None, None),
        "cyq_get_stage_factor": (None, 0, 0, None),
        "cyq_autotune": (None,) * 9 + (1, 1, None),
        "cyq_get_launch_shapes": (None, None, None, None, 1),
        "cyq_set_launch_shapes": (None, None, None, 1),
        "cyq_set_pcr_tail": (None, 1),
        "cyq_get_pcr_tail": (None, ctypes.byref(one)),
        "cyq_set_factor_path": (None, 1),
        "cyq_get_factor_path": (None, None, None),
        "cyq_set_sweep_path": (None, 1),
        "cyq_get_sweep_path": (None, None, None),
        "cyq_assemble_newton": (None, None, None, None),
        "cyq_tune_segments": (None,) * 9 + (1, 1, None, None),
        "cyq_pivot_eval": (None,) * 6 + (-1, None),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == INVALID, name
    for name in ("cyq_kkt_size", "cyq_workspace_bytes", "cyq_last_launch_count"):
        assert getattr(L, name)(None) == -1, name
    L.cyq_destroy(None)
