"""The C ABI library builds, loads without a GPU, and exports every symbol
include/qvts.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qvts.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w \*]*?\b([a-z][a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith(("sizeof",))))


@pytest.fixture(scope="module")
def libpath():
    from paper_1810_00204_gb300 import build
    return build.build()


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("qv_model_build", "mdp_value_iterate", "belief_predict", "belief_correct", "leaf_value",
              "qv_tree_plan", "qv_tree_plan_batched", "qv_plan_create", "qv_plan_run", "qv_plan_read",
              "qv_tree_backward", "mdp_value_iterate_checkpointed", "mdp_value_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1810_00204_gb300 import _native
    assert sorted(_native.SIGNATURES) == _declared()
    L = _native.lib()
    assert L.qv_version().decode().startswith("qvts-gb300")


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_1810_00204_gb300 import _native
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "libqvts.so"))
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(ImportError):
        _native.lib()


def test_invalid_arguments_are_rejected_without_gpu(libpath):
    """Host-side validation runs before any CUDA call."""
    from paper_1810_00204_gb300 import _native as N
    L = N.lib()
    assert L.qv_model_build(0, 5, 8, None, None, 1, 1, 0, None, None) == N.QV_ERR_INVALID
    # device pointers are never dereferenced by the sizing call: any non-null value
    m = N.qv_model_t(4, 5, 7, 16, 1, 0, 0.1, 0.9, 0.95, None, 32, 3)    # bad pitch
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None)
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0
    assert b"pitch" in L.qv_last_error()
    m = N.qv_model_t(4, 5, 8, 16, 1, 0, 0.1, 0.9, 0.95, None, 32, 3)
    p = N.qv_plan_params_t(2, 0, 0, 0, 0, 0, None)                # K = 0
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0
    p = N.qv_plan_params_t(N.QV_MAX_DEPTH + 1, 4, 0, 0, 0, 0, None)
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None)
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) > 0
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None, 0, 9)          # items_per_cta above 8
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None, 4096, 4)
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) > 0
    assert L.qv_plan_autotune_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) >= \
        L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p))
    # the anytime stop: a budget in ms, >= 0 (0 = none), fused leaves only
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None, 0, 0, 0, 5.0)
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) > 0
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None, 0, 0, 0, -1.0)
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None, 0, 0, 0, float("nan"))
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, N.QV_LEAF_MATERIALISE, None, 0, 0, 0, 5.0)
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0
    assert b"deadline" in L.qv_last_error()
    # the deepest fused level's form: auto (contraction) or the per-child stencil
    for form in (N.QV_DEEPEST_AUTO, N.QV_DEEPEST_STENCIL):
        p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None, 0, 0, 0, 0.0, form)
        assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) > 0
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None, 0, 0, 0, 0.0, 2)
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0
    assert b"deepest_form" in L.qv_last_error()
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None)
    m.num_beacons = N.QV_MAX_BEACONS + 1
    assert L.qv_plan_workspace_bytes(1, ctypes.byref(m), ctypes.byref(p)) == 0


def test_adjoint_arguments_are_rejected_without_gpu(libpath):
    from paper_1810_00204_gb300 import _native as N
    L = N.lib()
    assert L.qv_tree_backward_workspace_bytes(None, 0) == 0
    assert L.qv_tree_backward(None, 0, 1.0, None, None, None, None, None, None, 0, None) == N.QV_ERR_INVALID
    m = N.qv_model_t(4, 5, 8, 16, 1, 0, 0.1, 0.9, 0.95, None, 32, 3)
    assert L.mdp_value_backward_workspace_bytes(ctypes.byref(m), 0) == 0
    assert L.mdp_value_backward_workspace_bytes(ctypes.byref(m), 16) > 0
    assert L.mdp_value_backward(ctypes.byref(m), 200, 16, None, None, None, None, None, 0, None) == N.QV_ERR_INVALID
    assert L.mdp_value_iterate_checkpointed(ctypes.byref(m), 0, 16, 16, 16, 16, 16, 0, None) == N.QV_ERR_INVALID


def test_model9_arguments_rejected_without_gpu(libpath):
    """qv9_create validates its arguments before it reads the map back."""
    from paper_1810_00204_gb300 import _native as N
    L = N.lib()
    h = ctypes.c_void_p()
    fake = 0x1000  # never dereferenced: every case below fails validation first

    def create(H=10, W=10, goal=5, slip=0.1, ps=0.95, gamma=0.95, depth=2, K=4, null=False):
        s = N.qv9_model_t(H, W, None if null else fake, goal, slip, ps, gamma)
        return L.qv9_create(ctypes.byref(s), depth, K, ctypes.byref(h))

    assert L.qv9_create(None, 2, 4, ctypes.byref(h)) == N.QV_ERR_INVALID
    for kw in (dict(null=True), dict(H=0), dict(W=0), dict(goal=100), dict(goal=-1), dict(slip=0.4),
               dict(ps=0.3), dict(ps=1.2), dict(gamma=1.0), dict(depth=0), dict(depth=4), dict(K=0), dict(K=17)):
        assert create(**kw) == N.QV_ERR_INVALID, kw
    assert L.qv9_workspace_bytes(None) == 0
    v = N.qv9_level_view_t()
    assert L.qv9_level(None, 0, ctypes.byref(v)) == N.QV_ERR_INVALID
    r = N.qv9_plan_result_t()
    assert L.qv9_plan(None, None, None, 0, 0, ctypes.byref(r), None) == N.QV_ERR_INVALID


def test_model9_binding_checks_tensor_shapes():
    """The binding refuses Q and b0 of the wrong shape, type or place before
    it calls the library (the C ABI cannot check sizes)."""
    import torch
    from paper_1810_00204_gb300 import api
    m = object.__new__(api.Model9)   # no handle: the checks come first
    m.H, m.W = 4, 5
    with pytest.raises(ValueError):
        m.plan(torch.zeros(9, 4, 5))                      # on the host
    with pytest.raises(ValueError):
        m._check_grid(torch.zeros(5, 4, 5), (9, 4, 5), "Q")
    with pytest.raises(ValueError):
        m._check_grid(torch.zeros(9, 4, 5, dtype=torch.float64), (9, 4, 5), "Q")


def test_noalloc_binding_checks_tensors_before_the_library():
    """belief_correct_noalloc's binding refuses host, mistyped or wrongly
    shaped tensors before it calls the library, whose C ABI takes bare
    pointers and would write through them."""
    import torch
    from paper_1810_00204_gb300 import api

    class _M:  # stands in for a Model: only its grid shape and device are read
        H, P, device = 4, 8, torch.device("cuda", 0)
    m = _M()
    g = torch.zeros(4, 8)
    with pytest.raises(ValueError):
        api.belief_correct_noalloc(m, g, 0, g, torch.zeros(1))          # all on the host
    with pytest.raises(ValueError):
        api._check_tensor(torch.zeros(4, 5), (4, 8), "cpu", "f", "out")  # wrong shape (and place)
    with pytest.raises(ValueError):
        api._check_tensor(torch.zeros(1, dtype=torch.float64), None, "cpu", "f", "pz")
    with pytest.raises(ValueError):
        api._check_tensor(torch.zeros(8, 4).t(), (4, 8), "cpu", "f", "bbar")  # not contiguous


def test_injected_faults_are_reported_before_any_device_work(libpath, monkeypatch):
    """QVTS_FAULT=oom|invalid: the instrumented calls return the injected
    status and a message naming it before they read any argument or touch a
    device (here there is none), so the fake pointers below are never used."""
    from paper_1810_00204_gb300 import _native as N
    L = N.lib()
    fake = ctypes.c_void_p(0x1000)
    m = N.qv_model_t(4, 5, 8, 16, 1, 0, 0.1, 0.9, 0.95, None, 32, 3)
    p = N.qv_plan_params_t(2, 4, 0, 0, 0, 0, None)
    h = ctypes.c_void_p()
    qp = (ctypes.c_void_p * 1)(0x1000)
    monkeypatch.setenv("QVTS_FAULT", "oom")
    st = L.qv_plan_create(1, ctypes.byref(m), qp, qp, ctypes.byref(p), fake, 1 << 20, ctypes.byref(h), None)
    assert st == N.QV_ERR_WORKSPACE and b"QVTS_FAULT=oom" in L.qv_last_error()
    monkeypatch.setenv("QVTS_FAULT", "invalid")
    st = L.qv_plan_create(1, ctypes.byref(m), qp, qp, ctypes.byref(p), fake, 1 << 20, ctypes.byref(h), None)
    assert st == N.QV_ERR_INVALID and b"QVTS_FAULT=invalid" in L.qv_last_error()
    assert L.belief_predict(ctypes.byref(m), fake, 0, fake, None) == N.QV_ERR_INVALID
    assert b"QVTS_FAULT=invalid" in L.qv_last_error()
    assert not h.value


def test_debug_build_exports_the_same_symbols():
    """The bounds-checked build (-DQV_BOUNDS_CHECK) compiles and has the same ABI."""
    from paper_1810_00204_gb300 import build
    L = ctypes.CDLL(build.build(debug=True))
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
