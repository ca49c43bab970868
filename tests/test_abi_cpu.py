"""Host-side checks of the C ABI (no GPU needed).

* libwf.so builds for sm_103a and exports every function include/wf.h declares, each documented
  with its passage of the paper (or that it has none) and its errors;
* the calls that need no device behave as documented: defaults, error strings,
  argument validation before any CUDA call, and WF_ECUDA (not a crash) when no
  device is present.
"""
import ctypes
import os
import re

import pytest

from paper_2604_19370_gb300.build import build_library


@pytest.fixture(scope="module")
def libpath():
    return build_library()


def _declared(root):
    text = open(os.path.join(root, "include", "wf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wf_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(libpath, repo_root):
    L = ctypes.CDLL(libpath)
    names = _declared(repo_root)
    assert "wf_create" in names and "wf_step" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_every_declaration_is_documented(repo_root):
    # the comment above each declaration cites the paper's passage or says that it has none, and
    # states the call's errors (or that it returns none)
    src = open(os.path.join(repo_root, "include", "wf.h")).read()
    undocumented = []
    for m in re.finditer(r"^(?:int|void|const char\*)\s+(wf_\w+)\(", src, re.M):
        before = src[:m.start()]
        end = before.rfind("*/")
        comment = before[before.rfind("/*", 0, end):end]
        cites = "Sec." in comment or "counterpart" in comment or "paper" in comment
        errors = any(k in comment for k in ("Errors", "WF_E", "error", "No return value", "never NULL"))
        if not (cites and errors):
            undocumented.append(m.group(1))
    assert not undocumented, undocumented


def test_defaults_and_strings(libpath):
    from paper_2604_19370_gb300 import wf

    p = wf.wf_params_default()
    assert p.rho == 1.293 and p.kappa == 0.3 and p.T_ig == 800.0 and p.A_r == 1e-4
    assert abs(p.delta_x - 0.7) < 1e-15 and abs(p.delta_z - 0.075) < 1e-15
    assert p.scheme == wf.WF_PR and p.precision == wf.WF_FP32
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8):
        assert wf.wf_strerror(code) != "unknown status code"
    assert wf.wf_strerror(-99) == "unknown status code"


def test_argument_validation_without_device(libpath):
    from paper_2604_19370_gb300 import wf

    L = wf.lib()
    p = wf.wf_params_default()
    h = ctypes.c_void_p()
    for nx, ny, deg, dt in [(0, 4, 2, 1e-3), (4, 4, 0, 1e-3), (4, 4, 4, 1e-3), (4, 4, 2, 0.0), (4, 4, 2, -1.0)]:
        assert L.wf_create(nx, ny, deg, dt, ctypes.byref(p), ctypes.byref(h)) == wf.WF_EINVAL
        assert not h.value
    bad = wf.wf_params_default(scheme=7)
    assert L.wf_create(4, 4, 2, 1e-3, ctypes.byref(bad), ctypes.byref(h)) == wf.WF_EINVAL
    bad = wf.wf_params_default(rho=-1.0)
    assert L.wf_create(4, 4, 2, 1e-3, ctypes.byref(bad), ctypes.byref(h)) == wf.WF_EINVAL
    assert L.wf_step(None, 1) == wf.WF_EINVAL
    assert L.wf_sync(None) == wf.WF_EINVAL
    assert L.wf_get_dims(None, None, None, None, None) == wf.WF_EINVAL
    assert L.wf_set_state_f32(None, None, None, 0) == wf.WF_EINVAL
    assert L.wf_get_state_f32(None, None, None, 0) == wf.WF_EINVAL
    assert L.wf_batch_set_states(None, None, None, 0) == wf.WF_EINVAL
    assert L.wf_batch_set_states_f32(None, None, None, 0) == wf.WF_EINVAL
    assert L.wf_batch_get_states(None, None, None, 0) == wf.WF_EINVAL
    assert L.wf_batch_get_states_f32(None, None, None, 0) == wf.WF_EINVAL
    d = ctypes.c_double()
    buf = ctypes.create_string_buffer(64)
    assert L.wf_measure_host_link(None, buf, 64, ctypes.byref(d), ctypes.byref(d), ctypes.byref(d)) == wf.WF_EINVAL
    assert L.wf_measure_host_link(buf, buf, 0, ctypes.byref(d), ctypes.byref(d), ctypes.byref(d)) == wf.WF_EINVAL
    assert L.wf_measure_host_link(buf, buf, 64, None, ctypes.byref(d), ctypes.byref(d)) == wf.WF_EINVAL
    L.wf_destroy(None)


def test_no_device_reports_cuda_error(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2604_19370_gb300 import wf

    L = wf.lib()
    p = wf.wf_params_default()
    h = ctypes.c_void_p()
    assert L.wf_create(8, 8, 2, 1e-3, ctypes.byref(p), ctypes.byref(h)) == wf.WF_ECUDA
    assert not h.value


def test_server_and_batch_argument_checks(libpath):
    from paper_2604_19370_gb300 import wf

    L = wf.lib()
    s = ctypes.c_void_p()
    assert L.wf_server_create(0, 4, ctypes.byref(s)) == wf.WF_EINVAL
    assert L.wf_server_create(1 << 20, 0, ctypes.byref(s)) == wf.WF_EINVAL
    assert L.wf_submit(None, None, None) == wf.WF_EINVAL
    assert L.wf_poll(None, 1, None) == wf.WF_EINVAL
    L.wf_server_destroy(None)
    h = ctypes.c_void_p()
    p = wf.wf_params_default()
    assert L.wf_batch_create(8, 8, 2, 1e-3, ctypes.byref(p), 0, ctypes.byref(h)) == wf.WF_EINVAL
    assert L.wf_batch_activate(None, 0, 1) == wf.WF_EINVAL
    assert L.wf_batch_capacity(None) == wf.WF_EINVAL


def test_tuning_argument_checks_without_device(libpath):
    from paper_2604_19370_gb300 import wf

    L = wf.lib()
    assert L.wf_autotune(None, 1) == wf.WF_EINVAL
    assert L.wf_get_tuning(None, None) == wf.WF_EINVAL
    assert L.wf_set_tuning(None, None) == wf.WF_EINVAL


def test_mms_argument_checks_without_device(libpath):
    from paper_2604_19370_gb300 import wf

    L = wf.lib()
    assert L.wf_set_mms(None, None) == wf.WF_EINVAL
    assert L.wf_get_time(None, None) == wf.WF_EINVAL


def test_mean_wind_argument_checks_without_device(libpath):
    from paper_2604_19370_gb300 import wf

    L = wf.lib()
    assert L.wf_set_mean_wind(None, 0, 1.0, 0.0) == wf.WF_EINVAL


def test_launch_counter_without_device(libpath):
    from paper_2604_19370_gb300 import wf

    L = wf.lib()
    assert L.wf_launch_count(None) == wf.WF_EINVAL
    assert wf.wf_launch_count() >= 0
