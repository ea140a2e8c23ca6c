"""The C ABI library builds, loads and exports every entry point that
include/serbf.h declares; host-side argument checks work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2505_02350_gb300 import build
    build.build()
    from paper_2505_02350_gb300 import _native
    return _native


def _declared():
    src = open(os.path.join(ROOT, "include", "serbf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(serbf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ["serbf_build_neighbors", "serbf_forward", "serbf_backward", "serbf_step", "serbf_add_kernels",
              "serbf_refine", "serbf_bin_points", "serbf_normalize_sdf", "serbf_prune"]:
        assert n in names


def test_library_exports_every_declared_symbol(native):
    lib = C.CDLL(native.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(native.symbols())


def test_version_and_status_strings(native):
    assert b"sm_103a" in native.lib.serbf_version()
    assert native.lib.serbf_status_string(native.SERBF_ECAPACITY) == b"capacity exceeded"


def test_config_defaults_match_algorithm3(native):
    c = native.config_default()
    assert (c.eps, c.tau1, c.tau2, c.tau_m, c.tau_d) == (1e-7, 0.9, 1.1, 0.02, 0.01)
    assert (c.tau_l1, c.tau_l2, c.k_l1, c.k_l2, c.T_e, c.M_e) == (5.0, 0.5, 50, 10, 1600, 2000)
    assert (c.lr, c.lr_p2, c.lr_min) == (0.01, 1e-3, 1e-5)
    assert native.lib.serbf_config_default(None) == native.SERBF_EINVAL


def test_struct_sizes_match_header(native):
    assert C.sizeof(native.Config) == 160
    assert native.STATE_BYTES == 48 + 32 + 64 * 8 + 256 * 4


def test_workspace_sizing_is_host_only(native):
    s = native.WsSizes(1000, 64, 512, 256, 1024, 4, 0)
    b = native.serbf_workspace_bytes(s)
    assert b > 1000 * 16
    bad = native.WsSizes(0, 64, 512, 256, 1024, 4, 0)
    assert native.lib.serbf_workspace_bytes(C.byref(bad), C.byref(C.c_size_t())) == native.SERBF_EINVAL
    big = native.WsSizes(1000, 64, 512, 256, 1024, 4, 0)
    bigger = native.serbf_workspace_bytes(native.WsSizes(2000, 64, 512, 256, 1024, 4, 0))
    assert bigger > native.serbf_workspace_bytes(big)


def test_entry_points_reject_null_arguments_before_any_launch(native):
    L = native.lib
    E = native.SERBF_EINVAL
    assert L.serbf_forward(None, None, None, None, None, None, None, None, None) == E
    assert L.serbf_backward(None, None, None, None, None, None, None, None) == E
    assert L.serbf_step(None, None, None, None, None, None, None, None, None) == E
    assert L.serbf_prune(None, None, None, None, None, None) == E
    assert L.serbf_build_neighbors(None, None, None, None, None, None, None, None) == E
    assert L.serbf_add_kernels(None, None, None, None, None, None, None, None, None, None, 0, None, None) == E
    assert L.serbf_normalize_sdf(None, None, 0, None, None, None) == E
    assert L.serbf_gather(None, None, None, 5, None) == E
    assert L.serbf_state_init(None, None, None) == E
    g = native.Grid()
    assert L.serbf_bin_points(None, None, None, 1, C.byref(g), None, None, None, None, None, None) == E
    ws = native.workspace_struct()
    assert L.serbf_status(C.addressof(ws), None, None, 0, None) == E  # uninitialised workspace
    assert L.serbf_workspace_release(None) == E
    assert L.serbf_workspace_release(C.addressof(ws)) == E


def test_uninitialised_workspace_is_rejected(native):
    ws = native.workspace_struct()
    pts = native.Points(None, None, None, None, 0)
    prm = native.Params(None, None, 1)
    cfg = native.config_default()
    assert native.lib.serbf_forward(C.byref(pts), C.byref(prm), C.byref(cfg), None, None, None, None,
                                    C.addressof(ws), None) == native.SERBF_EINVAL


def test_batch_entry_points_check_arguments_on_the_host(native):
    L = native.lib
    E = native.SERBF_EINVAL
    b = C.c_size_t()
    assert L.serbf_batch_bytes(0, C.byref(b)) == E
    assert L.serbf_batch_bytes(1025, C.byref(b)) == E
    assert L.serbf_batch_bytes(64, C.byref(b)) == native.SERBF_OK and b.value > 0
    bb = native.batch_struct()
    assert L.serbf_epoch_batched(C.addressof(bb), None) == E  # not initialised
    assert L.serbf_batch_warps(C.addressof(bb)) == E
    assert L.serbf_batch_init(C.addressof(bb), None, 1, 0, None, 0, None) == E
    # a field without a workspace is rejected before anything touches the device
    f = (native.Field * 1)()
    cfg = native.config_default()
    f[0].cfg = C.pointer(cfg)
    assert L.serbf_batch_init(C.addressof(bb), f, 1, 0, C.c_void_p(256), 1 << 20, None) == E
    assert L.serbf_batch_init(C.addressof(bb), f, 1, 3, C.c_void_p(256), 1 << 20, None) == E  # bad split

