"""CPU checks of the boundary: the library builds for sm_103a, loads without a
GPU, and exports every entry point include/dco_stereo.h declares."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_02300_gb300 import binding
    return binding


def test_header_declares_the_boundary(lib):
    names = lib.header_functions()
    for required in ("dco_stereo_create", "dco_stereo_match", "dco_stereo_destroy", "dco_stereo_match_batch",
                     "dco_stereo_census", "dco_stereo_arms", "dco_stereo_cost_volume", "dco_stereo_lr_check",
                     "dco_stereo_match_host", "dco_params_default", "dco_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    missing = [n for n in lib.header_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    p = lib.Params.default()
    assert (p.lambda_ad, p.lambda_census, p.gamma_l) == (10.0, 40.0, 1.0)
    assert abs(p.eps - 0.8) < 1e-7
    assert (p.census_w, p.census_h, p.arm_l1, p.arm_l2, p.tau1, p.tau2, p.lr_tol) == (9, 7, 34, 17, 20, 6, 1)
    L = lib.lib()
    assert L.dco_status_string(0) == b"ok"
    assert L.dco_status_string(3) == b"workspace budget exceeded"
    assert L.dco_params_default(None) == lib.DCO_EINVAL
    # workspace sizing is host arithmetic: per-pixel buffers plus one pass of slices
    ws = lib.Stereo.workspace_bytes(640, 480, 64, p)
    npx = 640 * 480
    assert ws >= npx * (2 * 16 + 2 * 4 + 2 * 2)
    assert ws < npx * 64 * 4 * 2 + npx * 80   # never more than one full slice pair
    assert lib.Stereo.workspace_bytes(8, 8, 9, p) == 0          # D > W
    assert lib.Stereo.workspace_bytes(1920, 1080, 256, p) < 2 * 1920 * 1080 * 256  # no full volume
    bad = lib.Params.default(arm_l1=41)
    assert lib.Stereo.workspace_bytes(64, 64, 16, bad) == 0
    # Eq. 3's range [d_min, d_min + D - 1]: d_min >= 0, the largest disparity
    # at most 255 and below W
    ok = lib.Params.default(d_min=200)
    assert p.d_min == 0
    assert lib.Stereo.workspace_bytes(320, 64, 56, ok) > 0
    assert lib.Stereo.workspace_bytes(320, 64, 57, ok) == 0            # d = 256
    assert lib.Stereo.workspace_bytes(250, 64, 50, ok) > 0             # largest d = W - 1
    assert lib.Stereo.workspace_bytes(249, 64, 50, ok) == 0            # d_min + D > W
    assert lib.Stereo.workspace_bytes(64, 64, 16, lib.Params.default(d_min=-1)) == 0
    # tile shapes: 0 (automatic) or 32 .. 16384 positions; they do not
    # change the workspace
    for h, v, ok_ in ((0, 0, True), (32, 32, True), (16384, 96, True), (16, 0, False), (0, 31, False),
                      (-1, 0, False), (0, 16385, False)):
        ws_t = lib.Stereo.workspace_bytes(640, 480, 64, lib.Params.default(h_chunk=h, v_chunk=v))
        assert (ws_t == ws) if ok_ else (ws_t == 0), (h, v)
    # the slices hold D disparities, not d_min + D
    assert lib.Stereo.workspace_bytes(320, 64, 56, ok) == lib.Stereo.workspace_bytes(320, 64, 56, p)


def test_create_without_gpu_reports_an_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.lib().dco_stereo_create(ctypes.byref(h), 0, 0)
    assert rc != lib.DCO_OK and not h.value
