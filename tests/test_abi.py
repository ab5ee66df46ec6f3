"""The C ABI library loads, exports every declared symbol and validates arguments (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sgn():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_b", os.path.join(ROOT, "paper_1910_01997_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1910_01997_gb300 as sgn

    return sgn


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sgn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgn_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(sgn):
    names = declared_functions()
    assert len(names) >= 30
    lib = ctypes.CDLL(sgn.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_library_has_no_dynamic_cuda_runtime_dependency(sgn):
    # statically linked cudart: the library loads on hosts without a CUDA runtime in the loader path
    ctypes.CDLL(sgn.LIB_PATH)
    assert sgn.sgn_abi_version() == 4


def test_desc_defaults_and_validation(sgn):
    d = sgn.sgn_plan_desc_default(640, 480, 8, 5)
    assert (d.width, d.height, d.patch, d.max_frames) == (640, 480, 8, 5)
    assert abs(d.huber_k - 9 / 255) < 1e-7 and abs(d.lm_lambda - 1e-3) < 1e-9 and d.fp64_cond == 1e6
    assert d.optimize_normal == 1 and d.min_residuals == 8 and d.image_dtype == sgn.SGN_F32
    h = sgn.sgn_plan_create(d)
    assert sgn.sgn_plan_num_surfels(h) == 80 * 60
    assert sgn.sgn_plan_workspace_bytes(h) > 640 * 480 * 16 * 5
    sgn.sgn_plan_destroy(h)
    bad = [("patch", 5), ("patch", 32), ("width", 4), ("height", 20000), ("max_frames", 0), ("max_frames", 17),
           ("image_dtype", 7), ("huber_k", 0.0), ("huber_k", float("nan")), ("lm_lambda", -1.0),
           ("optimize_normal", 2), ("min_residuals", -1), ("fp64_cond", float("nan")), ("lm_adaptive", 3)]
    for field, value in bad:
        d2 = sgn.sgn_plan_desc_default(640, 480, 8, 5)
        setattr(d2, field, value)
        with pytest.raises(sgn.SgnError) as e:
            sgn.sgn_plan_create(d2)
        assert e.value.status == sgn.SGN_ERR_INVALID_ARGUMENT, field
        assert sgn.sgn_last_error()


def test_ragged_sizes_drop_partial_tiles(sgn):
    for (W, H, P) in ((157, 113, 8), (8, 8, 8), (17, 9, 4), (1920, 1080, 16)):
        h = sgn.sgn_plan_create(sgn.sgn_plan_desc_default(W, H, P, 2))
        assert sgn.sgn_plan_num_surfels(h) == (W // P) * (H // P)
        sgn.sgn_plan_destroy(h)


def test_mapping_validation(sgn):
    h = sgn.sgn_plan_create(sgn.sgn_plan_desc_default(64, 64, 4, 2))
    sgn.sgn_plan_set_mapping(h, 16, 128)
    for lanes, block in ((32, 256), (4, 256), (8, 48), (8, 512)):
        with pytest.raises(sgn.SgnError):
            sgn.sgn_plan_set_mapping(h, lanes, block)
    sgn.sgn_plan_destroy(h)


def test_calls_on_an_unbound_plan_fail_cleanly(sgn):
    h = sgn.sgn_plan_create(sgn.sgn_plan_desc_default(64, 64, 8, 2))
    with pytest.raises(sgn.SgnError) as e:
        sgn.sgn_run(h, 3)
    assert e.value.status == sgn.SGN_ERR_NOT_BOUND
    with pytest.raises(sgn.SgnError) as e:
        sgn.sgn_sync(h, 0)
    assert e.value.status == sgn.SGN_ERR_NOT_BOUND
    with pytest.raises(sgn.SgnError):
        sgn.sgn_set_intrinsics(h, -1.0, 1.0, 0.0, 0.0)
    sgn.sgn_set_intrinsics(h, 56.0, 56.0, 31.5, 31.5)
    for call in (lambda: sgn.sgn_read_results(h, 0, 0, 0, 0, 0, 0, 0, sgn.SGN_DEVICE),
                 lambda: sgn.sgn_read_surfels(h, 0, 0, 0, 0, 0, sgn.SGN_HOST),
                 lambda: sgn.sgn_read_depth_map(h, 0, 0, sgn.SGN_HOST)):
        with pytest.raises(sgn.SgnError) as e:
            call()
        assert e.value.status == sgn.SGN_ERR_NOT_BOUND
    sgn.sgn_plan_destroy(h)


def test_batch_host_side_checks(sgn):
    b = sgn.sgn_batch_create(2)
    h = sgn.sgn_plan_create(sgn.sgn_plan_desc_default(64, 64, 8, 2))
    sgn.sgn_batch_add(b, h)
    sgn.sgn_batch_add(b, h)
    with pytest.raises(sgn.SgnError):
        sgn.sgn_batch_add(b, h)  # full
    assert sgn.sgn_batch_workspace_bytes(b) > 0
    with pytest.raises(sgn.SgnError) as e:
        sgn.sgn_batch_run(b, 3)
    assert e.value.status == sgn.SGN_ERR_NOT_BOUND
    with pytest.raises(sgn.SgnError):
        sgn.sgn_batch_set_schedule(b, 3, 64)
    sgn.sgn_batch_destroy(b)
    sgn.sgn_plan_destroy(h)


def test_circular_surfel_desc_validation(sgn):
    d = sgn.sgn_plan_desc_default(128, 96, 8, 3)
    d.surfel_radius = 8 / 3.5449077  # area of the 8x8 tile
    h = sgn.sgn_plan_create(d)
    sgn.sgn_plan_destroy(h)
    for radius, adaptive in ((-1.0, 0), (0.3, 0), (16.5, 0), (float("nan"), 0), (13.0, 0), (4.0, 1)):
        d = sgn.sgn_plan_desc_default(128, 96, 8, 3)
        d.surfel_radius, d.lm_adaptive = radius, adaptive
        with pytest.raises(sgn.SgnError) as e:
            sgn.sgn_plan_create(d)
        assert e.value.status == sgn.SGN_ERR_INVALID_ARGUMENT, (radius, adaptive)


def test_transfer_and_render_argument_checks(sgn):
    """Host-side checks of the frame-change and render calls, taken before any device work."""
    lib = ctypes.CDLL(sgn.LIB_PATH)
    D4, D12 = ctypes.c_double * 4, ctypes.c_double * 12
    cam, bad_cam = D4(140.0, 140.0, 79.5, 59.5), D4(-1.0, 140.0, 79.5, 59.5)
    rigid = D12(1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0)
    scaled = D12(2, 0, 0, 0, 0, 2, 0, 0, 0, 0, 2, 0)
    host = (ctypes.c_float * 16)()
    p = ctypes.cast(host, ctypes.c_void_p)
    transfer = lambda c, T, n, ptr: sgn._status("sgn_transfer_surfels", c, T, n, ptr, ptr, ptr, ptr, ptr, ptr, ptr, None)
    assert transfer(bad_cam, rigid, 1, p) == sgn.SGN_ERR_INVALID_ARGUMENT
    assert transfer(cam, scaled, 1, p) == sgn.SGN_ERR_INVALID_ARGUMENT
    assert transfer(cam, rigid, -1, p) == sgn.SGN_ERR_INVALID_ARGUMENT
    assert transfer(cam, rigid, 0, None) == sgn.SGN_OK  # nothing to move
    assert transfer(cam, rigid, 2, p) == sgn.SGN_ERR_INVALID_ARGUMENT  # host memory
    assert "device memory" in sgn.sgn_last_error()

    def render(c, W, H, n, radius, ptr):
        return sgn._status("sgn_render_surfels", c, W, H, n, ptr, ptr, ptr, ptr, radius, ptr, ptr, ptr, None)

    assert render(bad_cam, 160, 120, 1, 3.0, p) == sgn.SGN_ERR_INVALID_ARGUMENT
    for W, H in ((0, 120), (160, 0), (16385, 120)):
        assert render(cam, W, H, 1, 3.0, p) == sgn.SGN_ERR_INVALID_ARGUMENT
    assert render(cam, 160, 120, -1, 3.0, p) == sgn.SGN_ERR_INVALID_ARGUMENT
    for radius in (0.0, -2.0, float("nan"), 2000.0):
        assert render(cam, 160, 120, 1, radius, p) == sgn.SGN_ERR_INVALID_ARGUMENT
    assert render(cam, 160, 120, 1, 3.0, p) == sgn.SGN_ERR_INVALID_ARGUMENT  # host memory
    assert lib.sgn_abi_version() == 4
