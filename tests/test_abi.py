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
    assert sgn.sgn_abi_version() == 2


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
        sgn.sgn_batch_set_schedule(b, 2, 64)
    sgn.sgn_batch_destroy(b)
    sgn.sgn_plan_destroy(h)
