"""The C-ABI library builds, loads and exports every entry point include/ballcorr.h
declares; argument validation that happens before any device work is checked on CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1711_05075_gb300 as bc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ballcorr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:[a-z_]+\s+)*[a-z_]+\s*\*?\s*(bc_[a-z_]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("bc_create", "bc_destroy", "bc_shape_create", "bc_shapes_create", "bc_shape_destroy", "bc_correlate", "bc_sweep",
              "bc_pairs", "bc_sync",
              "bc_last_error", "bc_version", "bc_profile_begin", "bc_profile_end", "bc_stage_name",
              "bc_shape_moments", "bc_mlp_create", "bc_mlp_destroy", "bc_mlp_features", "bc_mlp_predict",
              "bc_mlp_grads", "bc_mlp_train_step", "bc_mlp_train", "bc_mlp_state", "bc_learned_sweep", "bc_mlp_param_count", "bc_topk", "bc_sweep_plan", "bc_plan_run",
              "bc_plan_destroy", "bc_score", "bc_score_sweep", "bc_query_create", "bc_query_eval", "bc_query_destroy",
              "bc_lift_create", "bc_lift_correlate", "bc_lift_destroy", "bc_get_tuning", "bc_set_tuning", "bc_autotune",
              "bc_correlate_noalloc", "bc_selftest_wait", "bc_learned_sweep_avg", "bc_shape_moments_rot",
              "bc_mlp_features_rows", "bc_mlp_set_features", "bc_mlp_rotated_moments",
              "bc_learned_sweep_cascade", "bc_learned_sweep_coarse"):
        assert f in names


def test_library_exports_every_declared_symbol():
    L = bc.lib()
    for f in declared_functions():
        assert hasattr(L, f), f
    assert "sm_103a" in bc.bc_version()


def _status(fn):
    try:
        fn()
    except bc.BallCorrError as e:
        return e.status, str(e)
    return 0, ""


@pytest.mark.parametrize("kw,status", [
    (dict(N=33, W=6, radii=[0.1]), 5),
    (dict(N=32, W=1, radii=[0.1]), 1),
    (dict(N=32, W=12, radii=[0.1]), 1),
    (dict(N=32, W=6, radii=[]), 1),
    (dict(N=32, W=6, radii=[0.1] * 9), 1),
    (dict(N=32, W=6, radii=[-0.1]), 1),
    (dict(N=32, W=6, radii=[0.1], period=0.0), 1),
    (dict(N=32, W=6, radii=[0.1], sigma=3), 5),
    (dict(N=32, W=6, radii=[0.1], precision=2), 5),
])
def test_create_rejects_bad_parameters_before_device_work(kw, status):
    st, msg = _status(lambda: bc.bc_create(**kw))
    assert st == status, msg
    assert bc.lib().bc_last_error().decode()


def test_null_arguments_are_rejected():
    L = bc.lib()
    assert L.bc_create(None, None, None) == 1
    assert L.bc_destroy(None) == 0
    assert L.bc_shape_destroy(None) == 0
    assert L.bc_shape_create(None, None, None, 0, 0, None) == 1
    assert L.bc_shapes_create(None, 0, None, None, None, 0, None) == 1
    assert L.bc_correlate(None, None, None, None, 1, None, 1) == 1
    assert L.bc_sync(None) == 1
    assert L.bc_selftest_wait(None) == 1
    assert L.bc_profile_begin(None, 4) == 1
    assert L.bc_profile_end(None, None) == 1
    assert [bc.lib().bc_stage_name(i).decode() for i in range(7)] == [
        "prepare", "spread", "fft_z", "fft_y", "fft_x", "ifft_y", "ifft_z"]
    assert bc.lib().bc_stage_name(7).decode() == ""
    assert L.bc_mlp_create(None, 64, None, None) == 1
    assert L.bc_mlp_destroy(None) == 0
    assert bc.bc_mlp_param_count(256) == 256 * 132 + 256 + 256 * 256 + 256 + 256 + 1

    # added entry points: null arguments fail before any device work
    assert L.bc_score(None, None, None, None, 1, ctypes.c_double(0.1), ctypes.c_double(2.0), None, 1) == 1
    assert L.bc_score_sweep(None, None, None, None, 1, 0, ctypes.c_double(0.1), ctypes.c_double(2.0), None, None, 1) == 1
    assert L.bc_query_create(None, None, None, None, 10, None) == 1
    assert L.bc_query_eval(None, None, 1, None, 1) == 1
    assert L.bc_query_destroy(None) == 0
    assert L.bc_lift_correlate(None, None, 0, None, 0, None, None, 1, None, 1) == 1
    assert L.bc_lift_destroy(None) == 0
    assert L.bc_get_tuning(None, None) == 1
    assert L.bc_set_tuning(None, None) == 1
    assert L.bc_autotune(None, None, None, 0, None) == 1
    assert L.bc_learned_sweep_avg(None, None, None, None, None, 1, 1, None, 0, None, None, None, None) == 1


@pytest.mark.parametrize("kw,status", [
    (dict(N=48, Nr=16, L=0.1), 5),
    (dict(N=32, Nr=12, L=0.1), 5),
    (dict(N=32, Nr=16, L=0.0), 1),
    (dict(N=32, Nr=16, L=0.1, period=-1.0), 1),
    (dict(N=32, Nr=16, L=0.1, period_r=0.0), 1),
])
def test_lift_create_rejects_bad_parameters_before_device_work(kw, status):
    st, msg = _status(lambda: bc.bc_lift_create(**kw))
    assert st == status, msg


def test_tuning_struct_matches_the_header():
    src = open(os.path.join(ROOT, "include", "ballcorr.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} bc_tuning;", src).group(1)
    fields = re.findall(r"int\s+(\w+);", body)
    assert fields == [f for f, _ in bc.bc_tuning._fields_]
    body = re.search(r"typedef struct \{([^}]*)\} bc_lift_params;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(?:int|double)\s+(\w+);", body)
    assert fields == [f for f, _ in bc.bc_lift_params._fields_]


def test_shape_arrays_marshalling_on_the_host():
    # The binding's argument marshalling for shape uploads (no device work): host
    # arrays of any float/int type and layout become contiguous FP32 (n, 3) and int32 (n).
    x = np.arange(12, dtype=np.float64).reshape(3, 4)[:, :3]  # non-contiguous float64
    lv = [0, 1, 1]
    xa, la, dev = bc.Shape._arrays(x, lv)
    assert dev == 0 and xa.dtype == np.float32 and la.dtype == np.int32
    assert xa.shape == (3, 3) and xa.flags["C_CONTIGUOUS"] and la.flags["C_CONTIGUOUS"]
    np.testing.assert_array_equal(xa, x.astype(np.float32))
    np.testing.assert_array_equal(la, np.array(lv, np.int32))
    xe, le, _ = bc.Shape._arrays(np.zeros((0, 3)), np.zeros(0))
    assert xe.shape == (0, 3) and le.shape == (0,)
