"""The C-ABI library loads and exports every entry point include/dp.h declares
(no GPU needed: nothing here launches a kernel)."""
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(dp_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2407_14675_gb300 import build, dp
    build.build()
    return dp.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["dp_grid_create", "dp_grid_destroy", "dp_value_iterate", "dp_policy_iterate",
              "dp_feedback_control", "dp_simulate_closed_loop", "dp_get_value", "dp_get_policy",
              "dp_last_error", "dp_batch_create", "dp_batch_policy_iterate", "dp_batch_autotune",
              "dp_policy_evaluate"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_same_names(lib):
    from paper_2407_14675_gb300 import dp
    for n in _declared():
        assert hasattr(dp, n), n


def test_struct_layouts_match_header():
    # field names of the ctypes mirrors appear in the header in the same order
    from paper_2407_14675_gb300 import dp
    src = open(os.path.join(ROOT, "include", "dp.h")).read()
    for struct in (dp.dp_grid_desc, dp.dp_solve_opts, dp.dp_solve_stats, dp.dp_grid_info, dp.dp_mlp_train_opts,
                   dp.dp_mlp_train_stats, dp.dp_batch_stats):
        name = struct.__name__
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, flags=re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"(\w+)(?:\[\d\])?\s*[,;]", body)
        assert fields == [f for f, _ in struct._fields_], name


def test_invalid_descriptor_is_rejected_without_gpu_work(lib):
    # validation runs before any CUDA call
    from paper_2407_14675_gb300 import dp
    from paper_2407_14675_gb300 import workloads as W
    d = dp.desc_from_problem(W.config0(), stream=0)
    d.beta = 1.5
    import ctypes as C
    h = C.c_void_p()
    rc = lib.dp_grid_create(C.byref(d), C.byref(h))
    assert rc == dp.DP_EINVAL and not h.value
    assert "beta" in dp.dp_last_error()


def test_binding_constants_match_header():
    # every DP_* number the binding exports equals the header's #define
    from paper_2407_14675_gb300 import dp
    src = open(os.path.join(ROOT, "include", "dp.h")).read()
    defines = dict((k, int(v)) for k, v in re.findall(r"#define\s+(DP_[A-Z0-9_]+)\s+(-?\d+)", src))
    names = [n for n in dir(dp) if n.startswith("DP_") and isinstance(getattr(dp, n), int)]
    assert len(names) >= 20
    for n in names:
        assert n in defines, n
        assert getattr(dp, n) == defines[n], n
    for n in ("DP_EVAL_JACOBI", "DP_EVAL_GMRES", "DP_EVAL_DIAG", "DP_SWEEP_EVAL_DIAG", "DP_SWEEP_VI_DIAG",
              "DP_GMRES_MAX_RESTART"):
        assert n in names


def test_network_parameter_layout_matches_the_library(lib):
    # the flat FP32 vector of dp.h: W1 (256 x 4, row = output), b1, W2, b2, W3,
    # b3, W4 (3 x 256), b4 -- the library's count, the binding's flattening and
    # the reference network's shapes agree, and flattening round-trips
    from paper_2407_14675_gb300 import dp, workloads as W
    params = W.mlp_init_params(seed=3)
    shapes = [(W_.shape, b.shape) for W_, b in params]
    assert shapes == [((256, 4), (256,)), ((256, 256), (256,)), ((256, 256), (256,)), ((3, 256), (3,))]
    flat = dp.flatten_params(params)
    assert flat.dtype == np.float32
    assert lib.dp_mlp_param_count() == flat.size == 4 * 256 + 256 + 2 * (256 * 256 + 256) + 3 * 256 + 3
    back = dp.unflatten_params(flat)
    for (W0, b0), (W1, b1) in zip(params, back):
        assert np.array_equal(np.float32(W0), W1) and np.array_equal(np.float32(b0), b1)
    # the offsets dp.h implies: b1 right after W1, W4 right after b3
    assert np.array_equal(flat[1024:1280], np.float32(params[0][1]))
    assert np.array_equal(flat[-3 - 768:-3].reshape(3, 256), np.float32(params[3][0]))
