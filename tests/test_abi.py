"""The C-ABI library loads and exports every symbol the header declares; host-side
argument validation rejects bad input before any CUDA work (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libmvct():
    from paper_1903_10088_gb300 import build

    path = build.build()
    from paper_1903_10088_gb300 import mvct

    return mvct.load_library(path)


def header_functions():
    txt = open(os.path.join(ROOT, "include", "mvct.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mvct_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = header_functions()
    for f in ["mvct_plan_create", "mvct_plan_destroy", "mvct_forward", "mvct_back", "mvct_tv_grad",
              "mvct_recon", "mvct_last_error", "mvct_objective", "mvct_recon_opts_init"]:
        assert f in names


def test_library_exports_every_declared_symbol(libmvct):
    for name in header_functions():
        assert hasattr(libmvct, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1903_10088_gb300 import mvct

    assert set(header_functions()) <= set(mvct.EXPORTS)


def oracle_default_rule():
    import oracle

    return oracle.LAMBDA_RULES[oracle.DEFAULTS["lambda_rule"]]


def test_struct_layouts_match_header(libmvct):
    """The opts defaults come back through ctypes with the paper's constants, which
    only works if the binding's struct layout matches the header's."""
    from paper_1903_10088_gb300 import mvct

    o = mvct.ReconOpts()
    libmvct.mvct_recon_opts_init(ctypes.byref(o))
    assert (o.lambda0, o.dlambda_up, o.dlambda_down) == (0.01, 1e-4, 2e-4)
    assert (o.mu0, o.kappa, o.tv_eps, o.barrier_timeout_ms) == (0.05, 50.0, 1e-6, 2000.0)
    assert o.lambda_rule == mvct.LAMBDA_RULES["pass_sliding"] == oracle_default_rule()
    assert o.init_from_input == 0 and not o.d_best_out and not o.lambda_schedule


@pytest.mark.parametrize("field,value", [("n", 0), ("n", 5000), ("n_views", 0), ("n_channels", 0),
                                         ("fov_cm", -1.0), ("sad_cm", 20.0),
                                         ("fan_angle_rad", 4.0), ("view0_rad", float("nan"))])
def test_plan_create_rejects_bad_geometry(libmvct, field, value):
    from paper_1903_10088_gb300 import mvct, phantom

    g = mvct.geometry(phantom.GEOM_128)
    setattr(g, field, value)
    h = ctypes.c_void_p()
    rc = libmvct.mvct_plan_create(ctypes.byref(g), 10, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert libmvct.mvct_last_error()


@pytest.mark.parametrize("S", [0, 3, 201, 2000])
def test_plan_create_rejects_bad_subset_count(libmvct, S):
    from paper_1903_10088_gb300 import mvct, phantom

    g = mvct.geometry(phantom.GEOM_128)  # 200 views
    h = ctypes.c_void_p()
    assert libmvct.mvct_plan_create(ctypes.byref(g), S, ctypes.byref(h)) == -1


def test_null_plan_calls_fail_cleanly(libmvct):
    assert libmvct.mvct_forward(None, None, None, 0, None) == -1
    assert libmvct.mvct_back(None, None, None, 0, None) == -1
    assert libmvct.mvct_tv_grad(None, None, 1e-6, None, None, None) == -1
    assert libmvct.mvct_recon(None, None, None, 0.0, 1, None, None, None, None) == -1
    libmvct.mvct_plan_destroy(None)


@pytest.mark.parametrize("eps", [0.0, -1e-6, 1e-50, 1e-40, float("inf"), float("nan"), 1e300])
def test_tv_eps_that_is_not_a_normal_float_is_rejected(libmvct, eps):
    """eps enters every pixel term in FP32: a value that rounds to 0 or to a
    subnormal float (or overflows) would give 0 * rsqrt(0) = NaN gradients on
    flat regions, so it is refused before any CUDA call (the dummy pointers are
    never touched)."""
    bogus = ctypes.c_void_p(0x1000)
    assert libmvct.mvct_tv_grad_noalloc(bogus, 8, eps, bogus, None, None) == -1
    assert b"normal float" in libmvct.mvct_last_error()


def test_smallest_normal_float_eps_passes_the_check(libmvct):
    """FLT_MIN itself is accepted by the eps check: the call gets past it and fails
    only later, for want of a device, with another message."""
    bogus = ctypes.c_void_p(0x1000)
    libmvct.mvct_tv_grad_noalloc(bogus, 8, 1.1754944e-38, bogus, None, None)
    assert b"normal float" not in libmvct.mvct_last_error()
