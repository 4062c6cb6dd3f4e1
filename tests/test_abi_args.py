"""Host-side argument checks of the C ABI: calls with invalid arguments return ES_ERR_ARG
before any CUDA call, so they run without a GPU."""
import ctypes

import pytest

from paper_2407_05568_gb300 import es
from paper_2407_05568_gb300 import workloads as wl


@pytest.fixture(scope="module")
def L():
    from paper_2407_05568_gb300 import build
    build.build()
    return es.lib()


def _params(**over):
    p = es.make_params(wl.riemann_2d(16, seed=5))
    for k, v in over.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("field,value", [("dim", 3), ("n1", 4), ("n2", 0), ("precision", 7), ("tile", 6),
                                         ("tile", -1), ("cfl", 0.0), ("sign_tol", 0.5), ("kappa", 3),
                                         ("jacobi_sweeps", -1), ("R", 0.0), ("weno_eps", 0.0)])
def test_create_rejects_bad_params(L, field, value):
    h = ctypes.c_void_p()
    p = _params(**{field: value})
    assert L.es_create(ctypes.byref(h), ctypes.byref(p), None) == es.ES_ERR_ARG
    assert not h.value


def test_create_rejects_walls_in_the_mixed_form(L):
    p = es.make_params(wl.sine_2d(16), precision="mixed")
    p.bc[0] = es.ES_BC["reflect"]
    h = ctypes.c_void_p()
    assert L.es_create(ctypes.byref(h), ctypes.byref(p), None) == es.ES_ERR_ARG


def test_create_rejects_mixed_period_mismatch(L):
    w = wl.sine_2d(16)
    p = es.make_params(w, precision="mixed")
    p.period[0] = 0.9                       # the FP32 displacement is periodic only for period = n dxi
    h = ctypes.c_void_p()
    assert L.es_create(ctypes.byref(h), ctypes.byref(p), None) == es.ES_ERR_ARG


@pytest.mark.parametrize("B,Cin,Cout,H,W", [(1, 3, 32, 16, 16), (1, 32, 5, 16, 16), (0, 4, 32, 16, 16),
                                            (1, 4, 32, 0, 16), (1, 64, 32, 8, 8)])
def test_nn_shapes_rejected(L, B, Cin, Cout, H, W):
    dummy = ctypes.c_void_p(16)
    assert L.es_nn_workspace_bytes(B, Cin, Cout, H, W) == 0
    assert L.es_nn_conv_forward(dummy, dummy, dummy, ctypes.c_void_p(32), B, Cin, Cout, H, W, 0, dummy, 1 << 20,
                                None) == es.ES_ERR_ARG
    assert L.es_nn_conv_forward_bf16(dummy, dummy, dummy, ctypes.c_void_p(32), B, Cin, Cout, H, W, 0,
                                     None) == es.ES_ERR_ARG


def test_nn_null_and_aliasing_rejected(L):
    a = ctypes.c_void_p(16)
    assert L.es_nn_conv_forward(None, a, a, a, 1, 4, 32, 16, 16, 0, a, 1 << 20, None) == es.ES_ERR_ARG
    assert L.es_nn_conv_forward(a, a, a, a, 1, 4, 32, 16, 16, 0, ctypes.c_void_p(64), 1 << 20, None) == es.ES_ERR_ARG
    assert L.es_nn_conv_forward(ctypes.c_void_p(8), a, a, ctypes.c_void_p(24), 1, 4, 32, 16, 16, 0, a, 4,
                                None) == es.ES_ERR_ARG                 # workspace too small
    assert L.es_nn_mse(a, a, a, a, 0, None) == es.ES_ERR_ARG
    assert L.es_nn_adam(a, None, a, a, a, 10, ctypes.c_float(1e-3), ctypes.c_float(0.9), ctypes.c_float(0.999),
                        ctypes.c_float(1e-8), 0, None) == es.ES_ERR_ARG  # step counts from 1


def test_batch_rejects_bad_lengths_and_params(L):
    p = es.batch_params(wl.UNITS_A)
    lengths = (ctypes.c_int * 3)(200, 7, 300)
    h = ctypes.c_void_p()
    assert L.es_batch_create(ctypes.byref(h), ctypes.byref(p), 3, lengths, None) == es.ES_ERR_ARG
    ok = (ctypes.c_int * 2)(200, 300)
    q = es.batch_params(wl.UNITS_A)
    q.dim = 2
    assert L.es_batch_create(ctypes.byref(h), ctypes.byref(q), 2, ok, None) == es.ES_ERR_ARG
    q = es.batch_params(wl.UNITS_A)
    q.precision = es.ES_PREC["fp64"]
    assert L.es_batch_create(ctypes.byref(h), ctypes.byref(q), 2, ok, None) == es.ES_ERR_ARG
    assert L.es_batch_create(ctypes.byref(h), ctypes.byref(p), 0, ok, None) == es.ES_ERR_ARG


def test_null_context_rejected(L):
    assert L.es_check(None) == es.ES_ERR_ARG
    assert L.es_steps(None, None, None, None, 1, ctypes.c_double(1.0)) == es.ES_ERR_ARG
    assert L.es_launch_count(None) == 0
    assert L.es_batch_check(None) == es.ES_ERR_ARG
