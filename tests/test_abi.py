"""C-ABI checks that need no GPU.

libkkm.so builds with nvcc (it cross-compiles without a GPU) and loads. It
exports every function include/kkm.h declares, and it rejects invalid
arguments on the host before any CUDA call. No compute call is made here.
"""
import ctypes

import numpy as np
import os
import re
import shutil

import pytest

from paper_2410_05902_gb300 import build as kbuild
from paper_2410_05902_gb300 import kkm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kkm.h")


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    path = kbuild.build()
    return kkm.load(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:kkm_status|int32_t|const char\*)\s+(kkm_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("kkm_init", "kkm_step", "kkm_assign", "kkm_objective", "kkm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} declared in kkm.h but not exported"


def test_version(lib):
    assert lib.kkm_version() == 2


def _init(lib, **over):
    args = dict(X=ctypes.c_void_p(0x1000), n=100, d=8, ldx=8, k=4, b=32)
    args.update(over)
    kern = over.pop("kernel", kkm.kkm_kernel(kkm.KKM_GAUSSIAN, 2.0, 0.0, 2))
    cfg = over.pop("cfg", kkm.kkm_config(50, kkm.KKM_LR_BETA, 0.0, kkm.KKM_PREC_FP32, 0, 7))
    ctx = ctypes.c_void_p()
    st = lib.kkm_init(ctypes.byref(ctx), args["X"], args["n"], args["d"], args["ldx"], args["k"],
                      ctypes.byref(args.get("kernel", kern)), args["b"],
                      ctypes.byref(args.get("cfg", cfg)), None, None)
    return st, ctx


@pytest.mark.parametrize("over,needle", [
    (dict(n=0), "n must be"),
    (dict(d=0), "d must be"),
    (dict(ldx=4), "ldx"),
    (dict(k=0), "k must be"),
    (dict(k=200), "k must be"),
    (dict(b=0), "b must be"),
    (dict(X=None), "required"),
    (dict(kernel=kkm.kkm_kernel(kkm.KKM_GAUSSIAN, -1.0, 0.0, 2)), "kernel param"),
    (dict(kernel=kkm.kkm_kernel(9, 1.0, 0.0, 2)), "unknown kernel"),
    (dict(kernel=kkm.kkm_kernel(kkm.KKM_POLY, 1.0, 0.0, 0)), "degree"),
    (dict(cfg=kkm.kkm_config(50, 7, 0.0, 0, 0, 0)), "learning rate"),
    (dict(cfg=kkm.kkm_config(50, kkm.KKM_LR_CONST, 1.5, 0, 0, 0)), "eta"),
    (dict(cfg=kkm.kkm_config(50, 0, 0.0, 9, 0, 0)), "precision"),
    (dict(cfg=kkm.kkm_config(0, 0, 0.0, 0, 0, 0)), "max_iters"),
    (dict(cfg=kkm.kkm_config(50, 0, 0.0, 0, 0, 0, 96, 0)), "dist_tile"),
    (dict(cfg=kkm.kkm_config(50, 0, 0.0, 0, 0, 0, 0, 7)), "algo"),
    (dict(cfg=kkm.kkm_config(50, 0, 0.0, 0, 0, 0, 0, 1)), "tau"),
])
def test_init_rejects_invalid_arguments_on_host(lib, over, needle):
    st, ctx = _init(lib, **over)
    assert st == kkm.KKM_EINVAL
    assert not ctx.value
    assert needle in lib.kkm_last_error(None).decode()


def test_null_context_calls(lib):
    assert lib.kkm_destroy(None) == kkm.KKM_OK
    assert lib.kkm_step(None, None, None, None, None, None) == kkm.KKM_EINVAL
    assert lib.kkm_sync(None) == kkm.KKM_EINVAL
    assert lib.kkm_flush(None) == kkm.KKM_EINVAL
    assert lib.kkm_steps(None, 5) == kkm.KKM_EINVAL
    assert lib.kkm_steps_host(None, 5, None, None, None) == kkm.KKM_EINVAL
    out = ctypes.c_double()
    assert lib.kkm_objective(None, None, 0, 0, ctypes.byref(out)) == kkm.KKM_EINVAL


def test_group_create_validates_on_host(lib):
    g = ctypes.c_void_p()
    assert lib.kkm_group_create(None, None, 1, None) == kkm.KKM_EINVAL
    assert lib.kkm_group_create(ctypes.byref(g), None, 0, None) == kkm.KKM_EINVAL
    assert not g.value
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.kkm_group_create(ctypes.byref(g), arr, 1, None) == kkm.KKM_EINVAL
    assert b"null run" in lib.kkm_group_last_error(None)
    assert lib.kkm_group_step(None) == kkm.KKM_EINVAL
    assert lib.kkm_group_destroy(None) == kkm.KKM_OK


def test_kmeanspp_validates_on_host(lib):
    out = np.zeros(4, np.int64)
    kern = kkm.kkm_kernel(kkm.KKM_GAUSSIAN, 1.0, 0.0, 2)
    ptr = out.ctypes.data_as(ctypes.c_void_p)
    assert lib.kkm_kmeanspp(None, 10, 3, 3, 4, ctypes.byref(kern), 0, ptr, None) == kkm.KKM_EINVAL
    assert lib.kkm_kmeanspp(ctypes.c_void_p(16), 3, 3, 3, 4, ctypes.byref(kern), 0, ptr, None) == kkm.KKM_EINVAL
    assert b"k must be" in lib.kkm_last_error(None)
    bad = kkm.kkm_kernel(kkm.KKM_GAUSSIAN, -1.0, 0.0, 2)
    assert lib.kkm_kmeanspp(ctypes.c_void_p(16), 10, 3, 3, 4, ctypes.byref(bad), 0, ptr, None) == kkm.KKM_EINVAL


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        kkm.load(str(tmp_path / "missing.so"))


def test_tensor_core_forms_refuse_other_devices(lib):
    """The BF16, split-BF16 and TF32 forms run only on the tcgen05 passes built
    for sm_103a: any other device gets KKM_ENOTSUP, never a CUDA-core stand-in."""
    for prec in (kkm.KKM_PREC_BF16, kkm.KKM_PREC_BF16X3, kkm.KKM_PREC_TF32):
        assert lib.kkm_form_supported(prec, 10, 3) == kkm.KKM_OK
        for cc in ((10, 0), (9, 0), (12, 0), (8, 9), (10, 1)):
            assert lib.kkm_form_supported(prec, *cc) == kkm.KKM_ENOTSUP
    for cc in ((10, 3), (9, 0), (8, 0)):
        assert lib.kkm_form_supported(kkm.KKM_PREC_FP32, *cc) == kkm.KKM_OK
    assert lib.kkm_form_supported(7, 10, 3) == kkm.KKM_EINVAL
    assert lib.kkm_form_supported(-1, 10, 3) == kkm.KKM_EINVAL


def test_probe_rejects_bad_arguments(lib):
    a, b = ctypes.c_double(), ctypes.c_double()
    assert lib.kkm_probe_unit_rate(3, 10, ctypes.byref(a), ctypes.byref(b), None) == kkm.KKM_EINVAL
    assert lib.kkm_probe_unit_rate(-1, 10, ctypes.byref(a), ctypes.byref(b), None) == kkm.KKM_EINVAL
    assert lib.kkm_probe_unit_rate(0, 0, ctypes.byref(a), ctypes.byref(b), None) == kkm.KKM_EINVAL
    assert lib.kkm_probe_unit_rate(0, 1 << 25, ctypes.byref(a), ctypes.byref(b), None) == kkm.KKM_EINVAL
    assert lib.kkm_probe_unit_rate(0, 10, None, ctypes.byref(b), None) == kkm.KKM_EINVAL


def _lloyd_init(lib, **over):
    args = dict(X=ctypes.c_void_p(0x1000), n=100, d=8, ldx=8, k=4, precision=kkm.KKM_PREC_FP32, chunk_rows=0,
                kernel=kkm.kkm_kernel(kkm.KKM_GAUSSIAN, 2.0, 0.0, 2), init=np.arange(4, dtype=np.int64))
    args.update(over)
    run = ctypes.c_void_p()
    init = args["init"]
    ip = None if init is None else init.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    st = lib.kkm_lloyd_init(ctypes.byref(run), args["X"], args["n"], args["d"], args["ldx"], args["k"],
                            ctypes.byref(args["kernel"]), args["precision"], ip, args["chunk_rows"], None)
    return st, run


@pytest.mark.parametrize("over,needle", [
    (dict(n=0), "n must be"),
    (dict(d=0), "d must be"),
    (dict(ldx=4), "ldx"),
    (dict(k=0), "k must be"),
    (dict(k=200), "k must be"),
    (dict(X=None), "required"),
    (dict(init=None), "required"),
    (dict(init=np.array([0, 1, 2, 100], np.int64)), "init_idx"),
    (dict(init=np.array([0, 1, -1, 3], np.int64)), "init_idx"),
    (dict(chunk_rows=100), "chunk_rows"),
    (dict(chunk_rows=-128), "chunk_rows"),
    (dict(precision=9), "precision"),
    (dict(kernel=kkm.kkm_kernel(kkm.KKM_LAPLACIAN, 0.0, 0.0, 2)), "kernel param"),
    (dict(kernel=kkm.kkm_kernel(kkm.KKM_POLY, 1.0, 0.0, 9)), "degree"),
])
def test_lloyd_init_rejects_bad_arguments(lib, over, needle):
    st, run = _lloyd_init(lib, **over)
    assert st == kkm.KKM_EINVAL
    assert not run.value
    assert needle in lib.kkm_lloyd_last_error(None).decode()


def test_lloyd_calls_reject_a_null_handle(lib):
    assert lib.kkm_lloyd_iterate(None, 1) == kkm.KKM_EINVAL
    assert lib.kkm_lloyd_read(None, None, None, None) == kkm.KKM_EINVAL
    assert lib.kkm_lloyd_distances(None, None) == kkm.KKM_EINVAL
    assert lib.kkm_lloyd_destroy(None) == kkm.KKM_OK


@pytest.mark.parametrize("limit,arrive", [(10, 0), (6_000_000_000, 0), (1_000_000, 2)])
def test_bounded_wait_probe_rejects_bad_arguments(lib, limit, arrive):
    assert lib.kkm_probe_bounded_wait(limit, arrive, None) == kkm.KKM_EINVAL
