"""Thin Python binding of libkkm (include/kkm.h), argument marshalling only.

The module-level functions carry the C names (``kkm_init``, ``kkm_step``, ...)
and take raw integer pointers. ``KKM`` wraps one context for callers that
hold PyTorch CUDA tensors: it passes ``data_ptr()`` values and the current
CUDA stream, and every step of the method runs in the library's kernels.
There is no CPU fallback. If libkkm.so has not been built, loading fails with
an error.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_uint8, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkkm.so")

KKM_OK, KKM_EINVAL, KKM_ENOMEM, KKM_ECUDA, KKM_ETIMEOUT, KKM_ESTATE, KKM_ENOTSUP = range(7)
KKM_GAUSSIAN, KKM_LAPLACIAN, KKM_LINEAR, KKM_POLY = range(4)
KKM_LR_BETA, KKM_LR_CONST, KKM_LR_SKLEARN = 0, 1, 2
LEARNING_RATES = {"beta": KKM_LR_BETA, "const": KKM_LR_CONST, "sklearn": KKM_LR_SKLEARN}
KKM_ALGO_WINDOWS, KKM_ALGO_TABLE = 0, 1
ALGOS = {"windows": KKM_ALGO_WINDOWS, "table": KKM_ALGO_TABLE}
KKM_PREC_FP32, KKM_PREC_BF16, KKM_PREC_BF16X3, KKM_PREC_TF32 = 0, 1, 2, 3
PRECISIONS = {"fp32": KKM_PREC_FP32, "bf16": KKM_PREC_BF16, "bf16x3": KKM_PREC_BF16X3, "tf32": KKM_PREC_TF32}
KERNELS = {"gaussian": KKM_GAUSSIAN, "laplacian": KKM_LAPLACIAN, "linear": KKM_LINEAR,
           "poly": KKM_POLY}
_STATUS = {0: "KKM_OK", 1: "KKM_EINVAL", 2: "KKM_ENOMEM", 3: "KKM_ECUDA", 4: "KKM_ETIMEOUT",
           5: "KKM_ESTATE", 6: "KKM_ENOTSUP"}


class kkm_kernel(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("param", c_double), ("coef0", c_double), ("degree", c_int32)]


class kkm_config(ctypes.Structure):
    _fields_ = [("tau", c_int32), ("lr", c_int32), ("eta", c_double), ("precision", c_int32),
                ("max_iters", c_int32), ("seed", c_uint64), ("dist_tile", c_int32), ("algo", c_int32)]


class KKMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None
_P = c_void_p


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libkkm.so (built by paper_2410_05902_gb300.build) and declare its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libkkm.so is not built ({p}); run paper_2410_05902_gb300.build.build()")
    lib = ctypes.CDLL(p)
    sigs = {
        "kkm_version": ([], c_int32),
        "kkm_last_error": ([_P], ctypes.c_char_p),
        "kkm_init": ([POINTER(_P), _P, c_int64, c_int32, c_int64, c_int32, POINTER(kkm_kernel),
                      c_int32, POINTER(kkm_config), POINTER(c_int64), _P], c_int32),
        "kkm_step": ([_P, _P, _P, _P, _P, _P], c_int32),
        "kkm_step_host": ([_P, _P, _P, _P], c_int32),
        "kkm_steps_host": ([_P, c_int64, _P, _P, _P], c_int32),
        "kkm_assign": ([_P, _P, c_int64, c_int64, _P, _P, _P], c_int32),
        "kkm_objective": ([_P, _P, c_int64, c_int64, POINTER(c_double)], c_int32),
        "kkm_objective_fwd": ([_P, _P, c_int64, c_int64, _P, c_double, _P, _P], c_int32),
        "kkm_objective_bwd": ([_P, _P, c_int64, c_int64, _P, c_double, _P, _P, c_int64, _P], c_int32),
        "kkm_sync": ([_P], c_int32),
        "kkm_flush": ([_P], c_int32),
        "kkm_steps": ([_P, c_int64], c_int32),
        "kkm_get_state_sizes": ([_P, POINTER(c_int64), POINTER(c_int64)], c_int32),
        "kkm_get_state": ([_P, POINTER(c_int64), _P, _P, _P, _P, _P, _P, _P, _P], c_int32),
        "kkm_set_state": ([_P, c_int64, _P, _P, _P, _P, _P, _P, _P, _P], c_int32),
        "kkm_stats": ([_P, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64), c_int32], c_int32),
        "kkm_timing_enable": ([_P, c_int32], c_int32),
        "kkm_graph_enable": ([_P, c_int32], c_int32),
        "kkm_timing_read": ([_P, POINTER(c_int64), POINTER(c_double), c_int32], c_int32),
        "kkm_launches": ([_P, POINTER(c_int64), c_int32], c_int32),
        "kkm_distances_noalloc": ([_P, c_int64, c_int64, c_int32, _P, c_int64, c_int64, _P, _P, _P,
                                   c_int32, POINTER(kkm_kernel), _P, _P, _P], c_int32),
        "kkm_noalloc_last_error": ([], ctypes.c_char_p),
        "kkm_form_supported": ([c_int32, c_int32, c_int32], c_int32),
        "kkm_probe_unit_rate": ([c_int32, c_int64, POINTER(c_double), POINTER(c_double), _P], c_int32),
        "kkm_probe_bounded_wait": ([c_int64, c_int32, _P], c_int32),
        "kkm_destroy": ([_P], c_int32),
        "kkm_step_eval": ([_P, _P, _P, _P], c_int32),
        "kkm_kmeanspp": ([_P, c_int64, c_int32, c_int64, c_int32, POINTER(kkm_kernel), c_uint64, _P, _P], c_int32),
        "kkm_fit": ([_P, c_int64, c_double, POINTER(c_int64), POINTER(c_double)], c_int32),
        "kkm_get_cum_counts": ([_P, _P], c_int32),
        "kkm_set_cum_counts": ([_P, _P], c_int32),
        "kkm_group_create": ([POINTER(_P), _P, c_int32, _P], c_int32),
        "kkm_group_step": ([_P], c_int32),
        "kkm_group_launches": ([_P, POINTER(c_int64), POINTER(c_int32), c_int32], c_int32),
        "kkm_group_set_chains": ([_P, c_int32], c_int32),
        "kkm_group_sync": ([_P], c_int32),
        "kkm_group_last_error": ([_P], ctypes.c_char_p),
        "kkm_group_destroy": ([_P], c_int32),
        "kkm_lloyd_init": ([POINTER(_P), _P, c_int64, c_int32, c_int64, c_int32, POINTER(kkm_kernel), c_int32,
                            POINTER(c_int64), c_int64, _P], c_int32),
        "kkm_lloyd_iterate": ([_P, c_int32], c_int32),
        "kkm_lloyd_read": ([_P, POINTER(c_double), POINTER(c_int64), POINTER(c_int64)], c_int32),
        "kkm_lloyd_assignments": ([_P, _P, _P], c_int32),
        "kkm_lloyd_distances": ([_P, _P], c_int32),
        "kkm_lloyd_center_norms": ([_P, _P], c_int32),
        "kkm_lloyd_info": ([_P, POINTER(c_int64), POINTER(c_int32), POINTER(c_int64)], c_int32),
        "kkm_lloyd_destroy": ([_P], c_int32),
        "kkm_lloyd_last_error": ([_P], ctypes.c_char_p),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def _check(status: int, ctx) -> None:
    if status != KKM_OK:
        msg = load().kkm_last_error(ctx)
        raise KKMError(status, msg.decode() if msg else "")


def _np_ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(c_void_p)


# ------------------------------------------------------- C-named wrappers
def kkm_version() -> int:
    return load().kkm_version()


def kkm_init(X_ptr: int, n: int, d: int, ldx: int, k: int, kernel: kkm_kernel, b: int,
             cfg: kkm_config, init_idx: np.ndarray | None, stream: int):
    ctx = c_void_p()
    ii = None if init_idx is None else np.ascontiguousarray(init_idx, dtype=np.int64)
    st = load().kkm_init(ctypes.byref(ctx), X_ptr, n, d, ldx, k, ctypes.byref(kernel), b,
                         ctypes.byref(cfg), None if ii is None else ii.ctypes.data_as(POINTER(c_int64)),
                         stream)
    _check(st, None)
    return ctx


def kkm_step(ctx, batch_idx: int | None, forced_assign: int | None, assign_out: int | None,
             dist_out: int | None, batch_obj_out: int | None) -> None:
    _check(load().kkm_step(ctx, batch_idx, forced_assign, assign_out, dist_out, batch_obj_out), ctx)


def kkm_step_host(ctx, batch_idx: np.ndarray | None, assign_out: np.ndarray | None,
                  batch_obj_out: np.ndarray | None) -> None:
    _check(load().kkm_step_host(ctx, _np_ptr(batch_idx), _np_ptr(assign_out), _np_ptr(batch_obj_out)), ctx)


def kkm_steps_host(ctx, n: int, batch_idx: np.ndarray | None, assign_out: np.ndarray | None,
                   batch_obj_out: np.ndarray | None) -> None:
    _check(load().kkm_steps_host(ctx, int(n), _np_ptr(batch_idx), _np_ptr(assign_out), _np_ptr(batch_obj_out)),
           ctx)


def kkm_assign(ctx, Q: int, m: int, ldq: int, assign_out: int | None, mind_out: int | None,
               dist_out: int | None) -> None:
    _check(load().kkm_assign(ctx, Q, m, ldq, assign_out, mind_out, dist_out), ctx)


def kkm_objective(ctx, Q: int | None, m: int, ldq: int) -> float:
    out = c_double()
    _check(load().kkm_objective(ctx, Q, m, ldq, ctypes.byref(out)), ctx)
    return out.value


def kkm_objective_fwd(ctx, Q: int, m: int, ldq: int, assign: int, log_sigma: float, loss_out: int,
                      delta_out: int | None) -> None:
    _check(load().kkm_objective_fwd(ctx, Q, m, ldq, assign, float(log_sigma), loss_out, delta_out), ctx)


def kkm_objective_bwd(ctx, Q: int, m: int, ldq: int, assign: int, log_sigma: float, grad_loss: int,
                      grad_q: int, ldg: int, grad_log_sigma: int) -> None:
    _check(load().kkm_objective_bwd(ctx, Q, m, ldq, assign, float(log_sigma), grad_loss, grad_q, ldg,
                                    grad_log_sigma), ctx)


def kkm_kmeanspp(X_ptr: int, n: int, d: int, ldx: int, k: int, kernel: kkm_kernel, seed: int,
                 stream: int | None) -> np.ndarray:
    out = np.zeros(k, np.int64)
    _check(load().kkm_kmeanspp(X_ptr, n, d, ldx, k, ctypes.byref(kernel), int(seed) & ((1 << 64) - 1),
                               _np_ptr(out), stream), None)
    return out


def kmeanspp(X, k: int, kernel: str = "gaussian", param: float = 1.0, coef0: float = 0.0, degree: int = 2,
             seed: int = 0, stream=None) -> np.ndarray:
    """Kernel k-means++ seeding on the GPU: k data indices of the CUDA float32 tensor X."""
    import torch
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32 and X.dim() == 2
            and X.stride(1) == 1):
        raise TypeError("X must be a row-contiguous 2-D float32 CUDA tensor")
    st = stream if stream is not None else torch.cuda.current_stream(X.device)
    kern = kkm_kernel(KERNELS[kernel], float(param), float(coef0), int(degree))
    with torch.cuda.device(X.device):
        return kkm_kmeanspp(X.data_ptr(), X.shape[0], X.shape[1], X.stride(0), int(k), kern, seed, st.cuda_stream)


def kkm_sync(ctx) -> None:
    _check(load().kkm_sync(ctx), ctx)


def kkm_flush(ctx) -> None:
    _check(load().kkm_flush(ctx), ctx)


def kkm_steps(ctx, n: int) -> None:
    _check(load().kkm_steps(ctx, int(n)), ctx)


def kkm_stats(ctx, reset: bool = False) -> tuple[int, int, int]:
    a, b_, c = c_int64(), c_int64(), c_int64()
    _check(load().kkm_stats(ctx, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c), int(reset)), ctx)
    return a.value, b_.value, c.value


def kkm_timing_enable(ctx, enable) -> None:
    """enable: False/0 off, True/1 one launch per record, R > 1: R back-to-back launches."""
    _check(load().kkm_timing_enable(ctx, int(enable)), ctx)


def kkm_graph_enable(ctx, enable: bool) -> None:
    _check(load().kkm_graph_enable(ctx, int(enable)), ctx)


def kkm_timing_read(ctx, reset: bool = False) -> tuple[int, float]:
    n, ms = c_int64(), c_double()
    _check(load().kkm_timing_read(ctx, ctypes.byref(n), ctypes.byref(ms), int(reset)), ctx)
    return n.value, ms.value


def kkm_launches(ctx, reset: bool = False) -> int:
    n = c_int64()
    _check(load().kkm_launches(ctx, ctypes.byref(n), int(reset)), ctx)
    return n.value


def kkm_distances_noalloc(Q: int, m: int, ldq: int, d: int, Y: int, S: int, ldy: int, w: int,
                          seg_off: int, cnorm: int, k: int, kernel: kkm_kernel | None, dist_out: int | None,
                          assign_out: int | None, stream: int | None) -> None:
    """Distances and argmin against caller-held centers, with no allocation
    (kkm.h). m = 0 only loads the call's scratch and kernels on the current
    device; kernel may then be None."""
    lib = load()
    kp = ctypes.byref(kernel) if kernel is not None else None
    st = lib.kkm_distances_noalloc(Q, m, ldq, d, Y, S, ldy, w, seg_off, cnorm, k, kp,
                                   dist_out, assign_out, stream)
    if st != KKM_OK:
        raise KKMError(st, lib.kkm_noalloc_last_error().decode())


def _lcheck(status: int, run) -> None:
    if status != KKM_OK:
        msg = load().kkm_lloyd_last_error(run)
        raise KKMError(status, msg.decode() if msg else "")


def kkm_lloyd_init(X_ptr: int, n: int, d: int, ldx: int, k: int, kernel: kkm_kernel, precision: int,
                   init_idx, chunk_rows: int, stream: int | None):
    run = c_void_p()
    ii = np.ascontiguousarray(init_idx, dtype=np.int64)
    if ii.shape != (k,):
        raise ValueError("init_idx must hold k indices")
    st = load().kkm_lloyd_init(ctypes.byref(run), X_ptr, n, d, ldx, k, ctypes.byref(kernel), precision,
                               ii.ctypes.data_as(POINTER(c_int64)), chunk_rows, stream)
    _lcheck(st, None)
    return run


def kkm_lloyd_iterate(run, iters: int) -> None:
    _lcheck(load().kkm_lloyd_iterate(run, iters), run)


def kkm_lloyd_read(run) -> tuple[float, int, int]:
    o, ch, it = c_double(), c_int64(), c_int64()
    _lcheck(load().kkm_lloyd_read(run, ctypes.byref(o), ctypes.byref(ch), ctypes.byref(it)), run)
    return o.value, ch.value, it.value


def kkm_lloyd_assignments(run, assign_out: int | None, mind_out: int | None) -> None:
    _lcheck(load().kkm_lloyd_assignments(run, assign_out, mind_out), run)


def kkm_lloyd_distances(run, dist_out: int) -> None:
    _lcheck(load().kkm_lloyd_distances(run, dist_out), run)


def kkm_lloyd_center_norms(run, k: int) -> np.ndarray:
    out = np.zeros(k, np.float64)
    _lcheck(load().kkm_lloyd_center_norms(run, _np_ptr(out)), run)
    return out


def kkm_lloyd_info(run) -> tuple[int, int, int]:
    la, ch, rows = c_int64(), c_int32(), c_int64()
    _lcheck(load().kkm_lloyd_info(run, ctypes.byref(la), ctypes.byref(ch), ctypes.byref(rows)), run)
    return la.value, ch.value, rows.value


def kkm_lloyd_destroy(run) -> None:
    load().kkm_lloyd_destroy(run)


def kkm_probe_bounded_wait(limit_ns: int, arrive: bool, stream: int | None = None) -> int:
    """Status of one bounded mbarrier wait of the tcgen05 passes (KKM_ETIMEOUT when nothing arrives)."""
    return load().kkm_probe_bounded_wait(int(limit_ns), 1 if arrive else 0, stream)


def kkm_probe_unit_rate(op: int, iters: int, stream: int | None = None) -> tuple[float, float]:
    """(operations per SM per clock, operations per second) of one unit (see kkm.h)."""
    a, b_ = c_double(), c_double()
    st = load().kkm_probe_unit_rate(int(op), int(iters), ctypes.byref(a), ctypes.byref(b_), stream)
    if st != KKM_OK:
        raise KKMError(st, "kkm_probe_unit_rate failed")
    return a.value, b_.value


def unit_rates() -> dict:
    """MUFU ex2.approx, scalar FP32 FMA and packed f32x2 FMA rates of the current device."""
    ex2, ex2_s = kkm_probe_unit_rate(0, 65536)
    fma, fma_s = kkm_probe_unit_rate(1, 262144)
    fma2, fma2_s = kkm_probe_unit_rate(2, 131072)
    return {"ex2_per_clk_sm": ex2, "ex2_per_s": ex2_s, "ffma_per_clk_sm": fma, "ffma_per_s": fma_s,
            "ffma2_fp32_per_clk_sm": fma2, "ffma2_fp32_per_s": fma2_s}


def kkm_get_state(ctx, k: int) -> dict:
    rows, blocks = c_int64(), c_int64()
    _check(load().kkm_get_state_sizes(ctx, ctypes.byref(rows), ctypes.byref(blocks)), ctx)
    it = c_int64()
    out = {
        "rows_per_center": np.zeros(k, np.int32), "row_idx": np.zeros(rows.value, np.int64),
        "row_w": np.zeros(rows.value, np.float64), "blocks_per_center": np.zeros(k, np.int32),
        "block_iter": np.zeros(blocks.value, np.int64), "block_count": np.zeros(blocks.value, np.int32),
        "c1_kept": np.zeros(k, np.uint8), "cnorm": np.zeros(k, np.float64),
    }
    _check(load().kkm_get_state(ctx, ctypes.byref(it), *[_np_ptr(out[key]) for key in (
        "rows_per_center", "row_idx", "row_w", "blocks_per_center", "block_iter", "block_count",
        "c1_kept", "cnorm")]), ctx)
    out["iteration"] = it.value
    out["cum_counts"] = np.zeros(k, np.int64)
    _check(load().kkm_get_cum_counts(ctx, _np_ptr(out["cum_counts"])), ctx)
    return out


def kkm_set_state(ctx, state: dict) -> None:
    arrs = [np.ascontiguousarray(state[key], dtype=dt) for key, dt in (
        ("rows_per_center", np.int32), ("row_idx", np.int64), ("row_w", np.float64),
        ("blocks_per_center", np.int32), ("block_iter", np.int64), ("block_count", np.int32),
        ("c1_kept", np.uint8), ("cnorm", np.float64))]
    _check(load().kkm_set_state(ctx, int(state["iteration"]), *[_np_ptr(a) for a in arrs]), ctx)
    if "cum_counts" in state:
        cc = np.ascontiguousarray(state["cum_counts"], dtype=np.int64)
        _check(load().kkm_set_cum_counts(ctx, _np_ptr(cc)), ctx)


def kkm_step_eval(ctx, batch_idx: int | None, obj_before: int, obj_after: int) -> None:
    _check(load().kkm_step_eval(ctx, batch_idx, obj_before, obj_after), ctx)


def kkm_fit(ctx, max_iters: int, eps: float) -> tuple[int, float]:
    done, imp = c_int64(), c_double()
    _check(load().kkm_fit(ctx, int(max_iters), float(eps), ctypes.byref(done), ctypes.byref(imp)), ctx)
    return done.value, imp.value


def kkm_destroy(ctx) -> None:
    _check(load().kkm_destroy(ctx), None)


# ------------------------------------------------------------ torch wrapper
class KKM:
    """One clustering run on the current CUDA device (tensors in, tensors out).

    X is a CUDA float32 tensor (n x d, row stride >= d). It is kept alive
    here because the library reads batches and support rows from it. kernel is
    one of "gaussian", "laplacian", "linear" or "poly". param is kappa for the
    Gaussian kernel and sigma for the Laplacian kernel.
    """

    def __init__(self, X, k: int, b: int, kernel: str = "gaussian", param: float = 1.0,
                 coef0: float = 0.0, degree: int = 2, tau: int = 200, lr: str = "beta",
                 eta: float = 0.0, precision: str = "fp32", seed: int = 0, init_idx=None,
                 max_iters: int = 0, stream=None, dist_tile: int = 0, algo: str = "windows"):
        import torch
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
            raise TypeError("X must be a 2-D float32 CUDA tensor")
        if X.stride(1) != 1:
            raise ValueError("X rows must be contiguous")
        self._torch = torch
        self.X = X
        self.n, self.d = X.shape
        self.k, self.b = int(k), int(b)
        self.stream = stream if stream is not None else torch.cuda.current_stream(X.device)
        kern = kkm_kernel(KERNELS[kernel], float(param), float(coef0), int(degree))
        cfg = kkm_config(int(tau), LEARNING_RATES[lr], float(eta),
                         PRECISIONS[precision], int(max_iters), int(seed) & ((1 << 64) - 1), int(dist_tile),
                         ALGOS[algo])
        if isinstance(init_idx, str):
            if init_idx != "kmeans++":
                raise ValueError("init_idx: indices, None, or 'kmeans++'")
            init_idx = kmeanspp(X, self.k, kernel, param, coef0, degree, seed=seed, stream=self.stream)
        with torch.cuda.device(X.device):
            self.ctx = kkm_init(X.data_ptr(), self.n, self.d, X.stride(0), self.k, kern, self.b, cfg,
                                None if init_idx is None else np.asarray(init_idx), self.stream.cuda_stream)

    @staticmethod
    def _ptr(t):
        return None if t is None else t.data_ptr()

    def step(self, batch_idx=None, forced_assign=None, assign_out=None, dist_out=None, obj_out=None):
        """One iteration. Optional outputs are CUDA tensors the caller allocated."""
        kkm_step(self.ctx, self._ptr(batch_idx), self._ptr(forced_assign), self._ptr(assign_out),
                 self._ptr(dist_out), self._ptr(obj_out))

    def steps(self, n: int):
        """n iterations with the built-in sampler, no outputs (16 per graph replay when graphs are on)."""
        kkm_steps(self.ctx, n)

    def step_host(self, batch_idx: np.ndarray | None = None):
        """One iteration with host buffers; returns (assignments, f_B) as numpy / float."""
        bi = None if batch_idx is None else np.ascontiguousarray(batch_idx, dtype=np.int32)
        a = np.zeros(self.b, np.int32)
        o = np.zeros(1, np.float64)
        kkm_step_host(self.ctx, bi, a, o)
        return a, float(o[0])

    def steps_host(self, batch_idx: np.ndarray | None = None, n: int | None = None):
        """n iterations with host buffers (batch_idx: n x b indices, or None and n
        for the built-in sampler); returns (assignments n x b, f_B per step)."""
        if batch_idx is None:
            if n is None:
                raise ValueError("give batch_idx or n")
            bi = None
        else:
            bi = np.ascontiguousarray(batch_idx, dtype=np.int32).reshape(-1, self.b)
            n = bi.shape[0]
        a = np.zeros((n, self.b), np.int32)
        o = np.zeros(n, np.float64)
        kkm_steps_host(self.ctx, n, bi, a, o)
        return a, o

    def assign(self, Q, want_dist: bool = False):
        torch = self._torch
        m = Q.shape[0]
        a = torch.empty(m, dtype=torch.int32, device=Q.device)
        md = torch.empty(m, dtype=torch.float32, device=Q.device)
        dist = torch.empty((m, self.k), dtype=torch.float32, device=Q.device) if want_dist else None
        kkm_assign(self.ctx, Q.data_ptr(), m, Q.stride(0), a.data_ptr(), md.data_ptr(), self._ptr(dist))
        return a, md, dist

    def objective(self, Q=None) -> float:
        if Q is None:
            return kkm_objective(self.ctx, None, 0, 0)
        return kkm_objective(self.ctx, Q.data_ptr(), Q.shape[0], Q.stride(0))

    def objective_fwd(self, Q, assign, log_sigma: float, want_delta: bool = False):
        """Batch objective at fixed assignments (device scalar) and optionally Delta per row."""
        torch = self._torch
        loss = torch.empty(1, dtype=torch.float64, device=Q.device)
        delta = torch.empty(Q.shape[0], dtype=torch.float32, device=Q.device) if want_delta else None
        kkm_objective_fwd(self.ctx, Q.data_ptr(), Q.shape[0], Q.stride(0), assign.data_ptr(), log_sigma,
                          loss.data_ptr(), self._ptr(delta))
        return loss, delta

    def objective_bwd(self, Q, assign, log_sigma: float, grad_loss):
        """(grad Q, grad log_sigma) of grad_loss * objective (grad_loss: 1-element float64 CUDA tensor)."""
        torch = self._torch
        gq = torch.empty(Q.shape, dtype=torch.float32, device=Q.device)
        gs = torch.empty(1, dtype=torch.float64, device=Q.device)
        kkm_objective_bwd(self.ctx, Q.data_ptr(), Q.shape[0], Q.stride(0), assign.data_ptr(), log_sigma,
                          grad_loss.data_ptr(), gq.data_ptr(), gq.stride(0), gs.data_ptr())
        return gq, gs

    def step_eval(self, batch_idx=None):
        """One iteration plus f_B before and after the update on the same batch (device scalars)."""
        torch = self._torch
        before = torch.empty(1, dtype=torch.float64, device=self.X.device)
        after = torch.empty(1, dtype=torch.float64, device=self.X.device)
        kkm_step_eval(self.ctx, self._ptr(batch_idx), before.data_ptr(), after.data_ptr())
        return before, after

    def fit(self, max_iters: int, eps: float):
        """Iterate until the batch improvement drops below eps (Sec. 5); (iterations, last improvement)."""
        return kkm_fit(self.ctx, max_iters, eps)

    def sync(self):
        kkm_sync(self.ctx)

    def flush(self):
        """Queue the weight update the last step left pending (asynchronous)."""
        kkm_flush(self.ctx)

    def get_state(self) -> dict:
        return kkm_get_state(self.ctx, self.k)

    def set_state(self, state: dict):
        kkm_set_state(self.ctx, state)

    def stats(self, reset: bool = False):
        return kkm_stats(self.ctx, reset)

    def timing(self, enable):
        kkm_timing_enable(self.ctx, enable)

    def graph(self, enable: bool):
        kkm_graph_enable(self.ctx, enable)

    def timing_read(self, reset: bool = False):
        return kkm_timing_read(self.ctx, reset)

    def launches(self, reset: bool = False) -> int:
        return kkm_launches(self.ctx, reset)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            kkm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lloyd:
    """Full-batch kernel k-means (kernel Lloyd) through kkm_lloyd_*: every
    iteration assigns all points, then moves every center with points to the
    mean of its points in feature space (the baseline of Sec. 6)."""

    def __init__(self, X, k: int, init_idx, kernel: str = "gaussian", param: float = 1.0, coef0: float = 0.0,
                 degree: int = 2, precision: str = "fp32", chunk_rows: int = 0, stream=None):
        import torch
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
            raise TypeError("X must be a 2-D float32 CUDA tensor")
        if X.stride(1) != 1:
            raise ValueError("X rows must be contiguous")
        self._torch = torch
        self.n, self.d = X.shape
        self.k = int(k)
        self.device = X.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(X.device)
        kern = kkm_kernel(KERNELS[kernel], float(param), float(coef0), int(degree))
        with torch.cuda.device(X.device):
            self.run = kkm_lloyd_init(X.data_ptr(), self.n, self.d, X.stride(0), self.k, kern,
                                      PRECISIONS[precision], init_idx, int(chunk_rows), self.stream.cuda_stream)

    def iterate(self, iters: int = 1) -> None:
        """Queue `iters` iterations (asynchronous)."""
        kkm_lloyd_iterate(self.run, iters)

    def read(self) -> tuple[float, int, int]:
        """(f_X at the current centers, assignments changed by the last assignment, iterations run)."""
        return kkm_lloyd_read(self.run)

    def assignments(self):
        """(assignments int32 (n,), min_j Delta float32 (n,)) as CUDA tensors."""
        torch = self._torch
        a = torch.empty(self.n, dtype=torch.int32, device=self.device)
        md = torch.empty(self.n, dtype=torch.float32, device=self.device)
        kkm_lloyd_assignments(self.run, a.data_ptr(), md.data_ptr())
        return a, md

    def distances(self):
        """Delta(x, C_j) as an (n, k) float32 CUDA tensor."""
        out = self._torch.empty((self.n, self.k), dtype=self._torch.float32, device=self.device)
        kkm_lloyd_distances(self.run, out.data_ptr())
        return out

    def center_norms(self) -> np.ndarray:
        return kkm_lloyd_center_norms(self.run, self.k)

    def info(self) -> tuple[int, int, int]:
        """(kernels launched, Gram-pass chunks per iteration, rows per chunk)."""
        return kkm_lloyd_info(self.run)

    def close(self) -> None:
        if self.run:
            kkm_lloyd_destroy(self.run)
            self.run = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
