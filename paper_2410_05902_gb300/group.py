"""Batched runs: many independent clustering runs stepped as one CUDA graph,
with per-run kernel variants picked by measurement.

``Group(runs)`` wraps kkm_group_*: one ``step()`` advances every run by one
iteration, as one launch per step phase over all runs (and one per Gram pass
and class of runs that share a kernel template); from the second step on the
step is replayed as one CUDA graph. ``autotune`` picks, for one run shape,
the fastest of the candidate variants (precision form and distance-pass
tile width) by timing graph-replayed steps with CUDA events. Every default
candidate meets a 1e-4 bound on the objective's relative error: FP32 and
split-BF16 products at FP32 level, TF32 products (10-bit mantissa) at
4e-5 or below on the measured workloads (d from 16 to 784); plain BF16 is
left out, as it reaches 2e-4 at d = 16.
"""
from __future__ import annotations

import ctypes
from ctypes import c_void_p

from .kkm import KKM, KKMError, load

# (precision, distance-pass tile width); 0 = the form's default
DEFAULT_CANDIDATES = (("fp32", 0), ("bf16x3", 64), ("bf16x3", 128), ("bf16x3", 256), ("tf32", 128),
                      ("tf32", 256))


class Group:
    """A set of runs stepped together (the runs stay owned by the caller)."""

    def __init__(self, runs: list[KKM], stream=None):
        import torch
        self.runs = list(runs)
        lib = load()
        arr = (c_void_p * len(self.runs))(*[r.ctx.value if isinstance(r.ctx, c_void_p) else r.ctx
                                            for r in self.runs])
        self._g = c_void_p()
        st = lib.kkm_group_create(ctypes.byref(self._g), arr, len(self.runs),
                                  None if stream is None else stream.cuda_stream)
        if st != 0:
            raise KKMError(st, lib.kkm_group_last_error(None).decode())
        self.stream = stream

    def _check(self, st):
        if st != 0:
            lib = load()
            raise KKMError(st, lib.kkm_group_last_error(self._g).decode())

    def step(self):
        self._check(load().kkm_group_step(self._g))

    def sync(self):
        self._check(load().kkm_group_sync(self._g))

    def set_chains(self, chains: int):
        """Before the first step: step the runs as `chains` concurrent chains of
        per-phase launches, or (chains = 0) each run on a graph branch of its own."""
        self._check(load().kkm_group_set_chains(self._g, int(chains)))

    def launches(self, reset: bool = False) -> tuple[int, int]:
        """(kernels the group's steps launched, kernels per group step)."""
        la, per = ctypes.c_int64(), ctypes.c_int32()
        self._check(load().kkm_group_launches(self._g, ctypes.byref(la), ctypes.byref(per), int(reset)))
        return la.value, per.value

    def close(self):
        if getattr(self, "_g", None) is not None and self._g.value:
            load().kkm_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def time_steps(run: KKM, steps: int) -> float:
    """Milliseconds per graph-replayed step of one run (CUDA events on its stream)."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    run.sync()
    ev0.record(run.stream)
    for _ in range(steps):
        run.step()
    ev1.record(run.stream)
    run.sync()
    return ev0.elapsed_time(ev1) / steps


def autotune(X, k: int, b: int, kernel: str, param: float, tau: int, init_idx, candidates=DEFAULT_CANDIDATES,
             warm: int = 20, iters: int = 10, seed: int = 0):
    """(best (precision, tile), {candidate: ms per step}) for one run shape."""
    times = {}
    for prec, tile in candidates:
        run = KKM(X, k, b, kernel=kernel, param=param, tau=tau, precision=prec, dist_tile=tile,
                  init_idx=init_idx, seed=seed)
        run.graph(True)
        for _ in range(warm):
            run.step()
        times[(prec, tile)] = time_steps(run, iters)
        run.close()
    best = min(times, key=times.get)
    return best, times
