"""Run groups (kkm_group_*): a group step is exactly one step of every run.

Runs of different shapes and precision forms stepped through one group must
end in the same state, bit for bit, as identical runs stepped on their own
(the same kernels run; only the launch structure differs). Each run's own
parity with the FP64 oracle is covered by test_gpu_parity.py.
"""
import numpy as np
import pytest

from paper_2410_05902_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

SPECS = [  # (spec, precision, distance tile)
    (inputs.RunSpec(3000, 16, 7, 256, 1), "fp32", 0),
    (inputs.RunSpec(2500, 64, 12, 512, 2), "bf16x3", 64),
    (inputs.RunSpec(4000, 40, 5, 128, 3), "bf16", 128),
    (inputs.RunSpec(1500, 100, 20, 256, 4), "bf16x3", 128),
    (inputs.RunSpec(6000, 256, 30, 1024, 5), "bf16x3", 0),
]


def _make(spec, precision, tile, seed):
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKM
    X, _ = spec.make()
    sigma = inputs.median_sigma(X, seed=1)
    Xd = torch.from_numpy(X).cuda()
    return KKM(Xd, spec.k, spec.b, kernel="gaussian", param=2 * sigma * sigma, tau=40, precision=precision,
               dist_tile=tile, seed=seed, init_idx=inputs.init_indices(spec.n, spec.k, seed=seed))


def _same_state(a, b):
    for key in a:
        va, vb = np.asarray(a[key]), np.asarray(b[key])
        assert va.shape == vb.shape and np.array_equal(va, vb), key


def test_group_steps_equal_individual_steps():
    from paper_2410_05902_gb300.group import Group
    grouped = [_make(sp, p, t, 10 + i) for i, (sp, p, t) in enumerate(SPECS)]
    alone = [_make(sp, p, t, 10 + i) for i, (sp, p, t) in enumerate(SPECS)]
    g = Group(grouped)
    for _ in range(7):
        g.step()
    g.sync()
    for r in alone:
        for _ in range(7):
            r.step()
        r.sync()
    for ra, rb in zip(grouped, alone):
        _same_state(ra.get_state(), rb.get_state())
    # a few more group steps keep working after the graph was captured
    for _ in range(3):
        g.step()
    g.sync()
    g.close()
    for r in grouped + alone:
        r.close()


def test_autotune_returns_a_measured_candidate():
    torch = torch_cuda()
    from paper_2410_05902_gb300.group import DEFAULT_CANDIDATES, autotune
    spec = inputs.RunSpec(5000, 64, 16, 512, 9)
    X, _ = spec.make()
    sigma = inputs.median_sigma(X, seed=1)
    Xd = torch.from_numpy(X).cuda()
    best, times = autotune(Xd, spec.k, spec.b, "gaussian", 2 * sigma * sigma, 40,
                           inputs.init_indices(spec.n, spec.k, seed=1), warm=5, iters=5)
    assert set(times) == set(DEFAULT_CANDIDATES)
    assert best in times and all(t > 0 for t in times.values())
    assert times[best] == min(times.values())
