"""Run groups (kkm_group_*): a group step is exactly one step of every run.

Runs of different shapes, precision forms, tile widths and kernels stepped
through one group must end in the same state, bit for bit, as identical runs
stepped on their own, whichever launch structure the group uses: one launch
per phase over all runs (one chain or three concurrent chains), or every
run's own kernels on a graph branch of its own. Each run's own
parity with the FP64 oracle is covered by test_gpu_parity.py.
"""
import numpy as np
import pytest

from paper_2410_05902_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

SPECS = [  # (spec, precision, distance tile, kernel)
    (inputs.RunSpec(3000, 16, 7, 256, 1), "fp32", 0, "gaussian"),
    (inputs.RunSpec(2500, 64, 12, 512, 2), "bf16x3", 64, "gaussian"),
    (inputs.RunSpec(4000, 40, 5, 128, 3), "bf16", 128, "gaussian"),
    (inputs.RunSpec(1500, 100, 20, 256, 4), "bf16x3", 128, "gaussian"),
    (inputs.RunSpec(6000, 256, 30, 1024, 5), "bf16x3", 0, "gaussian"),
    (inputs.RunSpec(3500, 32, 9, 512, 6), "tf32", 128, "gaussian"),
    (inputs.RunSpec(2000, 24, 6, 384, 7), "bf16x3", 128, "laplacian"),
    (inputs.RunSpec(2200, 48, 11, 256, 8), "bf16x3", 64, "gaussian"),   # same class as run 1
]
# distance-pass classes (form, kernel, tile): fp32; bf16x3/64; bf16/128; bf16x3/128; bf16x3/256; tf32/128;
# bf16x3/128 Laplacian. Window-pass classes ignore the tile: fp32, bf16x3, bf16, tf32, bf16x3 Laplacian.
N_DIST, N_WINDOW = 7, 5


def _make(spec, precision, tile, kernel, seed):
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKM
    X, _ = spec.make()
    sigma = inputs.median_sigma(X, seed=1)
    Xd = torch.from_numpy(X).cuda()
    param = 2 * sigma * sigma if kernel == "gaussian" else sigma
    return KKM(Xd, spec.k, spec.b, kernel=kernel, param=param, tau=40, precision=precision,
               dist_tile=tile, seed=seed, init_idx=inputs.init_indices(spec.n, spec.k, seed=seed))


def _same_state(a, b):
    for key in a:
        va, vb = np.asarray(a[key]), np.asarray(b[key])
        assert va.shape == vb.shape and np.array_equal(va, vb), key


@pytest.mark.parametrize("chains", [0, 1, 3])
def test_group_steps_equal_individual_steps(chains):
    from paper_2410_05902_gb300.group import Group
    grouped = [_make(sp, p, t, kn, 10 + i) for i, (sp, p, t, kn) in enumerate(SPECS)]
    alone = [_make(sp, p, t, kn, 10 + i) for i, (sp, p, t, kn) in enumerate(SPECS)]
    g = Group(grouped)
    if chains == 1:
        # one launch per phase over all runs, one per Gram pass and class
        assert g.launches()[1] == 5 + N_DIST + N_WINDOW
    else:
        g.set_chains(chains)
    if chains == 0:
        assert g.launches()[1] == 7 * len(SPECS)    # every run's own seven kernels on a branch of its own
    per_step = g.launches()[1]
    for _ in range(7):
        g.step()
    g.sync()
    for r in alone:
        for _ in range(7):
            r.step()
        r.sync()
    for ra, rb in zip(grouped, alone):
        _same_state(ra.get_state(), rb.get_state())
    # the captured graph (steps 2 on) keeps matching the runs stepped alone
    for _ in range(5):
        g.step()
    g.sync()
    for r in alone:
        for _ in range(5):
            r.step()
        r.sync()
    for ra, rb in zip(grouped, alone):
        _same_state(ra.get_state(), rb.get_state())
    assert g.launches()[0] == 12 * per_step
    with pytest.raises(Exception):
        g.set_chains(2)              # only before the first step
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
