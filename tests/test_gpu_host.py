"""kkm_step_host (host buffers through the context's device-mapped staging area)
against kkm_step with device buffers, and the back-to-back timing mode against
plain steps: twin contexts on the same data, seed and initial centers must
give bit-identical assignments, objectives and states."""
import numpy as np
import pytest

from paper_2410_05902_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _twins(precision, graph, n=3000, d=24, k=8, b=256, tau=80):
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKM
    X, _ = inputs.isotropic_mixture(n, d, k, seed=31)
    sigma = inputs.median_sigma(X, seed=1)
    Xd = torch.from_numpy(X).cuda()
    init = inputs.init_indices(n, k, seed=32)
    runs = [KKM(Xd, k, b, kernel="gaussian", param=2 * sigma * sigma, tau=tau, precision=precision, seed=9,
                init_idx=init) for _ in range(2)]
    for r in runs:
        r.graph(graph)
    return torch, runs, n, b


def _same_state(a, b):
    sa, sb = a.get_state(), b.get_state()
    for key in sa:
        assert np.array_equal(np.asarray(sa[key]), np.asarray(sb[key])), key


@pytest.mark.parametrize("precision,graph", [("bf16x3", True), ("fp32", False), ("bf16", True)])
def test_step_host_matches_device_step(precision, graph):
    torch, (h, dv), n, b = _twins(precision, graph)
    a_dev = torch.empty(b, dtype=torch.int32, device="cuda")
    o_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    batches = inputs.batch_stream(n, b, 6, seed=33)
    for i in range(12):
        # explicit batches first, then the built-in sampler
        B = batches[i] if i < 6 else None
        a_host, f_host = h.step_host(B)
        dv.step(None if B is None else torch.from_numpy(B.astype(np.int32)).cuda(), None, a_dev, None, o_dev)
        dv.sync()
        assert np.array_equal(a_host, a_dev.cpu().numpy()), i
        assert f_host == float(o_dev.cpu()[0]), i
    _same_state(h, dv)
    h.close()
    dv.close()


def test_back_to_back_timing_leaves_results_unchanged():
    """Timing mode R > 1 launches the distance pass R times per step; the pass
    is idempotent, so the run must match an untimed twin exactly."""
    torch, (t, p), n, b = _twins("bf16", False)
    t.timing(20)
    a1 = torch.empty(b, dtype=torch.int32, device="cuda")
    a2 = torch.empty(b, dtype=torch.int32, device="cuda")
    for B in inputs.batch_stream(n, b, 8, seed=34):
        bi = torch.from_numpy(B.astype(np.int32)).cuda()
        t.step(bi, None, a1)
        p.step(bi, None, a2)
        t.sync()
        p.sync()
        assert torch.equal(a1, a2)
    n_rec, ms = t.timing_read(reset=True)
    t.timing(False)
    assert n_rec == 8 and ms > 0.0
    _same_state(t, p)
    t.close()
    p.close()


@pytest.mark.parametrize("precision,graph", [("bf16", True), ("fp32", False)])
def test_deferred_weight_update_applied_once(precision, graph):
    """A step leaves its weight update pending until the next step or the next
    call that reads the centers. Twin runs: one steps straight through, the
    other flushes, synchronises, reads the state and scores queries between
    its steps (each of which queues the pending update once). Assignments,
    batch objectives and final states must agree bit for bit."""
    torch, (a, b_), n, b = _twins(precision, graph)
    Xq = a.X[:300].contiguous()
    outs = []
    for r, busy in ((a, False), (b_, True)):
        res = []
        o = torch.empty(1, dtype=torch.float64, device="cuda")     # fixed outputs: the graph replays
        asg = torch.empty(b, dtype=torch.int32, device="cuda")
        for i in range(10):
            r.step(None, None, asg, None, o)
            if busy:
                if i % 3 == 0:
                    r.flush()
                    r.flush()                    # nothing left to apply
                elif i % 3 == 1:
                    r.get_state()
                else:
                    r.assign(Xq)
                r.sync()
            res.append((asg.cpu().numpy(), float(o.cpu()[0])))
        r.sync()
        outs.append(res)
    for i, ((aa, fa), (ab, fb)) in enumerate(zip(*outs)):
        assert np.array_equal(aa, ab), i
        assert fa == fb, i
    _same_state(a, b_)
    a.close()
    b_.close()


@pytest.mark.parametrize("precision,graph", [("bf16", True), ("fp32", False)])
def test_steps_match_single_steps(precision, graph):
    """kkm_steps(n) (16 iterations per graph replay, the rest one by one) gives
    the same centers, bit for bit, as n calls of kkm_step with the sampler."""
    torch, (a, b_), n, b = _twins(precision, graph)
    a.steps(37)
    for _ in range(37):
        b_.step()
    a.sync()
    b_.sync()
    _same_state(a, b_)
    a.steps(16)
    for _ in range(16):
        b_.step()
    assert a.stats()[0] == b_.stats()[0] == 53
    _same_state(a, b_)
    a.close()
    b_.close()


@pytest.mark.parametrize("precision,graph", [("bf16", True), ("bf16x3", True), ("fp32", False)])
def test_steps_host_matches_single_host_steps(precision, graph):
    """kkm_steps_host (chunks of 16 through two staging slots, one graph per
    slot) gives, bit for bit, the assignments, f_B values and final state of
    one kkm_step_host call per step: a context's first call (its first step
    goes one at a time), two full chunks and a ragged tail, then a call with
    the built-in sampler and a call of zero steps."""
    torch, (m, s1), n, b = _twins(precision, graph)
    batches = np.stack(inputs.batch_stream(n, b, 41, seed=35)).astype(np.int32)
    a_m, f_m = m.steps_host(batches)
    for i in range(41):
        a_s, f_s = s1.step_host(batches[i])
        assert np.array_equal(a_m[i], a_s), i
        assert f_m[i] == f_s, i
    _same_state(m, s1)
    a_m, f_m = m.steps_host(None, n=19)
    for i in range(19):
        a_s, f_s = s1.step_host(None)
        assert np.array_equal(a_m[i], a_s), i
        assert f_m[i] == f_s, i
    a_m, f_m = m.steps_host(None, n=0)
    assert a_m.shape == (0, b) and f_m.shape == (0,)
    _same_state(m, s1)
    assert m.stats()[0] == s1.stats()[0] == 60
    m.close()
    s1.close()

