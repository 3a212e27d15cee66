"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Protocols:
  teacher-forced   the oracle's state is loaded into the GPU (kkm_set_state),
                   both take one step on the same batch with the GPU forced to
                   the oracle's assignment, and every output is compared:
                   distances, argmin, f_B, counts, and the new windows,
                   weights and center norms.
  free-running     both run from the same initial centers on the same batch
                   stream. f_B and the assignments are compared every
                   iteration until a certified near-tie legitimately flips an
                   assignment.
"""
import numpy as np
import pytest

import oracle
from paper_2410_05902_gb300 import inputs
from gpu_helpers import (CN_RTOL, DIST_TOL, OBJ_TOL, OBJ_TOL_FORM, Pair, compare_states, dist_rel_err,
                         near_tie_ok, torch_cuda)

pytestmark = pytest.mark.gpu


def small_data(n=2000, d=16, c=10, seed=12345):
    X, _ = inputs.isotropic_mixture(n, d, c, seed=seed)
    return X


def teacher_forced(pair, batches, w_rtol=1e-12, cn_rtol=1e-6, check_assign=True):
    tol = DIST_TOL[pair.precision]
    worst = 0.0
    for B in batches:
        ora_state = pair.ora.state()
        pair.gpu.set_state(ora_state)
        rec = pair.ora.step(B)
        d, a, f = pair.gpu_step(B, forced=rec.assign)
        err = dist_rel_err(d, rec.dist)
        worst = max(worst, err)
        assert err <= tol, f"iteration {rec.iteration}: distance rel err {err:.3e} > {tol}"
        if check_assign:
            ok, nbad = near_tie_ok(a, rec, pair.abs_tol(rec))
            assert ok, f"iteration {rec.iteration}: {nbad} assignments differ outside near-ties"
        assert abs(f - rec.batch_objective) <= OBJ_TOL_FORM[pair.precision] * abs(rec.batch_objective) + 1e-12
        compare_states(pair.gpu.get_state(), pair.ora.state(), w_rtol=w_rtol, cn_rtol=cn_rtol)
    return worst


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "bf16", "tf32"])
def test_teacher_forced_small(precision):
    X = small_data()
    p = Pair(X, k=10, b=256, tau=200, precision=precision)
    batches = inputs.batch_stream(len(X), 256, 12, seed=21)
    teacher_forced(p, batches, cn_rtol=CN_RTOL[precision])
    p.close()


def test_free_running_small_fp32():
    """50 iterations of the small mixture (n=2000, d=16, k=10, b=256, tau=200)."""
    X = small_data()
    p = Pair(X, k=10, b=256, tau=200, precision="fp32")
    batches = inputs.batch_stream(len(X), 256, 50, seed=22)
    for B in batches:
        rec = p.ora.step(B)
        d, a, f = p.gpu_step(B)
        assert dist_rel_err(d, rec.dist) <= DIST_TOL["fp32"]
        assert abs(f - rec.batch_objective) <= OBJ_TOL * rec.batch_objective
        if not np.array_equal(a, rec.assign):
            ok, _ = near_tie_ok(a, rec, p.abs_tol(rec))
            assert ok
            break                       # a certified tie flipped: trajectories may diverge now
    compare_states(p.gpu.get_state(), p.ora.state())
    p.close()


def test_builtin_sampler_is_splitmix64():
    X = small_data(n=3000, d=8, c=4)
    p = Pair(X, k=4, b=300, tau=0, max_iters=3, seed=987654321)
    for it in (1, 2):
        B = oracle.batch_indices(987654321, it, 300, len(X))
        rec = p.ora.step(B)
        p.gpu.step(None, None, p.assign, p.dist, p.obj)
        p.torch.cuda.synchronize()
        np.testing.assert_array_equal(p.assign.cpu().numpy(), rec.assign)
    compare_states(p.gpu.get_state(), p.ora.state())   # row_idx carries the sampled indices
    p.close()


@pytest.mark.parametrize("kernel,extra", [
    ("laplacian", {}),
    ("linear", {}),
    ("poly", {"coef0": 1.0, "degree": 2}),
])
def test_other_kernels_teacher_forced(kernel, extra):
    rng = np.random.default_rng(4)
    X = small_data(n=600, d=12, c=5)
    if kernel in ("linear", "poly"):
        X = (X / 4.0).astype(np.float32)          # keep polynomial values moderate
    param = 1.0 if kernel in ("linear", "poly") else None
    p = Pair(X, k=5, b=96, kernel=kernel, param=param, tau=60, **extra)
    batches = inputs.batch_stream(len(X), 96, 8, seed=int(rng.integers(1 << 30)))
    teacher_forced(p, batches, cn_rtol=1e-5)
    p.close()


@pytest.mark.parametrize("n,d,k,b,tau", [
    (500, 13, 3, 77, 50),     # ragged d (not a multiple of 16/64) and b (not a multiple of 64/128)
    (400, 70, 1, 64, 30),     # a single center
    (300, 5, 7, 33, 1),       # tau = 1: only the newest block survives
    (300, 9, 4, 200, 500),    # tau larger than anything reached: no truncation
    (2500, 3, 12, 1000, 64),  # many centers, large batch, tiny d
    (3000, 8, 80, 1024, 64),  # more than 64 centers: sort/plan scans a center per thread
    (4000, 8, 80, 2048, 64),  # the same over two 1024-row chunks of the stable sort
])
def test_edge_shapes_teacher_forced(n, d, k, b, tau):
    X = small_data(n=n, d=d, c=max(k, 2))
    p = Pair(X, k=k, b=b, tau=tau)
    batches = inputs.batch_stream(n, b, 6, seed=n + d)
    teacher_forced(p, batches)
    p.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_window_compaction_free_running(precision):
    """Each center's region holds cap = 2*tau + 4*b + 8 rows. With tau=10 and b=40 that is 188
    rows, while a center receives about 20 rows per iteration. So over 40 iterations every
    window is copied back to the start of its region several times. The windows, weights and
    norms must still match the oracle, which has no such storage."""
    X = small_data(n=400, d=6, c=2)
    p = Pair(X, k=2, b=40, tau=10, precision=precision)
    for B in inputs.batch_stream(len(X), 40, 40, seed=17):
        rec = p.ora.step(B)
        d, a, f = p.gpu_step(B)
        assert dist_rel_err(d, rec.dist) <= DIST_TOL[precision]
        if not np.array_equal(a, rec.assign):
            ok, _ = near_tie_ok(a, rec, p.abs_tol(rec))
            assert ok
            pytest.skip("a certified near-tie flipped an assignment; trajectories diverge")
    compare_states(p.gpu.get_state(), p.ora.state(), cn_rtol=1e-5)
    p.close()


def test_untruncated_algorithm1():
    X = small_data(n=800, d=10, c=4)
    p = Pair(X, k=4, b=64, tau=0, max_iters=10)
    teacher_forced(p, inputs.batch_stream(len(X), 64, 10, seed=5))
    for j in range(4):                    # Algorithm 1 keeps C_1 and every block
        assert p.ora.center(j).c1_kept
    p.close()


def test_full_rate_and_empty_clusters():
    """Every point forced into center 0: alpha_0 = 1 erases the old center and the
    other centers, being empty, must not change (alpha = 0)."""
    X = small_data(n=500, d=6, c=3)
    p = Pair(X, k=3, b=50, tau=20)
    B = inputs.batch_stream(len(X), 50, 1, seed=9)[0]
    p.gpu.set_state(p.ora.state())
    forced = np.zeros(50, dtype=np.int64)
    rec = p.ora.step(B, forced_assign=forced)
    p.gpu_step(B, forced=forced)
    compare_states(p.gpu.get_state(), p.ora.state())
    assert rec.alpha[0] == 1.0 and np.all(rec.alpha[1:] == 0.0)
    p.close()


def test_duplicate_batch_rows_and_const_rate():
    X = small_data(n=50, d=4, c=2)
    p = Pair(X, k=2, b=40, tau=25, lr="const", eta=0.5)
    batches = inputs.batch_stream(len(X), 40, 6, seed=2)   # 40 draws from 50 points repeat
    teacher_forced(p, batches)
    p.close()


def test_assign_and_objective_queries():
    X = small_data(n=1500, d=16, c=6)
    p = Pair(X, k=6, b=128, tau=100)
    for B in inputs.batch_stream(len(X), 128, 5, seed=31):
        p.ora.step(B)
        p.gpu_step(B)
    p.gpu.set_state(p.ora.state())
    torch = p.torch
    Q = torch.from_numpy(X[:700]).cuda()
    a, md, dist = p.gpu.assign(Q, want_dist=True)
    ref = p.ora.distances(X[:700].astype(np.float64))
    assert dist_rel_err(dist.cpu().numpy(), ref) <= DIST_TOL["fp32"]
    order = np.sort(ref, 1)
    scale = float(np.max(np.abs(ref)))
    bad = np.nonzero(a.cpu().numpy() != ref.argmin(1))[0]
    assert np.all(order[bad, 1] - order[bad, 0] <= DIST_TOL["fp32"] * scale)
    assert np.max(np.abs(md.cpu().numpy() - ref.min(1))) <= DIST_TOL["fp32"] * scale
    f_gpu = p.gpu.objective()
    f_ref = p.ora.objective()
    assert abs(f_gpu - f_ref) <= OBJ_TOL * f_ref
    p.close()


def test_image_like_full_size_first_iterations():
    """The MNIST-shaped workload at full size (70000 x 784, k=10, b=1024, tau=200):
    the first three iterations from the same start, on both sides."""
    X, _ = inputs.image_like(70000, seed=12345)
    p = Pair(X, k=10, b=1024, tau=200, precision="fp32")
    for B in inputs.batch_stream(len(X), 1024, 3, seed=41):
        rec = p.ora.step(B)
        d, a, f = p.gpu_step(B)
        assert dist_rel_err(d, rec.dist) <= DIST_TOL["fp32"]
        ok, _ = near_tie_ok(a, rec, p.abs_tol(rec))
        assert ok and np.array_equal(a, rec.assign)
        assert abs(f - rec.batch_objective) <= OBJ_TOL * rec.batch_objective
    compare_states(p.gpu.get_state(), p.ora.state())
    p.close()


def test_invalid_batch_index_poisons_context():
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKMError
    X = small_data(n=200, d=4, c=2)
    p = Pair(X, k=2, b=16, tau=10)
    bad = torch.full((16,), 10_000, dtype=torch.int32, device="cuda")   # rejected, never read
    p.gpu.step(bad)
    with pytest.raises(KKMError, match="KKM_EINVAL"):
        p.gpu.sync()
    with pytest.raises(KKMError, match="KKM_ESTATE"):
        p.gpu.step(None)
    p.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_graph_replay_matches_eager(precision):
    """kkm_graph_enable: the captured step gives bit-identical windows, weights,
    norms and objectives to eager steps, with the built-in sampler."""
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKM
    X = small_data(n=3000, d=20, c=6)
    Xd = torch.from_numpy(X).cuda()
    init = inputs.init_indices(len(X), 6, seed=4)
    runs = [KKM(Xd, 6, 200, kernel="gaussian", param=40.0, tau=80, precision=precision, seed=99,
                init_idx=init) for _ in range(2)]
    runs[1].graph(True)
    objs = [[], []]
    obj = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(25):
        for r, run in enumerate(runs):
            run.step(None, None, None, None, obj)
            torch.cuda.synchronize()
            objs[r].append(float(obj.cpu()[0]))
    assert objs[0] == objs[1]
    a, b = runs[0].get_state(), runs[1].get_state()
    for key in a:
        np.testing.assert_array_equal(np.asarray(a[key]), np.asarray(b[key]), err_msg=key)
    for run in runs:
        run.close()


@pytest.mark.parametrize("precision,d,tile", [("bf16x3", 200, 128), ("bf16", 200, 64), ("bf16x3", 784, 128),
                                              ("bf16", 784, 256), ("bf16x3", 784, 256), ("bf16x3", 96, 64),
                                              ("tf32", 200, 128), ("tf32", 784, 256), ("tf32", 40, 64)])
def test_teacher_forced_wide_rows_tensor_path(precision, d, tile):
    """Wide rows give the tcgen05 passes several K-slices per tile (d=784: 13), with
    64-, 128- and 256-row support tiles in the distance pass."""
    X, _ = inputs.image_like(3000, seed=7, d=d, classes=8)
    p = Pair(X, k=8, b=512, tau=120, precision=precision, dist_tile=tile)
    batches = inputs.batch_stream(len(X), 512, 6, seed=23)
    teacher_forced(p, batches, cn_rtol=CN_RTOL[precision])
    p.close()


def test_image_like_full_size_split_bf16():
    """The MNIST-shaped workload at full size on the tensor-core path (split BF16)."""
    X, _ = inputs.image_like(70000, seed=12345)
    p = Pair(X, k=10, b=1024, tau=200, precision="bf16x3")
    for B in inputs.batch_stream(len(X), 1024, 3, seed=41):
        rec = p.ora.step(B)
        d, a, f = p.gpu_step(B)
        assert dist_rel_err(d, rec.dist) <= DIST_TOL["bf16x3"]
        ok, _ = near_tie_ok(a, rec, p.abs_tol(rec))
        assert ok
        if not np.array_equal(a, rec.assign):
            return                       # a certified near-tie flipped; trajectories diverge
        assert abs(f - rec.batch_objective) <= OBJ_TOL * rec.batch_objective
    compare_states(p.gpu.get_state(), p.ora.state(), cn_rtol=1e-6)
    p.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_sklearn_rate_teacher_forced(precision):
    """The sklearn rate b_i^j / N^j with N^j carried in the state (kkm_get/set_cum_counts)."""
    X = small_data(n=1500, d=12, c=6)
    p = Pair(X, k=6, b=128, tau=80, lr="sklearn", precision=precision)
    teacher_forced(p, inputs.batch_stream(len(X), 128, 8, seed=41))
    p.close()


def test_sklearn_rate_free_running():
    X = small_data(n=1200, d=8, c=5)
    p = Pair(X, k=5, b=96, tau=60, lr="sklearn")
    for B in inputs.batch_stream(len(X), 96, 20, seed=42):
        rec = p.ora.step(B)
        d, a, f = p.gpu_step(B)
        assert dist_rel_err(d, rec.dist) <= DIST_TOL["fp32"]
        assert abs(f - rec.batch_objective) <= OBJ_TOL * rec.batch_objective
        if not np.array_equal(a, rec.assign):
            assert near_tie_ok(a, rec, p.abs_tol(rec))[0]
            break
    compare_states(p.gpu.get_state(), p.ora.state())
    p.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_step_eval_objectives(precision):
    """f_{B_i}(C_i) and f_{B_i}(C_{i+1}) of kkm_step_eval against the oracle's
    batch objective before the update and its objective on the same batch after."""
    X = small_data()
    p = Pair(X, k=10, b=256, tau=200, precision=precision)
    torch = p.torch
    for B in inputs.batch_stream(len(X), 256, 6, seed=23):
        p.gpu.set_state(p.ora.state())
        rec = p.ora.step(B)
        after_ref = p.ora.objective(X[B].astype(np.float64))
        before, after = p.gpu.step_eval(torch.from_numpy(B.astype(np.int32)).cuda())
        p.gpu.sync()
        assert abs(float(before.cpu()[0]) - rec.batch_objective) <= OBJ_TOL * rec.batch_objective
        assert abs(float(after.cpu()[0]) - after_ref) <= OBJ_TOL * after_ref
    p.close()


def test_fit_stops_at_the_first_small_improvement():
    """kkm_fit stops after the first iteration whose improvement
    f_{B_i}(C_i) - f_{B_i}(C_{i+1}) is below eps (Sec. 5); a twin run stepped
    with kkm_step_eval (same built-in sampler, same kernels) shows the same
    improvements."""
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKM
    X = small_data()
    sigma = inputs.median_sigma(X, seed=1)
    Xd = torch.from_numpy(X).cuda()
    init = inputs.init_indices(len(X), 10, seed=3)
    mk = lambda: KKM(Xd, 10, 256, kernel="gaussian", param=2 * sigma * sigma, tau=200, seed=5, init_idx=init)
    eps = 2e-3
    a, b = mk(), mk()
    done, last = a.fit(100, eps)
    imps = []
    for _ in range(done):
        before, after = b.step_eval()
        imps.append(float(before.cpu()[0]) - float(after.cpu()[0]))
    assert 1 <= done <= 100
    assert imps[-1] == last
    assert all(v >= eps for v in imps[:-1])
    assert done == 100 or last < eps
    a.close()
    b.close()


@pytest.mark.parametrize("precision,tile,kernel", [("bf16", 256, "gaussian"), ("bf16x3", 128, "gaussian"),
                                                   ("tf32", 256, "laplacian"), ("bf16x3", 64, "laplacian")])
def test_teacher_forced_many_items_per_cta(precision, tile, kernel):
    """More distance-pass items than SMs, so each CTA runs several and the two
    epilogue groups alternate (one item per CTA runs both groups on it)."""
    torch = torch_cuda()
    X = small_data(n=12000, d=48, c=40, seed=77)
    p = Pair(X, k=40, b=2048, kernel=kernel, tau=60, precision=precision, dist_tile=tile)
    batches = inputs.batch_stream(len(X), 2048, 4, seed=78)
    p.gpu.stats(reset=True)
    teacher_forced(p, batches, cn_rtol=CN_RTOL[precision])
    steps, _, tiles = p.gpu.stats(reset=True)
    items = (2048 // 128) * tiles / steps
    assert items > 2 * torch.cuda.get_device_properties(0).multi_processor_count
    p.close()
