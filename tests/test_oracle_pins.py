"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests retypes the oracle's own formulas. Each one checks the
oracle against one of the following:
  * a published test vector (SplitMix64),
  * a closed form derived by hand (the 1-D linear-kernel example),
  * a library routine that implements a definition (scipy's cdist),
  * an independent formulation: explicit feature vectors for the linear and
    degree-2 polynomial kernels, and textbook Lloyd,
  * an identity or bound the paper proves: the Sec. 4 norm recurrence, the
    Kanungo et al. lemma and the norm and objective bounds of Sec. 5, and the
    truncation lemma of Sec. 4.1.
Each is chosen so that a plausible slip fails it: a dropped C_1 term, a wrong
decay index, a renormalised truncated center, a sign error in the cross term,
or a transposed kernel argument.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import GAUSSIAN, LAPLACIAN, LINEAR, POLY, Kernel, MiniBatchKernelKMeans
from paper_2410_05902_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- sampler
def test_splitmix64_published_vector():
    lines = [l.split("#")[0].strip() for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))]
    lines = [l for l in lines if l]
    seed = int(lines[0].split()[1])
    expected = [int(v) for v in lines[1:]]
    assert [oracle.splitmix64(seed, c) for c in range(len(expected))] == expected


def test_index_below_is_multiply_high():
    n = 70000
    assert oracle.index_below(0, n) == 0
    assert oracle.index_below((1 << 64) - 1, n) == n - 1
    assert oracle.index_below(1 << 63, n) == n // 2
    idx = oracle.batch_indices(7, 1, 20000, 10)
    assert idx.min() >= 0 and idx.max() <= 9
    counts = np.bincount(idx, minlength=10)
    assert np.all(np.abs(counts - 2000) < 200)          # loose uniformity
    # iteration i uses counters (i-1)*b .. (i-1)*b+b-1
    b2 = oracle.batch_indices(7, 2, 5, 1000)
    assert b2[0] == oracle.index_below(oracle.splitmix64(7, 5), 1000)


# ----------------------------------------------------------------- kernels
def test_kernel_closed_forms():
    x, y = np.array([0.0, 0.0]), np.array([3.0, 4.0])       # ||x - y|| = 5, <x,y> = 0
    assert oracle.kernel_matrix(x, y, Kernel(GAUSSIAN, 10.0))[0, 0] == pytest.approx(math.exp(-2.5), rel=1e-15)
    assert oracle.kernel_matrix(x, y, Kernel(LAPLACIAN, 2.0))[0, 0] == pytest.approx(math.exp(-2.5), rel=1e-15)
    a, c = np.array([1.0, 2.0]), np.array([3.0, -1.0])      # <a,c> = 1
    assert oracle.kernel_matrix(a, c, Kernel(LINEAR))[0, 0] == 1.0
    assert oracle.kernel_matrix(a, c, Kernel(POLY, coef0=2.0, degree=3))[0, 0] == 27.0


@pytest.mark.parametrize("kind,param", [(GAUSSIAN, 7.5), (LAPLACIAN, 1.7)])
def test_kernel_matches_scipy_cdist(kind, param):
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(0)
    A, B = rng.normal(size=(13, 5)), rng.normal(size=(17, 5))
    D = cdist(A, B, "euclidean")
    ref = np.exp(-D ** 2 / param) if kind == GAUSSIAN else np.exp(-D / param)
    np.testing.assert_allclose(oracle.kernel_matrix(A, B, Kernel(kind, param)), ref, rtol=1e-13)


@pytest.mark.parametrize("kern", [Kernel(GAUSSIAN, 3.0), Kernel(LAPLACIAN, 1.5), Kernel(LINEAR),
                                  Kernel(POLY, coef0=1.0, degree=2)])
def test_kernel_symmetric_psd(kern):
    rng = np.random.default_rng(1)
    A = rng.normal(size=(40, 6))
    G = oracle.kernel_matrix(A, A, kern)
    np.testing.assert_array_equal(G, G.T)
    assert np.linalg.eigvalsh(G).min() > -1e-9 * max(1.0, np.abs(G).max())
    np.testing.assert_allclose(np.diag(G), oracle.kernel_diag(A, kern), rtol=1e-14)
    w = rng.random(40)
    np.testing.assert_allclose(oracle.kernel_wsum(A[:7], A, w, kern), G[:7] @ w, rtol=1e-12)


def test_gaussian_gamma_is_one_golden_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "gamma_table.txt")) if l.strip() and not l.startswith("#")]
    gauss = [float(r[2]) for r in rows if r[1] == "gaussian"]
    assert len(gauss) == 4
    X, _ = inputs.isotropic_mixture(300, 16, 5, seed=3)
    kern = Kernel(GAUSSIAN, 2 * inputs.median_sigma(X, seed=0) ** 2)
    gamma = math.sqrt(np.max(np.diag(oracle.kernel_matrix(X, X, kern))))
    for g in gauss:
        assert gamma == pytest.approx(g, abs=5e-4)          # table rounds to 3 s.f.


# ------------------------------------------------- hand-derived 1-D example
def test_tiny_linear_1d_closed_form():
    """X = (0, 1, 10, 11), K(x,y) = xy, k = 2, C_1 = (x=0, x=10), batch = all four.

    Iteration 1 assigns {0,1} -> 0 and {10,11} -> 1, so b^j = 2 and
    alpha = sqrt(2/4) = 1/sqrt(2). Untruncated: C^0 = alpha/2 and
    C^1 = 10 + alpha/2. With tau = 2, the window after iteration 2 is {2}
    (b_2 = 2 >= tau), so C_1 and block 1 are dropped and the truncated center
    keeps only alpha * cm(B_2) with its untruncated weight: 0.5*alpha and
    10.5*alpha, not renormalised.
    """
    X = np.array([[0.0], [1.0], [10.0], [11.0]])
    a = 1.0 / math.sqrt(2.0)
    batch = np.arange(4)
    m = MiniBatchKernelKMeans(X, 2, Kernel(LINEAR), 4, [0, 2], tau=None)
    r1 = m.step(batch)
    np.testing.assert_allclose(r1.dist, [[0, 100], [1, 81], [100, 0], [121, 1]], atol=1e-12)
    assert r1.batch_objective == pytest.approx(0.5)
    np.testing.assert_array_equal(r1.counts, [2, 2])
    np.testing.assert_allclose(r1.alpha, [a, a], rtol=1e-15)
    c0, c1 = a / 2, 10 + a / 2
    np.testing.assert_allclose(r1.cnorm_after, [c0 ** 2, c1 ** 2], rtol=1e-12)
    r2 = m.step(batch)
    np.testing.assert_allclose(r2.dist[:, 0], (X[:, 0] - c0) ** 2, rtol=1e-12)
    np.testing.assert_allclose(r2.dist[:, 1], (X[:, 0] - c1) ** 2, rtol=1e-12)

    t = MiniBatchKernelKMeans(X, 2, Kernel(LINEAR), 4, [0, 2], tau=2)
    t.step(batch)
    assert t.center(0).c1_kept                     # window reaches iteration 1: untruncated
    t.step(batch)
    rep0, rep1 = t.center(0), t.center(1)
    assert not rep0.c1_kept and rep0.blocks == [(2, 2)]
    np.testing.assert_allclose(rep0.w @ X[rep0.idx, 0], 0.5 * a, rtol=1e-14)
    np.testing.assert_allclose(rep1.w @ X[rep1.idx, 0], 10.5 * a, rtol=1e-14)
    np.testing.assert_allclose(t.center_norms(), [(0.5 * a) ** 2, (10.5 * a) ** 2], rtol=1e-12)


# -------------------------------------- linear kernel = explicit mini-batch
def _explicit_minibatch(X, init_idx, batches, alpha_fn, k):
    """Mini-batch k-means on explicit vectors (Sec. 1, "Mini-batch k-means")."""
    C = X[init_idx].astype(np.float64).copy()
    recs = []
    for B in batches:
        P = X[B]
        D = ((P[:, None, :] - C[None, :, :]) ** 2).sum(-1)
        a = np.argmin(D, axis=1)
        cnt = np.bincount(a, minlength=k)
        alpha = alpha_fn(cnt)
        recs.append((D, a))
        for j in range(k):
            if cnt[j]:
                C[j] = (1 - alpha[j]) * C[j] + alpha[j] * P[a == j].mean(0)
    return recs, C


def test_linear_kernel_equals_explicit_minibatch_kmeans():
    X, _ = inputs.isotropic_mixture(400, 3, 4, seed=5)
    X = X.astype(np.float64)
    k, b = 4, 32
    init = inputs.init_indices(len(X), k, seed=1)
    batches = inputs.batch_stream(len(X), b, 12, seed=2)
    m = MiniBatchKernelKMeans(X, k, Kernel(LINEAR), b, init, tau=None)
    recs, C = _explicit_minibatch(X, init, batches, lambda c: np.sqrt(c / b), k)
    for B, (D, a) in zip(batches, recs):
        r = m.step(B)
        np.testing.assert_allclose(r.dist, D, rtol=1e-9, atol=1e-9)
        np.testing.assert_array_equal(r.assign, a)
    for j in range(k):
        rep = m.center(j)
        np.testing.assert_allclose(rep.w @ X[rep.idx], C[j], rtol=1e-10, atol=1e-12)


def test_sklearn_rate_is_the_running_mean():
    """With the sklearn rate b_i^j / N^j (N^j cumulative) and the linear
    kernel, an untruncated center is the plain mean of every point ever
    assigned to it (the init point until the first assignment) -- computed
    here directly from the assignments, with no weights."""
    X, _ = inputs.isotropic_mixture(300, 3, 4, seed=8)
    X = X.astype(np.float64)
    k, b = 4, 24
    init = inputs.init_indices(len(X), k, seed=2)
    m = MiniBatchKernelKMeans(X, k, Kernel(LINEAR), b, init, tau=None, lr="sklearn")
    members = [[] for _ in range(k)]
    for B in inputs.batch_stream(len(X), b, 10, seed=3):
        centers = np.array([X[members[j]].mean(axis=0) if members[j] else X[init[j]] for j in range(k)])
        r = m.step(B)
        expect = ((X[B][:, None, :] - centers[None, :, :]) ** 2).sum(axis=2)
        np.testing.assert_allclose(r.dist, expect, rtol=1e-9, atol=1e-9)
        for x, a in zip(B, r.assign):
            members[a].append(x)
        np.testing.assert_array_equal(m.cumulative_counts(), [len(v) for v in members])
    for j in range(k):
        rep = m.center(j)
        np.testing.assert_allclose(rep.w @ X[rep.idx], X[members[j]].mean(axis=0), rtol=1e-10, atol=1e-12)


def test_truncated_distances_equal_explicit_vectors():
    """With finite tau the oracle's kernel-trick distances equal explicit ones to sum_s w_s x_s."""
    X, _ = inputs.isotropic_mixture(300, 4, 3, seed=6)
    X = X.astype(np.float64)
    m = MiniBatchKernelKMeans(X, 3, Kernel(LINEAR), 24, [0, 1, 2], tau=20)
    for B in inputs.batch_stream(len(X), 24, 10, seed=3):
        reps = [m.center(j) for j in range(3)]
        C = np.stack([r.w @ X[r.idx] for r in reps])
        r = m.step(B)
        D = ((X[B][:, None, :] - C[None]) ** 2).sum(-1)
        np.testing.assert_allclose(r.dist, D, rtol=1e-9, atol=1e-9)
    assert any(not m.center(j).c1_kept for j in range(3))   # truncation did happen


def test_state_distances_equal_explicit_vectors():
    """Distances against an explicit window state: with the linear kernel they are
    squared distances to the explicit centroids sum_s w_s y_s, and the returned
    norms are ||sum_s w_s y_s||^2. With the Gaussian kernel they equal the
    oracle's own distances for the state it holds."""
    X, _ = inputs.isotropic_mixture(300, 5, 3, seed=16)
    X = X.astype(np.float64)
    m = MiniBatchKernelKMeans(X, 3, Kernel(LINEAR), 32, [4, 5, 6], tau=24)
    for B in inputs.batch_stream(len(X), 32, 8, seed=5):
        m.step(B)
    st = m.state()
    off = np.concatenate([[0], np.cumsum(st["rows_per_center"])])
    C = np.stack([st["row_w"][off[j]:off[j + 1]] @ X[st["row_idx"][off[j]:off[j + 1]]] for j in range(3)])
    Q = X[:40]
    d, cn = oracle.state_distances(X, Q, st, Kernel(LINEAR))
    np.testing.assert_allclose(d, ((Q[:, None, :] - C[None]) ** 2).sum(-1), rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(cn, (C * C).sum(1), rtol=1e-10)
    kg = Kernel(GAUSSIAN, 20.0)
    g = MiniBatchKernelKMeans(X, 3, kg, 32, [4, 5, 6], tau=24)
    for B in inputs.batch_stream(len(X), 32, 6, seed=8):
        g.step(B)
    d2, cn2 = oracle.state_distances(X, Q, g.state(), kg)
    np.testing.assert_allclose(d2, g.distances(Q), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(cn2, g.center_norms(), rtol=1e-12)


# ------------------------------------------- degree-2 polynomial, brute force
def _poly2_features(X, c):
    n, d = X.shape
    cols = []
    for i in range(d):
        for j in range(i, d):
            f = X[:, i] * X[:, j]
            cols.append(f if i == j else math.sqrt(2.0) * f)
    for i in range(d):
        cols.append(math.sqrt(2.0 * c) * X[:, i])
    cols.append(np.full(n, c))
    return np.stack(cols, 1)


def test_poly2_matches_explicit_feature_map():
    rng = np.random.default_rng(9)
    X = rng.normal(size=(40, 3))
    c = 0.7
    F = _poly2_features(X, c)
    kern = Kernel(POLY, coef0=c, degree=2)
    np.testing.assert_allclose(oracle.kernel_matrix(X, X, kern), F @ F.T, rtol=1e-12, atol=1e-12)
    k, b = 3, 8
    batches = inputs.batch_stream(len(X), b, 6, seed=4)
    m = MiniBatchKernelKMeans(X, k, kern, b, [0, 1, 2], tau=None)
    recs, C = _explicit_minibatch(F, np.array([0, 1, 2]), batches, lambda cnt: np.sqrt(cnt / b), k)
    for B, (D, a) in zip(batches, recs):
        r = m.step(B)
        np.testing.assert_allclose(r.dist, D, rtol=1e-9, atol=1e-9)
        np.testing.assert_array_equal(r.assign, a)


# ---------------------------------------------------- full-batch kernel Lloyd
def test_identity_batch_rate_one_is_kernel_lloyd():
    """b = n, the whole dataset as the batch and alpha = 1 give Lloyd in feature space."""
    X, _ = inputs.isotropic_mixture(120, 2, 3, seed=8)
    X = X.astype(np.float64)
    n, k = len(X), 3
    init = np.array([0, 1, 2])
    # textbook Lloyd on explicit vectors (linear kernel)
    C = X[init].copy()
    m = MiniBatchKernelKMeans(X, k, Kernel(LINEAR), n, init, tau=None, lr="const", eta=1.0)
    for _ in range(6):
        D = ((X[:, None] - C[None]) ** 2).sum(-1)
        a = np.argmin(D, 1)
        r = m.step(np.arange(n))
        np.testing.assert_array_equal(r.assign, a)
        np.testing.assert_allclose(r.dist, D, rtol=1e-9, atol=1e-9)
        for j in range(k):
            if np.any(a == j):
                C[j] = X[a == j].mean(0)
    # Gaussian kernel: the Lloyd objective f_X never increases
    g = MiniBatchKernelKMeans(X, k, Kernel(GAUSSIAN, 4.0), n, init, tau=None, lr="const", eta=1.0)
    objs = [g.step(np.arange(n)).batch_objective for _ in range(6)]
    assert all(b <= a + 1e-12 for a, b in zip(objs, objs[1:]))


# -------------------------------------------------------- paper identities
def test_norm_recurrence_of_sec4():
    """Sec. 4: ||C'||^2 = (1-a)^2||C||^2 + 2a(1-a)<C,cm(B)> + a^2||cm(B)||^2 (untruncated)."""
    X, _ = inputs.isotropic_mixture(200, 5, 3, seed=10)
    kern = Kernel(GAUSSIAN, 6.0)
    b, k = 30, 3
    m = MiniBatchKernelKMeans(X, k, kern, b, [0, 1, 2], tau=None)
    Xd = X.astype(np.float64)
    for B in inputs.batch_stream(len(X), b, 8, seed=5):
        r = m.step(B)
        for j in range(k):
            rows = B[r.assign == j]
            if len(rows) == 0:
                assert r.cnorm_after[j] == pytest.approx(r.cnorm_before[j], rel=1e-12)
                continue
            a = r.alpha[j]
            # <phi(x), C> = (K(x,x) + ||C||^2 - Delta(x, C)) / 2 for the assigned rows
            inner = (1.0 + r.cnorm_before[j] - r.dist[r.assign == j, j]) / 2
            cm_c = inner.mean()
            cm_cm = oracle.kernel_matrix(Xd[rows], Xd[rows], kern).mean()
            rec = (1 - a) ** 2 * r.cnorm_before[j] + 2 * a * (1 - a) * cm_c + a * a * cm_cm
            assert r.cnorm_after[j] == pytest.approx(rec, rel=1e-11, abs=1e-13)


def test_kanungo_identity():
    """Delta(S, C) = Delta(S, cm(S)) + |S| Delta(C, cm(S)) for C a current center."""
    X, _ = inputs.isotropic_mixture(150, 4, 3, seed=11)
    kern = Kernel(GAUSSIAN, 5.0)
    m = MiniBatchKernelKMeans(X, 3, kern, 20, [0, 1, 2], tau=15)
    for B in inputs.batch_stream(len(X), 20, 5, seed=6):
        m.step(B)
    S = np.arange(10, 30)
    rep = m.center(1)
    lhs = m.distances(X[S])[:, 1].sum()
    uni = np.full(len(S), 1.0 / len(S))
    d_S_cm = sum(oracle.distance_to_combination(X, X[s], S, uni, kern) for s in S)
    # Delta(C, cm(S)) = ||C - cm(S)||^2 as one signed combination
    diff = oracle.combination_norm2(X, np.concatenate([rep.idx, S]), np.concatenate([rep.w, -uni]), kern)
    assert lhs == pytest.approx(d_S_cm + len(S) * diff, rel=1e-10)


def test_gaussian_bounds_and_weight_sums():
    X, _ = inputs.isotropic_mixture(500, 8, 5, seed=12)
    kern = Kernel(GAUSSIAN, 2 * inputs.median_sigma(X, seed=1) ** 2)
    b, k = 64, 5
    init = inputs.init_indices(len(X), k, seed=2)
    t = MiniBatchKernelKMeans(X, k, kern, b, init, tau=40)
    u = MiniBatchKernelKMeans(X, k, kern, b, init, tau=None)
    for B in inputs.batch_stream(len(X), b, 15, seed=7):
        for m in (t, u):
            r = m.step(B)
            assert r.dist.min() >= -1e-12 and r.dist.max() <= 4.0 + 1e-12     # 0 <= Delta <= 4 gamma^2
            assert np.all(r.cnorm_after <= 1.0 + 1e-12)                        # ||C|| <= gamma
        for j in range(k):
            assert u.center(j).w.sum() == pytest.approx(1.0, abs=1e-13)       # convex combination
            wt = t.center(j).w
            assert np.all(wt >= 0) and wt.sum() <= 1.0 + 1e-13


def test_window_definition_properties():
    """Q_i^j: sum over the window >= tau, dropping its oldest block gives < tau,
    the sum is <= tau + b, the start never moves back, and C_hat = C while min Q = 1."""
    X, _ = inputs.isotropic_mixture(400, 4, 4, seed=13)
    kern = Kernel(GAUSSIAN, 8.0)
    tau, b, k = 50, 40, 4
    m = MiniBatchKernelKMeans(X, k, kern, b, [0, 1, 2, 3], tau=tau)
    prev = [1] * k
    for B in inputs.batch_stream(len(X), b, 25, seed=8):
        m.step(B)
        for j in range(k):
            rep = m.center(j)
            counts = [c for it, c in rep.blocks if it > 0]
            total = sum(counts)
            assert total <= tau + b
            if rep.window_start > 1:
                assert total >= tau and total - counts[0] < tau
            else:
                assert rep.c1_kept and m.truncation_error(j) == 0.0
            assert rep.window_start >= prev[j]
            prev[j] = rep.window_start
    assert max(prev) > 1


def test_truncation_lemma_bound():
    """Sec. 4.1 lemma: tau = ceil(b ln^2(28 gamma / eps)) gives ||C_hat - C|| <= eps / 28."""
    X, _ = inputs.isotropic_mixture(300, 4, 3, seed=14)
    kern = Kernel(GAUSSIAN, 2 * inputs.median_sigma(X, seed=2) ** 2)
    b, eps = 8, 4.0
    tau = math.ceil(b * math.log(28.0 / eps) ** 2)
    m = MiniBatchKernelKMeans(X, 3, kern, b, [0, 1, 2], tau=tau)
    truncated = False
    for B in inputs.batch_stream(len(X), b, 60, seed=9):
        m.step(B)
        for j in range(3):
            err2 = m.truncation_error(j)
            truncated |= err2 > 0
            assert err2 <= (eps / 28.0) ** 2 * (1 + 1e-12)
    assert truncated


def test_empty_cluster_unchanged_and_full_rate_erases():
    X, _ = inputs.isotropic_mixture(200, 3, 2, seed=15)
    kern = Kernel(GAUSSIAN, 3.0)
    m = MiniBatchKernelKMeans(X, 2, kern, 10, [0, 1], tau=None)
    # force every point into center 0: center 1 is empty (alpha = 0), center 0 has alpha = 1
    B = np.arange(10)
    before = m.center(1)
    r = m.step(B, forced_assign=np.zeros(10, dtype=np.int64))
    assert r.alpha[1] == 0.0 and r.alpha[0] == 1.0
    after = m.center(1)
    np.testing.assert_array_equal(after.idx, before.idx)
    np.testing.assert_array_equal(after.w, before.w)
    assert r.cnorm_after[1] == pytest.approx(r.cnorm_before[1], rel=1e-14)
    rep0 = m.center(0)
    assert rep0.w[0] == 0.0                                  # C_1 weight (1 - 1) = 0
    np.testing.assert_allclose(rep0.w[1:], 0.1)
    assert r.cnorm_after[0] == pytest.approx(oracle.kernel_matrix(X[B], X[B], kern).mean(), rel=1e-12)


# -------------------------------------------------------------- k-means++
def test_kmeanspp_d2_sampling():
    X = np.array([[0.0], [0.0], [5.0], [10.0]])
    kern = Kernel(LINEAR)
    for seed in range(20):
        ch = oracle.kmeanspp(X, 3, kern, seed)
        assert ch[0] == oracle.index_below(oracle.splitmix64(seed, 0), 4)
        assert len(set(X[ch, 0].tolist())) == 3          # zero-D^2 points are never re-picked
    # second-pick frequencies follow D^2 / sum D^2 from a fixed first pick
    X2 = np.array([[0.0], [1.0], [3.0]])
    picks = np.zeros(3)
    for seed in range(3000):
        ch = oracle.kmeanspp(X2, 2, kern, seed)
        if ch[0] == 0:
            picks[ch[1]] += 1
    p = picks / picks.sum()
    np.testing.assert_allclose(p, [0.0, 0.1, 0.9], atol=0.04)
