"""FP64 oracle of truncated mini-batch kernel k-means (test infrastructure only).

This is a plain restatement of Algorithm 2 (Appendix A) with the truncated
centers of Eq. (1), Sec. 4.1. With ``tau=None`` it is Algorithm 1 (Sec. 4).
It is slow on purpose and uses no recurrences.

* Each center is rebuilt every iteration from the full history of assigned
  blocks B_l^j and learning rates alpha_l^j. The unrolled center expression
  of Sec. 4.1 gives block l the weight alpha_l * prod_{z=l+1..i}(1 - alpha_z)
  and C_1 the weight prod_{z=1..i}(1 - alpha_z).
* The window Q_i^j follows its Sec. 4.1 definition. It runs from iteration i
  back to the latest iteration m with sum_{l=m..i} b_l^j >= tau. If no such m
  exists, it runs back to iteration 1. The printed subscript b_i^j inside that
  sum is read as b_l^j.
* Eq. (1): while min Q_i^j > 1 only the window's blocks are kept, with their
  untruncated weights and no renormalisation. Otherwise the center equals the
  untruncated one, C_1 term included.
* Distances are the kernel-trick expansion of Sec. 1 ("Lloyd's algorithm in
  feature space") with every term computed directly:
  Delta(x, C) = K(x,x) - 2 sum_s w_s K(x, y_s) + sum_{s,t} w_s w_t K(y_s, y_t).
* Assignment is the argmin of Algorithms 1/2. Ties, which the analysis breaks
  arbitrarily, go to the lowest center index.
* The learning rate is the beta rate alpha = sqrt(b_i^j / b) of Schwartzman
  (2023), the one the truncation lemma's proof uses (Sec. 4.1), or a constant.
  An empty cluster has alpha = 0 and its center does not change.

Every FP64 value here comes from these definitions, never from the CUDA path.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .kernels import Kernel, kernel_diag, kernel_matrix, kernel_wsum


@dataclass
class StepRecord:
    """Everything one iteration i computes (all FP64 / int64)."""

    iteration: int
    batch: np.ndarray          # (b,) data indices of B_i
    dist: np.ndarray           # (b, k) Delta(x, C_i^j)
    assign: np.ndarray         # (b,) argmin_j, ties to the lowest j
    gap: np.ndarray            # (b,) second-smallest minus smallest distance
    counts: np.ndarray         # (k,) b_i^j
    alpha: np.ndarray          # (k,) alpha_i^j
    batch_objective: float     # f_{B_i}(C_i) = mean_x min_j Delta(x, C_i^j)
    cnorm_before: np.ndarray   # (k,) ||C_i^j||^2
    cnorm_after: np.ndarray    # (k,) ||C_{i+1}^j||^2


@dataclass
class CenterRep:
    """A center as an explicit weighted sum of feature vectors of data points.

    ``idx`` and ``w`` list the support rows in window order: C_1 first (when it
    is kept), then the blocks from oldest to newest, each block in batch order.
    ``blocks`` lists the (iteration, count) pairs of the kept blocks in the
    same order, with C_1 as iteration 0 and count 1.
    """

    idx: np.ndarray
    w: np.ndarray
    blocks: list = field(default_factory=list)
    c1_kept: bool = True
    window_start: int = 1


def combination_norm2(X, idx, w, kernel: Kernel) -> float:
    """||sum_s w_s phi(x_{idx_s})||^2 = sum_{s,t} w_s w_t K(x_s, x_t), directly."""
    X = np.asarray(X, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    Y = X[idx]
    return float(w @ kernel_matrix(Y, Y, kernel) @ w)


def distance_to_combination(X, q, idx, w, kernel: Kernel) -> float:
    """Delta(q, sum_s w_s phi(x_s)) for one point q given by value (Sec. 3 notation)."""
    X = np.asarray(X, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)[None, :]
    cross = kernel_wsum(q, X[np.asarray(idx, dtype=np.int64)], w, kernel)[0]
    return float(kernel_diag(q, kernel)[0] - 2.0 * cross + combination_norm2(X, idx, w, kernel))


def state_distances(X, Q, state: dict, kernel: Kernel):
    """Delta(q, C^j) for every row q of Q against centers given explicitly by a
    window state (the layout of ``MiniBatchKernelKMeans.state``: support rows
    center by center with their weights), plus ||C^j||^2 of each center.

    Every term is computed directly from Eq. (1)'s weighted sum of feature
    vectors, as in ``MiniBatchKernelKMeans.distances``: the center norms are
    sum_{s,t} w_s w_t K(y_s, y_t), not a carried value. The state's own
    ``cnorm`` entry is not read. Returns (dist (m, k), cnorm (k,)).
    """
    X = np.asarray(X, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    if Q.ndim == 1:
        Q = Q[None, :]
    rows = np.asarray(state["rows_per_center"], dtype=np.int64)
    idx = np.asarray(state["row_idx"], dtype=np.int64)
    w = np.asarray(state["row_w"], dtype=np.float64)
    k = len(rows)
    off = np.concatenate([[0], np.cumsum(rows)])
    kqq = kernel_diag(Q, kernel)
    out = np.empty((Q.shape[0], k), dtype=np.float64)
    cn = np.empty(k, dtype=np.float64)
    for j in range(k):
        ij, wj = idx[off[j]:off[j + 1]], w[off[j]:off[j + 1]]
        Y = X[ij]
        cn[j] = float(wj @ kernel_matrix(Y, Y, kernel) @ wj) if len(ij) else 0.0
        cross = kernel_wsum(Q, Y, wj, kernel) if len(ij) else np.zeros(Q.shape[0])
        out[:, j] = kqq - 2.0 * cross + cn[j]
    return out, cn


class MiniBatchKernelKMeans:
    """Algorithm 2 (``tau`` an int) or Algorithm 1 (``tau=None``), FP64."""

    def __init__(self, X, k: int, kernel: Kernel, b: int, init_idx, tau: int | None = None,
                 lr: str = "beta", eta: float | None = None):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        if self.X.ndim != 2:
            raise ValueError("X must be n x d")
        self.n, self.d = self.X.shape
        self.k, self.b, self.tau, self.kernel = int(k), int(b), tau, kernel
        self.init_idx = np.asarray(init_idx, dtype=np.int64).copy()
        if self.init_idx.shape != (self.k,):
            raise ValueError("one initial point per center")
        if lr not in ("beta", "const", "sklearn"):
            raise ValueError("lr must be 'beta', 'const' or 'sklearn'")
        if lr == "const" and eta is None:
            raise ValueError("the constant rate needs eta")
        self.lr, self.eta = lr, eta
        self.iteration = 1                       # the centers held are C_i, i = iteration
        self.blocks = [[] for _ in range(self.k)]   # B_l^j for l = 1 .. iteration-1
        self.alphas = [[] for _ in range(self.k)]   # alpha_l^j for the same l
        self._rep_cache: dict = {}

    # ---------------------------------------------------------------- centers
    def window_start(self, j: int) -> int:
        """min Q_{i-1}^j for the centers C_i held now (1 if nothing is truncated)."""
        last = self.iteration - 1
        if self.tau is None or last == 0:
            return 1
        total = 0
        for ell in range(last, 0, -1):
            total += len(self.blocks[j][ell - 1])
            if total >= self.tau:
                return ell
        return 1

    def center(self, j: int, truncated: bool = True) -> CenterRep:
        """Support rows and weights of center j as held now (C_i or its truncation)."""
        key = (self.iteration, j, truncated)
        if key in self._rep_cache:
            return self._rep_cache[key]
        last = self.iteration - 1
        alphas = np.asarray(self.alphas[j], dtype=np.float64)
        # decay[l-1] = prod_{z=l+1..last} (1 - alpha_z); decay of C_1 is prod over all z.
        one_minus = 1.0 - alphas
        decay = np.ones(last, dtype=np.float64)
        for ell in range(last - 1, 0, -1):
            decay[ell - 1] = decay[ell] * one_minus[ell]
        c1_weight = float(np.prod(one_minus)) if last > 0 else 1.0
        m = self.window_start(j) if truncated else 1
        idx, w, blocks = [], [], []
        c1_kept = m == 1
        if c1_kept:
            idx.append(np.array([self.init_idx[j]], dtype=np.int64))
            w.append(np.array([c1_weight]))
            blocks.append((0, 1))
        for ell in range(m, last + 1):
            rows = self.blocks[j][ell - 1]
            if len(rows) == 0:
                continue
            coef = alphas[ell - 1] * decay[ell - 1] / len(rows)
            idx.append(np.asarray(rows, dtype=np.int64))
            w.append(np.full(len(rows), coef))
            blocks.append((ell, len(rows)))
        rep = CenterRep(idx=np.concatenate(idx) if idx else np.zeros(0, np.int64),
                        w=np.concatenate(w) if w else np.zeros(0),
                        blocks=blocks, c1_kept=c1_kept, window_start=m)
        self._rep_cache[key] = rep
        return rep

    def center_norm(self, j: int, truncated: bool = True) -> float:
        """||C^j||^2 = sum_{s,t} w_s w_t K(y_s, y_t), computed directly."""
        key = ("norm", self.iteration, j, truncated)
        if key not in self._rep_cache:
            rep = self.center(j, truncated)
            Y = self.X[rep.idx]
            self._rep_cache[key] = float(rep.w @ kernel_matrix(Y, Y, self.kernel) @ rep.w)
        return self._rep_cache[key]

    def center_norms(self, truncated: bool = True) -> np.ndarray:
        return np.array([self.center_norm(j, truncated) for j in range(self.k)])

    def truncation_error(self, j: int) -> float:
        """||C_hat^j - C^j||^2 for the centers held now.

        The untruncated center minus the truncated one is the C_1 term plus the
        blocks older than the window, all with their untruncated weights. This
        squared norm is computed directly from that difference.
        """
        full = self.center(j, truncated=False)
        trunc = self.center(j, truncated=True)
        ndrop = len(full.idx) - len(trunc.idx)
        if ndrop == 0:
            return 0.0
        Y = self.X[full.idx[:ndrop]]
        w = full.w[:ndrop]
        return float(w @ kernel_matrix(Y, Y, self.kernel) @ w)

    # -------------------------------------------------------------- distances
    def distances(self, Q, truncated: bool = True) -> np.ndarray:
        """Delta(q, C^j) for every row q of Q (points given by value), shape (m, k)."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        if Q.ndim == 1:
            Q = Q[None, :]
        kqq = kernel_diag(Q, self.kernel)
        out = np.empty((Q.shape[0], self.k), dtype=np.float64)
        for j in range(self.k):
            rep = self.center(j, truncated)
            cross = kernel_wsum(Q, self.X[rep.idx], rep.w, self.kernel)
            out[:, j] = kqq - 2.0 * cross + self.center_norm(j, truncated)
        return out

    def objective(self, Q=None) -> float:
        """f_A(C) = (1/|A|) sum_a min_j Delta(a, C^j); A = X when Q is None."""
        Q = self.X if Q is None else Q
        return float(np.mean(np.min(self.distances(Q), axis=1)))

    # -------------------------------------------------------------- iteration
    def cumulative_counts(self) -> np.ndarray:
        """N^j: points assigned to center j over all iterations so far."""
        return np.array([sum(len(B) for B in self.blocks[j]) for j in range(self.k)], dtype=np.int64)

    def learning_rate(self, counts: np.ndarray) -> np.ndarray:
        """alpha_i^j for this iteration's counts b_i^j (0 for an empty cluster).

        beta:    sqrt(b_i^j / b) (Sec. 4.1);
        const:   eta;
        sklearn: b_i^j / N^j with N^j the cumulative count including this
                 batch, the running-mean rate of mini-batch k-means as
                 scikit-learn implements it (the "sklearn" learning rate the
                 experiments of Sec. 6 compare with).
        """
        counts = np.asarray(counts, dtype=np.float64)
        if self.lr == "beta":
            return np.sqrt(counts / self.b)
        if self.lr == "sklearn":
            total = self.cumulative_counts() + counts
            return np.where(counts > 0, counts / np.where(total > 0, total, 1.0), 0.0)
        return np.where(counts > 0, float(self.eta), 0.0)

    def step(self, batch, forced_assign=None) -> StepRecord:
        """One iteration of Algorithm 2 on the batch ``batch`` (data indices).

        ``forced_assign`` replaces the argmin (teacher forcing in tests); the
        distances are still computed and returned.
        """
        batch = np.asarray(batch, dtype=np.int64)
        if batch.shape != (self.b,):
            raise ValueError(f"batch of {self.b} indices expected")
        if batch.min(initial=0) < 0 or batch.max(initial=0) >= self.n:
            raise ValueError("batch index out of range")
        cn_before = self.center_norms()
        dist = self.distances(self.X[batch])
        order = np.sort(dist, axis=1)
        gap = order[:, 1] - order[:, 0] if self.k > 1 else np.full(self.b, np.inf)
        assign = np.argmin(dist, axis=1) if forced_assign is None else \
            np.asarray(forced_assign, dtype=np.int64)
        counts = np.bincount(assign, minlength=self.k).astype(np.int64)
        alpha = self.learning_rate(counts)
        fB = float(np.mean(dist[np.arange(self.b), np.argmin(dist, axis=1)]))
        for j in range(self.k):
            self.blocks[j].append(batch[assign == j])
            self.alphas[j].append(float(alpha[j]))
        it = self.iteration
        self.iteration += 1
        self._rep_cache.clear()
        return StepRecord(iteration=it, batch=batch, dist=dist, assign=assign, gap=gap,
                          counts=counts, alpha=alpha, batch_objective=fB,
                          cnorm_before=cn_before, cnorm_after=self.center_norms())

    # ------------------------------------------------------------------ state
    def state(self) -> dict:
        """The held centers in the window layout (support rows, blocks, norms)."""
        reps = [self.center(j) for j in range(self.k)]
        return {
            "iteration": self.iteration,
            "rows_per_center": np.array([len(r.idx) for r in reps], dtype=np.int64),
            "row_idx": np.concatenate([r.idx for r in reps]) if reps else np.zeros(0, np.int64),
            "row_w": np.concatenate([r.w for r in reps]) if reps else np.zeros(0),
            "blocks_per_center": np.array([len(r.blocks) for r in reps], dtype=np.int64),
            "block_iter": np.array([bk[0] for r in reps for bk in r.blocks], dtype=np.int64),
            "block_count": np.array([bk[1] for r in reps for bk in r.blocks], dtype=np.int64),
            "c1_kept": np.array([r.c1_kept for r in reps], dtype=bool),
            "cnorm": self.center_norms(),
            "cum_counts": self.cumulative_counts(),
        }
