"""Seeded synthetic inputs for mini-batch kernel k-means workloads.

This module holds data generators and workload recipes only. It contains none
of the clustering method's arithmetic. The CUDA path, the oracle tests and the
benchmark all draw their inputs from it.

The paper's datasets (MNIST, PenDigits, Letters, HAR; Sec. 6) are not
available. These mixtures stand in for their shapes:

* ``isotropic_mixture``: c components with means ~ N(0, mean_var * I) and unit
  variance, equal sizes, seeded shuffle (PenDigits/Letters scale, d = 16).
* ``image_like``: n x 784 values in [0, 1], about 80% exact zeros. Each of 10
  latent classes has a fixed random mask over 25% of the dimensions. A point
  keeps each masked dimension with p = 0.8, with value ~ Beta(2, 2). This is
  MNIST's shape, not its content.
* ``anisotropic_mixture``: c components with covariance Q diag(lam) Q^T, where
  Q is Haar-orthogonal and lam is log-uniform in [1, cond] with cond ~ U[1, 100],
  rescaled to mean 1.

``median_sigma`` is the median heuristic for the kernel bandwidth: the median
pairwise Euclidean distance over a seeded subsample, in FP64. The Gaussian
kernel then uses kappa = 2 sigma^2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def isotropic_mixture(n: int, d: int, c: int, seed: int, mean_var: float = 4.0):
    """(X float32 n x d, labels int64): equal-size isotropic unit-variance mixture."""
    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, np.sqrt(mean_var), size=(c, d))
    labels = np.arange(n) % c
    rng.shuffle(labels)
    X = means[labels] + rng.normal(size=(n, d))
    return X.astype(np.float32), labels.astype(np.int64)


def image_like(n: int, seed: int, d: int = 784, classes: int = 10, mask_frac: float = 0.25,
               keep_p: float = 0.8):
    """(X float32 n x d in [0,1] with ~80% zeros, labels): class-masked Beta(2,2) values."""
    rng = np.random.default_rng(seed)
    masks = np.zeros((classes, d), dtype=bool)
    m = int(round(mask_frac * d))
    for c in range(classes):
        masks[c, rng.choice(d, size=m, replace=False)] = True
    labels = np.arange(n) % classes
    rng.shuffle(labels)
    X = np.zeros((n, d), dtype=np.float32)
    chunk = 8192
    for s in range(0, n, chunk):
        lab = labels[s:s + chunk]
        keep = masks[lab] & (rng.random((len(lab), d)) < keep_p)
        vals = rng.beta(2.0, 2.0, size=(len(lab), d)).astype(np.float32)
        X[s:s + chunk] = np.where(keep, vals, np.float32(0.0))
    return X, labels.astype(np.int64)


def anisotropic_mixture(n: int, d: int, c: int, seed: int, mean_var: float = 4.0,
                        max_cond: float = 100.0):
    """(X float32 n x d, labels): mixture with random covariances of condition <= max_cond."""
    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, np.sqrt(mean_var), size=(c, d))
    factors = []
    for _ in range(c):
        q, r = np.linalg.qr(rng.normal(size=(d, d)))
        q = q * np.sign(np.diag(r))[None, :]
        cond = rng.uniform(1.0, max_cond)
        lam = np.exp(rng.uniform(0.0, np.log(cond), size=d))
        lam = lam / lam.mean()
        factors.append(q * np.sqrt(lam)[None, :])
    labels = np.arange(n) % c
    rng.shuffle(labels)
    X = np.empty((n, d), dtype=np.float32)
    chunk = 65536
    for s in range(0, n, chunk):
        lab = labels[s:s + chunk]
        z = rng.normal(size=(len(lab), d))
        out = np.empty((len(lab), d))
        for comp in np.unique(lab):
            sel = lab == comp
            out[sel] = z[sel] @ factors[comp].T + means[comp]
        X[s:s + chunk] = out.astype(np.float32)
    return X, labels.astype(np.int64)


def median_sigma(X, seed: int, sample: int = 2000) -> float:
    """Median pairwise Euclidean distance over a seeded subsample of min(n, sample) rows.

    FP64. With an even number of pairs the median is the mean of the two middle values.
    """
    X = np.asarray(X)
    rng = np.random.default_rng(seed)
    m = min(X.shape[0], sample)
    rows = rng.choice(X.shape[0], size=m, replace=False)
    S = X[rows].astype(np.float64)
    sq = np.einsum("ij,ij->i", S, S)
    G = sq[:, None] + sq[None, :] - 2.0 * (S @ S.T)
    iu = np.triu_indices(m, k=1)
    return float(np.median(np.sqrt(np.maximum(G[iu], 0.0))))


def init_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct data indices, uniform without replacement."""
    return np.random.default_rng(seed).choice(n, size=k, replace=False).astype(np.int64)


def batch_stream(n: int, b: int, iters: int, seed: int) -> np.ndarray:
    """(iters, b) batch indices, uniform with replacement."""
    return np.random.default_rng(seed).integers(0, n, size=(iters, b), dtype=np.int64)


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload (shape, generator and method parameters)."""

    name: str
    n: int
    d: int
    k: int
    b: int
    tau: int
    iters: int
    kind: str            # generator: "isotropic", "image", "anisotropic"
    components: int
    data_seed: int = 12345

    def make(self):
        if self.kind == "isotropic":
            return isotropic_mixture(self.n, self.d, self.components, self.data_seed)
        if self.kind == "image":
            return image_like(self.n, self.data_seed, d=self.d, classes=self.components)
        if self.kind == "anisotropic":
            return anisotropic_mixture(self.n, self.d, self.components, self.data_seed)
        raise ValueError(self.kind)


WORKLOADS = {
    # PenDigits/Letters-scale mixture: 10 isotropic Gaussians, 200 points each.
    "small": Workload("small", n=2000, d=16, k=10, b=256, tau=200, iters=50,
                      kind="isotropic", components=10),
    # MNIST-shaped: 70000 x 784, ~80% zeros, 10 latent classes.
    "image": Workload("image", n=70000, d=784, k=10, b=1024, tau=200, iters=200,
                      kind="image", components=10),
    # 1e6 x 128 anisotropic 100-component mixture.
    "precision": Workload("precision", n=1_000_000, d=128, k=100, b=4096, tau=200, iters=200,
                          kind="anisotropic", components=100),
    # 2e5 x 64, 50 isotropic components.
    "differentiation": Workload("differentiation", n=200_000, d=64, k=50, b=2048, tau=200,
                                iters=200, kind="isotropic", components=50),
}


@dataclass(frozen=True)
class RunSpec:
    """One independent clustering run of a batched sweep."""

    n: int
    d: int
    k: int
    b: int
    data_seed: int

    def make(self):
        """Isotropic mixture with k_true = k components."""
        return isotropic_mixture(self.n, self.d, self.k, self.data_seed)


def batching_specs(count: int = 64, seed: int = 777, n_range=(5000, 200000), dims=(16, 64, 256),
                   k_range=(5, 200), batches=(256, 512, 1024, 2048), n_scale: float = 1.0):
    """The batched-sweep workload: ``count`` runs with n uniform in n_range
    (times n_scale), d from dims, k uniform in k_range, b from batches, all
    drawn from one seeded generator."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        d = int(rng.choice(dims))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        b = int(rng.choice(batches))
        out.append(RunSpec(max(int(n * n_scale), k), d, k, b, data_seed=seed * 1000 + i))
    return out
