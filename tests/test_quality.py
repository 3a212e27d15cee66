"""External clustering indices (ARI, NMI) against scikit-learn's, and their
closed-form special cases."""
import numpy as np
import pytest

from paper_2410_05902_gb300.quality import adjusted_rand, normalized_mutual_info


def test_special_cases():
    a = np.array([0, 0, 1, 1, 2, 2])
    assert adjusted_rand(a, a) == 1.0
    assert normalized_mutual_info(a, a) == pytest.approx(1.0)
    assert adjusted_rand(a, a[::-1] * 7 + 3) == 1.0          # relabelling does not matter
    assert normalized_mutual_info(a, np.zeros(6)) == 0.0


@pytest.mark.parametrize("seed", range(5))
def test_against_scikit_learn(seed):
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 5, size=300)
    b = np.where(rng.random(300) < 0.6, a, rng.integers(0, 7, size=300))
    assert adjusted_rand(a, b) == pytest.approx(metrics.adjusted_rand_score(a, b), abs=1e-12)
    assert normalized_mutual_info(a, b) == pytest.approx(metrics.normalized_mutual_info_score(a, b), abs=1e-12)
