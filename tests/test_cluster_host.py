"""Grouping of cell masks (Sec. 3.2) through the C ABI's host-only mlvs_cluster, against the
oracle's cluster().  Integer work: labels and representative masks must agree exactly."""
import numpy as np
import pytest

from oracle import cluster as ocl
from paper_2609_35258_b300 import mlvs as M


def _masks(seed, nrow, nb, nproto, flip):
    """Rows drawn from a few prototype masks (values 0..3) with a fraction `flip` of blocks
    changed, so that the rows form near-duplicate families and exact duplicates."""
    rng = np.random.default_rng(seed)
    proto = rng.integers(0, 4, size=(nproto, nb))
    rows = proto[rng.integers(0, nproto, size=nrow)].copy()
    mask = rng.random(rows.shape) < flip
    rows[mask] = rng.integers(0, 4, size=int(mask.sum()))
    return rows.astype(np.uint8)


@pytest.mark.parametrize("seed,nrow,nb,nproto,flip,tau", [
    (1, 200, 49, 3, 0.02, 0.05),
    (2, 500, 169, 6, 0.05, 0.07),
    (3, 300, 25, 2, 0.2, 0.035),
    (4, 64, 9, 4, 0.3, 0.0),      # tau = 0: only identical masks share a cluster
    (5, 100, 16, 3, 0.1, 1.0),    # tau = 1: one cluster
])
def test_cluster_matches_oracle(seed, nrow, nb, nproto, flip, tau):
    K = _masks(seed, nrow, nb, nproto, flip)
    lab, reps = M.mlvs_cluster(K, tau)
    olab, oreps = ocl.cluster(K, tau)
    np.testing.assert_array_equal(lab, olab)
    np.testing.assert_array_equal(reps, oreps)


def test_cluster_ties_and_threshold_edge():
    # two masks with equal frequency: the lexicographically smaller one seeds cluster 0;
    # a third at distance exactly tau from the first joins it (d <= tau)
    nb = 6
    a = np.array([0, 0, 1, 1, 2, 2], dtype=np.uint8)
    b = np.array([0, 0, 1, 1, 2, 3], dtype=np.uint8)   # d(a, b) = 1/18
    c = np.array([3, 3, 3, 3, 3, 3], dtype=np.uint8)
    K = np.stack([b, a, c, b, a, c, c])
    tau = 1.0 / 18.0
    lab, reps = M.mlvs_cluster(K, tau)
    olab, oreps = ocl.cluster(K, tau)
    np.testing.assert_array_equal(lab, olab)
    np.testing.assert_array_equal(reps, oreps)
    # c is the most frequent: cluster 0; a before b on the tie; b joins a at d == tau
    assert lab[2] == 0 and lab[1] == lab[0] == 1
    np.testing.assert_array_equal(reps[1], np.minimum(a, b))


def test_cluster_empty_and_single():
    lab, reps = M.mlvs_cluster(np.zeros((0, 4), dtype=np.uint8), 0.1)
    assert lab.shape == (0,) and reps.shape == (0, 4)
    lab, reps = M.mlvs_cluster(np.full((1, 4), 2, dtype=np.uint8), 0.1)
    assert list(lab) == [0] and reps.tolist() == [[2, 2, 2, 2]]
