"""Grouping of cellwise masks into representative spaces (oracle; test infrastructure).  Sec. 3.2.

 * graded distance d(Ma, Mb) = sum_b |kappa_a(b) - kappa_b(b)| / (3 N_b)  (Eq. after the kappa
   definition);
 * deduplicate, order unique patterns by descending frequency, seed the first cluster with
   the most frequent one, assign every next pattern to the nearest existing centre when the
   distance is <= tau_clust, otherwise open a new cluster;
 * enclosing mask kappa_rep(b) = min over members (the kappa_rep equation).

Readings: the centre of a cluster is its seeding pattern and does not move; equal
frequencies are ordered by the lexicographic order of the kappa row; equal distances go to
the lower cluster index.
"""
from __future__ import annotations

import numpy as np


def graded_distance(ka, kb):
    """Graded distance between two masks, Sec. 3.2 (the equation after the kappa definition)."""
    ka = np.asarray(ka).ravel()
    kb = np.asarray(kb).ravel()
    return float(np.sum(np.abs(ka.astype(np.int64) - kb.astype(np.int64)))) / (3.0 * ka.size)


def cluster(kappas, tau):
    """kappas: [ncell, Nb] integer array.  Returns (labels [ncell], reps [ncluster, Nb]).
    Sec. 3.2, Eq. kappa_rep."""
    K = np.asarray(kappas, dtype=np.int64)
    ncell = K.shape[0]
    uniq, inv, counts = np.unique(K, axis=0, return_inverse=True, return_counts=True)
    inv = np.asarray(inv).ravel()
    # descending frequency, ties by lexicographic order of the row (np.unique sorts rows)
    order = sorted(range(len(uniq)), key=lambda u: (-counts[u], u))
    centres = []
    ulabel = np.empty(len(uniq), dtype=np.int64)
    for u in order:
        if not centres:
            centres.append(u)
            ulabel[u] = 0
            continue
        d = [graded_distance(uniq[u], uniq[c]) for c in centres]
        j = int(np.argmin(d))
        if d[j] <= tau:
            ulabel[u] = j
        else:
            centres.append(u)
            ulabel[u] = len(centres) - 1
    labels = ulabel[inv]
    reps = np.stack([np.min(K[labels == c], axis=0) for c in range(len(centres))])
    assert labels.shape[0] == ncell
    return labels, reps
