"""Test infrastructure: match the CUDA library's cells to the oracle's.

Both sides number columns by their own mesh generators; cells are matched by
the flat-triangle centroid of their column (unique to ~1e-9) and the layer.
"""
import numpy as np
from scipy.spatial import cKDTree


def column_permutation(centroids_gpu, centroids_oracle):
    """perm[g] = oracle column of GPU column g."""
    tree = cKDTree(centroids_oracle)
    dist, perm = tree.query(centroids_gpu, k=1)
    assert np.all(dist < 1e-9), f"unmatched columns (max distance {dist.max():.3e})"
    assert len(np.unique(perm)) == len(perm), "column matching is not a bijection"
    return perm


def cell_permutation(col_perm, nlayers):
    """Index array idx with v_gpu = v_oracle[idx] (COLUMN layout on both)."""
    return (np.asarray(col_perm)[:, None] * nlayers + np.arange(nlayers)[None, :]).reshape(-1)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
