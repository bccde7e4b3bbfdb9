"""Helpers shared by the GPU parity tests (comparison rules, not arithmetic of
the method)."""
import numpy as np


def knn_mismatches(X64, idx_gpu, idx_ref, d_ref, rows=None, tie_rel=1e-6):
    """Rows whose GPU neighbour list differs from the FP64 brute force in a way
    the tie rule does not excuse.  The GPU list must hold valid neighbours of
    the query (computed here in FP64), sorted by distance, and at every
    position its distance must agree with the oracle's within ``tie_rel``
    relative (positions may swap only between near-equal distances)."""
    rows = np.arange(idx_gpu.shape[0]) if rows is None else np.asarray(rows)
    bad = []
    for r_i, q in enumerate(rows):
        g = idx_gpu[r_i]
        if np.array_equal(g, idx_ref[r_i]):
            continue
        if len(set(g.tolist())) != g.size or np.any(g < 0) or np.any(g >= X64.shape[0]):
            bad.append(int(q))
            continue
        dg = ((X64[g] - X64[q][None, :]) ** 2).sum(1)
        dr = d_ref[r_i]
        scale = np.maximum(np.abs(dr), 1e-300)
        if np.any(np.abs(dg - dr) > tie_rel * scale):
            bad.append(int(q))
    return bad


def rel_err(got, ref, floor=0.0):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), floor)
