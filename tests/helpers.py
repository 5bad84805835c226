"""Shared test helpers: parity comparison against the oracle."""
import os

import numpy as np

TOL = 1e-12   # per-coefficient bound: |gpu - oracle| <= TOL * sum_pairs |term|


RANK_BLOCKS = [slice(0, 1), slice(1, 4), slice(4, 10), slice(10, 20)]


def rank_block_sums(S, axis=1):
    """S summed over the components of the same order (0 | 1-3 | 4-9 | 10-19;
    a 3-component axis is one block).  The kernels derive the z-z trace
    components of each order from the others (the derivative tensors are
    harmonic), so the rounding error of a coefficient is bounded by the
    magnitude sums of its order block, not of its own terms alone."""
    S = np.asarray(S, dtype=np.float64)
    blocks = RANK_BLOCKS if S.shape[axis] == 20 else [slice(0, S.shape[axis])]
    out = np.empty_like(S)
    for sl in blocks:
        idx = [slice(None)] * S.ndim
        idx[axis] = sl
        out[tuple(idx)] = S[tuple(idx)].sum(axis=axis, keepdims=True)
    return out


def parity_ratio(got, ref, S, block_axis=None):
    """max over entries of |got - ref| / S (entries with S == 0 must match
    exactly); with ``block_axis`` S is summed over each order block first."""
    got, ref, S = (np.asarray(a, dtype=np.float64) for a in (got, ref, S))
    if block_axis is not None:
        S = rank_block_sums(S, block_axis)
    err = np.abs(got - ref)
    zero = S == 0
    if np.any(err[zero] != 0):
        return np.inf
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(zero, 0.0, err / np.where(zero, 1.0, S))
    return float(np.max(r)) if r.size else 0.0


def assert_parity(got, ref, S, tol=TOL, what="", block_axis=None):
    r = parity_ratio(got, ref, S, block_axis)
    assert r <= tol, f"{what}: max |gpu - oracle| / S = {r:.3e} > {tol:.0e}"
    return r


def oracle_threads(orc):
    orc.set_threads(max(1, os.cpu_count() or 1))


def sample_targets(tree, count, seed, levels=None):
    """[count, 2] (node, cell) pairs spread over nodes (optionally some levels)."""
    rng = np.random.default_rng(seed)
    nodes = np.arange(tree.n)
    if levels is not None:
        nodes = nodes[np.isin(tree.level, levels)]
    pick = rng.choice(nodes, size=count, replace=True)
    cells = rng.integers(0, 512, size=count)
    return np.stack([pick, cells], axis=1).astype(np.int32)
