"""Shared test helpers: parity comparison against the oracle."""
import os

import numpy as np

TOL = 1e-12   # per-coefficient bound: |gpu - oracle| <= TOL * sum_pairs |term|


def parity_ratio(got, ref, S):
    """max over entries of |got - ref| / S (entries with S == 0 must match exactly)."""
    got, ref, S = (np.asarray(a, dtype=np.float64) for a in (got, ref, S))
    err = np.abs(got - ref)
    zero = S == 0
    if np.any(err[zero] != 0):
        return np.inf
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(zero, 0.0, err / np.where(zero, 1.0, S))
    return float(np.max(r)) if r.size else 0.0


def assert_parity(got, ref, S, tol=TOL, what=""):
    r = parity_ratio(got, ref, S)
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
