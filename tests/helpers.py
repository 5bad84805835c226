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


def oracle_full_solve_at(orc, tree, M, m, cells):
    """The oracle's full multilevel solve at the given leaf cells only: each
    cell's own passes plus its ancestors' passes, shifted down level by level
    (the local-expansion shift between geometric cell centres); S follows the
    same chain with |d|.  Returns (L, S) [k, 20]."""
    idx = tree.index()
    chains, need = [], {}
    for node, cell in cells:
        lv = int(tree.level[node])
        g = 8 * tree.coord[node] + np.array([cell % 8, (cell // 8) % 8, cell // 64])
        chain = []
        for l in range(lv + 1):
            gl = g >> (lv - l)
            nd = idx[(l, *(gl // 8))]
            cc = int(gl[0] % 8 + 8 * (gl[1] % 8) + 64 * (gl[2] % 8))
            chain.append((nd, cc, gl, l))
            need[(nd, cc)] = None
        chains.append(chain)
    tg = np.array(list(need), dtype=np.int32)
    r1 = orc.run_pass(tree, "multipole", M=M, targets=tg)
    r2 = orc.run_pass(tree, "monopole", m=m, targets=tg)
    Lp = {k: r1["L"][i] + r2["L"][i] for i, k in enumerate(need)}
    Sp = {k: r1["S"][i] + r2["S"][i] for i, k in enumerate(need)}
    L, S = [], []
    for chain in chains:
        nd, cc, gl, l = chain[0]
        acc, sacc = Lp[(nd, cc)].copy(), Sp[(nd, cc)].copy()
        for (nd, cc, gl, l), (_, _, gp, lp) in zip(chain[1:], chain[:-1]):
            h, hp = tree.h0 / 2 ** l, tree.h0 / 2 ** lp
            d = (gl + 0.5) * h - (gp + 0.5) * hp
            acc = Lp[(nd, cc)] + orc.l2l(acc, d)
            sacc = Sp[(nd, cc)] + orc.l2l(sacc, np.abs(d))
        L.append(acc)
        S.append(sacc)
    return np.array(L), np.array(S)
