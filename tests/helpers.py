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


# stored components: 0; x y z; xx xy xz yy yz zz; xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
_E20 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
        (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1),
        (0, 1, 2), (0, 0, 3)]
_C20 = {e: c for c, e in enumerate(_E20)}


def _k(*idx):
    e = [0, 0, 0]
    for a in idx:
        e[a] += 1
    return _C20[tuple(e)]


def expansion_forces(M, L, Lc=None):
    """[k, 3] forces on k cells with moments M [k, 20] in fields L [k, 20]:
    F_i = -(M0 L_i + sum_j M_j L_ij + 1/2 sum_jk M_jk L_ijk) - M0 Lc_i."""
    F = np.zeros((M.shape[0], 3))
    for i in range(3):
        f = M[:, 0] * L[:, _k(i)]
        for j in range(3):
            f = f + M[:, _k(j)] * L[:, _k(i, j)]
            for l in range(3):
                f = f + 0.5 * M[:, _k(j, l)] * L[:, _k(i, j, l)]
        if Lc is not None:
            f = f + M[:, 0] * Lc[:, i]
        F[:, i] = -f
    return F


def spin_torques(M, L):
    """[k, 3] torques of the local fields on the cells' mass distributions
    about their centres: tau_i = -eps_ijk sum_I L[k + I] M[j + I] / I!."""
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    tau = np.zeros((M.shape[0], 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                if eps[i, j, k] == 0:
                    continue
                acc = L[:, _k(k)] * M[:, _k(j)]
                for a in range(3):
                    acc = acc + L[:, _k(k, a)] * M[:, _k(j, a)]
                    for b in range(3):
                        acc = acc + 0.5 * L[:, _k(k, a, b)] * M[:, _k(j, a, b)]
                tau[:, i] -= eps[i, j, k] * acc
    return tau


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    """Rows of a fixture under tests/golden/ as a float64 array (``#`` lines
    are the header: workload, recipe, columns)."""
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", dtype=np.float64, ndmin=2)


def load_golden_constants(name):
    """``name value`` rows of a fixture as a dict of floats."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, val = line.split()
                out[key] = float(val)
    return out


def golden_forward_columns(rows):
    """(targets [k, 2], L, S [k, 20], Lc, Sc [k, 3]) of forward_small_adaptive.txt."""
    return (rows[:, :2].astype(np.int32), rows[:, 2:22], rows[:, 22:42], rows[:, 42:45], rows[:, 45:48])


def golden_adjoint_columns(rows):
    """(cells [k, 2], Mbar, SM [k, 20], mbar, Sm [k]) of adjoint_small_adaptive.txt."""
    return (rows[:, :2].astype(np.int32), rows[:, 2:22], rows[:, 22:42], rows[:, 42], rows[:, 43])


def load_golden_script():
    """tests/golden/make_golden.py as a module (its tree and input recipe)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod
