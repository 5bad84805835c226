"""Shared test helpers: parity comparison against the oracle."""
import os

import numpy as np

TOL = 1e-12   # per-coefficient bound: |gpu - oracle| <= TOL * sum_pairs |term|

# The oracle's S treats every derivative value as one exact number, but a
# derivative is itself a sum of terms (a pairing sum of g_k(r) times
# coordinates), and any evaluation of it -- the oracle's pairing sum, the
# library's table -- rounds by a few units of those terms' magnitude sum.
# Where the terms cancel exactly (d^xyy G at (-6,-3,0), d^yyz G at (0,2,4))
# that rounding is all that is left, and S of a coefficient fed by such
# pairs alone is zero or rounding noise.  The oracle's SD counts each
# contraction term with its derivative's terms expanded; the bar allows
# DERIV_TOL (45 units of roundoff) of SD on top of TOL of S.
DERIV_TOL = 1e-14


def eff(S, SD):
    """The magnitude sum the bar divides by, in units of TOL: S + SD *
    DERIV_TOL / TOL."""
    return np.asarray(S, dtype=np.float64) + (DERIV_TOL / TOL) * np.asarray(SD, dtype=np.float64)


def fwd_scale(r, lc=False):
    """eff() of a forward pass result of the oracle (its L, or with ``lc`` its Lc)."""
    return eff(r["Sc"], r["SDc"]) if lc else eff(r["S"], r["SD"])


def adjoint_with_scale(orc, *args, **kw):
    """The oracle's transposed sum and the eff() of its magnitude sums."""
    out, S, SD = orc.pass_adjoint(*args, with_s=True, with_sd=True, **kw)
    return out, eff(S, SD)


# The kernels accumulate 16 of the 20 coefficients of an expansion and derive
# the other four from them, because every derivative tensor of G = -1/r is
# harmonic (a zero trace over any index pair).  A derived coefficient is a
# different formula, not a different summation order, so its rounding is
# bounded by the magnitude sums of the coefficients it is computed from, not
# by its own.  For each derived component (storage index): the (source index,
# weight) pairs of its formula.
#   Taylor coefficients L:      zz = -(xx + yy), xzz = -(xxx + xyy),
#                               yzz = -(xxy + yyy), zzz = -(xxz + yyz)
#   moment adjoints Mbar (the gradient with respect to the raw moments, whose
#   unique components carry multiplicities 1, 3, 3, 6):
#                               zz = -(xx + yy), xzz = -(3 xxx + xyy),
#                               yzz = -(xxy + 3 yyy), zzz = -(xxz + yyz) / 3
DERIVED = {
    "L": {9: ((4, 1.0), (7, 1.0)), 15: ((10, 1.0), (13, 1.0)),
          18: ((11, 1.0), (16, 1.0)), 19: ((12, 1.0), (17, 1.0))},
    "Mbar": {9: ((4, 1.0), (7, 1.0)), 15: ((10, 3.0), (13, 1.0)),
             18: ((11, 1.0), (16, 3.0)), 19: ((12, 1.0 / 3.0), (17, 1.0 / 3.0))},
}


def coefficient_scale(S, kind=None, axis=1):
    """The per-coefficient denominator of the parity bar: the oracle's own sum
    of |terms| S for every accumulated coefficient; for a derived one (kind
    "L" or "Mbar", 20 components along ``axis``) the weighted S of the
    coefficients its formula reads.  kind None (Lc, mbar, masses): S itself."""
    S = np.asarray(S, dtype=np.float64)
    if kind is None:
        return S
    assert S.shape[axis] == 20, (kind, S.shape)
    out = S.copy()
    Sm = np.moveaxis(S, axis, 0)
    om = np.moveaxis(out, axis, 0)
    for q, srcs in DERIVED[kind].items():
        om[q] = sum(w * Sm[k] for k, w in srcs)
    return out


def parity_ratio(got, ref, S, kind=None, axis=1):
    """max over entries of |got - ref| / scale, scale the per-coefficient
    denominator of ``coefficient_scale`` (entries with scale 0 must match
    exactly)."""
    got, ref = (np.asarray(a, dtype=np.float64) for a in (got, ref))
    S = coefficient_scale(S, kind, axis)
    err = np.abs(got - ref)
    zero = S == 0
    if np.any(err[zero] != 0):
        return np.inf
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(zero, 0.0, err / np.where(zero, 1.0, S))
    return float(np.max(r)) if r.size else 0.0


def own_s_ratio(got, ref, S):
    """The same ratio with every coefficient's own S (derived ones included),
    reported beside the bar, not asserted."""
    return parity_ratio(got, ref, S, None)


def assert_parity(got, ref, S, tol=TOL, what="", kind=None, axis=1):
    r = parity_ratio(got, ref, S, kind, axis)
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


def oracle_full_solve_at(orc, tree, M, m, cells, kind="L"):
    """The oracle's full multilevel solve at the given leaf cells only: each
    cell's own passes plus its ancestors' passes, shifted down level by level
    (the local-expansion shift between geometric cell centres); S follows the
    same chain with |d|, starting from each pass's per-coefficient scale
    (``coefficient_scale`` of kind "L": the passes derive four coefficients,
    the shift then moves all 20; kind None chains the oracle's own S).
    Returns (L, S) [k, 20]; compare with kind None."""
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
    S12 = fwd_scale(r1) + fwd_scale(r2) if kind is not None else r1["S"] + r2["S"]
    Sp = {k: coefficient_scale(S12[i], kind, axis=0) for i, k in enumerate(need)}
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


def full_solve_scale(orc, tree, M, m, centres=None, kind="L"):
    """[n, 20, 512] per-coefficient scale of the full multilevel solve at
    every cell: each cell's pass scale (the oracle's S of both passes through
    ``coefficient_scale`` of kind "L") plus its parent cell's full scale
    shifted down by |d|, d the offset between the two expansion centres
    (geometric, or ``centres`` [n, 3, 512]); kind None chains the oracle's
    own S.  Compare with kind None."""
    r1 = orc.run_pass_grid(tree, "multipole", M=M, centres=centres)
    r2 = orc.run_pass_grid(tree, "monopole", m=m, centres=centres)
    S = coefficient_scale(fwd_scale(r1) + fwd_scale(r2) if kind is not None else r1["S"] + r2["S"], kind, axis=1)
    idx = tree.index()
    cell = np.arange(512)
    local = np.stack([cell % 8, (cell // 8) % 8, cell // 64], 1)
    for node in np.argsort(tree.level, kind="stable"):
        lv = int(tree.level[node])
        if lv == 0:
            continue
        g = 8 * tree.coord[node] + local
        gp = g >> 1
        parent = idx[(lv - 1, *(tree.coord[node] // 2))]
        pcell = (gp % 8) @ np.array([1, 8, 64])
        if centres is None:
            h = tree.h0 / 2 ** lv
            d = (g + 0.5) * h - (gp + 0.5) * (2 * h)
        else:
            d = centres[node].T - centres[parent][:, pcell].T
        for c in range(512):
            S[node, :, c] += orc.l2l(S[parent, :, pcell[c]], np.abs(d[c]))
    return S


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
