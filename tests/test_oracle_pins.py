"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each pin is chosen so that a plausible mistake (a dropped term, a wrong sign,
factorial or multiplicity, a transposed index, a missed or doubled pair)
fails at least one of them:

* Green's-function derivatives against sympy's symbolic differentiation.
* Cell moments and their M2M shift against exact polynomial integrals.
* Every term of the n + m <= 3 contraction against brute-force point
  clusters: the error of the local Taylor model must fall as the 4th power
  of the cluster and evaluation radius (a wrong order-k term leaves an error
  of order k <= 3).  The angular-momentum term must lift the order of the
  gradient and force errors from 3 to 4 the same way.
* Newton's third law over closed pair sets; harmonicity of the expansions.
* Pair coverage: a single point mass through the full multilevel solve must
  give -1/r at every other leaf cell (a missed or doubled pair would not).
* Full solve against the brute-force pairwise sum, against the closed-form
  potentials of a uniform sphere and of an n = 1 polytrope, and against the
  exact potential of piecewise-constant cells (closed-form cube integrals,
  themselves checked by cubature and the point-mass limit).
* The transposed sums against the forward passes (dot-product identity).
* Virtual descendants of a coarse leaf against explicitly refined leaves.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
import sympy

import synth

# storage order of the 20 (35) components: sorted index tuples, lexicographic
def _exps(maxrank=4):
    out = []
    for k in range(maxrank + 1):
        for t in itertools.combinations_with_replacement(range(3), k):
            out.append(tuple(t.count(a) for a in range(3)))
    return out


EXPS = _exps(4)
EXP20 = EXPS[:20]
RANK = np.array([sum(e) for e in EXPS])


def _fact(e):
    return math.factorial(e[0]) * math.factorial(e[1]) * math.factorial(e[2])


def taylor(L, delta):
    """sum over stored J of L[J] delta^J / J!  (the local expansion)."""
    return sum(L[c] * np.prod(np.power(delta, EXP20[c])) / _fact(EXP20[c]) for c in range(20))


def point_cluster_moments(mu, pos, centre):
    """Raw moments sum mu (y - X)^K of point masses (definition of a moment)."""
    d = pos - centre
    return np.array([np.sum(mu * np.prod(d ** np.array(e), axis=1)) for e in EXP20])


# ---------------------------------------------------------------------------
# derivatives of G = -1/r
# ---------------------------------------------------------------------------

def test_component_order_matches_storage_convention(orc):
    assert orc.component_exponents().tolist() == [list(e) for e in EXPS]


@pytest.mark.parametrize("R", [(1, 2, 2), (3, -4, 12), (-2, 3, 6), (1, 1, 1), (0, 0, 5), (-7, 0, 3)])
def test_D_matches_sympy(orc, R):
    x, y, z = sympy.symbols("x y z", real=True)
    G = -1 / sympy.sqrt(x ** 2 + y ** 2 + z ** 2)
    sub = {x: sympy.Integer(R[0]), y: sympy.Integer(R[1]), z: sympy.Integer(R[2])}
    got = orc.D(np.array(R, dtype=float))
    for c, e in enumerate(EXPS):
        expr = sympy.diff(G, x, e[0], y, e[1], z, e[2])
        exact = float(sympy.N(expr.subs(sub), 40))
        scale = 1.0 / np.linalg.norm(R) ** (RANK[c] + 1)
        assert abs(got[c] - exact) <= 1e-14 * max(abs(exact), scale), (R, e, got[c], exact)


@pytest.mark.parametrize("R", [(0, 2, 4), (-6, -3, 0), (3, -1, 2), (0.7, -2.5, 1.3)])
def test_D_abs_matches_sympy_term_magnitudes(orc, R):
    """The magnitude sums of the derivatives' terms (the scale SD of the
    parity bar): write G = f(u), u = x^2 + y^2 + z^2; sympy expands d^K f(u)
    into sum_j f^(j)(u) Q_j(x, y, z), whose terms for one j share a sign, so
    the magnitude sum is sum_j |f^(j)(u)| Q_j(|x|, |y|, |z|) (Q_j has
    non-negative coefficients).  Where the derivative cancels exactly, the
    magnitude sum stays of the derivative's order of size."""
    x, y, z, u = sympy.symbols("x y z u", real=True)
    f = sympy.Function("f")
    F = -u ** sympy.Rational(-1, 2)
    expr0 = f(x ** 2 + y ** 2 + z ** 2)
    Ra = [abs(sympy.nsimplify(v)) for v in R]
    u0 = sum(sympy.nsimplify(v) ** 2 for v in R)
    got = orc.D_abs(np.array(R, dtype=float))
    for c, e in enumerate(EXPS):
        d = sympy.expand(sympy.diff(expr0, x, e[0], y, e[1], z, e[2]))
        total = sympy.Integer(0)
        for j in range(RANK[c] + 1):
            fj = f(x ** 2 + y ** 2 + z ** 2) if j == 0 else sympy.Subs(sympy.Derivative(f(u), (u, j)), u,
                                                                       x ** 2 + y ** 2 + z ** 2)
            Q = sympy.expand(d.coeff(fj))
            poly = sympy.Poly(Q, x, y, z) if Q != 0 else None
            if poly is None:
                continue
            assert all(co >= 0 for co in poly.coeffs()), (e, j, Q)
            fval = sympy.diff(F, u, j).subs(u, u0)
            total += abs(fval) * poly.as_expr().subs({x: Ra[0], y: Ra[1], z: Ra[2]})
        exact = float(sympy.N(total, 40))
        assert abs(got[c] - exact) <= 1e-14 * exact, (R, e, got[c], exact)
        assert got[c] >= abs(orc.D(np.array(R, dtype=float))[c]) * (1 - 1e-15)
    if tuple(R) == (0, 2, 4):
        c = EXPS.index((0, 2, 1))
        assert orc.D(np.array(R, dtype=float))[c] == 0.0 and got[c] > 0.1 / 20 ** 2


# ---------------------------------------------------------------------------
# moments
# ---------------------------------------------------------------------------

def _axis_int(e, lo, hi):
    """exact int_lo^hi t^e dt with Fractions"""
    return (Fraction(hi) ** (e + 1) - Fraction(lo) ** (e + 1)) / (e + 1)


def test_cube_moments_exact(orc):
    tree = synth.single_subgrid(level=2, h=0.5, leaf=True)
    rho = np.full((1, 512), 1.75)
    M = orc.moments(tree, rho)
    h = Fraction(1, 2)
    for c, e in enumerate(EXP20):
        exact = Fraction(7, 4)
        for a in range(3):
            exact *= _axis_int(e[a], -h / 2, h / 2)
        assert M[0, c, 77] == pytest.approx(float(exact), rel=1e-15, abs=1e-300)


def test_m2m_matches_exact_integrals(orc):
    tree = synth.uniform_tree(1, h_leaf=1.0)     # root (h=2) + 8 leaves (h=1)
    rng = np.random.default_rng(11)
    rho = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    M = orc.moments(tree, rho)
    idx = tree.index()
    root = idx[(0, 0, 0, 0)]
    for cell in (0, 9, 200, 511):
        gp = np.array([cell % 8, (cell // 8) % 8, cell // 64])
        XP = (gp + 0.5) * 2.0
        exact = np.zeros(20)
        for b in itertools.product((0, 1), repeat=3):
            gc = 2 * gp + np.array(b)
            node = idx[(1, *(gc // 8))]
            cc = int((gc % 8) @ np.array([1, 8, 64]))
            lo = gc * 1.0 - XP
            for c, e in enumerate(EXP20):
                v = Fraction(rho[node, cc])
                for a in range(3):
                    v *= _axis_int(e[a], Fraction(lo[a]), Fraction(lo[a] + 1))
                exact[c] += float(v)
        np.testing.assert_allclose(M[root, :, cell], exact, rtol=1e-13, atol=1e-13 * exact[0])


# ---------------------------------------------------------------------------
# the contraction, term by term, against brute-force point clusters
# ---------------------------------------------------------------------------

def _single_node_tree():
    return synth.single_subgrid(level=1, h=1.0, leaf=False)   # h = 1 cells, no halo


def _cell(i, j, k):
    return i + 8 * j + 64 * k


def _order(errs, scales):
    return np.polyfit(np.log(scales), np.log(errs), 1)[0]


def _cluster(rng, k=7):
    mu = rng.uniform(0.2, 1.0, size=k)
    u = rng.standard_normal((k, 3))
    return mu, u


def test_multipole_pass_taylor_order(orc):
    """L from the multipole pass reproduces the direct potential of a random
    point cluster with error O(s^4) when the cluster radius and the
    evaluation offset both scale with s."""
    tree = _single_node_tree()
    rng = np.random.default_rng(5)
    mu, u = _cluster(rng)
    A, B = (0, 0, 0), (4, 1, 0)          # |o|^2 = 17 > 12, parents at (2,0,0): far
    XA, XB = np.array(A) + 0.5, np.array(B) + 0.5
    dirs = rng.standard_normal((6, 3))
    errs, scales = [], [0.4, 0.2, 0.1, 0.05]
    for s in scales:
        M = np.zeros((1, 20, 512))
        pos = XB + s * u
        M[0, :, _cell(*B)] = point_cluster_moments(mu, pos, XB)
        r = orc.run_pass(tree, "multipole", M=M, targets=[[0, _cell(*A)]])
        L = r["L"][0]
        e = 0.0
        for d in dirs:
            delta = s * d / np.linalg.norm(d)
            exact = -np.sum(mu / np.linalg.norm(XA + delta - pos, axis=1))
            e = max(e, abs(taylor(L, delta) - exact))
        errs.append(e)
    order = _order(errs, scales)
    assert 3.7 < order < 4.4, (errs, order)


def test_multipole_pass_exact_for_point_masses(orc):
    """With point masses (no higher moments) every L[J] is an exact derivative,
    so L[0] equals the direct sum -sum m / r to rounding."""
    tree = _single_node_tree()
    rng = np.random.default_rng(6)
    M = np.zeros((1, 20, 512))
    M[0, 0] = rng.uniform(0.5, 1.5, 512)
    A = _cell(3, 4, 2)
    r = orc.run_pass(tree, "multipole", M=M, targets=[[0, A]])
    gA = np.array([3, 4, 2])
    exact = 0.0
    n = 0
    for c in range(512):
        g = np.array([c % 8, (c // 8) % 8, c // 64])
        o = g - gA
        n2 = o @ o
        op = np.floor_divide(gA % 2 + o, 2)
        if n2 > 12 and op @ op <= 12:
            exact -= M[0, 0, c] / math.sqrt(n2)
            n += 1
    assert r["npairs"] == n
    assert r["L"][0, 0] == pytest.approx(exact, rel=1e-14)


def test_monopole_pass_taylor_order(orc):
    """Point-mass sources: the only error of the local model is the degree-3
    truncation in the evaluation offset, O(s^4)."""
    tree = synth.single_subgrid(level=1, h=1.0, leaf=True)
    rng = np.random.default_rng(7)
    m = np.zeros((1, 512))
    srcs = [(5, 1, 2), (0, 6, 6), (3, 2, 3)]   # two far, one near
    for s_ in srcs:
        m[0, _cell(*s_)] = rng.uniform(0.5, 1.5)
    A = (1, 2, 3)
    XA = np.array(A) + 0.5
    r = orc.run_pass(tree, "monopole", m=m, targets=[[0, _cell(*A)]])
    L = r["L"][0]
    dirs = rng.standard_normal((6, 3))
    errs, scales = [], [0.4, 0.2, 0.1, 0.05]
    for s in scales:
        e = 0.0
        for d in dirs:
            delta = s * d / np.linalg.norm(d)
            exact = -sum(m[0, _cell(*q)] / np.linalg.norm(XA + delta - (np.array(q) + 0.5)) for q in srcs)
            e = max(e, abs(taylor(L, delta) - exact))
        errs.append(e)
    order = _order(errs, scales)
    assert 3.7 < order < 4.4, (errs, order)


def _force(Mt, L, Lc=None):
    """F_i = -(M0 L_i + sum_j M_j L_ij + 1/2 sum_jk M_jk L_ijk) - m Lc_i,
    full index sums over the stored symmetric components."""
    comp = {e: c for c, e in enumerate(EXP20)}

    def key(*idx):
        e = [0, 0, 0]
        for a in idx:
            e[a] += 1
        return comp[tuple(e)]
    F = np.zeros(3)
    for i in range(3):
        f = Mt[0] * L[key(i)]
        for j in range(3):
            f += Mt[key(j)] * L[key(i, j)]
        for j in range(3):
            for k in range(3):
                f += 0.5 * Mt[key(j, k)] * L[key(i, j, k)]
        if Lc is not None:
            f += Mt[0] * Lc[i]
        F[i] = -f
    return F


def test_angular_term_lifts_gradient_order(orc):
    """A point-mass target and a random-cluster source: L1 alone has an O(s^3)
    gradient error (the source octupole term is truncated); L1 + Lc is O(s^4)."""
    tree = _single_node_tree()
    rng = np.random.default_rng(8)
    mu, u = _cluster(rng)
    A, B = (0, 0, 0), (4, 1, 0)
    XA, XB = np.array(A) + 0.5, np.array(B) + 0.5
    e1, e2, scales = [], [], [0.4, 0.2, 0.1, 0.05]
    for s in scales:
        M = np.zeros((1, 20, 512))
        pos = XB + s * u
        M[0, :, _cell(*B)] = point_cluster_moments(mu, pos, XB)
        M[0, 0, _cell(*A)] = 1.0          # target: unit point mass
        r = orc.run_pass(tree, "multipole", M=M, targets=[[0, _cell(*A)]])
        L, Lc = r["L"][0], r["Lc"][0]
        R = XA - pos
        exact = np.sum(mu[:, None] * R / np.linalg.norm(R, axis=1)[:, None] ** 3, axis=0)
        e1.append(np.max(np.abs(L[1:4] - exact)))
        e2.append(np.max(np.abs(L[1:4] + Lc - exact)))
    o1, o2 = _order(e1, scales), _order(e2, scales)
    assert 2.7 < o1 < 3.4, (e1, o1)
    assert 3.7 < o2 < 4.4, (e2, o2)


def test_angular_term_lifts_force_order_for_cluster_target(orc):
    """A random-cluster target and a point-mass source: the force on the target
    cluster from the expansion has an O(s^3) error without Lc, O(s^4) with it
    (this pins the -(m_B/m_A) M3_A part of the correction)."""
    tree = _single_node_tree()
    rng = np.random.default_rng(9)
    mu, u = _cluster(rng)
    A, B = (0, 0, 0), (4, 1, 0)
    XA, XB = np.array(A) + 0.5, np.array(B) + 0.5
    mB = 1.3
    e1, e2, scales = [], [], [0.4, 0.2, 0.1, 0.05]
    for s in scales:
        M = np.zeros((1, 20, 512))
        pos = XA + s * u
        MA = point_cluster_moments(mu, pos, XA)
        M[0, :, _cell(*A)] = MA
        M[0, 0, _cell(*B)] = mB
        r = orc.run_pass(tree, "multipole", M=M, targets=[[0, _cell(*A)]])
        L, Lc = r["L"][0], r["Lc"][0]
        R = pos - XB
        exact = -np.sum(mu[:, None] * mB * R / np.linalg.norm(R, axis=1)[:, None] ** 3, axis=0)
        e1.append(np.max(np.abs(_force(MA, L) - exact)))
        e2.append(np.max(np.abs(_force(MA, L, Lc) - exact)))
    o1, o2 = _order(e1, scales), _order(e2, scales)
    assert 2.7 < o1 < 3.4, (e1, o1)
    assert 3.7 < o2 < 4.4, (e2, o2)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

def _traces(L):
    comp = {e: c for c, e in enumerate(EXP20)}
    t2 = L[..., comp[(2, 0, 0)]] + L[..., comp[(0, 2, 0)]] + L[..., comp[(0, 0, 2)]]
    t3 = [L[..., comp[(3, 0, 0)]] + L[..., comp[(1, 2, 0)]] + L[..., comp[(1, 0, 2)]],
          L[..., comp[(2, 1, 0)]] + L[..., comp[(0, 3, 0)]] + L[..., comp[(0, 1, 2)]],
          L[..., comp[(2, 0, 1)]] + L[..., comp[(0, 2, 1)]] + L[..., comp[(0, 0, 3)]]]
    return t2, t3


def test_harmonic_and_isotropic_cancellation(orc):
    tree = _single_node_tree()
    M = synth.random_moments(tree, seed=12)
    r = orc.run_pass_grid(tree, "multipole", M=M)
    L, S = r["L"], r["S"]
    t2, t3 = _traces(L.transpose(0, 2, 1))
    assert np.max(np.abs(t2)) <= 1e-13 * np.max(S[:, 4:10])
    for t in t3:
        assert np.max(np.abs(t)) <= 1e-13 * np.max(S[:, 10:20])
    # an isotropic second moment contributes nothing
    Mi = M.copy()
    for c in (4, 7, 9):
        Mi[:, c] += 0.37
    ri = orc.run_pass_grid(tree, "multipole", M=Mi)
    assert np.max(np.abs(ri["L"] - L)) <= 1e-13 * np.max(S)


@pytest.mark.parametrize("with_lc", [False, True])
def test_newton_third_law_multipole(orc, with_lc):
    """Over a pair set closed under o -> -o (one isolated sub-grid) the
    expansion forces sum to zero to rounding, with and without Lc."""
    tree = _single_node_tree()
    M = synth.random_moments(tree, seed=13)
    r = orc.run_pass_grid(tree, "multipole", M=M)
    L, Lc = r["L"][0].T, r["Lc"][0].T
    F = np.array([_force(M[0, :, a], L[a], Lc[a] if with_lc else None) for a in range(512)])
    scale = np.sum(np.abs(F))
    assert np.max(np.abs(F.sum(axis=0))) <= 1e-13 * scale


def test_newton_third_law_monopole_level(orc):
    tree = synth.uniform_level(1, 1.0)     # 8 leaf sub-grids, 16^3 cells
    rng = np.random.default_rng(14)
    m = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    r = orc.run_pass_grid(tree, "monopole", m=m)
    F = -(m[:, None, :] * r["L"][:, 1:4, :])
    assert np.max(np.abs(F.sum(axis=(0, 2)))) <= 1e-13 * np.sum(np.abs(F))


# ---------------------------------------------------------------------------
# local-expansion shift
# ---------------------------------------------------------------------------

def test_l2l_is_exact_taylor_shift_of_cubic(orc):
    rng = np.random.default_rng(15)
    for _ in range(5):
        Lp = rng.standard_normal(20)
        d = rng.uniform(-0.7, 0.7, 3)
        Lc = orc.l2l(Lp, d)
        for _ in range(5):
            delta = rng.uniform(-1, 1, 3)
            assert taylor(Lc, delta) == pytest.approx(taylor(Lp, d + delta), rel=1e-13, abs=1e-13)


# ---------------------------------------------------------------------------
# full multilevel solve
# ---------------------------------------------------------------------------

def _leaf_cells(tree):
    pos, ids = [], []
    for i in np.nonzero(tree.is_leaf)[0]:
        pos.append(synth.cell_centres(tree, i))
        ids.append(np.stack([np.full(512, i), np.arange(512)], axis=1))
    return np.concatenate(pos), np.concatenate(ids)


@pytest.mark.parametrize("src", [(0, 0, 0), (9, 4, 13), (15, 15, 15)])
def test_single_mass_covered_exactly_once(orc, src):
    """One unit point mass: the full solve must give -1/r at every other leaf
    cell (a pair missed by the stencils would give 0, a doubled pair -2/r)."""
    tree = synth.uniform_tree(1, 1.0)
    pos, ids = _leaf_cells(tree)
    idx = tree.index()
    node = idx[(1, src[0] // 8, src[1] // 8, src[2] // 8)]
    cell = (src[0] % 8) + 8 * (src[1] % 8) + 64 * (src[2] % 8)
    rho = np.zeros((tree.n, 512))
    rho[node, cell] = 1.0                       # h = 1: mass 1
    L = orc.full_solve(tree, rho)
    phi = L[ids[:, 0], 0, ids[:, 1]]
    r = np.linalg.norm(pos - (np.array(src) + 0.5), axis=1)
    mask = r > 0
    rel = np.abs(phi[mask] + 1.0 / r[mask]) * r[mask]
    assert np.max(rel) < 2e-2, np.max(rel)
    assert phi[~mask][0] == 0.0


def test_full_solve_matches_direct_sum(orc):
    tree = synth.uniform_tree(1, 1.0)
    rng = np.random.default_rng(16)
    rho = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    L = orc.full_solve(tree, rho)
    pos, ids = _leaf_cells(tree)
    m = rho[ids[:, 0], ids[:, 1]]
    sample = rng.choice(len(pos), 300, replace=False)
    for k in sample:
        d = np.linalg.norm(pos - pos[k], axis=1)
        d[k] = np.inf
        exact = -np.sum(m / d)
        grad = np.sum(m[:, None] * (pos[k] - pos) / d[:, None] ** 3, axis=0)
        got = L[ids[k, 0], :, ids[k, 1]]
        assert abs(got[0] - exact) < 2e-4 * abs(exact)
        assert np.max(np.abs(got[1:4] - grad)) < 1e-2 * np.max(np.abs(grad)) + 1e-3 * abs(exact) / 16


@pytest.mark.slow
def test_uniform_sphere_closed_form_converges(orc):
    """Phi of a uniform sphere, -M (3R^2 - r^2) / (2R^3) inside: the voxelised
    full solve approaches it as the sphere gets more cells."""
    errs = []
    tree = synth.uniform_tree(1, 1.0)            # 16^3 leaf cells
    pos, ids = _leaf_cells(tree)
    c = np.full(3, 8.0)
    for R in (3.0, 6.0):
        inside = np.linalg.norm(pos - c, axis=1) < R
        rho = np.zeros((tree.n, 512))
        rho[ids[inside, 0], ids[inside, 1]] = 1.0
        L = orc.full_solve(tree, rho)
        phi = L[ids[:, 0], 0, ids[:, 1]]
        Mtot = inside.sum()                          # discrete mass
        r = np.linalg.norm(pos - c, axis=1)
        exact = np.where(r < R, -Mtot * (3 * R * R - r * r) / (2 * R ** 3), -Mtot / r)
        core = r < R / 2
        errs.append(np.max(np.abs(phi[core] - exact[core]) / np.abs(exact[core])))
    assert errs[1] < errs[0] and errs[1] < 0.05, errs


# ---------------------------------------------------------------------------
# exact potential of piecewise-constant cells (homogeneous rectangular prisms)
# ---------------------------------------------------------------------------

def _prism_F(x, y, z):
    """An antiderivative F of 1/r with d^3 F / dx dy dz = 1/r (the closed form
    behind the potential of a homogeneous rectangular prism, Nagy 1966 and
    Waldvogel 1976), for coordinates that are all non-zero."""
    r = np.sqrt(x * x + y * y + z * z)
    return (x * y * np.log(z + r) + y * z * np.log(x + r) + z * x * np.log(y + r)
            - 0.5 * x * x * np.arctan(y * z / (x * r))
            - 0.5 * y * y * np.arctan(z * x / (y * r))
            - 0.5 * z * z * np.arctan(x * y / (z * r)))


def prism_integral(lo, hi):
    """The integral of dV / r over the box [lo, hi] (coordinates relative to
    the field point; [..., 3] arrays): F summed over the 8 corners with the
    sign of a nested definite integral."""
    lo = np.asarray(lo, dtype=float)
    hi = np.asarray(hi, dtype=float)
    tot = 0.0
    for i, j, k in itertools.product((0, 1), repeat=3):
        tot = tot + (-1) ** (3 - i - j - k) * _prism_F((hi if i else lo)[..., 0], (hi if j else lo)[..., 1],
                                                       (hi if k else lo)[..., 2])
    return tot


def test_prism_integral_closed_form():
    """The box integral against adaptive cubature (a box off the field point),
    against the unit cube's integral about its centre reduced to a smooth 2-D
    integral (int over [0,1]^3 of dV/r = 3/2 int over [0,1]^2 of
    ds dt / sqrt(1 + s^2 + t^2), by the pyramids where one coordinate is the
    largest), and far away against the point mass: a cube's first multipole
    beyond its mass that does not vanish is of order 4, so the difference
    falls as d^-5."""
    from scipy import integrate
    lo, hi = np.array([0.7, -1.3, 2.1]), np.array([1.9, -0.2, 3.0])
    num = integrate.tplquad(lambda z, y, x: 1.0 / math.sqrt(x * x + y * y + z * z), lo[0], hi[0], lo[1], hi[1],
                            lo[2], hi[2], epsabs=1e-13, epsrel=1e-12)[0]
    assert abs(prism_integral(lo, hi) - num) < 1e-11 * num
    pyr = integrate.dblquad(lambda t, s: 1.0 / math.sqrt(1 + s * s + t * t), 0, 1, 0, 1,
                            epsabs=1e-14, epsrel=1e-14)[0]
    # [-1/2, 1/2]^3 = 8 octants, each a quarter of [0, 1]^3 (dV/8, 1/r x 2)
    assert abs(prism_integral([-0.5] * 3, [0.5] * 3) - 2 * 1.5 * pyr) < 1e-12
    u = np.array([1.0, 0.37, 0.61])
    u /= np.linalg.norm(u)
    c5 = [(prism_integral(d * u - 0.5, d * u + 0.5) - 1.0 / d) * d ** 5 for d in (4.0, 8.0, 16.0)]
    assert c5[0] > 0 and max(c5) / min(c5) < 1.01, c5


def test_full_solve_against_exact_voxel_potential(orc):
    """Every leaf cell a homogeneous cube: the exact potential at sampled cell
    centres is the sum of closed-form cube integrals.  The method, by its
    definition, takes near cells (0 < |o|^2 <= 12) as point masses and omits
    the cell's own potential; with those terms put back at their exact
    values, what separates the full solve from the exact potential is the
    truncation of the multipole expansions and the down-pass alone.  That
    must stay far below the near-field model error (a dropped or mis-signed
    coarse-level term would exceed it: a coarse cell's dipole alone is of
    order 1e-2 of its pair's potential)."""
    tree = synth.uniform_tree(1, 1.0)          # 16^3 leaf cells, h = 1
    rng = np.random.default_rng(61)
    rho = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    L = orc.full_solve(tree, rho)
    pos, ids = _leaf_cells(tree)
    dens = rho[ids[:, 0], ids[:, 1]]
    i_self = prism_integral([-0.5] * 3, [0.5] * 3)
    trunc, model = [], []
    for k in rng.choice(len(pos), 64, replace=False):
        d = pos - pos[k]
        n2 = np.rint(np.sum(d * d, axis=1)).astype(np.int64)
        cube = prism_integral(d - 0.5, d + 0.5)
        exact = -np.sum(dens * cube)                                    # self included
        near, far = (n2 > 0) & (n2 <= 12), n2 > 12
        method = -np.sum(dens[far] * cube[far]) - np.sum(dens[near] / np.sqrt(n2[near]))
        got = L[ids[k, 0], 0, ids[k, 1]]
        trunc.append(abs(got - method) / abs(exact))
        model.append(abs(method - (exact + dens[k] * i_self)) / abs(exact))
    assert max(trunc) < 2e-5, max(trunc)
    assert max(trunc) < 0.2 * min(model), (max(trunc), min(model))
    assert max(model) < 5e-4, max(model)


@pytest.mark.slow
def test_polytrope_closed_form_converges(orc):
    """n = 1 polytrope (G = 1): rho = sin(xi)/xi, xi = pi r / R, whose potential
    inside is -(4 R^2 / pi)(1 + sin(xi)/xi).  The full solve plus each cell's
    own potential (closed form) approaches it at second order in h / R, the
    order of sampling the density at cell centres."""
    i_self = prism_integral([-0.5] * 3, [0.5] * 3)
    errs = []
    for leaf_level, R in ((1, 3.0), (1, 6.0), (2, 12.0)):
        tree = synth.uniform_tree(leaf_level, 1.0)
        pos, ids = _leaf_cells(tree)
        c = np.full(3, 4.0 * 2 ** leaf_level)         # the domain centre, a cell corner
        r = np.linalg.norm(pos - c, axis=1)
        xi = np.pi * r / R
        dens = np.where(r < R, np.sinc(xi / np.pi), 0.0)
        rho = np.zeros((tree.n, 512))
        rho[ids[:, 0], ids[:, 1]] = dens
        L = orc.full_solve(tree, rho)
        phi = L[ids[:, 0], 0, ids[:, 1]] - dens * i_self
        exact = np.where(r < R, -(4 * R * R / np.pi) * (1 + np.sinc(xi / np.pi)), -(4 * R ** 3 / np.pi) / r)
        errs.append(np.max(np.abs(phi - exact) / np.abs(exact)))
    assert errs[0] / errs[1] > 3 and errs[1] / errs[2] > 3 and errs[2] < 2e-3, errs


# ---------------------------------------------------------------------------
# adjoints
# ---------------------------------------------------------------------------

def _small_adaptive():
    def refine(level, coord, h0):
        return level == 1 and tuple(coord) in {(0, 0, 0), (1, 0, 0)}
    return synth.adaptive_tree(refine, 1, 2, 16.0)


@pytest.mark.parametrize("which", ["single", "adaptive"])
def test_multipole_adjoint_dot_product(orc, which):
    tree = _single_node_tree() if which == "single" else _small_adaptive()
    rng = np.random.default_rng(17)
    M = synth.random_moments(tree, seed=18)
    Lbar = rng.standard_normal((tree.n, 20, 512))
    L = orc.run_pass_grid(tree, "multipole", M=M)["L"]
    Mbar = orc.pass_adjoint(tree, "multipole", Lbar)
    a, b = np.sum(L * Lbar), np.sum(M * Mbar)
    assert a == pytest.approx(b, rel=1e-12)


@pytest.mark.parametrize("which", ["level", "adaptive"])
def test_monopole_adjoint_dot_product(orc, which):
    tree = synth.uniform_level(1, 1.0) if which == "level" else _small_adaptive()
    rng = np.random.default_rng(19)
    m = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    Lbar = rng.standard_normal((tree.n, 20, 512))
    L = orc.run_pass_grid(tree, "monopole", m=m)["L"]
    mbar = orc.pass_adjoint(tree, "monopole", Lbar)
    assert np.sum(L * Lbar) == pytest.approx(np.sum(m * mbar), rel=1e-12)


# ---------------------------------------------------------------------------
# virtual descendants of a coarse leaf
# ---------------------------------------------------------------------------

def test_virtual_descendants_equal_refined_leaves(orc):
    """A coarse leaf seen from a finer level holds 1/8^d of its cell mass in
    each virtual descendant: identical to refining it into real leaves."""
    tree = _small_adaptive()
    rng = np.random.default_rng(20)
    m = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    idx = tree.index()
    # refine one coarse level-1 leaf explicitly
    coarse = (1, 1, 1, 0)
    assert tree.is_leaf[idx[coarse]] == 1
    lv, co, lf = list(tree.level), [tuple(c) for c in tree.coord], list(tree.is_leaf)
    k = idx[coarse]
    lf[k] = 0
    new_m = [m[i] for i in range(tree.n)]
    for b in itertools.product((0, 1), repeat=3):
        cc = (2 * coarse[1] + b[0], 2 * coarse[2] + b[1], 2 * coarse[3] + b[2])
        lv.append(2)
        co.append(cc)
        lf.append(1)
        child = np.empty(512)
        for a in range(512):
            g = np.array([a % 8, (a // 8) % 8, a // 64]) + 8 * np.array(cc)
            gp = g // 2 - 8 * np.array(coarse[1:])
            child[a] = m[k, gp[0] + 8 * gp[1] + 64 * gp[2]] / 8
        new_m.append(child)
    ref = synth.Tree(np.array(lv, np.int32), np.array(co, np.int32), np.array(lf, np.uint8), tree.h0)
    m2 = np.array(new_m)
    targets = [[i, a] for i in range(tree.n) if tree.level[i] == 2 for a in range(0, 512, 37)]
    r1 = orc.run_pass(tree, "monopole", m=m, targets=targets)
    r2 = orc.run_pass(ref, "monopole", m=m2, targets=targets)
    assert r1["npairs"] == r2["npairs"]
    np.testing.assert_allclose(r1["L"], r2["L"], rtol=0, atol=1e-14 * np.max(r1["S"]))


# ---------------------------------------------------------------------------
# centre-of-mass expansion centres
# ---------------------------------------------------------------------------

def test_com_moments_exact(orc):
    """Root cells of a two-level tree: the centre is the mass-weighted mean of
    the 8 child cubes' centres, the dipole vanishes, and every moment equals
    the exact integral of the piecewise-constant density about that centre."""
    tree = synth.uniform_tree(1, h_leaf=1.0)
    rng = np.random.default_rng(21)
    rho = rng.integers(1, 9, size=(tree.n, 512)).astype(float) / 4.0   # exact in binary
    M, C = orc.moments_com(tree, rho)
    idx = tree.index()
    root = idx[(0, 0, 0, 0)]
    for cell in (0, 77, 300, 511):
        gp = np.array([cell % 8, (cell // 8) % 8, cell // 64])
        kids = []
        for b in itertools.product((0, 1), repeat=3):
            gc = 2 * gp + np.array(b)
            node = idx[(1, *(gc // 8))]
            kids.append((Fraction(rho[node, int((gc % 8) @ np.array([1, 8, 64]))]), gc))
        mass = sum(r for r, _ in kids)
        X = [sum(r * (Fraction(int(gc[a])) + Fraction(1, 2)) for r, gc in kids) / mass for a in range(3)]
        np.testing.assert_allclose(C[root, :, cell], [float(x) for x in X], rtol=1e-15)
        exact = np.zeros(20)
        for c, e in enumerate(EXP20):
            v = Fraction(0)
            for r, gc in kids:
                t = r
                for a in range(3):
                    t *= _axis_int(e[a], Fraction(int(gc[a])) - X[a], Fraction(int(gc[a]) + 1) - X[a])
                v += t
            exact[c] = float(v)
        scale = exact[0] * np.array([1.0] + [1.0] * 3 + [1.0] * 6 + [1.0] * 10)
        np.testing.assert_allclose(M[root, :, cell], exact, rtol=0, atol=1e-13 * scale.max())
        assert np.max(np.abs(M[root, 1:4, cell])) <= 1e-14 * exact[0]


def test_off_centre_expansions_taylor_order(orc):
    """Target and source expansions about arbitrary points inside their cells:
    the local model of a random point cluster still errs as O(s^4)."""
    tree = _single_node_tree()
    rng = np.random.default_rng(22)
    mu, u = _cluster(rng)
    A, B = (0, 0, 0), (4, 1, 0)
    XA = np.array(A) + 0.5 + rng.uniform(-0.3, 0.3, 3)
    XB = np.array(B) + 0.5 + rng.uniform(-0.3, 0.3, 3)
    dirs = rng.standard_normal((6, 3))
    errs, scales = [], [0.4, 0.2, 0.1, 0.05]
    for s in scales:
        M = np.zeros((1, 20, 512))
        C = synth.cell_centres(tree, 0).T.reshape(1, 3, 512).copy()
        C[0, :, _cell(*A)] = XA
        C[0, :, _cell(*B)] = XB
        pos = XB + s * u
        M[0, :, _cell(*B)] = point_cluster_moments(mu, pos, XB)
        r = orc.run_pass(tree, "multipole", M=M, targets=[[0, _cell(*A)]], centres=C)
        L = r["L"][0]
        e = 0.0
        for d in dirs:
            delta = s * d / np.linalg.norm(d)
            exact = -np.sum(mu / np.linalg.norm(XA + delta - pos, axis=1))
            e = max(e, abs(taylor(L, delta) - exact))
        errs.append(e)
    order = _order(errs, scales)
    assert 3.7 < order < 4.4, (errs, order)


def test_com_full_solve_matches_direct_sum(orc):
    tree = synth.uniform_tree(1, 1.0)
    rng = np.random.default_rng(23)
    rho = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    L = orc.full_solve(tree, rho, com=True)
    pos, ids = _leaf_cells(tree)
    m = rho[ids[:, 0], ids[:, 1]]
    for k in rng.choice(len(pos), 200, replace=False):
        d = np.linalg.norm(pos - pos[k], axis=1)
        d[k] = np.inf
        exact = -np.sum(m / d)
        assert abs(L[ids[k, 0], 0, ids[k, 1]] - exact) < 2e-4 * abs(exact)


@pytest.mark.parametrize("pass_kind", ["multipole", "monopole"])
def test_com_adjoint_dot_product(orc, pass_kind):
    """With the expansion centres held fixed, each pass is linear in its
    sources, so the transposed sum satisfies <L(M; C), Lbar> = <M, Mbar(C)>;
    the forward side with centres is pinned by the Taylor-order test above.
    The adaptive tree has multipole, leaf and virtual sources."""
    tree = _small_adaptive()
    rng = np.random.default_rng(24)
    rho = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    M, C = orc.moments_com(tree, rho)
    Lbar = rng.standard_normal((tree.n, 20, 512))
    if pass_kind == "multipole":
        src = synth.random_moments(tree, seed=25)
        L = orc.run_pass_grid(tree, "multipole", M=src, centres=C)["L"]
    else:
        src = rng.uniform(0.5, 1.5, size=(tree.n, 512))
        L = orc.run_pass_grid(tree, "monopole", m=src, centres=C)["L"]
    bar = orc.pass_adjoint(tree, pass_kind, Lbar, centres=C)
    assert np.sum(L * Lbar) == pytest.approx(np.sum(src * bar), rel=1e-12)
    # and the centres matter: the geometric-centre adjoint differs
    geo = orc.pass_adjoint(tree, pass_kind, Lbar)
    assert np.max(np.abs(geo - bar)) > 1e-6 * np.max(np.abs(bar))


# ---------------------------------------------------------------------------
# coarse leaf targets next to refined sub-grids (virtual refinement)
# ---------------------------------------------------------------------------

def test_newton_third_law_adaptive_tree(orc):
    """On a 2:1-balanced adaptive tree every pair of both passes appears from
    both sides -- fine cells see a coarse leaf's virtual children, and the
    coarse leaf, refined virtually, sees the fine cells -- so the expansion
    forces of all cells of all levels sum to zero to rounding."""
    tree = _small_adaptive()
    rng = np.random.default_rng(26)
    rho = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    M = orc.moments(tree, rho)
    m = np.ascontiguousarray(M[:, 0, :])
    r1 = orc.run_pass_grid(tree, "multipole", M=M)
    r2 = orc.run_pass_grid(tree, "monopole", m=m)
    L = r1["L"] + r2["L"]
    F = np.array([_force(M[i, :, a], L[i, :, a], r1["Lc"][i, :, a]) for i in range(tree.n) for a in range(512)])
    scale = np.sum(np.abs(F))
    assert np.max(np.abs(F.sum(axis=0))) <= 1e-13 * scale, (F.sum(axis=0), scale)


def test_coarse_target_sees_fine_mass_through_virtual_children(orc):
    """One unit mass in a fine cell next to a coarse leaf: a coarse cell whose
    refined neighbour is near gets the mean over its 8 virtual children of
    -1/r and of its gradient R/r^3; a coarse cell farther away gets nothing
    from the point-mass pass (it sees the refined cell's multipole)."""
    tree = _small_adaptive()
    idx = tree.index()
    assert tree.is_leaf[idx[(1, 0, 1, 0)]] == 1 and tree.is_leaf[idx[(1, 0, 0, 0)]] == 0
    m = np.zeros((tree.n, 512))
    fine = np.array([3, 15, 3])                                   # level-2 global cell
    m[idx[(2, *(fine // 8))], _cell(*(fine % 8))] = 1.0
    hc = tree.h0 / 4.0
    coarse = idx[(1, 0, 1, 0)]
    for g in ((1, 8, 1), (1, 9, 1), (1, 12, 1)):                  # level-1 global cells
        near = np.sum((np.array(g) - fine // 2) ** 2) <= 12
        r = orc.run_pass(tree, "monopole", m=m, targets=[[coarse, _cell(*(np.array(g) % 8))]])
        L = r["L"][0]
        if not near:
            assert np.all(L == 0.0)
            continue
        want0, want1 = 0.0, np.zeros(3)
        for cv in itertools.product((0, 1), repeat=3):
            R = (2 * np.array(g) + np.array(cv) - fine) * hc          # X_v - X_s
            d = np.linalg.norm(R)
            want0 += -1.0 / d / 8.0
            want1 += R / d ** 3 / 8.0
        assert L[0] == pytest.approx(want0, rel=1e-14)
        np.testing.assert_allclose(L[1:4], want1, rtol=1e-14)


def test_mirror_symmetry(orc):
    """Mirroring the density of a uniform tree across the x mid-plane mirrors
    the coefficients of both passes: L'(x) = S L(X - x), S negating the
    components of odd x-order (D(-R) = (-1)^k D(R) and the mirror-symmetric
    stencils)."""
    tree = synth.uniform_tree(1, 1.0)
    rng = np.random.default_rng(27)
    rho = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    idx = tree.index()

    def mirror(field):
        out = np.empty_like(field)
        for (l, x, y, z), i in idx.items():
            j = idx[(l, 2 ** l - 1 - x, y, z)]
            f = field[j].reshape(field.shape[1:-1] + (8, 8, 8))    # [..., z, y, x]
            out[i] = f[..., ::-1].reshape(field.shape[1:])
        return out
    rho_m = mirror(rho)
    M, Mm = orc.moments(tree, rho), orc.moments(tree, rho_m)
    L = orc.run_pass_grid(tree, "multipole", M=M)["L"] + orc.run_pass_grid(tree, "monopole", m=M[:, 0])["L"]
    Lm = orc.run_pass_grid(tree, "multipole", M=Mm)["L"] + orc.run_pass_grid(tree, "monopole", m=Mm[:, 0])["L"]
    sign = np.array([-1.0 if e[0] % 2 else 1.0 for e in EXP20])[None, :, None]
    want = sign * mirror(L)
    scale = np.max(np.abs(L), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(Lm - want) / scale) < 1e-13


def test_sampled_full_solve_helper_matches_whole_grid(orc):
    """The tests' per-cell full solve (own passes plus the ancestors' passes
    shifted down) reproduces the oracle's whole-grid full solve."""
    from helpers import full_solve_scale, oracle_full_solve_at
    tree = synth.uniform_tree(1, 1.0)
    rng = np.random.default_rng(28)
    rho = rng.uniform(0.5, 1.5, size=(tree.n, 512))
    L, S = orc.full_solve(tree, rho, with_s=True)
    M = orc.moments(tree, rho)
    cells = [(int(i), int(c)) for i in np.nonzero(tree.is_leaf)[0][:3] for c in (0, 77, 511)]
    Lc, Sc = oracle_full_solve_at(orc, tree, M, np.ascontiguousarray(M[:, 0, :]), cells, kind=None)
    for k, (i, c) in enumerate(cells):
        np.testing.assert_allclose(Lc[k], L[i, :, c], rtol=0, atol=1e-13 * np.max(S[i, :, c]))
        np.testing.assert_allclose(Sc[k], S[i, :, c], rtol=1e-12)
    # the whole-grid chain of the same scale
    Sg = full_solve_scale(orc, tree, M, np.ascontiguousarray(M[:, 0, :]), kind=None)
    np.testing.assert_allclose(Sg, S, rtol=1e-12)
    # the bar's scale: at the root level, the accumulated coefficients'
    # S + 1e-2 SD of both passes, the derived ones the sums they are formed from
    Sd = full_solve_scale(orc, tree, M, np.ascontiguousarray(M[:, 0, :]))
    r1 = orc.run_pass_grid(tree, "multipole", M=M)
    r2 = orc.run_pass_grid(tree, "monopole", m=np.ascontiguousarray(M[:, 0, :]))
    Se = r1["S"] + r2["S"] + 1e-2 * (r1["SD"] + r2["SD"])
    root = np.nonzero(tree.level == 0)[0]
    acc = [q for q in range(20) if q not in (9, 15, 18, 19)]
    np.testing.assert_allclose(Sd[root][:, acc], Se[root][:, acc], rtol=1e-12)
    np.testing.assert_allclose(Sd[root][:, 9], Se[root][:, 4] + Se[root][:, 7], rtol=1e-12)
    assert np.all(Sd[:, acc] >= S[:, acc] * (1 - 1e-12))


_EPS = np.zeros((3, 3, 3))
_EPS[0, 1, 2] = _EPS[1, 2, 0] = _EPS[2, 0, 1] = 1.0
_EPS[0, 2, 1] = _EPS[2, 1, 0] = _EPS[1, 0, 2] = -1.0


def _spin_torque(Mt, L):
    """Torque of the local field on a cell's mass distribution about its
    centre: tau_i = -eps_ijk sum_I L[k + I] M[j + I] / I! (full index sums,
    |I| <= 2)."""
    comp = {e: c for c, e in enumerate(EXP20)}

    def key(*idx):
        e = [0, 0, 0]
        for a in idx:
            e[a] += 1
        return comp[tuple(e)]
    tau = np.zeros(3)
    for i, j, k in itertools.product(range(3), repeat=3):
        if _EPS[i, j, k] == 0:
            continue
        acc = L[key(k)] * Mt[key(j)]
        for a in range(3):
            acc += L[key(k, a)] * Mt[key(j, a)]
        for a, b in itertools.product(range(3), repeat=2):
            acc += 0.5 * L[key(k, a, b)] * Mt[key(j, a, b)]
        tau[i] -= _EPS[i, j, k] * acc
    return tau


@pytest.mark.parametrize("seed", [20, 21, 22])
def test_angular_term_conserves_angular_momentum(orc, seed):
    """Masses and octupoles only (the case the angular term is for): over an
    isolated sub-grid the total torque of the expansion forces about the
    origin, orbital X x F plus the spin torque, is O(1) without Lc and
    vanishes to rounding with it -- which fixes the term's sign and form."""
    tree = _single_node_tree()
    M = synth.random_moments(tree, seed=seed)
    M[0, 1:10, :] = 0.0
    r = orc.run_pass_grid(tree, "multipole", M=M)
    L, Lc = r["L"][0].T, r["Lc"][0].T
    X = synth.cell_centres(tree, 0)

    def torque(with_lc):
        T, scale = np.zeros(3), 0.0
        for a in range(512):
            F = _force(M[0, :, a], L[a], Lc[a] if with_lc else None)
            t = np.cross(X[a], F) + _spin_torque(M[0, :, a], L[a])
            T += t
            scale += np.sum(np.abs(np.cross(X[a], F)))
        return np.linalg.norm(T), scale
    t0, scale = torque(False)
    t1, _ = torque(True)
    assert t0 > 1e-5 * scale
    assert t1 <= 1e-14 * scale, (t0, t1, scale)


@pytest.mark.parametrize("low, high", [(1, 17), (0, 16), (4, 20)])
def test_levels_sixteen_apart_do_not_alias(orc, low, high):
    """Node lookups tell levels apart over the whole range 0..20: two leaf
    sub-grids with the same coordinates on levels 16 apart each see only
    their own unit mass, as the exact near-field point-mass potential
    -1 / (|o| h), and nothing from the other."""
    tree = synth.two_level_forest(low, high, (1, 0, 0) if low > 0 else (0, 0, 0))
    for k in range(2):
        c0 = 3 + 8 * 4 + 64 * 2
        m = np.zeros((tree.n, 512))
        m[k, c0] = 1.0
        L = orc.run_pass_grid(tree, "monopole", m=m)["L"]
        assert np.all(L[1 - k] == 0.0)
        h = tree.h(tree.level[k])
        ijk = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")[::-1], -1).reshape(-1, 3)
        o = ijk - ijk[c0]
        r2 = np.sum(o * o, axis=1)
        seen = L[k, 0] != 0.0
        near = (r2 > 0) & (r2 <= 12)
        # near pairs always, far pairs of this level where their parents are
        # not well separated: each seen cell holds the exact point-mass value
        assert np.all(seen[near]) and not seen[c0]
        np.testing.assert_allclose(L[k, 0, seen], -1.0 / (np.sqrt(r2[seen]) * h), rtol=1e-15)


def test_massless_targets_have_no_angular_term(orc):
    """The angular term divides by the target's mass; a target without mass
    gets exactly zero there (no 0/0) and finite coefficients, while massive
    targets of the same sub-grid keep a non-zero term."""
    tree = _single_node_tree()
    M = synth.random_moments(tree, seed=19)
    massless = np.zeros(512, dtype=bool)
    massless[::5] = True
    M[0, 0, massless] = 0.0
    r = orc.run_pass_grid(tree, "multipole", M=M)
    assert np.all(np.isfinite(r["L"])) and np.all(np.isfinite(r["Lc"]))
    assert np.all(r["Lc"][0][:, massless] == 0.0)
    assert np.all(np.abs(r["Lc"][0][:, ~massless]).max(axis=0) > 0)
