"""Workload generators: octrees of 8^3-cell sub-grids and the fields on them.

Conventions (shared by every consumer):

* A tree is a ``Tree`` with ``level[n]``, ``coord[n,3]`` (integer node position
  at its level, ``0 <= coord < 2**level``), ``is_leaf[n]`` and ``h0`` (the cell
  size at level 0).  The cell size at level ``l`` is ``h0 / 2**l``.  Every node
  carries an 8x8x8 sub-grid (Sec. 2.1 of the paper); cell ``(i, j, k)`` of a node
  has flat index ``i + 8*j + 64*k`` and its centre at
  ``(8*coord + (i, j, k) + 0.5) * h_l``.
* ``is_leaf`` marks the source class of a node's cells: leaf cells act as point
  masses (monopole sources) and receive near-field interactions; non-leaf cells
  act as multipole sources.  A non-leaf node need not have children (the
  isolated single sub-grid workload uses one such node).
* Nodes are ordered by level, then Morton order of ``coord``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Tree", "cell_centres", "single_subgrid", "uniform_tree", "uniform_level", "two_level_forest",
    "adaptive_tree", "balance_2to1", "polytrope_density", "sample_density",
    "uniform_random_density", "random_moments", "binary_star_field",
    "sparse_lbar", "choose_probes", "config1", "config2", "config3", "config4_probes",
    "config5_step", "STAR_FLOOR",
]

STAR_FLOOR = 1e-10
N1 = 8           # cells per sub-grid edge
NCELL = 512      # cells per sub-grid


@dataclasses.dataclass
class Tree:
    level: np.ndarray      # int32 [n]
    coord: np.ndarray      # int32 [n, 3]
    is_leaf: np.ndarray    # uint8 [n]
    h0: float

    @property
    def n(self) -> int:
        return int(self.level.shape[0])

    def h(self, level):
        return self.h0 / (2.0 ** np.asarray(level))

    def index(self):
        return {(int(l), int(c[0]), int(c[1]), int(c[2])): i
                for i, (l, c) in enumerate(zip(self.level, self.coord))}

    def counts(self):
        lv = self.level
        return {int(l): (int(np.sum(lv == l)), int(np.sum((lv == l) & (self.is_leaf == 1))))
                for l in np.unique(lv)}


def _morton(c):
    x, y, z = (int(v) for v in c)
    key = 0
    for b in range(21):
        key |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
    return key


def _make_tree(nodes, leaves, h0):
    items = sorted(nodes, key=lambda t: (t[0], _morton(t[1:])))
    level = np.array([t[0] for t in items], dtype=np.int32)
    coord = np.array([t[1:] for t in items], dtype=np.int32).reshape(-1, 3)
    is_leaf = np.array([1 if t in leaves else 0 for t in items], dtype=np.uint8)
    return Tree(level, coord, is_leaf, float(h0))


def _children(t):
    l, x, y, z = t
    return [(l + 1, 2 * x + a, 2 * y + b, 2 * z + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]


def _leaves_of(nodes):
    return {t for t in nodes if _children(t)[0] not in nodes}


def cell_centres(tree: Tree, node: int) -> np.ndarray:
    """[512, 3] cell-centre positions of one node, flat index i + 8 j + 64 k."""
    h = tree.h0 / 2.0 ** int(tree.level[node])
    k, j, i = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    loc = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    return (8.0 * tree.coord[node].astype(np.float64) + loc + 0.5) * h


def single_subgrid(level: int = 1, h: float = 1.0, leaf: bool = False) -> Tree:
    """One isolated sub-grid; every halo cell around it is empty (zero)."""
    nodes = {(level, 0, 0, 0)}
    leaves = nodes if leaf else set()
    return _make_tree(nodes, leaves, h * 2.0 ** level)


def uniform_tree(leaf_level: int, h_leaf: float = 1.0) -> Tree:
    """Complete octree: every level 0..leaf_level full, leaves at leaf_level."""
    nodes = set()
    for l in range(leaf_level + 1):
        s = 2 ** l
        for z in range(s):
            for y in range(s):
                for x in range(s):
                    nodes.add((l, x, y, z))
    leaves = {t for t in nodes if t[0] == leaf_level}
    return _make_tree(nodes, leaves, h_leaf * 2.0 ** leaf_level)


def uniform_level(leaf_level: int, h_leaf: float = 1.0) -> Tree:
    """Only the leaf level of a uniform tree (no coarse levels)."""
    s = 2 ** leaf_level
    nodes = {(leaf_level, x, y, z) for z in range(s) for y in range(s) for x in range(s)}
    return _make_tree(nodes, nodes, h_leaf * 2.0 ** leaf_level)


def two_level_forest(low: int = 1, high: int = 17, coord=(1, 0, 0)) -> Tree:
    """Two isolated leaf sub-grids with the same integer coordinates, one on
    level ``low`` and one on level ``high`` (h = 1 there), and no other node:
    a tree whose levels differ by 16 puts the two at positions that a level
    field of 4 bits cannot tell apart."""
    nodes = {(low, *coord), (high, *coord)}
    return _make_tree(nodes, nodes, 2.0 ** high)


def balance_2to1(nodes: set) -> set:
    """Refine until every node's parent has all its 26 same-level neighbours.

    This makes leaves that touch (face, edge or corner) differ by at most one
    level.  ``nodes`` must be closed under taking parents and siblings.
    """
    nodes = set(nodes)

    def ensure(t):
        if t in nodes:
            return
        l, x, y, z = t
        parent = (l - 1, x >> 1, y >> 1, z >> 1)
        ensure(parent)
        for c in _children(parent):
            nodes.add(c)

    changed = True
    while changed:
        changed = False
        for t in sorted(nodes):
            l, x, y, z = t
            if l < 2:
                continue
            pl, px, py, pz = l - 1, x >> 1, y >> 1, z >> 1
            s = 2 ** pl
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        q = (pl, px + dx, py + dy, pz + dz)
                        if min(q[1:]) < 0 or max(q[1:]) >= s:
                            continue
                        if q not in nodes:
                            ensure(q)
                            changed = True
    return nodes


def adaptive_tree(refine, min_level: int, max_level: int, h0: float) -> Tree:
    """Octree full down to ``min_level``; a node below max_level with
    ``refine(level, coord, h0)`` true gets 8 children; then 2:1 balanced."""
    nodes = set()
    for l in range(min_level + 1):
        s = 2 ** l
        nodes |= {(l, x, y, z) for z in range(s) for y in range(s) for x in range(s)}
    frontier = [t for t in nodes if t[0] == min_level]
    while frontier:
        nxt = []
        for t in frontier:
            if t[0] < max_level and refine(t[0], np.array(t[1:]), h0):
                for c in _children(t):
                    nodes.add(c)
                    nxt.append(c)
        frontier = nxt
    nodes = balance_2to1(nodes)
    return _make_tree(nodes, _leaves_of(nodes), h0)


# ----------------------------------------------------------------------------
# density fields
# ----------------------------------------------------------------------------

def polytrope_density(x: np.ndarray, centre, radius: float, rho_c: float = 1.0,
                      floor: float = STAR_FLOOR) -> np.ndarray:
    """n = 1 polytrope rho_c sin(xi)/xi with xi = pi r / R inside R, ``floor`` outside."""
    r = np.linalg.norm(x - np.asarray(centre, dtype=np.float64), axis=-1)
    xi = np.pi * r / radius
    with np.errstate(invalid="ignore", divide="ignore"):
        core = np.where(xi > 0, np.sin(xi) / np.where(xi > 0, xi, 1.0), 1.0)
    rho = np.where(r < radius, rho_c * core, 0.0)
    return np.maximum(rho, floor)


def sample_density(tree: Tree, field) -> np.ndarray:
    """[n, 512] densities sampled at the cell centres of every node."""
    out = np.empty((tree.n, NCELL), dtype=np.float64)
    for i in range(tree.n):
        out[i] = field(cell_centres(tree, i))
    return out


def uniform_random_density(tree: Tree, seed: int, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(tree.n, NCELL))


def random_moments(tree: Tree, seed: int, positive_mass: bool = True) -> np.ndarray:
    """[n, 20, 512] stress moments: component of order m ~ N(0,1) h^(m+3)
    (mass ~ U[0.5, 1.5] h^3 when ``positive_mass``)."""
    rng = np.random.default_rng(seed)
    orders = np.array([0] + [1] * 3 + [2] * 6 + [3] * 10)
    h = tree.h(tree.level)[:, None, None]
    M = rng.standard_normal((tree.n, 20, NCELL)) * h ** (orders[None, :, None] + 3)
    if positive_mass:
        M[:, 0, :] = rng.uniform(0.5, 1.5, size=(tree.n, NCELL)) * h[:, 0, :] ** 3
    return M


def sparse_lbar(tree: Tree, count: int, seed: int):
    """L-bar [n, 20, 512] that is N(0,1) in all 20 components on ``count``
    random cells (duplicates merged) and zero elsewhere, and those cells as
    [k, 2] (node, cell) sorted pairs."""
    rng = np.random.default_rng(seed)
    cells = np.unique(np.stack([rng.integers(0, tree.n, count), rng.integers(0, NCELL, count)], 1), axis=0)
    Lbar = np.zeros((tree.n, 20, NCELL))
    Lbar[cells[:, 0], :, cells[:, 1]] = rng.standard_normal((len(cells), 20))
    return Lbar, cells.astype(np.int32)


def choose_probes(n_cells: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_cells, size=count, replace=False)).astype(np.int64)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def config1(seed: int = 1):
    """One isolated 8^3 sub-grid (h = 1) with empty halo; rho ~ U[0.5, 1.5];
    its cells act as multipole sources."""
    tree = single_subgrid(level=1, h=1.0, leaf=False)
    return tree, uniform_random_density(tree, seed)


def config2(leaf_level: int = 3, radius: float = 28.0):
    """Uniform 64^3 leaf level (512 sub-grids, h = 1) plus coarse levels 0-2,
    holding an n = 1 polytrope of radius 28 centred on the domain centre."""
    tree = uniform_tree(leaf_level, 1.0)
    side = 8.0 * 2 ** leaf_level
    centre = (side / 2,) * 3
    rho = sample_density(tree, lambda x: polytrope_density(x, centre, radius))
    return tree, rho


def _star_refine(stars, threshold=1e-3):
    """Refine a node whose box comes within the radius where the star density
    drops to ``threshold`` * rho_c (sinc(xi) = threshold)."""
    # xi_t solves sin(xi)/xi = threshold on (0, pi): bisection
    lo, hi = 1.0, math.pi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.sin(mid) / mid > threshold:
            lo = mid
        else:
            hi = mid
    frac = lo / math.pi

    def refine(level, coord, h0):
        size = 8.0 * h0 / 2 ** level
        lo_c = coord * size
        hi_c = lo_c + size
        for (c, R, rc) in stars:
            c = np.asarray(c)
            d = np.maximum(0.0, np.maximum(lo_c - c, c - hi_c))
            if np.linalg.norm(d) < R * frac and rc > 0:
                return True
        return False
    return refine


def config3(seed: int = 3, radius_l3_cells: float = 7.0):
    """Adaptive octree, levels 3-6 (finest h = 1): one polytrope with a seeded
    centre; nodes are refined where rho > 1e-3 rho_c, then 2:1 balanced."""
    rng = np.random.default_rng(seed)
    h0 = 64.0                     # level-6 cells have h = 1
    side = 8 * h0
    R = radius_l3_cells * 8.0     # a level-3 cell is 8 finest cells
    centre = side / 2 + rng.uniform(-0.05, 0.05, size=3) * side
    stars = [(centre, R, 1.0)]
    tree = adaptive_tree(_star_refine(stars), 3, 6, h0)
    rho = sample_density(tree, lambda x: polytrope_density(x, centre, R))
    return tree, rho, dict(centre=centre, radius=R)


def config4_probes(n_cells: int = 262144, seed: int = 4, count: int = 1000):
    return choose_probes(n_cells, count, seed)


def binary_star_field(angle: float, side: float, r1=24.0, r2=19.0, sep=60.0, q=0.5):
    """Two n = 1 polytropes (mass ratio q, radii r1, r2, separation sep) whose
    centres are rotated by ``angle`` about the z axis through the domain centre.
    Returns (field(x), stars) with stars = [(centre, R, rho_c)]."""
    rc1 = 1.0
    rc2 = q * rc1 * (r1 / r2) ** 3
    m1_frac = 1.0 / (1.0 + q)
    cx = side / 2
    d1, d2 = -sep * (1 - m1_frac), sep * m1_frac     # centre of mass at the domain centre
    ca, sa = math.cos(angle), math.sin(angle)
    c1 = np.array([cx + d1 * ca, cx + d1 * sa, cx])
    c2 = np.array([cx + d2 * ca, cx + d2 * sa, cx])

    def field(x):
        a = polytrope_density(x, c1, r1, rc1, floor=0.0)
        b = polytrope_density(x, c2, r2, rc2, floor=0.0)
        return np.maximum(a + b, STAR_FLOOR)
    return field, [(c1, r1, rc1), (c2, r2, rc2)]


def config5_step(step: int, side: float = 390.0, min_level: int = 3, max_level: int = 7):
    """Binary-star workload at time step ``step``: the field is rotated by
    0.01 * step rad; the adaptive tree (levels 3-7) is rebuilt for it."""
    field, stars = binary_star_field(0.01 * step, side)
    h0 = side / 8.0
    tree = adaptive_tree(_star_refine(stars), min_level, max_level, h0)
    rho = sample_density(tree, field)
    return tree, rho
