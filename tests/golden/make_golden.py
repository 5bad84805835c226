"""Write the stored expected values under tests/golden/.

Every value here comes from the CPU oracle (``oracle/``), on inputs from the
seeded generators (``synth``), or from exact arithmetic (mpmath); nothing is
taken from the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py

The fixtures are plain text: ``#`` header lines state the workload, the
inputs' recipe and the columns; every other line is one row of
whitespace-separated numbers, floats written with 17 significant digits
(round-trip exact).
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

SEED_MOMENTS = 71
SEED_TARGETS = 72
SEED_LBAR = 73
N_TARGETS = 40
N_LBAR = 60


def small_adaptive_tree():
    """25 sub-grids: the root, 8 at level 1 of which (0,0,0) and (1,1,0) are
    refined, 16 leaves at level 2; h0 = 16 (leaf cells of level 2: h = 1).
    The two refined nodes' leaves have coarse level-1 leaves as neighbours,
    so the halo holds virtual descendants and coarse leaves are refined
    virtually as targets."""
    def refine(level, coord, h0):
        return level == 1 and tuple(coord) in {(0, 0, 0), (1, 1, 0)}
    return synth.adaptive_tree(refine, 1, 2, 16.0)


def inputs(tree):
    """Stress moments (every one of the 20 components non-zero, so dipole,
    quadrupole, octupole and angular terms all contribute), the point masses
    their order-0 row, the sampled targets and the sparse L-bar."""
    M = synth.random_moments(tree, seed=SEED_MOMENTS)
    m = np.ascontiguousarray(M[:, 0, :])
    targets = sample_cells(tree, N_TARGETS, SEED_TARGETS)
    Lbar, lbar_cells = synth.sparse_lbar(tree, N_LBAR, SEED_LBAR)
    return M, m, targets, Lbar, lbar_cells


def sample_cells(tree, count, seed):
    """[count, 2] distinct (node, cell) pairs, half of them in non-leaf
    sub-grids (multipole targets and sources) and half in leaf sub-grids."""
    rng = np.random.default_rng(seed)
    out = []
    for nodes in (np.flatnonzero(~tree.is_leaf.astype(bool)), np.flatnonzero(tree.is_leaf.astype(bool))):
        k = count // 2 if not out else count - count // 2
        flat = rng.choice(len(nodes) * 512, size=k, replace=False)
        out.append(np.stack([nodes[flat // 512], flat % 512], 1))
    return np.concatenate(out).astype(np.int32)


def _fmt(row):
    return " ".join(str(int(v)) if isinstance(v, (int, np.integer)) else f"{float(v):.17g}" for v in row)


def write_forward(tree, M, m, targets, path):
    r1 = oracle.run_pass(tree, "multipole", M=M, targets=targets)
    r2 = oracle.run_pass(tree, "monopole", m=m, targets=targets)
    L, S = r1["L"] + r2["L"], r1["S"] + r2["S"]
    with open(path, "w") as f:
        f.write("# Forward interactions (multipole pass with angular term + point-mass pass) at sampled cells.\n")
        f.write("# Method: Sec. 2.1 (FMM gravity on an octree of 8^3 sub-grids), Sec. 2.2.1 (one sub-grid plus\n")
        f.write("# its ghost layers per kernel), Sec. 4.1.1 (FP64); pass definitions as read for this library:\n")
        f.write("# order-3 Cartesian expansions, |J|+|I| <= 3 truncation, theta = 0.5 opening rule on integer\n")
        f.write("# offsets, virtual descendants of coarser leaves, angular-momentum correction Lc.\n")
        f.write("# Tree: adaptive, 25 sub-grids (root; level 1 with (0,0,0) and (1,1,0) refined; 16 level-2\n")
        f.write(f"# leaves), h0 = 16.  Inputs: M = synth.random_moments(tree, seed={SEED_MOMENTS}), m = M[:, 0, :].\n")
        f.write(f"# Targets: {N_TARGETS} distinct cells, sample_cells(tree, {N_TARGETS}, {SEED_TARGETS}): half in non-leaf, "
                "half in leaf sub-grids.\n")
        f.write("# Written by tests/golden/make_golden.py from the CPU oracle.\n")
        f.write("# columns: node cell L[0..19] S[0..19] Lc[0..2] Sc[0..2]   (S = sum over pairs of |term|)\n")
        for k in range(len(targets)):
            f.write(_fmt([targets[k, 0], targets[k, 1], *L[k], *S[k], *r1["Lc"][k], *r1["Sc"][k]]) + "\n")


def write_adjoint(tree, Lbar, lbar_cells, targets, path):
    Mb, SM = oracle.pass_adjoint(tree, "multipole", Lbar, with_s=True, targets=lbar_cells)
    mb, Sm = oracle.pass_adjoint(tree, "monopole", Lbar, with_s=True, targets=lbar_cells)
    with open(path, "w") as f:
        f.write("# Adjoint (transposed sum of both passes) at sampled source cells.\n")
        f.write("# Method: the transpose of the forward interactions of forward_small_adaptive.txt (same pairs,\n")
        f.write("# roles of target and source swapped; virtual descendants restricted onto their coarse leaf).\n")
        f.write("# Tree: as forward_small_adaptive.txt.  Input: L-bar = synth.sparse_lbar(tree, "
                f"{N_LBAR}, {SEED_LBAR})\n")
        f.write("# (N(0,1) in all 20 components at those cells, zero elsewhere).  Rows: the sampled cells of\n")
        f.write("# forward_small_adaptive.txt, now read as sources.\n")
        f.write("# Written by tests/golden/make_golden.py from the CPU oracle.\n")
        f.write("# columns: node cell Mbar[0..19] SM[0..19] mbar Sm   (S = sum over pairs of |term|)\n")
        for k in range(len(targets)):
            nd, c = targets[k]
            f.write(_fmt([nd, c, *Mb[nd, :, c], *SM[nd, :, c], mb[nd, c], Sm[nd, c]]) + "\n")


def write_closed_forms(path):
    import mpmath as mp
    mp.mp.dps = 30
    cube_centre = 3 * mp.log(2 + mp.sqrt(3)) - mp.pi / 2
    with open(path, "w") as f:
        f.write("# Closed forms (exact arithmetic, 30 digits), not from any implementation.\n")
        f.write("# unit_cube_centre: the integral of dV / r over the unit cube [-1/2, 1/2]^3 about its centre,\n")
        f.write("# = 3 ln(2 + sqrt 3) - pi/2.  By symmetry it is 8 (1/2)^2 I, I the integral over [0,1]^3 about\n")
        f.write("# the corner; I splits into three pyramids by the largest coordinate, and in the one where x is\n")
        f.write("# largest y = x s, z = x t give int_0^1 x dx J = J / 2, J = int_[0,1]^2 ds dt / sqrt(1 + s^2 + t^2)\n")
        f.write("# = ln(2 + sqrt 3) - pi/6; so the integral is 3 J.  Its negative is the potential (G = 1, unit\n")
        f.write("# density) of a homogeneous cube at its centre, the building block of the exact voxel potential\n")
        f.write("# the full solve is checked against.\n")
        f.write("# Written by tests/golden/make_golden.py (mpmath).\n")
        f.write("# columns: name value\n")
        f.write(f"unit_cube_centre {mp.nstr(cube_centre, 25)}\n")


def main():
    oracle.build()
    tree = small_adaptive_tree()
    M, m, targets, Lbar, lbar_cells = inputs(tree)
    write_forward(tree, M, m, targets, os.path.join(HERE, "forward_small_adaptive.txt"))
    write_adjoint(tree, Lbar, lbar_cells, targets, os.path.join(HERE, "adjoint_small_adaptive.txt"))
    write_closed_forms(os.path.join(HERE, "closed_forms.txt"))


if __name__ == "__main__":
    main()
