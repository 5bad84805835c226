"""Stored expected values (tests/golden/) against the CPU oracle.

The fixtures were written by tests/golden/make_golden.py from the oracle and
from exact arithmetic; these tests re-derive them so that any later change to
the oracle's arithmetic, or to the seeded input recipe, shows up here, and
they pin the exact cube integral behind the voxel-potential check to its
closed form.  The CUDA path is compared with the same fixtures in
test_gpu_golden.py, without running the oracle.
"""
import numpy as np

from helpers import (golden_adjoint_columns, golden_forward_columns, load_golden, load_golden_constants,
                     load_golden_script, parity_ratio)
from test_oracle_pins import prism_integral

make_golden = load_golden_script()


def _inputs():
    tree = make_golden.small_adaptive_tree()
    return (tree, *make_golden.inputs(tree))


def test_golden_forward_reproduced_by_oracle(orc):
    tree, M, m, targets, _, _ = _inputs()
    tg, L, S, Lc, Sc = golden_forward_columns(load_golden("forward_small_adaptive.txt"))
    np.testing.assert_array_equal(tg, targets)
    r1 = orc.run_pass(tree, "multipole", M=M, targets=tg)
    r2 = orc.run_pass(tree, "monopole", m=m, targets=tg)
    assert parity_ratio(r1["L"] + r2["L"], L, S) <= 1e-15
    assert parity_ratio(r1["Lc"], Lc, Sc) <= 1e-15
    np.testing.assert_allclose(r1["S"] + r2["S"], S, rtol=1e-15)
    # the fixture exercises every kind of pair: non-leaf targets (multipole
    # sources, angular term) and leaf targets (point masses)
    assert np.all(np.abs(Lc[:20]).max(axis=1) > 0) and np.all(Lc[20:] == 0)


def test_golden_adjoint_reproduced_by_oracle(orc):
    tree, _, _, _, Lbar, lbar_cells = _inputs()
    cells, Mb, SM, mb, Sm = golden_adjoint_columns(load_golden("adjoint_small_adaptive.txt"))
    Mo, SMo = orc.pass_adjoint(tree, "multipole", Lbar, with_s=True, targets=lbar_cells)
    mo, Smo = orc.pass_adjoint(tree, "monopole", Lbar, with_s=True, targets=lbar_cells)
    assert parity_ratio(Mo[cells[:, 0], :, cells[:, 1]], Mb, SM) <= 1e-15
    assert parity_ratio(mo[cells[:, 0], cells[:, 1]], mb, Sm) <= 1e-15
    assert np.count_nonzero(Mb.any(axis=1)) == 20 and np.count_nonzero(mb) == 20


def test_cube_integral_matches_stored_closed_form():
    """The homogeneous-prism integral used by the voxel-potential pin, about
    the unit cube's centre, equals the stored 3 ln(2 + sqrt 3) - pi/2."""
    c = load_golden_constants("closed_forms.txt")["unit_cube_centre"]
    assert abs(prism_integral([-0.5] * 3, [0.5] * 3) - c) <= 4e-15 * c
    # scaling: a cube of side a about its centre integrates to a^2 times it
    assert abs(prism_integral([-1.5] * 3, [1.5] * 3) - 9.0 * c) <= 4e-15 * 9.0 * c
