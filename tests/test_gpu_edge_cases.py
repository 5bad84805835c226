"""GPU edge cases: the deepest levels the interface allows, cells without
mass, and all-zero inputs, each through the C ABI against the oracle (or an
exact expected value)."""
import numpy as np
import pytest
import torch

import synth
from helpers import adjoint_with_scale, assert_parity, fwd_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ot():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2303_08058_b300 as ot
    ot.load()
    return ot


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("low, high", [(1, 17), (2, 18), (4, 20)])
def test_levels_sixteen_apart(ot, orc, low, high):
    """Two leaf sub-grids with equal coordinates on levels 16 apart (up to
    the deepest level, 20): the grid is accepted (not taken for a duplicate
    node), the forward and the adjoint match the oracle at every cell, and
    a level beyond 20 is refused."""
    tree = synth.two_level_forest(low, high, (1, 0, 0))
    rng = np.random.default_rng(81 + low)
    m = rng.uniform(0.5, 1.5, (tree.n, 512)) * tree.h(tree.level)[:, None] ** 3
    M = np.zeros((tree.n, 20, 512))
    M[:, 0, :] = m
    g = ot.OTGrid.from_tree(tree)
    L, _ = g.interactions(dev(M), dev(m))
    Lbar = rng.standard_normal((tree.n, 20, 512))
    _, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    g.check()
    r = orc.run_pass_grid(tree, "monopole", m=m)
    assert_parity(host(L), r["L"], fwd_scale(r), what="L", kind="L")
    assert g.info()["pairs_monopole"] == r["npairs"] > 0
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar)
    assert_parity(host(mb), mo, Sm, what="mbar")
    with pytest.raises(ot.OTError, match="OT_EINVAL"):
        ot.OTGrid(np.array([21], np.int32), np.zeros((1, 3), np.int32), np.ones(1, np.uint8), 1.0)


def test_deep_node_inside_a_coarse_leaf_refused(ot):
    """A level-16 sub-grid inside the level-0 root leaf would see the root's
    cells as virtual descendants 16 levels down; the library serves at most
    5 (2:1-balanced trees need 1) and refuses the grid with a message."""
    tree = synth.two_level_forest(0, 16, (0, 0, 0))
    with pytest.raises(ot.OTError, match="OT_EINVAL.*virtual descendant 16 levels"):
        ot.OTGrid.from_tree(tree)


def _small_adaptive():
    def refine(level, coord, h0):
        return level == 1 and tuple(coord) in {(0, 0, 0), (1, 1, 0)}
    return synth.adaptive_tree(refine, 1, 2, 16.0)


def test_cells_without_mass(ot, orc):
    """Stress moments in which a fifth of the cells carry no mass but keep
    their higher moments: no division by a zero mass reaches the output,
    the angular term of a massless target is exactly zero, and every
    coefficient matches the oracle."""
    tree = _small_adaptive()
    M = synth.random_moments(tree, seed=82)
    rng = np.random.default_rng(83)
    massless = rng.random((tree.n, 512)) < 0.2
    M[:, 0, :][massless] = 0.0
    m = np.ascontiguousarray(M[:, 0, :])
    g = ot.OTGrid.from_tree(tree)
    L, Lc = g.interactions(dev(M), dev(m))
    torch.cuda.synchronize()
    g.check()
    L, Lc = host(L), host(Lc)
    assert np.all(np.isfinite(L)) and np.all(np.isfinite(Lc))
    nonleaf = ~tree.is_leaf.astype(bool)
    sel = massless & nonleaf[:, None]
    assert sel.any() and np.all(Lc.transpose(0, 2, 1)[sel] == 0.0)
    r1 = orc.run_pass_grid(tree, "multipole", M=M)
    r2 = orc.run_pass_grid(tree, "monopole", m=m)
    assert_parity(L, r1["L"] + r2["L"], fwd_scale(r1) + fwd_scale(r2), what="L", kind="L")
    assert_parity(Lc, r1["Lc"], fwd_scale(r1, lc=True), what="Lc")


def test_all_zero_inputs_give_exact_zeros(ot):
    """Zero densities give zero moments, zero coefficients and a zero angular
    term; a zero L-bar gives zero gradients: exactly, with no NaN from the
    massless targets."""
    tree = _small_adaptive()
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(torch.zeros((tree.n, 512), dtype=torch.float64, device="cuda"))
    L, Lc = g.interactions(M, m)
    Mb, mb = g.backward(torch.zeros((tree.n, 20, 512), dtype=torch.float64, device="cuda"))
    rb = g.moments_backward(Mb, mb)
    torch.cuda.synchronize()
    g.check()
    for t in (M, m, L, Lc, Mb, mb, rb):
        assert torch.count_nonzero(t).item() == 0 and bool(torch.isfinite(t).all())
