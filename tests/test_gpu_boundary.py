"""Coarse-fine boundaries on the GPU: the coarse leaf targets refined
virtually (their near sources in refined sub-grids seen through the leaf's
virtual children), checked by the properties that hold at any size -- every
pair appears from both sides, so the expansion forces of all cells of all
levels sum to zero -- and by the grid's rejection of trees the rule cannot
serve.  Parity with the oracle on these pairs is in the adaptive-tree tests
of the other GPU files."""
import numpy as np
import pytest
import torch

import synth

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


# stored components: 0; x y z; xx xy xz yy yz zz; xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
_E = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
      (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1),
      (0, 1, 2), (0, 0, 3)]
_C = {e: c for c, e in enumerate(_E)}


def _key(*idx):
    e = [0, 0, 0]
    for a in idx:
        e[a] += 1
    return _C[tuple(e)]


def total_force(M, L, Lc):
    """Sum over all cells of F_i = -(M0 L_i + sum_j M_j L_ij + 1/2 sum_jk M_jk
    L_ijk) - M0 Lc_i (full index sums over the stored symmetric components),
    and the sum of |F|."""
    F = []
    for i in range(3):
        f = M[:, 0] * L[:, _key(i)]
        for j in range(3):
            f = f + M[:, _key(j)] * L[:, _key(i, j)]
        for j in range(3):
            for k in range(3):
                f = f + 0.5 * M[:, _key(j, k)] * L[:, _key(i, j, k)]
        f = f + M[:, 0] * Lc[:, i]
        F.append(-f)
    F = torch.stack(F)
    return F.sum(dim=(1, 2)).cpu().numpy(), float(F.abs().sum())


def _unbalanced_tree():
    """Root, all 8 level-1 nodes; (1,1,0,0) refined, and its child (2,2,0,0),
    which touches the leaf (1,0,0,0), refined again."""
    nodes = {(0, 0, 0, 0)}
    nodes |= {(1, x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)}
    nodes |= {(2, 2 + x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)}
    nodes |= {(3, 4 + x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)}
    nodes = sorted(nodes)
    parents = {(l - 1, x >> 1, y >> 1, z >> 1) for (l, x, y, z) in nodes if l > 0}
    level = np.array([t[0] for t in nodes], np.int32)
    coord = np.array([t[1:] for t in nodes], np.int32)
    leaf = np.array([0 if t in parents else 1 for t in nodes], np.uint8)
    return level, coord, leaf


def test_unbalanced_tree_rejected(ot):
    level, coord, leaf = _unbalanced_tree()
    with pytest.raises(ot.OTError, match="OT_EINVAL.*2:1"):
        ot.OTGrid(level, coord, leaf, 16.0)


@pytest.mark.parametrize("cfg", ["adaptive", "binary"])
def test_newton_third_law_full_size(ot, cfg):
    """Config 3 (4,641 sub-grids) and the binary star (9,481 sub-grids): the
    forces of all cells of all levels, from both passes and the angular
    term, sum to zero to rounding."""
    tree, rho = synth.config3()[:2] if cfg == "adaptive" else synth.config5_step(0)
    g = ot.OTGrid.from_tree(tree)
    info = g.info()
    assert info["pairs_refined"] > 0 and info["pairs_virtual"] > 0
    M, m = g.moments(dev(rho))
    L, Lc = g.interactions(M, m)
    torch.cuda.synchronize()
    g.check()
    Fsum, Fabs = total_force(M, L, Lc)
    assert np.max(np.abs(Fsum)) <= 1e-12 * Fabs, (Fsum, Fabs)


def test_newton_third_law_com_centres(ot):
    """The same with centre-of-mass expansion centres (every pair antisymmetric
    about its own centres)."""
    tree, rho, _ = synth.config3()
    g = ot.OTGrid.from_tree(tree)
    M, m, C = g.moments_com(dev(rho))
    L, Lc = g.interactions_com(M, m, C)
    torch.cuda.synchronize()
    g.check()
    Fsum, Fabs = total_force(M, L, Lc)
    assert np.max(np.abs(Fsum)) <= 1e-12 * Fabs, (Fsum, Fabs)


def test_adaptive_atomic_adjoint_equals_fixed_order(ot):
    """On config 3 the point-mass adjoint by target (atomic adds, refined near
    sources included) equals the fixed-order gather (which reaches the coarse
    leaves' virtual children from the fine side) to rounding."""
    tree, rho, _ = synth.config3()
    g = ot.OTGrid.from_tree(tree)
    Lbar = dev(np.random.default_rng(110).standard_normal((tree.n, 20, 512)))
    Mb1, mb1 = g.backward(Lbar)
    g.set_deterministic(True)
    Mb2, mb2 = g.backward(Lbar)
    torch.cuda.synchronize()
    g.check()
    assert torch.equal(Mb1, Mb2)
    scale = float(mb2.abs().max())
    assert float((mb1 - mb2).abs().max()) <= 1e-13 * scale
