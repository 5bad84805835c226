"""Centre-of-mass expansion centres on the GPU: moments and centres, both
passes with the derivatives evaluated per pair at R = C_A - C_B, the adjoint
with the centres held fixed, and the down-pass, against the oracle's
explicit-centre functions.  Every oracle input comes from the seeded
generators or the oracle itself."""
import numpy as np
import pytest
import torch

import synth
from helpers import adjoint_with_scale, assert_parity, full_solve_scale, fwd_scale, oracle_threads, sample_targets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ot():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2303_08058_b300 as ot
    ot.load()
    return ot


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    oracle_threads(oracle)
    return oracle


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def _small_adaptive():
    """25 sub-grids: root, 8 at level 1 (two refined), 16 leaves at level 2."""
    def refine(l, c, h0):
        return l == 1 and tuple(c) in {(0, 0, 0), (1, 1, 0)}
    return synth.adaptive_tree(refine, 1, 2, 16.0)


TREES = {
    "uniform": lambda: synth.uniform_tree(1, 1.0),
    "adaptive": _small_adaptive,
    "root_leaf": lambda: synth.single_subgrid(0, 1.0, leaf=True),
    "leaf_level": lambda: synth.uniform_level(1, 1.0),
}


def all_targets(tree):
    return np.stack(np.meshgrid(np.arange(tree.n), np.arange(512), indexing="ij"), -1).reshape(-1, 2).astype(np.int32)


def at_targets(L, tg):
    return L[tg[:, 0], :, tg[:, 1]]


def oracle_com_inputs(orc, tree, rho):
    M, C = orc.moments_com(tree, rho)
    return M, np.ascontiguousarray(M[:, 0, :]), C


def oracle_com_passes(orc, tree, M, m, C, tg):
    r1 = orc.run_pass(tree, "multipole", M=M, targets=tg, centres=C)
    r2 = orc.run_pass(tree, "monopole", m=m, targets=tg, centres=C)
    return r1["L"] + r2["L"], fwd_scale(r1) + fwd_scale(r2), r1["Lc"], fwd_scale(r1, lc=True)


def geometric_centres(tree):
    return np.stack([synth.cell_centres(tree, i).T for i in range(tree.n)])


# ---------------------------------------------------------------------------
# moments and centres
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["uniform", "adaptive"])
def test_com_moments_match_oracle(ot, orc, which):
    tree = TREES[which]()
    rho = synth.uniform_random_density(tree, seed=91)
    g = ot.OTGrid.from_tree(tree)
    M, m, C = g.moments_com(dev(rho))
    torch.cuda.synchronize()
    Mo, Co = orc.moments_com(tree, rho)
    extent = 8.0 * tree.h0
    assert np.max(np.abs(host(C) - Co)) <= 1e-14 * extent
    # a shift by the rounding of the centre moves order k by ~k M_(k-1) dX
    h = tree.h(tree.level)[:, None, None]
    k = np.array([0] + [1] * 3 + [2] * 6 + [3] * 10)[None, :, None]
    scale = np.abs(Mo[:, :1, :]) * (h + extent) ** k
    assert np.all(np.abs(host(M) - Mo) <= 1e-13 * scale + 1e-300)
    np.testing.assert_array_equal(host(m), host(M)[:, 0, :])
    # the centres are really centres of mass: dipoles vanish to rounding
    nonleaf = tree.is_leaf == 0
    dip = np.abs(host(M)[nonleaf, 1:4, :])
    assert np.all(dip <= 1e-12 * np.abs(Mo[nonleaf, :1, :]) * extent)


# ---------------------------------------------------------------------------
# the passes with explicit centres
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["uniform", "adaptive", "root_leaf", "leaf_level"])
def test_com_passes_all_cells(ot, orc, which):
    """Every cell of trees with every source class (multipole, leaf, virtual
    descendants of coarse leaves) and every stencil (root, far, near)."""
    tree = TREES[which]()
    rho = synth.uniform_random_density(tree, seed=92)
    M, m, C = oracle_com_inputs(orc, tree, rho)
    g = ot.OTGrid.from_tree(tree)
    Cg = C.copy()
    Cg[tree.is_leaf == 1] = np.nan      # never read: leaf cells sit at their geometric centres
    L, Lc = g.interactions_com(dev(M), dev(m), dev(Cg))
    torch.cuda.synchronize()
    g.check()
    tg = all_targets(tree)
    Lo, S, Lco, Sc = oracle_com_passes(orc, tree, M, m, C, tg)
    assert_parity(at_targets(host(L), tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(host(Lc), tg), Lco, Sc, what="Lc")


@pytest.mark.parametrize("seed", [93, 94])
def test_com_random_moments_random_centres(ot, orc, seed):
    """Random moments of every order about centres scattered inside their
    cells: every contraction term, and the angular term with target and
    source octupoles, at non-integer separations."""
    tree = synth.single_subgrid(1, 0.5)
    M = synth.random_moments(tree, seed=seed)
    rng = np.random.default_rng(seed + 100)
    h = tree.h(1)
    C = geometric_centres(tree) + rng.uniform(-0.3, 0.3, size=(1, 3, 512)) * h
    g = ot.OTGrid.from_tree(tree)
    L, Lc = g.interactions_com(dev(M), None, dev(C))
    L2, Lc2 = g.multipole(dev(M), centres=dev(C))
    torch.cuda.synchronize()
    r = orc.run_pass_grid(tree, "multipole", M=M, centres=C)
    assert_parity(host(L), r["L"], fwd_scale(r), what="L", kind="L")
    assert_parity(host(Lc), r["Lc"], fwd_scale(r, lc=True), what="Lc")
    assert np.max(np.abs(r["Lc"])) > 0
    assert torch.equal(L, L2) and torch.equal(Lc, Lc2)


def test_com_monopole_only_and_split_passes(ot, orc):
    """m-only call against the oracle's point-mass pass, and the two single
    passes summing to the fused call."""
    tree = _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=95)
    M, m, C = oracle_com_inputs(orc, tree, rho)
    g = ot.OTGrid.from_tree(tree)
    L2, _ = g.interactions_com(None, dev(m), dev(C))
    L1, Lc1 = g.interactions_com(dev(M), None, dev(C))
    L, Lc = g.interactions_com(dev(M), dev(m), dev(C))
    torch.cuda.synchronize()
    r2 = orc.run_pass_grid(tree, "monopole", m=m, centres=C)
    assert_parity(host(L2), r2["L"], fwd_scale(r2), what="L (point masses)", kind="L")
    r1 = orc.run_pass_grid(tree, "multipole", M=M, centres=C)
    S = fwd_scale(r1) + fwd_scale(r2)
    assert_parity(host(L1) + host(L2), host(L), S, what="split vs fused", kind="L")
    assert torch.equal(Lc, Lc1)


def test_com_path_with_geometric_centres_matches_table_path(ot, orc):
    """Geometric centres through the per-pair path give the table path's
    result (both against the geometric-centre oracle)."""
    tree = _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=96)
    M = orc.moments(tree, rho)
    m = np.ascontiguousarray(M[:, 0, :])
    C = geometric_centres(tree)
    g = ot.OTGrid.from_tree(tree)
    Lcom, Lccom = g.interactions_com(dev(M), dev(m), dev(C))
    Ltab, Lctab = g.interactions(dev(M), dev(m))
    torch.cuda.synchronize()
    tg = all_targets(tree)
    r1 = orc.run_pass(tree, "multipole", M=M, targets=tg)
    r2 = orc.run_pass(tree, "monopole", m=m, targets=tg)
    for L, Lc in ((Lcom, Lccom), (Ltab, Lctab)):
        assert_parity(at_targets(host(L), tg), r1["L"] + r2["L"], fwd_scale(r1) + fwd_scale(r2), what="L", kind="L")
        assert_parity(at_targets(host(Lc), tg), r1["Lc"], fwd_scale(r1, lc=True), what="Lc")


# ---------------------------------------------------------------------------
# adjoint with the centres held fixed
# ---------------------------------------------------------------------------

def _sparse_lbar(tree, count, seed):
    rng = np.random.default_rng(seed)
    tg = np.unique(np.stack([rng.integers(0, tree.n, count), rng.integers(0, 512, count)], 1), axis=0)
    Lbar = np.zeros((tree.n, 20, 512))
    Lbar[tg[:, 0], :, tg[:, 1]] = rng.standard_normal((len(tg), 20))
    return Lbar, tg.astype(np.int32)


@pytest.mark.parametrize("deterministic", [False, True])
@pytest.mark.parametrize("which", ["uniform", "adaptive", "leaf_level"])
def test_com_adjoint_matches_oracle(ot, orc, which, deterministic):
    tree = TREES[which]()
    rho = synth.uniform_random_density(tree, seed=97)
    _, _, C = oracle_com_inputs(orc, tree, rho)
    Lbar, tg = _sparse_lbar(tree, 300, 98)
    g = ot.OTGrid.from_tree(tree)
    g.set_deterministic(deterministic)
    Cg = C.copy()
    Cg[tree.is_leaf == 1] = np.nan
    Mb, mb = g.backward_com(dev(Lbar), dev(Cg))
    torch.cuda.synchronize()
    g.check()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar, targets=tg, centres=C)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=tg, centres=C)
    assert_parity(host(Mb), Mo, SM, what="Mbar", kind="Mbar")
    assert_parity(host(mb), mo, Sm, what="mbar")
    assert np.max(np.abs(mo)) > 0


def test_com_adjoint_dot_product_binary_star(ot, orc):
    """<L(M, m; C), Lbar> = <M, Mbar> + <m, mbar> on the binary-star octree
    (levels 3-7, virtual descendants) with dense N(0, 1) Lbar."""
    tree, rho = synth.config5_step(0)
    M, m, C = oracle_com_inputs(orc, tree, rho)
    rng = np.random.default_rng(99)
    Mr = synth.random_moments(tree, seed=100)
    Lbar = dev(rng.standard_normal((tree.n, 20, 512)))
    g = ot.OTGrid.from_tree(tree)
    Md, md, Cd = dev(Mr), dev(m), dev(C)
    L, _ = g.interactions_com(Md, md, Cd, want_lc=False)
    Mb, mb = g.backward_com(Lbar, Cd)
    torch.cuda.synchronize()
    g.check()
    lhs = float((L * Lbar).sum())
    rhs = float((Md * Mb).sum() + (md * mb).sum())
    assert lhs == pytest.approx(rhs, rel=1e-11)


# ---------------------------------------------------------------------------
# down-pass and the full solve
# ---------------------------------------------------------------------------

def test_com_atomic_adjoint_equals_fixed_order(ot, orc):
    tree, rho = synth.config5_step(3)
    _, _, C = oracle_com_inputs(orc, tree, rho)
    Lbar = dev(np.random.default_rng(106).standard_normal((tree.n, 20, 512)))
    g = ot.OTGrid.from_tree(tree)
    Cd = dev(C)
    Mb1, mb1 = g.backward_com(Lbar, Cd)
    g.set_deterministic(True)
    Mb2, mb2 = g.backward_com(Lbar, Cd)
    torch.cuda.synchronize()
    assert torch.equal(Mb1, Mb2)
    scale = float(mb2.abs().max())
    assert float((mb1 - mb2).abs().max()) <= 1e-13 * scale


def test_com_l2l_adjoint_dot_product(ot, orc):
    tree = _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=101)
    _, _, C = oracle_com_inputs(orc, tree, rho)
    rng = np.random.default_rng(102)
    x = rng.standard_normal((tree.n, 20, 512))
    y = rng.standard_normal((tree.n, 20, 512))
    g = ot.OTGrid.from_tree(tree)
    Lx = g.l2l_com(dev(x), dev(C))
    Ly = g.l2l_com_backward(dev(y), dev(C))
    torch.cuda.synchronize()
    assert np.sum(host(Lx) * y) == pytest.approx(np.sum(x * host(Ly)), rel=1e-12)


@pytest.mark.parametrize("which", ["uniform", "adaptive"])
def test_com_full_solve_matches_oracle(ot, orc, which):
    """GPU moments and centres, both passes and the down-pass against the
    oracle's full solve about centres of mass."""
    tree = TREES[which]()
    rho = synth.uniform_random_density(tree, seed=103)
    g = ot.OTGrid.from_tree(tree)
    L, _, _ = g.solve_com(dev(rho))
    torch.cuda.synchronize()
    Lo = orc.full_solve(tree, rho, com=True)
    Mo, Co = orc.moments_com(tree, rho)
    So = full_solve_scale(orc, tree, Mo, np.ascontiguousarray(Mo[:, 0, :]), centres=Co)
    assert_parity(host(L), Lo, So, what="L")


# ---------------------------------------------------------------------------
# full-size workloads, sampled
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("cfg", ["polytrope64", "binary"])
def test_com_full_size_sampled(ot, orc, cfg):
    tree, rho = synth.config2() if cfg == "polytrope64" else synth.config5_step(7)
    M, m, C = oracle_com_inputs(orc, tree, rho)
    g = ot.OTGrid.from_tree(tree)
    L, Lc = g.interactions_com(dev(M), dev(m), dev(C))
    torch.cuda.synchronize()
    g.check()
    tg = np.concatenate([sample_targets(tree, 100, 104), sample_targets(tree, 40, 105, levels=[0, 1, 2])])
    Lo, S, Lco, Sc = oracle_com_passes(orc, tree, M, m, C, tg)
    assert_parity(at_targets(host(L), tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(host(Lc), tg), Lco, Sc, what="Lc")
    # the GPU's own moments and centres on the same tree
    Mg, _, Cg = g.moments_com(dev(rho))
    torch.cuda.synchronize()
    assert np.max(np.abs(host(Cg) - C)) <= 1e-14 * 8.0 * tree.h0
