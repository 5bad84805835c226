"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: every Taylor coefficient within 1e-12 * S of the oracle, S being the
oracle's sum of |terms| for that coefficient (the two differ in summation
order, FMA contraction and the traceless reduction only).
"""
import numpy as np
import pytest
import torch

import synth
from helpers import adjoint_with_scale, assert_parity, fwd_scale, oracle_threads, sample_targets

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


def oracle_moments(orc, tree, rho):
    """(M, m) from the oracle: inputs of the pass parity tests never come from
    the GPU (the GPU moments are checked against these separately)."""
    M = orc.moments(tree, rho)
    return M, np.ascontiguousarray(M[:, 0, :])


def gpu_fused(ot, tree, rho=None, M=None, m=None, schedule=None, orc=None):
    g = ot.OTGrid.from_tree(tree)
    if schedule is not None:
        g.set_schedule(*schedule)
    if M is None and orc is not None:
        M, m = oracle_moments(orc, tree, rho)
    if M is None:
        Md, md = g.moments(dev(rho))
    else:
        Md, md = dev(M), dev(m)
    L, Lc = g.interactions(Md, md)
    torch.cuda.synchronize()
    g.check()
    return g, host(Md), host(md), host(L), host(Lc)


def oracle_both(orc, tree, M, m, targets=None):
    r1 = orc.run_pass(tree, "multipole", M=M, targets=targets)
    r2 = orc.run_pass(tree, "monopole", m=m, targets=targets)
    return r1["L"] + r2["L"], fwd_scale(r1) + fwd_scale(r2), r1["Lc"], fwd_scale(r1, lc=True), r1["npairs"], r2["npairs"]


def at_targets(L, targets):
    return L[targets[:, 0], :, targets[:, 1]]


def all_targets(tree):
    return np.stack(np.meshgrid(np.arange(tree.n), np.arange(512), indexing="ij"), -1).reshape(-1, 2).astype(np.int32)


# ---------------------------------------------------------------------------
# moments
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["uniform", "adaptive", "single"])
def test_moments_match_oracle(ot, orc, which):
    if which == "uniform":
        tree = synth.uniform_tree(1, 1.0)
    elif which == "adaptive":
        tree = synth.adaptive_tree(lambda l, c, h0: l == 1 and tuple(c) in {(0, 0, 0), (1, 1, 0)}, 1, 3, 32.0)
    else:
        tree = synth.single_subgrid(1, 1.0)
    rho = synth.uniform_random_density(tree, seed=31)
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(dev(rho))
    Mo = orc.moments(tree, rho)
    scale = np.abs(Mo[:, :1, :]) * (tree.h(tree.level)[:, None, None] ** np.array(
        [0] + [1] * 3 + [2] * 6 + [3] * 10)[None, :, None])
    assert np.all(np.abs(host(M) - Mo) <= 1e-14 * scale + 1e-300)
    np.testing.assert_array_equal(host(m), host(M)[:, 0, :])


def test_moments_backward_dot_product(ot):
    tree = synth.adaptive_tree(lambda l, c, h0: l == 1 and tuple(c) == (0, 1, 0), 1, 3, 32.0)
    rng = np.random.default_rng(32)
    rho = rng.uniform(0.5, 1.5, (tree.n, 512))
    Mb = rng.standard_normal((tree.n, 20, 512))
    mb = rng.standard_normal((tree.n, 512))
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(dev(rho))
    rb = g.moments_backward(dev(Mb), dev(mb))
    lhs = np.sum(host(M) * Mb) + np.sum(host(m) * mb)
    rhs = np.sum(rho * host(rb))
    assert lhs == pytest.approx(rhs, rel=1e-12)


# ---------------------------------------------------------------------------
# forward passes, small cases (every cell)
# ---------------------------------------------------------------------------

def test_config1_multipole_all_cells(ot, orc):
    """One isolated sub-grid of multipole cells (monopole + quadrupole moments)."""
    tree, rho = synth.config1()
    g = ot.OTGrid.from_tree(tree)
    M, _ = oracle_moments(orc, tree, rho)
    L, Lc = g.multipole(dev(M))
    torch.cuda.synchronize()
    r = orc.run_pass_grid(tree, "multipole", M=M)
    assert_parity(host(L), r["L"], fwd_scale(r), what="L", kind="L")
    assert_parity(host(Lc), r["Lc"], fwd_scale(r, lc=True), what="Lc")
    assert g.info()["pairs_multipole"] == r["npairs"]


@pytest.mark.parametrize("seed", [41, 42])
def test_single_subgrid_random_moments_all_terms(ot, orc, seed):
    """Random moments of every order exercise every contraction term and the
    angular correction (target and source octupoles)."""
    tree = synth.single_subgrid(1, 0.5)
    M = synth.random_moments(tree, seed=seed)
    g = ot.OTGrid.from_tree(tree)
    L, Lc = g.multipole(dev(M))
    torch.cuda.synchronize()
    r = orc.run_pass_grid(tree, "multipole", M=M)
    assert_parity(host(L), r["L"], fwd_scale(r), what="L", kind="L")
    assert_parity(host(Lc), r["Lc"], fwd_scale(r, lc=True), what="Lc")
    assert np.max(np.abs(r["Lc"])) > 0


def test_root_leaf_subgrid_root_and_near_stencils(ot, orc):
    """A lone root leaf: root stencil (all well-separated pairs) plus near pairs."""
    tree = synth.single_subgrid(0, 1.0, leaf=True)
    rng = np.random.default_rng(43)
    m = rng.uniform(0.5, 1.5, (1, 512))
    g = ot.OTGrid.from_tree(tree)
    L = g.monopole(dev(m))
    torch.cuda.synchronize()
    r = orc.run_pass_grid(tree, "monopole", m=m)
    assert_parity(host(L), r["L"], fwd_scale(r), what="L", kind="L")
    assert g.info()["pairs_monopole"] == r["npairs"] == 512 * 511


def test_monopole_uniform_level(ot, orc):
    tree = synth.uniform_level(1, 1.0)
    rng = np.random.default_rng(44)
    m = rng.uniform(0.5, 1.5, (tree.n, 512))
    g = ot.OTGrid.from_tree(tree)
    L = g.monopole(dev(m))
    torch.cuda.synchronize()
    r = orc.run_pass_grid(tree, "monopole", m=m)
    assert_parity(host(L), r["L"], fwd_scale(r), what="L", kind="L")
    assert g.info()["pairs_monopole"] == r["npairs"]


def test_fused_uniform_tree_with_coarse_levels(ot, orc):
    tree = synth.uniform_tree(1, 1.0)
    rho = synth.uniform_random_density(tree, seed=45)
    g, M, m, L, Lc = gpu_fused(ot, tree, rho, orc=orc)
    tg = all_targets(tree)
    Lo, S, Lco, Sc, n1, n2 = oracle_both(orc, tree, M, m, tg)
    assert_parity(at_targets(L, tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(Lc, tg), Lco, Sc, what="Lc")
    info = g.info()
    assert (info["pairs_multipole"], info["pairs_monopole"]) == (n1, n2)


def _small_adaptive():
    """25 sub-grids: root, 8 at level 1 (two refined), 16 leaves at level 2."""
    def refine(l, c, h0):
        return l == 1 and tuple(c) in {(0, 0, 0), (1, 1, 0)}
    return synth.adaptive_tree(refine, 1, 2, 16.0)


def test_fused_adaptive_virtual_descendants(ot, orc):
    """Mixed levels: virtual descendants of coarse leaves in the halo, near
    pairs with refined (multipole) neighbours, mixed-class warps."""
    tree = _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=46)
    g, M, m, L, Lc = gpu_fused(ot, tree, rho, orc=orc)
    info = g.info()
    assert info["pairs_virtual"] > 0 and info["n_virtual"] > 0
    tg = all_targets(tree)
    Lo, S, Lco, Sc, n1, n2 = oracle_both(orc, tree, M, m, tg)
    assert_parity(at_targets(L, tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(Lc, tg), Lco, Sc, what="Lc")
    assert (info["pairs_multipole"], info["pairs_monopole"]) == (n1, n2)


def _refined_faces_tree():
    """89 sub-grids: levels 0-2 full, two level-2 nodes refined, so that level-2
    leaves have refined face neighbours on each of the three axes and the
    refined nodes (and their parents) have leaf neighbours."""
    def refine(l, c, h0):
        return l == 2 and tuple(c) in {(1, 2, 1), (2, 1, 2)}
    tree = synth.adaptive_tree(refine, 2, 3, 8.0)
    assert tree.n == 1 + 8 + 64 + 16
    return tree


def test_leaf_targets_next_to_refined_faces_every_cell(ot, orc):
    """Leaf targets whose multipole sources sit in refined face neighbours on
    each of the three axes walk those sources paired with their reflections
    along an axis parallel to the refined face (or alone), and non-leaf
    targets their point masses likewise; every cell of the tree against the
    oracle, both passes."""
    tree = _refined_faces_tree()
    rho = synth.uniform_random_density(tree, seed=47)
    g, M, m, L, Lc = gpu_fused(ot, tree, rho, orc=orc)
    tg = all_targets(tree)
    Lo, S, Lco, Sc, n1, n2 = oracle_both(orc, tree, M, m, tg)
    assert_parity(at_targets(L, tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(Lc, tg), Lco, Sc, what="Lc")
    info = g.info()
    assert (info["pairs_multipole"], info["pairs_monopole"]) == (n1, n2)
    # the multipole pass alone (the launch with the axis-pair walk)
    L1, _ = g.multipole(dev(M))
    r1 = orc.run_pass(tree, "multipole", M=M, targets=tg)
    assert_parity(at_targets(host(L1), tg), r1["L"], fwd_scale(r1), what="L multipole pass", kind="L")


def test_separate_passes_equal_fused(ot):
    tree = _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=47)
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(dev(rho))
    L1, Lc1 = g.multipole(M)
    L1 = g.monopole(m, L1)
    L2, Lc2 = g.interactions(M, m)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(Lc1), host(Lc2))
    np.testing.assert_allclose(host(L1), host(L2), rtol=1e-13, atol=1e-13 * np.abs(host(L2)).max())


def test_schedules_are_bitwise_identical(ot):
    """Persistent, graph-replayed and per-sub-grid launches run the same
    per-target summation order: identical bits.  On this small tree every
    sub-grid's items run as list chunks (the cap is the minimum), so the
    chunk combination is part of what must agree."""
    tree = _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=48)
    outs = []
    for sched in [(0, 4, 0, True), (0, 2, 1, False), (1, 4, 0, False), (0, 8, 0, True)]:
        g = ot.OTGrid.from_tree(tree)
        info = g.info()
        assert info["chunked_subgrids"] > 0
        assert 0 < info["fp64_ops_fwd"] < info["ops_fwd"] and 0 < info["fp64_ops_adj"] < info["ops_adj"]
        assert 0 < info["fp64_ops_fwd_multi"] < info["fp64_ops_fwd"]
        assert info["fp64_ops_fwd_multi"] < info["ops_fwd_multi"] < info["ops_fwd"]
        g.set_schedule(*sched)
        g.set_deterministic(True)
        M, m = g.moments(dev(rho))
        for _ in range(2):   # second call replays the graph
            L, Lc = g.interactions(M, m)
        Lb = dev(np.random.default_rng(1).standard_normal((tree.n, 20, 512)))
        Mb, mb = g.backward(Lb)
        torch.cuda.synchronize()
        outs.append([host(L), host(Lc), host(Mb), host(mb)])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------

def _sparse_lbar(tree, count, seed):
    """L-bar non-zero (all 20 components) on `count` random target cells only,
    so the oracle's scatter can be restricted to exactly those targets."""
    rng = np.random.default_rng(seed)
    tg = np.unique(np.stack([rng.integers(0, tree.n, count), rng.integers(0, 512, count)], 1), axis=0)
    Lbar = np.zeros((tree.n, 20, 512))
    Lbar[tg[:, 0], :, tg[:, 1]] = rng.standard_normal((len(tg), 20))
    return Lbar, tg.astype(np.int32)


def test_adjoint_dense_single_subgrid(ot, orc):
    tree = synth.single_subgrid(1, 1.0)
    Lbar = np.random.default_rng(50).standard_normal((1, 20, 512))
    g = ot.OTGrid.from_tree(tree)
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar)
    assert_parity(host(Mb), Mo, SM, what="Mbar", kind="Mbar")
    assert np.all(host(mb) == 0)


@pytest.mark.parametrize("deterministic", [False, True])
@pytest.mark.parametrize("which", ["uniform_tree", "adaptive", "leaf_level"])
def test_adjoint_matches_oracle_transposed_sum(ot, orc, which, deterministic):
    tree = {"uniform_tree": lambda: synth.uniform_tree(1, 1.0),
            "adaptive": _small_adaptive,
            "leaf_level": lambda: synth.uniform_level(1, 1.0)}[which]()
    Lbar, tg = _sparse_lbar(tree, 300, 51)
    g = ot.OTGrid.from_tree(tree)
    g.set_deterministic(deterministic)
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar, targets=tg)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=tg)
    assert_parity(host(Mb), Mo, SM, what="Mbar", kind="Mbar")
    assert_parity(host(mb), mo, Sm, what="mbar")
    assert np.max(np.abs(mo)) > 0


def test_refined_faces_adjoint_against_oracle(ot, orc):
    """The point-mass adjoint by target (non-leaf targets' point masses in
    axis pairs, atomic adds) and the multipole gather on the tree with
    refined faces on all three axes, against the oracle's transposed sums."""
    tree = _refined_faces_tree()
    Lbar, tg = _sparse_lbar(tree, 600, 52)
    g = ot.OTGrid.from_tree(tree)
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    g.check()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar, targets=tg)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=tg)
    assert_parity(host(Mb), Mo, SM, what="Mbar", kind="Mbar")
    assert_parity(host(mb), mo, Sm, what="mbar")
    assert np.max(np.abs(mo)) > 0


def test_atomic_adjoint_equals_fixed_order_adjoint(ot):
    """The default point-mass adjoint (target-ordered, atomic adds) and the
    fixed-order gather agree to rounding on a dense L-bar; the multipole
    half is the same gather in both modes (bitwise equal)."""
    tree = _small_adaptive()
    Lbar = dev(np.random.default_rng(55).standard_normal((tree.n, 20, 512)))
    g = ot.OTGrid.from_tree(tree)
    Mb1, mb1 = g.backward(Lbar)
    g.set_deterministic(True)
    Mb2, mb2 = g.backward(Lbar)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(Mb1), host(Mb2))
    a, b = host(mb1), host(mb2)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


def test_adjoint_dot_product_gpu(ot):
    tree = _small_adaptive()
    rng = np.random.default_rng(52)
    M = synth.random_moments(tree, seed=53)
    m = rng.uniform(0.5, 1.5, (tree.n, 512))
    Lbar = rng.standard_normal((tree.n, 20, 512))
    g = ot.OTGrid.from_tree(tree)
    L, _ = g.interactions(dev(M), dev(m), want_lc=False)
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    lhs = np.sum(host(L) * Lbar)
    rhs = np.sum(M * host(Mb)) + np.sum(m * host(mb))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_autograd_matches_central_differences(ot):
    """loss = sum over probes of (L0)^2 on a small uniform tree; gradient with
    respect to densities via the adjoint kernels against central differences.
    The loss is exactly quadratic in rho, so central differences have no
    truncation error at any step: a relative step of 1e-3 keeps the rounding
    of the two loss evaluations (each a few 1e-15 of the loss, divided by
    the step) near 1e-7 of the derivative."""
    tree = synth.uniform_tree(1, 1.0)
    rho0 = synth.sample_density(tree, lambda x: synth.polytrope_density(x, (8.0, 8.0, 8.0), 6.0))
    leaf_nodes = np.nonzero(tree.is_leaf)[0]
    rng = np.random.default_rng(54)
    probes = np.stack([rng.choice(leaf_nodes, 50), rng.integers(0, 512, 50)], 1)
    g = ot.OTGrid.from_tree(tree)
    rho = dev(rho0).requires_grad_(True)
    L = ot.potential_and_gradient(g, rho)
    loss = (L[probes[:, 0], 0, probes[:, 1]] ** 2).sum()
    loss.backward()
    grad = host(rho.grad)

    def f(r):
        with torch.no_grad():
            Lr = ot.potential_and_gradient(g, dev(r))
            return float((Lr[probes[:, 0], 0, probes[:, 1]] ** 2).sum())
    cells = [(int(n), int(c)) for n, c in zip(rng.choice(leaf_nodes, 16), rng.integers(0, 512, 16))]
    cells += [(0, 100), (int(np.nonzero(tree.level == 0)[0][0]), 7)]   # coarse nodes: gradient 0
    loss0 = float(loss.detach())
    for (n, c) in cells:
        step = 1e-3 * max(rho0[n, c], 1e-3)
        rp, rm = rho0.copy(), rho0.copy()
        rp[n, c] += step
        rm[n, c] -= step
        fd = (f(rp) - f(rm)) / (2 * step)
        scale = max(abs(fd), 1e-6 * np.max(np.abs(grad)))
        noise = 64 * np.finfo(np.float64).eps * abs(loss0) / step
        assert abs(grad[n, c] - fd) <= 1e-6 * scale + noise, (n, c, grad[n, c], fd, noise)


# ---------------------------------------------------------------------------
# full-size workloads in the benchmark's launch configuration (sampled)
# ---------------------------------------------------------------------------

def test_config2_full_size_sampled(ot, orc):
    tree, rho = synth.config2()
    g, M, m, L, Lc = gpu_fused(ot, tree, rho, orc=orc)
    tg = np.concatenate([sample_targets(tree, 96, 61, levels=[3]), sample_targets(tree, 48, 62, levels=[0, 1, 2])])
    Lo, S, Lco, Sc, _, _ = oracle_both(orc, tree, M, m, tg)
    assert_parity(at_targets(L, tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(Lc, tg), Lco, Sc, what="Lc")
    # every leaf cell: potential negative, the field points inward (towards the star centre)
    leaf = tree.level == 3
    assert np.all(L[leaf, 0, :] < 0)


def test_config2_every_coarse_cell(ot, orc):
    """Every cell of levels 0-2 of the 64^3 workload (73 sub-grids, 37,376
    cells: the root's walk, every chunked item, every angular-term lane)
    against the oracle, forward; and the multipole adjoint at every one of
    those cells for an L-bar dense on levels 0-1 and on 512 sampled level-2
    cells (a coarse source is seen by targets of its own level only, so its
    M-bar is the complete transposed sum of that L-bar; the oracle's scatter
    is serial, hence the sample)."""
    tree, rho = synth.config2()
    g, M, m, L, Lc = gpu_fused(ot, tree, rho, orc=orc)
    coarse = np.nonzero(tree.level <= 2)[0]
    assert len(coarse) == 73
    tg = np.stack(np.meshgrid(coarse, np.arange(512), indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
    Lo, S, Lco, Sc, _, _ = oracle_both(orc, tree, M, m, tg)
    assert_parity(at_targets(L, tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(Lc, tg), Lco, Sc, what="Lc")
    del L, Lc
    Lbar = np.zeros((tree.n, 20, 512))
    rng = np.random.default_rng(66)
    lvl2 = tg[tree.level[tg[:, 0]] == 2]
    sp = np.concatenate([tg[tree.level[tg[:, 0]] <= 1], lvl2[rng.choice(len(lvl2), 512, replace=False)]])
    Lbar[sp[:, 0], :, sp[:, 1]] = rng.standard_normal((len(sp), 20))
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar, targets=sp)
    assert_parity(host(Mb)[coarse], Mo[coarse], SM[coarse], what="Mbar", kind="Mbar")
    assert np.all(host(mb) == 0)


def test_config2_adjoint_full_size_dot_product(ot):
    tree, rho = synth.config2()
    rng = np.random.default_rng(63)
    Lbar = rng.standard_normal((tree.n, 20, 512))
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(dev(rho))
    L, _ = g.interactions(M, m, want_lc=False)
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    lhs = np.sum(host(L) * Lbar)
    rhs = np.sum(host(M) * host(Mb)) + np.sum(host(m) * host(mb))
    assert lhs == pytest.approx(rhs, rel=1e-11)


def test_config2_adjoint_sampled_against_oracle(ot, orc):
    """Sampled sources of the full-size adjoint against the oracle's transposed
    sum restricted to those sources (probe-style L-bar: L0 at 1000 cells)."""
    tree, rho = synth.config2()
    probes = synth.config4_probes()
    leaf_nodes = np.nonzero(tree.level == 3)[0]
    Lbar = np.zeros((tree.n, 20, 512))
    Lbar[leaf_nodes[probes // 512], 0, probes % 512] = np.random.default_rng(64).standard_normal(len(probes))
    g = ot.OTGrid.from_tree(tree)
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    tg = np.stack([leaf_nodes[probes // 512], probes % 512], 1).astype(np.int32)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=tg)
    assert_parity(host(mb), mo, Sm, what="mbar")
    assert np.all(host(Mb) == 0)    # L-bar only on leaf cells: no multipole source sees it


@pytest.mark.parametrize("cfg", ["config3", "config5"])
def test_adaptive_workloads_sampled(ot, orc, cfg):
    if cfg == "config3":
        tree, rho, _ = synth.config3()
    else:
        tree, rho = synth.config5_step(0)
    g, M, m, L, Lc = gpu_fused(ot, tree, rho, orc=orc)
    info = g.info()
    assert info["pairs_virtual"] > 0
    tg = sample_targets(tree, 160, 65)
    Lo, S, Lco, Sc, _, _ = oracle_both(orc, tree, M, m, tg)
    assert_parity(at_targets(L, tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(Lc, tg), Lco, Sc, what="Lc")


# ---------------------------------------------------------------------------
# boundary behaviour
# ---------------------------------------------------------------------------

def test_abi_rejects_bad_input(ot):
    lvl = np.array([1, 1], np.int32)
    with pytest.raises(ot.OTError, match="OT_EINVAL"):
        ot.OTGrid(lvl, np.zeros((2, 3), np.int32), np.ones(2, np.uint8), 1.0)      # duplicate node
    with pytest.raises(ot.OTError, match="OT_EINVAL"):
        ot.OTGrid(np.array([1], np.int32), np.array([[2, 0, 0]], np.int32), np.ones(1, np.uint8), 1.0)
    with pytest.raises(ot.OTError, match="OT_EINVAL"):
        ot.OTGrid(np.array([1], np.int32), np.zeros((1, 3), np.int32), np.ones(1, np.uint8), -1.0)
    tree = synth.single_subgrid(1, 1.0)
    g = ot.OTGrid.from_tree(tree)
    M = torch.zeros(1 * 20 * 512 + 1, dtype=torch.float64, device="cuda")
    L = torch.zeros(20 * 512, dtype=torch.float64, device="cuda")
    import ctypes
    from paper_2303_08058_b300 import _lib
    lib = _lib.load()
    st = lib.ot_multipole_interactions(g.handle, ctypes.c_void_p(M.data_ptr() + 8), None,
                                       ctypes.c_void_p(L.data_ptr()), None, None)
    assert st == _lib.OT_EINVAL and b"aligned" in lib.ot_last_error()
    st = lib.ot_multipole_interactions(g.handle, ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(M.data_ptr() + 8),
                                       ctypes.c_void_p(L.data_ptr()), None, None)
    assert st == _lib.OT_EINVAL and b"C is not 16-byte aligned" in lib.ot_last_error()
    st = lib.ot_interactions_com(g.handle, None, None, ctypes.c_void_p(M.data_ptr()),
                                 ctypes.c_void_p(L.data_ptr()), None, None)
    assert st == _lib.OT_EINVAL and b"both NULL" in lib.ot_last_error()
    assert lib.ot_interactions(None, None, None, None, None, None) == _lib.OT_EINVAL
    g.check()
    # a destroyed handle is refused, not used
    g2 = ot.OTGrid.from_tree(tree)
    h = ctypes.c_void_p(g2.handle.value)
    g2.close()
    assert lib.ot_multipole_interactions(h, ctypes.c_void_p(M.data_ptr()), None, ctypes.c_void_p(L.data_ptr()),
                                         None, None) == _lib.OT_EINVAL
    assert b"not live" in lib.ot_last_error()
    assert lib.ot_grid_destroy(h) == _lib.OT_EINVAL
    # the binding checks element counts and devices (the library cannot)
    with pytest.raises(ValueError, match="elements"):
        g.multipole(torch.zeros(20 * 512 - 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError, match="elements"):
        g.interactions(torch.zeros(1, 20, 512, dtype=torch.float64, device="cuda"),
                       torch.zeros(1, 512, dtype=torch.float64, device="cuda"),
                       L=torch.zeros(1, 3, 512, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError, match="float64"):
        g.moments(torch.zeros(1, 512, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError, match="probe writes"):
        ot.fp64_fma_probe(torch.zeros(100, dtype=torch.float64, device="cuda"), 1, 10)


def test_fp64_probe_runs(ot):
    out = torch.zeros(148 * 256, dtype=torch.float64, device="cuda")
    for variant in (0, 1, 2):
        ot.fp64_fma_probe(out, 148, 10, variant)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(host(out))) and np.all(host(out) > 0)


@pytest.mark.parametrize("mechanism", [0, 1, 2, 3, 4])
def test_completion_study_results_and_stats(ot, orc, mechanism):
    """Per-sub-grid launches over 4 streams, whatever signals their
    completion (stream sync, host callback, event polling by the launching
    thread or by a host thread pool, one batched launch), give the oracle's
    result at every cell of the small adaptive tree, and the batched
    launch's bits; the stats are sane."""
    tree = _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=90)
    M, m = oracle_moments(orc, tree, rho)
    g = ot.OTGrid.from_tree(tree)
    L_ref, Lc_ref = g.interactions(dev(M), dev(m))
    stats, L, Lc = g.completion_study(dev(M), dev(m), mechanism, n_streams=4)
    torch.cuda.synchronize()
    tg = all_targets(tree)
    Lo, S, Lco, Sc, _, _ = oracle_both(orc, tree, M, m, tg)
    assert_parity(at_targets(host(L), tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(host(Lc), tg), Lco, Sc, what="Lc")
    np.testing.assert_array_equal(host(Lc), host(Lc_ref))
    scale = np.max(np.abs(host(L_ref)))
    assert np.max(np.abs(host(L) - host(L_ref))) <= 1e-13 * scale
    assert stats["launches"] == (1 if mechanism == 3 else tree.n)
    assert 0 < stats["mean_latency_us"] <= stats["max_latency_us"]
    assert stats["wall_ms"] > 0


def test_launch_count_direct_and_graphed(ot):
    """ot_launch_count: the forward and the adjoint count the same kernels
    whether their calls launch them directly or replay them from CUDA graphs
    (recording a graph counts none)."""
    tree = _small_adaptive()
    rho = dev(synth.uniform_random_density(tree, seed=140))
    Lbar = dev(np.random.default_rng(141).standard_normal((tree.n, 20, 512)))
    counts = []
    for graph in (False, True):
        g = ot.OTGrid.from_tree(tree)
        g.set_schedule(ot.OT_SCHED_PERSISTENT, 4, 0, graph)
        M, m = g.moments(rho)
        L, Lc = g.interactions(M, m)           # records the graphs when enabled
        Mb, mb = g.backward(Lbar)
        torch.cuda.synchronize()
        c0 = ot.launch_count()
        for _ in range(3):
            g.interactions(M, m, L, Lc)
            g.backward(Lbar, Mb, mb)
        torch.cuda.synchronize()
        counts.append(ot.launch_count() - c0)
        g.close()
    assert counts[0] == counts[1] > 0 and counts[0] % 3 == 0, counts


def test_autotune_cache(ot, tmp_path):
    """A tuned tile shape is stored under the tree's and device's key and
    applied without timing by the next grid on the same tree."""
    tree = synth.uniform_tree(1, 1.0)
    rho = synth.uniform_random_density(tree, seed=130)
    cache = str(tmp_path / "tiles.json")
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(dev(rho))
    L, Lc = g.zeros(tree.n, 20, 512), g.zeros(tree.n, 3, 512)
    first = g.autotune(M, m, L, Lc, cache=cache)
    assert not first["cached"]
    g2 = ot.OTGrid.from_tree(tree)
    second = g2.autotune(M, m, L, Lc, cache=cache)
    assert second["cached"]
    info = g2.info()
    assert (info["warps_per_block"], info["blocks_per_sm"]) == (first["warps_per_block"], first["blocks_per_sm"])
    L2, _ = g2.interactions(M, m)
    L1, _ = g.interactions(M, m)
    torch.cuda.synchronize()
    assert torch.equal(L1, L2)
    other = ot.OTGrid.from_tree(synth.uniform_tree(2, 1.0))
    assert other.config_key() != g.config_key()


def test_step_host_matches_separate_calls(ot):
    """The overlapped host-buffer step (copies on a side stream) returns what
    the separate calls return, bit for bit, and again when its buffers are
    reused (fixed-order adjoint, so the comparison is exact)."""
    tree = _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=150)
    Lbar = np.random.default_rng(151).standard_normal((tree.n, 20, 512))
    g = ot.OTGrid.from_tree(tree)
    g.set_deterministic(True)
    rho_pin = torch.as_tensor(rho).pin_memory()
    Lbar_pin = torch.as_tensor(Lbar).pin_memory()
    L_out = torch.empty((tree.n, 20, 512), dtype=torch.float64).pin_memory()
    rb_out = torch.empty((tree.n, 512), dtype=torch.float64).pin_memory()
    M, m = g.moments(dev(rho))
    L, _ = g.interactions(M, m)
    Mb, mb = g.backward(dev(Lbar))
    rb = g.moments_backward(Mb, mb)
    torch.cuda.synchronize()
    work = g.step_host(rho_pin, Lbar_pin, L_out, rb_out)
    torch.cuda.synchronize()
    assert torch.equal(L_out, L.cpu()) and torch.equal(rb_out, rb.cpu())
    L_out.zero_()
    rb_out.zero_()
    g.step_host(rho_pin, Lbar_pin, L_out, rb_out, work)
    torch.cuda.synchronize()
    assert torch.equal(L_out, L.cpu()) and torch.equal(rb_out, rb.cpu())


@pytest.mark.parametrize("seed", [160, 161])
def test_angular_term_conserves_angular_momentum_gpu(ot, seed):
    """The GPU's multipole pass with its angular term on masses and
    octupoles: the total torque (orbital plus spin) over an isolated sub-grid
    vanishes to rounding; without Lc it is O(1)."""
    from helpers import expansion_forces, spin_torques
    tree = synth.single_subgrid(1, 1.0)
    M = synth.random_moments(tree, seed=seed)
    M[0, 1:10, :] = 0.0
    g = ot.OTGrid.from_tree(tree)
    L, Lc = g.multipole(dev(M))
    torch.cuda.synchronize()
    Mc, Lh, Lch = M[0].T, host(L)[0].T, host(Lc)[0].T
    X = synth.cell_centres(tree, 0)
    tau = spin_torques(Mc, Lh)
    F0 = expansion_forces(Mc, Lh)
    F1 = expansion_forces(Mc, Lh, Lch)
    scale = np.sum(np.abs(np.cross(X, F0)))
    T0 = np.linalg.norm(np.sum(np.cross(X, F0) + tau, axis=0))
    T1 = np.linalg.norm(np.sum(np.cross(X, F1) + tau, axis=0))
    assert T0 > 1e-5 * scale
    assert T1 <= 1e-13 * scale, (T0, T1, scale)


@pytest.mark.parametrize("cfg", ["config2", "config3", "config5"])
def test_full_size_random_moment_stress(ot, orc, cfg):
    """The full-size workloads with stress moments (all 20 components
    ~ N(0,1) h^(m+3), masses ~ U[0.5, 1.5] h^3) in place of the physical
    ones: every multipole term and the angular term carry weight at every
    non-leaf source.  Forward at sampled cells of every level, adjoint
    for a sparse L-bar against the oracle's transposed sum."""
    if cfg == "config2":
        tree = synth.config2()[0]
    elif cfg == "config3":
        tree = synth.config3()[0]
    else:
        tree = synth.config5_step(0)[0]
    M = synth.random_moments(tree, seed=91)
    m = np.ascontiguousarray(M[:, 0, :])
    g, _, _, L, Lc = gpu_fused(ot, tree, M=M, m=m)
    levels = np.unique(tree.level)
    tg = np.concatenate([sample_targets(tree, 24, 92 + int(l), levels=[int(l)]) for l in levels])
    Lo, S, Lco, Sc, _, _ = oracle_both(orc, tree, M, m, tg)
    assert_parity(at_targets(L, tg), Lo, S, what="L", kind="L")
    assert_parity(at_targets(Lc, tg), Lco, Sc, what="Lc")
    assert np.abs(Lco).max() > 0
    del L, Lc
    Lbar, sp = _sparse_lbar(tree, 150, 93)
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    g.check()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar, targets=sp)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=sp)
    assert_parity(host(Mb), Mo, SM, what="Mbar", kind="Mbar")
    assert_parity(host(mb), mo, Sm, what="mbar")
