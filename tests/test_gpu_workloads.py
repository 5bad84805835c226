"""Full-size workloads on the GPU: the differentiation workload (loss over
1000 probe cells of the 64^3 polytrope, gradient by the adjoint kernels) and
the rotating binary-star octree, checked against the oracle."""
import numpy as np
import pytest
import torch

import synth
from helpers import adjoint_with_scale, assert_parity, fwd_scale, oracle_full_solve_at, oracle_threads, sample_targets

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


def test_config4_probe_loss_gradient(ot, orc):
    """loss = sum over 1000 seeded probe cells of (L0)^2 on the 64^3 grid;
    d loss / d rho for all 262,144 leaf densities through the adjoint kernels,
    against the oracle's transposed sum and central differences."""
    tree, rho_h = synth.config2()
    leaf_nodes = np.nonzero(tree.level == 3)[0]
    probes = synth.config4_probes()
    pn, pc = leaf_nodes[probes // 512], probes % 512
    g = ot.OTGrid.from_tree(tree)
    rho = dev(rho_h).requires_grad_(True)
    L = ot.potential_and_gradient(g, rho)
    loss = (L[pn, 0, pc] ** 2).sum()
    loss.backward()
    grad = host(rho.grad)
    g.check()

    # oracle: with h = 1, d loss / d rho of a leaf cell is its point-mass
    # adjoint for L-bar = 2 L0 at the probes (leaf moments reach the loss only
    # through their masses; coarse densities are not used at all)
    Lbar = np.zeros((tree.n, 20, 512))
    Lbar[pn, 0, pc] = 2.0 * host(L)[pn, 0, pc]
    tg = np.stack([pn, pc], 1).astype(np.int32)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=tg)
    assert_parity(grad[leaf_nodes], mo[leaf_nodes], Sm[leaf_nodes], what="d loss / d rho")
    assert np.all(grad[tree.level < 3] == 0)

    # central differences, relative step 1e-6, on 64 cells inside the star
    rng = np.random.default_rng(5)
    inside = np.argwhere(rho_h[leaf_nodes] > 1e-3)
    pick = inside[rng.choice(len(inside), 64, replace=False)]

    def f(r):
        with torch.no_grad():
            Lr = ot.potential_and_gradient(g, dev(r))
            return float((Lr[pn, 0, pc] ** 2).sum())
    loss0 = float(loss.detach())
    for (k, c) in pick:
        n = leaf_nodes[k]
        step = 1e-6 * rho_h[n, c]
        rp, rm = rho_h.copy(), rho_h.copy()
        rp[n, c] += step
        rm[n, c] -= step
        fd = (f(rp) - f(rm)) / (2 * step)
        # FD of a quadratic is exact up to rounding: the relative bound, plus
        # one ulp of the loss (the rounding of each loss evaluation) per step
        noise = np.finfo(np.float64).eps * abs(loss0) / step
        assert abs(grad[n, c] - fd) <= 1e-4 * abs(fd) + noise, (n, c, grad[n, c], fd, noise)


@pytest.mark.parametrize("step", [0, 7, 19])
def test_config5_binary_star_steps(ot, orc, step):
    """Rotating binary star on an adaptive octree (levels 3-7, ~8,300 leaves):
    forward of both passes at sampled cells, adjoint against the oracle's
    transposed sum for a sparse L-bar, and the dot-product identity for the
    workload's dense N(0,1) L-bar."""
    tree, rho = synth.config5_step(step)
    g = ot.OTGrid.from_tree(tree)
    Mh = orc.moments(tree, rho)            # oracle inputs never come from the GPU
    mh = np.ascontiguousarray(Mh[:, 0, :])
    M, m = dev(Mh), dev(mh)
    L, Lc = g.interactions(M, m)
    torch.cuda.synchronize()
    info = g.info()
    assert info["pairs_virtual"] > 0 and info["n_virtual"] > 0
    tg = sample_targets(tree, 120, 100 + step)
    r1 = orc.run_pass(tree, "multipole", M=Mh, targets=tg)
    r2 = orc.run_pass(tree, "monopole", m=mh, targets=tg)
    assert_parity(host(L)[tg[:, 0], :, tg[:, 1]], r1["L"] + r2["L"], fwd_scale(r1) + fwd_scale(r2), what="L", kind="L")
    assert_parity(host(Lc)[tg[:, 0], :, tg[:, 1]], r1["Lc"], fwd_scale(r1, lc=True), what="Lc")

    rng = np.random.default_rng(200 + step)
    sp = np.unique(sample_targets(tree, 200, 300 + step), axis=0)
    Lbar = np.zeros((tree.n, 20, 512))
    Lbar[sp[:, 0], :, sp[:, 1]] = rng.standard_normal((len(sp), 20))
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar, targets=sp)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=sp)
    assert_parity(host(Mb), Mo, SM, what="Mbar", kind="Mbar")
    assert_parity(host(mb), mo, Sm, what="mbar")

    Lbar_d = dev(rng.standard_normal((tree.n, 20, 512)))
    L2, _ = g.interactions(M, m, want_lc=False)
    Mb2, mb2 = g.backward(Lbar_d)
    lhs = float((L2 * Lbar_d).sum())
    rhs = float((M * Mb2).sum() + (m * mb2).sum())
    assert lhs == pytest.approx(rhs, rel=1e-11)
    g.check()
    g.close()


@pytest.mark.parametrize("axis", [0, 2])
def test_mirror_symmetry_full_size(ot, axis):
    """The 64^3 workload with its density mirrored across the x (or z)
    mid-plane: the GPU's coefficients of both passes mirror, with the
    components of odd order along that axis negated.  Exercises the +-o
    pairing, the parity-dependent lists and the z-halves of the warp layout."""
    tree, rho = synth.config2()
    rho = rho * (1.0 + 0.3 * np.random.default_rng(120 + axis).random(rho.shape))   # break the star's symmetry
    idx = tree.index()
    exps = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
            (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1),
            (0, 1, 2), (0, 0, 3)]

    def mirror(field):
        out = np.empty_like(field)
        for (l, x, y, z), i in idx.items():
            c = [x, y, z]
            c[axis] = 2 ** l - 1 - c[axis]
            j = idx[(l, *c)]
            f = field[j].reshape(field.shape[1:-1] + (8, 8, 8))            # [..., z, y, x]
            out[i] = np.flip(f, axis=f.ndim - 1 - axis).reshape(field.shape[1:])
        return out
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(dev(rho))
    L, Lc = g.interactions(M, m)
    Mm, mm = g.moments(dev(mirror(rho)))
    Lm, Lcm = g.interactions(Mm, mm)
    torch.cuda.synchronize()
    sign = np.array([-1.0 if e[axis] % 2 else 1.0 for e in exps])[None, :, None]
    want = sign * mirror(host(L))
    scale = np.max(np.abs(host(L)), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(host(Lm) - want) / scale) < 1e-12
    # the angular term is a force: its component along the axis flips
    sc = np.array([-1.0 if a == axis else 1.0 for a in range(3)])[None, :, None]
    want_c = sc * mirror(host(Lc))
    scale_c = np.max(np.abs(host(Lc)), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(host(Lcm) - want_c) / scale_c) < 1e-12


def test_config4_full_solve_probe_loss_gradient(ot, orc):
    """The differentiation workload on the full multilevel potential: loss =
    sum over the 1000 probe cells of Phi^2, Phi = L0 after moments, both
    passes and the down-pass; the gradient for all leaf densities through the
    adjoint chain (down-pass, passes, moments transposed).  Phi at the probes
    against the oracle's full solve there; the gradient against central
    differences."""
    tree, rho_h = synth.config2()
    leaf_nodes = np.nonzero(tree.level == 3)[0]
    probes = synth.config4_probes()
    pn, pc = leaf_nodes[probes // 512], probes % 512
    g = ot.OTGrid.from_tree(tree)
    rho = dev(rho_h).requires_grad_(True)
    L = ot.potential_and_gradient(g, rho, full=True)
    loss = (L[pn, 0, pc] ** 2).sum()
    loss.backward()
    grad = host(rho.grad)
    g.check()

    Mo = orc.moments(tree, rho_h)
    Lo, So = oracle_full_solve_at(orc, tree, Mo, np.ascontiguousarray(Mo[:, 0, :]), list(zip(pn, pc)))
    assert_parity(host(L)[pn, :, pc], Lo, So, what="full-solve L at the probes")

    rng = np.random.default_rng(6)
    inside = np.argwhere(rho_h[leaf_nodes] > 1e-3)
    pick = inside[rng.choice(len(inside), 48, replace=False)]

    def f(r):
        with torch.no_grad():
            Lr = ot.potential_and_gradient(g, dev(r), full=True)
            return float((Lr[pn, 0, pc] ** 2).sum())
    loss0 = float(loss.detach())
    for (k, c) in pick:
        n = leaf_nodes[k]
        step = 1e-6 * rho_h[n, c]
        rp, rm = rho_h.copy(), rho_h.copy()
        rp[n, c] += step
        rm[n, c] -= step
        fd = (f(rp) - f(rm)) / (2 * step)
        noise = np.finfo(np.float64).eps * abs(loss0) / step
        assert abs(grad[n, c] - fd) <= 1e-4 * abs(fd) + noise, (n, c, grad[n, c], fd, noise)


def _boundary_nodes(tree):
    """Leaf nodes with a refined (non-leaf) neighbour of their level, and
    non-leaf nodes with a leaf neighbour of their level or a coarser leaf
    covering a neighbour position (a virtual source)."""
    idx = tree.index()

    def kind(l, q):
        if any(v < 0 or v >= (1 << l) for v in q):
            return None
        j = idx.get((l, *q))
        if j is not None:
            return "leaf" if tree.is_leaf[j] else "multi"
        for d in range(1, l + 1):
            j = idx.get((l - d, *(v >> d for v in q)))
            if j is not None:
                return "leaf" if tree.is_leaf[j] else None
        return None

    leaf_next_multi, multi_next_leaf = [], []
    for i in range(tree.n):
        l, c = int(tree.level[i]), [int(v) for v in tree.coord[i]]
        if l == 0:
            continue
        kinds = {kind(l, (c[0] + dx, c[1] + dy, c[2] + dz))
                 for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1) if (dx, dy, dz) != (0, 0, 0)}
        if tree.is_leaf[i] and "multi" in kinds:
            leaf_next_multi.append(i)
        if not tree.is_leaf[i] and "leaf" in kinds:
            multi_next_leaf.append(i)
    return np.array(leaf_next_multi), np.array(multi_next_leaf)


def test_config5_coarse_fine_targets_sampled(ot, orc):
    """The binary star's first tree at full size, sampled where the walks
    that pair sources with their reflections along one axis run: cells of
    leaf targets next to refined sub-grids (their multipole sources) and of
    non-leaf targets next to leaves (their point masses), forward of both
    passes and the adjoint of a sparse L-bar on those cells."""
    tree, rho = synth.config5_step(0)
    leaves, nonleaves = _boundary_nodes(tree)
    assert len(leaves) > 1000 and len(nonleaves) > 500
    rng = np.random.default_rng(400)
    tg = np.concatenate([
        np.stack([rng.choice(leaves, 96), rng.integers(0, 512, 96)], 1),
        np.stack([rng.choice(nonleaves, 96), rng.integers(0, 512, 96)], 1)]).astype(np.int32)
    tg = np.unique(tg, axis=0)
    g = ot.OTGrid.from_tree(tree)
    Mh = orc.moments(tree, rho)
    mh = np.ascontiguousarray(Mh[:, 0, :])
    L, Lc = g.interactions(dev(Mh), dev(mh))
    torch.cuda.synchronize()
    r1 = orc.run_pass(tree, "multipole", M=Mh, targets=tg)
    r2 = orc.run_pass(tree, "monopole", m=mh, targets=tg)
    assert_parity(host(L)[tg[:, 0], :, tg[:, 1]], r1["L"] + r2["L"], fwd_scale(r1) + fwd_scale(r2), what="L", kind="L")
    assert_parity(host(Lc)[tg[:, 0], :, tg[:, 1]], r1["Lc"], fwd_scale(r1, lc=True), what="Lc")
    Lbar = np.zeros((tree.n, 20, 512))
    Lbar[tg[:, 0], :, tg[:, 1]] = rng.standard_normal((len(tg), 20))
    Mb, mb = g.backward(dev(Lbar))
    torch.cuda.synchronize()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar, targets=tg)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=tg)
    assert_parity(host(Mb), Mo, SM, what="Mbar", kind="Mbar")
    assert_parity(host(mb), mo, Sm, what="mbar")
    g.check()
    g.close()
