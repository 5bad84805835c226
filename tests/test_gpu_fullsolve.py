"""The complete multilevel solve on the GPU (moments, both passes, L2L
down-pass) against the oracle's full solve, closed forms, and its adjoint."""
import numpy as np
import pytest
import torch

import synth
from helpers import assert_parity, full_solve_scale, oracle_threads

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
    def refine(l, c, h0):
        return l == 1 and tuple(c) in {(0, 0, 0), (1, 1, 0)}
    return synth.adaptive_tree(refine, 1, 2, 16.0)


@pytest.mark.parametrize("which", ["uniform", "adaptive"])
def test_full_solve_matches_oracle(ot, orc, which):
    tree = synth.uniform_tree(1, 1.0) if which == "uniform" else _small_adaptive()
    rho = synth.uniform_random_density(tree, seed=71)
    g = ot.OTGrid.from_tree(tree)
    L, _ = g.solve(dev(rho))
    torch.cuda.synchronize()
    Lo = orc.full_solve(tree, rho)
    Mo = orc.moments(tree, rho)
    So = full_solve_scale(orc, tree, Mo, np.ascontiguousarray(Mo[:, 0, :]))
    assert_parity(host(L), Lo, So, what="L")


def test_l2l_adjoint_dot_product(ot):
    tree, _ = synth.config2()
    g = ot.OTGrid.from_tree(tree)
    rng = np.random.default_rng(72)
    x = rng.standard_normal((tree.n, 20, 512))
    y = rng.standard_normal((tree.n, 20, 512))
    Lx = g.l2l(dev(x))
    Ly = g.l2l_backward(dev(y))
    torch.cuda.synchronize()
    assert np.sum(host(Lx) * y) == pytest.approx(np.sum(x * host(Ly)), rel=1e-12)


def _leaf_cells(tree):
    ids = np.concatenate([np.stack([np.full(512, i), np.arange(512)], 1) for i in np.nonzero(tree.is_leaf)[0]])
    pos = np.concatenate([synth.cell_centres(tree, i) for i in np.nonzero(tree.is_leaf)[0]])
    return ids, pos


def test_single_mass_full_size_every_pair_once(ot):
    """One unit mass in the 64^3 tree: -1/r at every other leaf cell."""
    tree, _ = synth.config2()
    ids, pos = _leaf_cells(tree)
    rho = np.zeros((tree.n, 512))
    k = 123457
    rho[ids[k, 0], ids[k, 1]] = 1.0
    g = ot.OTGrid.from_tree(tree)
    L, _ = g.solve(dev(rho))
    phi = host(L)[ids[:, 0], 0, ids[:, 1]]
    r = np.linalg.norm(pos - pos[k], axis=1)
    mask = r > 0
    rel = np.abs(phi[mask] + 1.0 / r[mask]) * r[mask]
    assert np.max(rel) < 2e-2, np.max(rel)
    assert phi[k] == 0.0


def test_polytrope_closed_form(ot):
    """n = 1 polytrope, R = 28, rho_c = 1 (G = 1):
    Phi = -(4 rho_c R^2 / pi) (1 + sin(xi)/xi), xi = pi r / R, inside."""
    tree, rho = synth.config2()
    ids, pos = _leaf_cells(tree)
    g = ot.OTGrid.from_tree(tree)
    L, _ = g.solve(dev(rho))
    phi = host(L)[ids[:, 0], 0, ids[:, 1]]
    R = 28.0
    r = np.linalg.norm(pos - 32.0, axis=1)
    xi = np.pi * r / R
    exact = -(4 * R * R / np.pi) * (1 + np.sin(xi) / xi)
    core = r < R / 2
    err = np.max(np.abs(phi[core] - exact[core]) / np.abs(exact[core]))
    assert err < 5e-3, err
    # the field points inwards
    gvec = -host(L)[ids[core, 0], 1:4, ids[core, 1]]
    assert np.all(np.sum(gvec * (pos[core] - 32.0), axis=1) <= 0)


def test_full_solve_autograd_central_differences(ot):
    tree = synth.uniform_tree(1, 1.0)
    rho0 = synth.sample_density(tree, lambda x: synth.polytrope_density(x, (8.0, 8.0, 8.0), 6.0))
    leaf_nodes = np.nonzero(tree.is_leaf)[0]
    rng = np.random.default_rng(73)
    probes = np.stack([rng.choice(leaf_nodes, 40), rng.integers(0, 512, 40)], 1)
    g = ot.OTGrid.from_tree(tree)
    rho = dev(rho0).requires_grad_(True)
    L = ot.potential_and_gradient(g, rho, full=True)
    loss = (L[probes[:, 0], 0, probes[:, 1]] ** 2).sum()
    loss.backward()
    grad = host(rho.grad)

    def f(r):
        with torch.no_grad():
            Lr = ot.potential_and_gradient(g, dev(r), full=True)
            return float((Lr[probes[:, 0], 0, probes[:, 1]] ** 2).sum())
    loss0 = float(loss.detach())
    for n, c in zip(rng.choice(leaf_nodes, 12), rng.integers(0, 512, 12)):
        step = 1e-6 * max(rho0[n, c], 1e-3)
        rp, rm = rho0.copy(), rho0.copy()
        rp[n, c] += step
        rm[n, c] -= step
        fd = (f(rp) - f(rm)) / (2 * step)
        noise = np.finfo(np.float64).eps * abs(loss0) / step
        assert abs(grad[n, c] - fd) <= 1e-4 * abs(fd) + noise, (n, c, grad[n, c], fd)
