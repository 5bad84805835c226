"""Double-float contractions against the oracle: point masses only
(OT_PREC_DF64_POINT_MASS) and the multipole contractions with the angular
term too (OT_PREC_DF64), under the same 1e-12 bound on each coefficient as
the FP64 path."""
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


def _small_adaptive():
    def refine(l, c, h0):
        return l == 1 and tuple(c) in {(0, 0, 0), (1, 1, 0)}
    return synth.adaptive_tree(refine, 1, 2, 16.0)


PRECS = ["point_mass", "both"]


def _prec(ot, name):
    return ot.OT_PREC_DF64_POINT_MASS if name == "point_mass" else ot.OT_PREC_DF64


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["leaf_level", "root_leaf", "adaptive", "uniform_tree"])
def test_df64_all_cells(ot, orc, which, prec):
    tree = {"leaf_level": lambda: synth.uniform_level(1, 1.0),
            "root_leaf": lambda: synth.single_subgrid(0, 1.0, leaf=True),
            "adaptive": _small_adaptive,
            "uniform_tree": lambda: synth.uniform_tree(1, 1.0)}[which]()
    rho = synth.uniform_random_density(tree, seed=81)
    g = ot.OTGrid.from_tree(tree)
    g.set_precision(_prec(ot, prec))
    Mh = orc.moments(tree, rho)            # oracle inputs never come from the GPU
    mh = np.ascontiguousarray(Mh[:, 0, :])
    L, Lc = g.interactions(dev(Mh), dev(mh))
    torch.cuda.synchronize()
    g.check()
    tg = np.stack(np.meshgrid(np.arange(tree.n), np.arange(512), indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
    r1 = orc.run_pass(tree, "multipole", M=Mh, targets=tg)
    r2 = orc.run_pass(tree, "monopole", m=mh, targets=tg)
    got = host(L)[tg[:, 0], :, tg[:, 1]]
    assert_parity(got, r1["L"] + r2["L"], fwd_scale(r1) + fwd_scale(r2), what="L", kind="L")
    assert_parity(host(Lc)[tg[:, 0], :, tg[:, 1]], r1["Lc"], fwd_scale(r1, lc=True), what="Lc")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("cfg", ["config2", "config5"])
def test_df64_full_size_sampled(ot, orc, cfg, prec):
    tree, rho = synth.config2() if cfg == "config2" else synth.config5_step(3)
    g = ot.OTGrid.from_tree(tree)
    Mh = orc.moments(tree, rho)
    mh = np.ascontiguousarray(Mh[:, 0, :])
    M, m = dev(Mh), dev(mh)
    L64, _ = g.interactions(M, m, want_lc=False)
    L64 = host(L64)
    g.set_precision(_prec(ot, prec))
    Ldf, _ = g.interactions(M, m, want_lc=False)
    torch.cuda.synchronize()
    Ldf = host(Ldf)
    tg = sample_targets(tree, 200, 82)
    r2 = orc.run_pass(tree, "monopole", m=mh, targets=tg)
    r1 = orc.run_pass(tree, "multipole", M=Mh, targets=tg)
    assert_parity(Ldf[tg[:, 0], :, tg[:, 1]], r1["L"] + r2["L"], fwd_scale(r1) + fwd_scale(r2), what="L", kind="L")
    # every cell: double-float within 1e-12 of the FP64 path relative to the
    # coefficient-order block magnitude of the FP64 result
    scale = np.max(np.abs(L64), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(Ldf - L64) / scale) < 1e-12


@pytest.mark.parametrize("seed", [140, 141])
def test_df64_random_moments_every_term(ot, orc, seed):
    """Random moments of every order through the double-float multipole
    contraction and angular term (single sub-grid: root, far pairs, paired and
    single entries)."""
    tree = synth.single_subgrid(1, 0.5)
    M = synth.random_moments(tree, seed=seed)
    g = ot.OTGrid.from_tree(tree)
    g.set_precision(ot.OT_PREC_DF64)
    L, Lc = g.multipole(dev(M))
    torch.cuda.synchronize()
    g.check()
    r = orc.run_pass_grid(tree, "multipole", M=M)
    assert_parity(host(L), r["L"], fwd_scale(r), what="L", kind="L")
    assert_parity(host(Lc), r["Lc"], fwd_scale(r, lc=True), what="Lc")


def test_df64_multipole_pass_differs_from_fp64_by_rounding_only(ot):
    """The double-float mode really runs a different arithmetic (results not
    bitwise equal to FP64) yet stays within the bound of the FP64 result."""
    tree, rho = synth.config2()
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(dev(rho))
    L64, Lc64 = g.interactions(M, m)
    L64, Lc64 = host(L64), host(Lc64)
    g.set_precision(ot.OT_PREC_DF64)
    Ldf, Lcdf = g.interactions(M, m)
    torch.cuda.synchronize()
    Ldf, Lcdf = host(Ldf), host(Lcdf)
    assert not np.array_equal(Ldf, L64)
    scale = np.max(np.abs(L64), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(Ldf - L64) / scale) < 1e-12
    scale_c = np.max(np.abs(Lc64), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(Lcdf - Lc64) / scale_c) < 1e-11


def _sparse_lbar(tree, count, seed):
    rng = np.random.default_rng(seed)
    tg = np.unique(np.stack([rng.integers(0, tree.n, count), rng.integers(0, 512, count)], 1), axis=0)
    Lbar = np.zeros((tree.n, 20, 512))
    Lbar[tg[:, 0], :, tg[:, 1]] = rng.standard_normal((len(tg), 20))
    return Lbar, tg.astype(np.int32)


@pytest.mark.parametrize("which", ["uniform_tree", "adaptive", "leaf_level"])
def test_df64_adjoint_matches_oracle(ot, orc, which):
    """The double-float adjoint (multipole gather and point-mass scatter)
    against the oracle's transposed sums under the same 1e-12 bound."""
    tree = {"leaf_level": lambda: synth.uniform_level(1, 1.0),
            "adaptive": _small_adaptive,
            "uniform_tree": lambda: synth.uniform_tree(1, 1.0)}[which]()
    Lbar, tg = _sparse_lbar(tree, 300, 142)
    g = ot.OTGrid.from_tree(tree)
    g.set_precision(ot.OT_PREC_DF64)
    Mb, mb = g.backward(dev(Lbar))
    Mb1, _ = g.backward(dev(Lbar), want=(True, False))      # the multipole half alone
    torch.cuda.synchronize()
    g.check()
    Mo, SM = adjoint_with_scale(orc, tree, "multipole", Lbar, targets=tg)
    mo, Sm = adjoint_with_scale(orc, tree, "monopole", Lbar, targets=tg)
    assert_parity(host(Mb), Mo, SM, what="Mbar", kind="Mbar")
    assert_parity(host(Mb1), Mo, SM, what="Mbar (alone)", kind="Mbar")
    assert_parity(host(mb), mo, Sm, what="mbar")


@pytest.mark.parametrize("cfg", ["config2", "config5"])
def test_df64_adjoint_full_size_close_to_fp64(ot, cfg):
    """Dense N(0,1) L-bar on the full-size grids: the double-float adjoint
    within 1e-12 of the FP64 adjoint relative to each component's largest
    magnitude, and really a different arithmetic."""
    tree, _ = synth.config2() if cfg == "config2" else synth.config5_step(2)
    Lbar = dev(np.random.default_rng(143).standard_normal((tree.n, 20, 512)))
    g = ot.OTGrid.from_tree(tree)
    Mb64, mb64 = g.backward(Lbar)
    g.set_precision(ot.OT_PREC_DF64)
    Mbd, mbd = g.backward(Lbar)
    torch.cuda.synchronize()
    Mb64, mb64, Mbd, mbd = host(Mb64), host(mb64), host(Mbd), host(mbd)
    assert not np.array_equal(Mbd, Mb64)
    sM = np.max(np.abs(Mb64), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(Mbd - Mb64) / np.where(sM > 0, sM, 1.0)) < 1e-12
    assert np.max(np.abs(mbd - mb64)) < 1e-12 * np.max(np.abs(mb64))
