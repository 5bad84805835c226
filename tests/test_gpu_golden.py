"""GPU parity against the stored expected values of tests/golden/.

The same seeded inputs the fixtures were written from (an adaptive tree with
virtual descendants, stress moments in all 20 components, a sparse L-bar) go
through the C ABI; the results at the stored cells must lie within
1e-12 * S of the stored oracle values, S summed over each order block as in
the other parity tests.  No oracle code runs here.
"""
import numpy as np
import pytest
import torch

from helpers import (assert_parity, golden_adjoint_columns, golden_forward_columns, load_golden,
                     load_golden_script)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2303_08058_b300 as ot
    ot.load()
    mg = load_golden_script()
    tree = mg.small_adaptive_tree()
    M, m, targets, Lbar, lbar_cells = mg.inputs(tree)
    return ot, tree, M, m, Lbar


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_gpu_forward_matches_golden(case):
    ot, tree, M, m, _ = case
    tg, L, S, Lc, Sc = golden_forward_columns(load_golden("forward_small_adaptive.txt"))
    g = ot.OTGrid.from_tree(tree)
    Lg, Lcg = g.interactions(_dev(M), _dev(m))
    torch.cuda.synchronize()
    g.check()
    Lg, Lcg = Lg.cpu().numpy(), Lcg.cpu().numpy()
    assert_parity(Lg[tg[:, 0], :, tg[:, 1]], L, S, what="L", kind="L")
    assert_parity(Lcg[tg[:, 0], :, tg[:, 1]], Lc, Sc, what="Lc")


@pytest.mark.parametrize("deterministic", [False, True])
def test_gpu_adjoint_matches_golden(case, deterministic):
    ot, tree, _, _, Lbar = case
    cells, Mb, SM, mb, Sm = golden_adjoint_columns(load_golden("adjoint_small_adaptive.txt"))
    g = ot.OTGrid.from_tree(tree)
    g.set_deterministic(deterministic)
    Mbg, mbg = g.backward(_dev(Lbar))
    torch.cuda.synchronize()
    g.check()
    Mbg, mbg = Mbg.cpu().numpy(), mbg.cpu().numpy()
    assert_parity(Mbg[cells[:, 0], :, cells[:, 1]], Mb, SM, what="Mbar", kind="Mbar")
    assert_parity(mbg[cells[:, 0], cells[:, 1]], mb, Sm, what="mbar")
