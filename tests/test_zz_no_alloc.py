"""The allocation-free multipole entry point, called through the C ABI.

Callers recording a CUDA graph by stream capture, real-time loops that forbid
allocator calls after set-up, and hosts whose device memory belongs to another
allocator cannot let the library cudaMalloc while they call it.
ot_multipole_interactions_noalloc serves them: its scratch lives in one static
device array of fixed size.  This checks that it returns what the regular
entry point returns, on two calls in a row (the second reuses the array with
the first call's contents still in it), that both agree with the oracle,
that a call leaves the device's allocated memory unchanged, and that it
rejects a grid whose multipole sub-grids do not fit the array.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from helpers import assert_parity, fwd_scale, oracle_threads, sample_targets

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


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_multipole_matches_regular_entry_point(ot, orc):
    from paper_2303_08058_b300 import _lib
    lib = _lib.load()
    tree, rho = synth.config2()          # 73 multipole sub-grids: 4.6 MiB of the 16 MiB array
    M = orc.moments(tree, rho)           # the oracle's moments: the comparison below takes no GPU input
    g = ot.OTGrid.from_tree(tree)
    Md = torch.as_tensor(M, device="cuda")
    L_ref, Lc_ref = g.multipole(Md)
    torch.cuda.synchronize()
    L_ref, Lc_ref = L_ref.cpu().numpy(), Lc_ref.cpu().numpy()
    tg = np.concatenate([sample_targets(tree, 64, 171, levels=[0, 1, 2]), sample_targets(tree, 32, 172, levels=[3])])
    r = orc.run_pass(tree, "multipole", M=M, targets=tg)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [torch.empty((tree.n, 20, 512), dtype=torch.float64, device="cuda") for _ in range(2)]
    outcs = [torch.empty((tree.n, 3, 512), dtype=torch.float64, device="cuda") for _ in range(2)]
    # the first call on the device sets up the array's address
    assert lib.ot_multipole_interactions_noalloc(g.handle, _p(Md), _p(outs[0]), _p(outcs[0]), stream) == _lib.OT_OK
    torch.cuda.synchronize()
    for call in range(2):
        L, Lc = outs[call], outcs[call]
        L.fill_(np.nan)
        Lc.fill_(np.nan)
        torch.cuda.synchronize()
        alloc0 = torch.cuda.memory_allocated()
        free0, _ = torch.cuda.mem_get_info()
        st = lib.ot_multipole_interactions_noalloc(g.handle, _p(Md), _p(L), _p(Lc), stream)
        assert st == _lib.OT_OK, lib.ot_last_error()
        torch.cuda.synchronize()
        # the call allocated nothing, neither through torch nor from the device
        assert torch.cuda.memory_allocated() == alloc0
        assert torch.cuda.mem_get_info()[0] == free0
        Ln, Lcn = L.cpu().numpy(), Lc.cpu().numpy()
        # another instruction path (FP64, no x tables, no chunks): the
        # regular entry point's result within the parity bar, per coefficient
        # scale of the oracle, and the oracle's own values
        Lt = Ln[tg[:, 0], :, tg[:, 1]]
        assert_parity(Lt, r["L"], fwd_scale(r), what=f"call {call}: L vs oracle", kind="L")
        assert_parity(Lcn[tg[:, 0], :, tg[:, 1]], r["Lc"], fwd_scale(r, lc=True), what=f"call {call}: Lc vs oracle")
        assert_parity(Lt, L_ref[tg[:, 0], :, tg[:, 1]], fwd_scale(r), tol=2e-12, what=f"call {call}: L vs regular",
                      kind="L")
        scale = np.max(np.abs(L_ref), axis=(0, 2), keepdims=True)
        assert np.all(np.abs(Ln - L_ref) <= 1e-12 * scale), f"call {call}"
        cscale = np.max(np.abs(Lc_ref), axis=(0, 2), keepdims=True)
        assert np.all(np.abs(Lcn - Lc_ref) <= 1e-12 * cscale), f"call {call}"
    g.check()
    g.close()


def test_noalloc_rejects_grids_beyond_its_scratch(ot):
    from paper_2303_08058_b300 import _lib
    lib = _lib.load()
    # 300 childless multipole sub-grids at level 5: 300 x 64 KiB > 16 MiB
    coord = np.array([[x, y, 0] for y in range(10) for x in range(30)], dtype=np.int32)
    g = ot.OTGrid(np.full(300, 5, np.int32), coord, np.zeros(300, np.uint8), 32.0)
    M = torch.zeros((300, 20, 512), dtype=torch.float64, device="cuda")
    L = torch.zeros((300, 20, 512), dtype=torch.float64, device="cuda")
    st = lib.ot_multipole_interactions_noalloc(g.handle, _p(M), _p(L), None, None)
    assert st == _lib.OT_EINVAL
    assert b"static scratch holds 256" in lib.ot_last_error()
    assert lib.ot_multipole_interactions_noalloc(None, _p(M), _p(L), None, None) == _lib.OT_EINVAL
    g.close()
