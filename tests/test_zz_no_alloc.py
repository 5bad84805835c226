"""The allocation-free multipole entry point, called through the C ABI.

Callers recording a CUDA graph by stream capture, real-time loops that forbid
allocator calls after set-up, and hosts whose device memory belongs to another
allocator cannot let the library cudaMalloc while they call it.
ot_multipole_interactions_noalloc serves them: its scratch lives in one static
device array of fixed size.  This checks that it returns what the regular
entry point returns, on two calls in a row (the second reuses the array with
the first call's contents still in it), and that it rejects a grid whose
multipole sub-grids do not fit the array.
"""
import ctypes

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


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_multipole_matches_regular_entry_point(ot):
    from paper_2303_08058_b300 import _lib
    lib = _lib.load()
    tree, rho = synth.config2()          # 73 multipole sub-grids: 4.6 MiB of the 16 MiB array
    g = ot.OTGrid.from_tree(tree)
    M, m = g.moments(torch.as_tensor(rho, device="cuda"))
    L_ref, Lc_ref = g.multipole(M)
    torch.cuda.synchronize()
    L_ref, Lc_ref = L_ref.cpu().numpy(), Lc_ref.cpu().numpy()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        L = torch.full((tree.n, 20, 512), np.nan, dtype=torch.float64, device="cuda")
        Lc = torch.full((tree.n, 3, 512), np.nan, dtype=torch.float64, device="cuda")
        st = lib.ot_multipole_interactions_noalloc(g.handle, _p(M), _p(L), _p(Lc), stream)
        assert st == _lib.OT_OK, lib.ot_last_error()
        torch.cuda.synchronize()
        Ln, Lcn = L.cpu().numpy(), Lc.cpu().numpy()
        # same kernels and summation order: equal within the parity tolerance
        # (1e-12 of each coefficient's scale) -- in practice bit for bit
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
