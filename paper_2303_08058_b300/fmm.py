"""Python face of the library: a grid handle over the C ABI and the autograd
Function.  Device memory and streams come from PyTorch; every step of the
interaction path (moments, both passes, adjoints) runs in libotfmm's kernels.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np
import torch

from . import _lib

NCOMP = 20
NCELL = 512


def _ptr(t):
    if t is None:
        return None
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class OTGrid:
    """Handle of one octree of 8^3 sub-grids on the current CUDA device.

    level [n], coord [n, 3], is_leaf [n] describe the nodes (see include/ot.h);
    h0 is the cell size at level 0.
    """

    def __init__(self, level, coord, is_leaf, h0: float, stream=None):
        self.lib = _lib.load()
        self.level = np.ascontiguousarray(level, dtype=np.int32)
        self.coord = np.ascontiguousarray(coord, dtype=np.int32).reshape(-1, 3)
        self.is_leaf = np.ascontiguousarray(is_leaf, dtype=np.uint8)
        self.n = int(self.level.shape[0])
        self.h0 = float(h0)
        self.device = torch.device("cuda", torch.cuda.current_device())
        desc = _lib.GridDesc(self.n, self.level.ctypes.data, self.coord.ctypes.data, self.is_leaf.ctypes.data,
                             self.h0, 12, 0)
        handle = ctypes.c_void_p()
        _lib.check(self.lib.ot_grid_create(ctypes.byref(desc), _stream(stream), ctypes.byref(handle)))
        self.handle = handle

    @classmethod
    def from_tree(cls, tree, stream=None):
        return cls(tree.level, tree.coord, tree.is_leaf, tree.h0, stream=stream)

    # -- lifetime ------------------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.check(self.lib.ot_grid_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers -------------------------------------------------------------------
    def _p(self, t, comps):
        """Pointer of a [n][comps][512] float64 tensor on this grid's device;
        the library cannot check sizes, so the binding does."""
        if t is None:
            return None
        if t.numel() != self.n * comps * NCELL:
            raise ValueError(f"expected {self.n} x {comps} x {NCELL} elements, got shape {tuple(t.shape)}")
        if t.device != self.device:
            raise ValueError(f"tensor on {t.device}, grid on {self.device}")
        return _ptr(t)

    def zeros(self, *shape):
        return torch.zeros(*shape, dtype=torch.float64, device=self.device)

    def info(self) -> dict:
        out = _lib.GridInfo()
        _lib.check(self.lib.ot_grid_info(self.handle, ctypes.byref(out)))
        return out.as_dict()

    def check(self, stream=None):
        _lib.check(self.lib.ot_grid_check(self.handle, _stream(stream)))

    def set_schedule(self, schedule=_lib.OT_SCHED_PERSISTENT, warps_per_block=4, blocks_per_sm=0, use_graph=True):
        _lib.check(self.lib.ot_set_schedule(self.handle, int(schedule), int(warps_per_block), int(blocks_per_sm),
                                            int(bool(use_graph))))

    def set_precision(self, mode=_lib.OT_PREC_FP64):
        """OT_PREC_FP64, or OT_PREC_DF64_POINT_MASS (double-float point-mass
        contractions on the FP32 pipe, see include/ot.h)."""
        _lib.check(self.lib.ot_set_precision(self.handle, int(mode)))

    def set_deterministic(self, on=True):
        """Fixed-order (bit-reproducible) adjoint instead of the atomic one."""
        _lib.check(self.lib.ot_set_deterministic(self.handle, int(bool(on))))

    def config_key(self) -> str:
        """Hash of the tree and the device: the key of a tuned tile shape."""
        h = hashlib.sha1()
        for a in (self.level, self.coord, self.is_leaf, np.float64(self.h0)):
            h.update(np.ascontiguousarray(a).tobytes())
        h.update(torch.cuda.get_device_name(self.device).encode())
        return h.hexdigest()

    def autotune(self, M, m, L, Lc=None, stream=None, cache=None):
        """Time the fused launch over tile shapes and keep the fastest.  With
        ``cache`` (a JSON file path) a shape tuned before for the same tree on
        the same device is applied without timing, and new results are added."""
        key = self.config_key()
        if cache is not None and os.path.exists(cache):
            with open(cache) as f:
                hit = json.load(f).get(key)
            if hit is not None:
                self.set_schedule(_lib.OT_SCHED_PERSISTENT, hit["warps_per_block"], hit["blocks_per_sm"],
                                  bool(self.info()["graphs_enabled"]))
                return dict(hit, cached=True)
        w, b, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _lib.check(self.lib.ot_autotune(self.handle, self._p(M, NCOMP), self._p(m, 1), self._p(L, NCOMP),
                                        self._p(Lc, 3), _stream(stream), ctypes.byref(w), ctypes.byref(b),
                                        ctypes.byref(ms)))
        out = dict(warps_per_block=w.value, blocks_per_sm=b.value, ms=ms.value)
        if cache is not None:
            table = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    table = json.load(f)
            table[key] = out
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1)
            os.replace(tmp, cache)
        return dict(out, cached=False)

    def completion_study(self, M, m, mechanism, n_streams=1, timeout_s=60.0, L=None, Lc=None):
        """Per-sub-grid launches with completion signalled by mechanism 0 (stream
        sync), 1 (host callback), 2 (event polling by the launching thread),
        4 (event polling by a pool of host threads) or 3 (one batched launch)."""
        L = L if L is not None else self.zeros(self.n, NCOMP, NCELL)
        Lc = Lc if Lc is not None else self.zeros(self.n, 3, NCELL)
        out = _lib.CompletionStats()
        _lib.check(self.lib.ot_completion_study(self.handle, self._p(M, NCOMP), self._p(m, 1), self._p(L, NCOMP),
                                                self._p(Lc, 3), int(mechanism), int(n_streams), float(timeout_s),
                                                ctypes.byref(out)))
        return {name: getattr(out, name) for name, _ in out._fields_}, L, Lc

    # -- the path ------------------------------------------------------------------
    def moments(self, rho, M=None, m=None, stream=None):
        M = M if M is not None else self.zeros(self.n, NCOMP, NCELL)
        m = m if m is not None else self.zeros(self.n, NCELL)
        _lib.check(self.lib.ot_moments(self.handle, self._p(rho, 1), self._p(M, NCOMP), self._p(m, 1),
                                       _stream(stream)))
        return M, m

    def moments_backward(self, Mbar=None, mbar=None, rhobar=None, stream=None):
        rhobar = rhobar if rhobar is not None else self.zeros(self.n, NCELL)
        _lib.check(self.lib.ot_moments_backward(self.handle, self._p(Mbar, NCOMP), self._p(mbar, 1),
                                                self._p(rhobar, 1), _stream(stream)))
        return rhobar

    def multipole(self, M, L=None, Lc=None, want_lc=True, centres=None, stream=None):
        L = L if L is not None else self.zeros(self.n, NCOMP, NCELL)
        if Lc is None and want_lc:
            Lc = self.zeros(self.n, 3, NCELL)
        _lib.check(self.lib.ot_multipole_interactions(self.handle, self._p(M, NCOMP), self._p(centres, 3),
                                                      self._p(L, NCOMP), self._p(Lc, 3), _stream(stream)))
        return L, Lc

    def monopole(self, m, L=None, stream=None):
        L = L if L is not None else self.zeros(self.n, NCOMP, NCELL)
        _lib.check(self.lib.ot_monopole_interactions(self.handle, self._p(m, 1), self._p(L, NCOMP), _stream(stream)))
        return L

    def interactions(self, M, m, L=None, Lc=None, want_lc=True, stream=None):
        L = L if L is not None else self.zeros(self.n, NCOMP, NCELL)
        if Lc is None and want_lc:
            Lc = self.zeros(self.n, 3, NCELL)
        _lib.check(self.lib.ot_interactions(self.handle, self._p(M, NCOMP), self._p(m, 1), self._p(L, NCOMP),
                                            self._p(Lc, 3), _stream(stream)))
        return L, Lc

    # -- centre-of-mass expansion centres ----------------------------------------
    def moments_com(self, rho, M=None, m=None, C=None, stream=None):
        """(M, m, C): moments about the cells' centres of mass (ot_moments_com)."""
        M = M if M is not None else self.zeros(self.n, NCOMP, NCELL)
        m = m if m is not None else self.zeros(self.n, NCELL)
        C = C if C is not None else self.zeros(self.n, 3, NCELL)
        _lib.check(self.lib.ot_moments_com(self.handle, self._p(rho, 1), self._p(M, NCOMP), self._p(m, 1),
                                           self._p(C, 3), _stream(stream)))
        return M, m, C

    def interactions_com(self, M, m, C, L=None, Lc=None, want_lc=True, stream=None):
        """Both passes (either source may be None) about explicit centres C."""
        L = L if L is not None else self.zeros(self.n, NCOMP, NCELL)
        if Lc is None and want_lc and M is not None:
            Lc = self.zeros(self.n, 3, NCELL)
        _lib.check(self.lib.ot_interactions_com(self.handle, self._p(M, NCOMP), self._p(m, 1), self._p(C, 3),
                                                self._p(L, NCOMP), self._p(Lc, 3), _stream(stream)))
        return L, Lc

    def backward_com(self, Lbar, C, Mbar=None, mbar=None, want=(True, True), stream=None):
        """Adjoint of interactions_com with the centres held fixed."""
        if Mbar is None and want[0]:
            Mbar = self.zeros(self.n, NCOMP, NCELL)
        if mbar is None and want[1]:
            mbar = self.zeros(self.n, NCELL)
        _lib.check(self.lib.ot_interactions_backward_com(self.handle, self._p(Lbar, NCOMP), self._p(C, 3),
                                                         self._p(Mbar, NCOMP), self._p(mbar, 1), _stream(stream)))
        return Mbar, mbar

    def l2l_com(self, L, C, stream=None):
        _lib.check(self.lib.ot_l2l_com(self.handle, self._p(C, 3), self._p(L, NCOMP), _stream(stream)))
        return L

    def l2l_com_backward(self, Lbar, C, stream=None):
        _lib.check(self.lib.ot_l2l_com_backward(self.handle, self._p(C, 3), self._p(Lbar, NCOMP), _stream(stream)))
        return Lbar

    def solve_com(self, rho, stream=None):
        """Full multilevel solve about centres of mass: (L, Lc, C)."""
        M, m, C = self.moments_com(rho, stream=stream)
        L, Lc = self.interactions_com(M, m, C, stream=stream)
        self.l2l_com(L, C, stream=stream)
        return L, Lc, C

    def l2l(self, L, stream=None):
        """In-place down-pass: adds every parent's shifted expansion (ot_l2l)."""
        return _l2l(self, L, stream)

    def l2l_backward(self, Lbar, stream=None):
        return _l2l_backward(self, Lbar, stream)

    def solve(self, rho, stream=None):
        """Full multilevel solve: moments, both passes, L2L.  Returns L (leaf
        L[:,0] is the potential) and Lc."""
        M, m = self.moments(rho, stream=stream)
        L, Lc = self.interactions(M, m, stream=stream)
        self.l2l(L, stream=stream)
        return L, Lc

    def step_buffers(self) -> dict:
        """The device buffers (and the side stream) ``step_host`` works in:
        rho, Lbar, M, m, L, Lc, Mb, mb, rb, allocated once.  Calls that run on
        them directly (moments, interactions, backward, moments_backward)
        replay the same graphs as step_host."""
        return {"copy": torch.cuda.Stream(device=self.device),
                "rho": self.zeros(self.n, NCELL), "Lbar": self.zeros(self.n, NCOMP, NCELL),
                "M": self.zeros(self.n, NCOMP, NCELL), "m": self.zeros(self.n, NCELL),
                "L": self.zeros(self.n, NCOMP, NCELL), "Lc": self.zeros(self.n, 3, NCELL),
                "Mb": self.zeros(self.n, NCOMP, NCELL), "mb": self.zeros(self.n, NCELL),
                "rb": self.zeros(self.n, NCELL)}

    def step_host(self, rho_h, Lbar_h, L_h, rhobar_h, work=None, stream=None):
        """One forward + adjoint step between pinned host buffers: rho_h [n, 512]
        and Lbar_h [n, 20, 512] in; L_h [n, 20, 512] (both passes) and rhobar_h
        [n, 512] (the density adjoint of Lbar through both passes and the
        moments) out; the angular term is computed (work["Lc"]) but stays on
        the device.  The large copies run on a side stream, overlapped with
        the kernels: Lbar uploads (after rho) during the moments and the
        forward, L downloads during the adjoint.  ``work`` (a dict this method fills on
        first use) keeps the device buffers between calls.  Asynchronous on
        ``stream``; the outputs are ready when it completes."""
        main = stream if stream is not None else torch.cuda.current_stream()
        if work is None:
            work = {}
        if not work:
            work.update(self.step_buffers())
        cp = work["copy"]
        rho_in, lbar_in, fwd_done = (torch.cuda.Event() for _ in range(3))
        with torch.cuda.stream(main):
            work["rho"].copy_(rho_h, non_blocking=True)
        rho_in.record(main)
        # the L-bar upload after the densities' (host-to-device copies from two
        # streams can queue on one copy engine, and the moments need rho
        # first); waiting on main also means the previous step released the
        # buffers
        cp.wait_event(rho_in)
        with torch.cuda.stream(cp):
            work["Lbar"].copy_(Lbar_h, non_blocking=True)
            lbar_in.record(cp)
        self.moments(work["rho"], work["M"], work["m"], stream=main)
        self.interactions(work["M"], work["m"], work["L"], work["Lc"], stream=main)
        fwd_done.record(main)
        with torch.cuda.stream(cp):
            cp.wait_event(fwd_done)
            L_h.copy_(work["L"], non_blocking=True)
        main.wait_event(lbar_in)
        self.backward(work["Lbar"], work["Mb"], work["mb"], stream=main)
        self.moments_backward(work["Mb"], work["mb"], work["rb"], stream=main)
        with torch.cuda.stream(main):
            rhobar_h.copy_(work["rb"], non_blocking=True)
        main.wait_stream(cp)
        return work

    def backward(self, Lbar, Mbar=None, mbar=None, want=(True, True), stream=None):
        if Mbar is None and want[0]:
            Mbar = self.zeros(self.n, NCOMP, NCELL)
        if mbar is None and want[1]:
            mbar = self.zeros(self.n, NCELL)
        _lib.check(self.lib.ot_interactions_backward(self.handle, self._p(Lbar, NCOMP), self._p(Mbar, NCOMP),
                                                     self._p(mbar, 1), _stream(stream)))
        return Mbar, mbar


def _l2l(grid, L, stream=None):
    _lib.check(grid.lib.ot_l2l(grid.handle, grid._p(L, NCOMP), _stream(stream)))
    return L


def _l2l_backward(grid, Lbar, stream=None):
    _lib.check(grid.lib.ot_l2l_backward(grid.handle, grid._p(Lbar, NCOMP), _stream(stream)))
    return Lbar


# FMAs one thread runs per round of each probe variant
FP64_PROBE_FMA_PER_ROUND = {0: 16, 1: 16, 2: 1024}


def fp64_fma_probe(out, blocks, iters, variant=0, stream=None):
    """FP64 FMA probe: writes blocks x 256 doubles into ``out``; a thread runs
    FP64_PROBE_FMA_PER_ROUND[variant] FMAs per round."""
    lib = _lib.load()
    if out.numel() < int(blocks) * 256:
        raise ValueError(f"out holds {out.numel()} doubles, the probe writes {int(blocks) * 256}")
    _lib.check(lib.ot_fp64_fma_probe(_ptr(out), int(blocks), int(iters), int(variant), _stream(stream)))


def launch_count() -> int:
    """Kernels the library has launched in this process (graph replays count
    every kernel they hold; recording a graph counts none)."""
    lib = _lib.load()
    n = ctypes.c_int64(0)
    _lib.check(lib.ot_launch_count(ctypes.byref(n)))
    return int(n.value)


class FMMInteractions(torch.autograd.Function):
    """rho [n, 512] -> L [n, 20, 512]: moments and both passes, and with
    ``full`` the L2L down-pass (the complete multilevel solve).

    The backward runs the adjoint kernels (L2L transposed, transposed stencil,
    moments transposed); nothing from the forward pass is stored (every map is
    linear in rho, so the adjoint needs only the grid)."""

    @staticmethod
    def forward(ctx, grid: OTGrid, rho, full: bool = False):
        M, m = grid.moments(rho.contiguous())
        L, _ = grid.interactions(M, m, want_lc=False)
        if full:
            grid.l2l(L)
        ctx.grid, ctx.full = grid, full
        return L

    @staticmethod
    def backward(ctx, Lbar):
        grid = ctx.grid
        Lbar = Lbar.contiguous().clone() if ctx.full else Lbar.contiguous()
        if ctx.full:
            grid.l2l_backward(Lbar)
        Mbar, mbar = grid.backward(Lbar)
        rhobar = grid.moments_backward(Mbar, mbar)
        return None, rhobar, None


def potential_and_gradient(grid: OTGrid, rho, full: bool = False):
    """Differentiable L (potential, gradient, ...) of every cell from rho;
    ``full`` adds the L2L down-pass (the whole multilevel solve)."""
    return FMMInteractions.apply(grid, rho, full)
