"""CPU FP64 oracle of the FMM cell-interaction passes -- TEST INFRASTRUCTURE.

Only ``tests/``, the package's ``smoke()`` check and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never imports, links or
calls it, and the two share no code; both read their inputs from ``synth``.

The arithmetic lives in ``ot_oracle.c`` (plain C, FP64, compiled without fast
math or FMA contraction); this module only builds it and marshals numpy arrays.
See ``ot_oracle.c`` for the formulas and the passage of the paper each follows.

Parity pins (tests/test_oracle_*.py) check it against sympy derivatives,
exact polynomial integrals, brute-force point-mass sums, closed-form
potentials and conservation invariants.  The angular-momentum correction is
pinned by its antisymmetry (Newton III), by its being the missing order-(1,3)
gradient term, and by the exact cancellation of the total torque for masses
and octupoles; that it is the cited method's exact expression is a reading.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ot_oracle.c")
_LIB = os.path.join(_HERE, "libot_oracle.so")
_lib = None

NCOMP = 20
NCELL = 512


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.oracle_D.argtypes = [P, P]
    lib.oracle_D.restype = None
    lib.oracle_comp_exponents.argtypes = [I, P]
    lib.oracle_comp_exponents.restype = I
    lib.oracle_moments.argtypes = [I, P, P, P, ctypes.c_double, P, P]
    lib.oracle_moments.restype = I
    lib.oracle_pass.argtypes = [I, P, P, P, ctypes.c_double, P, P, I, I, P, P, P, P, P]
    lib.oracle_pass.restype = ctypes.c_longlong
    lib.oracle_pass_adjoint.argtypes = [I, P, P, P, ctypes.c_double, I, P, P, P, P]
    lib.oracle_pass_adjoint.restype = I
    lib.oracle_pass_adjoint_targets.argtypes = [I, P, P, P, ctypes.c_double, I, P, P, P, P, I, P]
    lib.oracle_pass_adjoint_targets.restype = ctypes.c_longlong
    lib.oracle_pass_adjoint_centres.argtypes = [I, P, P, P, ctypes.c_double, P, I, P, P, P, P, I, P]
    lib.oracle_pass_adjoint_centres.restype = ctypes.c_longlong
    lib.oracle_moments_com.argtypes = [I, P, P, P, ctypes.c_double, P, P, P]
    lib.oracle_moments_com.restype = I
    lib.oracle_pass_centres.argtypes = [I, P, P, P, ctypes.c_double, P, P, P, I, I, P, P, P, P, P]
    lib.oracle_pass_centres.restype = ctypes.c_longlong
    lib.oracle_pass_scales.argtypes = [I, P, P, P, ctypes.c_double, P, P, P, I, I, P, P, P, P, P, P, P]
    lib.oracle_pass_scales.restype = ctypes.c_longlong
    lib.oracle_pass_adjoint_scales.argtypes = [I, P, P, P, ctypes.c_double, P, I, P, P, P, P, P, I, P]
    lib.oracle_pass_adjoint_scales.restype = ctypes.c_longlong
    lib.oracle_D_abs.argtypes = [P, P]
    lib.oracle_D_abs.restype = None
    lib.oracle_full_solve_com.argtypes = [I, P, P, P, ctypes.c_double, P, I, P, P]
    lib.oracle_full_solve_com.restype = I
    lib.oracle_l2l.argtypes = [P, P, P]
    lib.oracle_l2l.restype = None
    lib.oracle_full_solve.argtypes = [I, P, P, P, ctypes.c_double, P, P, P]
    lib.oracle_full_solve.restype = I
    lib.oracle_set_threads.argtypes = [I]
    lib.oracle_set_threads.restype = None
    lib.oracle_get_threads.argtypes = []
    lib.oracle_get_threads.restype = I
    _lib = lib
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _tree_args(tree):
    level = np.ascontiguousarray(tree.level, dtype=np.int32)
    coord = np.ascontiguousarray(tree.coord, dtype=np.int32)
    leaf = np.ascontiguousarray(tree.is_leaf, dtype=np.uint8)
    return level, coord, leaf


def set_threads(k: int) -> None:
    _load().oracle_set_threads(int(k))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def component_exponents():
    """[35, 3] exponent triples of the stored components (ranks 0..4)."""
    lib = _load()
    out = np.zeros((35, 3), dtype=np.int32)
    e = np.zeros(3, dtype=np.int32)
    for c in range(35):
        lib.oracle_comp_exponents(c, _p(e))
        out[c] = e
    return out


def D(R) -> np.ndarray:
    """Derivatives of G = -1/r of orders 0..4 at R (35 stored components)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.zeros(35)
    _load().oracle_D(_p(R), _p(out))
    return out


def moments(tree, rho) -> np.ndarray:
    """[n, 20, 512] cell moments: uniform-cube moments for childless nodes,
    exact M2M of the children otherwise."""
    level, coord, leaf = _tree_args(tree)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    M = np.zeros((tree.n, NCOMP, NCELL))
    _load().oracle_moments(tree.n, _p(level), _p(coord), _p(leaf), tree.h0, _p(rho), _p(M))
    return M


def moments_com(tree, rho):
    """(M [n,20,512], C [n,3,512]): moments about centre-of-mass expansion centres."""
    level, coord, leaf = _tree_args(tree)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    M = np.zeros((tree.n, NCOMP, NCELL))
    C = np.zeros((tree.n, 3, NCELL))
    _load().oracle_moments_com(tree.n, _p(level), _p(coord), _p(leaf), tree.h0, _p(rho), _p(M), _p(C))
    return M, C


def run_pass(tree, pass_kind: str, M=None, m=None, targets=None, centres=None, with_sd: bool = True):
    """Evaluate one pass for the listed targets ([k, 2] node, cell) or all cells.

    Returns dict(L=[k,20], S=[k,20], npairs=int) plus Lc, Sc ([k,3]) for the
    multipole pass.  ``pass_kind`` is "multipole" (sources = non-leaf cells,
    uses M) or "monopole" (sources = leaf cells and virtual descendants of
    coarser leaves, uses m).  S sums the |terms| of each coefficient; with
    ``with_sd`` SD (and SDc) sums them with every derivative's own terms
    expanded (see ``D_abs``)."""
    level, coord, leaf = _tree_args(tree)
    kind = {"multipole": 1, "monopole": 2}[pass_kind]
    if targets is None:
        nt = tree.n * NCELL
        tg = None
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int32).reshape(-1, 2)
        nt = tg.shape[0]
    Mv = np.ascontiguousarray(M, dtype=np.float64) if M is not None else None
    mv = np.ascontiguousarray(m, dtype=np.float64) if m is not None else None
    if kind == 1 and Mv is None:
        raise ValueError("multipole pass needs M")
    if kind == 2 and mv is None:
        raise ValueError("monopole pass needs m")
    L = np.zeros((nt, NCOMP))
    S = np.zeros((nt, NCOMP))
    Lc = np.zeros((nt, 3))
    Sc = np.zeros((nt, 3))
    SD = np.zeros((nt, NCOMP)) if with_sd else None
    SDc = np.zeros((nt, 3)) if with_sd and kind == 1 else None
    Cv = np.ascontiguousarray(centres, dtype=np.float64) if centres is not None else None
    npairs = _load().oracle_pass_scales(tree.n, _p(level), _p(coord), _p(leaf), tree.h0, _p(Mv), _p(mv), _p(Cv),
                                        kind, nt, _p(tg), _p(L), _p(Lc), _p(S), _p(Sc), _p(SD), _p(SDc))
    out = dict(L=L, S=S, npairs=int(npairs))
    if with_sd:
        out["SD"] = SD
    if kind == 1:
        out.update(Lc=Lc, Sc=Sc)
        if with_sd:
            out["SDc"] = SDc
    return out


def run_pass_grid(tree, pass_kind, M=None, m=None, centres=None):
    """All cells; returns L [n,20,512] (and Lc [n,3,512]) in the library layout."""
    r = run_pass(tree, pass_kind, M=M, m=m, centres=centres)
    n = tree.n
    out = dict(L=r["L"].reshape(n, NCELL, NCOMP).transpose(0, 2, 1).copy(),
               S=r["S"].reshape(n, NCELL, NCOMP).transpose(0, 2, 1).copy(),
               SD=r["SD"].reshape(n, NCELL, NCOMP).transpose(0, 2, 1).copy(), npairs=r["npairs"])
    if "Lc" in r:
        out["Lc"] = r["Lc"].reshape(n, NCELL, 3).transpose(0, 2, 1).copy()
        out["Sc"] = r["Sc"].reshape(n, NCELL, 3).transpose(0, 2, 1).copy()
        out["SDc"] = r["SDc"].reshape(n, NCELL, 3).transpose(0, 2, 1).copy()
    return out


def pass_adjoint(tree, pass_kind: str, Lbar, with_s: bool = False, targets=None, centres=None,
                 with_sd: bool = False):
    """Transposed sum of a pass: Mbar [n,20,512] (multipole) or mbar [n,512];
    with ``with_s`` also the matching sum of |terms| S, and with ``with_sd``
    after it the same sums with every derivative's terms expanded (SD).
    ``targets`` ([k, 2] node, cell) restricts the scatter to those target
    cells; ``centres`` ([n, 3, 512]) are expansion centres held fixed
    (default geometric)."""
    level, coord, leaf = _tree_args(tree)
    kind = {"multipole": 1, "monopole": 2}[pass_kind]
    Lbar = np.ascontiguousarray(Lbar, dtype=np.float64)
    Mbar = np.zeros((tree.n, NCOMP, NCELL))
    mbar = np.zeros((tree.n, NCELL))
    S = np.zeros_like(Mbar if kind == 1 else mbar)
    SD = np.zeros_like(S) if with_sd else None
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int32).reshape(-1, 2)
    Cv = None if centres is None else np.ascontiguousarray(centres, dtype=np.float64)
    npairs = _load().oracle_pass_adjoint_scales(tree.n, _p(level), _p(coord), _p(leaf), tree.h0, _p(Cv), kind,
                                                _p(Lbar), _p(Mbar), _p(mbar), _p(S), _p(SD),
                                                0 if tg is None else tg.shape[0], _p(tg))
    out = Mbar if kind == 1 else mbar
    if with_s == "pairs":
        return out, int(npairs)
    if with_s and with_sd:
        return out, S, SD
    return (out, S) if with_s else out


def D_abs(R) -> np.ndarray:
    """[35] magnitude sums of the terms of each derivative of G = -1/r at R
    (the pairing sum of ``D`` with every term in absolute value)."""
    out = np.zeros(35)
    _load().oracle_D_abs(_p(np.ascontiguousarray(R, dtype=np.float64)), _p(out))
    return out


def l2l(Lp, d) -> np.ndarray:
    Lp = np.ascontiguousarray(Lp, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(NCOMP)
    _load().oracle_l2l(_p(Lp), _p(d), _p(out))
    return out


def full_solve(tree, rho, with_s: bool = False, com: bool = False):
    """[n, 20, 512] total local expansion of every cell (potential = [:, 0]);
    with ``with_s`` also the matching sums of |terms|; ``com`` uses
    centre-of-mass expansion centres (expansions about the cells' centres of
    mass, shifted between them)."""
    level, coord, leaf = _tree_args(tree)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    L = np.zeros((tree.n, NCOMP, NCELL))
    S = np.zeros((tree.n, NCOMP, NCELL)) if with_s else None
    _load().oracle_full_solve_com(tree.n, _p(level), _p(coord), _p(leaf), tree.h0, _p(rho), int(com), _p(L), _p(S))
    return (L, S) if with_s else L
