"""CPU-side checks of the boundary: the shared library loads, exports every
entry point include/ot.h declares, and rejects bad arguments before touching
the device; the generated contraction code is current; the product package
never imports the oracle."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2303_08058_b300")


def header_functions():
    text = open(os.path.join(ROOT, "include", "ot.h")).read()
    return sorted(set(re.findall(r"^(?:ot_status|const char\*)\s+(ot_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_08058_b300 import build, _lib
    build.build()
    return _lib.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_2303_08058_b300 import _lib
    decl = header_functions()
    assert len(decl) >= 14
    assert sorted(_lib.EXPORTS) == decl
    for name in decl:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(PKG, "libotfmm.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (ot_\w+)$", out, flags=re.M))
    assert set(decl) <= exported


def test_library_is_built_for_sm_103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", os.path.join(PKG, "libotfmm.so")],
                         capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_host_argument_checks_without_device(lib):
    from paper_2303_08058_b300 import _lib
    out = ctypes.c_void_p()
    assert lib.ot_grid_create(None, None, ctypes.byref(out)) == _lib.OT_EINVAL
    assert b"desc" in lib.ot_last_error()
    desc = _lib.GridDesc(0, None, None, None, 1.0, 12, 0)
    assert lib.ot_grid_create(ctypes.byref(desc), None, ctypes.byref(out)) == _lib.OT_EINVAL
    lv = np.array([1], np.int32)
    co = np.zeros((1, 3), np.int32)
    lf = np.ones(1, np.uint8)
    desc = _lib.GridDesc(1, lv.ctypes.data, co.ctypes.data, lf.ctypes.data, 1.0, 24, 0)
    assert lib.ot_grid_create(ctypes.byref(desc), None, ctypes.byref(out)) == _lib.OT_ENOTSUP
    desc = _lib.GridDesc(1, lv.ctypes.data, co.ctypes.data, lf.ctypes.data, float("nan"), 12, 0)
    assert lib.ot_grid_create(ctypes.byref(desc), None, ctypes.byref(out)) == _lib.OT_EINVAL
    assert lib.ot_grid_destroy(None) == _lib.OT_OK
    assert lib.ot_set_schedule(None, 0, 4, 0, 1) == _lib.OT_EINVAL
    assert lib.ot_interactions(None, None, None, None, None, None) == _lib.OT_EINVAL
    assert lib.ot_fp64_fma_probe(None, 1, 1, 0, None) == _lib.OT_EINVAL
    assert lib.ot_fp64_fma_probe(ctypes.c_void_p(0x1000), 1, 1, 3, None) == _lib.OT_EINVAL
    assert b"variant" in lib.ot_last_error()
    # the launch counter reads a host counter: no device needed
    assert lib.ot_launch_count(None) == _lib.OT_EINVAL
    cnt = ctypes.c_int64(-1)
    assert lib.ot_launch_count(ctypes.byref(cnt)) == _lib.OT_OK and cnt.value >= 0
    # a pointer that is not a live grid handle is refused before any use
    fake = ctypes.c_void_p(0x1000)
    assert lib.ot_grid_destroy(fake) == _lib.OT_EINVAL
    assert b"not live" in lib.ot_last_error()
    assert lib.ot_grid_info(fake, ctypes.byref(_lib.GridInfo())) == _lib.OT_EINVAL
    assert lib.ot_interactions(fake, None, None, None, None, None) == _lib.OT_EINVAL
    assert lib.ot_multipole_interactions_noalloc(fake, None, None, None, None) == _lib.OT_EINVAL


def test_generated_contraction_code_is_current():
    sys.path.insert(0, os.path.join(PKG, "csrc"))
    try:
        import gen_contract
    finally:
        sys.path.pop(0)
    text = gen_contract.emit()
    assert text == open(os.path.join(PKG, "csrc", "ot_contract.inc")).read()
    assert gen_contract.emit_counts() == open(os.path.join(PKG, "csrc", "ot_contract_counts.h")).read()
    body = text.split("ot_multi_fwd")[1].split("}")[0]
    assert body.count("fma(") == 70
    body = text.split("ot_mono_fwd")[1].split("}")[0]
    assert body.count("fma(") == 16


def test_product_never_touches_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".inc", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "ot_oracle" not in text, f


def test_generated_trees_are_2to1_balanced():
    tree, _, _ = synth.config3()
    idx = tree.index()
    leaves = [(int(l), *map(int, c)) for l, c, f in zip(tree.level, tree.coord, tree.is_leaf) if f]
    leafset = set(leaves)

    def covering_leaf(l, q):
        for d in range(0, l + 1):
            t = (l - d, q[0] >> d, q[1] >> d, q[2] >> d)
            if t in leafset:
                return t
        return None
    for (l, x, y, z) in leaves[::7]:
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    q = (x + dx, y + dy, z + dz)
                    if min(q) < 0 or max(q) >= 2 ** l:
                        continue
                    if (l, *q) in idx and not tree.is_leaf[idx[(l, *q)]]:
                        # refined neighbour: its children touching us must be leaves
                        continue
                    cl = covering_leaf(l, q)
                    assert cl is None or l - cl[0] <= 1


def test_generated_pair_derivatives_match_sympy(tmp_path):
    """The per-pair derivative routines of the explicit-centre kernels,
    compiled as host C++ (they use only fma, sqrt and division), against
    sympy's exact derivatives of -1/r at integer and fractional separations,
    for exactly the components each routine promises."""
    import shutil
    import subprocess

    import sympy
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    sys.path.insert(0, os.path.join(PKG, "csrc"))
    try:
        import gen_contract
    finally:
        sys.path.pop(0)
    text = open(os.path.join(PKG, "csrc", "ot_contract.inc")).read()

    def routine(name):
        start = text.index(f"__device__ __forceinline__ void {name}(")
        return text[start:text.index("\n}\n", start) + 3]
    names = list(gen_contract.DERIV_SETS)
    src = "#include <cmath>\nusing std::fma; using std::sqrt;\n#define __device__\n#define __forceinline__ inline\n"
    for name in names:
        src += routine(name)
        src += (f'extern "C" void c_{name}(double x, double y, double z, double* o) {{ double d[36];'
                f' for (int i = 0; i < 36; ++i) d[i] = 1e300; {name}(x, y, z, d);'
                f' for (int i = 0; i < 36; ++i) o[i] = d[i]; }}\n')
    (tmp_path / "d.cpp").write_text(src)
    so = str(tmp_path / "d.so")
    subprocess.run(["g++", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, str(tmp_path / "d.cpp")],
                   check=True)
    lib = ctypes.CDLL(so)
    x, y, z = sympy.symbols("x y z", real=True)
    G = -1 / sympy.sqrt(x * x + y * y + z * z)
    for R in [(3, -4, 12), (1.25, 0.5, -2.75), (-0.3, 2.2, 0.9), (0, 0, 5), (7, 1, 1)]:
        sub = {x: sympy.Rational(R[0]), y: sympy.Rational(R[1]), z: sympy.Rational(R[2])}
        r = float(np.linalg.norm(R))
        exact = [float(sympy.N(sympy.diff(G, x, e[0], y, e[1], z, e[2]).subs(sub), 40))
                 for e in gen_contract.ROW[:35]]
        for name in names:
            out = (ctypes.c_double * 36)()
            getattr(lib, f"c_{name}")(ctypes.c_double(R[0]), ctypes.c_double(R[1]), ctypes.c_double(R[2]), out)
            want = set(gen_contract.DERIV_SETS[name])
            for q in range(36):
                if q not in want:
                    assert out[q] == 1e300, (name, q)      # untouched
                    continue
                e = gen_contract.ROW[q]
                scale = 1.0 / r ** (sum(e) + 1)
                assert abs(out[q] - exact[q]) <= 1e-14 * max(abs(exact[q]), scale), (name, R, e, out[q], exact[q])


def test_multipole_class_contraction_matches_its_members(tmp_path):
    """The reflection-class contraction of multipole sources, compiled as host
    C++, against the per-source contraction (ot_multi_fwd + ot_angular_fwd)
    of each member with the derivatives at its own offset, for every zero
    pattern, with and without the angular term, and with members missing;
    the variant with the x butterflies prebuilt; the same for the transposed
    gather (ot_multi_adj per target member)."""
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    text = open(os.path.join(PKG, "csrc", "ot_contract.inc")).read()

    def routine(name):
        start = text.index(f"__device__ __forceinline__ void {name}(")
        return text[start:text.index("\n}\n", start) + 3]
    src = ("#include <cmath>\nusing std::fma; using std::sqrt;\n#define __device__\n#define __forceinline__ inline\n"
           "#define __restrict__\n#define __ldg(p) (*(p))\nconstexpr int NCELL = 1;\n")
    for name in ["ot_multi_fwd", "ot_angular_fwd", "ot_multi_adj", "ot_deriv31_at"]:
        src += routine(name)
    for Z in range(7):
        for ang in ("", "_ang"):
            src += routine(f"ot_mclass_fwd_z{Z}{ang}")
        src += routine(f"ot_mclass_adj_z{Z}")
    for Z in (0, 2, 4, 6):
        for ang in ("", "_ang"):
            src += routine(f"ot_mclass_fwd_x_z{Z}{ang}")
    src += "typedef void (*x_fn)(double (&)[16], double (&)[3], double (&)[9], const double* const (&)[4], const double*);\n"
    src += "static x_fn x_table[2][4] = {{" + ", ".join(f"ot_mclass_fwd_x_z{Z}" for Z in (0, 2, 4, 6)) + "}, {" + \
        ", ".join(f"ot_mclass_fwd_x_z{Z}_ang" for Z in (0, 2, 4, 6)) + "}};\n"
    for Z in (0, 2, 4, 6):
        src += routine(f"ot_mclass_adj_x_z{Z}")
    src += "typedef void (*adjx_fn)(double (&)[16], const double* const (&)[4], const double*);\n"
    src += "static adjx_fn adjx_table[4] = {" + ", ".join(f"ot_mclass_adj_x_z{Z}" for Z in (0, 2, 4, 6)) + "};\n"
    src += "typedef void (*adj_fn)(double (&)[16], const double* const (&)[8], const double*);\n"
    src += "static adj_fn adj_table[7] = {" + ", ".join(f"ot_mclass_adj_z{Z}" for Z in range(7)) + "};\n"
    src += "typedef void (*cls_fn)(double (&)[16], double (&)[3], double (&)[9], const double* const (&)[8], const double*);\n"
    src += "static cls_fn table[2][7] = {{" + ", ".join(f"ot_mclass_fwd_z{Z}" for Z in range(7)) + "}, {" + \
        ", ".join(f"ot_mclass_fwd_z{Z}_ang" for Z in range(7)) + "}};\n"
    src += r'''
extern "C" void run_class(int Z, int ang, const double* r, int mask, const double* row, double* out) {
    double a[16] = {0}, c[3] = {0}, t4[9] = {0};
    const double* p[8];
    for (int i = 0; i < 8; ++i) p[i] = ((mask >> i) & 1) ? r + 16 * i : nullptr;
    table[ang][Z](a, c, t4, p, row);
    for (int i = 0; i < 16; ++i) out[i] = a[i];
    for (int i = 0; i < 3; ++i) out[16 + i] = c[i];
    for (int i = 0; i < 9; ++i) out[19 + i] = t4[i];
}
extern "C" void run_members(int ox, int oy, int oz, int ang, const double* r, int mask, double* out) {
    double a[16] = {0}, c[3] = {0}, t4[9] = {0};
    for (int i = 0; i < 8; ++i) {
        if (!((mask >> i) & 1)) continue;
        double d[36] = {0};
        const int sx = (i & 1) ? -ox : ox, sy = (i & 2) ? -oy : oy, sz = (i & 4) ? -oz : oz;
        ot_deriv31_at(-1.0 * sx, -1.0 * sy, -1.0 * sz, d);
        double rr[16];
        for (int q = 0; q < 16; ++q) rr[q] = r[16 * i + q];
        ot_multi_fwd(a, rr, d);
        if (ang) ot_angular_fwd(c, t4, rr, rr[0], d);
    }
    for (int i = 0; i < 16; ++i) out[i] = a[i];
    for (int i = 0; i < 3; ++i) out[16 + i] = c[i];
    for (int i = 0; i < 9; ++i) out[19 + i] = t4[i];
}
extern "C" void run_class_x(int Z, int ang, const double* r, int mask, const double* row, double* out) {
    // the x butterflies of the members at the four (y, z) sign positions
    double S[4][32];
    const double* p[4];
    for (int q = 0; q < 4; ++q) {
        for (int k = 0; k < 16; ++k) {
            const int ip = q << 1, im = (q << 1) | 1;
            const double vp = ((mask >> ip) & 1) ? r[16 * ip + k] : 0.0;
            const double vm = ((mask >> im) & 1) ? r[16 * im + k] : 0.0;
            S[q][2 * k] = vp + vm;
            S[q][2 * k + 1] = vp - vm;
        }
        p[q] = S[q];
    }
    double a[16] = {0}, c[3] = {0}, t4[9] = {0};
    x_table[ang][Z >> 1](a, c, t4, p, row);
    for (int i = 0; i < 16; ++i) out[i] = a[i];
    for (int i = 0; i < 3; ++i) out[16 + i] = c[i];
    for (int i = 0; i < 9; ++i) out[19 + i] = t4[i];
}
extern "C" void run_class_adj(int Z, const double* r, int mask, const double* row, double* out) {
    double g[16] = {0};
    const double* p[8];
    for (int i = 0; i < 8; ++i) p[i] = ((mask >> i) & 1) ? r + 16 * i : nullptr;
    adj_table[Z](g, p, row);
    for (int i = 0; i < 16; ++i) out[i] = g[i];
}
extern "C" void run_class_adj_x(int Z, const double* r, int mask, const double* row, double* out) {
    double S[4][32];
    const double* p[4];
    for (int q = 0; q < 4; ++q) {
        for (int k = 0; k < 16; ++k) {
            const int ip = q << 1, im = (q << 1) | 1;
            const double vp = ((mask >> ip) & 1) ? r[16 * ip + k] : 0.0;
            const double vm = ((mask >> im) & 1) ? r[16 * im + k] : 0.0;
            S[q][2 * k] = vp + vm;
            S[q][2 * k + 1] = vp - vm;
        }
        p[q] = S[q];
    }
    double g[16] = {0};
    adjx_table[Z >> 1](g, p, row);
    for (int i = 0; i < 16; ++i) out[i] = g[i];
}
extern "C" void run_members_adj(int ox, int oy, int oz, const double* r, int mask, double* out) {
    double g[16] = {0};
    for (int i = 0; i < 8; ++i) {
        if (!((mask >> i) & 1)) continue;
        double d[36] = {0};
        const int sx = (i & 1) ? -ox : ox, sy = (i & 2) ? -oy : oy, sz = (i & 4) ? -oz : oz;
        ot_deriv31_at(1.0 * sx, 1.0 * sy, 1.0 * sz, d);     // target at +s*o from the source
        double lb[16];
        for (int q = 0; q < 16; ++q) lb[q] = r[16 * i + q];
        ot_multi_adj(g, lb, d);
    }
    for (int i = 0; i < 16; ++i) out[i] = g[i];
}
extern "C" void row_at(int ox, int oy, int oz, double* out) {
    double d[36] = {0};
    ot_deriv31_at(-1.0 * ox, -1.0 * oy, -1.0 * oz, d);
    for (int q = 0; q < 36; ++q) out[q] = d[q];
}
'''
    (tmp_path / "c.cpp").write_text(src)
    so = str(tmp_path / "c.so")
    subprocess.run(["g++", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, str(tmp_path / "c.cpp")],
                   check=True)
    lib = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    rng = np.random.default_rng(7)
    for (ox, oy, oz) in [(3, 2, 5), (0, 4, 1), (2, 0, 3), (3, 1, 0), (0, 0, 5), (0, 6, 0), (4, 0, 0), (7, 7, 7)]:
        Z = (ox == 0) | ((oy == 0) << 1) | ((oz == 0) << 2)
        allowed = [i for i in range(8) if not (i & Z)]
        row = np.zeros(36)
        lib.row_at(ox, oy, oz, row.ctypes.data_as(dp))
        for ang in (0, 1):
            for trial in range(4):
                mask = sum(1 << i for i in allowed if trial == 0 or rng.random() < 0.6)
                r = rng.standard_normal((8, 16))
                got, want = np.zeros(28), np.zeros(28)
                lib.run_class(Z, ang, r.ctypes.data_as(dp), mask, row.ctypes.data_as(dp), got.ctypes.data_as(dp))
                lib.run_members(ox, oy, oz, ang, r.ctypes.data_as(dp), mask, want.ctypes.data_as(dp))
                scale = np.max(np.abs(want)) + 1e-300
                assert np.max(np.abs(got - want)) <= 1e-13 * scale, ((ox, oy, oz), ang, mask, got - want)
                if not ang:
                    assert np.all(got[16:] == 0)
                if not (Z & 1):       # the x stage prebuilt
                    gx = np.zeros(28)
                    lib.run_class_x(Z, ang, r.ctypes.data_as(dp), mask, row.ctypes.data_as(dp), gx.ctypes.data_as(dp))
                    assert np.max(np.abs(gx - want)) <= 1e-13 * scale, ((ox, oy, oz), ang, mask, "x")
        # the gather by source: targets at +s*o, the table row of -o
        mrow = np.zeros(36)
        lib.row_at(-ox, -oy, -oz, mrow.ctypes.data_as(dp))
        for trial in range(4):
            mask = sum(1 << i for i in allowed if trial == 0 or rng.random() < 0.6)
            r = rng.standard_normal((8, 16))
            got, want = np.zeros(16), np.zeros(16)
            lib.run_class_adj(Z, r.ctypes.data_as(dp), mask, mrow.ctypes.data_as(dp), got.ctypes.data_as(dp))
            lib.run_members_adj(ox, oy, oz, r.ctypes.data_as(dp), mask, want.ctypes.data_as(dp))
            assert np.max(np.abs(got - want)) <= 1e-13 * (np.max(np.abs(want)) + 1e-300), ((ox, oy, oz), mask)
            if not (Z & 1):
                gx = np.zeros(16)
                lib.run_class_adj_x(Z, r.ctypes.data_as(dp), mask, mrow.ctypes.data_as(dp), gx.ctypes.data_as(dp))
                assert np.max(np.abs(gx - want)) <= 1e-13 * (np.max(np.abs(want)) + 1e-300), ((ox, oy, oz), mask)
