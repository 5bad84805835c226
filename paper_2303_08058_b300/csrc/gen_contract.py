"""Emit ot_contract.inc: straight-line FP64 contraction code for the kernels.

Run as ``python gen_contract.py`` (the build does it when the .inc is stale).

The kernels contract with the *traceless-reduced* index sets.  Every
derivative tensor d^k G of G = -1/r is harmonic (traceless in every index
pair), so

* of a target's 20 Taylor coefficients only the 16 whose multi-index has at
  most one z (``IND16`` below) are accumulated; the other 4 follow per cell
  from zz = -(xx + yy), xzz = -(xxx + xyy), yzz = -(xxy + yyy),
  zzz = -(xxz + yyz);
* a source's second and third moments enter only through 5 and 7 reduced
  combinations (the z-z traces folded into the other components), so the
  16 reduced source moments use the same index set ``IND16``.

With both sides reduced, one multipole pair costs 70 FMAs for the 16
coefficients (instead of 84 with all 20 components), one point-mass pair 16
(instead of 20), and the transposed (adjoint) contractions cost the same.

Paired offsets.  When a target's list holds both o and -o, the two sources
share one table row: d^k G(-R) = (-1)^k d^k G(R), so with the sum s and the
difference d of the two sources' (reduced) moments, every FMA takes s when
its derivative has even order and d when odd.  Two point-mass pairs then
cost 16 FMAs + 2 adds, two multipole pairs 70 FMAs + 32 adds (+ 30 FMAs for
the angular term, whose derivatives are all of order 4); the multipole
adjoint pairs the same way on the two targets' L-bar.

Double-float variants (FP32 pairs hi + lo, see ot_kernels.cu) of the
point-mass contractions read a second table of 32 floats per offset: the
hi parts of the 16 IND16 derivatives, then their lo parts.

Derivative-table row layout (36 doubles per integer offset):
  [0..15]  the IND16 components of ranks 0..3
  [16..19] zz, xzz, yzz, zzz
  [20..34] rank 4 in storage order (xxxx xxxy xxxz xxyy xxyz xxzz xyyy xyyz
           xyzz xzzz yyyy yyyz yyzz yzzz zzzz)
  [35]     padding
"""
import itertools
import os

IND16 = [(0, 0, 0),
         (1, 0, 0), (0, 1, 0), (0, 0, 1),
         (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
         (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (0, 3, 0), (0, 2, 1)]
EXTRA = [(0, 0, 2), (1, 0, 2), (0, 1, 2), (0, 0, 3)]
RANK4 = [tuple(t.count(a) for a in range(3))
         for t in itertools.combinations_with_replacement(range(3), 4)]
ROW = IND16 + EXTRA + RANK4
ROWIDX = {e: i for i, e in enumerate(ROW)}
assert len(ROW) == 35


def rank(e):
    return sum(e)


def add(a, b):
    return tuple(x + y for x, y in zip(a, b))


R3 = [k for k, e in enumerate(IND16) if rank(e) == 3]          # reduced octupole slots 9..15
# independent rank-4 components (at most one z) accumulated for the
# angular term's target-side sum, and the three derived ones
T4 = [e for e in RANK4 if e[2] <= 1]
T4IDX = {e: i for i, e in enumerate(T4)}
assert len(T4) == 9


def t4_expr(e):
    """expression of a rank-4 component (z count <= 2) in the t4[] accumulators"""
    if e[2] <= 1:
        return f"t4[{T4IDX[e]}]"
    # e has zz: d_{..zz} = -d_{..xx} - d_{..yy}
    base = (e[0], e[1], e[2] - 2)
    return f"(-{t4_expr(add(base, (2, 0, 0)))} - {t4_expr(add(base, (0, 2, 0)))})"


def _flops(e):
    """Algorithmic FLOPs of a sympy expression as the emitted code evaluates
    it: n-1 per n-ary sum or product (a factor -1 is a sign, not a product),
    k-1 products for an integer power k."""
    import sympy
    if e.is_Atom:
        return 0
    sub = sum(_flops(a) for a in e.args)
    if e.is_Add:
        return sub + len(e.args) - 1
    if e.is_Mul:
        factors = [a for a in e.args if a != -1]
        return sub + max(len(factors) - 1, 0)
    if e.is_Pow and e.exp.is_Integer and e.exp > 1:
        return _flops(e.base) + int(e.exp) - 1
    raise ValueError(f"unexpected node {e.func}")


# Derivative components each per-pair routine produces (row layout): the
# point-mass contractions read orders 0-3 of the reduced basis (0..15), the
# multipole contractions orders 0-3 with three extra traces (0..18), the
# angular term 12 of the order-4 components (20..28, 30..32).
DERIV_SETS = {
    "ot_deriv16_at": list(range(16)),
    "ot_deriv19_at": list(range(19)),
    "ot_deriv31_at": list(range(19)) + list(range(20, 29)) + [30, 31, 32],
}


def _deriv_plan(indices):
    """Which components of DERIV_SETS' index list are evaluated as polynomials
    and which follow from the Laplace identity d_zz = -d_xx - d_yy: a
    component with two or more z derivatives is -(K + (2,0,-2)) - (K + (0,2,-2)),
    recursively, so only components with at most one z are polynomials."""
    direct, derived = set(), []

    def need(e):
        if e[2] < 2:
            direct.add(e)
            return
        for sub in ((e[0] + 2, e[1], e[2] - 2), (e[0], e[1] + 2, e[2] - 2)):
            need(sub)
        if e not in derived:
            derived.append(e)
    for q in indices:
        need(ROW[q])
    derived.sort(key=lambda e: e[2])          # fewer z first: operands come before their users
    return sorted(direct, key=lambda e: (sum(e), e)), derived


def deriv_flops(name):
    """FLOPs of one call of a generated derivative routine: r^2 (5), 1/sqrt
    (2), r^-2 and the powers r^-(2k+1), the cse'd polynomials, one scaling
    product per polynomial component, two per component from the Laplace
    identity."""
    direct, derived = _deriv_plan(DERIV_SETS[name])
    polys, repl, reduced = _deriv_polys(direct)
    kmax = max(k for k, _ in polys)
    return (5 + 2 + 1 + kmax + sum(_flops(v) for _, v in repl) + sum(_flops(P) for P in reduced) + len(polys)
            + 2 * len(derived))


def _deriv_polys(exps):
    import sympy
    x, y, z = sympy.symbols("x y z", real=True)
    r2 = x * x + y * y + z * z
    G = -1 / sympy.sqrt(r2)
    polys = []
    for e in exps:
        k = rank(e)
        expr = sympy.diff(G, x, e[0], y, e[1], z, e[2]) if k else G
        P = sympy.expand(sympy.simplify(expr * r2 ** sympy.Rational(2 * k + 1, 2)))
        assert P.is_polynomial(x, y, z), (e, P)
        polys.append((k, P))
    repl, reduced = sympy.cse([P for _, P in polys], symbols=sympy.numbered_symbols("t"))
    return polys, repl, reduced


def deriv_code(name):
    """Straight-line code for the derivative components DERIV_SETS[name] of
    G = -1/r at R = (x, y, z): with sympy, d^K G = P_K(x, y, z) r^-(2k+1) for
    a polynomial P_K of degree k (components with at most one z derivative;
    the polynomials share subexpressions, cse), and the components with two
    or more z derivatives from the Laplace identity.  Entries of d outside
    the set are left untouched."""
    import re

    import sympy
    indices = DERIV_SETS[name]
    direct, derived = _deriv_plan(indices)
    polys, repl, reduced = _deriv_polys(direct)
    lines = [f"__device__ __forceinline__ void {name}(double x, double y, double z, double (&d)[36]) {{\n",
             "  const double r2 = fma(x, x, fma(y, y, z * z));\n",
             "  const double ir = 1.0 / sqrt(r2);\n",
             "  const double ir2 = ir * ir;\n",
             "  const double s0 = ir;\n"]
    for k in range(1, max(k for k, _ in polys) + 1):
        lines.append(f"  const double s{k} = s{k - 1} * ir2;\n")

    def cc(e):
        # integer powers as products (no pow calls), integer constants as doubles
        t = sympy.ccode(e)
        t = re.sub(r"pow\((\w+), 4\)", r"((\1 * \1) * (\1 * \1))", t)
        t = re.sub(r"pow\((\w+), 3\)", r"(\1 * \1 * \1)", t)
        t = re.sub(r"pow\((\w+), 2\)", r"(\1 * \1)", t)
        assert "pow" not in t, t
        return re.sub(r"(?<![\w.])(\d+)(?![\w.])", r"\1.0", t)

    def var(e):
        return f"k{e[0]}{e[1]}{e[2]}"
    for sym, val in repl:
        lines.append(f"  const double {sym} = {cc(val)};\n")
    for e, (k, _), P in zip(direct, polys, reduced):
        lines.append(f"  const double {var(e)} = ({cc(P)}) * s{k};\n")
    for e in derived:
        a, b = (e[0] + 2, e[1], e[2] - 2), (e[0], e[1] + 2, e[2] - 2)
        lines.append(f"  const double {var(e)} = -({var(a)} + {var(b)});\n")
    for q in indices:
        lines.append(f"  d[{q}] = {var(ROW[q])};\n")
    lines.append("}\n\n")
    return "".join(lines)


# ---------------------------------------------------------------------------
# reflection classes of multipole sources
#
# The sources at t + s*o (s in {+1, -1}^3 per axis, o >= 0) see one table row
# up to signs: d^K G at -s*o is s^K d^K G at -o, s^K = prod_a s_a^K_a, whose
# value depends only on the parity pattern pi(K) of K.  A term
# a[J] += r_s[K] d[J + K] summed over the members becomes
# d[J + K] * W_K[pi(J) ^ pi(K)], W_K the Walsh-Hadamard transform of the
# members' K-th moments over the sign axes (W_K[pi] = sum_i (-1)^|i & pi|
# r_i[K], member i negated on the axes set in i).  Each source component
# needs only the transform outputs its terms use; an axis with a zero offset
# component (bit set in Z) has one member and its odd-order derivatives are
# exactly zero, so terms with pi & Z drop out.
# ---------------------------------------------------------------------------

def parity(e):
    return (e[0] & 1) | ((e[1] & 1) << 1) | ((e[2] & 1) << 2)


def mclass_terms(Z, ang):
    """per source component k: [(output pi, target kind, index, row index)]"""
    out = {k: [] for k in range(16)}
    for j, ej in enumerate(IND16):
        for k, ek in enumerate(IND16):
            if rank(ej) + rank(ek) <= 3:
                e = add(ej, ek)
                if not (parity(e) & Z):
                    out[k].append((parity(e), "a", j, ROWIDX[e]))
    if ang:
        for i in range(3):
            ei = tuple(1 if a == i else 0 for a in range(3))
            for k in R3:
                e = add(ei, IND16[k])
                if not (parity(e) & Z):
                    out[k].append((parity(e), "c", i, ROWIDX[e]))
        for q, e in enumerate(T4):
            if not (parity(e) & Z):
                out[0].append((parity(e), "t4", q, ROWIDX[e]))
    return out


def transform_plan(Z, need, first=None):
    """butterflies computing the transform outputs `need` of the members
    {i : i & Z == 0}: the stage order with the fewest adds (with `first`, the
    orders starting with that axis; the caller then loads stage 1 instead of
    computing it).  Returns (ops, number of stages) with ops = [(stage,
    index, op, lhs index, rhs index)]."""
    bits = [b for b in range(3) if not (Z >> b) & 1]
    best = None
    for order in itertools.permutations(bits):
        if first is not None and order[0] != first:
            continue
        needed = [None] * (len(order) + 1)
        needed[len(order)] = set(need)
        for t in range(len(order), 0, -1):
            b = 1 << order[t - 1]
            prev = set()
            for x in needed[t]:
                prev |= {x & ~b, x | b}
            needed[t - 1] = prev
        ops = []
        for t in range(1, len(order) + 1):
            b = 1 << order[t - 1]
            for x in sorted(needed[t]):
                lo, hi = x & ~b, x | b
                ops.append((t, x, "+" if x == lo else "-", lo, hi))
        cost = len([op for op in ops if first is None or op[0] > 1])
        if best is None or cost < best[2]:
            best = (ops, len(order), cost)
    return best[0], best[1]


def mclass_fwd_code(Z, ang):
    name = f"ot_mclass_fwd_z{Z}" + ("_ang" if ang else "")
    lines = [f"__device__ __forceinline__ void {name}(double (&a)[16], double (&c)[3], double (&t4)[9],\n"
             f"    const double* const (&src)[8], const double* __restrict__ row) {{\n"]
    members = [i for i in range(8) if not (i & Z)]
    terms = mclass_terms(Z, ang)
    n_add = n_fma = 0
    for k in range(16):
        if not terms[k]:
            continue
        lines.append("  {\n")
        for i in members:
            lines.append(f"    const double v0_{i} = src[{i}] ? __ldg(src[{i}] + {k} * NCELL) : 0.0;\n")
        need = sorted({pi for (pi, _, _, _) in terms[k]})
        ops, nst = transform_plan(Z, need)
        for (t, x, op, lo, hi) in ops:
            lines.append(f"    const double v{t}_{x} = v{t - 1}_{lo} {op} v{t - 1}_{hi};\n")
        n_add += len(ops)
        for (pi, kind, idx, di) in terms[k]:
            w = f"v{nst}_{pi}"
            lines.append(f"    {kind}[{idx}] = fma({w}, __ldg(row + {di}), {kind}[{idx}]);\n")
            n_fma += 1
        lines.append("  }\n")
    lines.append("}\n\n")
    return name, "".join(lines), n_add, n_fma


def mclass_fwd_x_code(Z, ang):
    """ot_mclass_fwd_code with the x stage prebuilt: for a class with a > 0
    (Z without bit 0) the members' x butterflies r(q + a x) +- r(q - a x) at
    the four positions q = t + (0, +-b, +-c) are read from a table built once
    per call (pos[q] points at component 0's sum; its difference and the
    other components follow at stride NCELL)"""
    assert not (Z & 1)
    name = f"ot_mclass_fwd_x_z{Z}" + ("_ang" if ang else "")
    lines = [f"__device__ __forceinline__ void {name}(double (&a)[16], double (&c)[3], double (&t4)[9],\n"
             f"    const double* const (&pos)[4], const double* __restrict__ row) {{\n"]
    terms = mclass_terms(Z, ang)
    n_add = n_fma = n_ld = 0
    for k in range(16):
        if not terms[k]:
            continue
        lines.append("  {\n")
        need = sorted({pi for (pi, _, _, _) in terms[k]})
        ops, nst = transform_plan(Z, need, first=0)
        for (t, x, op, lo, hi) in ops:
            if t == 1:
                q = (x >> 1) & 3
                lines.append(f"    const double v1_{x} = pos[{q}] ? __ldg(pos[{q}] + {2 * k + (x & 1)} * NCELL) : 0.0;\n")
                n_ld += 1
            else:
                lines.append(f"    const double v{t}_{x} = v{t - 1}_{lo} {op} v{t - 1}_{hi};\n")
                n_add += 1
        for (pi, kind, idx, di) in terms[k]:
            lines.append(f"    {kind}[{idx}] = fma(v{nst}_{pi}, __ldg(row + {di}), {kind}[{idx}]);\n")
            n_fma += 1
        lines.append("  }\n")
    lines.append("}\n\n")
    return name, "".join(lines), n_add, n_fma


def xy_plan(Z, need):
    """the transform with the x and y stages prebuilt (order x, y, then z):
    the stage-2 values to load and the z stage's butterflies"""
    order = [0, 1] + ([2] if not (Z >> 2) & 1 else [])
    needed = [None] * (len(order) + 1)
    needed[len(order)] = set(need)
    for t in range(len(order), 0, -1):
        b = 1 << order[t - 1]
        prev = set()
        for x in needed[t]:
            prev |= {x & ~b, x | b}
        needed[t - 1] = prev
    ops = []
    for t in range(3, len(order) + 1):
        b = 1 << order[t - 1]
        for x in sorted(needed[t]):
            lo, hi = x & ~b, x | b
            ops.append((t, x, "+" if x == lo else "-", lo, hi))
    return sorted(needed[2]), ops, len(order)


def mclass_fwd_xy_code(Z, ang):
    """ot_mclass_fwd_code with the x and y stages prebuilt: for a class with
    a, b > 0 (Z without bits 0, 1) whose (x, y) members are all present or all
    absent at each z sign, the transforms over x and y of the members' reduced
    moments at the positions q = t + (0, 0, +-c) are read from a table built
    once per call (pos[r] points at component 0's channel 0 at the z member r,
    0 for +c and 1 for -c; channel ch = x parity + 2 y parity of component k
    at pos[r] + 4 k NCELL + ch: a cell's four channels are adjacent and read
    as two 16-byte pairs)"""
    assert not (Z & 3)
    name = f"ot_mclass_fwd_xy_z{Z}" + ("_ang" if ang else "")
    lines = [f"__device__ __forceinline__ void {name}(double (&a)[16], double (&c)[3], double (&t4)[9],\n"
             f"    const double* const (&pos)[2], const double* __restrict__ row) {{\n"]
    terms = mclass_terms(Z, ang)
    n_add = n_fma = 0
    for k in range(16):
        if not terms[k]:
            continue
        lines.append("  {\n")
        need = sorted({pi for (pi, _, _, _) in terms[k]})
        loads, ops, nst = xy_plan(Z, need)
        pairs = sorted({((x >> 2) & 1, (x >> 1) & 1) for x in loads})
        for (r, h) in pairs:
            lines.append(f"    const double2 p{r}{h} = pos[{r}] ? __ldg(reinterpret_cast<const double2*>(pos[{r}] + "
                         f"{4 * k} * NCELL + {2 * h})) : make_double2(0.0, 0.0);\n")
        for x in loads:
            r, h = (x >> 2) & 1, (x >> 1) & 1
            lines.append(f"    const double v2_{x} = p{r}{h}.{'y' if x & 1 else 'x'};\n")
        for (t, x, op, lo, hi) in ops:
            lines.append(f"    const double v{t}_{x} = v{t - 1}_{lo} {op} v{t - 1}_{hi};\n")
            n_add += 1
        for (pi, kind, idx, di) in terms[k]:
            lines.append(f"    {kind}[{idx}] = fma(v{nst}_{pi}, __ldg(row + {di}), {kind}[{idx}]);\n")
            n_fma += 1
        lines.append("  }\n")
    lines.append("}\n\n")
    return name, "".join(lines), n_add, n_fma


def mclass_adj_code(Z):
    """the transpose (multipole gather by source): the members are targets,
    per target component j the transform of their reduced L-bar feeds
    g[k] += W_j[pi(j + k)] d[j + k]"""
    name = f"ot_mclass_adj_z{Z}"
    lines = [f"__device__ __forceinline__ void {name}(double (&g)[16], const double* const (&src)[8],\n"
             f"    const double* __restrict__ row) {{\n"]
    members = [i for i in range(8) if not (i & Z)]
    terms = {j: [] for j in range(16)}
    for j, ej in enumerate(IND16):
        for k, ek in enumerate(IND16):
            if rank(ej) + rank(ek) <= 3:
                e = add(ej, ek)
                if not (parity(e) & Z):
                    terms[j].append((parity(e), k, ROWIDX[e]))
    n_add = n_fma = 0
    for j in range(16):
        if not terms[j]:
            continue
        lines.append("  {\n")
        for i in members:
            lines.append(f"    const double v0_{i} = src[{i}] ? __ldg(src[{i}] + {j} * NCELL) : 0.0;\n")
        need = sorted({pi for (pi, _, _) in terms[j]})
        ops, nst = transform_plan(Z, need)
        for (t, x, op, lo, hi) in ops:
            lines.append(f"    const double v{t}_{x} = v{t - 1}_{lo} {op} v{t - 1}_{hi};\n")
        n_add += len(ops)
        for (pi, k, di) in terms[j]:
            lines.append(f"    g[{k}] = fma(v{nst}_{pi}, __ldg(row + {di}), g[{k}]);\n")
            n_fma += 1
        lines.append("  }\n")
    lines.append("}\n\n")
    return name, "".join(lines), n_add, n_fma


def mclass_adj_x_code(Z):
    """ot_mclass_adj_code with the x stage prebuilt (the member targets'
    L-bar x butterflies at the positions q = B + (0, +-b, +-c))"""
    assert not (Z & 1)
    name = f"ot_mclass_adj_x_z{Z}"
    lines = [f"__device__ __forceinline__ void {name}(double (&g)[16], const double* const (&pos)[4],\n"
             f"    const double* __restrict__ row) {{\n"]
    terms = {j: [] for j in range(16)}
    for j, ej in enumerate(IND16):
        for k, ek in enumerate(IND16):
            if rank(ej) + rank(ek) <= 3:
                e = add(ej, ek)
                if not (parity(e) & Z):
                    terms[j].append((parity(e), k, ROWIDX[e]))
    n_add = n_fma = 0
    for j in range(16):
        if not terms[j]:
            continue
        lines.append("  {\n")
        need = sorted({pi for (pi, _, _) in terms[j]})
        ops, nst = transform_plan(Z, need, first=0)
        for (t, x, op, lo, hi) in ops:
            if t == 1:
                q = (x >> 1) & 3
                lines.append(f"    const double v1_{x} = pos[{q}] ? __ldg(pos[{q}] + {2 * j + (x & 1)} * NCELL) : 0.0;\n")
            else:
                lines.append(f"    const double v{t}_{x} = v{t - 1}_{lo} {op} v{t - 1}_{hi};\n")
                n_add += 1
        for (pi, k, di) in terms[j]:
            lines.append(f"    g[{k}] = fma(v{nst}_{pi}, __ldg(row + {di}), g[{k}]);\n")
            n_fma += 1
        lines.append("  }\n")
    lines.append("}\n\n")
    return name, "".join(lines), n_add, n_fma


def emit():
    out = []
    w = out.append
    w("// Generated by gen_contract.py -- do not edit.\n")
    w("// Traceless-reduced FP64 contractions; see gen_contract.py for the layout.\n\n")

    # point-mass source: a[J] += mass * d[J]
    w("__device__ __forceinline__ void ot_mono_fwd(double (&a)[16], double mass, const double (&d)[36]) {\n")
    for j in range(16):
        w(f"  a[{j}] = fma(mass, d[{j}], a[{j}]);\n")
    w("}\n\n")

    # multipole source: a[J] += sum_K r[K] d[J+K]
    terms = []
    for j, ej in enumerate(IND16):
        for k, ek in enumerate(IND16):
            if rank(ej) + rank(ek) <= 3:
                terms.append((j, k, ROWIDX[add(ej, ek)]))
    assert len(terms) == 70, len(terms)
    w("// 70 FMAs\n")
    w("__device__ __forceinline__ void ot_multi_fwd(double (&a)[16], const double (&r)[16], const double (&d)[36]) {\n")
    # order: by source component so consecutive FMAs hit different accumulators
    for k in range(16):
        for (j, kk, di) in terms:
            if kk == k:
                w(f"  a[{j}] = fma(r[{k}], d[{di}], a[{j}]);\n")
    w("}\n\n")

    # angular term, source part: c[i] += sum_{K in R3} r[K] d[e_i + K];
    # target part accumulator: t4[q] += mB * d[q]
    w("// 21 + 9 FMAs\n")
    w("__device__ __forceinline__ void ot_angular_fwd(double (&c)[3], double (&t4)[9], const double (&r)[16],\n"
      "                                               double mB, const double (&d)[36]) {\n")
    for i in range(3):
        ei = tuple(1 if a == i else 0 for a in range(3))
        for k in R3:
            w(f"  c[{i}] = fma(r[{k}], d[{ROWIDX[add(ei, IND16[k])]}], c[{i}]);\n")
    for q, e in enumerate(T4):
        w(f"  t4[{q}] = fma(mB, d[{ROWIDX[e]}], t4[{q}]);\n")
    w("}\n\n")

    # angular epilogue: out[i] = sum_{K in R3} rA[K] * T4[e_i + K]
    w("__device__ __forceinline__ void ot_angular_target(double (&out)[3], const double (&t4)[9], const double (&rA)[16]) {\n")
    for i in range(3):
        ei = tuple(1 if a == i else 0 for a in range(3))
        parts = [f"rA[{k}] * {t4_expr(add(ei, IND16[k]))}" for k in R3]
        w(f"  out[{i}] = " + " + ".join(parts) + ";\n")
    w("}\n\n")

    # adjoint, multipole source: g[K] += sum_J lb[J] d[J+K]
    w("// 70 FMAs\n")
    w("__device__ __forceinline__ void ot_multi_adj(double (&g)[16], const double (&lb)[16], const double (&d)[36]) {\n")
    for j in range(16):
        for (jj, k, di) in terms:
            if jj == j:
                w(f"  g[{k}] = fma(lb[{j}], d[{di}], g[{k}]);\n")
    w("}\n\n")

    # paired point-mass sources: a[J] += (even order ? s : d) * d[J]
    w("// paired: 16 FMAs for two point-mass pairs (s = m+ + m-, d = m+ - m-)\n")
    w("__device__ __forceinline__ void ot_mono_fwd_pair(double (&a)[16], double s, double dm, const double (&d)[36]) {\n")
    for j in range(16):
        w(f"  a[{j}] = fma({'s' if rank(IND16[j]) % 2 == 0 else 'dm'}, d[{j}], a[{j}]);\n")
    w("}\n\n")

    # point masses paired by a reflection along one axis A (the member at o'
    # is o with its A component negated): a[J] += (J_A even ? s : dm) * d[J]
    for A, name in enumerate("xyz"):
        w(f"// paired along {name}: 16 FMAs for two point-mass pairs at o and o reflected along {name}\n"
          f"// (s = m(o) + m(o'), dm = m(o) - m(o'), d the row of o)\n")
        w(f"__device__ __forceinline__ void ot_mono_fwd_{name}pair(double (&a)[16], double s, double dm,\n"
          f"                                                  const double (&d)[36]) {{\n")
        for j in range(16):
            w(f"  a[{j}] = fma({'s' if IND16[j][A] % 2 == 0 else 'dm'}, d[{j}], a[{j}]);\n")
        w("}\n\n")

    # paired multipole sources: a[J] += (even order of J+K ? rs[K] : rd[K]) * d[J+K]
    w("// paired: 70 FMAs for two multipole pairs (rs = r+ + r-, rd = r+ - r-)\n")
    w("__device__ __forceinline__ void ot_multi_fwd_pair(double (&a)[16], const double (&rs)[16], const double (&rd)[16],\n"
      "                                                  const double (&d)[36]) {\n")
    for k in range(16):
        for (j, kk, di) in terms:
            if kk == k:
                src = "rs" if rank(ROW[di]) % 2 == 0 else "rd"
                w(f"  a[{j}] = fma({src}[{k}], d[{di}], a[{j}]);\n")
    w("}\n\n")

    # multipole sources paired by a reflection along one axis A: the member
    # at o' (o with its A component negated) sees d^K G(o') = (-1)^{K_A}
    # d^K G(o), so a[J] += (K_A of J+K even ? rs[K] : rd[K]) * d[J+K] with
    # the row of o
    for A, name in enumerate("xyz"):
        w(f"// paired along {name}: 70 FMAs for two multipole pairs at o and o reflected along {name}\n"
          f"// (rs = r(o) + r(o'), rd = r(o) - r(o'), d the row of o)\n")
        w(f"__device__ __forceinline__ void ot_multi_fwd_{name}pair(double (&a)[16], const double (&rs)[16],\n"
          f"                                                   const double (&rd)[16], const double (&d)[36]) {{\n")
        for k in range(16):
            for (j, kk, di) in terms:
                if kk == k:
                    src = "rs" if ROW[di][A] % 2 == 0 else "rd"
                    w(f"  a[{j}] = fma({src}[{k}], d[{di}], a[{j}]);\n")
        w("}\n\n")

    # paired multipole adjoint: g[K] += sum_J (even order of J+K ? ls[J] : ld[J]) * d[J+K]
    w("// paired: 70 FMAs for two targets (ls = lb+ + lb-, ld = lb+ - lb-)\n")
    w("__device__ __forceinline__ void ot_multi_adj_pair(double (&g)[16], const double (&ls)[16], const double (&ld)[16],\n"
      "                                                  const double (&d)[36]) {\n")
    for j in range(16):
        for (jj, k, di) in terms:
            if jj == j:
                src = "ls" if rank(ROW[di]) % 2 == 0 else "ld"
                w(f"  g[{k}] = fma({src}[{j}], d[{di}], g[{k}]);\n")
    w("}\n\n")

    # adjoint, point-mass source: g[s] += sum_J lb[J] d[J]  (4 partial sums)
    w("// 16 FMAs\n")
    w("__device__ __forceinline__ void ot_mono_adj(double (&g)[4], const double (&lb)[16], const double (&d)[36]) {\n")
    for j in range(16):
        w(f"  g[{j % 4}] = fma(lb[{j}], d[{j}], g[{j % 4}]);\n")
    w("}\n\n")
    # point-mass adjoint organised by target: even- and odd-order parts of
    # <lb, d>; the source at t+o receives e+q, the one at t-o receives e-q
    w("// 16 FP64 ops: e = even-order part, q = odd-order part of <lb, d>\n")
    w("__device__ __forceinline__ void ot_mono_adj_split(double& e, double& q, const double (&lb)[16],\n"
      "                                                  const double (&d)[36]) {\n")
    first = {0: True, 1: True}
    for j in range(16):
        par = rank(IND16[j]) % 2
        v = "e" if par == 0 else "q"
        if first[par]:
            w(f"  {v} = lb[{j}] * d[{j}];\n")
            first[par] = False
        else:
            w(f"  {v} = fma(lb[{j}], d[{j}], {v});\n")
    w("}\n\n")

    # the same split by the parity of J_A: the source at t+o receives e + q,
    # the one at o reflected along A receives e - q
    for A, name in enumerate("xyz"):
        w(f"// 16 FP64 ops: e = the part of <lb, d> with an even {name} order, q = the odd part\n")
        w(f"__device__ __forceinline__ void ot_mono_adj_split_{name}(double& e, double& q, const double (&lb)[16],\n"
          f"                                                    const double (&d)[36]) {{\n")
        first = {0: True, 1: True}
        for j in range(16):
            par = IND16[j][A] % 2
            v = "e" if par == 0 else "q"
            if first[par]:
                w(f"  {v} = lb[{j}] * d[{j}];\n")
                first[par] = False
            else:
                w(f"  {v} = fma(lb[{j}], d[{j}], {v});\n")
        w("}\n\n")

    # double-float (FP32 hi + lo) point-mass contraction, paired form:
    # a[J] += x * D[J] with x = s (even order) or dm (odd order); the row
    # holds hi[0..15] then lo[0..15]
    w("// double-float: 16 products for two point-mass pairs (x = s or dm by order parity)\n")
    w("__device__ __forceinline__ void ot_mono_fwd_pair_df(float (&ah)[16], float (&al)[16], float sh, float sl,\n"
      "                                                    float dh, float dl, const float (&r)[32]) {\n")
    for j in range(16):
        even = rank(IND16[j]) % 2 == 0
        xh, xl = ("sh", "sl") if even else ("dh", "dl")
        w(f"  df_fma(ah[{j}], al[{j}], {xh}, {xl}, r[{j}], r[{16 + j}]);\n")
    w("}\n\n")
    w("// double-float: 16 products for one point-mass pair\n")
    w("__device__ __forceinline__ void ot_mono_fwd_df(float (&ah)[16], float (&al)[16], float mh, float ml,\n"
      "                                               const float (&r)[32]) {\n")
    for j in range(16):
        w(f"  df_fma(ah[{j}], al[{j}], mh, ml, r[{j}], r[{16 + j}]);\n")
    w("}\n\n")

    # double-float multipole contractions.  The table row is a float2 pair
    # (hi, lo) per derivative component, read from L1 as each component is
    # needed; terms are grouped by component so its pair dies after its terms.
    by_di = {}
    for (j, k, di) in terms:
        by_di.setdefault(di, []).append((j, k))
    w("// double-float, paired: 70 products for two multipole pairs (rs = r+ + r-, rd = r+ - r-)\n")
    w("__device__ __forceinline__ void ot_multi_fwd_pair_df(float (&ah)[16], float (&al)[16], const float (&rsh)[16],\n"
      "                                                     const float (&rsl)[16], const float (&rdh)[16],\n"
      "                                                     const float (&rdl)[16], const float2* __restrict__ row) {\n")
    for di in sorted(by_di):
        w(f"  {{\n    const float2 d = __ldg(row + {di});\n")
        src = "rs" if rank(ROW[di]) % 2 == 0 else "rd"
        for (j, k) in by_di[di]:
            w(f"    df_fma(ah[{j}], al[{j}], {src}h[{k}], {src}l[{k}], d.x, d.y);\n")
        w("  }\n")
    w("}\n\n")
    w("// double-float: 70 products for one multipole pair\n")
    w("__device__ __forceinline__ void ot_multi_fwd_df(float (&ah)[16], float (&al)[16], const float (&rh)[16],\n"
      "                                                const float (&rl)[16], const float2* __restrict__ row) {\n")
    for di in sorted(by_di):
        w(f"  {{\n    const float2 d = __ldg(row + {di});\n")
        for (j, k) in by_di[di]:
            w(f"    df_fma(ah[{j}], al[{j}], rh[{k}], rl[{k}], d.x, d.y);\n")
        w("  }\n")
    w("}\n\n")
    # angular term in double-float: c[i] += sum_{K in R3} r[K] d[e_i + K];
    # t4[q] += mB d[q] (rank-4 components: even, so paired entries use sums)
    ang = {}
    for i in range(3):
        ei = tuple(1 if a == i else 0 for a in range(3))
        for k in R3:
            ang.setdefault(ROWIDX[add(ei, IND16[k])], []).append(("c", i, k))
    for q, e in enumerate(T4):
        ang.setdefault(ROWIDX[e], []).append(("t", q, None))
    w("// double-float angular term: 21 + 9 products\n")
    w("__device__ __forceinline__ void ot_angular_fwd_df(float (&ch)[3], float (&cl)[3], float (&th)[9], float (&tl)[9],\n"
      "                                                  const float (&rh)[16], const float (&rl)[16],\n"
      "                                                  const float2* __restrict__ row) {\n")
    for di in sorted(ang):
        w(f"  {{\n    const float2 d = __ldg(row + {di});\n")
        for (kind, i, k) in ang[di]:
            if kind == "c":
                w(f"    df_fma(ch[{i}], cl[{i}], rh[{k}], rl[{k}], d.x, d.y);\n")
            else:
                w(f"    df_fma(th[{i}], tl[{i}], rh[0], rl[0], d.x, d.y);\n")
        w("  }\n")
    w("}\n\n")

    # double-float adjoint contractions (transposes of the above)
    w("// double-float adjoint, paired: g[K] += sum_J (even order of J+K ? ls[J] : ld[J]) * d[J+K]\n")
    w("__device__ __forceinline__ void ot_multi_adj_pair_df(float (&gh)[16], float (&gl)[16], const float (&lsh)[16],\n"
      "                                                     const float (&lsl)[16], const float (&ldh)[16],\n"
      "                                                     const float (&ldl)[16], const float2* __restrict__ row) {\n")
    for di in sorted(by_di):
        w(f"  {{\n    const float2 d = __ldg(row + {di});\n")
        src = "ls" if rank(ROW[di]) % 2 == 0 else "ld"
        for (j, k) in by_di[di]:
            w(f"    df_fma(gh[{k}], gl[{k}], {src}h[{j}], {src}l[{j}], d.x, d.y);\n")
        w("  }\n")
    w("}\n\n")
    w("// double-float adjoint, one target: g[K] += sum_J lb[J] d[J+K]\n")
    w("__device__ __forceinline__ void ot_multi_adj_df(float (&gh)[16], float (&gl)[16], const float (&lh)[16],\n"
      "                                                const float (&ll)[16], const float2* __restrict__ row) {\n")
    for di in sorted(by_di):
        w(f"  {{\n    const float2 d = __ldg(row + {di});\n")
        for (j, k) in by_di[di]:
            w(f"    df_fma(gh[{k}], gl[{k}], lh[{j}], ll[{j}], d.x, d.y);\n")
        w("  }\n")
    w("}\n\n")
    w("// double-float point-mass adjoint of one entry: the even- and odd-order\n"
      "// parts (e, q) of <lb, d> in fresh double-float accumulators\n")
    w("__device__ __forceinline__ void ot_mono_adj_split_df(float& eh, float& el, float& qh, float& ql,\n"
      "                                                     const float (&lh)[16], const float (&ll)[16],\n"
      "                                                     const float (&r)[32]) {\n")
    w("  eh = 0.0f;\n  el = 0.0f;\n  qh = 0.0f;\n  ql = 0.0f;\n")
    for j in range(16):
        v = "e" if rank(IND16[j]) % 2 == 0 else "q"
        w(f"  df_fma({v}h, {v}l, lh[{j}], ll[{j}], r[{j}], r[{16 + j}]);\n")
    w("}\n\n")

    # multipole sources by reflection class
    w("// multipole sources of one reflection class, zero pattern Z (see\n"
      "// gen_contract.py): src[i] the reduced moments of member i (stride NCELL)\n"
      "// or null, row the table row of the class's representative offset\n")
    for Z in range(7):
        for ang in (False, True):
            name, code, n_add, n_fma = mclass_fwd_code(Z, ang)
            w(f"// {n_add} adds + {n_fma} FMAs\n")
            w(code)
    for Z in (0, 2, 4, 6):
        for ang in (False, True):
            name, code, n_add, n_fma = mclass_fwd_x_code(Z, ang)
            w(f"// x stage prebuilt: {n_add} adds + {n_fma} FMAs\n")
            w(code)
    w("template <int Z, bool ANG>\n"
      "__device__ __forceinline__ void ot_mclass_fwd_x(double (&a)[16], double (&c)[3], double (&t4)[9],\n"
      "                                                const double* const (&pos)[4], const double* __restrict__ row) {\n")
    for i, Z in enumerate((0, 2, 4, 6)):
        w(f"  {'if' if i == 0 else 'else if'} constexpr (Z == {Z}) {{\n"
          f"    if constexpr (ANG) ot_mclass_fwd_x_z{Z}_ang(a, c, t4, pos, row);\n"
          f"    else ot_mclass_fwd_x_z{Z}(a, c, t4, pos, row);\n  }}\n")
    w("}\n\n")
    for Z in (0, 4):
        for ang in (False, True):
            name, code, n_add, n_fma = mclass_fwd_xy_code(Z, ang)
            w(f"// x and y stages prebuilt: {n_add} adds + {n_fma} FMAs\n")
            w(code)
    w("template <int Z, bool ANG>\n"
      "__device__ __forceinline__ void ot_mclass_fwd_xy(double (&a)[16], double (&c)[3], double (&t4)[9],\n"
      "                                                 const double* const (&pos)[2], const double* __restrict__ row) {\n")
    for i, Z in enumerate((0, 4)):
        w(f"  {'if' if i == 0 else 'else if'} constexpr (Z == {Z}) {{\n"
          f"    if constexpr (ANG) ot_mclass_fwd_xy_z{Z}_ang(a, c, t4, pos, row);\n"
          f"    else ot_mclass_fwd_xy_z{Z}(a, c, t4, pos, row);\n  }}\n")
    w("}\n\n")
    for Z in range(7):
        name, code, n_add, n_fma = mclass_adj_code(Z)
        w(f"// adjoint: {n_add} adds + {n_fma} FMAs\n")
        w(code)
    for Z in (0, 2, 4, 6):
        name, code, n_add, n_fma = mclass_adj_x_code(Z)
        w(f"// adjoint, x stage prebuilt: {n_add} adds + {n_fma} FMAs\n")
        w(code)
    w("template <int Z>\n"
      "__device__ __forceinline__ void ot_mclass_adj_x(double (&g)[16], const double* const (&pos)[4],\n"
      "                                                const double* __restrict__ row) {\n")
    for i, Z in enumerate((0, 2, 4, 6)):
        w(f"  {'if' if i == 0 else 'else if'} constexpr (Z == {Z}) ot_mclass_adj_x_z{Z}(g, pos, row);\n")
    w("}\n\n")
    w("template <int Z>\n"
      "__device__ __forceinline__ void ot_mclass_adj(double (&g)[16], const double* const (&src)[8],\n"
      "                                              const double* __restrict__ row) {\n")
    for Z in range(7):
        w(f"  {'if' if Z == 0 else 'else if'} constexpr (Z == {Z}) ot_mclass_adj_z{Z}(g, src, row);\n")
    w("}\n\n")
    w("template <int Z, bool ANG>\n"
      "__device__ __forceinline__ void ot_mclass_fwd(double (&a)[16], double (&c)[3], double (&t4)[9],\n"
      "                                              const double* const (&src)[8], const double* __restrict__ row) {\n")
    for Z in range(7):
        w(f"  {'if' if Z == 0 else 'else if'} constexpr (Z == {Z}) {{\n"
          f"    if constexpr (ANG) ot_mclass_fwd_z{Z}_ang(a, c, t4, src, row);\n"
          f"    else ot_mclass_fwd_z{Z}(a, c, t4, src, row);\n  }}\n")
    w("}\n\n")

    # derivatives at an arbitrary separation (centre-of-mass expansion centres)
    w("// derivatives of -1/r (row layout) at R = (x, y, z), the components each\n")
    w("// contraction reads: point masses, multipole sources, multipole sources\n")
    w("// with the angular term\n")
    for name in DERIV_SETS:
        w(deriv_code(name))
    w("// algorithmic FLOPs of one call of each (sqrt and the division count one each)\n")
    for name in DERIV_SETS:
        w(f"constexpr int {name.upper().replace('OT_DERIV', 'OT_DERIV').replace('_AT', '')}_FLOPS = "
          f"{deriv_flops(name)};\n")
    w("\n")

    # the same with the row of -o: odd-order derivatives negated
    w("// 16 FMAs (derivatives of the negated offset)\n")
    w("__device__ __forceinline__ void ot_mono_adj_neg(double (&g)[4], const double (&lb)[16], const double (&d)[36]) {\n")
    for j in range(16):
        sign = "" if rank(IND16[j]) % 2 == 0 else "-"
        w(f"  g[{j % 4}] = fma({sign}lb[{j}], d[{j}], g[{j % 4}]);\n")
    w("}\n")
    return "".join(out)


def emit_counts():
    """ot_contract_counts.h: operation counts of the generated routines that
    the host code's cost model and FLOP accounting use"""
    out = ["// Generated by gen_contract.py -- do not edit.\n",
           "// Operation counts of generated contractions (host and device).\n",
           "#pragma once\n\n",
           "// FP64 adds and FMAs of ot_mclass_fwd_z<Z>[_ang], indexed [ang][Z]\n"]
    adds, fmas = {}, {}
    for Z in range(7):
        for ang in (False, True):
            _, _, adds[ang, Z], fmas[ang, Z] = mclass_fwd_code(Z, ang)
    for name, tab in (("OT_MCLASS_ADDS", adds), ("OT_MCLASS_FMAS", fmas)):
        out.append(f"constexpr int {name}[2][7] = {{" + ", ".join(
            "{" + ", ".join(str(tab[ang, Z]) for Z in range(7)) + "}" for ang in (False, True)) + "};\n")
    out.append("// FP64 adds of ot_mclass_fwd_x_z<Z>[_ang] (x stage prebuilt; 0 for Z with bit 0), [ang][Z]\n")
    xa = {(ang, Z): (mclass_fwd_x_code(Z, ang)[2] if not (Z & 1) else 0) for ang in (False, True) for Z in range(7)}
    out.append("constexpr int OT_MCLASS_X_ADDS[2][7] = {" + ", ".join(
        "{" + ", ".join(str(xa[ang, Z]) for Z in range(7)) + "}" for ang in (False, True)) + "};\n")
    out.append("// FP64 adds of ot_mclass_fwd_xy_z<Z>[_ang] (x and y stages prebuilt; 0 for Z with bit 0 or 1), [ang][Z]\n")
    xya = {(ang, Z): (mclass_fwd_xy_code(Z, ang)[2] if not (Z & 3) else 0) for ang in (False, True) for Z in range(7)}
    out.append("constexpr int OT_MCLASS_XY_ADDS[2][7] = {" + ", ".join(
        "{" + ", ".join(str(xya[ang, Z]) for Z in range(7)) + "}" for ang in (False, True)) + "};\n")
    ax = [mclass_adj_x_code(Z)[2] if not (Z & 1) else 0 for Z in range(7)]
    out.append("// FP64 adds of ot_mclass_adj_x_z<Z> (x stage prebuilt; 0 for Z with bit 0)\n")
    out.append("constexpr int OT_MCLASS_ADJ_X_ADDS[7] = {" + ", ".join(str(a) for a in ax) + "};\n")
    out.append("// FP64 adds and FMAs of ot_mclass_adj_z<Z>\n")
    cnt = [mclass_adj_code(Z)[2:] for Z in range(7)]
    out.append("constexpr int OT_MCLASS_ADJ_ADDS[7] = {" + ", ".join(str(a) for a, _ in cnt) + "};\n")
    out.append("constexpr int OT_MCLASS_ADJ_FMAS[7] = {" + ", ".join(str(f) for _, f in cnt) + "};\n")
    return "".join(out)


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "ot_contract.inc"), "w") as f:
        f.write(emit())
    with open(os.path.join(here, "ot_contract_counts.h"), "w") as f:
        f.write(emit_counts())
